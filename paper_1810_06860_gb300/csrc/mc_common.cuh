// Shared declarations of the GB300 fast-SVT library: error plumbing, device
// memory, and the host-side launchers of every kernel.  Internal header.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/mc.h"

namespace mc {

// ---- errors ---------------------------------------------------------------
void set_error(const std::string &msg);
struct Err {
  mc_status st;
  std::string msg;
};
// Thrown only inside the library; the C ABI catches every Err.
[[noreturn]] void fail(mc_status st, const std::string &msg);

#define MC_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      ::mc::fail(MC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)
// Every kernel launch of the library goes through MC_CHECK_LAUNCH, which also
// counts it (mc_launch_count).
void count_launch();
// Keeps the copy of Y into CSC order on the handle's own stream (no second
// stream): the serving form runs many handles at once, and twice as many
// streams as hardware work queues would put unrelated jobs' work behind a
// second stream's event wait.
void handle_single_stream(mc_handle h);
#define MC_CHECK_LAUNCH()          \
  do {                             \
    MC_CUDA(cudaGetLastError());   \
    ::mc::count_launch();          \
  } while (0)
#define MC_REQUIRE(cond, msg)                                                           \
  do {                                                                                  \
    if (!(cond)) ::mc::fail(MC_EINVAL, msg);                                            \
  } while (0)

// ---- device memory ----------------------------------------------------------
// A growable device buffer owned by a handle; allocation goes through the
// handle's allocator hook or cudaMallocAsync on its stream.
struct Alloc {
  mc_allocator hook{};
  bool has_hook = false;
  cudaStream_t stream = nullptr;
  void *get(size_t bytes);
  void put(void *p, size_t bytes);
};

struct DBuf {
  void *p = nullptr;
  size_t cap = 0;
  template <class T>
  T *as() const { return static_cast<T *>(p); }
  void reserve(Alloc &a, size_t bytes);   // contents not preserved
  void release(Alloc &a);
};

// Releases the listed buffers when it leaves scope, so a temporary buffer is
// returned to the allocator also when a later step throws.
struct BufGuard {
  Alloc &a;
  std::vector<DBuf *> bufs;
  BufGuard(Alloc &a_, std::initializer_list<DBuf *> b) : a(a_), bufs(b) {}
  BufGuard(const BufGuard &) = delete;
  BufGuard &operator=(const BufGuard &) = delete;
  ~BufGuard() {
    for (DBuf *b : bufs) b->release(a);
  }
};

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---- work decomposition of a compressed sparse matrix -----------------------
// Rows (or columns, for the CSC copy) are cut into segments of at most SEG
// entries.  A row with one segment is written directly by the warp that owns
// it; a longer row writes one partial per segment and a fix-up pass adds them
// in segment order (deterministic, no atomics).
constexpr int SEG = 256;
struct SegPlan {
  int64_t nseg = 0;      // number of segments (every row has >= 1, empty rows too)
  int64_t nsplit = 0;    // number of rows with > 1 segment
  int64_t nslot = 0;     // partial slots (segments of split rows)
  DBuf seg;              // int4[nseg]  (row, first entry, one past the last, partial slot or -1)
  DBuf split_row;        // int32[nsplit] rows with several segments
  DBuf split_slot;       // int32[nsplit+1] first slot of each split row
};

// ---- launchers (k_rng.cu) ---------------------------------------------------
void launch_omega(cudaStream_t st, int64_t n, int k, int ld, uint64_t seed, uint64_t call_id,
                  int col0, float *out, uint32_t *words);

// ---- launchers (k_sparse.cu) ------------------------------------------------
// Build CSC arrays (col_ptr, row_idx, perm: CSC position -> CSR position) from
// CSR on the device.  tmp must hold >= 4*(n+1) + 4*nnz bytes.
void build_csc(cudaStream_t st, int64_t m, int64_t n, int64_t nnz, const int *row_ptr,
               const int *col, int *col_ptr, int *row_idx, int *perm, void *tmp);
size_t csc_tmp_bytes(int64_t m, int64_t n);
// int64 row_ptr -> int32 with monotonicity/range checks (flags[0] |= 1 on error)
void convert_rowptr(cudaStream_t st, int64_t m, int64_t nnz, const int64_t *rp64, int *rp32, int *flags);
// Validate CSR (sorted unique columns, indices in range, finite values).
// flags: device int[3] (0 ok); host reads back.
void validate_csr(cudaStream_t st, int64_t m, int64_t n, const int *row_ptr, const int *col,
                  const float *val, int *flags);
// COO (any order; rows int64, cols int32, device) -> CSR (row_ptr int64,
// col, val; device).  flags[1] |= 1 for an index out of range, |= 2 for a
// repeated (row, col); flags[2] |= 1 for a non-finite value.
void coo_to_csr(cudaStream_t st, Alloc &a, int64_t m, int64_t n, int64_t nnz, const int64_t *rows, const int *cols,
                const float *vals, int64_t *row_ptr, int *col, float *val, int *flags);
void plan_segments(cudaStream_t st, Alloc &a, int64_t rows, const int *ptr, SegPlan &plan);
// out (rows x K, ld_out) = A (CSR ptr/idx/val) * X (cols x K, ld_x).  K, ld_x,
// ld_out multiples of 4 (padded columns must be zero in X).  partial must hold
// plan.nslot * K floats.
// rows_in: rows of X (sizes the column chunks so the panel slice stays in L2).
// Launch shape of the SpMM: gathers in flight per lane group (u), CTA size
// (threads: 128 or 256) and column-chunk width; 0 selects the default.  The
// lane-group count depends on the panel width only, so no choice changes the
// order of any sum: every shape gives the same bits.
struct SpmmCfg {
  int u = 0, threads = 0, chunk = 0;
};
std::vector<SpmmCfg> spmm_candidates(int K, int64_t rows_in);
// What the candidate list depends on: lane groups per warp and the default
// column chunk for a panel of K columns and rows_in rows.
int spmm_groups(int K, int64_t rows_in);
int default_chunk(int64_t rows_in);
void spmm(cudaStream_t st, const SegPlan &plan, const int *idx, const float *val, int64_t rows_in,
          const float *X, int ld_x, int K, float *out, int ld_out, float *partial, const SpmmCfg &cfg = SpmmCfg{});
// As spmm with a bf16 panel X (K, ld_x multiples of 8, K <= 256), float32
// accumulation and output (mixed-precision form).
void spmm_bf16(cudaStream_t st, const SegPlan &plan, const int *idx, const float *val, const void *Xbf, int ld_x,
               int K, float *out, int ld_out, float *partial);
// out (rows x ld_out, bf16) = round(in[:, 0:cols]), zero columns after cols.
void to_bf16(cudaStream_t st, int64_t rows, int cols, const float *in, int ld_in, void *out, int ld_out);
// y = P_Phi(M) scaled: y[e] = alpha * mval[e]
void scale_values(cudaStream_t st, int64_t nnz, const float *src, float alpha, float *dst);
// Yc[p] = Y[perm[p]]
void mirror_values(cudaStream_t st, int64_t nnz, const int *perm, const float *y, float *yc);
// Fused SVT update over Phi in CSR order (Alg. 6 steps 15-17):
//   x_e = <Us[row_e, 0:r], V[col_e, 0:r]>,  res = M_e - x_e,
//   per-block sums of res^2 into block_sq (double, sddmm_partials() entries),
//   y_e += delta * res (only if update != 0).  x_out (optional) receives x_e.
//   Returns the number of block partials written.  Columns r..ld-1 of Us and
//   V must be zero up to the next multiple of 4.
int sddmm_update(cudaStream_t st, int64_t nnz, const int *rix, const int *col, const float *mval, float *y,
                 const float *Us, int ld_us, const float *V, int ld_v, int r, float delta, int update,
                 double *block_sq, float *x_out);
int sddmm_partials();
// The SpMM's gathers alone (k_sparse.cu): rows idx[e] of the panel P (ldp a
// multiple of 4, K columns) loaded in 16-byte slices by lane groups, summed
// into sink (grid * 256 floats); the ceiling for the SpMM's gathers.
void gather_probe(cudaStream_t st, int64_t nnz, const int *idx, const float *P, int ldp, int K, float *sink,
                  int grid);
// rix[e] = row of CSR entry e.
void expand_rows(cudaStream_t st, int64_t m, const int *rp, int *rix);
// Deterministic sum of a double array into out[0] (one block, fixed order).
void sum_doubles(cudaStream_t st, const double *in, int64_t count, double *out);
// sum of squares of a float array, deterministic, into out[0] (double).
void sumsq_floats(cudaStream_t st, const float *in, int64_t count, double *scratch, double *out);
// Evaluate X = Us V^T at listed positions.
void sample_lowrank(cudaStream_t st, int64_t count, const int64_t *rows, const int64_t *cols,
                    const float *Us, int ld_us, const float *V, int ld_v, int r, float *out);

// ---- launchers (k_dense.cu) -------------------------------------------------
// C (K1 x K2, ld_c) = X^T Y summed over R rows; X (R x K1, ld_x), Y (R x K2,
// ld_y).  sym: X == Y and only the lower triangle is needed (mirrored).
// partial: scratch of gemm_tn_scratch_floats(R, K1, K2) floats.
size_t gemm_tn_scratch_floats(int64_t R, int K1, int K2);
// skip (device int, may be NULL): when it holds a nonzero value the kernels
// return without work (a CholeskyQR pass found unnecessary on the device).
// Shapes the tensor-core kernel takes (K1, K2 <= 256, K2 > 16) run there
// unless MC_TN_TC=0; err (device int, may be NULL) receives its wait-expiry code.
void gemm_tn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y,
             int ld_y, float *C, int ld_c, bool sym, float *partial, const int *skip = nullptr,
             int *err = nullptr);
// The SIMT kernels alone.
void gemm_tn_simt(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y, int ld_y,
                  float *C, int ld_c, float *partial, const int *skip = nullptr, bool sym = false);
// The fixed-order sum of nsplit partial K1p x K2p tiles into C (K1 x K2).
void gemm_tn_reduce_partials(cudaStream_t st, int K1, int K2, int nsplit, const float *partial, int K1p, int K2p,
                             float *C, int ld_c, const int *skip);
// C (K1 x K2) = X1^T X2 on the tensor cores (k_tc.cu, 3xTF32, warp-specialised):
// K1, K2 <= 256, leading dimensions multiples of 4, panels 16-byte aligned.
bool gemm_tn_tc_supported(int64_t R, int K1, int K2, const void *X1, int ld1, const void *X2, int ld2);
size_t gemm_tn_tc_scratch_floats(int64_t R, int K1, int K2);
void gemm_tn_tc(cudaStream_t st, int64_t R, int K1, int K2, const float *X1, int ld1, const float *X2, int ld2,
                float *C, int ld_c, float *partial, int *err, const int *skip);
// Z (R x K2, ld_z) = beta * Z + alpha * X (R x K1, ld_x) * W (K1 x K2, ld_w) * diag(colscale)
// colscale may be NULL (ones).  Z may not alias X.  copy_if (device int, may
// be NULL; 16 < K1 == K2 <= 64 only): when it holds a nonzero value, Z = X.
// Shapes the tensor-core kernel takes (K2 > 16) run there unless MC_NN_TC=0;
// err (device int, may be NULL) receives its wait-expiry code.
void gemm_nn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *W,
             int ld_w, const float *colscale, float alpha, float beta, float *Z, int ld_z,
             const int *copy_if = nullptr, int *err = nullptr);
// The SIMT kernels alone (thread-per-row for K2 <= 16, W in shared memory for
// K1 <= 64, tiled otherwise).
void gemm_nn_simt(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *W,
                  int ld_w, const float *colscale, float alpha, float beta, float *Z, int ld_z,
                  const int *copy_if = nullptr);
// out (K x ncp) = W[:, 0:ncols], zero columns ncols..ncp-1
void select_cols(cudaStream_t st, int K, const float *W, int ld_w, int ncols, int ncp, float *out);
// In-place Cholesky of the K x K Gram G (ld) followed by inversion of the
// factor: Rinv (K x K, ld) = R^{-1} with G + shift I = R^T R.  Pivots <= tiny
// (zero columns) give an identity row/column so zero columns stay zero.
// shift_rel: shift = shift_rel * trace(G) / K.  ref_diag (optional, device, K
// floats): column norms^2 before a projection; columns with G_jj <= ref_tol *
// ref_diag[j] are treated as absent (dependent on the earlier blocks).
// skip_if (device int, may be NULL): return without work when it is nonzero.
// set_skip (device int, may be NULL; K <= 128): receives 1 when G is within
// 1e-2 of the identity entry by entry (the input block was already
// orthonormal to that level, so one more pass would change nothing), else 0.
void chol_inv(cudaStream_t st, int K, const float *G, int ld, float shift_rel, const float *ref_diag,
              float ref_tol, float *Rinv, const int *skip_if = nullptr, int *set_skip = nullptr);
// out[c] = sum_r X[r][c]^2 (deterministic).  scratch: colsumsq_scratch_floats(K).
size_t colsumsq_scratch_floats(int K);
void colsumsq(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *out, float *scratch);
// Gram on the tensor cores (k_tc.cu): G = X^T X for K <= 256, ld % 4 == 0,
// X 16-byte aligned.  partial: gram_tc_scratch_floats(R, K) floats.  err
// (device int, may be NULL) receives a nonzero code if a bounded wait expired.
// One cooperative launch for a narrow Krylov block (K <= 32): column norms
// (use_ref), two projections against Qp (R x cols), CholeskyQR passes (the
// first shifted by shift_rel * trace / K and with the dependence test
// G_jj <= ref_tol * norm_j^2; the third skipped when the second pass's Gram
// is within 1e-2 of I), result into out.  Qp's rows are staged in shared
// memory when they fit, else read from global memory.  Returns false
// (nothing launched) when the block's rows do not fit the CTAs' shared
// memory, rows are not 16-byte aligned, or the device has no cooperative
// launch; the caller then takes the separate kernels.
size_t orth_narrow_scratch_floats(int64_t R, int K, int cols);
bool orth_narrow(cudaStream_t st, int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out,
                 int ldo, bool use_ref, float shift_rel, float ref_tol, float *scratch);
size_t gram_tc_scratch_floats(int64_t R, int K);
bool gram_tc_supported(int K, int ld, const void *X);
void gram_tc(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *G, int ld_g, float *partial, int *err);
// Z (R x N, ld_z) = beta Z + alpha X (R x K, ld_x) W (K x N, ld_w) diag(colscale)
// on the tensor cores (k_tc.cu, 3xTF32).  Supported: N <= 256, K and N
// rounded up to 32 and 16 with a product of at most 16384, ld_x % 4 == 0, X
// 16-byte aligned.  err as for gram_tc (codes shifted by 4 bits).
bool gemm_nn_tc_supported(int64_t R, int K, int N, const void *X, int ld_x);
void gemm_nn_tc(cudaStream_t st, int64_t R, int K, int N, const float *X, int ld_x, const float *W, int ld_w,
                const float *colscale, float alpha, float beta, float *Z, int ld_z, int *err,
                const int *copy_if = nullptr);
// Top-kw eigenpairs of the symmetric K x K matrix A (lower triangle read).
// lam: kw floats descending; W: K x kw (ld_w).  work: eig_work_bytes(K, kw).
size_t eig_work_bytes(int K, int kw);
void eig_topk(cudaStream_t st, int K, int kw, const float *A, int lda, float *lam, float *W, int ld_w,
              void *work);


// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the previous kernel on the stream is finishing, so its
// launch overlaps that kernel's tail; it calls pdl_wait() before anything
// else, which returns once the previous kernel has completed and its writes
// are visible (for an ordinary launch it returns at once).  MC_PDL=0 turns
// the overlap off.
bool use_pdl();
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next kernel on the stream (if launched with launch_pdl) be
// scheduled now; it still waits in pdl_wait() for this kernel's completion
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  static_assert(sizeof...(KArgs) == sizeof...(Args), "launch_pdl: every kernel argument is passed");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MC_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for a kernel once per
// device and size (the launch paths call it before every launch; the driver
// call is not free on a path of a hundred launches per iteration).
void smem_attr(const void *fn, int bytes);
template <typename F>
inline void smem_attr(F *fn, int bytes) {
  smem_attr(reinterpret_cast<const void *>(fn), bytes);
}

// Blocked right-looking Cholesky of the lower triangle of a 64 x 64 matrix in
// shared memory (As[a][b], b <= a; 256 threads, all of which call it).  Every
// entry takes its updates one fused multiply-add at a time in pivot order,
// as the unblocked right-looking loop does, so the result is that loop's:
// on return As holds L below the diagonal (column j scaled by 1/sqrt of the
// pivot), the diagonal keeps the pivots A[j][j] before scaling, invd[j] =
// 1/sqrt(pivot) (0 for a pivot at or below drop) and flags[j] = 0 for a
// dropped pivot (otherwise untouched).  In 16-column blocks: (1) one warp
// factors the diagonal block, lane a holding row a in registers and each
// step's column passed by shuffles; (2) a thread per row below solves it
// against the block; (3) a thread per entry applies the block's rank-16
// update to the trailing matrix; three block barriers per block.
__device__ __forceinline__ void chol64_blocked(float (*As)[65], float drop, float *invd, float *flags) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned full = 0xffffffffu;
  for (int j0 = 0; j0 < 64; j0 += 16) {
    // (1) the diagonal block: lane a (and a + 16) holds row j0 + a
    if (wid == 0) {
      const int a = lane & 15;
      float r[16];
#pragma unroll
      for (int b = 0; b < 16; ++b) r[b] = b <= a ? As[j0 + a][j0 + b] : 0.f;
      auto diag_step = [&](const int j) {
        const float pj = __shfl_sync(full, r[j], j);
        const bool keep = pj > drop;
        const float inv = keep ? rsqrtf(pj) : 0.f;
        if (a > j) r[j] *= inv;
        const float la = r[j];
#pragma unroll
        for (int b = j + 1; b < 16; ++b) {
          const float lb = __shfl_sync(full, la, b);
          if (a >= b) r[b] = fmaf(-la, lb, r[b]);
        }
        if (lane == 0) {
          invd[j0 + j] = inv;
          if (!keep) flags[j0 + j] = 0.f;
        }
      };
#pragma unroll
      for (int j = 0; j < 8; ++j) diag_step(j);
#pragma unroll
      for (int j = 8; j < 16; ++j) diag_step(j);
      if (lane < 16) {
#pragma unroll
        for (int b = 0; b < 16; ++b)
          if (b <= a) As[j0 + a][j0 + b] = r[b];
      }
    }
    __syncthreads();
    // (2) the rows below it
    const int j1 = j0 + 16;
    if (j1 + tid < 64) {
      const int a = j1 + tid;
      float r[16];
#pragma unroll
      for (int b = 0; b < 16; ++b) r[b] = As[a][j0 + b];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float l = r[j] * invd[j0 + j];
        r[j] = l;
#pragma unroll
        for (int b = j + 1; b < 16; ++b) r[b] = fmaf(-l, As[j0 + b][j0 + j], r[b]);
      }
#pragma unroll
      for (int b = 0; b < 16; ++b) As[a][j0 + b] = r[b];
    }
    __syncthreads();
    // (3) the trailing matrix
    if (j1 < 64) {
#pragma unroll 4
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u, a = e >> 6, b = e & 63;
        if (b < j1 || b > a) continue;
        float v = As[a][b];
#pragma unroll
        for (int k = 0; k < 16; ++k) v = fmaf(-As[a][j0 + k], As[b][j0 + k], v);
        As[a][b] = v;
      }
    }
    __syncthreads();
  }
}

}  // namespace mc
