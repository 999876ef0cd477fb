// Gram G = X^T X of a tall float32 panel (R x K, K <= 256) on the fifth-
// generation tensor cores: the B = A^T A step of eigSVD (Alg. 3 step 1) and
// the Gram of each CholeskyQR pass.
//
// One CTA of 128 threads per row range.  TMA loads 32-row stages of the panel
// as 32-column boxes (128-byte rows, 128-byte swizzle) into a double-buffered
// shared-memory ring.  The threads split every value into a TF32 "hi" part
// and a TF32 remainder "lo" (both rounded to nearest) and write both
// transposed into the K-major 128-byte-swizzled operand layout (the panel's
// rows are the reduction dimension; a 32-row stage is exactly one 128-byte
// swizzle row per panel column).  One thread issues tcgen05.mma kind::tf32 and
// accumulates hi*hi + hi*lo + lo*hi into float32 accumulators in tensor
// memory, which gives about float32 accuracy.
// Up to K = 128 one 128 x N tile covers the Gram; above, a second 128-row tile
// covers the remaining upper block.  Each CTA writes its partial Gram; a
// reduction kernel adds the partials in a fixed order.  Every wait on an
// mbarrier is bounded: on expiry the kernel records an error code and
// finishes its outstanding work before it returns.
#include "mc_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace mc {
namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_KT = 32;                 // panel rows per stage (4 MMA k-steps of 8)
constexpr int TC_BOX_BYTES = 32 * TC_KT * 4;  // one 32-column box: 4 KiB
constexpr int TC_MAX_BOXES = 8;           // K <= 256
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bulk tensor stores from shared memory (plain, or added to what global
// memory holds), grouped for completion by the issuing thread.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_add_2d(const CUtensorMap *map, const void *src, int x, int y) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int P>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(P) : "memory");
}
template <int P>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(P) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand in 128-byte-swizzled
// atoms (8 rows of 128 bytes = 32 tf32 along K, 1024 bytes per atom): the
// stride between 8-row groups is 1024 bytes; the leading offset is unused for
// this layout.  A k-step of 8 elements advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused): 16 bytes
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset: 1024 bytes
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
  d |= static_cast<uint64_t>(2) << 61;  // 128-byte swizzle
  return d;
}

// Instruction descriptor: D f32, A/B tf32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                                  // D format: f32
         | (2u << 7)                                // A format: tf32
         | (2u << 10)                               // B format: tf32
         | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  // load and wait in one statement: the registers are defined only after the wait
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Split of a float32 value for 3xTF32 products: hi is the value rounded to
// the nearest TF32 number (10-bit mantissa, ties away from zero), the
// remainder x - hi is exact in float32 and is rounded the same way, so
// hi + lo carries x to about 2^-24 relative, as float32 does (truncating both
// parts would leave 2^-22).
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void tf32_split(float x, float &h, float &l) {
  h = tf32_rn(x);
  l = tf32_rn(x - h);
}

struct TcSmem {
  // 1024-byte aligned ring: raw / hi / lo, two stages each, boxes of 4 KiB
  static constexpr size_t stage_bytes = (size_t)TC_MAX_BOXES * TC_BOX_BYTES;  // 32 KiB
  static constexpr size_t total = 6 * stage_bytes + 1024;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap xmap, int64_t R, int K, int nbox, int two_tiles, int N0,
               uint32_t tmem_cols, int64_t rows_per_cta, float *__restrict__ partial, int Kp, int *__restrict__ err) {
  extern __shared__ __align__(1024) uint8_t tc_raw_smem[];
  __shared__ __align__(8) uint64_t full_bar[2];
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_raw_smem) + 1023) & ~uintptr_t(1023));
  uint8_t *raw[2] = {base, base + TcSmem::stage_bytes};
  uint8_t *hi[2] = {base + 2 * TcSmem::stage_bytes, base + 3 * TcSmem::stage_bytes};
  uint8_t *lo[2] = {base + 4 * TcSmem::stage_bytes, base + 5 * TcSmem::stage_bytes};
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t r0 = blockIdx.x * rows_per_cta;
  const int64_t r1 = min(R, r0 + rows_per_cta);
  const int S = r1 > r0 ? static_cast<int>((r1 - r0 + TC_KT - 1) / TC_KT) : 0;
  const uint32_t stage_tx = static_cast<uint32_t>(nbox) * TC_BOX_BYTES;

  if (tid == 0) {
    mbar_init(&full_bar[0], 1);
    mbar_init(&full_bar[1], 1);
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  auto issue_loads = [&](int s, int b) {
    mbar_expect_tx(&full_bar[b], stage_tx);
    const int y = static_cast<int>(r0 + (int64_t)s * TC_KT);
    for (int j = 0; j < nbox; ++j) tma_load_2d(raw[b] + j * TC_BOX_BYTES, &xmap, 32 * j, y, &full_bar[b]);
  };
  // tid 0 issues every load and every MMA: it alone tracks how far both got,
  // for a clean exit after an expired wait
  int issued = 0, committed = -1;
  if (tid == 0)
    for (; issued < S && issued < 2; ++issued) issue_loads(issued, issued);

  const uint32_t id0 = idesc_tf32(128, N0);
  const uint32_t id1 = idesc_tf32(128, 128);
  const int nvec = nbox * TC_BOX_BYTES / 16;  // float4 per stage
  for (int s = 0; s < S; ++s) {
    const int b = s & 1;
    bool ok = mbar_wait(&full_bar[b], (s >> 1) & 1);
    if (ok && s >= 2) ok = mbar_wait(&mma_bar[b], ((s - 2) >> 1) & 1);
    if (!ok) atomicOr(&s_fail, 1);
    // split into tf32 hi and float32 lo and transpose: the TMA tile holds
    // element (r, c) (stage row r = reduction index, panel column c) at
    //   box(c/32) * 4096 + r * 128 + (((c % 32) / 4) ^ (r % 8)) * 16 + (c % 4) * 4;
    // the K-major operand stores it at
    //   (c / 8) * 1024 + (c % 8) * 128 + ((r / 4) ^ (c % 8)) * 16 + (r % 4) * 4.
    const float4 *src = reinterpret_cast<const float4 *>(raw[b]);
    float *dh = reinterpret_cast<float *>(hi[b]);
    float *dl = reinterpret_cast<float *>(lo[b]);
    // a warp takes one 4-column group of a box across its 32 rows (lane = row):
    // the swizzled reads and the transposed writes are then free of bank conflicts
    for (int q = tid; q < nvec; q += TC_THREADS) {
      const int box = q >> 8, k4 = (q >> 5) & 7, r = q & 31;  // 256 float4 per box
      const int c0 = box * 32 + k4 * 4;
      const float4 v = src[box * 256 + r * 8 + (k4 ^ (r & 7))];
      const float vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u;
        const int off = (c >> 3) * 256 + (c & 7) * 32 + ((((r >> 2) ^ (c & 7)) & 7) << 2) + (r & 3);
        float h, l;
        tf32_split(vals[u], h, l);
        dh[off] = h;
        dl[off] = l;
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (s_fail) break;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(hi[b]), al = smem_u32(lo[b]);
      for (int kg = 0; kg < TC_KT / 8; ++kg) {
        const uint32_t ko = kg * 32;  // next 8 elements along K
        const uint32_t acc0 = (s > 0 || kg > 0) ? 1u : 0u;
        // tile 0: rows 0..127 of G (panel columns 0..127), columns 0..N0-1
        mma_tf32(tmem, smem_desc(ah + ko), smem_desc(ah + ko), id0, acc0);
        mma_tf32(tmem, smem_desc(ah + ko), smem_desc(al + ko), id0, 1u);
        mma_tf32(tmem, smem_desc(al + ko), smem_desc(ah + ko), id0, 1u);
        if (two_tiles) {
          // tile 1: rows 128..255, columns 128..255 (16 atoms = 16 KiB further)
          const uint32_t o1 = 16 * 1024 + ko;
          const uint32_t d1 = tmem + static_cast<uint32_t>(N0);
          mma_tf32(d1, smem_desc(ah + o1), smem_desc(ah + o1), id1, acc0);
          mma_tf32(d1, smem_desc(ah + o1), smem_desc(al + o1), id1, 1u);
          mma_tf32(d1, smem_desc(al + o1), smem_desc(ah + o1), id1, 1u);
        }
      }
      mma_commit(&mma_bar[b]);
      committed = s;
      if (s + 2 < S) {
        issue_loads(s + 2, b);
        issued = s + 3;
      }
    }
    __syncwarp();  // warp 0 reconverges after thread 0's issue
  }
  __syncwarp();
  __syncthreads();
  if (tid == 0) {
    // The last commit covers every MMA issued before it: wait for it.  Then
    // wait for the loads of stages that no MMA consumed (only after an early
    // exit): on each barrier the phase waited for is the latest one armed, so
    // a completed phase returns at once.  All waits are bounded.
    if (committed >= 0 && !mbar_wait(&mma_bar[committed & 1], (committed >> 1) & 1)) atomicOr(&s_fail, 2);
    for (int t = committed + 1; t < issued; ++t) mbar_wait(&full_bar[t & 1], (t >> 1) & 1);
  }
  __syncwarp();
  __syncthreads();
  // read the accumulators only after a complete run
  const bool have = S > 0 && !s_fail;
  tc_fence_after();
  float *out = partial + (size_t)blockIdx.x * Kp * Kp;
  const int row = 32 * wid + lane;  // accumulator lane = row within the tile
  for (int tile = 0; tile < (two_tiles ? 2 : 1); ++tile) {
    const int ncols = tile == 0 ? N0 : 128;
    const int grow = tile * 128 + row;
    const int gcol0 = tile * 128;
    const uint32_t tcol = tile == 0 ? 0u : static_cast<uint32_t>(N0);
    for (int c = 0; c < ncols; c += 16) {
      float v[16] = {};
      // have is the same in every thread: the warp-wide load is skipped as a whole
      if (have) tmem_ld16(tmem + (static_cast<uint32_t>(32 * wid) << 16) + tcol + c, v);
      if (grow < Kp) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int gc = gcol0 + c + i;
          if (gc < Kp) out[(size_t)grow * Kp + gc] = v[i];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  if (tid == 0 && s_fail && err) atomicOr(err, s_fail);
}

// G (K x K, ld_g) = sum of the partials.  Partial entries are valid in rows
// 0..127 and in columns >= 128; the block rows >= 128, columns < 128 is read
// transposed from rows < 128.
__global__ void __launch_bounds__(256)
gram_tc_reduce_kernel(int K, int nsplit, const float *__restrict__ partial, int Kp, float *__restrict__ G, int ld_g) {
  // a block covers 32 outputs with 8 lanes of split groups each (fixed order)
  __shared__ float sh[8][33];
  const int64_t total = (int64_t)K * K;
  const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
  for (int64_t base = (int64_t)blockIdx.x * 32; base < total; base += (int64_t)gridDim.x * 32) {
    const int64_t t = base + o;
    float acc = 0.f;
    int i = 0, j = 0;
    if (t < total) {
      i = static_cast<int>(t / K);
      j = static_cast<int>(t % K);
      int si = i, sj = j;
      if (i >= 128 && j < 128) {
        si = j;
        sj = i;
      }
      const float *p = partial + (size_t)si * Kp + sj;
      for (int sp = g; sp < nsplit; sp += 8) acc += p[(size_t)sp * Kp * Kp];
    }
    sh[g][o] = acc;
    __syncthreads();
    if (g == 0 && t < total) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) v += sh[q][o];
      G[(int64_t)i * ld_g + j] = v;
    }
    __syncthreads();
  }
}

// ---- panel times small factor on the tensor cores ---------------------------
// Z (R x N) = alpha X (R x K) W (K x N) diag(colscale) + beta Z, float32 in and
// out, for K_p N_p <= 16384 (K_p = K rounded up to 32, N_p = N rounded up to
// 16): the block products of the Krylov orthonormalisation (X R^{-1},
// X - Q_prev C) and the Ritz factors U = Q W, V = B^T W S^{-1} (Alg. 5 step
// 11, Alg. 3 step 4).  TMA brings 128-row x 32-column boxes of X (128-byte
// rows, 128-byte swizzle), which is already the K-major operand layout of
// tcgen05.mma; W, staged once per CTA, is written transposed into the same
// layout as hi and lo parts; the product accumulates hi*hi + hi*lo + lo*hi in
// float32 in tensor memory (about float32 accuracy).
constexpr int NT_BM = 128, NT_KC = 32;
constexpr int NT_BOX_BYTES = NT_BM * NT_KC * 4;  // 16 KiB
constexpr int NT_MAX_W = 16384;                   // K_p * N_p floats
constexpr size_t NT_SMEM_LIMIT = 226 * 1024;

// The kernel is warp-specialised: 512 threads in roles that hand boxes to each other through mbarriers:
//   warp 0, lane 0   TMA producer: loads box g into stage g % nst once the
//                    MMAs of box g - nst released it (the first nst boxes
//                    before W is staged);
//   warp 1, lane 0   MMA issuer: hi*hi + hi*lo + lo*hi per 8-column step into
//                    one of two TMEM accumulators (tiles alternate), releases
//                    the stage (commit) and, after a tile's last box, hands
//                    the accumulator to the epilogue (commit);
//   warps 4..11      split each landed box in place into TF32 hi and lo and
//                    signal the issuer;
//   warps 12..15     epilogue: each reads its 32 accumulator rows (tcgen05.ld,
//                    lanes 32 (w % 4) ..), scales them and stages 32 columns
//                    at a time in its own shared memory (one or two
//                    buffers), from where one lane hands them to a bulk
//                    tensor store (beta = 0) or a bulk tensor add into Z
//                    (beta = 1), then frees the accumulator.  Other beta
//                    values, or a Z the tensor map cannot describe, take
//                    float4 stores from the staging buffer instead.
// So the split of box g + 1, the MMAs of box g and the epilogue of the
// previous tile run at the same time.  Every wait is bounded: an expiry sets
// a shared failure flag that ends every role's loop; each role then waits
// (bounded) for its own outstanding copies or MMAs before the block frees its
// tensor memory.
constexpr int NW_THREADS = 512;
constexpr int NW_MAXST = 4;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool failed(const volatile int *f) { return *f != 0; }

__global__ void __launch_bounds__(NW_THREADS, 1)
gemm_nn_tc_ws_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap zmap, int zmode,
                     int ebuf, int cat, int64_t R, int K, int N, int Kp, int Np,
                     uint32_t tmem_cols, int nst, const float *__restrict__ W, int ld_w,
                     const float *__restrict__ colscale, float alpha, float beta, float *__restrict__ Z, int ld_z,
                     int *__restrict__ err, const int *__restrict__ copy_if, int ld_x, const float *__restrict__ Xp) {
  extern __shared__ __align__(1024) uint8_t nw_raw_smem[];
  __shared__ __align__(8) uint64_t full_bar[NW_MAXST], split_bar[NW_MAXST], empty_bar[NW_MAXST];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail;
  pdl_wait();
  pdl_trigger();
  if (copy_if && *copy_if) {
    // copy mode (the factor is the identity): Z = X, K == N
    for (int64_t e = blockIdx.x * (int64_t)NW_THREADS + threadIdx.x; e < R * K; e += (int64_t)gridDim.x * NW_THREADS) {
      const int64_t r = e / K;
      const int c = static_cast<int>(e % K);
      Z[r * ld_z + c] = Xp[r * ld_x + c];
    }
    return;
  }
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(nw_raw_smem) + 1023) & ~uintptr_t(1023));
  const int kchunks = Kp / NT_KC;
  const size_t wbytes = (size_t)Kp * Np * 4;
  uint8_t *whi = base, *wlo = base + wbytes;
  uint8_t *stg = base + 2 * wbytes;                                         // nst x (hi, lo) boxes
  float *epi = reinterpret_cast<float *>(stg + (size_t)nst * 2 * NT_BOX_BYTES);  // 4 warps x ebuf x 32 x 32 floats
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (R + NT_BM - 1) / NT_BM;
  const int my_tiles = blockIdx.x < ntiles ? static_cast<int>((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int G = my_tiles * kchunks;
  const int pre = min(nst, G);  // boxes in flight before W is staged
  volatile int *vfail = &s_fail;
  auto box_hi = [&](int s) { return stg + (size_t)s * 2 * NT_BOX_BYTES; };
  auto box_lo = [&](int s) { return stg + (size_t)s * 2 * NT_BOX_BYTES + NT_BOX_BYTES; };
  auto issue = [&](int s, int kc, int tl) {
    const int64_t tile = blockIdx.x + (int64_t)tl * gridDim.x;
    mbar_expect_tx(&full_bar[s], NT_BOX_BYTES);
    tma_load_2d(box_hi(s), &xmap, kc * NT_KC, static_cast<int>(tile * NT_BM), &full_bar[s]);
  };

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&split_bar[s], 8);   // one arrival per split warp
      mbar_init(&empty_bar[s], 1);   // MMA commit
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf_bar[a], 1);    // MMA commit
      mbar_init(&acce_bar[a], 4);    // one arrival per epilogue warp
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the first boxes do not depend on W: their copies overlap its staging
    for (int g = 0; g < pre; ++g) issue(g, g % kchunks, g / kchunks);
  }
  if (wid == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // W^T (N_p x K_p, K-major, 128-byte swizzle) as hi and lo: element (n, k) of
  // column block kc at kc * N_p * 128 + (n / 8) * 1024 + (n % 8) * 128 +
  // (((k % 32) / 4) ^ (n % 8)) * 16 + (k % 4) * 4 of its part; with cat the
  // parts interleave by column block, [hi | lo] as 2 N_p operand rows per
  // block (one MMA then takes X_hi against both).  Eight loads per thread
  // are in flight before their values are split and stored.
  for (int e0 = tid; e0 < Kp * Np; e0 += 8 * NW_THREADS) {
    float w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * NW_THREADS, k = e / Np, n = e % Np;
      w[u] = (e < Kp * Np && k < K && n < N) ? W[(int64_t)k * ld_w + n] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * NW_THREADS, k = e / Np, n = e % Np;
      if (e >= Kp * Np) break;
      const int kc = k / NT_KC, kl = k % NT_KC;
      float h, lw;
      tf32_split(w[u], h, lw);
      const size_t off = (size_t)kc * Np * 128 * (cat ? 2 : 1) + (n >> 3) * 1024 + (n & 7) * 128 +
                         (((kl >> 2) ^ (n & 7)) << 4) + (kl & 3) * 4;
      *reinterpret_cast<float *>(whi + off) = h;
      *reinterpret_cast<float *>((cat ? whi + (size_t)Np * 128 : wlo) + off) = lw;
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const unsigned fullm = 0xffffffffu;
  if (wid == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      // the loop runs only when pre == nst, so box g = pre reuses stage 0
      int issued = pre, s = 0, kc = pre % kchunks, tl = pre / kchunks;
      uint32_t eph = 0;
      for (int g = pre; g < G; ++g) {
        if (failed(vfail)) break;
        if (!mbar_wait(&empty_bar[s], eph)) {
          atomicOr(&s_fail, 1);
          break;
        }
        issue(s, kc, tl);
        issued = g + 1;
        if (++s == nst) {
          s = 0;
          eph ^= 1u;
        }
        if (++kc == kchunks) {
          kc = 0;
          ++tl;
        }
      }
      // every issued copy lands before the block exits: the last one per stage
      // is the latest phase armed there (a completed one returns at once)
      for (int g = max(0, issued - nst); g < issued; ++g) mbar_wait(&full_bar[g % nst], (g / nst) & 1);
    }
  } else if (wid == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      // A single thread issues every MMA, so the loop keeps its stage, phase,
      // chunk and tile counters incrementally and moves descriptors by adding
      // address units (16 bytes) instead of rebuilding them.
      const uint32_t idesc = idesc_tf32(NT_BM, Np), idesc2 = idesc_tf32(NT_BM, 2 * Np);
      const uint64_t wstep = static_cast<uint64_t>(Np) * 128 * (cat ? 2 : 1) >> 4;  // one 32-row block of W^T
      const uint64_t xstep = static_cast<uint64_t>(2 * NT_BOX_BYTES) >> 4;  // one (hi, lo) stage
      const uint64_t dwh = smem_desc(smem_u32(whi)), dwl = smem_desc(smem_u32(wlo)), dx = smem_desc(smem_u32(stg));
      int committed = -1;
      uint32_t committed_ph = 0;
      int s = 0, kc = 0, tl = 0;
      uint32_t ph = 0;
      for (int g = 0; g < G; ++g) {
        if (failed(vfail)) break;
        const int a = tl & 1;
        if (kc == 0 && tl >= 2 && !mbar_wait(&acce_bar[a], ((tl >> 1) - 1) & 1)) {
          atomicOr(&s_fail, 2);
          break;
        }
        if (!mbar_wait(&split_bar[s], ph)) {
          atomicOr(&s_fail, 4);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + static_cast<uint32_t>(a * Np * (cat ? 2 : 1));
        const uint64_t ah = dx + s * xstep, al = ah + (NT_BOX_BYTES >> 4);
        const uint64_t bh = dwh + kc * wstep, bl = dwl + kc * wstep;
        if (cat) {
          // X_hi [W_hi | W_lo] into accumulator columns [0, Np) and [Np, 2 Np),
          // X_lo W_hi into [0, Np); the epilogue adds the two halves
#pragma unroll
          for (int ks = 0; ks < NT_KC / 8; ++ks) {
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(d, ah + 2 * ks, bh + 2 * ks, idesc2, acc0);
            mma_tf32(d, al + 2 * ks, bh + 2 * ks, idesc, 1u);
          }
        } else {
#pragma unroll
          for (int ks = 0; ks < NT_KC / 8; ++ks) {
            const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(d, ah + 2 * ks, bh + 2 * ks, idesc, acc0);  // 8 columns = 32 bytes further
            mma_tf32(d, ah + 2 * ks, bl + 2 * ks, idesc, 1u);
            mma_tf32(d, al + 2 * ks, bh + 2 * ks, idesc, 1u);
          }
        }
        mma_commit(&empty_bar[s]);
        if (kc == kchunks - 1) mma_commit(&accf_bar[a]);
        committed = s;
        committed_ph = ph;
        if (++s == nst) {
          s = 0;
          ph ^= 1u;
        }
        if (++kc == kchunks) {
          kc = 0;
          ++tl;
        }
      }
      // the last commit covers every MMA issued before it
      if (committed >= 0 && !mbar_wait(&empty_bar[committed], committed_ph)) atomicOr(&s_fail, 64);
    }
  } else if (wid >= 4 && wid < 12) {
    // ---- split into TF32 hi (in place) and float32 lo ----
    const int st = tid - 128;
    int s = 0;
    uint32_t ph = 0;
    for (int g = 0; g < G; ++g, s = s + 1 == nst ? 0 : s + 1, ph ^= s == 0 ? 1u : 0u) {
      if (__any_sync(fullm, failed(vfail))) break;
      const bool ok = mbar_wait(&full_bar[s], ph);
      if (!__all_sync(fullm, ok)) {
        atomicOr(&s_fail, 8);
        break;
      }
      float4 *hi4 = reinterpret_cast<float4 *>(box_hi(s));
      float4 *lo4 = reinterpret_cast<float4 *>(box_lo(s));
#pragma unroll 4
      for (int q = st; q < NT_BOX_BYTES / 16; q += 256) {
        const float4 v = hi4[q];
        float4 h, l;
        tf32_split(v.x, h.x, l.x);
        tf32_split(v.y, h.y, l.y);
        tf32_split(v.z, h.z, l.z);
        tf32_split(v.w, h.w, l.w);
        hi4[q] = h;
        lo4[q] = l;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&split_bar[s]);
    }
  } else if (wid >= 12) {
    // ---- epilogue: accumulator rows 32 (w % 4) .. + 31 of each tile ----
    const int ew = wid - 12;
    const bool vec_out = ld_z % 4 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15u) == 0;
    int chunk = 0;         // 32-column chunks staged by this warp
    bool pending = false;  // lane 0: bulk stores issued (their reads of the buffers may be in flight)
    for (int tl = 0; tl < my_tiles; ++tl) {
      if (__any_sync(fullm, failed(vfail))) break;
      const int a = tl & 1;
      const bool ok = mbar_wait(&accf_bar[a], (tl >> 1) & 1);
      if (!__all_sync(fullm, ok)) {
        atomicOr(&s_fail, 16);
        break;
      }
      tc_fence_after();
      const int64_t row0 = ((int64_t)blockIdx.x + (int64_t)tl * gridDim.x) * NT_BM + 32 * ew;
      for (int c0 = 0; c0 < N; c0 += 32, ++chunk) {
        // 32 rows x 32 columns, row = lane, float4 q of a row at q ^ (row % 8):
        // the 128-byte-swizzled box of the bulk tensor store
        float *bf = epi + (size_t)(ew * ebuf + chunk % ebuf) * 1024;
        float4 *buf4 = reinterpret_cast<float4 *>(bf);
        if (zmode != 0) {
          // the store that last read this buffer has finished reading it
          if (lane == 0 && pending) {
            if (ebuf == 2) bulk_wait_read<1>();
            else bulk_wait_read<0>();
          }
          __syncwarp();
        }
        for (int c = 0; c < 32 && c0 + c < N; c += 16) {
          float v[16];
          const uint32_t ta = tmem + (static_cast<uint32_t>(32 * ew) << 16) +
                              static_cast<uint32_t>(a * Np * (cat ? 2 : 1) + c0 + c);
          tmem_ld16(ta, v);
          if (cat) {
            float v2[16];
            tmem_ld16(ta + static_cast<uint32_t>(Np), v2);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += v2[k];
          }
          if (zmode != 0) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int col = c0 + c + k;
              v[k] = col < N ? v[k] * alpha * (colscale ? colscale[col] : 1.0f) : 0.f;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            buf4[lane * 8 + (((c >> 2) + u) ^ (lane & 7))] =
                make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        }
        if (zmode != 0) {
          fence_proxy_async();
          __syncwarp();
          // rows past R and columns past N are clipped by the tensor map
          if (lane == 0 && row0 < R) {
            if (zmode == 1) tma_store_2d(&zmap, bf, c0, static_cast<int>(row0));
            else tma_add_2d(&zmap, bf, c0, static_cast<int>(row0));
            bulk_commit();
            pending = true;
          }
          continue;
        }
        __syncwarp();
        for (int e = lane; e < 32 * 8; e += 32) {
          const int rr = e >> 3, q = e & 7, col = c0 + 4 * q;
          const int64_t grow = row0 + rr;
          if (grow >= R || col >= N) continue;
          const float4 v4 = buf4[rr * 8 + (q ^ (rr & 7))];
          const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
          float *z = Z + grow * ld_z + col;
          if (vec_out && col + 3 < N) {
            float o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = vv[i] * alpha * (colscale ? colscale[col + i] : 1.0f);
            if (beta != 0.f) {
              const float4 zo = *reinterpret_cast<const float4 *>(z);
              o[0] += beta * zo.x;
              o[1] += beta * zo.y;
              o[2] += beta * zo.z;
              o[3] += beta * zo.w;
            }
            *reinterpret_cast<float4 *>(z) = make_float4(o[0], o[1], o[2], o[3]);
          } else {
            for (int i = 0; i < 4 && col + i < N; ++i)
              z[i] = (beta != 0.f ? beta * z[i] : 0.f) + vv[i] * alpha * (colscale ? colscale[col + i] : 1.0f);
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[a]);
    }
    // every bulk store has completed before the block exits
    if (lane == 0 && pending) bulk_wait_all<0>();
  }
  // The producer and issuer roles ran on lane 0 alone: the warp reconverges
  // before the block barrier, which must count every warp only once it has
  // left its role (the tensor memory is freed after it).
  __syncwarp();
  __syncthreads();
  tc_fence_after();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  if (tid == 0 && s_fail && err) atomicOr(err, s_fail << 8);
}

// ---- X1^T X2 on the tensor cores (Grams and projections) --------------------
// C (K1 x K2) = X1^T X2 summed over R rows, X1 (R x K1) and X2 (R x K2) tall
// float32 panels, K1, K2 <= 256: the Grams of the block orthonormalisation
// (Alg. 5 steps 3-7 as CholeskyQR, Lemmas 2-3), its projections Q_prev^T X
// and the Ritz Gram B B^T (Alg. 5 step 9, Alg. 3 step 1).  The MMA's
// reduction dimension is the panels' rows, so every 32-row stage is
// transposed into the K-major operand layout (as in gram_tc_kernel).  Each
// CTA covers a range of rows and writes one partial K1_p x K2_p tile; a
// fixed-order reduction adds the partials.
//
// Warp-specialised, 384 threads, two rings in shared memory:
//   warp 0, lane 0   TMA producer: raw stages of 32 nsub rows (nsub = 1, 2
//                    or 4), the 32-column boxes of X1 (and of X2 unless it
//                    is X1), once the splitters released the raw stage (tall
//                    boxes: fewer, larger copies);
//   warps 4..11      split each 32-row part of a raw stage into TF32 hi and
//                    lo (rounded to nearest) and write both transposed into
//                    a split stage, handing it to the issuer; the raw stage
//                    is released after its last part;
//   warp 1, lane 0   MMA issuer: hi*hi + hi*lo + lo*hi for every 8-row step
//                    into one accumulator per 128 columns of X1 (for the Gram
//                    of 33..64 columns one MMA, hi^T [hi | lo], see below),
//                    releasing the split stage by a commit;
//   warps 8..11      after the last stage, read the accumulators (tcgen05.ld)
//                    and write the partial tile.
// The MMAs take the 32-row parts in row order.  Every wait is bounded; an
// expiry ends every role, each drains its own copies or MMAs, and the error
// code goes to err.
constexpr int TT_THREADS = 384, TT_KT = 32, TT_MAXST = 6;
constexpr int TT_BOX = TT_KT * 32 * 4;  // 32 rows x 32 columns: 4 KiB

__global__ void __launch_bounds__(TT_THREADS, 1)
gemm_tn_tc_ws_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, int same,
                     int sym, int64_t R, int nbA, int nbB, int Np, int mt, uint32_t tmem_cols, int nsub, int nr,
                     int ns, int64_t rows_per_cta, float *__restrict__ partial, int K1p, int K2p,
                     int *__restrict__ err, const int *__restrict__ skip) {
  extern __shared__ __align__(1024) uint8_t tt_raw_smem[];
  __shared__ __align__(8) uint64_t full_bar[TT_MAXST], rawfree_bar[TT_MAXST], split_bar[TT_MAXST],
      splitfree_bar[TT_MAXST];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int s_fail;
  pdl_wait();
  pdl_trigger();
  if (skip && *skip) return;  // a pass the previous one made unnecessary
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tt_raw_smem) + 1023) & ~uintptr_t(1023));
  const int nbr = nbA + (same ? 0 : nbB);                  // raw boxes per stage
  const int rb = TT_KT * nsub;                             // rows per raw stage
  const size_t box_bytes = (size_t)rb * 128;               // one 32-column box of a raw stage
  const size_t raw_bytes = (size_t)nbr * box_bytes;
  const size_t spl_bytes = (size_t)(4 * mt + (same ? 0 : nbB)) * TT_BOX;  // one of hi / lo
  auto raw = [&](int s) { return base + (size_t)s * raw_bytes; };
  auto hi = [&](int s) { return base + (size_t)nr * raw_bytes + (size_t)s * 2 * spl_bytes; };
  auto lo = [&](int s) { return base + (size_t)nr * raw_bytes + (size_t)s * 2 * spl_bytes + spl_bytes; };
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t r0 = blockIdx.x * rows_per_cta;
  const int64_t r1 = min(R, r0 + rows_per_cta);
  const int S = r1 > r0 ? static_cast<int>((r1 - r0 + TT_KT - 1) / TT_KT) : 0;  // 32-row parts
  const int SR = (S + nsub - 1) / nsub;                                           // raw stages
  volatile int *vfail = &s_fail;
  const unsigned fullm = 0xffffffffu;

  if (tid == 0) {
    for (int s = 0; s < nr; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&rawfree_bar[s], 8);  // one arrival per split warp
    }
    for (int s = 0; s < ns; ++s) {
      mbar_init(&split_bar[s], 8);
      mbar_init(&splitfree_bar[s], 1);  // MMA commit
    }
    mbar_init(&acc_bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // A (X1^T) is laid out as 4 mt boxes (128 columns per accumulator: the MMA
  // reads 128 rows of A whatever K1), B (X2^T) follows unless it is A
  const int aboxes = 4 * mt;
  if (wid == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      int issued = 0, s = 0;
      uint32_t ph = 0;  // parity of raw stage s's current use
      int y = static_cast<int>(r0);
      for (int g = 0; g < SR; ++g, y += rb) {
        if (failed(vfail)) break;
        if (g >= nr && !mbar_wait(&rawfree_bar[s], ph ^ 1u)) {
          atomicOr(&s_fail, 1);
          break;
        }
        mbar_expect_tx(&full_bar[s], static_cast<uint32_t>(raw_bytes));
        for (int j = 0; j < nbA; ++j) tma_load_2d(raw(s) + j * box_bytes, &amap, 32 * j, y, &full_bar[s]);
        if (!same)
          for (int j = 0; j < nbB; ++j) tma_load_2d(raw(s) + (nbA + j) * box_bytes, &bmap, 32 * j, y, &full_bar[s]);
        issued = g + 1;
        if (++s == nr) {
          s = 0;
          ph ^= 1u;
        }
      }
      for (int g = max(0, issued - nr); g < issued; ++g) mbar_wait(&full_bar[g % nr], (g / nr) & 1);
    }
  } else if (wid == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      // one thread issues every MMA: incremental stage and phase, descriptors
      // moved by adding address units (16 bytes)
      const uint32_t idesc = idesc_tf32(128, Np), idesc_sym = idesc_tf32(128, 128);
      const uint64_t sstep = static_cast<uint64_t>(2 * spl_bytes) >> 4;
      const uint64_t dh0 = smem_desc(smem_u32(hi(0))), dl0 = smem_desc(smem_u32(lo(0)));
      const uint64_t boff = same ? 0 : static_cast<uint64_t>(aboxes * TT_BOX) >> 4;
      int committed = -1, ncommit = 0, s = 0;
      uint32_t ph = 0, committed_ph = 0;
      for (int g = 0; g < S; ++g) {
        if (failed(vfail)) break;
        if (!mbar_wait(&split_bar[s], ph)) {
          atomicOr(&s_fail, 4);
          break;
        }
        tc_fence_after();
        const uint64_t ah = dh0 + s * sstep, al = dl0 + s * sstep, bh = ah + boff, bl = al + boff;
        if (sym) {
          // the Gram of at most 64 columns: the stage holds [hi | lo] as 128
          // operand rows, so one MMA per 8-row step gives hi^T hi (columns
          // 0..63) and hi^T lo (64..127); lo^T hi is the latter's transpose
#pragma unroll
          for (int ks = 0; ks < TT_KT / 8; ++ks)
            mma_tf32(tmem, ah + 2 * ks, ah + 2 * ks, idesc_sym, (g > 0 || ks > 0) ? 1u : 0u);
        } else if (mt == 1) {
#pragma unroll
          for (int ks = 0; ks < TT_KT / 8; ++ks) {
            const uint32_t acc0 = (g > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(tmem, ah + 2 * ks, bh + 2 * ks, idesc, acc0);  // 8 rows = 32 bytes further
            mma_tf32(tmem, ah + 2 * ks, bl + 2 * ks, idesc, 1u);
            mma_tf32(tmem, al + 2 * ks, bh + 2 * ks, idesc, 1u);
          }
        } else {
#pragma unroll
          for (int ks = 0; ks < TT_KT / 8; ++ks) {
            const uint32_t acc0 = (g > 0 || ks > 0) ? 1u : 0u;
            for (int t = 0; t < mt; ++t) {
              const uint32_t d = tmem + static_cast<uint32_t>(t * Np);
              const uint64_t ao = static_cast<uint64_t>(t) * 1024 + 2 * ks;  // 128 columns = 16 KiB further
              mma_tf32(d, ah + ao, bh + 2 * ks, idesc, acc0);
              mma_tf32(d, ah + ao, bl + 2 * ks, idesc, 1u);
              mma_tf32(d, al + ao, bh + 2 * ks, idesc, 1u);
            }
          }
        }
        mma_commit(&splitfree_bar[s]);
        committed = s;
        committed_ph = ph;
        ++ncommit;
        if (++s == ns) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (S > 0 && ncommit == S) mma_commit(&acc_bar);
      if (committed >= 0 && !mbar_wait(&splitfree_bar[committed], committed_ph)) atomicOr(&s_fail, 8);
    }
  } else if (wid >= 4) {
    // ---- transpose and split ----
    const int st = tid - 128;
    int sr = 0, ss = 0, sub = 0;
    uint32_t phr = 0, phs = 0;
    for (int g = 0; g < S; ++g) {
      if (__any_sync(fullm, failed(vfail))) break;
      bool ok = sub != 0 || mbar_wait(&full_bar[sr], phr);
      if (ok && g >= ns) ok = mbar_wait(&splitfree_bar[ss], phs ^ 1u);
      if (!__all_sync(fullm, ok)) {
        atomicOr(&s_fail, 2);
        break;
      }
      // raw box j holds element (row r of the stage, column 32 j + cc) at
      //   j * 32 rb + r * 32 + (((cc / 4) ^ (r % 8)) * 4) + cc % 4   (floats);
      // part sub takes rows r = 32 sub + rr, and the K-major operand stores
      // global column c at
      //   (c / 8) * 256 + (c % 8) * 32 + (((rr / 4) ^ (c % 8)) * 4) + rr % 4,
      // with B's columns after A's 4 mt boxes (for the folded Gram, lo at
      // column c + 64 of the same operand).  A warp takes one 4-column group
      // of a box across its 32 rows (lane = row): conflict-free.
      const float4 *src = reinterpret_cast<const float4 *>(raw(sr)) + sub * TT_KT * 8;
      float *dh = reinterpret_cast<float *>(hi(ss)), *dl = reinterpret_cast<float *>(lo(ss));
#pragma unroll 2
      for (int q = st; q < nbr * 256; q += 256) {
        const int box = q >> 8, k4 = (q >> 5) & 7, r = q & 31;
        const int obox = box < nbA ? box : aboxes + (box - nbA);
        const int c0 = obox * 32 + k4 * 4;
        const float4 v = src[box * (rb * 8) + r * 8 + (k4 ^ (r & 7))];
        const float vals[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + u;
          const int off = (c >> 3) * 256 + (c & 7) * 32 + ((((r >> 2) ^ (c & 7)) & 7) << 2) + (r & 3);
          float h, l;
          tf32_split(vals[u], h, l);
          dh[off] = h;
          if (sym) dh[off + 2048] = l;  // column c + 64 of the same operand
          else dl[off] = l;
        }
      }
      fence_proxy_async();
      __syncwarp();
      const bool last_part = sub == nsub - 1;
      if (lane == 0) {
        mbar_arrive(&split_bar[ss]);
        if (last_part) mbar_arrive(&rawfree_bar[sr]);
      }
      if (++ss == ns) {
        ss = 0;
        phs ^= 1u;
      }
      if (last_part) {
        sub = 0;
        if (++sr == nr) {
          sr = 0;
          phr ^= 1u;
        }
      } else {
        ++sub;
      }
    }
  }
  __syncwarp();  // lanes 1..31 of the producer and issuer warps wait for lane 0
  __syncthreads();
  if (wid >= 8) {
    // ---- partial tile: accumulator t holds rows 128 t .. of C, lane = row ----
    const int ew = wid - 8;
    bool ok = !__any_sync(fullm, failed(vfail)) && S > 0;
    if (ok) {
      const bool w = mbar_wait(&acc_bar, 0);
      if (!__all_sync(fullm, w)) {
        atomicOr(&s_fail, 16);
        ok = false;
      }
    }
    tc_fence_after();
    float *out = partial + (size_t)blockIdx.x * K1p * K2p;
    if (sym) {
      // G = hi^T hi + C + C^T with C = hi^T lo: rows 0..63 (warps 8, 9) put C
      // in shared memory (the stages are idle now), then every entry adds its
      // transpose
      float(*Ct)[65] = reinterpret_cast<float(*)[65]>(base);
      const int i = 32 * ew + lane;
      if (ew < 2) {
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float v[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = 0.f;
          if (ok) tmem_ld16(tmem + (static_cast<uint32_t>(32 * ew) << 16) + static_cast<uint32_t>(64 + c0), v);
#pragma unroll
          for (int k = 0; k < 16; ++k) Ct[i][c0 + k] = v[k];
        }
        asm volatile("bar.sync 1, 64;" ::: "memory");
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float a[16], b[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) a[k] = b[k] = 0.f;
          if (ok) {
            tmem_ld16(tmem + (static_cast<uint32_t>(32 * ew) << 16) + static_cast<uint32_t>(c0), a);
            tmem_ld16(tmem + (static_cast<uint32_t>(32 * ew) << 16) + static_cast<uint32_t>(64 + c0), b);
          }
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (c0 + k < K2p) out[(size_t)i * K2p + c0 + k] = (a[k] + b[k]) + Ct[c0 + k][i];
        }
      }
    }
    for (int t = 0; t < (sym ? 0 : mt); ++t) {
      const int i = t * 128 + 32 * ew + lane;
      for (int c0 = 0; c0 < Np; c0 += 16) {
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        if (ok) tmem_ld16(tmem + (static_cast<uint32_t>(32 * ew) << 16) + static_cast<uint32_t>(t * Np + c0), v);
        if (i < K1p) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (c0 + k < K2p) out[(size_t)i * K2p + c0 + k] = v[k];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  if (tid == 0 && s_fail && err) atomicOr(err, s_fail << 16);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    MC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    MC_REQUIRE(p != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int tc_nsplit(int64_t R) {
  const int64_t by_rows = std::max<int64_t>(1, (R + 4 * TC_KT - 1) / (4 * TC_KT));
  return static_cast<int>(std::min<int64_t>(152, by_rows));
}

}  // namespace

// ---- panel x small factor (tensor cores) --------------------------------------
namespace {
struct NtPlan {
  int Kp, Np, nst, ebuf;
  uint32_t cols;
  size_t smem;
};
// W's hi and lo parts, one or two 16 KiB epilogue staging tiles (two when
// that still leaves two box stages) and as many (hi, lo) box stages as fit
// (two to four); two accumulators of N_p columns in tensor memory
NtPlan nt_plan(int K, int N) {
  NtPlan p{};
  p.Kp = static_cast<int>(round_up(K, NT_KC));
  p.Np = static_cast<int>(round_up(N, 16));
  const size_t wfix = 2 * (size_t)p.Kp * p.Np * 4 + 1024;
  auto stages = [&](int ebuf) {
    const size_t fixed = wfix + (size_t)ebuf * 16 * 1024;
    return fixed < NT_SMEM_LIMIT ? static_cast<int>(std::min<size_t>(NW_MAXST, (NT_SMEM_LIMIT - fixed) /
                                                                                  (2 * NT_BOX_BYTES)))
                                 : 0;
  };
  p.ebuf = stages(2) >= 2 ? 2 : 1;
  p.nst = stages(p.ebuf);
  p.smem = wfix + (size_t)p.ebuf * 16 * 1024 + (size_t)p.nst * 2 * NT_BOX_BYTES;
  p.cols = 32;
  while (p.cols < static_cast<uint32_t>(2 * p.Np)) p.cols <<= 1;
  return p;
}
}  // namespace

// X_hi against [W_hi | W_lo] in one MMA per 8-column step for N <= 128
// (MC_NN_CAT=0: three MMAs per step into one accumulator).
bool use_nn_cat() {
  static const bool on = [] {
    const char *v = std::getenv("MC_NN_CAT");
    return !(v && v[0] == '0');
  }();
  return on;
}

bool gemm_nn_tc_supported(int64_t R, int K, int N, const void *X, int ld_x) {
  if (R < 1 || R >= (int64_t(1) << 31) || K < 1 || N < 1 || N > 256 || ld_x < K || ld_x % 4 != 0) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0) return false;
  const NtPlan p = nt_plan(K, N);
  return (int64_t)p.Kp * p.Np <= NT_MAX_W && p.nst >= 2;
}

void gemm_nn_tc(cudaStream_t st, int64_t R, int K, int N, const float *X, int ld_x, const float *W, int ld_w,
                const float *colscale, float alpha, float beta, float *Z, int ld_z, int *err, const int *copy_if) {
  MC_REQUIRE(gemm_nn_tc_supported(R, K, N, X, ld_x), "gemm_nn_tc: shape or alignment not supported");
  MC_REQUIRE(!copy_if || K == N, "gemm_nn_tc: the copy mode needs K == N");
  const NtPlan p = nt_plan(K, N);
  CUtensorMap map;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(R)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld_x) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(NT_KC), static_cast<cuuint32_t>(NT_BM)};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult cr = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), gdim, gstride, box,
                                  estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) fail(MC_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)cr));
  // Z through bulk tensor stores (beta 0) or adds (beta 1) when a tensor map
  // describes it: 16-byte aligned rows, at least one 32-column box wide
  CUtensorMap zmap;
  std::memset(&zmap, 0, sizeof(zmap));
  int zmode = 0;
  if ((beta == 0.f || beta == 1.f) && N >= 32 && ld_z % 4 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15u) == 0) {
    const cuuint64_t zdim[2] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(R)};
    const cuuint64_t zstride[1] = {static_cast<cuuint64_t>(ld_z) * sizeof(float)};
    const cuuint32_t zbox[2] = {32, 32};
    if (encode_fn()(&zmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Z, zdim, zstride, zbox, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      zmode = beta == 0.f ? 1 : 2;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    MC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t ntiles = (R + NT_BM - 1) / NT_BM;
  const int grid = static_cast<int>(std::min<int64_t>(ntiles, sms));
  smem_attr(gemm_nn_tc_ws_kernel, (int)NT_SMEM_LIMIT);
  const int cat = p.Np <= 128 && use_nn_cat() ? 1 : 0;
  uint32_t cols = p.cols;
  while (cat && cols < static_cast<uint32_t>(4 * p.Np)) cols <<= 1;
  launch_pdl(gemm_nn_tc_ws_kernel, dim3(grid), dim3(NW_THREADS), p.smem, st, map, zmap, zmode, p.ebuf, cat, R, K, N,
             p.Kp, p.Np, cols, p.nst, W, ld_w, colscale, alpha, beta, Z, ld_z, err, copy_if, ld_x, X);
  MC_CHECK_LAUNCH();
}

// ---- X1^T X2 (tensor cores) ----------------------------------------------------
namespace {
constexpr size_t TT_SMEM = 226 * 1024;
struct TtPlan {
  int K1p, K2p, nbA, nbB, Np, mt, nsub, nr, ns, nsplit;
  uint32_t cols;
  size_t smem;
  int64_t rows_per;
};
// Raw stages of 32 nsub rows (the tallest copies that leave two raw and two
// split stages), two raw stages, and up to four split stages.
TtPlan tt_plan(int64_t R, int K1, int K2, bool same) {
  TtPlan p{};
  p.K1p = static_cast<int>(round_up(K1, 32));
  p.K2p = static_cast<int>(round_up(K2, 32));
  p.nbA = p.K1p / 32;
  p.nbB = same ? 0 : p.K2p / 32;
  p.Np = static_cast<int>(round_up(K2, 16));
  p.mt = p.K1p > 128 ? 2 : 1;
  const size_t spl = (size_t)(4 * p.mt + p.nbB) * TT_BOX;
  p.nsub = 0;
  for (int nsub : {4, 2, 1}) {
    const size_t raw = (size_t)(p.nbA + p.nbB) * TT_BOX * nsub;
    for (int ns : {4, 3, 2}) {
      if (2 * raw + (size_t)ns * 2 * spl + 1024 <= TT_SMEM) {
        p.nsub = nsub;
        p.nr = 2;
        p.ns = ns;
        p.smem = 2 * raw + (size_t)ns * 2 * spl + 1024;
        break;
      }
    }
    if (p.nsub) break;
  }
  p.cols = 32;
  while (p.cols < static_cast<uint32_t>(p.mt * p.Np)) p.cols <<= 1;
  p.nsplit = tc_nsplit(R);
  p.rows_per = round_up((R + p.nsplit - 1) / p.nsplit, TT_KT);
  p.nsplit = static_cast<int>((R + p.rows_per - 1) / p.rows_per);
  return p;
}
CUtensorMap tt_map(const float *X, int64_t R, int K, int ld, int rows) {
  CUtensorMap map;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(R)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  const cuuint32_t box[2] = {32, static_cast<cuuint32_t>(rows)};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult cr = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), gdim, gstride, box,
                                  estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) fail(MC_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)cr));
  return map;
}
}  // namespace

// Grams of 33..64 columns with the cross terms folded into one MMA per step
// (MC_TN_SYM=0: three MMAs per step, hi*hi + hi*lo + lo*hi in one accumulator).
bool use_tn_sym() {
  static const bool on = [] {
    const char *v = std::getenv("MC_TN_SYM");
    return !(v && v[0] == '0');
  }();
  return on;
}

bool gemm_tn_tc_supported(int64_t R, int K1, int K2, const void *X1, int ld1, const void *X2, int ld2) {
  if (R < 1 || R >= (int64_t(1) << 31) || K1 < 1 || K2 < 1 || K1 > 256 || K2 > 256) return false;
  if (ld1 < K1 || ld2 < K2 || ld1 % 4 || ld2 % 4) return false;
  if (((reinterpret_cast<uintptr_t>(X1) | reinterpret_cast<uintptr_t>(X2)) & 15u) != 0) return false;
  return tt_plan(R, K1, K2, X1 == X2 && ld1 == ld2 && K1 == K2).nsub > 0;
}

size_t gemm_tn_tc_scratch_floats(int64_t R, int K1, int K2) {
  const TtPlan p = tt_plan(R, K1, K2, false);
  return (size_t)p.nsplit * p.K1p * p.K2p;
}

void gemm_tn_tc(cudaStream_t st, int64_t R, int K1, int K2, const float *X1, int ld1, const float *X2, int ld2,
                float *C, int ld_c, float *partial, int *err, const int *skip) {
  MC_REQUIRE(gemm_tn_tc_supported(R, K1, K2, X1, ld1, X2, ld2), "gemm_tn_tc: shape or alignment not supported");
  const bool same = X1 == X2 && ld1 == ld2 && K1 == K2;
  const TtPlan p = tt_plan(R, K1, K2, same);
  const CUtensorMap amap = tt_map(X1, R, K1, ld1, TT_KT * p.nsub);
  const CUtensorMap bmap = same ? amap : tt_map(X2, R, K2, ld2, TT_KT * p.nsub);
  smem_attr(gemm_tn_tc_ws_kernel, (int)TT_SMEM);
  // the Gram of 33..64 columns in one MMA per step (hi^T [hi | lo])
  const bool sym = same && p.nbA == 2 && p.mt == 1 && use_tn_sym();
  launch_pdl(gemm_tn_tc_ws_kernel, dim3(p.nsplit), dim3(TT_THREADS), p.smem, st, amap, bmap, same ? 1 : 0,
             sym ? 1 : 0, R, p.nbA, p.nbB, p.Np, p.mt, sym ? 128u : p.cols, p.nsub, p.nr, p.ns, p.rows_per, partial,
             p.K1p, p.K2p, err, skip);
  MC_CHECK_LAUNCH();
  gemm_tn_reduce_partials(st, K1, K2, p.nsplit, partial, p.K1p, p.K2p, C, ld_c, skip);
}

size_t gram_tc_scratch_floats(int64_t R, int K) {
  const int Kp = static_cast<int>(round_up(K, 32));
  return (size_t)tc_nsplit(R) * Kp * Kp;
}

bool gram_tc_supported(int K, int ld, const void *X) {
  return K >= 1 && K <= 256 && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

void gram_tc(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *G, int ld_g, float *partial, int *err) {
  MC_REQUIRE(gram_tc_supported(K, ld, X), "gram_tc: K must be <= 256, ld a multiple of 4, X 16-byte aligned");
  MC_REQUIRE(R >= 1 && R < (int64_t(1) << 31), "gram_tc: row count out of range");
  CUtensorMap map;
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(R)};
  const cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  const cuuint32_t box[2] = {32, static_cast<cuuint32_t>(TC_KT)};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult cr = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), gdim, gstride, box,
                                  estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) fail(MC_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)cr));
  const bool two = K > 128;
  const int N0 = two ? 256 : std::max(32, static_cast<int>(round_up(K, 32)));
  const int nbox = two ? 8 : 4;  // the A operand always spans 128 columns
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(N0 + (two ? 128 : 0))) cols <<= 1;
  const int Kp = static_cast<int>(round_up(K, 32));
  const int nsplit = tc_nsplit(R);
  const int64_t rows_per = round_up((R + nsplit - 1) / nsplit, TC_KT);
  const size_t smem = TcSmem::total;
  smem_attr(gram_tc_kernel, (int)smem);
  gram_tc_kernel<<<nsplit, TC_THREADS, smem, st>>>(map, R, K, nbox, two ? 1 : 0, N0, cols, rows_per, partial, Kp, err);
  MC_CHECK_LAUNCH();
  const int64_t total = (int64_t)K * K;
  const int nb = static_cast<int>(std::min<int64_t>((total + 31) / 32, 152 * 8));
  gram_tc_reduce_kernel<<<nb, 256, 0, st>>>(K, nsplit, partial, Kp, G, ld_g);
  MC_CHECK_LAUNCH();
}

}  // namespace mc
