// Sparse kernels of the SVT hot path: CSR ingest checks, the CSC copy, the
// sparse x dense-panel products Y X and Y^T X (Alg. 4/5 steps 2-8), the fused
// evaluation of the shrunk X on Phi with the update of Y (Alg. 6 steps 15-17),
// and deterministic reductions.
//
// Products: every row (a column for the CSC copy) is cut into segments of at
// most SEG entries, one warp per segment.  For panel width K <= 64 a warp
// splits into 32/(K/4) lane groups that walk alternate entries; each lane owns
// a float4 column slice of the panel row it gathers (128-bit loads), so one
// warp instruction gathers 2-4 panel rows.  Group sums are combined by warp
// shuffles in a fixed order and long rows are finished by a fix-up pass that
// adds their segment partials in order: results are deterministic and no
// atomics touch floating-point data.
#include "mc_common.cuh"

#include <algorithm>
#include <vector>

namespace mc {
namespace {

constexpr int kWarpsPerBlock = 8;

// ---------------------------------------------------------------- ingest ----
__global__ void rowptr_check_kernel(int64_t m, int64_t nnz, const int64_t *__restrict__ rp64,
                                    int *__restrict__ rp32, int *__restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = rp64[i];
    if (v < 0 || v > nnz || (i == 0 && v != 0) || (i == m && v != nnz) || (i < m && rp64[i + 1] < v))
      atomicOr(flags, 1);
    rp32[i] = static_cast<int>(v);
  }
}

__global__ void csr_check_kernel(int64_t m, int64_t n, const int *__restrict__ rp, const int *__restrict__ col,
                                 const float *__restrict__ val, int *__restrict__ flags) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int prev = -1;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int c = col[e];
    if (c < 0 || c >= n) atomicOr(flags + 1, 1);
    if (c <= prev) atomicOr(flags + 1, 2);
    prev = c;
    if (!isfinite(val[e])) atomicOr(flags + 2, 1);
  }
}

// Column histogram per row block (CTA b owns rows [r0, r1)).
__global__ void csc_count_kernel(int64_t m, int64_t n, int nblk, const int *__restrict__ rp,
                                 const int *__restrict__ col, int *__restrict__ cnt) {
  const int b = blockIdx.x;
  const int64_t r0 = m * b / nblk, r1 = m * (b + 1) / nblk;
  for (int64_t e = rp[r0] + threadIdx.x; e < rp[r1]; e += blockDim.x) atomicAdd(&cnt[(int64_t)b * n + col[e]], 1);
}

// Per column: exclusive prefix over row blocks (in place) and the total.
__global__ void csc_blockscan_kernel(int64_t n, int nblk, int *__restrict__ cnt, int *__restrict__ total) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int run = 0;
  for (int b = 0; b < nblk; ++b) {
    const int t = cnt[(int64_t)b * n + j];
    cnt[(int64_t)b * n + j] = run;
    run += t;
  }
  total[j] = run;
}

// Exclusive scan of count values into out[0..count] (single block).
__global__ void exclusive_scan_kernel(int64_t count, const int *__restrict__ in, int *__restrict__ out) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < count; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int v = i < count ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < count) out[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[count] = carry;
}

// Scatter rows in ascending order inside each row block: entries of one row
// have distinct columns, rows are visited in order, so the CSC order is
// (column, row) ascending and independent of scheduling.
__global__ void csc_scatter_kernel(int64_t m, int64_t n, int nblk, const int *__restrict__ rp,
                                   const int *__restrict__ col, const int *__restrict__ col_ptr,
                                   int *__restrict__ cursor, int *__restrict__ row_idx, int *__restrict__ perm) {
  const int b = blockIdx.x;
  const int64_t r0 = m * b / nblk, r1 = m * (b + 1) / nblk;
  int *cur = cursor + (int64_t)b * n;
  for (int64_t i = r0; i < r1; ++i) {
    for (int e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const int j = col[e];
      const int pos = col_ptr[j] + cur[j];
      cur[j] += 1;
      row_idx[pos] = static_cast<int>(i);
      perm[pos] = e;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- products ---
template <int G, int CH>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
spmm_seg_kernel(int64_t nseg, const int *__restrict__ seg_row, const int *__restrict__ seg_beg,
                const int *__restrict__ seg_end, const int *__restrict__ seg_slot,
                const int *__restrict__ idx, const float *__restrict__ val, const float *__restrict__ X,
                int ld_x, int K4, float *__restrict__ out, int ld_out, float *__restrict__ partial) {
  constexpr int L = 32 / G;  // lanes per group
  const int lane = threadIdx.x & 31;
  const int64_t seg = blockIdx.x * (int64_t)kWarpsPerBlock + (threadIdx.x >> 5);
  if (seg >= nseg) return;
  const int g = lane / L, li = lane % L;
  const int beg = seg_beg[seg], end = seg_end[seg];
  float4 acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int base = beg; base < end; base += 32) {
    const int e = base + lane;
    const int my_idx = e < end ? idx[e] : 0;
    const float my_val = e < end ? val[e] : 0.f;
    const int cnt = min(32, end - base);
#pragma unroll 4
    for (int t = 0; t < 32; t += G) {
      if (t >= cnt) break;
      const int src = t + g;
      const int j = __shfl_sync(0xffffffffu, my_idx, src);
      const float a = __shfl_sync(0xffffffffu, my_val, src);
      if (src < cnt) {
        const float4 *xr = reinterpret_cast<const float4 *>(X + (int64_t)j * ld_x);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int q = li + c * L;
          if (q < K4) {
            const float4 x = __ldg(xr + q);
            acc[c].x = fmaf(a, x.x, acc[c].x);
            acc[c].y = fmaf(a, x.y, acc[c].y);
            acc[c].z = fmaf(a, x.z, acc[c].z);
            acc[c].w = fmaf(a, x.w, acc[c].w);
          }
        }
      }
    }
  }
#pragma unroll
  for (int off = L; off < 32; off <<= 1) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, off);
      acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, off);
      acc[c].z += __shfl_xor_sync(0xffffffffu, acc[c].z, off);
      acc[c].w += __shfl_xor_sync(0xffffffffu, acc[c].w, off);
    }
  }
  if (g != 0) return;
  const int slot = seg_slot[seg];
  float4 *dst = slot < 0 ? reinterpret_cast<float4 *>(out + (int64_t)seg_row[seg] * ld_out)
                         : reinterpret_cast<float4 *>(partial + (int64_t)slot * (K4 * 4));
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int q = li + c * L;
    if (q < K4) dst[q] = acc[c];
  }
}

__global__ void spmm_fixup_kernel(int64_t nsplit, const int *__restrict__ split_row,
                                  const int *__restrict__ split_slot, const float *__restrict__ partial, int K,
                                  float *__restrict__ out, int ld_out) {
  const int64_t t = blockIdx.x;
  if (t >= nsplit) return;
  const int s0 = split_slot[t], s1 = split_slot[t + 1];
  float *o = out + (int64_t)split_row[t] * ld_out;
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    float acc = 0.f;
    for (int s = s0; s < s1; ++s) acc += partial[(int64_t)s * K + c];
    o[c] = acc;
  }
}

// ------------------------------------------------------------ elementwise ---
__global__ void scale_kernel(int64_t nnz, const float *__restrict__ src, float alpha, float *__restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = alpha * src[e];
}

__global__ void mirror_kernel(int64_t nnz, const int *__restrict__ perm, const float *__restrict__ y,
                              float *__restrict__ yc) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    yc[p] = __ldg(y + perm[p]);
}

// ------------------------------------------------------- fused SVT update ---
// One warp per CSR segment; the row's shrunk left factor Us[i, 0:r] is staged
// in shared memory and read as broadcasts; each lane takes one observed entry
// at a time and gathers V[j, 0:r] with 128-bit loads.  The dot product runs in
// a fixed order, so the same entry always gives the same x.
constexpr int kSddmmMaxR = 1024;
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
sddmm_update_kernel(int64_t nseg, const int *__restrict__ seg_row, const int *__restrict__ seg_beg,
                    const int *__restrict__ seg_end, const int *__restrict__ col, const float *__restrict__ mval,
                    float *__restrict__ y, const float *__restrict__ Us, int ld_us, const float *__restrict__ V,
                    int ld_v, int r, float delta, int update, double *__restrict__ seg_sq,
                    float *__restrict__ x_out) {
  extern __shared__ float4 sh_us4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t seg = blockIdx.x * (int64_t)kWarpsPerBlock + warp;
  const int r4 = (r + 3) >> 2;
  float4 *us = sh_us4 + warp * r4;
  float sq = 0.f;
  if (seg < nseg) {
    const int row = seg_row[seg];
    const float4 *src = reinterpret_cast<const float4 *>(Us + (int64_t)row * ld_us);
    for (int q = lane; q < r4; q += 32) us[q] = src[q];
    __syncwarp();
    const int beg = seg_beg[seg], end = seg_end[seg];
    for (int e = beg + lane; e < end; e += 32) {
      const float4 *vr = reinterpret_cast<const float4 *>(V + (int64_t)col[e] * ld_v);
      float x = 0.f;
      for (int q = 0; q < r4; ++q) {
        const float4 a = us[q];
        const float4 b = __ldg(vr + q);
        x = fmaf(a.x, b.x, x);
        x = fmaf(a.y, b.y, x);
        x = fmaf(a.z, b.z, x);
        x = fmaf(a.w, b.w, x);
      }
      const float res = mval[e] - x;
      sq = fmaf(res, res, sq);
      if (update) y[e] = fmaf(delta, res, y[e]);
      if (x_out) x_out[e] = x;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
  if (lane == 0 && seg < nseg) seg_sq[seg] = static_cast<double>(sq);
}

// ------------------------------------------------------------- reductions ---
__global__ void sum_doubles_kernel(const double *__restrict__ in, int64_t count, double *__restrict__ out) {
  __shared__ double sh[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += in[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < (unsigned)off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void sumsq_partial_kernel(const float *__restrict__ in, int64_t count, double *__restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    acc += v * v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < (unsigned)off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sample_lowrank_kernel(int64_t count, const int64_t *__restrict__ rows,
                                      const int64_t *__restrict__ cols, const float *__restrict__ Us, int ld_us,
                                      const float *__restrict__ V, int ld_v, int r, float *__restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const float *a = Us + rows[t] * ld_us;
    const float *b = V + cols[t] * ld_v;
    float x = 0.f;
    for (int c = 0; c < r; ++c) x = fmaf(a[c], b[c], x);
    out[t] = x;
  }
}

inline int grid_for(int64_t work, int threads, int cap = 152 * 16) {
  const int64_t b = (work + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// ================================================================ launchers ==
void validate_csr(cudaStream_t st, int64_t m, int64_t n, const int *row_ptr, const int *col, const float *val,
                  int *flags) {
  if (m <= 0) return;
  csr_check_kernel<<<grid_for(m, 256, 1 << 20), 256, 0, st>>>(m, n, row_ptr, col, val, flags);
  MC_CHECK_LAUNCH();
}

void convert_rowptr(cudaStream_t st, int64_t m, int64_t nnz, const int64_t *rp64, int *rp32, int *flags) {
  rowptr_check_kernel<<<grid_for(m + 1, 256), 256, 0, st>>>(m, nnz, rp64, rp32, flags);
  MC_CHECK_LAUNCH();
}

void build_csc(cudaStream_t st, int64_t m, int64_t n, int64_t nnz, const int *row_ptr, const int *col,
               int *col_ptr, int *row_idx, int *perm, void *tmp) {
  // tmp layout: total[n] | cnt[nblk * n]
  int nblk = static_cast<int>(std::min<int64_t>(256, std::max<int64_t>(1, (int64_t(1) << 24) / std::max<int64_t>(n, 1))));
  nblk = static_cast<int>(std::min<int64_t>(nblk, std::max<int64_t>(m, 1)));
  int *total = static_cast<int *>(tmp);
  int *cnt = total + round_up(n, 64);
  MC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)nblk * n, st));
  if (nnz > 0) {
    csc_count_kernel<<<nblk, 256, 0, st>>>(m, n, nblk, row_ptr, col, cnt);
    MC_CHECK_LAUNCH();
  }
  csc_blockscan_kernel<<<grid_for(n, 256, 1 << 20), 256, 0, st>>>(n, nblk, cnt, total);
  MC_CHECK_LAUNCH();
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(n, total, col_ptr);
  MC_CHECK_LAUNCH();
  if (nnz > 0) {
    csc_scatter_kernel<<<nblk, 256, 0, st>>>(m, n, nblk, row_ptr, col, col_ptr, cnt, row_idx, perm);
    MC_CHECK_LAUNCH();
  }
}

size_t csc_tmp_bytes(int64_t m, int64_t n) {
  int64_t nblk = std::min<int64_t>(256, std::max<int64_t>(1, (int64_t(1) << 24) / std::max<int64_t>(n, 1)));
  nblk = std::min<int64_t>(nblk, std::max<int64_t>(m, 1));
  return sizeof(int) * (size_t)(round_up(n, 64) + nblk * n);
}

// Host planner: cut rows into segments of <= SEG entries (see SegPlan).
void plan_segments(cudaStream_t st, Alloc &a, int64_t rows, const int *ptr, SegPlan &plan) {
  std::vector<int> hp(rows + 1);
  MC_CUDA(cudaMemcpyAsync(hp.data(), ptr, sizeof(int) * (rows + 1), cudaMemcpyDeviceToHost, st));
  MC_CUDA(cudaStreamSynchronize(st));
  std::vector<int> srow, sbeg, send, sslot, sprow, spslot;
  srow.reserve(rows + hp[rows] / SEG + 1);
  int slot = 0;
  for (int64_t i = 0; i < rows; ++i) {
    const int b = hp[i], e = hp[i + 1];
    const int len = e - b;
    const int ns = len <= SEG ? 1 : (len + SEG - 1) / SEG;
    if (ns == 1) {
      srow.push_back(static_cast<int>(i));
      sbeg.push_back(b);
      send.push_back(e);
      sslot.push_back(-1);
    } else {
      sprow.push_back(static_cast<int>(i));
      spslot.push_back(slot);
      for (int s = 0; s < ns; ++s) {
        srow.push_back(static_cast<int>(i));
        sbeg.push_back(b + s * SEG);
        send.push_back(std::min(e, b + (s + 1) * SEG));
        sslot.push_back(slot++);
      }
    }
  }
  spslot.push_back(slot);
  plan.nseg = static_cast<int64_t>(srow.size());
  plan.nsplit = static_cast<int64_t>(sprow.size());
  plan.nslot = slot;
  auto up = [&](DBuf &d, const std::vector<int> &v) {
    d.reserve(a, sizeof(int) * std::max<size_t>(1, v.size()));
    if (!v.empty()) MC_CUDA(cudaMemcpyAsync(d.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, st));
  };
  up(plan.seg_row, srow);
  up(plan.seg_beg, sbeg);
  up(plan.seg_end, send);
  up(plan.seg_slot, sslot);
  up(plan.split_row, sprow);
  up(plan.split_slot, spslot);
  MC_CUDA(cudaStreamSynchronize(st));
}

void spmm(cudaStream_t st, const SegPlan &plan, const int *idx, const float *val, const float *X, int ld_x, int K,
          float *out, int ld_out, float *partial) {
  if (plan.nseg == 0 || K <= 0) return;
  MC_REQUIRE(K % 4 == 0 && ld_x % 4 == 0 && ld_out % 4 == 0, "spmm: K and leading dims must be multiples of 4");
  const int K4 = K / 4;
  const int64_t blocks = (plan.nseg + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int threads = kWarpsPerBlock * 32;
#define MC_SPMM_ARGS                                                                                          \
  plan.nseg, plan.seg_row.as<int>(), plan.seg_beg.as<int>(), plan.seg_end.as<int>(), plan.seg_slot.as<int>(), \
      idx, val, X, ld_x, K4, out, ld_out, partial
  if (K4 <= 2) spmm_seg_kernel<16, 1><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 4) spmm_seg_kernel<8, 1><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 8) spmm_seg_kernel<4, 1><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 16) spmm_seg_kernel<2, 1><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 32) spmm_seg_kernel<1, 1><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 64) spmm_seg_kernel<1, 2><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 128) spmm_seg_kernel<1, 4><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else if (K4 <= 256) spmm_seg_kernel<1, 8><<<blocks, threads, 0, st>>>(MC_SPMM_ARGS);
  else MC_REQUIRE(false, "spmm: panel width above 1024");
#undef MC_SPMM_ARGS
  MC_CHECK_LAUNCH();
  if (plan.nsplit > 0) {
    spmm_fixup_kernel<<<static_cast<unsigned>(plan.nsplit), 128, 0, st>>>(
        plan.nsplit, plan.split_row.as<int>(), plan.split_slot.as<int>(), partial, K, out, ld_out);
    MC_CHECK_LAUNCH();
  }
}

void scale_values(cudaStream_t st, int64_t nnz, const float *src, float alpha, float *dst) {
  if (nnz <= 0) return;
  scale_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, src, alpha, dst);
  MC_CHECK_LAUNCH();
}

void mirror_values(cudaStream_t st, int64_t nnz, const int *perm, const float *y, float *yc) {
  if (nnz <= 0) return;
  mirror_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, perm, y, yc);
  MC_CHECK_LAUNCH();
}

void sddmm_update(cudaStream_t st, const SegPlan &plan, const int *col, const float *mval, float *y, const float *Us,
                  int ld_us, const float *V, int ld_v, int r, float delta, int update, double *seg_sq, float *x_out) {
  if (plan.nseg == 0) return;
  MC_REQUIRE(r >= 0 && r <= kSddmmMaxR, "sddmm: rank above 1024");
  MC_REQUIRE(ld_us % 4 == 0 && ld_v % 4 == 0, "sddmm: leading dims must be multiples of 4");
  const int r4 = (r + 3) / 4;
  const size_t smem = sizeof(float4) * (size_t)kWarpsPerBlock * std::max(r4, 1);
  const int64_t blocks = (plan.nseg + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (smem > 48 * 1024)
    MC_CUDA(cudaFuncSetAttribute(sddmm_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sddmm_update_kernel<<<blocks, kWarpsPerBlock * 32, smem, st>>>(
      plan.nseg, plan.seg_row.as<int>(), plan.seg_beg.as<int>(), plan.seg_end.as<int>(), col, mval, y, Us, ld_us, V,
      ld_v, r, delta, update, seg_sq, x_out);
  MC_CHECK_LAUNCH();
}

void sum_doubles(cudaStream_t st, const double *in, int64_t count, double *out) {
  sum_doubles_kernel<<<1, 1024, 0, st>>>(in, count, out);
  MC_CHECK_LAUNCH();
}

void sumsq_floats(cudaStream_t st, const float *in, int64_t count, double *scratch, double *out) {
  const int nb = grid_for(count, 256, 1024);
  sumsq_partial_kernel<<<nb, 256, 0, st>>>(in, count, scratch);
  MC_CHECK_LAUNCH();
  sum_doubles(st, scratch, nb, out);
}

void sample_lowrank(cudaStream_t st, int64_t count, const int64_t *rows, const int64_t *cols, const float *Us,
                    int ld_us, const float *V, int ld_v, int r, float *out) {
  if (count <= 0) return;
  sample_lowrank_kernel<<<grid_for(count, 256), 256, 0, st>>>(count, rows, cols, Us, ld_us, V, ld_v, r, out);
  MC_CHECK_LAUNCH();
}

}  // namespace mc
