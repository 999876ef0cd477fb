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

#include <vector>

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

namespace mc {
namespace {

constexpr int kWarpsPerBlock = 4;  // bf16 products: 128-thread CTAs (the faster shape measured)

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

// A warp per row, lanes along the row: every entry is compared with its
// left neighbour in the row (long Zipf rows no longer run on one thread).
__global__ void csr_check_kernel(int64_t m, int64_t n, const int *__restrict__ rp, const int *__restrict__ col,
                                 const float *__restrict__ val, int *__restrict__ flags) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  const int b = rp[w], e1 = rp[w + 1];
  int bad = 0, nonfin = 0;
  for (int e = b + lane; e < e1; e += 32) {
    const int c = col[e];
    if (c < 0 || c >= n) bad |= 1;
    if (e > b && c <= col[e - 1]) bad |= 2;
    if (!isfinite(val[e])) nonfin = 1;
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  nonfin = __reduce_or_sync(0xffffffffu, nonfin);
  if (lane == 0) {
    if (bad) atomicOr(flags + 1, bad);
    if (nonfin) atomicOr(flags + 2, 1);
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

// ------------------------------------------------------------- COO ingest ---
// Entries in any order: key = row * n + col (checked), a stable LSD radix
// sort of (key, original index) with 8-bit digits, then the CSR arrays.
constexpr int RS_THREADS = 256, RS_TILE = 4096;

__global__ void coo_keys_kernel(int64_t nnz, int64_t m, int64_t n, const int64_t *__restrict__ rows,
                                const int *__restrict__ cols, const float *__restrict__ vals,
                                unsigned long long *__restrict__ keys, int *__restrict__ idx, int *__restrict__ flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rows[e];
    const int c = cols[e];
    if (r < 0 || r >= m || c < 0 || c >= n) {
      atomicOr(flags + 1, 1);
      keys[e] = 0ull;
    } else {
      keys[e] = (unsigned long long)r * (unsigned long long)n + (unsigned long long)c;
    }
    if (!isfinite(vals[e])) atomicOr(flags + 2, 1);
    idx[e] = static_cast<int>(e);
  }
}

// digit counts per tile: hist[d * ntile + tile]
__global__ void __launch_bounds__(RS_THREADS)
radix_hist_kernel(int64_t nnz, const unsigned long long *__restrict__ keys, int shift, int *__restrict__ hist) {
  __shared__ int cnt[256];
  const int ntile = gridDim.x;
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * RS_TILE, b1 = min(nnz, b0 + RS_TILE);
  for (int64_t e = b0 + threadIdx.x; e < b1; e += RS_THREADS) atomicAdd(&cnt[(keys[e] >> shift) & 255ull], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntile + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter in order: within a tile, chunks of 256 entries; a warp ranks equal
// digits with a match mask, warps add the counts of the warps before them,
// and a running base per digit carries over from chunk to chunk (stable).
__global__ void __launch_bounds__(RS_THREADS)
radix_scatter_kernel(int64_t nnz, const unsigned long long *__restrict__ kin, const int *__restrict__ vin, int shift,
                     const int *__restrict__ offs, unsigned long long *__restrict__ kout, int *__restrict__ vout) {
  constexpr int NWP = RS_THREADS / 32;
  __shared__ int base[256];
  __shared__ int wc[NWP][256];
  const int ntile = gridDim.x, tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  base[tid] = offs[(int64_t)tid * ntile + blockIdx.x];
  const int64_t b0 = (int64_t)blockIdx.x * RS_TILE, b1 = min(nnz, b0 + RS_TILE);
  for (int64_t c0 = b0; c0 < b1; c0 += RS_THREADS) {
    for (int q = tid; q < NWP * 256; q += RS_THREADS) (&wc[0][0])[q] = 0;
    __syncthreads();
    const int64_t e = c0 + tid;
    const bool act = e < b1;
    unsigned long long key = act ? kin[e] : 0ull;
    const int dg = static_cast<int>((key >> shift) & 255ull);
    const unsigned amask = __ballot_sync(0xffffffffu, act);
    int wrank = 0;
    if (act) {
      const unsigned peers = __match_any_sync(amask, dg);
      wrank = __popc(peers & ((1u << lane) - 1u));
      if (wrank == 0) wc[wid][dg] = __popc(peers);
    }
    __syncthreads();
    if (act) {
      int pos = base[dg] + wrank;
      for (int w = 0; w < wid; ++w) pos += wc[w][dg];
      kout[pos] = key;
      vout[pos] = vin[e];
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < NWP; ++w) tot += wc[w][tid];
    base[tid] += tot;
    __syncthreads();
  }
}

// Exclusive scan of a long int array by one block, chunk after chunk.
__global__ void scan_long_kernel(int64_t count, const int *__restrict__ in, int *__restrict__ out) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < count; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
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
}

// CSR from the sorted keys: columns, values (gathered by original index),
// duplicates flagged, row counts for the row pointer.
__global__ void coo_csr_kernel(int64_t nnz, int64_t n, const unsigned long long *__restrict__ keys,
                               const int *__restrict__ idx, const float *__restrict__ vals, int *__restrict__ col,
                               float *__restrict__ val, int *__restrict__ rowcnt, int *__restrict__ flags) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[e];
    if (e > 0 && keys[e - 1] == k) atomicOr(flags + 1, 2);
    const int64_t r = static_cast<int64_t>(k / (unsigned long long)n);
    col[e] = static_cast<int>(k - (unsigned long long)r * (unsigned long long)n);
    val[e] = vals[idx[e]];
    atomicAdd(rowcnt + r, 1);
  }
}

__global__ void widen_rowptr_kernel(int64_t m, const int *__restrict__ rp32, int64_t *__restrict__ rp64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x)
    rp64[i] = rp32[i];
}

// --------------------------------------------------------------- products ---
// G lane groups per warp (a group owns one gathered panel row at a time), U
// gathers in flight per group.  Group g takes the segment's entries g, g + G,
// g + 2G, ... in that order whatever U and the block size are, so those two
// launch parameters (tuned at run time) never change the result's bits.
template <int G, int U>
__global__ void __launch_bounds__(256)
spmm_seg_kernel(int64_t nseg, const int4 *__restrict__ segs, const int *__restrict__ idx,
                const float *__restrict__ val, const float *__restrict__ X, int ld_x, int K4,
                float *__restrict__ out, int ld_out, float *__restrict__ partial) {
  pdl_wait();
  pdl_trigger();
  constexpr int L = 32 / G;  // lanes per group
  const int lane = threadIdx.x & 31;
  const int64_t seg = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (seg >= nseg) return;
  const int g = lane / L, li = lane % L;
  const int4 sd = segs[seg];  // (row, begin, end, partial slot or -1)
  const bool active = li < K4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int base = sd.y; base < sd.z; base += 32) {
    const int e = base + lane;
    // indices and values are streamed once: evict-first, so the L1 keeps
    // the gathered panel rows (popular columns are reused across rows)
    const int my_idx = e < sd.z ? __ldcs(idx + e) : 0;
    const float my_val = e < sd.z ? __ldcs(val + e) : 0.f;
    const int cnt = min(32, sd.z - base);
#pragma unroll
    for (int t0 = 0; t0 < 32; t0 += G * U) {
      if (t0 >= cnt) break;  // warp-uniform
      float4 xv[U];
      float av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int src = t0 + u * G + g;
        const int j = __shfl_sync(0xffffffffu, my_idx, src);
        av[u] = __shfl_sync(0xffffffffu, my_val, src);
        xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active && src < cnt) xv[u] = __ldg(reinterpret_cast<const float4 *>(X + (int64_t)j * ld_x) + li);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        acc.x = fmaf(av[u], xv[u].x, acc.x);
        acc.y = fmaf(av[u], xv[u].y, acc.y);
        acc.z = fmaf(av[u], xv[u].z, acc.z);
        acc.w = fmaf(av[u], xv[u].w, acc.w);
      }
    }
  }
#pragma unroll
  for (int off = L; off < 32; off <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off);
  }
  if (g != 0 || !active) return;
  float4 *dst = sd.w < 0 ? reinterpret_cast<float4 *>(out + (int64_t)sd.x * ld_out)
                         : reinterpret_cast<float4 *>(partial + (int64_t)sd.w * (K4 * 4));
  dst[li] = acc;
}

// Same work split with a BF16 panel (mixed-precision form): a lane owns 8
// consecutive columns (one 16-byte load of 8 bf16) and accumulates in float32.
template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
spmm_seg_bf16_kernel(int64_t nseg, const int4 *__restrict__ segs, const int *__restrict__ idx,
                     const float *__restrict__ val, const __nv_bfloat16 *__restrict__ X, int ld_x, int K8,
                     float *__restrict__ out, int ld_out, float *__restrict__ partial) {
  constexpr int L = 32 / G;
  constexpr int U = 1;  // one gather in flight per group (the faster choice measured)
  const int lane = threadIdx.x & 31;
  const int64_t seg = blockIdx.x * (int64_t)kWarpsPerBlock + (threadIdx.x >> 5);
  if (seg >= nseg) return;
  const int g = lane / L, li = lane % L;
  const int4 sd = segs[seg];
  const bool active = li < K8;
  float acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.f;
  for (int base = sd.y; base < sd.z; base += 32) {
    const int e = base + lane;
    const int my_idx = e < sd.z ? __ldcs(idx + e) : 0;
    const float my_val = e < sd.z ? __ldcs(val + e) : 0.f;
    const int cnt = min(32, sd.z - base);
#pragma unroll
    for (int t0 = 0; t0 < 32; t0 += G * U) {
      if (t0 >= cnt) break;  // warp-uniform
      uint4 xv[U];
      float av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int src = t0 + u * G + g;
        const int j = __shfl_sync(0xffffffffu, my_idx, src);
        av[u] = __shfl_sync(0xffffffffu, my_val, src);
        xv[u] = make_uint4(0u, 0u, 0u, 0u);
        if (active && src < cnt) xv[u] = __ldg(reinterpret_cast<const uint4 *>(X + (int64_t)j * ld_x) + li);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t w[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float lo = __uint_as_float(w[q] << 16), hi = __uint_as_float(w[q] & 0xFFFF0000u);
          acc[2 * q] = fmaf(av[u], lo, acc[2 * q]);
          acc[2 * q + 1] = fmaf(av[u], hi, acc[2 * q + 1]);
        }
      }
    }
  }
#pragma unroll
  for (int off = L; off < 32; off <<= 1)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
  if (g != 0 || !active) return;
  float *dst = sd.w < 0 ? out + (int64_t)sd.x * ld_out : partial + (int64_t)sd.w * (K8 * 8);
  float4 *d4 = reinterpret_cast<float4 *>(dst + li * 8);
  d4[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
  d4[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// Round a float32 panel to bf16 (nearest even); columns cols..ld_out-1 zero.
__global__ void to_bf16_kernel(int64_t rows, int cols, const float *__restrict__ in, int ld_in,
                               __nv_bfloat16 *__restrict__ out, int ld_out) {
  const int64_t total = rows * ld_out;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ld_out;
    const int c = static_cast<int>(t - r * ld_out);
    out[t] = __float2bfloat16_rn(c < cols ? in[r * ld_in + c] : 0.f);
  }
}

// A warp per (split row, group of 4 columns): lane l adds the row's segment
// partials l, l + 32, ... (four loads in flight), and the 32 lane sums meet
// in a fixed shuffle tree.  The order is the same for every launch shape; a
// column with hundreds of segments (the popular columns of rating data)
// takes a few load latencies instead of one per segment.
__global__ void spmm_fixup_kernel(int64_t nsplit, const int *__restrict__ split_row,
                                  const int *__restrict__ split_slot, const float *__restrict__ partial, int K,
                                  float *__restrict__ out, int ld_out) {
  pdl_wait();
  pdl_trigger();
  const int K4 = K / 4;
  const int lane = threadIdx.x & 31;
  const int64_t nw = nsplit * K4;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nw; w += wstride) {
    const int64_t i = w / K4;
    const int c4 = static_cast<int>(w - i * K4);
    const int s0 = split_slot[i], s1 = split_slot[i + 1];
    const float *src = partial + 4 * c4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = s0 + lane; b < s1; b += 4 * 32) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sg = b + 32 * u;
        v[u] = sg < s1 ? *reinterpret_cast<const float4 *>(src + (int64_t)sg * K) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.x += v[u].x;
        acc.y += v[u].y;
        acc.z += v[u].z;
        acc.w += v[u].w;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, off);
    }
    if (lane == 0) *reinterpret_cast<float4 *>(out + (int64_t)split_row[i] * ld_out + 4 * c4) = acc;
  }
}

// The same sums with a warp per split row and chunk of KM4 column groups
// (one chunk for panels of at most 4 KM4 columns): each lane loads a chunk
// of a segment's partial row (KM4 consecutive float4) in one pass over the
// row's segments, so the launch has fewer warps than column groups, each
// with the same few load latencies, and a segment's row is read in whole
// sectors.  Per column the order is that of spmm_fixup_kernel: the same bits.
template <int KM4>
__global__ void spmm_fixup_rows_kernel(int64_t nsplit, const int *__restrict__ split_row,
                                       const int *__restrict__ split_slot, const float *__restrict__ partial, int K,
                                       float *__restrict__ out, int ld_out, int nchunk) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wi < nsplit * nchunk; wi += wstride) {
    const int64_t i = wi / nchunk;
    const int cb = static_cast<int>(wi - i * nchunk) * KM4;  // first column group of the chunk
    const int K4 = K / 4 - cb;                               // column groups from cb on
    const float *part_c = partial + 4 * cb;
    const int s0 = split_slot[i], s1 = split_slot[i + 1];
    float4 acc[KM4];
#pragma unroll
    for (int c = 0; c < KM4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = s0 + lane; b < s1; b += 4 * 32) {
      float4 v[4][KM4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sg = b + 32 * u;
#pragma unroll
        for (int c = 0; c < KM4; ++c)
          v[u][c] = (sg < s1 && c < K4) ? *reinterpret_cast<const float4 *>(part_c + (int64_t)sg * K + 4 * c)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < KM4; ++c) {
          acc[c].x += v[u][c].x;
          acc[c].y += v[u][c].y;
          acc[c].z += v[u][c].z;
          acc[c].w += v[u][c].w;
        }
    }
#pragma unroll
    for (int c = 0; c < KM4; ++c) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, off);
        acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, off);
        acc[c].z += __shfl_xor_sync(0xffffffffu, acc[c].z, off);
        acc[c].w += __shfl_xor_sync(0xffffffffu, acc[c].w, off);
      }
    }
    if (lane == 0) {
      float4 *dst = reinterpret_cast<float4 *>(out + (int64_t)split_row[i] * ld_out + 4 * cb);
#pragma unroll
      for (int c = 0; c < KM4; ++c)
        if (c < K4) dst[c] = acc[c];
    }
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
// One thread per observed entry (grid-stride over a fixed grid, so every
// thread always sees the same entries): x_e = <Us[i,:], V[j,:]> with 128-bit
// loads (entries of one row are adjacent, so a warp's Us loads mostly hit
// one row), res = M_e - x_e, y_e += delta res, and sum res^2 per block in a
// fixed order.  The dot product order is fixed, so the same entry always
// gives the same x.
constexpr int kSddmmThreads = 256;
constexpr int kSddmmBlocks = 152 * 8;
__global__ void __launch_bounds__(kSddmmThreads)
sddmm_update_kernel(int64_t nnz, const int *__restrict__ rix, const int *__restrict__ col,
                    const float *__restrict__ mval, float *__restrict__ y, const float *__restrict__ Us, int ld_us,
                    const float *__restrict__ V, int ld_v, int r4, float delta, int update,
                    double *__restrict__ block_sq, float *__restrict__ x_out) {
  pdl_wait();
  pdl_trigger();
  __shared__ float wsum[kSddmmThreads / 32];
  float sq = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)kSddmmThreads + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * kSddmmThreads) {
    const float4 *a = reinterpret_cast<const float4 *>(Us + (int64_t)rix[e] * ld_us);
    const float4 *b = reinterpret_cast<const float4 *>(V + (int64_t)col[e] * ld_v);
    float x = 0.f;
    for (int q = 0; q < r4; ++q) {
      const float4 u = __ldg(a + q);
      const float4 v = __ldg(b + q);
      x = fmaf(u.x, v.x, x);
      x = fmaf(u.y, v.y, x);
      x = fmaf(u.z, v.z, x);
      x = fmaf(u.w, v.w, x);
    }
    const float res = mval[e] - x;
    sq = fmaf(res, res, sq);
    if (update) y[e] = fmaf(delta, res, y[e]);
    if (x_out) x_out[e] = x;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSddmmThreads / 32; ++w) t += wsum[w];
    block_sq[blockIdx.x] = t;
  }
}

// Row index of every CSR entry (the fused update walks entries, not rows).
__global__ void expand_rows_kernel(int64_t m, const int *__restrict__ rp, int *__restrict__ rix) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m) return;
  for (int e = rp[w] + lane; e < rp[w + 1]; e += 32) rix[e] = static_cast<int>(w);
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
  csr_check_kernel<<<static_cast<unsigned>((m * 32 + 255) / 256), 256, 0, st>>>(m, n, row_ptr, col, val, flags);
  MC_CHECK_LAUNCH();
}

void coo_to_csr(cudaStream_t st, Alloc &a, int64_t m, int64_t n, int64_t nnz, const int64_t *rows, const int *cols,
                const float *vals, int64_t *row_ptr, int *col, float *val, int *flags) {
  if (nnz <= 0) {
    MC_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t) * (m + 1), st));
    return;
  }
  const int64_t ntile = (nnz + RS_TILE - 1) / RS_TILE;
  DBuf k0, k1, v0, v1, hist, offs, cnt, rp32;
  BufGuard guard(a, {&k0, &k1, &v0, &v1, &hist, &offs, &cnt, &rp32});
  k0.reserve(a, sizeof(unsigned long long) * nnz);
  k1.reserve(a, sizeof(unsigned long long) * nnz);
  v0.reserve(a, sizeof(int) * nnz);
  v1.reserve(a, sizeof(int) * nnz);
  hist.reserve(a, sizeof(int) * 256 * ntile);
  offs.reserve(a, sizeof(int) * (256 * ntile + 1));
  coo_keys_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, m, n, rows, cols, vals, k0.as<unsigned long long>(),
                                                      v0.as<int>(), flags);
  MC_CHECK_LAUNCH();
  const unsigned long long maxkey = (unsigned long long)m * (unsigned long long)n - 1ull;
  int bits = 0;
  while (bits < 64 && (maxkey >> bits) != 0ull) ++bits;
  unsigned long long *kin = k0.as<unsigned long long>(), *kout = k1.as<unsigned long long>();
  int *vin = v0.as<int>(), *vout = v1.as<int>();
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<(unsigned)ntile, RS_THREADS, 0, st>>>(nnz, kin, shift, hist.as<int>());
    MC_CHECK_LAUNCH();
    scan_long_kernel<<<1, 1024, 0, st>>>(256 * ntile, hist.as<int>(), offs.as<int>());
    MC_CHECK_LAUNCH();
    radix_scatter_kernel<<<(unsigned)ntile, RS_THREADS, 0, st>>>(nnz, kin, vin, shift, offs.as<int>(), kout, vout);
    MC_CHECK_LAUNCH();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  cnt.reserve(a, sizeof(int) * (m + 1));
  rp32.reserve(a, sizeof(int) * (m + 1));
  MC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (m + 1), st));
  coo_csr_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, n, kin, vin, vals, col, val, cnt.as<int>(), flags);
  MC_CHECK_LAUNCH();
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(m, cnt.as<int>(), rp32.as<int>());
  MC_CHECK_LAUNCH();
  widen_rowptr_kernel<<<grid_for(m + 1, 256), 256, 0, st>>>(m, rp32.as<int>(), row_ptr);
  MC_CHECK_LAUNCH();
  MC_CUDA(cudaStreamSynchronize(st));
  for (DBuf *b : {&k0, &k1, &v0, &v1, &hist, &offs, &cnt, &rp32}) b->release(a);
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
  std::vector<int4> packed;
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
  packed.resize(srow.size());
  for (size_t t = 0; t < srow.size(); ++t) packed[t] = make_int4(srow[t], sbeg[t], send[t], sslot[t]);
  plan.seg.reserve(a, sizeof(int4) * std::max<size_t>(1, packed.size()));
  if (!packed.empty())
    MC_CUDA(cudaMemcpyAsync(plan.seg.p, packed.data(), sizeof(int4) * packed.size(), cudaMemcpyHostToDevice, st));
  up(plan.split_row, sprow);
  up(plan.split_slot, spslot);
  MC_CUDA(cudaStreamSynchronize(st));
}

int default_chunk(int64_t rows_in) {
  // column chunks of at most 128, narrower when the panel slice would not stay
  // resident in L2 next to the streamed indices (each chunk re-reads them)
  int chunk = 128;
  while (chunk > 32 && (double)rows_in * chunk * 4.0 > 40e6) chunk /= 2;
  return chunk;
}

namespace {
int lane_groups(int K4) { return K4 <= 2 ? 16 : (K4 <= 4 ? 8 : (K4 <= 8 ? 4 : (K4 <= 16 ? 2 : 1))); }

template <int G>
void launch_seg(int u, int64_t blocks, int threads, cudaStream_t st, int64_t nseg, const int4 *segs, const int *idx,
                const float *val, const float *X, int ld_x, int K4, float *out, int ld_out, float *partial) {
#define MC_SPMM_ARGS nseg, segs, idx, val, X, ld_x, K4, out, ld_out, partial
  if (u >= 4 && G * 4 <= 32) launch_pdl(spmm_seg_kernel<G, (G * 4 <= 32 ? 4 : 1)>, dim3(blocks), dim3(threads), 0, st, MC_SPMM_ARGS);
  else if (u >= 2 && G * 2 <= 32) launch_pdl(spmm_seg_kernel<G, (G * 2 <= 32 ? 2 : 1)>, dim3(blocks), dim3(threads), 0, st, MC_SPMM_ARGS);
  else launch_pdl(spmm_seg_kernel<G, 1>, dim3(blocks), dim3(threads), 0, st, MC_SPMM_ARGS);
#undef MC_SPMM_ARGS
}
}  // namespace

// Split-row sums by chunks of 8 column groups for K > 16 (MC_FIXUP_ROWS=0:
// a warp per column group).
static bool use_fixup_rows() {
  static const bool on = [] {
    const char *v = std::getenv("MC_FIXUP_ROWS");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Adds the partials of rows longer than one segment (K columns, a multiple of 4).
static void launch_fixup(cudaStream_t st, const SegPlan &plan, const float *partial, int K, float *out, int ld_out) {
  const int K4 = K / 4;
  const int *sr = plan.split_row.as<int>(), *ss = plan.split_slot.as<int>();
  if (K4 <= 4) {
    launch_pdl(spmm_fixup_rows_kernel<4>, dim3(grid_for(plan.nsplit * 32, 256, 1 << 20)), dim3(256), 0, st,
               plan.nsplit, sr, ss, partial, K, out, ld_out, 1);
  } else if (K4 <= 64 && use_fixup_rows()) {
    const int nchunk = (K4 + 7) / 8;
    launch_pdl(spmm_fixup_rows_kernel<8>, dim3(grid_for(plan.nsplit * nchunk * 32, 256, 1 << 20)), dim3(256), 0, st,
               plan.nsplit, sr, ss, partial, K, out, ld_out, nchunk);
  } else {
    launch_pdl(spmm_fixup_kernel, dim3(grid_for(plan.nsplit * K4 * 32, 256)), dim3(256), 0, st, plan.nsplit, sr, ss,
               partial, K, out, ld_out);
  }
  MC_CHECK_LAUNCH();
}

// Lane groups of a product: from the widest chunk the default chunking uses,
// so that every chunking the tuner tries fits the same groups.
int spmm_groups(int K, int64_t rows_in) { return lane_groups(std::min(K, default_chunk(rows_in)) / 4); }

std::vector<SpmmCfg> spmm_candidates(int K, int64_t rows_in) {
  const int G = spmm_groups(K, rows_in);
  const int dc = default_chunk(rows_in);
  std::vector<SpmmCfg> c;
  for (int u : {1, 2, 4}) {
    if (G * u > 32) continue;
    for (int threads : {128, 256}) c.push_back({u, threads, dc});
  }
  if (K > 32) c.push_back({1, 128, dc / 2});  // narrower chunks only: wider ones would need other groups
  return c;
}

void spmm(cudaStream_t st, const SegPlan &plan, const int *idx, const float *val, int64_t rows_in, const float *X,
          int ld_x, int K, float *out, int ld_out, float *partial, const SpmmCfg &cfg) {
  if (plan.nseg == 0 || K <= 0) return;
  MC_REQUIRE(K % 4 == 0 && ld_x % 4 == 0 && ld_out % 4 == 0, "spmm: K and leading dims must be multiples of 4");
  MC_REQUIRE(K <= 1024, "spmm: panel width above 1024");
  const int dc = default_chunk(rows_in);
  const int chunk = cfg.chunk > 0 ? std::min(dc, std::max(4, cfg.chunk / 4 * 4)) : dc;
  const int threads = cfg.threads == 256 ? 256 : 128;
  const int64_t wpb = threads / 32;
  const int64_t blocks = (plan.nseg + wpb - 1) / wpb;
  // the lane-group count follows the panel width and the default chunk, not
  // the chunk in use, so every chunking sums each column's entries in the
  // same order
  const int G = spmm_groups(K, rows_in);
  const int u = cfg.u > 0 ? cfg.u : 1;
  for (int c0 = 0; c0 < K; c0 += chunk) {
    const int kc = std::min(chunk, K - c0);
    const int K4 = kc / 4;
    MC_REQUIRE(K4 <= 32 / G, "spmm: chunk wider than the lane groups");
#define MC_SEG_ARGS u, blocks, threads, st, plan.nseg, plan.seg.as<int4>(), idx, val, X + c0, ld_x, K4, out + c0, ld_out, partial
    if (G == 16) launch_seg<16>(MC_SEG_ARGS);
    else if (G == 8) launch_seg<8>(MC_SEG_ARGS);
    else if (G == 4) launch_seg<4>(MC_SEG_ARGS);
    else if (G == 2) launch_seg<2>(MC_SEG_ARGS);
    else launch_seg<1>(MC_SEG_ARGS);
#undef MC_SEG_ARGS
    MC_CHECK_LAUNCH();
    if (plan.nsplit > 0) {
      launch_fixup(st, plan, partial, kc, out + c0, ld_out);
    }
  }
}

void spmm_bf16(cudaStream_t st, const SegPlan &plan, const int *idx, const float *val, const void *Xbf, int ld_x,
               int K, float *out, int ld_out, float *partial) {
  if (plan.nseg == 0 || K <= 0) return;
  MC_REQUIRE(K % 8 == 0 && ld_x % 8 == 0 && ld_out % 4 == 0 && K <= 256, "spmm_bf16: K and ld must be multiples of 8, K <= 256");
  const __nv_bfloat16 *X = static_cast<const __nv_bfloat16 *>(Xbf);
  const int K8 = K / 8;
  const int64_t blocks = (plan.nseg + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int threads = kWarpsPerBlock * 32;
#define MC_BF_ARGS plan.nseg, plan.seg.as<int4>(), idx, val, X, ld_x, K8, out, ld_out, partial
  if (K8 <= 1) spmm_seg_bf16_kernel<32><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
  else if (K8 <= 2) spmm_seg_bf16_kernel<16><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
  else if (K8 <= 4) spmm_seg_bf16_kernel<8><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
  else if (K8 <= 8) spmm_seg_bf16_kernel<4><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
  else if (K8 <= 16) spmm_seg_bf16_kernel<2><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
  else spmm_seg_bf16_kernel<1><<<blocks, threads, 0, st>>>(MC_BF_ARGS);
#undef MC_BF_ARGS
  MC_CHECK_LAUNCH();
  if (plan.nsplit > 0) {
    launch_fixup(st, plan, partial, K, out, ld_out);
  }
}

void to_bf16(cudaStream_t st, int64_t rows, int cols, const float *in, int ld_in, void *out, int ld_out) {
  const int64_t total = rows * ld_out;
  if (total <= 0) return;
  to_bf16_kernel<<<grid_for(total, 256), 256, 0, st>>>(rows, cols, in, ld_in, static_cast<__nv_bfloat16 *>(out),
                                                       ld_out);
  MC_CHECK_LAUNCH();
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

// ---- gather probe ------------------------------------------------------------
// The SpMM's panel-row gathers alone: a warp walks a contiguous chunk of an
// index stream (the CSR column or CSC row indices, in the product's entry
// order), its lane groups taking alternate entries as in spmm_seg_kernel, and
// each lane loads its 16-byte slices of the indexed row, with no products,
// partials or stores; a per-thread sum keeps the loads live.  Its rate is the
// ceiling for the product's gathers on the same matrix and panel width.
__global__ void __launch_bounds__(256)
gather_probe_kernel(int64_t nnz, const int *__restrict__ idx, const float4 *__restrict__ P, int ld4, int K4, int L,
                    float *__restrict__ sink) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = tid >> 5;
  const int lane = static_cast<int>(tid & 31), grp = lane / L, sub = lane % L, ngrp = 32 / L;
  const int64_t chunk = (nnz + nwarps - 1) / nwarps;
  const int64_t e0 = w * chunk, e1 = min(nnz, e0 + chunk);
  float acc = 0.f;
  for (int64_t e = e0 + grp; e < e1; e += ngrp) {
    const float4 *row = P + (int64_t)__ldg(idx + e) * ld4;
    for (int q = sub; q < K4; q += L) {
      const float4 v = __ldg(row + q);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  sink[tid] = acc;
}

void gather_probe(cudaStream_t st, int64_t nnz, const int *idx, const float *P, int ldp, int K, float *sink,
                  int grid) {
  const int K4 = (K + 3) / 4;
  int L = 1;
  while (L < K4 && L < 32) L <<= 1;
  gather_probe_kernel<<<grid, 256, 0, st>>>(nnz, idx, reinterpret_cast<const float4 *>(P), ldp / 4, K4, L, sink);
  MC_CHECK_LAUNCH();
}

int sddmm_update(cudaStream_t st, int64_t nnz, const int *rix, const int *col, const float *mval, float *y,
                 const float *Us, int ld_us, const float *V, int ld_v, int r, float delta, int update, double *block_sq,
                 float *x_out) {
  MC_REQUIRE(r >= 0, "sddmm: negative rank");
  MC_REQUIRE(ld_us % 4 == 0 && ld_v % 4 == 0 && ld_us >= r && ld_v >= r, "sddmm: bad leading dims");
  const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kSddmmBlocks, (nnz + kSddmmThreads - 1) / kSddmmThreads)));
  launch_pdl(sddmm_update_kernel, dim3(nb), dim3(kSddmmThreads), 0, st, nnz, rix, col, mval, y, Us, ld_us, V, ld_v,
             (r + 3) / 4, delta, update, block_sq, x_out);
  MC_CHECK_LAUNCH();
  return nb;
}

int sddmm_partials() { return kSddmmBlocks; }

void expand_rows(cudaStream_t st, int64_t m, const int *rp, int *rix) {
  if (m <= 0) return;
  const int64_t threads = m * 32;
  expand_rows_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(m, rp, rix);
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
