// Dense kernels of the rSVD hot path:
//   gemm_tn   C = X^T Y over the long dimension (Gram B = A^T A of eigSVD,
//             Alg. 3 step 1, and the block projections Q^T H)
//   gemm_nn   Z = beta Z + X W diag(s) (U = A V S^-1 of Alg. 3 step 4, the
//             Ritz vectors U = Q W of Alg. 5 step 11, H R^-1)
//   chol_inv  R^-1 of the Cholesky factor of a small Gram (block normalisation
//             standing in for lu() and orth(), which Lemmas 2-3 allow)
// All float32; every reduction runs in a fixed order (deterministic).
#include "mc_common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <mutex>

namespace mc {
namespace {

// ============================================================ gemm_tn ======
constexpr int TN_T = 64;   // output tile edge
constexpr int TN_RB = 32;  // rows staged per step

__global__ void __launch_bounds__(256)
gemm_tn_kernel(int64_t R, int K1, int K2, const float *__restrict__ X, int ld_x, const float *__restrict__ Y,
               int ld_y, int64_t rows_per_split, int tiles_j, bool sym, float *__restrict__ partial, int K1p,
               int K2p) {
  __shared__ __align__(16) float xs[TN_RB][TN_T];
  __shared__ __align__(16) float ys[TN_RB][TN_T];
  int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
  if (sym && tj < ti) return;  // lower tiles mirrored by the reducer
  const int split = blockIdx.y;
  const int64_t r0 = split * rows_per_split;
  const int64_t r1 = min(R, r0 + rows_per_split);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  float acc[4][4] = {};
  const int i0 = ti * TN_T, j0 = tj * TN_T;
  for (int64_t rb = r0; rb < r1; rb += TN_RB) {
    // stage 32 rows x 64 columns of X and Y (512 float4 each, 2 per thread)
    for (int q = tid; q < TN_RB * TN_T / 4; q += 256) {
      const int rr = q / (TN_T / 4), c4 = (q % (TN_T / 4)) * 4;
      const int64_t r = rb + rr;
      float4 vx = make_float4(0.f, 0.f, 0.f, 0.f), vy = vx;
      if (r < r1) {
        if (i0 + c4 < K1) vx = *reinterpret_cast<const float4 *>(X + r * ld_x + i0 + c4);
        if (j0 + c4 < K2) vy = *reinterpret_cast<const float4 *>(Y + r * ld_y + j0 + c4);
      }
      *reinterpret_cast<float4 *>(&xs[rr][c4]) = vx;
      *reinterpret_cast<float4 *>(&ys[rr][c4]) = vy;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < TN_RB; ++rr) {
      const float4 a = *reinterpret_cast<const float4 *>(&xs[rr][ty * 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&ys[rr][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  float *dst = partial + (int64_t)split * K1p * K2p;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u;
    *reinterpret_cast<float4 *>(dst + (int64_t)i * K2p + j0 + tx * 4) =
        make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
}

// ---- asynchronous global -> shared copies (cp.async, 16 bytes) -------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- gemm_tn for narrow panels (K1, K2 <= 64): one T x T output tile --------
// T in {16, 32, 64}.  The block's 256 threads form 256 / (T/4)^2 groups; a
// thread owns a 4 x 4 piece of the tile and its group walks every G-th row of
// the staged chunk.  Chunks of CH rows of X (and Y) stream through STAGES
// shared-memory buffers with cp.async, so loads of later chunks are in flight
// while a chunk is multiplied.  For the symmetric Gram the pieces below the
// diagonal are skipped (the reducer mirrors them).  The groups' sums are added
// in group order, and each block writes one partial tile.
constexpr int TNS_STAGES = 3;
template <int T>
struct TnSmall {
  static constexpr int TQ = T / 4, GT = TQ * TQ, G = 256 / GT, CH = (T == 64) ? 64 : 128;
  static constexpr size_t smem_bytes(bool same) { return sizeof(float) * TNS_STAGES * CH * T * (same ? 1 : 2); }
};

template <int T>
__global__ void __launch_bounds__(256)
gemm_tn_small_kernel(int64_t R, int K1, int K2, const float *__restrict__ X, int ld_x, const float *__restrict__ Y,
                     int ld_y, int64_t rows_per_split, int sym, int same, float *__restrict__ partial, int tiles_j,
                     int K1p, int K2p, const int *__restrict__ skip) {
  using P = TnSmall<T>;
  if (skip && *skip) return;  // a pass the previous one made unnecessary
  // output tile (ti, tj) of blockIdx.y; below-diagonal tiles of a Gram are mirrored by the reducer
  const int ti = blockIdx.y / tiles_j, tj = blockIdx.y % tiles_j;
  if (sym && tj < ti) return;
  const int i0 = ti * T, j0 = tj * T;
  X += i0;
  Y += j0;
  same = same && ti == tj;  // one staged panel serves both operands only on a diagonal tile
  extern __shared__ __align__(16) float tns[];
  float *xs = tns;                                          // [STAGES][CH][T]
  float *ys = same ? tns : tns + TNS_STAGES * P::CH * T;    // [STAGES][CH][T]
  const int tid = threadIdx.x;
  const int g = tid / P::GT, q = tid % P::GT, ty = q / P::TQ, tx = q % P::TQ;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_split;
  const int64_t r1 = min(R, r0 + rows_per_split);
  const int nchunks = r1 > r0 ? static_cast<int>((r1 - r0 + P::CH - 1) / P::CH) : 0;
  auto issue = [&](int c) {
    const int stg = c % TNS_STAGES;
    const int64_t rb = r0 + (int64_t)c * P::CH;
    for (int e = tid; e < P::CH * P::TQ; e += 256) {
      const int rr = e / P::TQ, c4 = (e % P::TQ) * 4;
      const int64_t r = rb + rr;
      const bool okx = r < r1 && i0 + c4 < K1;
      cp_async16(xs + ((size_t)stg * P::CH + rr) * T + c4, okx ? X + r * ld_x + c4 : X, okx ? 16 : 0);
      if (!same) {
        const bool oky = r < r1 && j0 + c4 < K2;
        cp_async16(ys + ((size_t)stg * P::CH + rr) * T + c4, oky ? Y + r * ld_y + c4 : Y, oky ? 16 : 0);
      }
    }
  };
#pragma unroll
  for (int c = 0; c < TNS_STAGES - 1; ++c) {
    if (c < nchunks) issue(c);
    cp_async_commit();
  }
  const bool active = i0 + ty * 4 < K1 && j0 + tx * 4 < K2 && !(sym && ti == tj && ty > tx);
  float acc[4][4] = {};
  for (int c = 0; c < nchunks; ++c) {
    if (c + TNS_STAGES - 1 < nchunks) issue(c + TNS_STAGES - 1);
    cp_async_commit();
    cp_async_wait<TNS_STAGES - 1>();
    __syncthreads();
    const int stg = c % TNS_STAGES;
    const float *xb = xs + (size_t)stg * P::CH * T, *yb = ys + (size_t)stg * P::CH * T;
    if (active) {
#pragma unroll 4
      for (int rr = g; rr < P::CH; rr += P::G) {
        const float4 a = *reinterpret_cast<const float4 *>(xb + rr * T + ty * 4);
        const float4 b = *reinterpret_cast<const float4 *>(yb + rr * T + tx * 4);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  float *dst = partial + (int64_t)blockIdx.x * K1p * K2p + (int64_t)i0 * K2p + j0;
  if (P::G == 1) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      *reinterpret_cast<float4 *>(dst + (int64_t)(ty * 4 + u) * K2p + tx * 4) =
          make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    return;
  }
  float *red = tns;  // [G][T][T], fits in the stage buffers
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<float4 *>(red + ((size_t)g * T + ty * 4 + u) * T + tx * 4) =
        make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  __syncthreads();
  for (int e = tid; e < T * T; e += 256) {
    float v = 0.f;
#pragma unroll
    for (int gg = 0; gg < P::G; ++gg) v += red[(size_t)gg * T * T + e];
    dst[(int64_t)(e / T) * K2p + e % T] = v;
  }
}

// Sum of the per-split partial tiles, in split order: a block covers 32
// outputs with 8 lanes of split groups each, then adds the 8 group sums in order.
__global__ void __launch_bounds__(256)
gemm_tn_reduce_kernel(int K1, int K2, int nsplit, const float *__restrict__ partial, int K1p, int K2p, bool sym,
                      int mirror, float *__restrict__ C, int ld_c, const int *__restrict__ skip = nullptr) {
  __shared__ float sh[8][33];
  pdl_wait();
  pdl_trigger();
  if (skip && *skip) return;
  const int64_t total = (int64_t)K1 * K2;
  const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t tile = (int64_t)K1p * K2p;
  for (int64_t base = (int64_t)blockIdx.x * 32; base < total; base += (int64_t)gridDim.x * 32) {
    const int64_t t = base + o;
    float acc = 0.f;
    int i = 0, j = 0;
    if (t < total) {
      i = static_cast<int>(t / K2);
      j = static_cast<int>(t % K2);
      int si = i, sj = j;
      if (sym && (j / mirror) < (i / mirror)) {  // piece below the diagonal: read the mirrored one
        si = j;
        sj = i;
      }
      const float *src = partial + (int64_t)si * K2p + sj;
      for (int sp = g; sp < nsplit; sp += 8) acc += src[sp * tile];
    }
    sh[g][o] = acc;
    __syncthreads();
    if (g == 0 && t < total) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) v += sh[q][o];
      C[(int64_t)i * ld_c + j] = v;
    }
    __syncthreads();
  }
}

// ---- gemm_nn with the small factor in shared memory --------------------------
// W (its K1 x 64 column slice for output columns j0 .. j0+63, zero-padded)
// stays in shared memory; 64-row chunks of X stream through cp.async
// buffers (three for K1 <= 64, two above).  Thread (ty, tx) computes rows
// 4 ty .. 4 ty + 3 and columns j0 + 4 tx .. + 3 of the chunk's output.
constexpr int NNS_BM = 64;
template <int KM1>
struct NnSmall {
  static constexpr int STAGES = KM1 <= 64 ? 3 : 2;
  static constexpr int LDX = KM1 + 4;  // padded row: the two row groups of a warp hit different banks
  static constexpr size_t smem = sizeof(float) * ((size_t)KM1 * 64 + (size_t)STAGES * NNS_BM * LDX);
};

// Z (R x K2) = alpha X W diag(colscale) + beta Z for narrow outputs
// (K2 <= KN <= 16, e.g. the factors U = Q W S of a low-rank estimate): a
// thread per row, W in shared memory read by broadcast, the row of X read
// with 16-byte loads; sums over k in ascending order as in the tiled kernels.
template <int KN>
__global__ void __launch_bounds__(256)
gemm_nn_narrow_kernel(int64_t R, int K1, int K2, const float *__restrict__ X, int ld_x, const float *__restrict__ W,
                      int ld_w, const float *__restrict__ colscale, float alpha, float beta, float *__restrict__ Z,
                      int ld_z) {
  extern __shared__ __align__(16) float wn[];  // K1 x KN, zero beyond K2
  for (int e = threadIdx.x; e < K1 * KN; e += blockDim.x) {
    const int k = e / KN, j = e % KN;
    wn[e] = j < K2 ? W[(int64_t)k * ld_w + j] : 0.f;
  }
  float sc[KN];
#pragma unroll
  for (int j = 0; j < KN; ++j) sc[j] = j < K2 ? alpha * (colscale ? colscale[j] : 1.0f) : 0.f;
  __syncthreads();
  const bool vec_in = ld_x % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
  const bool vec_out = K2 == KN && ld_z % 4 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15u) == 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const float *xr = X + r * ld_x;
    float acc[KN];
#pragma unroll
    for (int j = 0; j < KN; ++j) acc[j] = 0.f;
    int k = 0;
    if (vec_in)
      for (; k + 4 <= K1; k += 4) {
        const float4 x4 = __ldg(reinterpret_cast<const float4 *>(xr + k));
        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float4 *wr = reinterpret_cast<const float4 *>(wn + (k + t) * KN);
#pragma unroll
          for (int j4 = 0; j4 < KN / 4; ++j4) {
            const float4 w4 = wr[j4];
            acc[4 * j4 + 0] = fmaf(xv[t], w4.x, acc[4 * j4 + 0]);
            acc[4 * j4 + 1] = fmaf(xv[t], w4.y, acc[4 * j4 + 1]);
            acc[4 * j4 + 2] = fmaf(xv[t], w4.z, acc[4 * j4 + 2]);
            acc[4 * j4 + 3] = fmaf(xv[t], w4.w, acc[4 * j4 + 3]);
          }
        }
      }
    for (; k < K1; ++k) {
      const float xv = __ldg(xr + k);
#pragma unroll
      for (int j = 0; j < KN; ++j) acc[j] = fmaf(xv, wn[k * KN + j], acc[j]);
    }
    float *z = Z + r * ld_z;
    if (vec_out) {
#pragma unroll
      for (int j4 = 0; j4 < KN / 4; ++j4) {
        float4 o = make_float4(acc[4 * j4] * sc[4 * j4], acc[4 * j4 + 1] * sc[4 * j4 + 1],
                               acc[4 * j4 + 2] * sc[4 * j4 + 2], acc[4 * j4 + 3] * sc[4 * j4 + 3]);
        if (beta != 0.f) {
          const float4 pz = *reinterpret_cast<const float4 *>(z + 4 * j4);
          o.x += beta * pz.x;
          o.y += beta * pz.y;
          o.z += beta * pz.z;
          o.w += beta * pz.w;
        }
        *reinterpret_cast<float4 *>(z + 4 * j4) = o;
      }
    } else {
#pragma unroll
      for (int j = 0; j < KN; ++j) {
        if (j >= K2) continue;
        float o = acc[j] * sc[j];
        if (beta != 0.f) o += beta * z[j];
        z[j] = o;
      }
    }
  }
}

template <int KM1>
__global__ void __launch_bounds__(256)
gemm_nn_small_kernel(int64_t R, int K1, int K2, const float *__restrict__ X, int ld_x, const float *__restrict__ W,
                     int ld_w, const float *__restrict__ colscale, float alpha, float beta, float *__restrict__ Z,
                     int ld_z, int64_t chunks_per_block, const int *__restrict__ copy_if) {
  using P = NnSmall<KM1>;
  // copy mode (the factor is the identity: a pass the previous one made
  // unnecessary): Z = X, read through the same staging
  const bool copy = copy_if && *copy_if;
  extern __shared__ __align__(16) float nns[];
  float *ws = nns;                   // [KM1][64]
  float *xs = nns + KM1 * 64;        // [STAGES][BM][LDX]
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int j0 = blockIdx.y * 64;
  const int64_t nch_total = (R + NNS_BM - 1) / NNS_BM;
  const int64_t c0 = (int64_t)blockIdx.x * chunks_per_block;
  const int64_t c1 = min(nch_total, c0 + chunks_per_block);
  const int nch = c1 > c0 ? static_cast<int>(c1 - c0) : 0;
  const int K4 = (K1 + 3) / 4;
  auto issue = [&](int c) {
    const int stg = c % P::STAGES;
    const int64_t rb = (c0 + c) * NNS_BM;
    for (int e = tid; e < NNS_BM * (KM1 / 4); e += 256) {
      const int rr = e / (KM1 / 4), k4 = (e % (KM1 / 4)) * 4;
      const int64_t r = rb + rr;
      const bool ok = r < R && k4 < K1;
      cp_async16(xs + ((size_t)stg * NNS_BM + rr) * P::LDX + k4, ok ? X + r * ld_x + k4 : X, ok ? 16 : 0);
    }
  };
#pragma unroll
  for (int c = 0; c < P::STAGES - 1; ++c) {
    if (c < nch) issue(c);
    cp_async_commit();
  }
  for (int e = tid; e < KM1 * 64; e += 256) {
    const int k = e / 64, j = e % 64;
    ws[e] = (k < K1 && j0 + j < K2) ? W[(int64_t)k * ld_w + j0 + j] : 0.f;
  }
  float sc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = j0 + tx * 4 + v;
    sc[v] = j < K2 ? alpha * (colscale ? colscale[j] : 1.0f) : 0.f;
  }
  const bool vec_out = (ld_z % 4 == 0) && ((reinterpret_cast<uintptr_t>(Z) & 15u) == 0) && j0 + tx * 4 + 3 < K2;
  for (int c = 0; c < nch; ++c) {
    if (c + P::STAGES - 1 < nch) issue(c + P::STAGES - 1);
    cp_async_commit();
    cp_async_wait<P::STAGES - 1>();
    __syncthreads();
    const float *xb = xs + (size_t)(c % P::STAGES) * NNS_BM * P::LDX;
    float acc[4][4] = {};
    if (j0 + tx * 4 < K2) {
      if (copy) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = xb[(ty * 4 + u) * P::LDX + j0 + tx * 4 + v];
      }
      for (int k4 = 0; k4 < (copy ? 0 : K4); ++k4) {
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = *reinterpret_cast<const float4 *>(xb + (ty * 4 + u) * P::LDX + k4 * 4);
#pragma unroll
        for (int t = 0; t < 4; ++t) b[t] = *reinterpret_cast<const float4 *>(ws + (k4 * 4 + t) * 64 + tx * 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float av[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            acc[u][0] = fmaf(av[t], b[t].x, acc[u][0]);
            acc[u][1] = fmaf(av[t], b[t].y, acc[u][1]);
            acc[u][2] = fmaf(av[t], b[t].z, acc[u][2]);
            acc[u][3] = fmaf(av[t], b[t].w, acc[u][3]);
          }
        }
      }
      const int64_t rb = (c0 + c) * NNS_BM;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t r = rb + ty * 4 + u;
        if (r >= R) continue;
        float *z = Z + r * ld_z + j0 + tx * 4;
        if (copy) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (j0 + tx * 4 + v < K2) z[v] = acc[u][v];
        } else if (vec_out) {
          float4 o = make_float4(acc[u][0] * sc[0], acc[u][1] * sc[1], acc[u][2] * sc[2], acc[u][3] * sc[3]);
          if (beta != 0.f) {
            const float4 pz = *reinterpret_cast<const float4 *>(z);
            o.x += beta * pz.x;
            o.y += beta * pz.y;
            o.z += beta * pz.z;
            o.w += beta * pz.w;
          }
          *reinterpret_cast<float4 *>(z) = o;
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            if (j0 + tx * 4 + v >= K2) continue;
            z[v] = (beta != 0.f ? beta * z[v] : 0.f) + acc[u][v] * sc[v];
          }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

// ============================================================ gemm_nn ======
constexpr int NN_BM = 128, NN_BN = 64, NN_BK = 32;

__global__ void __launch_bounds__(256)
gemm_nn_kernel(int64_t R, int K1, int K2, const float *__restrict__ X, int ld_x, const float *__restrict__ W,
               int ld_w, const float *__restrict__ colscale, float alpha, float beta, float *__restrict__ Z,
               int ld_z) {
  __shared__ __align__(16) float xs[NN_BK][NN_BM + 4];
  __shared__ __align__(16) float ws[NN_BK][NN_BN];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t r0 = (int64_t)blockIdx.x * NN_BM;
  const int j0 = blockIdx.y * NN_BN;
  float acc[8][4] = {};
  for (int k0 = 0; k0 < K1; k0 += NN_BK) {
    // X tile: 128 rows x 32 k -> transposed into xs[k][row]
    for (int q = tid; q < NN_BM * NN_BK / 4; q += 256) {
      const int rr = q / (NN_BK / 4), kk = (q % (NN_BK / 4)) * 4;
      const int64_t r = r0 + rr;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < R) {
        const float *src = X + r * ld_x + k0 + kk;
        if (k0 + kk + 3 < K1) v = *reinterpret_cast<const float4 *>(src);
        else {
          float t[4] = {0.f, 0.f, 0.f, 0.f};
          for (int u = 0; u < 4; ++u)
            if (k0 + kk + u < K1) t[u] = src[u];
          v = make_float4(t[0], t[1], t[2], t[3]);
        }
      }
      xs[kk + 0][rr] = v.x;
      xs[kk + 1][rr] = v.y;
      xs[kk + 2][rr] = v.z;
      xs[kk + 3][rr] = v.w;
    }
    // W tile: 32 k x 64 columns
    for (int q = tid; q < NN_BK * NN_BN; q += 256) {
      const int kk = q / NN_BN, jj = q % NN_BN;
      ws[kk][jj] = (k0 + kk < K1 && j0 + jj < K2) ? W[(int64_t)(k0 + kk) * ld_w + j0 + jj] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < NN_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&xs[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&xs[kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&ws[kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int64_t r = r0 + ty * 8 + u;
    if (r >= R) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (j >= K2) continue;
      const float s = alpha * (colscale ? colscale[j] : 1.0f);
      float *z = Z + r * ld_z + j;
      *z = (beta != 0.f ? beta * *z : 0.f) + acc[u][v] * s;
    }
  }
}

// ============================================== chol_inv (narrow blocks) ==
// K <= 128: G + shift I = L L^T and L^{-1} together, right-looking, in shared
// memory.  Step j scales column j of L by 1/sqrt(pivot) and row j of the
// running right-hand side B (B = I at the start; row j of B becomes row j of
// L^{-1}); then every row a > j is updated by one warp over its entries:
// columns b <= j of B (B[a][b] -= L[a][j] X[j][b]) and columns j < b <= a of
// L (the trailing update).  Two barriers per step, K steps.  The diagonal of
// L is never overwritten (its final value is kept in dg), so the pivot of the
// next step can be read right after the second barrier.
__global__ void __launch_bounds__(1024)
chol_inv_small_kernel(int K, const float *__restrict__ G, int ld, float shift_rel, const float *__restrict__ ref_diag,
                      float ref_tol, float *__restrict__ Rinv, const int *__restrict__ skip_if,
                      int *__restrict__ set_skip, float skip3) {
  extern __shared__ float sh[];
  if (skip_if && *skip_if) return;  // a pass the previous one made unnecessary
  const int ls = (K % 2 == 0) ? K + 1 : K;  // odd row stride: column reads are conflict-free
  float *L = sh;                            // K x ls
  float *B = L + (size_t)K * ls;            // K x ls
  float *flags = B + (size_t)K * ls;        // K
  const int tid = threadIdx.x, nt = blockDim.x;
  const int wid = tid >> 5, lane = tid & 31, nw = nt >> 5;
  __shared__ float s_tr, s_max;
  if (tid < 32) {
    float tr = 0.f, mx = 0.f;
    for (int i = lane; i < K; i += 32) {
      const float gi = G[(int64_t)i * ld + i];
      tr += gi;
      mx = fmaxf(mx, gi);
    }
    for (int off = 16; off > 0; off >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, off);
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
      s_tr = tr;
      s_max = mx;
    }
  }
  for (int i = tid; i < K; i += nt)
    flags[i] = (ref_diag && !(G[(int64_t)i * ld + i] > ref_tol * ref_diag[i])) ? 0.f : 1.f;
  __syncthreads();
  const float shift = shift_rel * s_tr / K;
  const float drop = fmaxf(1e-30f, 1e-12f * s_max) + shift;
  float dev = 0.f;  // largest |G - I| over the lower triangle
  for (int t = tid; t < K * K; t += nt) {
    const int i = t / K, j = t % K;
    const bool live = flags[i] != 0.f && flags[j] != 0.f;
    const float g = j <= i ? G[(int64_t)i * ld + j] : 0.f;
    if (j <= i) dev = fmaxf(dev, fabsf(g - (i == j ? 1.f : 0.f)));
    L[i * ls + j] = (j <= i && live) ? g + (i == j ? shift : 0.f) : 0.f;
    B[i * ls + j] = (i == j) ? 1.f : 0.f;
  }
  if (set_skip) {
    __shared__ unsigned s_dev;
    if (tid == 0) s_dev = 0u;
    __syncthreads();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, off));
    if (lane == 0) atomicMax(&s_dev, __float_as_uint(dev));  // nonnegative floats order as their bits
    __syncthreads();
    if (tid == 0) *set_skip = __uint_as_float(s_dev) <= skip3 ? 1 : 0;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    const float d = L[j * ls + j];
    const bool keep = d > drop;
    const float inv = keep ? rsqrtf(d) : 0.f;
    // column j of L and row j of L^{-1}
    for (int i = j + 1 + tid; i < K; i += nt) L[i * ls + j] *= inv;
    for (int c = tid; c <= j; c += nt) B[j * ls + c] *= inv;
    if (tid == 0 && !keep) flags[j] = 0.f;
    __syncthreads();
    if (keep) {
      for (int a = j + 1 + wid; a < K; a += nw) {
        const float la = L[a * ls + j];
        for (int b = lane; b <= a; b += 32) {
          if (b <= j) B[a * ls + b] -= la * B[j * ls + b];
          else L[a * ls + b] -= la * L[b * ls + j];
        }
      }
    }
    __syncthreads();
  }
  // R^{-1} = (L^{-1})^T; rows and columns of dropped pivots are zero
  for (int t = tid; t < K * K; t += nt) {
    const int i = t / K, c = t % K;
    Rinv[t] = (flags[i] != 0.f && flags[c] != 0.f && c >= i) ? B[c * ls + i] : 0.f;
  }
}

// ============================================== chol_inv (K <= 64) =======
// The factorisation and inverse of chol_inv_small_kernel for K <= 64, with
// the same rounding (every entry takes its updates one fused multiply-add at
// a time, in pivot order), arranged for latency: the matrix is padded to 64
// with an identity block and factored in four 16-column blocks,
//   (1) the diagonal block by one warp, lane a holding row a in registers and
//       the column of each step passed by shuffles;
//   (2) the rows below it by a thread per row, registers again, the block's
//       L read as shared-memory broadcasts;
//   (3) the trailing matrix's rank-16 update by a thread per entry;
// three barriers per block.  L^{-1} follows by columns, four threads (one
// warp's lanes 4c'..4c'+3) per column holding its rows i = r (mod 4) in
// registers: step k scales entry (k, c) by the pivot's 1/sqrt and shuffles
// it to the other three, which update their rows i > k.  Pivots at or below
// the drop threshold give a zero column of L and a zero row of L^{-1}.
constexpr int CB_K = 64, CB_NB = 16, CB_THREADS = 256;
__global__ void __launch_bounds__(CB_THREADS)
chol_inv_blk_kernel(int K, const float *__restrict__ G, int ld, float shift_rel, const float *__restrict__ ref_diag,
                    float ref_tol, float *__restrict__ Rinv, const int *__restrict__ skip_if,
                    int *__restrict__ set_skip, float skip3) {
  __shared__ float As[CB_K][CB_K + 1];  // lower triangle: A, then L (its diagonal keeps the pivot)
  __shared__ float invd[CB_K], flags[CB_K], diagv[CB_K];
  __shared__ float s_tr, s_max;
  __shared__ unsigned s_dev;
  pdl_wait();
  pdl_trigger();
  if (skip_if && *skip_if) return;  // a pass the previous one made unnecessary
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned full = 0xffffffffu;
  // every load in flight at once: entry (i, j) = (e / 64, e % 64), e = tid + 256 u
  float g[16];
  float dev = 0.f;  // largest |G - I| over the lower triangle
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = tid + CB_THREADS * u, i = e >> 6, j = e & 63;
    g[u] = (i < K && j <= i) ? G[(int64_t)i * ld + j] : 0.f;
  }
  const float rd = (ref_diag && tid < K) ? ref_diag[tid] : 0.f;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = tid + CB_THREADS * u, i = e >> 6, j = e & 63;
    if (i < K && j <= i) dev = fmaxf(dev, fabsf(g[u] - (i == j ? 1.f : 0.f)));
    if (i == j && i < K) diagv[i] = g[u];
  }
  if (tid == 0) s_dev = 0u;
  __syncthreads();
  if (wid == 0) {
    float tr = 0.f, mx = 0.f;
    for (int i = lane; i < K; i += 32) {
      tr += diagv[i];
      mx = fmaxf(mx, diagv[i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      tr += __shfl_xor_sync(full, tr, off);
      mx = fmaxf(mx, __shfl_xor_sync(full, mx, off));
    }
    if (lane == 0) {
      s_tr = tr;
      s_max = mx;
    }
  }
  // a column that lost (almost) all of its norm to an earlier projection is
  // rounding noise: it is removed before factoring
  if (tid < CB_K) flags[tid] = (tid < K && ref_diag && !(diagv[tid] > ref_tol * rd)) ? 0.f : 1.f;
  if (set_skip) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dev = fmaxf(dev, __shfl_xor_sync(full, dev, off));
    if (lane == 0) atomicMax(&s_dev, __float_as_uint(dev));  // nonnegative floats order as their bits
  }
  __syncthreads();
  if (set_skip && tid == 0) *set_skip = __uint_as_float(s_dev) <= skip3 ? 1 : 0;
  const float shift = shift_rel * s_tr / K;
  const float drop = fmaxf(1e-30f, 1e-12f * s_max) + shift;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = tid + CB_THREADS * u, i = e >> 6, j = e & 63;
    if (j > i) continue;
    if (i < K) As[i][j] = (flags[i] != 0.f && flags[j] != 0.f) ? g[u] + (i == j ? shift : 0.f) : 0.f;
    else As[i][j] = i == j ? 1.f : 0.f;  // padding: an identity block, coupled to nothing
  }
  __syncthreads();
  chol64_blocked(As, drop, invd, flags);
  // L^{-1}: thread (c, r) holds entries (4q + r, c); at step k entry (k, c) is
  // final once scaled, and the rows below take its multiple
  const int c = tid >> 2, r = tid & 3, src0 = lane & ~3;
  float v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = 4 * q + r == c ? 1.f : 0.f;
  auto inv_step = [&](const int k) {
    if (r == (k & 3)) v[k >> 2] *= invd[k];
    const float x = __shfl_sync(full, v[k >> 2], src0 | (k & 3));
#pragma unroll
    for (int q = k >> 2; q < 16; ++q) {
      const int i = 4 * q + r;
      if (i > k) v[q] = fmaf(-As[i][k], x, v[q]);
    }
  };
  // four constant-trip loops unroll completely: every index into v is a constant
#pragma unroll
  for (int k = 0; k < 16; ++k) inv_step(k);
#pragma unroll
  for (int k = 16; k < 32; ++k) inv_step(k);
#pragma unroll
  for (int k = 32; k < 48; ++k) inv_step(k);
#pragma unroll
  for (int k = 48; k < 64; ++k) inv_step(k);
  // R^{-1} = (L^{-1})^T: row c of R^{-1} is column c of L^{-1}; rows and
  // columns of dropped pivots are zero
  if (c < K) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int rho = 4 * q + r;
      if (rho < K) Rinv[(int64_t)c * K + rho] = (rho >= c && flags[c] != 0.f && flags[rho] != 0.f) ? v[q] : 0.f;
    }
  }
}

// =========================================================== chol_inv ======
// One block.  G + shift I = L L^T (right-looking, warp per row of the trailing
// update); pivots below the drop threshold make their column "absent": its
// row of L^{-1} is zero, so the matching column of H R^{-1} is zero and the
// others ignore it.  L^{-1} by forward substitution, one thread per column,
// reading L as warp broadcasts; the result is written transposed: R^{-1}.
__global__ void __launch_bounds__(1024)
chol_inv_kernel(int K, const float *__restrict__ G, int ld, float shift_rel, const float *__restrict__ ref_diag,
                float ref_tol, float *__restrict__ Rinv, int X_in_smem) {
  extern __shared__ float sh[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int wid = tid >> 5, lane = tid & 31, nw = nt >> 5;
  float *L = sh;                                   // K x K, lower
  float *flags = sh + (size_t)K * K;               // K: 1 = kept
  float *X = X_in_smem ? flags + K : Rinv;         // K x K: L^{-1} (X[l][c])
  __shared__ float s_tr, s_max;
  if (tid < 32) {
    float tr = 0.f, mx = 0.f;
    for (int i = lane; i < K; i += 32) {
      const float gi = G[(int64_t)i * ld + i];
      tr += gi;
      mx = fmaxf(mx, gi);
    }
    for (int off = 16; off > 0; off >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, off);
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) {
      s_tr = tr;
      s_max = mx;
    }
  }
  // a column that lost (almost) all of its norm to an earlier projection is
  // rounding noise: remove it before factoring
  for (int i = tid; i < K; i += nt)
    flags[i] = (ref_diag && !(G[(int64_t)i * ld + i] > ref_tol * ref_diag[i])) ? 0.f : 1.f;
  __syncthreads();
  const float shift = shift_rel * s_tr / K;
  const float drop = fmaxf(1e-30f, 1e-12f * s_max) + shift;
  for (int t = tid; t < K * K; t += nt) {
    const int i = t / K, j = t % K;
    const bool live = flags[i] != 0.f && flags[j] != 0.f;
    L[t] = (j <= i && live) ? G[(int64_t)i * ld + j] + (i == j ? shift : 0.f) : 0.f;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    const float d = L[j * K + j];
    const bool keep = d > drop;
    const float inv = keep ? rsqrtf(d) : 0.f;
    __syncthreads();  // every thread has read the pivot before it is overwritten
    for (int i = j + 1 + tid; i < K; i += nt) L[i * K + j] *= inv;
    if (tid == 0) {
      L[j * K + j] = keep ? d * inv : 1.0f;
      flags[j] = keep ? flags[j] : 0.f;
    }
    __syncthreads();
    if (keep) {
      for (int a = j + 1 + wid; a < K; a += nw) {
        const float la = L[a * K + j];
        for (int b = j + 1 + lane; b <= a; b += 32) L[a * K + b] -= la * L[b * K + j];
      }
      __syncthreads();
    }
  }
  // forward substitution: column c of L^{-1}
  for (int c = tid; c < K; c += nt) {
    const bool kc = flags[c] != 0.f;
    for (int i = 0; i < K; ++i) {
      float x = 0.f;
      if (kc && i >= c && flags[i] != 0.f) {
        float a0 = (i == c) ? 1.0f : 0.0f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int l = c;
        for (; l + 3 < i; l += 4) {
          a0 -= L[i * K + l] * X[(int64_t)l * K + c];
          a1 -= L[i * K + l + 1] * X[(int64_t)(l + 1) * K + c];
          a2 -= L[i * K + l + 2] * X[(int64_t)(l + 2) * K + c];
          a3 -= L[i * K + l + 3] * X[(int64_t)(l + 3) * K + c];
        }
        for (; l < i; ++l) a0 -= L[i * K + l] * X[(int64_t)l * K + c];
        x = ((a0 + a1) + (a2 + a3)) / L[i * K + i];
      }
      X[(int64_t)i * K + c] = x;
    }
  }
  __syncthreads();
  if (X_in_smem) {
    for (int t = tid; t < K * K; t += nt) {
      const int i = t / K, j = t % K;
      Rinv[t] = X[(int64_t)j * K + i];  // R^{-1} = (L^{-1})^T
    }
  } else {
    for (int t = tid; t < K * K; t += nt) {
      const int i = t / K, j = t % K;
      if (i < j) {
        const float a = Rinv[(int64_t)i * K + j], b = Rinv[(int64_t)j * K + i];
        Rinv[(int64_t)i * K + j] = b;
        Rinv[(int64_t)j * K + i] = a;
      }
    }
  }
}

// Column sums of squares of X (R x K): per-chunk partials, then an ordered sum.
// A block's 256 threads cover K4 = ceil(K/4) float4 columns and 256 / K4 row
// lanes (K4 <= 64); lane sums are added in lane order in shared memory.
__global__ void __launch_bounds__(256)
colsumsq_partial_kernel(int64_t R, int K, const float *__restrict__ X, int ld, int64_t rows_per,
                        float *__restrict__ part) {
  __shared__ float4 sh[256];
  const int K4 = (K + 3) / 4;
  const int lanes = 256 / K4;
  const int tid = threadIdx.x, c4 = tid % K4, rl = tid / K4;
  const int64_t r0 = blockIdx.x * rows_per, r1 = min(R, r0 + rows_per);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (rl < lanes) {
#pragma unroll 4
    for (int64_t r = r0 + rl; r < r1; r += lanes) {
      const float4 v = *reinterpret_cast<const float4 *>(X + r * ld + c4 * 4);
      acc.x = fmaf(v.x, v.x, acc.x);
      acc.y = fmaf(v.y, v.y, acc.y);
      acc.z = fmaf(v.z, v.z, acc.z);
      acc.w = fmaf(v.w, v.w, acc.w);
    }
  }
  sh[tid] = acc;
  __syncthreads();
  if (tid < K4) {
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int l = 0; l < lanes; ++l) {
      const float4 u = sh[l * K4 + tid];
      t.x += u.x;
      t.y += u.y;
      t.z += u.z;
      t.w += u.w;
    }
    const float tv[4] = {t.x, t.y, t.z, t.w};
    for (int q = 0; q < 4; ++q)
      if (tid * 4 + q < K) part[(int64_t)blockIdx.x * K + tid * 4 + q] = tv[q];
  }
}

// Columns beyond 256 (or unaligned panels): one thread per column.
__global__ void colsumsq_partial_wide_kernel(int64_t R, int K, const float *__restrict__ X, int ld, int64_t rows_per,
                                             float *__restrict__ part) {
  const int64_t r0 = blockIdx.x * rows_per, r1 = min(R, r0 + rows_per);
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) {
      const float v = X[r * ld + c];
      acc = fmaf(v, v, acc);
    }
    part[(int64_t)blockIdx.x * K + c] = acc;
  }
}

// One block per column: a fixed-order tree over the chunk partials.
__global__ void colsumsq_reduce_kernel(int K, int nchunk, const float *__restrict__ part, float *__restrict__ out) {
  __shared__ float sh[256];
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int b = threadIdx.x; b < nchunk; b += blockDim.x) acc += part[(int64_t)b * K + c];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < (unsigned)off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// out (K x ncp) = W[:, 0:ncols] with zero columns up to ncp
__global__ void select_cols_kernel(int K, const float *__restrict__ W, int ld_w, int ncols, int ncp,
                                   float *__restrict__ out) {
  const int64_t total = (int64_t)K * ncp;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = static_cast<int>(t / ncp), j = static_cast<int>(t % ncp);
    out[t] = j < ncols ? W[(int64_t)i * ld_w + j] : 0.f;
  }
}

// ===================================== narrow block orthonormalisation ====
// One cooperative kernel for a whole Krylov block of width K <= 32 (the
// narrow blocks of the SVT iteration): optional column norms before the
// projection (the dependence test), two projections against the earlier
// blocks Qp (X -= Qp (Qp^T X)), then CholeskyQR passes: a shifted one, a
// plain one, and a third unless the shifted pass already left the block
// orthonormal to within 1e-2 (the separate kernels always run all three).
// Each CTA keeps its
// rows of X and Qp in shared memory for the whole sequence; every reduction
// over rows is per-CTA partials, a grid barrier, a fixed-order sum split
// across the CTAs, and a second barrier.  The K x K Cholesky-inverse is
// repeated by every CTA (it is tiny), so its result needs no barrier.
constexpr int ON_THREADS = 256;
constexpr int ON_MAXK = 32;

struct OrthNarrowArgs {
  int64_t R, rows_per;
  int K, cols, ldx, ldq, ldo, use_ref;
  int q_smem;        // 1: rows of Qp staged in shared memory; 0: read from global (L2)
  float skip3;       // max |G - I| of the second pass that makes the third redundant
  float *X;          // R x K (clobbered)
  const float *Qp;   // R x cols
  float *out;        // R x K
  float *part;       // nblk x max(cols K + K, K K)
  float *fin;        // cols K + K + K K
  float shift_rel, ref_tol;
};

// sum over the CTAs' partials of entries [0, count): a warp per entry, lane l
// adds partials l, l + 32, ... and the lanes' sums meet in a fixed shuffle tree
__device__ __forceinline__ void on_reduce(const OrthNarrowArgs &a, int count, int stride, float *dst) {
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (ON_THREADS / 32) + (threadIdx.x >> 5), nw = nb * (ON_THREADS / 32);
  constexpr int BATCH = 8;  // independent loads in flight per lane
  for (int e = gw; e < count; e += nw) {
    float acc = 0.f;
    for (int b0 = lane; b0 < nb; b0 += 32 * BATCH) {
      float v[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int b = b0 + 32 * u;
        v[u] = b < nb ? a.part[(int64_t)b * stride + e] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) acc += v[u];  // partials lane, lane + 32, ... in order
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) dst[e] = acc;
  }
}

// Row strides of the shared-memory copies: multiples of 4 floats (16-byte
// rows) with an odd number of 16-byte groups, so eight consecutive rows read
// with 16-byte loads fall in distinct bank groups.
__host__ __device__ inline int on_ld(int w) {
  const int w4 = (w + 3) / 4 * 4;
  return ((w4 / 4) & 1) ? w4 : w4 + 4;
}

// partial[ti][tj] (4 x 4 tiles) of A^T B over the CTA's rows, A = As (width
// na, stride lda), B = Bs (width nb4*4, stride ldb); tiles with ti > tj are
// skipped when upper.  Groups of threads take interleaved rows; their tile
// sums meet in shared memory in group order.  Writes count = na4*4 x nb4*4
// values (row-major, width nb4*4) to dst.
__device__ __forceinline__ void on_tile_products(const float *As, int lda, int na4, const float *Bs, int ldb, int nb4,
                                                 int nr, bool upper, float *red, float *dst) {
  const int tid = threadIdx.x;
  const int T = na4 * nb4;
  const int G = max(1, ON_THREADS / T);
  float acc[4][4] = {};
  const int tile = tid % T, g = tid / T;
  const int ti = tile / nb4, tj = tile % nb4;
  const bool act = g < G && tid < T * G && !(upper && ti > tj);
  if (act)
    for (int r = g; r < nr; r += G) {
      const float4 x = *reinterpret_cast<const float4 *>(As + r * lda + 4 * ti);
      const float4 y = *reinterpret_cast<const float4 *>(Bs + r * ldb + 4 * tj);
      const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
    }
  if (tid < T * G)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) red[(size_t)tid * 16 + u * 4 + v] = act ? acc[u][v] : 0.f;
  __syncthreads();
  const int W = nb4 * 4;
  for (int o = tid; o < T * 16; o += ON_THREADS) {
    const int t = o / 16, e = o % 16;
    float sum = 0.f;
    for (int q = 0; q < G; ++q) sum += red[(size_t)(q * T + t) * 16 + e];
    const int i = (t / nb4) * 4 + e / 4, j = (t % nb4) * 4 + e % 4;
    dst[i * W + j] = sum;
  }
  __syncthreads();
}

template <int KM>
__global__ void __launch_bounds__(ON_THREADS, KM <= 16 ? 2 : 1) orth_narrow_kernel(OrthNarrowArgs a) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float onsm[];
  const int K = a.K, cols = a.cols, tid = threadIdx.x;
  const int K4 = (K + 3) / 4, C4 = (cols + 3) / 4, KW = K4 * 4, CW = C4 * 4;
  const int ldh = on_ld(K), ldqs = on_ld(cols);
  const int64_t r0 = blockIdx.x * a.rows_per;
  const int64_t r1 = a.R < r0 + a.rows_per ? a.R : r0 + a.rows_per;
  const int nr = r1 > r0 ? static_cast<int>(r1 - r0) : 0;
  float *Hs = onsm;                                   // rows_per x ldh (zero beyond K)
  float *Qsm = Hs + (size_t)a.rows_per * ldh;         // rows_per x ldqs when staged
  float *Ms = Qsm + (a.q_smem ? (size_t)a.rows_per * ldqs : 0);  // CW x KW (C) or KW x KW (G)
  // this CTA's rows of Qp: the staged copy, or the rows in global memory (L2)
  const float *Qs = a.q_smem ? Qsm : a.Qp + (cols > 0 ? r0 * a.ldq : 0);
  const int ldq = a.q_smem ? ldqs : a.ldq;
  float *red = Ms + (size_t)max(CW, KW) * KW;         // ON_THREADS x 16
  float *Ls = red + (size_t)ON_THREADS * 16;          // K x (K+1): Cholesky factor
  float *Bs = Ls + (size_t)K * (K + 1);               // K x (K+1): running inverse
  float *fl = Bs + (size_t)K * (K + 1);               // K flags
  float *refs = fl + K;                               // K column norms^2
  const int stride = max(CW * KW + KW, KW * KW);  // per-CTA partials of C (+ norms) or of G
  float *fin_C = a.fin, *fin_G = a.fin + stride;

  // rows of X and Qp into shared memory, 16 bytes per copy (K, cols, the
  // leading dimensions and the bases are multiples of 4 floats); columns
  // K..ldh and cols..ldq are never read
  for (int t = tid; t < nr * K4; t += ON_THREADS) {
    const int r = t / K4, c = t % K4;
    cp_async16(Hs + r * ldh + 4 * c, a.X + (r0 + r) * a.ldx + 4 * c, 16);
  }
  if (a.q_smem)
    for (int t = tid; t < nr * C4; t += ON_THREADS) {
      const int r = t / C4, c = t % C4;
      cp_async16(Qsm + r * ldqs + 4 * c, a.Qp + (r0 + r) * a.ldq + 4 * c, 16);
    }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();

  // X -= Qp (Qp^T X), twice; the column norms^2 before the projection (the
  // dependence test of the first pass) ride along with the first product
  const int nref = a.use_ref ? K : 0;
  for (int rep = 0; rep < 2 && cols > 0; ++rep) {
    float *dst = a.part + (int64_t)blockIdx.x * stride;
    on_tile_products(Qs, ldq, C4, Hs, ldh, K4, nr, false, red, dst);
    if (rep == 0)
      for (int c = tid; c < nref; c += ON_THREADS) {
        float acc = 0.f;
        for (int r = 0; r < nr; ++r) acc = fmaf(Hs[r * ldh + c], Hs[r * ldh + c], acc);
        dst[CW * KW + c] = acc;
      }
    grid.sync();
    on_reduce(a, CW * KW + (rep == 0 ? nref : 0), stride, fin_C);
    grid.sync();
    for (int o = tid; o < CW * KW; o += ON_THREADS) Ms[o] = fin_C[o];
    if (rep == 0)
      for (int c = tid; c < nref; c += ON_THREADS) refs[c] = fin_C[CW * KW + c];
    __syncthreads();
    // a thread per row: out = h - q C with q (the row of Qp) read 4 at a time
    for (int r = tid; r < nr; r += ON_THREADS) {
      float out[KM];
#pragma unroll
      for (int j4 = 0; j4 < KM / 4; ++j4) {
        const float4 h4 = j4 < K4 ? *reinterpret_cast<const float4 *>(Hs + r * ldh + 4 * j4) : make_float4(0, 0, 0, 0);
        out[4 * j4 + 0] = h4.x;
        out[4 * j4 + 1] = h4.y;
        out[4 * j4 + 2] = h4.z;
        out[4 * j4 + 3] = h4.w;
      }
      for (int i4 = 0; i4 < C4; ++i4) {
        const float4 q4 = *reinterpret_cast<const float4 *>(Qs + r * ldq + 4 * i4);
        const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float *crow = Ms + (4 * i4 + u) * KW;
#pragma unroll
          for (int j4 = 0; j4 < KM / 4; ++j4) {
            if (j4 < K4) {
              const float4 c4 = *reinterpret_cast<const float4 *>(crow + 4 * j4);
              out[4 * j4 + 0] = fmaf(-qv[u], c4.x, out[4 * j4 + 0]);
              out[4 * j4 + 1] = fmaf(-qv[u], c4.y, out[4 * j4 + 1]);
              out[4 * j4 + 2] = fmaf(-qv[u], c4.z, out[4 * j4 + 2]);
              out[4 * j4 + 3] = fmaf(-qv[u], c4.w, out[4 * j4 + 3]);
            }
          }
        }
      }
#pragma unroll
      for (int j4 = 0; j4 < KM / 4; ++j4)
        if (j4 < K4)
          *reinterpret_cast<float4 *>(Hs + r * ldh + 4 * j4) =
              make_float4(out[4 * j4], out[4 * j4 + 1], out[4 * j4 + 2], out[4 * j4 + 3]);
    }
    __syncthreads();
  }

  // CholeskyQR passes: X <- X R^{-1} with X^T X + shift I = R^T R, the first
  // shifted.  The third is skipped when the second pass's Gram is within
  // skip3 of the identity on its live columns: its input then has a
  // condition number near 1, one pass leaves O(u) orthogonality (the
  // CholeskyQR2 bound) and a third would change nothing that matters.  Every
  // CTA reduces the same Gram in the same order, so all take the same branch.
  __shared__ int s_skip3;
  if (tid == 0) s_skip3 = 0;
  for (int pass = 0; pass < 3; ++pass) {
    on_tile_products(Hs, ldh, K4, Hs, ldh, K4, nr, true, red, a.part + (int64_t)blockIdx.x * stride);
    grid.sync();
    on_reduce(a, KW * KW, stride, fin_G);
    grid.sync();
    // G (upper triangle reduced; mirrored) -> L L^T and L^{-1}, as chol_inv:
    // the lower triangle of G into Ls in one parallel read; then one warp
    // factors it in registers, lane r holding row r of the trailing matrix
    // and of the inverse, the pivot column and row broadcast by shuffles
    for (int t = tid; t < K * K; t += ON_THREADS) {
      const int i = t / K, j = t % K;
      Ls[i * (K + 1) + j] = j <= i ? fin_G[j * KW + i] : 0.f;
    }
    __syncthreads();
    if (tid < 32) {
      const int lane = tid;
      const unsigned full = 0xffffffffu;
      if (lane < K)
        fl[lane] = (pass == 0 && a.use_ref && !(Ls[lane * (K + 1) + lane] > a.ref_tol * refs[lane])) ? 0.f : 1.f;
      float tr = 0.f, mx = 0.f;  // the same order on every lane
      for (int i = 0; i < K; ++i) {
        const float g = Ls[i * (K + 1) + i];
        tr += g;
        mx = fmaxf(mx, g);
      }
      const float shift = (pass == 0 ? a.shift_rel : 0.f) * tr / K;
      const float drop = fmaxf(1e-30f, 1e-12f * mx) + shift;
      if (pass == 1) {
        // largest |G - I| over live columns (zero columns, dropped before, excluded)
        float dev = 0.f;
        if (lane < K && Ls[lane * (K + 1) + lane] > 0.5f)
          for (int c = 0; c <= lane; ++c)
            if (Ls[c * (K + 1) + c] > 0.5f) dev = fmaxf(dev, fabsf(Ls[lane * (K + 1) + c] - (c == lane ? 1.f : 0.f)));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dev = fmaxf(dev, __shfl_xor_sync(full, dev, off));
        if (lane == 0) s_skip3 = dev <= a.skip3;
      }
      __syncwarp();
      const int rl = min(lane, K - 1);  // clamped indices: every load is in bounds, all issue at once
      const bool live_r = lane < K && fl[rl] != 0.f;
      float lr_[KM], br_[KM];
#pragma unroll
      for (int c = 0; c < KM; ++c) {
        const int cl = min(c, K - 1);
        const float g = Ls[rl * (K + 1) + cl];
        const bool live = live_r && c < K && c <= lane && fl[cl] != 0.f;
        lr_[c] = live ? g + (c == lane ? shift : 0.f) : 0.f;
        br_[c] = c == lane ? 1.f : 0.f;
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < KM; ++j) {
        if (j >= K) continue;  // uniform; keeps every register index static
        const float d = __shfl_sync(full, lr_[j], j);
        const bool keep = d > drop;
        const float inv = keep ? rsqrtf(d) : 0.f;
        if (lane > j) lr_[j] *= inv;  // column j of L below the diagonal
        if (lane == j) {
#pragma unroll
          for (int c = 0; c <= j; ++c) br_[c] *= inv;  // row j of L^{-1}
        }
        if (lane == 0 && !keep) fl[j] = 0.f;
        if (keep) {
          const float lr = lr_[j];
#pragma unroll
          for (int b = 0; b < KM; ++b) {
            if (b <= j) {  // L^{-1}[r][b] -= L[r][j] L^{-1}[j][b]
              const float bjb = __shfl_sync(full, br_[b], j);
              if (lane > j) br_[b] -= lr * bjb;
            } else {       // trailing L[r][b] -= L[r][j] L[b][j], b <= r
              const float lbj = __shfl_sync(full, lr_[j], b);
              if (lane > j && b <= lane) lr_[b] -= lr * lbj;
            }
          }
        }
      }
      if (lane < K) {
#pragma unroll
        for (int c = 0; c < KM; ++c)
          if (c < K) Bs[lane * (K + 1) + c] = br_[c];
      }
    }
    __syncthreads();
    // X <- X R^{-1}, R^{-1}[l][c] = L^{-1}[c][l] (kept l, c only), a thread per row
    for (int r = tid; r < nr; r += ON_THREADS) {
      float h[KM], o[KM];
#pragma unroll
      for (int l4 = 0; l4 < KM / 4; ++l4) {
        const float4 h4 = l4 < K4 ? *reinterpret_cast<const float4 *>(Hs + r * ldh + 4 * l4) : make_float4(0, 0, 0, 0);
        h[4 * l4 + 0] = h4.x;
        h[4 * l4 + 1] = h4.y;
        h[4 * l4 + 2] = h4.z;
        h[4 * l4 + 3] = h4.w;
      }
#pragma unroll
      for (int l = 0; l < KM; ++l) h[l] = (l < K && fl[l] != 0.f) ? h[l] : 0.f;
#pragma unroll
      for (int c = 0; c < KM; ++c) {
        float acc = 0.f;
        if (c < K && fl[c] != 0.f) {
#pragma unroll
          for (int l = 0; l <= c; ++l) acc = fmaf(h[l], Bs[c * (K + 1) + l], acc);
        }
        o[c] = acc;
      }
#pragma unroll
      for (int c4 = 0; c4 < KM / 4; ++c4)
        if (c4 < K4)
          *reinterpret_cast<float4 *>(Hs + r * ldh + 4 * c4) = make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
    }
    __syncthreads();
    if (pass == 1 && s_skip3) break;
  }
  for (int t = tid; t < nr * K4; t += ON_THREADS) {
    const int r = t / K4, c = t % K4;
    *reinterpret_cast<float4 *>(a.out + (r0 + r) * a.ldo + 4 * c) =
        *reinterpret_cast<const float4 *>(Hs + r * ldh + 4 * c);
  }
}

}  // namespace

// ================================================================ launchers ==
size_t colsumsq_scratch_floats(int K) { return (size_t)608 * K; }

void colsumsq(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *out, float *scratch) {
  if (K <= 0) return;
  const int nchunk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(608, (R + 63) / 64)));
  const int64_t rows_per = (R + nchunk - 1) / nchunk;
  if (K <= 256 && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0)
    colsumsq_partial_kernel<<<nchunk, 256, 0, st>>>(R, K, X, ld, rows_per, scratch);
  else
    colsumsq_partial_wide_kernel<<<nchunk, 128, 0, st>>>(R, K, X, ld, rows_per, scratch);
  MC_CHECK_LAUNCH();
  colsumsq_reduce_kernel<<<K, 256, 0, st>>>(K, nchunk, scratch, out);
  MC_CHECK_LAUNCH();
}

void select_cols(cudaStream_t st, int K, const float *W, int ld_w, int ncols, int ncp, float *out) {
  const int64_t total = (int64_t)K * ncp;
  if (total <= 0) return;
  const int nb = static_cast<int>(std::min<int64_t>((total + 255) / 256, 1024));
  select_cols_kernel<<<nb, 256, 0, st>>>(K, W, ld_w, ncols, ncp, out);
  MC_CHECK_LAUNCH();
}

// tile edge of the pipelined kernel: one T x T tile for narrow panels,
// 64 x 64 tiles (a grid of them) for wider ones
static int tn_small_tile(int K1, int K2) {
  const int k = std::max(K1, K2);
  return k <= 16 ? 16 : (k <= 32 ? 32 : 64);
}
struct TnPlan {
  int T, K1p, K2p, tiles_i, tiles_j, nsplit;
  int64_t rps;
};
static TnPlan tn_plan(int64_t R, int K1, int K2, bool sym) {
  TnPlan pl{};
  pl.T = tn_small_tile(K1, K2);
  pl.K1p = (int)round_up(std::max(K1, 1), pl.T);
  pl.K2p = (int)round_up(std::max(K2, 1), pl.T);
  pl.tiles_i = pl.K1p / pl.T;
  pl.tiles_j = pl.K2p / pl.T;
  const int active = sym ? pl.tiles_i * (pl.tiles_i + 1) / 2 : pl.tiles_i * pl.tiles_j;
  const int64_t want = std::max<int64_t>(1, (304 + active - 1) / active);
  const int64_t ns = std::max<int64_t>(1, std::min<int64_t>(want, (R + 63) / 64));
  pl.rps = round_up((R + ns - 1) / ns, 64);
  pl.nsplit = static_cast<int>((R + pl.rps - 1) / pl.rps);
  return pl;
}

size_t gemm_tn_scratch_floats(int64_t R, int K1, int K2) {
  // the largest plan over sym / non-sym (sym has fewer active tiles, more splits)
  // and over the tensor-core kernel
  const TnPlan a = tn_plan(R, K1, K2, true), b = tn_plan(R, K1, K2, false);
  size_t n = std::max((size_t)a.nsplit * a.K1p * a.K2p, (size_t)b.nsplit * b.K1p * b.K2p);
  if (K1 <= 256 && K2 <= 256) n = std::max(n, gemm_tn_tc_scratch_floats(R, K1, K2));
  return n;
}

// MC_TN_TC=0 keeps the SIMT kernels for X1^T X2.
bool use_tn_tc() {
  static const bool on = [] {
    const char *v = std::getenv("MC_TN_TC");
    return !(v && v[0] == '0');
  }();
  return on;
}

void gemm_tn_reduce_partials(cudaStream_t st, int K1, int K2, int nsplit, const float *partial, int K1p, int K2p,
                             float *C, int ld_c, const int *skip) {
  const int64_t total = (int64_t)K1 * K2;
  const int nb = static_cast<int>(std::min<int64_t>((total + 31) / 32, 152 * 8));
  launch_pdl(gemm_tn_reduce_kernel, dim3(nb), dim3(256), 0, st, K1, K2, nsplit, static_cast<const float *>(partial), K1p,
             K2p, false, 4, C, ld_c, skip);
  MC_CHECK_LAUNCH();
}

template <int T>
static void launch_tn_small(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y,
                            int ld_y, bool symg, bool same, float *partial, const TnPlan &pl, const int *skip) {
  const size_t smem = TnSmall<T>::smem_bytes(same && pl.tiles_i * pl.tiles_j == 1);
  // the attribute is per kernel and process-wide: always set the largest size
  // any call needs, so concurrent callers on other threads never lower it
  smem_attr(gemm_tn_small_kernel<T>, (int)TnSmall<T>::smem_bytes(false));
  dim3 grid((unsigned)pl.nsplit, (unsigned)(pl.tiles_i * pl.tiles_j));
  gemm_tn_small_kernel<T><<<grid, 256, smem, st>>>(R, K1, K2, X, ld_x, Y, ld_y, pl.rps, symg ? 1 : 0, same ? 1 : 0,
                                                   partial, pl.tiles_j, pl.K1p, pl.K2p, skip);
  MC_CHECK_LAUNCH();
}

void gemm_tn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y, int ld_y, float *C,
             int ld_c, bool sym, float *partial, const int *skip, int *err) {
  if (K1 <= 0 || K2 <= 0) return;
  if (use_tn_tc() && K2 > 16 && gemm_tn_tc_supported(R, K1, K2, X, ld_x, Y, ld_y)) {
    gemm_tn_tc(st, R, K1, K2, X, ld_x, Y, ld_y, C, ld_c, partial, err, skip);
    return;
  }
  gemm_tn_simt(st, R, K1, K2, X, ld_x, Y, ld_y, C, ld_c, partial, skip, sym);
}

void gemm_tn_simt(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y, int ld_y,
                  float *C, int ld_c, float *partial, const int *skip, bool sym) {
  if (K1 <= 0 || K2 <= 0) return;
  MC_REQUIRE(ld_x % 4 == 0 && ld_y % 4 == 0, "gemm_tn: leading dims must be multiples of 4");
  MC_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15u) == 0,
             "gemm_tn: panels must be 16-byte aligned");
  const bool same = (X == Y && ld_x == ld_y && K1 == K2);
  const bool symg = sym && same;  // only a true Gram skips the lower tiles
  const TnPlan pl = tn_plan(R, K1, K2, symg);
  if (pl.T == 16) launch_tn_small<16>(st, R, K1, K2, X, ld_x, Y, ld_y, symg, same, partial, pl, skip);
  else if (pl.T == 32) launch_tn_small<32>(st, R, K1, K2, X, ld_x, Y, ld_y, symg, same, partial, pl, skip);
  else launch_tn_small<64>(st, R, K1, K2, X, ld_x, Y, ld_y, symg, same, partial, pl, skip);
  const int64_t total = (int64_t)K1 * K2;
  const int nb = static_cast<int>(std::min<int64_t>((total + 31) / 32, 152 * 8));
  launch_pdl(gemm_tn_reduce_kernel, dim3(nb), dim3(256), 0, st, K1, K2, pl.nsplit, static_cast<const float *>(partial),
             pl.K1p, pl.K2p, symg, 4, C, ld_c, skip);
  MC_CHECK_LAUNCH();
}

// Panel products with more than 16 output columns run on the tensor cores
// (k_tc.cu) where the shape fits; MC_NN_TC=0 keeps the SIMT kernels.
bool use_nn_tc() {
  static const bool on = [] {
    const char *v = std::getenv("MC_NN_TC");
    return !(v && v[0] == '0');
  }();
  return on;
}

void gemm_nn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *W, int ld_w,
             const float *colscale, float alpha, float beta, float *Z, int ld_z, const int *copy_if, int *err) {
  if (R <= 0 || K2 <= 0) return;
  if (use_nn_tc() && K2 > 16 && gemm_nn_tc_supported(R, K1, K2, X, ld_x) && (!copy_if || K1 == K2)) {
    gemm_nn_tc(st, R, K1, K2, X, ld_x, W, ld_w, colscale, alpha, beta, Z, ld_z, err, copy_if);
    return;
  }
  gemm_nn_simt(st, R, K1, K2, X, ld_x, W, ld_w, colscale, alpha, beta, Z, ld_z, copy_if);
}

void gemm_nn_simt(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *W, int ld_w,
                  const float *colscale, float alpha, float beta, float *Z, int ld_z, const int *copy_if) {
  if (R <= 0 || K2 <= 0) return;
  MC_REQUIRE(!copy_if || (K1 == K2 && K2 > 16 && K1 <= 64 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0),
             "gemm_nn: the copy mode needs the small-factor kernel (16 < K1 == K2 <= 64, X 16-byte aligned)");
  MC_REQUIRE(ld_x % 4 == 0, "gemm_nn: ld_x must be a multiple of 4");
  // narrow outputs: a thread per row (the 64-column tiles would leave most threads idle)
  if (K2 <= 16 && K1 <= 1024) {
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((R + 255) / 256, 152 * 8)));
#define MC_NN_NARROW(KN)                                                                                              \
  gemm_nn_narrow_kernel<KN><<<grid, 256, sizeof(float) * (size_t)K1 * KN, st>>>(R, K1, K2, X, ld_x, W, ld_w, colscale, \
                                                                              alpha, beta, Z, ld_z)
    if (K2 <= 4) MC_NN_NARROW(4);
    else if (K2 <= 8) MC_NN_NARROW(8);
    else {
      smem_attr(gemm_nn_narrow_kernel<16>, (int)(sizeof(float) * 1024 * 16));
      MC_NN_NARROW(16);
    }
#undef MC_NN_NARROW
    MC_CHECK_LAUNCH();
    return;
  }
  // K1 <= 64: W in shared memory, X streamed; wider K1 (the projections
  // against many earlier blocks) measured faster on the tiled kernel below
  if (K1 <= 64 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
    const int64_t nch = (R + NNS_BM - 1) / NNS_BM;
    const int tiles = (K2 + 63) / 64;
    const int per_sm = 3;
    const int64_t want = std::max<int64_t>(1, (int64_t)152 * per_sm / tiles);
    const int64_t per = std::max<int64_t>(1, (nch + want - 1) / want);
    const dim3 grid(static_cast<unsigned>((nch + per - 1) / per), static_cast<unsigned>(tiles));
#define MC_NN_SMALL(KM)                                                                                              \
  smem_attr(gemm_nn_small_kernel<KM>, (int)NnSmall<KM>::smem);                                                \
  gemm_nn_small_kernel<KM><<<grid, 256, NnSmall<KM>::smem, st>>>(R, K1, K2, X, ld_x, W, ld_w, colscale, alpha, beta, \
                                                                 Z, ld_z, per, copy_if)
    MC_NN_SMALL(64);
#undef MC_NN_SMALL
    MC_CHECK_LAUNCH();
    return;
  }
  dim3 grid(static_cast<unsigned>((R + NN_BM - 1) / NN_BM), static_cast<unsigned>((K2 + NN_BN - 1) / NN_BN));
  gemm_nn_kernel<<<grid, 256, 0, st>>>(R, K1, K2, X, ld_x, W, ld_w, colscale, alpha, beta, Z, ld_z);
  MC_CHECK_LAUNCH();
}

// The largest |G - I| of a CholeskyQR pass's Gram that makes the next pass
// redundant (MC_SKIP3_TOL overrides).
float skip3_tol() {
  static const float v = [] {
    const char *e = std::getenv("MC_SKIP3_TOL");
    return e ? static_cast<float>(std::atof(e)) : 1e-2f;
  }();
  return v;
}

// The blocked factorisation for K <= 64 (MC_CHOL_BLK=0: the unblocked
// shared-memory kernel for every K <= 128).
bool use_chol_blk() {
  static const bool on = [] {
    const char *v = std::getenv("MC_CHOL_BLK");
    return !(v && v[0] == '0');
  }();
  return on;
}

void chol_inv(cudaStream_t st, int K, const float *G, int ld, float shift_rel, const float *ref_diag, float ref_tol,
              float *Rinv, const int *skip_if, int *set_skip) {
  MC_REQUIRE(K >= 1 && K <= 1024, "chol_inv: K out of range");
  if (K <= CB_K && use_chol_blk()) {
    launch_pdl(chol_inv_blk_kernel, dim3(1), dim3(CB_THREADS), 0, st, K, G, ld, shift_rel, ref_diag, ref_tol, Rinv,
               skip_if, set_skip, skip3_tol());
    MC_CHECK_LAUNCH();
    return;
  }
  if (K <= 128) {
    const int ls = (K % 2 == 0) ? K + 1 : K;
    const size_t need = sizeof(float) * (2 * (size_t)K * ls + K);
    constexpr size_t kMax = sizeof(float) * (2 * 128 * 129 + 128);  // K = 128; fixed for concurrent callers
    smem_attr(chol_inv_small_kernel, (int)kMax);
    const int threads = K <= 32 ? 256 : (K <= 64 ? 512 : 1024);
    chol_inv_small_kernel<<<1, threads, need, st>>>(K, G, ld, shift_rel, ref_diag, ref_tol, Rinv, skip_if, set_skip,
                                                    skip3_tol());
    MC_CHECK_LAUNCH();
    return;
  }
  MC_REQUIRE(!skip_if && !set_skip, "chol_inv: the pass flags need K <= 128");
  const size_t base = sizeof(float) * ((size_t)K * K + K);
  MC_REQUIRE(base <= 220 * 1024, "chol_inv: block too wide for shared memory");
  const bool x_sm = base + sizeof(float) * (size_t)K * K <= 220 * 1024;
  const size_t need = x_sm ? base + sizeof(float) * (size_t)K * K : base;
  smem_attr(chol_inv_kernel, (int)(220 * 1024));
  const int threads = K <= 128 ? 256 : 1024;
  chol_inv_kernel<<<1, threads, need, st>>>(K, G, ld, shift_rel, ref_diag, ref_tol, Rinv, x_sm ? 1 : 0);
  MC_CHECK_LAUNCH();
}

static int64_t on_stride(int K, int cols) {
  const int64_t KW = (K + 3) / 4 * 4, CW = (cols + 3) / 4 * 4;
  return std::max(CW * KW + KW, KW * KW);
}

size_t orth_narrow_scratch_floats(int64_t R, int K, int cols) {
  (void)R;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int64_t nb_max = (int64_t)std::max(sms, 1) * 4;
  const int64_t st = on_stride(K, cols);
  return (size_t)(nb_max * st + 2 * st + 64);
}

static size_t on_smem(int64_t rows_per, int K, int cols, bool q_smem) {
  const int KW = (K + 3) / 4 * 4, CW = (cols + 3) / 4 * 4;
  return sizeof(float) * ((size_t)rows_per * on_ld(K) + (q_smem ? (size_t)rows_per * on_ld(cols) : 0) +
                          (size_t)std::max(CW, KW) * KW + (size_t)ON_THREADS * 16 + 2 * (size_t)K * (K + 1) +
                          2 * (size_t)K);
}

bool orth_narrow(cudaStream_t st, int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out,
                 int ldo, bool use_ref, float shift_rel, float ref_tol, float *scratch) {
  if (K < 1 || K > ON_MAXK || R < 1 || cols < 0) return false;
  // 16-byte copies of whole rows: widths, leading dimensions and bases in multiples of 4 floats
  if (K % 4 || cols % 4 || ldx % 4 || ldo % 4 || (cols > 0 && ldq % 4)) return false;
  if (((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(out) |
        (cols > 0 ? reinterpret_cast<uintptr_t>(Qp) : 0)) & 15u) != 0)
    return false;
  if (((cols + 3) / 4) * ((K + 3) / 4) > ON_THREADS) return false;  // one 4 x 4 tile of Qp^T X per thread at most
  int dev = 0, sms = 0, coop = 0;
  MC_CUDA(cudaGetDevice(&dev));
  MC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop || sms <= 0) return false;
  const bool small = K <= 16;
  const void *fn = small ? reinterpret_cast<const void *>(orth_narrow_kernel<16>)
                         : reinterpret_cast<const void *>(orth_narrow_kernel<32>);
  smem_attr(fn, 220 * 1024);
  // CTAs: one to four per SM, at least 32 rows each, the rows and the
  // panel slices of a CTA in at most 220 KB / CTAs-per-SM of shared memory
  // (MC_ORTH_PER_SM caps the CTAs per SM)
  static const int cap = [] {
    const char *v = std::getenv("MC_ORTH_PER_SM");
    return v ? std::max(1, std::min(4, std::atoi(v))) : 4;
  }();
  // first with the rows of Qp staged too; when they do not fit, Qp is read
  // from global memory (it stays in L2 between the four passes over it)
  for (int attempt = 0; attempt < 2; ++attempt)
  for (int per_sm = cap; per_sm >= 1; --per_sm) {
    const bool q_smem = attempt == 0 && cols > 0;
    if (attempt == 1 && cols == 0) break;
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (R + 31) / 32));
    const int64_t rows_per = (R + nb - 1) / nb;
    const size_t smem = on_smem(rows_per, K, cols, q_smem);
    if (smem > (size_t)220 * 1024 / per_sm) continue;
    int occ = 0;
    MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, ON_THREADS, smem));
    if ((int64_t)occ * sms < nb) continue;
    const int64_t stride = on_stride(K, cols);
    OrthNarrowArgs a{};
    a.skip3 = skip3_tol();
    a.R = R;
    a.rows_per = rows_per;
    a.K = K;
    a.cols = cols;
    a.ldx = ldx;
    a.ldq = ldq;
    a.ldo = ldo;
    a.use_ref = use_ref ? 1 : 0;
    a.q_smem = q_smem ? 1 : 0;
    a.X = X;
    a.Qp = Qp;
    a.out = out;
    a.part = scratch;
    a.fin = scratch + nb * stride;
    a.shift_rel = shift_rel;
    a.ref_tol = ref_tol;
    void *args[] = {&a};
    MC_CUDA(cudaLaunchCooperativeKernel(fn, dim3((unsigned)nb), dim3(ON_THREADS), args, smem, st));
    count_launch();
    return true;
  }
  return false;
}

// ===================================================== allocation-free Gram ==
// mc_gram_noalloc is for callers that cannot allocate device memory while they
// call this library: code that runs between the begin and end of a CUDA stream
// capture (cudaMalloc is not allowed there), host callbacks and allocator
// hooks, and hosts that hand every byte of device memory to their own pool
// and forbid other allocations.  Its scratch (the per-split partial tiles of
// the Gram) is a file-scope device array of kNoAllocScratchFloats floats
// (4 MiB) that every GPU which loads this library holds until the process
// exits.
namespace {

constexpr size_t kNoAllocScratchFloats = size_t(1) << 20;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array for the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in for the device
// symbol, so the address is looked up once per device with that device
// current and cached.
float *noalloc_scratch_for_current_device(int *dev_out) {
  int dev = -1;
  MC_CUDA(cudaGetDevice(&dev));
  MC_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, "mc_gram_noalloc: device index above 63");
  *dev_out = dev;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    MC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<float *>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

}  // namespace mc

extern "C" mc_status mc_gram_noalloc(int64_t R, int K, const float *X, int ld, float *G, int ldg, void *stream) {
  using namespace mc;
  try {
    MC_REQUIRE(R >= 1 && K >= 1, "mc_gram_noalloc: R and K must be >= 1");
    MC_REQUIRE(X != nullptr && G != nullptr, "mc_gram_noalloc: null X or G");
    MC_REQUIRE(ld >= K && ld % 4 == 0, "mc_gram_noalloc: ld must be >= K and a multiple of 4");
    MC_REQUIRE(ldg >= K, "mc_gram_noalloc: ldg must be >= K");
    // the kernel reads rows of X as float4: the base must be 16-byte aligned
    MC_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15u) == 0, "mc_gram_noalloc: X must be 16-byte aligned");
    MC_REQUIRE(is_device_ptr(X) && is_device_ptr(G), "mc_gram_noalloc: X and G must be device pointers");
    const int Kp = static_cast<int>(round_up(K, TN_T));
    const size_t tile_floats = (size_t)Kp * Kp;
    if (tile_floats > kNoAllocScratchFloats)
      fail(MC_EINVAL, "mc_gram_noalloc: K = " + std::to_string(K) +
                          " needs more scratch than the fixed 4 MiB array holds (maximum K is 1024)");
    int dev = -1;
    float *scratch = noalloc_scratch_for_current_device(&dev);
    // as gemm_tn, with the number of row splits capped by the scratch size
    const int ti = Kp / TN_T;
    const int64_t want = std::max<int64_t>(1, (152 * 4 + ti * ti - 1) / (ti * ti));
    const int64_t by_rows = std::max<int64_t>(1, R / 256);
    const int64_t by_scratch = static_cast<int64_t>(kNoAllocScratchFloats / tile_floats);
    const int nsplit = static_cast<int>(std::min<int64_t>(std::min<int64_t>(std::min<int64_t>(want, by_rows), by_scratch), 1024));
    const int64_t rps = round_up((R + nsplit - 1) / nsplit, TN_RB);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid(ti * ti, nsplit);
    gemm_tn_kernel<<<grid, 256, 0, st>>>(R, K, K, X, ld, X, ld, rps, ti, true, scratch, Kp, Kp);
    MC_CHECK_LAUNCH();
    const int64_t total = (int64_t)K * K;
    const int nb = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 8));
    gemm_tn_reduce_kernel<<<nb, 256, 0, st>>>(K, K, nsplit, scratch, Kp, Kp, true, TN_T, G, ldg);
    MC_CHECK_LAUNCH();
    return MC_OK;
  } catch (const Err &e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc &) {
    set_error("mc_gram_noalloc: host allocation failed");
    return MC_ENOMEM;
  } catch (const std::exception &e) {
    set_error(std::string("mc_gram_noalloc: ") + e.what());
    return MC_EINTERNAL;
  }
}
