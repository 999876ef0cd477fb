// Dense kernels of the rSVD hot path:
//   gemm_tn   C = X^T Y over the long dimension (Gram B = A^T A of eigSVD,
//             Alg. 3 step 1, and the block projections Q^T H)
//   gemm_nn   Z = beta Z + X W diag(s) (U = A V S^-1 of Alg. 3 step 4, the
//             Ritz vectors U = Q W of Alg. 5 step 11, H R^-1)
//   chol_inv  R^-1 of the Cholesky factor of a small Gram (block normalisation
//             standing in for lu() and orth(), which Lemmas 2-3 allow)
//   eig_topk  leading eigenpairs of a small symmetric matrix (Alg. 3 step 2)
// All float32; every reduction runs in a fixed order (deterministic).
#include "mc_common.cuh"

#include <algorithm>
#include <cfloat>
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

__global__ void gemm_tn_reduce_kernel(int K1, int K2, int nsplit, const float *__restrict__ partial, int K1p,
                                      int K2p, bool sym, float *__restrict__ C, int ld_c) {
  const int64_t total = (int64_t)K1 * K2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int i = static_cast<int>(t / K2), j = static_cast<int>(t % K2);
    int si = i, sj = j;
    if (sym && (j / TN_T) < (i / TN_T)) {  // tile below the diagonal: read the mirrored tile
      si = j;
      sj = i;
    }
    float acc = 0.f;
    for (int s = 0; s < nsplit; ++s) acc += partial[(int64_t)s * K1p * K2p + (int64_t)si * K2p + sj];
    C[(int64_t)i * ld_c + j] = acc;
  }
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

// =========================================================== chol_inv ======
// One block.  G + shift I = L L^T (right-looking), pivots below the drop
// threshold make their column "absent": its row of L^{-1} is zero, so the
// matching column of H R^{-1} is zero and the others ignore it.
__global__ void __launch_bounds__(1024)
chol_inv_kernel(int K, const float *__restrict__ G, int ld, float shift_rel, const float *__restrict__ ref_diag,
                float ref_tol, float *__restrict__ Rinv, float *__restrict__ gwork) {
  extern __shared__ float sh[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool in_smem = gwork == nullptr;
  float *L = in_smem ? sh : gwork;  // K x K (lower), then L^{-1}
  float *flags = in_smem ? sh + (size_t)K * K : sh;  // K floats: 1 = kept
  __shared__ float s_tr, s_max;
  if (tid == 0) {
    float tr = 0.f, mx = 0.f;
    for (int i = 0; i < K; ++i) {
      tr += G[(int64_t)i * ld + i];
      mx = fmaxf(mx, G[(int64_t)i * ld + i]);
    }
    s_tr = tr;
    s_max = mx;
  }
  __syncthreads();
  const float shift = shift_rel * s_tr / K;
  const float drop = fmaxf(1e-30f, 1e-12f * s_max) + shift;
  // a column that lost (almost) all of its norm to an earlier projection is
  // rounding noise: remove it before factoring
  for (int i = tid; i < K; i += nt)
    flags[i] = (ref_diag && !(G[(int64_t)i * ld + i] > ref_tol * ref_diag[i])) ? 0.f : 1.f;
  __syncthreads();
  for (int t = tid; t < K * K; t += nt) {
    const int i = t / K, j = t % K;
    const bool live = flags[i] != 0.f && flags[j] != 0.f;
    L[t] = (j <= i && live) ? G[(int64_t)i * ld + j] + (i == j ? shift : 0.f) : 0.f;
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    const float d = L[j * K + j];
    const bool keep = d > drop;
    __syncthreads();  // every thread has read the pivot before it is overwritten
    // column j
    if (keep) {
      const float ljj = sqrtf(d), inv = 1.0f / ljj;
      for (int i = j + 1 + tid; i < K; i += nt) L[i * K + j] *= inv;
      if (tid == 0) L[j * K + j] = ljj;
    } else {
      for (int i = j + 1 + tid; i < K; i += nt) L[i * K + j] = 0.f;
      if (tid == 0) L[j * K + j] = 1.0f;
    }
    __syncthreads();
    if (tid == 0) flags[j] = keep ? 1.f : 0.f;
    __syncthreads();
    if (keep) {
      // trailing update of the lower triangle: L[a][b] -= L[a][j] L[b][j], j < b <= a
      const int n = K - j - 1;
      const int64_t tot = (int64_t)n * (n + 1) / 2;
      for (int64_t f = tid; f < tot; f += nt) {
        int a = static_cast<int>((sqrtf(8.0f * f + 1.0f) - 1.0f) * 0.5f);
        while ((int64_t)(a + 1) * (a + 2) / 2 <= f) ++a;
        while ((int64_t)a * (a + 1) / 2 > f) --a;
        const int b = static_cast<int>(f - (int64_t)a * (a + 1) / 2);
        const int ga = j + 1 + a, gb = j + 1 + b;
        L[ga * K + gb] -= L[ga * K + j] * L[gb * K + j];
      }
    }
    __syncthreads();
  }
  // L^{-1} by columns: thread c solves L x = e_c (forward substitution).
  // Written to the strictly upper part as scratch, then transposed out.
  for (int c = tid; c < K; c += nt) {
    // x_i for i >= c stored in Rinv column c temporarily (global), row-major Rinv[i][c]
    for (int i = 0; i < K; ++i) Rinv[(int64_t)i * K + c] = 0.f;
    if (flags[c] == 0.f) continue;
    for (int i = c; i < K; ++i) {
      if (flags[i] == 0.f) continue;
      float acc = (i == c) ? 1.0f : 0.0f;
      for (int l = c; l < i; ++l) acc -= L[i * K + l] * Rinv[(int64_t)l * K + c];
      Rinv[(int64_t)i * K + c] = acc / L[i * K + i];
    }
  }
  __syncthreads();
  // Rinv currently holds L^{-1} (row-major).  R^{-1} = (L^{-1})^T: transpose in place.
  for (int t = tid; t < K * K; t += nt) {
    const int i = t / K, j = t % K;
    if (i < j) {
      const float a = Rinv[(int64_t)i * K + j], b = Rinv[(int64_t)j * K + i];
      Rinv[(int64_t)i * K + j] = b;
      Rinv[(int64_t)j * K + i] = a;
    }
  }
}

// =========================================================== eig_topk ======
// One block of 1024 threads.
//  1. Householder reduction of the symmetric matrix (packed lower triangle)
//     to tridiagonal form T = Q^T A Q.
//  2. Sturm-count multisection for the kw largest eigenvalues of T.
//  3. Inverse iteration (partially pivoted tridiagonal LU, three solves from
//     a fixed pseudo-random start) for their eigenvectors.
//  4. Classical Gram-Schmidt, applied twice, in descending-eigenvalue order.
//  5. Back-transformation W = Q Z by the stored reflectors.
constexpr int EIG_THREADS = 1024;
constexpr size_t EIG_SMEM = 220 * 1024;

__device__ __forceinline__ int64_t pk(int r, int c) { return (int64_t)r * (r + 1) / 2 + c; }  // r >= c

__device__ float block_sum(float v, float *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__global__ void __launch_bounds__(EIG_THREADS, 1)
eig_topk_kernel(int K, int kw, const float *__restrict__ A, int lda, float *__restrict__ lam_out,
                float *__restrict__ W, int ld_w, float *__restrict__ gw, int P_in_smem, int Z_in_smem) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float red[40];
  const int tid = threadIdx.x, nt = blockDim.x;
  // --- layout ---
  float *d = sm;                 // K
  float *e = d + K;              // K
  float *beta = e + K;           // K
  float *v = beta + K;           // K
  float *pw = v + K;             // K
  float *lam = pw + K;           // kw
  float *lo = lam + kw;          // kw
  float *hi = lo + kw;           // kw
  float *hvec = hi + kw;         // kw
  float *base = hvec + kw;
  base = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(base) + 15) & ~uintptr_t(15));
  const int64_t npk = (int64_t)K * (K + 1) / 2;
  float *P = P_in_smem ? base : gw;
  float *gnext = P_in_smem ? gw : gw + round_up(npk, 64);
  float *Z;
  if (Z_in_smem) {
    Z = P_in_smem ? base + round_up(npk, 4) : base;
  } else {
    Z = gnext;
    gnext += round_up((int64_t)K * kw, 64);
  }
  float *fa = gnext;                      // inverse-iteration factors, [i * kw + t]
  float *fb = fa + (int64_t)K * kw;
  float *fc = fb + (int64_t)K * kw;
  float *fl = fc + (int64_t)K * kw;
  float *fp = fl + (int64_t)K * kw;

  // ---- load the lower triangle ----
  for (int64_t f = tid; f < npk; f += nt) {
    int r = static_cast<int>((sqrtf(8.0f * f + 1.0f) - 1.0f) * 0.5f);
    while (pk(r + 1, 0) <= f) ++r;
    while (pk(r, 0) > f) --r;
    const int c = static_cast<int>(f - pk(r, 0));
    P[f] = A[(int64_t)r * lda + c];
  }
  __syncthreads();

  // ---- 1. tridiagonalisation ----
  for (int i = 0; i + 2 < K; ++i) {
    const int n = K - 1 - i;  // length of the column below the diagonal
    float part = 0.f;
    for (int a = 1 + tid; a < n; a += nt) {
      const float x = P[pk(i + 1 + a, i)];
      part += x * x;
    }
    const float sigma = block_sum(part, red);
    const float x0 = P[pk(i + 1, i)];
    const float dd = P[pk(i, i)];
    float bt = 0.f, alpha = x0;
    if (sigma > 0.f) {
      const float mu = sqrtf(x0 * x0 + sigma);
      alpha = x0 <= 0.f ? mu : -mu;
      const float v0 = x0 - alpha;
      bt = 2.0f / (v0 * v0 + sigma);
      __syncthreads();
      if (tid == 0) P[pk(i + 1, i)] = v0;
    }
    if (tid == 0) {
      d[i] = dd;
      e[i] = alpha;
      beta[i] = bt;
    }
    __syncthreads();
    if (bt == 0.f) continue;
    for (int a = tid; a < n; a += nt) v[a] = P[pk(i + 1 + a, i)];
    __syncthreads();
    // p = bt * A' v with A' the trailing block (rows/cols i+1..K-1)
    {
      int tpr = 32;
      while (tpr > 1 && (int64_t)n * tpr > nt) tpr >>= 1;
      const int rows_per_pass = nt / tpr;
      for (int a0 = 0; a0 < n; a0 += rows_per_pass) {
        const int a = a0 + tid / tpr, q = tid % tpr;
        float s = 0.f;
        if (a < n) {
          const int ra = i + 1 + a;
          for (int b = q; b < n; b += tpr) {
            const int rb = i + 1 + b;
            s += (rb <= ra ? P[pk(ra, rb)] : P[pk(rb, ra)]) * v[b];
          }
        }
        for (int off = tpr >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (a < n && q == 0) pw[a] = bt * s;
      }
    }
    __syncthreads();
    float vp = 0.f;
    for (int a = tid; a < n; a += nt) vp += v[a] * pw[a];
    const float c = 0.5f * bt * block_sum(vp, red);
    for (int a = tid; a < n; a += nt) pw[a] -= c * v[a];  // w
    __syncthreads();
    // A' -= v w^T + w v^T on the lower triangle: warp per row, interleaved
    {
      const int wid = tid >> 5, lane = tid & 31, nw = nt >> 5;
      for (int a = wid; a < n; a += nw) {
        const float va = v[a], wa = pw[a];
        float *row = P + pk(i + 1 + a, i + 1);
        for (int b = lane; b <= a; b += 32) row[b] -= va * pw[b] + wa * v[b];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (K >= 2) {
      d[K - 2] = P[pk(K - 2, K - 2)];
      e[K - 2] = P[pk(K - 1, K - 2)];
    }
    d[K - 1] = P[pk(K - 1, K - 1)];
    e[K - 1] = 0.f;
    if (K >= 2) beta[K - 2] = 0.f;
    beta[K - 1] = 0.f;
  }
  __syncthreads();

  // ---- 2. eigenvalues by multisection ----
  __shared__ float s_glo, s_ghi, s_pivmin;
  if (tid == 0) {
    float glo = FLT_MAX, ghi = -FLT_MAX, emax = 0.f;
    for (int a = 0; a < K; ++a) {
      const float r = (a > 0 ? fabsf(e[a - 1]) : 0.f) + (a + 1 < K ? fabsf(e[a]) : 0.f);
      glo = fminf(glo, d[a] - r);
      ghi = fmaxf(ghi, d[a] + r);
      if (a + 1 < K) emax = fmaxf(emax, e[a] * e[a]);
    }
    const float span = fmaxf(ghi - glo, fmaxf(fabsf(glo), fabsf(ghi)) * 1e-6f) + 1e-30f;
    s_glo = glo - 1e-3f * span;
    s_ghi = ghi + 1e-3f * span;
    s_pivmin = FLT_MIN * fmaxf(1.0f, emax);
  }
  __syncthreads();
  for (int t = tid; t < kw; t += nt) {
    lo[t] = s_glo;
    hi[t] = s_ghi;
  }
  __syncthreads();
  {
    int g = 32;
    while (g > 1 && kw * g > nt) g >>= 1;
    const int groups = nt / g;
    for (int t0 = 0; t0 < kw; t0 += groups) {
      const int t = t0 + tid / g, q = tid % g;
      const int target = K - 1 - t;  // ascending index of the t-th largest
      for (int it = 0; it < 64; ++it) {
        float l = 0.f, h = 0.f;
        bool active = t < kw;
        if (active) {
          l = lo[t];
          h = hi[t];
          if (h - l <= 2.0f * FLT_EPSILON * fmaxf(fabsf(l), fabsf(h)) + s_pivmin) active = false;
        }
        bool any = __any_sync(0xffffffffu, active);
        // all lanes of a group share t, so the group agrees on 'active'
        if (!__syncthreads_or(any)) break;
        int cnt = 0;
        const float x = l + (h - l) * (float)(q + 1) / (float)(g + 1);
        if (active) {
          float qq = d[0] - x;
          cnt = qq < 0.f;
          for (int a = 1; a < K; ++a) {
            if (fabsf(qq) < s_pivmin) qq = -s_pivmin;
            qq = d[a] - x - __fdividef(e[a - 1] * e[a - 1], qq);
            cnt += qq < 0.f;
          }
        }
        // new interval: the largest probe with count <= target and the smallest with count > target
        float nl = l, nh = h;
        for (int s = 0; s < g; ++s) {
          const float xs = __shfl_sync(0xffffffffu, x, (tid & 31) / g * g + s);
          const int cs = __shfl_sync(0xffffffffu, cnt, (tid & 31) / g * g + s);
          if (cs <= target) nl = fmaxf(nl, xs);
          else nh = fminf(nh, xs);
        }
        __syncthreads();
        if (active && q == 0) {
          lo[t] = nl;
          hi[t] = fmaxf(nl, nh);
        }
        __syncthreads();
      }
    }
  }
  for (int t = tid; t < kw; t += nt) lam[t] = 0.5f * (lo[t] + hi[t]);
  __syncthreads();

  // ---- 3. inverse iteration, one thread per eigenvalue ----
  __shared__ float s_tnorm;
  if (tid == 0) s_tnorm = fmaxf(fabsf(s_glo), fabsf(s_ghi));
  __syncthreads();
  for (int t = tid; t < kw; t += nt) {
    const float lm = lam[t];
    const float tiny = fmaxf(FLT_EPSILON * s_tnorm, FLT_MIN);
    // factor T - lm I = P L U (LAPACK gttrf scheme): fa = diag(U), fb = 1st super,
    // fc = 2nd super, fl = multipliers, fp = interchange flags
    float a_cur = d[0] - lm, b_cur = K > 1 ? e[0] : 0.f;
    for (int a = 0; a + 1 < K; ++a) {
      const float c = e[a];
      const float a_next = d[a + 1] - lm;
      const float b_next = a + 2 < K ? e[a + 1] : 0.f;
      float l, du2 = 0.f, na, nb;
      int piv;
      if (fabsf(a_cur) >= fabsf(c)) {
        if (a_cur == 0.f) a_cur = tiny;
        l = c / a_cur;
        na = a_next - l * b_cur;
        nb = b_next;
        piv = 0;
      } else {
        l = a_cur / c;
        const float new_a = c;
        const float new_b = a_next;
        na = b_cur - l * a_next;
        du2 = b_next;
        nb = -l * b_next;
        a_cur = new_a;
        b_cur = new_b;
        piv = 1;
      }
      const int64_t o = (int64_t)a * kw + t;
      fa[o] = a_cur;
      fb[o] = b_cur;
      fc[o] = du2;
      fl[o] = l;
      fp[o] = piv ? 1.f : 0.f;
      a_cur = na;
      b_cur = nb;
    }
    if (a_cur == 0.f) a_cur = tiny;
    fa[(int64_t)(K - 1) * kw + t] = a_cur;
    fb[(int64_t)(K - 1) * kw + t] = 0.f;
    fc[(int64_t)(K - 1) * kw + t] = 0.f;
    for (int a = 0; a < K; ++a) {
      const int64_t o = (int64_t)a * kw + t;
      if (fabsf(fa[o]) < tiny) fa[o] = copysignf(tiny, fa[o]);
    }
    // start vector
    for (int a = 0; a < K; ++a)
      Z[(int64_t)a * kw + t] = (float)(hash32((uint32_t)(a * 7919 + t * 104729 + 12345)) >> 8) * (1.0f / 16777216.0f) - 0.5f;
    for (int rep = 0; rep < 3; ++rep) {
      // forward: apply P and L^{-1}
      for (int a = 0; a + 1 < K; ++a) {
        const int64_t o = (int64_t)a * kw + t;
        float ya = Z[o], yb = Z[o + kw];
        if (fp[o] != 0.f) {
          const float tmp = ya;
          ya = yb;
          yb = tmp - fl[o] * ya;
        } else {
          yb -= fl[o] * ya;
        }
        Z[o] = ya;
        Z[o + kw] = yb;
      }
      // backward with U
      float x1 = 0.f, x2 = 0.f, nrm = 0.f;
      for (int a = K - 1; a >= 0; --a) {
        const int64_t o = (int64_t)a * kw + t;
        const float x = (Z[o] - fb[o] * x1 - fc[o] * x2) / fa[o];
        Z[o] = x;
        x2 = x1;
        x1 = x;
        nrm = fmaxf(nrm, fabsf(x));
      }
      const float sc = nrm > 0.f ? 1.0f / nrm : 1.0f;
      for (int a = 0; a < K; ++a) Z[(int64_t)a * kw + t] *= sc;
    }
  }
  __syncthreads();

  // ---- 4. Gram-Schmidt twice, column by column ----
  for (int j = 0; j < kw; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      // h[l] = z_l . z_j for l < j
      if (j > 0) {
        int tpc = 32;
        while (tpc > 1 && j * tpc > nt) tpc >>= 1;
        const int per = nt / tpc;
        for (int l0 = 0; l0 < j; l0 += per) {
          const int l = l0 + tid / tpc, q = tid % tpc;
          float s = 0.f;
          if (l < j)
            for (int a = q; a < K; a += tpc) s += Z[(int64_t)a * kw + l] * Z[(int64_t)a * kw + j];
          for (int off = tpc >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          if (l < j && q == 0) hvec[l] = s;
        }
        __syncthreads();
        for (int a = tid; a < K; a += nt) {
          float s = 0.f;
          for (int l = 0; l < j; ++l) s += Z[(int64_t)a * kw + l] * hvec[l];
          Z[(int64_t)a * kw + j] -= s;
        }
        __syncthreads();
      }
      float part = 0.f;
      for (int a = tid; a < K; a += nt) {
        const float z = Z[(int64_t)a * kw + j];
        part += z * z;
      }
      const float nrm2 = block_sum(part, red);
      const float sc = nrm2 > 0.f ? rsqrtf(nrm2) : 0.f;
      for (int a = tid; a < K; a += nt) Z[(int64_t)a * kw + j] *= sc;
      __syncthreads();
    }
  }

  // ---- 5. back-transformation: Z <- H_0 H_1 ... H_{K-3} Z ----
  for (int i = K - 3; i >= 0; --i) {
    const float bt = beta[i];
    if (bt == 0.f) continue;
    const int n = K - 1 - i;
    for (int a = tid; a < n; a += nt) v[a] = P[pk(i + 1 + a, i)];
    __syncthreads();
    int tpc = 32;
    while (tpc > 1 && kw * tpc > nt) tpc >>= 1;
    const int per = nt / tpc;
    for (int t0 = 0; t0 < kw; t0 += per) {
      const int t = t0 + tid / tpc, q = tid % tpc;
      float s = 0.f;
      if (t < kw)
        for (int a = q; a < n; a += tpc) s += v[a] * Z[(int64_t)(i + 1 + a) * kw + t];
      for (int off = tpc >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (t < kw && q == 0) hvec[t] = bt * s;
    }
    __syncthreads();
    for (int64_t f = tid; f < (int64_t)n * kw; f += nt) {
      const int a = static_cast<int>(f / kw), t = static_cast<int>(f % kw);
      Z[(int64_t)(i + 1 + a) * kw + t] -= v[a] * hvec[t];
    }
    __syncthreads();
  }

  // ---- outputs ----
  for (int t = tid; t < kw; t += nt) lam_out[t] = lam[t];
  for (int64_t f = tid; f < (int64_t)K * kw; f += nt) {
    const int a = static_cast<int>(f / kw), t = static_cast<int>(f % kw);
    W[(int64_t)a * ld_w + t] = Z[f];
  }
}

// Column sums of squares of X (R x K): per-chunk partials, then an ordered sum.
__global__ void colsumsq_partial_kernel(int64_t R, int K, const float *__restrict__ X, int ld, int64_t rows_per,
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

__global__ void colsumsq_reduce_kernel(int K, int nchunk, const float *__restrict__ part, float *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < nchunk; ++b) acc += part[(int64_t)b * K + c];
    out[c] = acc;
  }
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

}  // namespace

// ================================================================ launchers ==
size_t colsumsq_scratch_floats(int K) { return (size_t)608 * K; }

void colsumsq(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *out, float *scratch) {
  if (K <= 0) return;
  const int nchunk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(608, (R + 63) / 64)));
  const int64_t rows_per = (R + nchunk - 1) / nchunk;
  colsumsq_partial_kernel<<<nchunk, 128, 0, st>>>(R, K, X, ld, rows_per, scratch);
  MC_CHECK_LAUNCH();
  colsumsq_reduce_kernel<<<(K + 127) / 128, 128, 0, st>>>(K, nchunk, scratch, out);
  MC_CHECK_LAUNCH();
}

void select_cols(cudaStream_t st, int K, const float *W, int ld_w, int ncols, int ncp, float *out) {
  const int64_t total = (int64_t)K * ncp;
  if (total <= 0) return;
  const int nb = static_cast<int>(std::min<int64_t>((total + 255) / 256, 1024));
  select_cols_kernel<<<nb, 256, 0, st>>>(K, W, ld_w, ncols, ncp, out);
  MC_CHECK_LAUNCH();
}

static int tn_splits(int64_t R, int tiles) {
  const int64_t want = std::max<int64_t>(1, (152 * 4 + tiles - 1) / std::max(tiles, 1));
  const int64_t max_by_rows = std::max<int64_t>(1, R / 256);
  return static_cast<int>(std::min<int64_t>(std::min<int64_t>(want, max_by_rows), 1024));
}

size_t gemm_tn_scratch_floats(int64_t R, int K1, int K2) {
  const int K1p = (int)round_up(std::max(K1, 1), TN_T), K2p = (int)round_up(std::max(K2, 1), TN_T);
  const int tiles = (K1p / TN_T) * (K2p / TN_T);
  return (size_t)tn_splits(R, tiles) * K1p * K2p;
}

void gemm_tn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *Y, int ld_y, float *C,
             int ld_c, bool sym, float *partial) {
  if (K1 <= 0 || K2 <= 0) return;
  MC_REQUIRE(ld_x % 4 == 0 && ld_y % 4 == 0, "gemm_tn: leading dims must be multiples of 4");
  const int K1p = (int)round_up(K1, TN_T), K2p = (int)round_up(K2, TN_T);
  const int ti = K1p / TN_T, tj = K2p / TN_T;
  const int nsplit = tn_splits(R, ti * tj);
  const int64_t rps = round_up((R + nsplit - 1) / nsplit, TN_RB);
  dim3 grid(ti * tj, nsplit);
  gemm_tn_kernel<<<grid, 256, 0, st>>>(R, K1, K2, X, ld_x, Y, ld_y, rps, tj, sym, partial, K1p, K2p);
  MC_CHECK_LAUNCH();
  const int64_t total = (int64_t)K1 * K2;
  const int nb = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 8));
  gemm_tn_reduce_kernel<<<nb, 256, 0, st>>>(K1, K2, nsplit, partial, K1p, K2p, sym, C, ld_c);
  MC_CHECK_LAUNCH();
}

void gemm_nn(cudaStream_t st, int64_t R, int K1, int K2, const float *X, int ld_x, const float *W, int ld_w,
             const float *colscale, float alpha, float beta, float *Z, int ld_z) {
  if (R <= 0 || K2 <= 0) return;
  MC_REQUIRE(ld_x % 4 == 0, "gemm_nn: ld_x must be a multiple of 4");
  dim3 grid(static_cast<unsigned>((R + NN_BM - 1) / NN_BM), static_cast<unsigned>((K2 + NN_BN - 1) / NN_BN));
  gemm_nn_kernel<<<grid, 256, 0, st>>>(R, K1, K2, X, ld_x, W, ld_w, colscale, alpha, beta, Z, ld_z);
  MC_CHECK_LAUNCH();
}

void chol_inv(cudaStream_t st, int K, const float *G, int ld, float shift_rel, const float *ref_diag, float ref_tol,
              float *Rinv) {
  MC_REQUIRE(K >= 1 && K <= 1024, "chol_inv: K out of range");
  const size_t need = sizeof(float) * ((size_t)K * K + K);
  MC_REQUIRE(need <= 200 * 1024, "chol_inv: block too wide for shared memory");
  MC_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024)));
  chol_inv_kernel<<<1, 1024, need, st>>>(K, G, ld, shift_rel, ref_diag, ref_tol, Rinv, nullptr);
  MC_CHECK_LAUNCH();
}

static void eig_layout(int K, int kw, bool &P_sm, bool &Z_sm) {
  const size_t fixed = sizeof(float) * (5 * (size_t)K + 4 * (size_t)kw) + 64;
  const size_t p = sizeof(float) * round_up((int64_t)K * (K + 1) / 2, 4);
  const size_t z = sizeof(float) * (size_t)K * kw;
  P_sm = fixed + p <= EIG_SMEM;
  Z_sm = fixed + (P_sm ? p : 0) + z <= EIG_SMEM;
}

size_t eig_work_bytes(int K, int kw) {
  bool P_sm, Z_sm;
  eig_layout(K, kw, P_sm, Z_sm);
  size_t f = 0;
  if (!P_sm) f += round_up((int64_t)K * (K + 1) / 2, 64);
  if (!Z_sm) f += round_up((int64_t)K * kw, 64);
  f += 5 * (size_t)K * kw;
  return sizeof(float) * f + 256;
}

void eig_topk(cudaStream_t st, int K, int kw, const float *A, int lda, float *lam, float *W, int ld_w, void *work) {
  MC_REQUIRE(K >= 1 && K <= 1024 && kw >= 1 && kw <= K, "eig_topk: sizes out of range");
  bool P_sm, Z_sm;
  eig_layout(K, kw, P_sm, Z_sm);
  MC_CUDA(cudaFuncSetAttribute(eig_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EIG_SMEM));
  eig_topk_kernel<<<1, EIG_THREADS, EIG_SMEM, st>>>(K, kw, A, lda, lam, W, ld_w, static_cast<float *>(work), P_sm ? 1 : 0,
                                                    Z_sm ? 1 : 0);
  MC_CHECK_LAUNCH();
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
    gemm_tn_reduce_kernel<<<nb, 256, 0, st>>>(K, K, nsplit, scratch, Kp, Kp, true, G, ldg);
    MC_CHECK_LAUNCH();
    return MC_OK;
  } catch (const Err &e) {
    set_error(e.msg);
    return e.st;
  }
}
