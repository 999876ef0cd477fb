// Small symmetric eigensolver: the kw largest eigenpairs of a K x K float32
// matrix, the eig() step of eigSVD (Alg. 3 step 2) applied to the Gram of
// B^T in rSVD-PI / rSVD-BKI (Alg. 4/5).
//
// Kernel 1 (one block of 1024 threads; 512 above K = 513): Householder
//   reduction to tridiagonal form T = Q^T A Q.  The packed lower triangle
//   lives in shared memory while it fits, else in global memory (L2); the
//   symmetric matrix-vector product reads every stored element once, row by
//   row (a warp per row, lanes along the row: coalesced, bank-conflict free),
//   keeping the transposed contributions in per-lane registers (8, 16 or 32
//   per lane for K up to 257, 513, 1025).  Four barriers per column.  The
//   reflectors go to global memory.
//   Sub-columns whose squared norm is below (eps max|A|)^2 are left as they
//   are (rounding residue of a rank-deficient Gram).
// Kernel 2 (one block of 1024 threads):
//   - Sturm-count multisection for the kw largest eigenvalues of T;
//   - inverse iteration, one thread per eigenvalue (pivoted tridiagonal LU,
//     three solves from a fixed pseudo-random start).  Eigenvalues within
//     1e-5 ||T|| of a neighbour form a cluster; their shifts are moved just
//     outside the cluster so that every direction of the cluster grows alike
//     and different starts give independent vectors;
//   - classical Gram-Schmidt applied twice (descending eigenvalue order);
//   - back-transformation by the reflectors, staged 16 at a time in shared
//     memory.
// Everything is float32; every reduction has a fixed order.
#include "mc_common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <cstring>

namespace mc {
namespace {

constexpr int EIG_THREADS = 1024;
constexpr int NW = EIG_THREADS / 32;
constexpr size_t EIG_SMEM = 220 * 1024;
constexpr int HV_CHUNK = 16;       // reflectors staged per back-transformation chunk
constexpr int ST_BISECT = 1, ST_INVIT = 2, ST_GS = 4, ST_BACK = 8, ST_ALL = 15;
constexpr int SPLIT_K = 256;       // above: inverse iteration and back-transformation on many CTAs
constexpr int SMALL_K = 128;       // up to here: 256-thread CTAs
constexpr int WY_MIN_KW = 16;      // blocked back-transformation from this many vectors

__device__ __forceinline__ int pk(int r, int c) { return r * (r + 1) / 2 + c; }  // r >= c

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// --------------------------------------------------------------- kernel 1 --
// PPR transposed-contribution registers per lane cover columns up to 32 PPR;
// THREADS threads (fewer for the widest case, to leave registers for them).
template <int NWT>
__device__ __forceinline__ float block_sum_n(float v, float *red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll 8
  for (int q = 0; q < NWT; ++q) t += red[q];
  return t;
}

// Householder tridiagonalisation for K <= 64: a thread per row of the full
// symmetric matrix, kept in shared memory with row stride 65 (a column read
// by the 32 threads of a warp hits 32 banks), two warps.  Each step forms
// the reflector of the column below the subdiagonal, p = beta A' v as one
// dot product per row, c = beta (v . p) / 2, w = p - c v, and
// A' -= v w^T + w v^T a row per thread: a handful of barriers per step
// instead of the warp-per-row reductions of the wider kernel.  Outputs
// (d, e, beta, reflectors in Hv) as eig_tridiag_kernel.
constexpr int TS_K = 64, TS_LD = TS_K + 1, TS_THREADS = 64;

__device__ __forceinline__ float ts_sum(float v, float (*red)[2], int &rb) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[rb][threadIdx.x >> 5] = v;
  __syncthreads();
  const float t = red[rb][0] + red[rb][1];
  rb ^= 1;
  return t;
}

__global__ void __launch_bounds__(TS_THREADS, 1)
eig_tridiag_small_kernel(int K, const float *__restrict__ A, int lda, float *__restrict__ g_d,
                         float *__restrict__ g_e, float *__restrict__ g_beta, float *__restrict__ Hv) {
  __shared__ float S[TS_K * TS_LD];
  __shared__ __align__(16) float vs[TS_K];
  __shared__ __align__(16) float ws[TS_K];
  __shared__ float red[2][2], s_amax[2];
  const int t = threadIdx.x;
  float amax = 0.f;
  for (int e = t; e < K * K; e += TS_THREADS) {
    const int r = e / K, c = e % K;
    const float x = r >= c ? A[(int64_t)r * lda + c] : A[(int64_t)c * lda + r];  // lower triangle read
    S[r * TS_LD + c] = x;
    amax = fmaxf(amax, fabsf(x));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((t & 31) == 0) s_amax[t >> 5] = amax;
  __syncthreads();
  amax = fmaxf(s_amax[0], s_amax[1]);
  // a sub-column below (eps |A|)^2 is rounding residue: not reflected (see eig_tridiag_kernel)
  const float sig_floor = fmaxf((FLT_EPSILON * amax) * (FLT_EPSILON * amax), 1e-37f);
  int rb = 0;
  for (int i = 0; i + 2 < K; ++i) {
    const int n = K - 1 - i;  // trailing rows and columns i + 1 .. K - 1
    const bool act = t < n;
    float *row = S + (i + 1 + t) * TS_LD + (i + 1);  // this thread's row of the trailing block
    const float x = act ? S[(i + 1 + t) * TS_LD + i] : 0.f;
    const float sigma = ts_sum(act && t >= 1 ? x * x : 0.f, red, rb);
    const float x0 = S[(i + 1) * TS_LD + i];
    float bt = 0.f, alpha = x0, v0 = 0.f;
    if (sigma > sig_floor) {
      const float mu = sqrtf(x0 * x0 + sigma);
      alpha = x0 <= 0.f ? mu : -mu;
      v0 = x0 - alpha;
      bt = 2.0f / (v0 * v0 + sigma);
    }
    const float vr = t == 0 ? v0 : x;
    if (t == 0) {
      g_d[i] = S[i * TS_LD + i];
      g_e[i] = alpha;
      g_beta[i] = bt;
    }
    if (act) Hv[(int64_t)i * K + t] = vr;
    if (bt == 0.f) continue;  // uniform: every thread has the same sigma
    if (act) vs[t] = vr;
    __syncthreads();
    // loads in batches of four ahead of their arithmetic: the compiler
    // cannot tell the row stores below from the vs / ws loads, so a plain
    // loop pays one shared-memory latency per element
    float p = 0.f;
    if (act) {
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
      int b = 0;
      for (; b + 4 <= n; b += 4) {
        const float r0 = row[b], r1 = row[b + 1], r2 = row[b + 2], r3 = row[b + 3];
        const float4 v4 = *reinterpret_cast<const float4 *>(vs + b);
        p0 = fmaf(r0, v4.x, p0);
        p1 = fmaf(r1, v4.y, p1);
        p2 = fmaf(r2, v4.z, p2);
        p3 = fmaf(r3, v4.w, p3);
      }
      for (; b < n; ++b) p0 = fmaf(row[b], vs[b], p0);
      p = ((p0 + p1) + (p2 + p3)) * bt;
    }
    const float c = 0.5f * bt * ts_sum(act ? vr * p : 0.f, red, rb);
    const float w = p - c * vr;
    if (act) ws[t] = w;
    __syncthreads();
    if (act) {
      int b = 0;
      for (; b + 4 <= n; b += 4) {
        const float r0 = row[b], r1 = row[b + 1], r2 = row[b + 2], r3 = row[b + 3];
        const float4 w4 = *reinterpret_cast<const float4 *>(ws + b);
        const float4 v4 = *reinterpret_cast<const float4 *>(vs + b);
        row[b] = r0 - (vr * w4.x + w * v4.x);
        row[b + 1] = r1 - (vr * w4.y + w * v4.y);
        row[b + 2] = r2 - (vr * w4.z + w * v4.z);
        row[b + 3] = r3 - (vr * w4.w + w * v4.w);
      }
      for (; b < n; ++b) row[b] -= vr * ws[b] + w * vs[b];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (K >= 2) {
      g_d[K - 2] = S[(K - 2) * TS_LD + (K - 2)];
      g_e[K - 2] = S[(K - 1) * TS_LD + (K - 2)];
      g_beta[K - 2] = 0.f;
    }
    g_d[K - 1] = S[(K - 1) * TS_LD + (K - 1)];
    g_e[K - 1] = 0.f;
    g_beta[K - 1] = 0.f;
  }
}

// Householder tridiagonalisation for 64 < K <= 256: a thread per row of
// the trailing matrix, the lower triangle packed in shared memory.  Row a's
// product with v reads its own contiguous part (columns <= a) and then walks
// down its column (entries (b, a), b > a: consecutive threads read
// consecutive words); the rank-2 update runs row-wise over the lower
// triangle.  Loads go four at a time ahead of their arithmetic.  Outputs as
// eig_tridiag_kernel.
constexpr int TM_K = 256, TM_THREADS = 256;

__device__ __forceinline__ float tm_sum(float v, float (*red)[TM_THREADS / 32], int &rb) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[rb][threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < TM_THREADS / 32; ++q) t += red[rb][q];
  rb ^= 1;
  return t;
}

__global__ void __launch_bounds__(TM_THREADS, 1)
eig_tridiag_mid_kernel(int K, const float *__restrict__ A, int lda, float *__restrict__ g_d,
                       float *__restrict__ g_e, float *__restrict__ g_beta, float *__restrict__ Hv) {
  extern __shared__ __align__(16) float P[];  // packed lower triangle, K (K + 1) / 2
  __shared__ __align__(16) float vs[TM_K];
  __shared__ __align__(16) float ws[TM_K];
  __shared__ float red[2][TM_THREADS / 32], s_amax[TM_THREADS / 32];
  const int t = threadIdx.x;
  float amax = 0.f;
  for (int e = t; e < K * K; e += TM_THREADS) {  // coalesced over A, lower triangle kept
    const int r = e / K, c = e % K;
    if (c > r) continue;
    const float x = A[(int64_t)r * lda + c];
    P[pk(r, c)] = x;
    amax = fmaxf(amax, fabsf(x));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((t & 31) == 0) s_amax[t >> 5] = amax;
  __syncthreads();
  amax = 0.f;
#pragma unroll
  for (int q = 0; q < TM_THREADS / 32; ++q) amax = fmaxf(amax, s_amax[q]);
  const float sig_floor = fmaxf((FLT_EPSILON * amax) * (FLT_EPSILON * amax), 1e-37f);
  int rb = 0;
  for (int i = 0; i + 2 < K; ++i) {
    const int n = K - 1 - i;
    const bool act = t < n;
    const int ga = i + 1 + t;  // this thread's row
    const float x = act ? P[pk(ga, i)] : 0.f;
    const float sigma = tm_sum(act && t >= 1 ? x * x : 0.f, red, rb);
    const float x0 = P[pk(i + 1, i)];
    float bt = 0.f, alpha = x0, v0 = 0.f;
    if (sigma > sig_floor) {
      const float mu = sqrtf(x0 * x0 + sigma);
      alpha = x0 <= 0.f ? mu : -mu;
      v0 = x0 - alpha;
      bt = 2.0f / (v0 * v0 + sigma);
    }
    const float vr = t == 0 ? v0 : x;
    if (t == 0) {
      g_d[i] = P[pk(i, i)];
      g_e[i] = alpha;
      g_beta[i] = bt;
    }
    if (act) Hv[(int64_t)i * K + t] = vr;
    if (bt == 0.f) continue;  // uniform
    if (act) vs[t] = vr;
    __syncthreads();
    float p = 0.f;
    float *row = P + pk(ga, i + 1);  // row ga, columns i + 1 .. ga
    if (act) {
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
      int b = 0;
      for (; b + 4 <= t + 1; b += 4) {
        const float r0 = row[b], r1 = row[b + 1], r2 = row[b + 2], r3 = row[b + 3];
        const float4 v4 = *reinterpret_cast<const float4 *>(vs + b);
        p0 = fmaf(r0, v4.x, p0);
        p1 = fmaf(r1, v4.y, p1);
        p2 = fmaf(r2, v4.z, p2);
        p3 = fmaf(r3, v4.w, p3);
      }
      for (; b <= t; ++b) p0 = fmaf(row[b], vs[b], p0);
      // column part: entries (i + 1 + b, ga) for b > t
      int idx = pk(i + 1 + b, ga);
      for (; b + 4 <= n; b += 4) {
        const int gb = i + 1 + b;
        const int i1 = idx + gb + 1, i2 = i1 + gb + 2, i3 = i2 + gb + 3;
        const float r0 = P[idx], r1 = P[i1], r2 = P[i2], r3 = P[i3];
        p0 = fmaf(r0, vs[b], p0);
        p1 = fmaf(r1, vs[b + 1], p1);
        p2 = fmaf(r2, vs[b + 2], p2);
        p3 = fmaf(r3, vs[b + 3], p3);
        idx = i3 + gb + 4;
      }
      for (; b < n; ++b) {
        p0 = fmaf(P[idx], vs[b], p0);
        idx += i + 2 + b;
      }
      p = ((p0 + p1) + (p2 + p3)) * bt;
    }
    const float c = 0.5f * bt * tm_sum(act ? vr * p : 0.f, red, rb);
    const float w = p - c * vr;
    if (act) ws[t] = w;
    __syncthreads();
    if (act) {
      int b = 0;
      for (; b + 4 <= t + 1; b += 4) {
        const float r0 = row[b], r1 = row[b + 1], r2 = row[b + 2], r3 = row[b + 3];
        const float4 w4 = *reinterpret_cast<const float4 *>(ws + b);
        const float4 v4 = *reinterpret_cast<const float4 *>(vs + b);
        row[b] = r0 - (vr * w4.x + w * v4.x);
        row[b + 1] = r1 - (vr * w4.y + w * v4.y);
        row[b + 2] = r2 - (vr * w4.z + w * v4.z);
        row[b + 3] = r3 - (vr * w4.w + w * v4.w);
      }
      for (; b <= t; ++b) row[b] -= vr * ws[b] + w * vs[b];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (K >= 2) {
      g_d[K - 2] = P[pk(K - 2, K - 2)];
      g_e[K - 2] = P[pk(K - 1, K - 2)];
      g_beta[K - 2] = 0.f;
    }
    g_d[K - 1] = P[pk(K - 1, K - 1)];
    g_e[K - 1] = 0.f;
    g_beta[K - 1] = 0.f;
  }
}

// Householder tridiagonalisation for 64 < K <= 256 with the lower triangle in
// registers (the fastest variant for this range).  512 threads: lane l holds
// the rows r = l + 32 a (a < 8), warp w the columns c = w + 16 b (b < 16);
// element (r, c) is kept when r >= c (at most 72 registers; the others hold
// zero).  Step j: the warp holding column j forms the reflector (warp
// reductions) and publishes v.  Every thread adds its elements' terms of
// p = beta A v twice over for the symmetric matrix: A(r, c) v(c) to row r
// (summed across the warps through shared memory) and, for r > c, A(r, c) v(r)
// to column c (summed across the lanes of the warp by a shuffle reduce-
// scatter).  A thread per row finishes p and the dot v.p, and every thread
// applies A -= v w^T + w v^T to its elements.  Three barriers per step; only
// columns of the trailing block (c > j) and blocks of 32 rows that reach
// into it are visited, warp-uniform tests.
// Outputs (d, e, beta, reflectors in Hv) as eig_tridiag_kernel.
constexpr int TR_K = 256, TR_THREADS = 512, TR_NW = TR_THREADS / 32;
constexpr int TR_A = 8, TR_B = 16;

// x[a][b] (column b of this thread's block) for a compile-time b
template <int B>
__device__ __forceinline__ void tr_col(const float (&x)[TR_A][TR_B], float (&col)[TR_A]) {
#pragma unroll
  for (int a = 0; a < TR_A; ++a) col[a] = (B <= 2 * a + 1) ? x[a][B] : 0.f;
}

__global__ void __launch_bounds__(TR_THREADS, 1)
eig_tridiag_reg_kernel(int K, const float *__restrict__ A, int lda, float *__restrict__ g_d,
                       float *__restrict__ g_e, float *__restrict__ g_beta, float *__restrict__ Hv) {
  pdl_wait();
  pdl_trigger();
  __shared__ float vs[2][TR_K], ps[2][TR_K], colp[TR_K];
  __shared__ float part[TR_NW][TR_K];
  __shared__ float dotp[2][TR_K / 32];
  __shared__ float s_beta[2], s_amax[TR_NW];
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const unsigned full = 0xffffffffu;
  for (int i = tid; i < TR_K; i += TR_THREADS) {
    vs[0][i] = 0.f;
    vs[1][i] = 0.f;
    ps[0][i] = 0.f;
    ps[1][i] = 0.f;
    colp[i] = 0.f;
  }
  // stored(a, b): b < 2a always; b == 2a when l >= w; b == 2a + 1 when l >= w + 16
  float x[TR_A][TR_B];
  float amax = 0.f;
#pragma unroll
  for (int a = 0; a < TR_A; ++a) {
#pragma unroll
    for (int b = 0; b < TR_B; ++b) {
      x[a][b] = 0.f;
      if (b > 2 * a + 1) continue;
      const int r = l + 32 * a, c = w + 16 * b;
      const bool keep = b < 2 * a || (b == 2 * a ? l >= w : l >= w + 16);
      if (keep && r < K && c < K) x[a][b] = A[(int64_t)r * lda + c];
      amax = fmaxf(amax, fabsf(x[a][b]));
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(full, amax, off));
  if (l == 0) s_amax[w] = amax;
  __syncthreads();
  amax = 0.f;
#pragma unroll
  for (int q = 0; q < TR_NW; ++q) amax = fmaxf(amax, s_amax[q]);
  const float sig_floor = fmaxf((FLT_EPSILON * amax) * (FLT_EPSILON * amax), 1e-37f);

  int buf = 0;
  for (int j = 0; j + 2 < K; ++j, buf ^= 1) {
    if (w == (j & 15)) {
      // column j (rows r = l + 32 a; zero where not stored, i.e. above the diagonal)
      float col[TR_A];
      switch (j >> 4) {
        case 0: tr_col<0>(x, col); break;
        case 1: tr_col<1>(x, col); break;
        case 2: tr_col<2>(x, col); break;
        case 3: tr_col<3>(x, col); break;
        case 4: tr_col<4>(x, col); break;
        case 5: tr_col<5>(x, col); break;
        case 6: tr_col<6>(x, col); break;
        case 7: tr_col<7>(x, col); break;
        case 8: tr_col<8>(x, col); break;
        case 9: tr_col<9>(x, col); break;
        case 10: tr_col<10>(x, col); break;
        case 11: tr_col<11>(x, col); break;
        case 12: tr_col<12>(x, col); break;
        case 13: tr_col<13>(x, col); break;
        case 14: tr_col<14>(x, col); break;
        default: tr_col<15>(x, col); break;
      }
      float sq = 0.f, mine_d = 0.f, mine_x0 = 0.f;
#pragma unroll
      for (int a = 0; a < TR_A; ++a) {
        const int r = l + 32 * a;
        if (r > j + 1) sq = fmaf(col[a], col[a], sq);
        if (a == (j >> 5)) mine_d = col[a];
        if (a == ((j + 1) >> 5)) mine_x0 = col[a];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(full, sq, off);
      const float dj = __shfl_sync(full, mine_d, j & 31);
      const float x0 = __shfl_sync(full, mine_x0, (j + 1) & 31);
      float bt = 0.f, alpha = x0, v0 = 0.f;
      if (sq > sig_floor) {
        const float mu = sqrtf(x0 * x0 + sq);
        alpha = x0 <= 0.f ? mu : -mu;
        v0 = x0 - alpha;
        bt = 2.0f / (v0 * v0 + sq);
      }
#pragma unroll
      for (int a = 0; a < TR_A; ++a) {
        const int r = l + 32 * a;
        if (r > j && r < K) {
          const float v = r == j + 1 ? v0 : col[a];
          vs[buf][r] = v;
          Hv[(int64_t)j * K + (r - j - 1)] = v;
        }
      }
      if (l == 0) {
        g_d[j] = dj;
        g_e[j] = alpha;
        g_beta[j] = bt;
        s_beta[buf] = bt;
      }
    }
    __syncthreads();
    const float bt = s_beta[buf];
    if (bt == 0.f) continue;  // uniform
    float vr[TR_A];
#pragma unroll
    for (int a = 0; a < TR_A; ++a) vr[a] = vs[buf][l + 32 * a];
    // ---- p = beta A v: row terms (rp) and transposed column terms (cp) ----
    float rp[TR_A], cp[TR_B];
#pragma unroll
    for (int a = 0; a < TR_A; ++a) rp[a] = 0.f;
#pragma unroll
    for (int b = 0; b < TR_B; ++b) {
      cp[b] = 0.f;
      const int c = w + 16 * b;
      if (c > j && c < K) {
        const float vc = vs[buf][c];
#pragma unroll
        for (int a = 0; a < TR_A; ++a) {
          if (b > 2 * a + 1) continue;
          if (32 * a + 31 <= j) continue;  // rows l + 32 a all outside the trailing block (warp-uniform)
          const float e = x[a][b];
          rp[a] = fmaf(e, vc, rp[a]);
          // the diagonal element (r == c) contributes once, to its row
          const bool diag = (b == 2 * a && l == w) || (b == 2 * a + 1 && l == w + 16);
          if (!diag) cp[b] = fmaf(e, vr[a], cp[b]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < TR_A; ++a) part[w][l + 32 * a] = rp[a];
    {
      // reduce-scatter of the 16 column sums over the 32 lanes: after the
      // levels on lane bits 4..1, lane l holds column b = l >> 1 (both lanes of a pair)
      float t8[8], t4[4], t2[2];
      const bool h4 = l & 16, h3 = l & 8, h2 = l & 4, h1 = l & 2;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float keep = h4 ? cp[i + 8] : cp[i], send = h4 ? cp[i] : cp[i + 8];
        t8[i] = keep + __shfl_xor_sync(full, send, 16);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float keep = h3 ? t8[i + 4] : t8[i], send = h3 ? t8[i] : t8[i + 4];
        t4[i] = keep + __shfl_xor_sync(full, send, 8);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float keep = h2 ? t4[i + 2] : t4[i], send = h2 ? t4[i] : t4[i + 2];
        t2[i] = keep + __shfl_xor_sync(full, send, 4);
      }
      const float keep = h1 ? t2[1] : t2[0], send = h1 ? t2[0] : t2[1];
      float t1 = keep + __shfl_xor_sync(full, send, 2);
      t1 += __shfl_xor_sync(full, t1, 1);
      const int c = w + 16 * (l >> 1);
      if ((l & 1) == 0 && c > j && c < K) colp[c] = t1;
    }
    __syncthreads();
    if (tid < TR_K) {
      const int r = tid;
      float pr = 0.f;
      if (r > j && r < K) {
        float s = colp[r];
#pragma unroll
        for (int q = 0; q < TR_NW; ++q) s += part[q][r];
        pr = bt * s;
        ps[buf][r] = pr;
      }
      float dv = pr * vs[buf][r];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) dv += __shfl_xor_sync(full, dv, off);
      if (l == 0) dotp[buf][tid >> 5] = dv;
    }
    __syncthreads();
    float dot = 0.f;
#pragma unroll
    for (int q = 0; q < TR_K / 32; ++q) dot += dotp[buf][q];
    const float cc = 0.5f * bt * dot;
    // ---- A -= v w^T + w v^T with w = p - c v ----
    float wr[TR_A];
#pragma unroll
    for (int a = 0; a < TR_A; ++a) wr[a] = ps[buf][l + 32 * a] - cc * vr[a];
#pragma unroll
    for (int b = 0; b < TR_B; ++b) {
      const int c = w + 16 * b;
      if (c > j && c < K) {
        const float vc = vs[buf][c], wc = ps[buf][c] - cc * vc;
#pragma unroll
        for (int a = 0; a < TR_A; ++a) {
          if (b > 2 * a + 1) continue;
          if (32 * a + 31 <= j) continue;  // rows that no later step reads
          const bool keep = b < 2 * a || (b == 2 * a ? l >= w : l >= w + 16);
          if (keep) x[a][b] -= vr[a] * wc + wr[a] * vc;
        }
      }
    }
  }
  // the last 2 x 2 block: each of its three elements is written by its owner
#pragma unroll
  for (int a = 0; a < TR_A; ++a) {
#pragma unroll
    for (int b = 0; b < TR_B; ++b) {
      if (b > 2 * a + 1) continue;
      const int r = l + 32 * a, c = w + 16 * b;
      if (r >= K || c >= K || r < c) continue;
      if (r == K - 2 && c == K - 2) g_d[K - 2] = x[a][b];
      if (r == K - 1 && c == K - 2) g_e[K - 2] = x[a][b];
      if (r == K - 1 && c == K - 1) g_d[K - 1] = x[a][b];
    }
  }
  if (tid == 0) {
    g_beta[K - 2] = 0.f;
    g_e[K - 1] = 0.f;
    g_beta[K - 1] = 0.f;
  }
}

template <int PPR, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
eig_tridiag_kernel(int K, const float *__restrict__ A, int lda, float *__restrict__ g_d, float *__restrict__ g_e,
                   float *__restrict__ g_beta, float *__restrict__ Hv, float *__restrict__ gP, int p_in_smem) {
  constexpr int NWT = THREADS / 32;
  constexpr int TMAX = 32 * PPR;
  extern __shared__ __align__(16) float sm[];
  __shared__ float red[2][32];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  float *vv = sm;                 // K
  float *pw = vv + K;             // K
  float *prow = pw + K;           // K
  float *dd = prow + K;           // K
  float *ppw = dd + K;            // NWT x TMAX
  float *P = p_in_smem ? ppw + NWT * TMAX : gP;

  float amax_part = 0.f;
  for (int r = wid; r < K; r += NWT)
    for (int c = lane; c <= r; c += 32) {
      const float x = A[(int64_t)r * lda + c];
      P[pk(r, c)] = x;
      amax_part = fmaxf(amax_part, fabsf(x));
    }
  // largest magnitude: a sub-column whose squared norm is below (eps |A|)^2 is
  // rounding residue (the trailing block of a rank-deficient Gram) and is not
  // reflected; reflecting it would divide by a denormal and overflow
  __shared__ float s_amax[NWT];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax_part = fmaxf(amax_part, __shfl_xor_sync(0xffffffffu, amax_part, off));
  if (lane == 0) s_amax[wid] = amax_part;
  __syncthreads();
  float amax = 0.f;
#pragma unroll 8
  for (int q = 0; q < NWT; ++q) amax = fmaxf(amax, s_amax[q]);
  const float sig_floor = fmaxf((FLT_EPSILON * amax) * (FLT_EPSILON * amax), 1e-37f);
  int rb = 0;  // alternating reduction buffer
  for (int i = 0; i + 2 < K; ++i) {
    const int n = K - 1 - i;
    float part = 0.f;
    for (int a = 1 + tid; a < n; a += THREADS) {
      const float x = P[pk(i + 1 + a, i)];
      vv[a] = x;
      part += x * x;
    }
    const float sigma = block_sum_n<NWT>(part, red[rb]);
    rb ^= 1;
    const float x0 = P[pk(i + 1, i)];
    float bt = 0.f, alpha = x0, v0 = 0.f;
    if (sigma > sig_floor) {
      const float mu = sqrtf(x0 * x0 + sigma);
      alpha = x0 <= 0.f ? mu : -mu;
      v0 = x0 - alpha;
      bt = 2.0f / (v0 * v0 + sigma);
    }
    if (tid == 0) {
      dd[i] = P[pk(i, i)];
      g_e[i] = alpha;
      g_beta[i] = bt;
      Hv[(int64_t)i * K] = v0;
    }
    for (int a = 1 + tid; a < n; a += THREADS) Hv[(int64_t)i * K + a] = vv[a];
    if (bt == 0.f) {
      __syncthreads();
      continue;
    }
    // p = A' v: warp per row a, lanes along the row (coalesced); the row's
    // transposed contributions A'(a,b) v_a (b < a) accumulate in pp[] of
    // lane b % 32, so the packed triangle is read once, by rows
    float pp[PPR];
#pragma unroll
    for (int j = 0; j < PPR; ++j) pp[j] = 0.f;
    for (int a = wid; a < n; a += NWT) {
      const float va = a == 0 ? v0 : vv[a];
      const float *row = P + pk(i + 1 + a, i + 1);
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < PPR; ++j) {
        const int b = lane + 32 * j;
        if (b <= a) {
          const float x = row[b];
          acc = fmaf(x, b == 0 ? v0 : vv[b], acc);
          if (b < a) pp[j] = fmaf(x, va, pp[j]);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) prow[a] = acc;
    }
#pragma unroll
    for (int j = 0; j < PPR; ++j) {
      const int b = lane + 32 * j;
      if (b < n) ppw[wid * TMAX + b] = pp[j];
    }
    __syncthreads();
    float vp = 0.f;
    for (int b = tid; b < n; b += THREADS) {
      float acc = prow[b];
#pragma unroll 8
      for (int w = 0; w < NWT; ++w) acc += ppw[w * TMAX + b];
      const float pb = bt * acc;
      pw[b] = pb;
      vp = fmaf(b == 0 ? v0 : vv[b], pb, vp);
    }
    const float c = 0.5f * bt * block_sum_n<NWT>(vp, red[rb]);
    rb ^= 1;
    // A' -= v w^T + w v^T with w = p - c v, lower triangle, warp per row
    for (int a = wid; a < n; a += NWT) {
      const float va = a == 0 ? v0 : vv[a];
      const float wa = pw[a] - c * va;
      float *row = P + pk(i + 1 + a, i + 1);
      for (int b = lane; b <= a; b += 32) {
        const float vb = b == 0 ? v0 : vv[b];
        const float wb = pw[b] - c * vb;
        row[b] -= va * wb + wa * vb;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (K >= 2) {
      dd[K - 2] = P[pk(K - 2, K - 2)];
      g_e[K - 2] = P[pk(K - 1, K - 2)];
      g_beta[K - 2] = 0.f;
    }
    dd[K - 1] = P[pk(K - 1, K - 1)];
    g_e[K - 1] = 0.f;
    g_beta[K - 1] = 0.f;
  }
  __syncthreads();
  for (int a = tid; a < K; a += THREADS) g_d[a] = dd[a];
}

// ------------------------------------------------- kernel 1, many CTAs --
// The same reduction for K > 256, where one SM's bandwidth to the matrix is
// the limit: a cooperative grid keeps the full symmetric matrix in global
// memory (L2).  Every CTA computes the Householder vector of the current
// column itself (same data, same order, same result), the warps of the grid
// share the rows of the trailing block for the product p = A v and for the
// rank-2 update, and two grid barriers per column separate the phases.  The
// update term v_r w_b + w_r v_b is formed with unfused roundings, so entry
// (r, b) and entry (b, r) stay bit-equal.
constexpr int CT_THREADS = 256;
__global__ void __launch_bounds__(CT_THREADS)
eig_tridiag_coop_kernel(int K, const float *__restrict__ A, int lda, float *__restrict__ Af, float *__restrict__ g_d,
                        float *__restrict__ g_e, float *__restrict__ g_beta, float *__restrict__ Hv,
                        float *__restrict__ g_p, float *__restrict__ g_part) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float ctm[];
  float *v = ctm;      // K
  float *w = v + K;    // K
  __shared__ float red[2][CT_THREADS / 32];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int nb = gridDim.x;
  const int64_t gt = (int64_t)blockIdx.x * CT_THREADS + tid, gstride = (int64_t)nb * CT_THREADS;
  // full symmetric copy from the lower triangle, and the largest magnitude
  float amax_part = 0.f;
  for (int64_t t = gt; t < (int64_t)K * K; t += gstride) {
    const int r = static_cast<int>(t / K), c = static_cast<int>(t % K);
    const float x = r >= c ? A[(int64_t)r * lda + c] : A[(int64_t)c * lda + r];
    Af[t] = x;
    amax_part = fmaxf(amax_part, fabsf(x));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax_part = fmaxf(amax_part, __shfl_xor_sync(0xffffffffu, amax_part, off));
  if (lane == 0) red[0][wid] = amax_part;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int q = 0; q < CT_THREADS / 32; ++q) m = fmaxf(m, red[0][q]);
    g_part[blockIdx.x] = m;
  }
  grid.sync();
  float amax = 0.f;
  for (int b = 0; b < nb; ++b) amax = fmaxf(amax, g_part[b]);
  const float sig_floor = fmaxf((FLT_EPSILON * amax) * (FLT_EPSILON * amax), 1e-37f);
  grid.sync();  // every CTA has read the maxima before the partials are reused
  const int gw = blockIdx.x * (CT_THREADS / 32) + wid, nwarps = nb * (CT_THREADS / 32);
  int rb = 0;
  for (int i = 0; i + 2 < K; ++i) {
    const int n = K - 1 - i;
    // Householder vector of column i (every CTA)
    float part = 0.f;
    for (int a = tid; a < n; a += CT_THREADS) {
      const float x = Af[(int64_t)(i + 1 + a) * K + i];
      v[a] = x;
      if (a >= 1) part += x * x;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) red[rb][wid] = part;
    __syncthreads();
    float sigma = 0.f;
#pragma unroll
    for (int q = 0; q < CT_THREADS / 32; ++q) sigma += red[rb][q];
    rb ^= 1;
    const float x0 = v[0];
    float bt = 0.f, alpha = x0, v0 = 0.f;
    if (sigma > sig_floor) {
      const float mu = sqrtf(x0 * x0 + sigma);
      alpha = x0 <= 0.f ? mu : -mu;
      v0 = x0 - alpha;
      bt = 2.0f / (v0 * v0 + sigma);
    }
    if (blockIdx.x == 0) {
      if (tid == 0) {
        g_d[i] = Af[(int64_t)i * K + i];
        g_e[i] = alpha;
        g_beta[i] = bt;
        Hv[(int64_t)i * K] = v0;
      }
      for (int a = 1 + tid; a < n; a += CT_THREADS) Hv[(int64_t)i * K + a] = v[a];
    }
    __syncthreads();
    if (tid == 0) v[0] = v0;
    __syncthreads();
    if (bt == 0.f) continue;  // uniform over the grid: no update, no barrier
    // p = bt A' v, a warp per row of the trailing block
    float vp = 0.f;
    for (int a = gw; a < n; a += nwarps) {
      const float *row = Af + (int64_t)(i + 1 + a) * K + (i + 1);
      float acc = 0.f;
      for (int b = lane; b < n; b += 32) acc = fmaf(row[b], v[b], acc);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      const float pa = bt * acc;
      if (lane == 0) g_p[a] = pa;
      vp = fmaf(v[a], pa, vp);  // the same in every lane of the warp
    }
    if (lane == 0) red[rb][wid] = vp;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int q = 0; q < CT_THREADS / 32; ++q) t += red[rb][q];
      g_part[blockIdx.x] = t;
    }
    rb ^= 1;
    grid.sync();
    float vps = 0.f;
    for (int b = 0; b < nb; ++b) vps += g_part[b];
    const float c = 0.5f * bt * vps;
    for (int a = tid; a < n; a += CT_THREADS) w[a] = g_p[a] - c * v[a];
    __syncthreads();
    // A' -= v w^T + w v^T, a warp per row
    for (int a = gw; a < n; a += nwarps) {
      float *row = Af + (int64_t)(i + 1 + a) * K + (i + 1);
      const float va = v[a], wa = w[a];
      for (int b = lane; b < n; b += 32) row[b] -= __fadd_rn(__fmul_rn(va, w[b]), __fmul_rn(wa, v[b]));
    }
    grid.sync();
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (K >= 2) {
      g_d[K - 2] = Af[(int64_t)(K - 2) * K + (K - 2)];
      g_e[K - 2] = Af[(int64_t)(K - 1) * K + (K - 2)];
      g_beta[K - 2] = 0.f;
    }
    g_d[K - 1] = Af[(int64_t)(K - 1) * K + (K - 1)];
    g_e[K - 1] = 0.f;
    g_beta[K - 1] = 0.f;
  }
}

// --------------------------------------------------------------- kernel 2 --
struct VecLayout {
  int ldz;         // odd row stride of Z
  int z_in_smem;   // Z in shared memory
  int batch;       // eigenvalues factored at once (factors in shared memory)
  int f_in_smem;
  int64_t g_z;     // float offsets into the global work area
  int64_t g_f;
};

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
eig_vectors_kernel(int K, int kw, const float *__restrict__ g_d, const float *__restrict__ g_e,
                   const float *__restrict__ g_beta, const float *__restrict__ Hv, float *__restrict__ lam_out,
                   float *__restrict__ W, int ld_w, float *__restrict__ gw, VecLayout lay, int stages) {
  constexpr int NWV = THREADS / 32;
  extern __shared__ __align__(16) float sm[];
  __shared__ float red[2][32];
  __shared__ float s_glo, s_ghi, s_pivmin;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int ldz = lay.ldz;
  float *d = sm;                  // K
  float *e = d + K;               // K
  float *beta = e + K;            // K
  float *lam = beta + K;          // kw
  float *lo = lam + kw;           // kw
  float *hi = lo + kw;            // kw
  float *hvec = hi + kw;          // kw
  float *part = hvec + kw;        // NW x 32
  float *hv = part + NWV * 32;     // HV_CHUNK x K
  float *wy = hv + (size_t)HV_CHUNK * K;  // blocked back-transformation: S, T (16 x 16 each), W (16 x kw)
  float *big = wy + 2 * HV_CHUNK * HV_CHUNK + (size_t)HV_CHUNK * kw;
  big = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(big) + 15) & ~uintptr_t(15));
  float *Z = lay.z_in_smem ? big : gw + lay.g_z;
  float *F = lay.f_in_smem ? (lay.z_in_smem ? big + (size_t)K * ldz : big) : gw + lay.g_f;
  const int B = lay.batch;

  for (int a = tid; a < K; a += THREADS) {
    d[a] = g_d[a];
    e[a] = g_e[a];
    beta[a] = g_beta[a];
  }
  __syncthreads();

  if (stages & ST_BISECT) {
  // ---- multisection ----
  if (tid < 32) {
    float glo = FLT_MAX, ghi = -FLT_MAX, emax = 0.f;
    for (int a = lane; a < K; a += 32) {
      const float r = (a > 0 ? fabsf(e[a - 1]) : 0.f) + (a + 1 < K ? fabsf(e[a]) : 0.f);
      glo = fminf(glo, d[a] - r);
      ghi = fmaxf(ghi, d[a] + r);
      if (a + 1 < K) emax = fmaxf(emax, e[a] * e[a]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, off));
      ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
      emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    }
    if (lane == 0) {
      const float span = fmaxf(ghi - glo, fmaxf(fabsf(glo), fabsf(ghi)) * 1e-6f) + 1e-30f;
      s_glo = glo - 1e-3f * span;
      s_ghi = ghi + 1e-3f * span;
      s_pivmin = FLT_MIN * fmaxf(1.0f, emax);
    }
  }
  __syncthreads();
  for (int t = tid; t < kw; t += THREADS) {
    lo[t] = s_glo;
    hi[t] = s_ghi;
  }
  __syncthreads();
  {
    int g = 32;
    while (g > 1 && kw * g > THREADS) g >>= 1;
    const int groups = THREADS / g;
    for (int t0 = 0; t0 < kw; t0 += groups) {
      const int t = t0 + tid / g, q = tid % g;
      const int target = K - 1 - t;
      for (int it = 0; it < 64; ++it) {
        float l = 0.f, h = 0.f;
        bool active = t < kw;
        if (active) {
          l = lo[t];
          h = hi[t];
          if (h - l <= 2.0f * FLT_EPSILON * fmaxf(fabsf(l), fabsf(h)) + s_pivmin) active = false;
        }
        if (!__syncthreads_or(active)) break;
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
        // the group's points increase with q: the new bracket is the highest
        // point whose count is <= target and the lowest whose count is above
        const unsigned gmask = (g == 32 ? 0xffffffffu : ((1u << g) - 1u)) << ((lane / g) * g);
        const unsigned below = __ballot_sync(0xffffffffu, cnt <= target) & gmask;
        const unsigned above = __ballot_sync(0xffffffffu, cnt > target) & gmask;
        const int lb = below ? 31 - __clz(below) : 0, la = above ? __ffs(above) - 1 : 0;
        const float xb = __shfl_sync(0xffffffffu, x, lb), xa = __shfl_sync(0xffffffffu, x, la);
        const float nl = below ? fmaxf(l, xb) : l;
        const float nh = above ? fminf(h, xa) : h;
        __syncthreads();
        if (active && q == 0) {
          lo[t] = nl;
          hi[t] = fmaxf(nl, nh);
        }
        __syncthreads();
      }
    }
  }
  for (int t = tid; t < kw; t += THREADS) lam[t] = 0.5f * (lo[t] + hi[t]);
  __syncthreads();

  for (int t = tid; t < kw; t += THREADS) lam_out[t] = lam[t];
  }  // ST_BISECT
  if (stages & ST_INVIT) {
  if (!(stages & ST_BISECT)) {
    for (int t = tid; t < kw; t += THREADS) lam[t] = lam_out[t];
    __syncthreads();
  }
  // ---- inverse iteration, B eigenvalues at a time ----
  const float tnorm = fmaxf(fabsf(s_glo), fabsf(s_ghi));
  const float tol_c = 1e-5f * tnorm;
  for (int t0 = 0; t0 < kw; t0 += B) {
    const int t = t0 + tid;
    if (tid < B && t < kw) {
      float *fa = F, *fb = F + (size_t)K * B, *fc = F + (size_t)2 * K * B, *fl = F + (size_t)3 * K * B;
      const bool clus = (t > 0 && lam[t - 1] - lam[t] <= tol_c) || (t + 1 < kw && lam[t] - lam[t + 1] <= tol_c);
      const float lm = lam[t] + (clus ? 2.0f * tol_c * (1.0f + 0.01f * (float)(t % 64)) : 0.f);
      const float tiny = fmaxf(FLT_EPSILON * tnorm, FLT_MIN);
      unsigned piv_bits[32];  // K <= 1024
#pragma unroll
      for (int q = 0; q < 32; ++q) piv_bits[q] = 0u;
      float a_cur = d[0] - lm, b_cur = K > 1 ? e[0] : 0.f;
      for (int a = 0; a + 1 < K; ++a) {
        const float cc = e[a];
        const float a_next = d[a + 1] - lm;
        const float b_next = a + 2 < K ? e[a + 1] : 0.f;
        float l, du2 = 0.f, na, nb;
        if (fabsf(a_cur) >= fabsf(cc)) {
          if (a_cur == 0.f) a_cur = tiny;
          l = __fdividef(cc, a_cur);
          na = a_next - l * b_cur;
          nb = b_next;
        } else {
          l = __fdividef(a_cur, cc);
          na = b_cur - l * a_next;
          du2 = b_next;
          nb = -l * b_next;
          a_cur = cc;
          b_cur = a_next;
          piv_bits[a >> 5] |= 1u << (a & 31);
        }
        const int o = a * B + tid;
        // the factors of inverse iteration need no correctly rounded division:
        // an error of a few ulps only perturbs the shift
        fa[o] = __fdividef(1.0f, fabsf(a_cur) < tiny ? copysignf(tiny, a_cur) : a_cur);
        fb[o] = b_cur;
        fc[o] = du2;
        fl[o] = l;
        a_cur = na;
        b_cur = nb;
      }
      {
        const int o = (K - 1) * B + tid;
        fa[o] = __fdividef(1.0f, fabsf(a_cur) < tiny ? copysignf(tiny, a_cur) : a_cur);
        fb[o] = 0.f;
        fc[o] = 0.f;
      }
      for (int a = 0; a < K; ++a)
        Z[(int64_t)a * ldz + t] =
            (float)(hash32((uint32_t)(a * 7919 + t * 104729 + 12345)) >> 8) * (1.0f / 16777216.0f) - 0.5f;
      for (int rep = 0; rep < 3; ++rep) {
        float ya = Z[t];
        for (int a = 0; a + 1 < K; ++a) {
          float yb = Z[(int64_t)(a + 1) * ldz + t];
          const float l = fl[a * B + tid];
          if (piv_bits[a >> 5] & (1u << (a & 31))) {
            const float tmp = ya;
            ya = yb;
            yb = tmp - l * ya;
          } else {
            yb -= l * ya;
          }
          Z[(int64_t)a * ldz + t] = ya;
          ya = yb;
        }
        float x1 = ya * fa[(K - 1) * B + tid], x2 = 0.f;
        Z[(int64_t)(K - 1) * ldz + t] = x1;
        float nrm = fabsf(x1);
        for (int a = K - 2; a >= 0; --a) {
          const int o = a * B + tid;
          const float xx = (Z[(int64_t)a * ldz + t] - fb[o] * x1 - fc[o] * x2) * fa[o];
          Z[(int64_t)a * ldz + t] = xx;
          x2 = x1;
          x1 = xx;
          nrm = fmaxf(nrm, fabsf(xx));
        }
        // an overflowed solve restarts from the scaled start vector
        const bool fin = nrm <= FLT_MAX;
        const float sc = fin ? (nrm > 0.f ? 1.0f / nrm : 1.0f) : 0.f;
        for (int a = 0; a < K; ++a) {
          const float z = Z[(int64_t)a * ldz + t];
          Z[(int64_t)a * ldz + t] =
              fin ? z * sc : (float)(hash32((uint32_t)(a * 7919 + t * 104729 + 12345)) >> 8) * (1.0f / 16777216.0f) - 0.5f;
        }
      }
    }
    __syncthreads();
  }

  }  // ST_INVIT
  if (stages & ST_GS) {
  // ---- Gram-Schmidt twice ----
  int rb = 0;
  for (int j = 0; j < kw; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      if (j > 0) {
        // h[l] = z_l . z_j: lanes along l, warps split the rows
        for (int c0 = 0; c0 < j; c0 += 32) {
          const int l = c0 + lane;
          float acc = 0.f;
          if (l < j)
            for (int a = wid; a < K; a += NWV) acc = fmaf(Z[(int64_t)a * ldz + l], Z[(int64_t)a * ldz + j], acc);
          part[wid * 32 + lane] = acc;
          __syncthreads();
          if (tid < 32 && c0 + tid < j) {
            float s = 0.f;
            for (int w = 0; w < NWV; ++w) s += part[w * 32 + tid];
            hvec[c0 + tid] = s;
          }
          __syncthreads();
        }
      }
      float nrm_part = 0.f;
      for (int a = tid; a < K; a += THREADS) {
        float z = Z[(int64_t)a * ldz + j];
        for (int l = 0; l < j; ++l) z = fmaf(-Z[(int64_t)a * ldz + l], hvec[l], z);
        Z[(int64_t)a * ldz + j] = z;
        nrm_part = fmaf(z, z, nrm_part);
      }
      const float nrm2 = block_sum_n<NWV>(nrm_part, red[rb]);
      rb ^= 1;
      const float sc = nrm2 > 0.f ? rsqrtf(nrm2) : 0.f;
      for (int a = tid; a < K; a += THREADS) Z[(int64_t)a * ldz + j] *= sc;
      __syncthreads();
    }
  }

  }  // ST_GS
  if (!(stages & ST_BACK)) return;
  // ---- back-transformation: Z <- H_0 H_1 ... H_{K-3} Z ----
  // up to one vector per warp: each warp applies the staged reflectors to its
  // vector with warp reductions (no block barrier per reflector); more
  // vectors: one reflector at a time across the block, and 16 at a time
  // (compact WY) when the vectors are many enough to amortise forming T
  if (kw <= NWV) {
  for (int top = K - 3; top >= 0; top -= HV_CHUNK) {
    const int lowi = max(0, top - HV_CHUNK + 1);
    for (int64_t f = tid; f < (int64_t)(top - lowi + 1) * K; f += THREADS) {
      const int r = static_cast<int>(f / K), a = static_cast<int>(f % K);
      hv[r * K + a] = Hv[(int64_t)(lowi + r) * K + a];
    }
    __syncthreads();
    if (wid < kw) {
      const int t = wid;
      for (int i = top; i >= lowi; --i) {
        const float bt = beta[i];
        if (bt == 0.f) continue;
        const int n = K - 1 - i;
        const float *v = hv + (i - lowi) * K;
        float acc = 0.f;
        for (int a = lane; a < n; a += 32) acc = fmaf(v[a], Z[(int64_t)(i + 1 + a) * ldz + t], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const float hb = bt * acc;
        for (int a = lane; a < n; a += 32) Z[(int64_t)(i + 1 + a) * ldz + t] -= v[a] * hb;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  } else if (kw < WY_MIN_KW) {
  for (int top = K - 3; top >= 0; top -= HV_CHUNK) {
    const int lowi = max(0, top - HV_CHUNK + 1);
    for (int64_t f = tid; f < (int64_t)(top - lowi + 1) * K; f += THREADS) {
      const int r = static_cast<int>(f / K), a = static_cast<int>(f % K);
      hv[r * K + a] = Hv[(int64_t)(lowi + r) * K + a];
    }
    __syncthreads();
    for (int i = top; i >= lowi; --i) {
      const float bt = beta[i];
      if (bt == 0.f) continue;
      const int n = K - 1 - i;
      const float *v = hv + (i - lowi) * K;
      for (int c0 = 0; c0 < kw; c0 += 32) {
        const int t = c0 + lane;
        float acc = 0.f;
        if (t < kw)
          for (int a = wid; a < n; a += NWV) acc = fmaf(v[a], Z[(int64_t)(i + 1 + a) * ldz + t], acc);
        part[wid * 32 + lane] = acc;
        __syncthreads();
        if (tid < 32 && c0 + tid < kw) {
          float s = 0.f;
          for (int w = 0; w < NWV; ++w) s += part[w * 32 + tid];
          hvec[c0 + tid] = bt * s;
        }
        __syncthreads();
      }
      for (int64_t f = tid; f < (int64_t)n * kw; f += THREADS) {
        const int a = static_cast<int>(f / kw), t = static_cast<int>(f % kw);
        Z[(int64_t)(i + 1 + a) * ldz + t] -= v[a] * hvec[t];
      }
      __syncthreads();
    }
  }

  } else {
  // H_lo ... H_hi = I - V T V^T (compact WY form, V's columns the reflectors in
  // ascending order, T upper triangular: T_jj = beta_j and column j above the
  // diagonal -beta_j T(0:j, 0:j) V(:, 0:j)^T v_j); then Z -= V (T (V^T Z)).
  float *S = wy, *T = wy + HV_CHUNK * HV_CHUNK, *Wb = wy + 2 * HV_CHUNK * HV_CHUNK;
  for (int top = K - 3; top >= 0; top -= HV_CHUNK) {
    const int lowi = max(0, top - HV_CHUNK + 1), nb = top - lowi + 1;
    // V (K x nb, column r = reflector lowi + r, zero above row lowi + r + 1)
    for (int64_t f = tid; f < (int64_t)nb * K; f += THREADS) {
      const int r = static_cast<int>(f / K), row = static_cast<int>(f % K);
      const int i = lowi + r;
      hv[r * K + row] = row >= i + 1 ? Hv[(int64_t)i * K + (row - i - 1)] : 0.f;
    }
    __syncthreads();
    // S = V^T V (nb x nb), a warp per entry
    for (int e = wid; e < nb * nb; e += NWV) {
      const int r = e / nb, c = e % nb;
      float acc = 0.f;
      if (c < r) acc = 0.f;
      else
        for (int row = lane; row < K; row += 32) acc = fmaf(hv[r * K + row], hv[c * K + row], acc);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) S[r * HV_CHUNK + c] = acc;  // upper triangle (r <= c) used
    }
    __syncthreads();
    // T, column by column (one warp; nb <= 16)
    if (wid == 0) {
      for (int j = 0; j < nb; ++j) {
        const float bj = beta[lowi + j];
        // T(i, j) for i < j: -bj * sum_{l=i}^{j-1} T(i, l) S(l, j)
        float tij = 0.f;
        if (lane < j) {
          for (int l = lane; l < j; ++l) tij = fmaf(T[lane * HV_CHUNK + l], S[l * HV_CHUNK + j], tij);
          tij *= -bj;
        }
        __syncwarp();
        if (lane < j) T[lane * HV_CHUNK + j] = tij;
        if (lane == j) T[j * HV_CHUNK + j] = bj;
        if (lane > j && lane < HV_CHUNK) T[lane * HV_CHUNK + j] = 0.f;
        __syncwarp();
      }
    }
    // W = V^T Z (nb x kw), a warp per entry
    for (int e = wid; e < nb * kw; e += NWV) {
      const int r = e / kw, t = e % kw;
      float acc = 0.f;
      for (int row = lowi + r + 1 + lane; row < K; row += 32) acc = fmaf(hv[r * K + row], Z[(int64_t)row * ldz + t], acc);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) Wb[r * kw + t] = acc;
    }
    __syncthreads();
    // W <- T W (in place by columns of W: each thread one column t)
    for (int t = tid; t < kw; t += THREADS) {
      float w[HV_CHUNK];
#pragma unroll
      for (int r = 0; r < HV_CHUNK; ++r) w[r] = r < nb ? Wb[r * kw + t] : 0.f;
#pragma unroll
      for (int r = 0; r < HV_CHUNK; ++r) {
        if (r < nb) {
          float acc = 0.f;
#pragma unroll
          for (int l = 0; l < HV_CHUNK; ++l)
            if (l >= r && l < nb) acc = fmaf(T[r * HV_CHUNK + l], w[l], acc);
          Wb[r * kw + t] = acc;
        }
      }
    }
    __syncthreads();
    // Z -= V W (rows lowi + 1 .. K-1)
    for (int64_t f = tid; f < (int64_t)(K - lowi - 1) * kw; f += THREADS) {
      const int row = lowi + 1 + static_cast<int>(f / kw), t = static_cast<int>(f % kw);
      float acc = 0.f;
      for (int r = 0; r < nb; ++r) acc = fmaf(hv[r * K + row], Wb[r * kw + t], acc);
      Z[(int64_t)row * ldz + t] -= acc;
    }
    __syncthreads();
  }

  }
  for (int64_t f = tid; f < (int64_t)K * kw; f += THREADS) {
    const int a = static_cast<int>(f / kw), t = static_cast<int>(f % kw);
    W[(int64_t)a * ld_w + t] = Z[(int64_t)a * ldz + t];
  }
}

// ---- wide matrices: the per-eigenvalue stages on many CTAs ------------------
// Inverse iteration for eigenvalue blockIdx.x (one thread; the LU factors and
// the vector in the CTA's shared memory), the same steps as in
// eig_vectors_kernel; the vector goes to Z (global, row stride ldz).
__global__ void __launch_bounds__(32)
eig_invit_kernel(int K, int kw, const float *__restrict__ g_d, const float *__restrict__ g_e,
                 const float *__restrict__ lam_g, float *__restrict__ Z, int ldz) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) float ism[];
  float *d = ism, *e = d + K, *fa = e + K, *fb = fa + K, *fc = fb + K, *fl = fc + K, *z = fl + K;
  const int lane = threadIdx.x, t = blockIdx.x;
  float glo = FLT_MAX, ghi = -FLT_MAX;
  for (int a = lane; a < K; a += 32) {
    d[a] = g_d[a];
    e[a] = g_e[a];
  }
  __syncwarp();
  for (int a = lane; a < K; a += 32) {
    const float r = (a > 0 ? fabsf(e[a - 1]) : 0.f) + (a + 1 < K ? fabsf(e[a]) : 0.f);
    glo = fminf(glo, d[a] - r);
    ghi = fmaxf(ghi, d[a] + r);
  }
  for (int off = 16; off > 0; off >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, off));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
  }
  const float span = fmaxf(ghi - glo, fmaxf(fabsf(glo), fabsf(ghi)) * 1e-6f) + 1e-30f;
  const float s_glo = glo - 1e-3f * span, s_ghi = ghi + 1e-3f * span;
  if (lane != 0) return;
  const float tnorm = fmaxf(fabsf(s_glo), fabsf(s_ghi));
  const float tol_c = 1e-5f * tnorm;
  const float lt = lam_g[t];
  const bool clus = (t > 0 && lam_g[t - 1] - lt <= tol_c) || (t + 1 < kw && lt - lam_g[t + 1] <= tol_c);
  const float lm = lt + (clus ? 2.0f * tol_c * (1.0f + 0.01f * (float)(t % 64)) : 0.f);
  const float tiny = fmaxf(FLT_EPSILON * tnorm, FLT_MIN);
  unsigned piv_bits[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) piv_bits[q] = 0u;
  float a_cur = d[0] - lm, b_cur = K > 1 ? e[0] : 0.f;
  for (int a = 0; a + 1 < K; ++a) {
    const float cc = e[a];
    const float a_next = d[a + 1] - lm;
    const float b_next = a + 2 < K ? e[a + 1] : 0.f;
    float l, du2 = 0.f, na, nb;
    if (fabsf(a_cur) >= fabsf(cc)) {
      if (a_cur == 0.f) a_cur = tiny;
      l = cc / a_cur;
      na = a_next - l * b_cur;
      nb = b_next;
    } else {
      l = a_cur / cc;
      na = b_cur - l * a_next;
      du2 = b_next;
      nb = -l * b_next;
      a_cur = cc;
      b_cur = a_next;
      piv_bits[a >> 5] |= 1u << (a & 31);
    }
    fa[a] = 1.0f / (fabsf(a_cur) < tiny ? copysignf(tiny, a_cur) : a_cur);
    fb[a] = b_cur;
    fc[a] = du2;
    fl[a] = l;
    a_cur = na;
    b_cur = nb;
  }
  fa[K - 1] = 1.0f / (fabsf(a_cur) < tiny ? copysignf(tiny, a_cur) : a_cur);
  fb[K - 1] = 0.f;
  fc[K - 1] = 0.f;
  for (int a = 0; a < K; ++a)
    z[a] = (float)(hash32((uint32_t)(a * 7919 + t * 104729 + 12345)) >> 8) * (1.0f / 16777216.0f) - 0.5f;
  for (int rep = 0; rep < 3; ++rep) {
    float ya = z[0];
    for (int a = 0; a + 1 < K; ++a) {
      float yb = z[a + 1];
      if (piv_bits[a >> 5] & (1u << (a & 31))) {
        const float tmp = ya;
        ya = yb;
        yb = tmp - fl[a] * ya;
      } else {
        yb -= fl[a] * ya;
      }
      z[a] = ya;
      ya = yb;
    }
    float x1 = ya * fa[K - 1], x2 = 0.f;
    z[K - 1] = x1;
    float nrm = fabsf(x1);
    for (int a = K - 2; a >= 0; --a) {
      const float xx = (z[a] - fb[a] * x1 - fc[a] * x2) * fa[a];
      z[a] = xx;
      x2 = x1;
      x1 = xx;
      nrm = fmaxf(nrm, fabsf(xx));
    }
    const bool fin = nrm <= FLT_MAX;
    const float sc = fin ? (nrm > 0.f ? 1.0f / nrm : 1.0f) : 0.f;
    for (int a = 0; a < K; ++a)
      z[a] = fin ? z[a] * sc
                 : (float)(hash32((uint32_t)(a * 7919 + t * 104729 + 12345)) >> 8) * (1.0f / 16777216.0f) - 0.5f;
  }
  for (int a = 0; a < K; ++a) Z[(int64_t)a * ldz + t] = z[a];
}

// Back-transformation of vector blockIdx.x by the reflectors (the vector in
// shared memory, each reflector read once from global memory), then W.
constexpr int BT_THREADS = 256;
__global__ void __launch_bounds__(BT_THREADS)
eig_backtr_kernel(int K, const float *__restrict__ g_beta, const float *__restrict__ Hv,
                  const float *__restrict__ Z, int ldz, float *__restrict__ W, int ld_w) {
  extern __shared__ __align__(16) float bsm[];
  __shared__ float red[2][BT_THREADS / 32];
  float *z = bsm;
  const int t = blockIdx.x, tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  for (int a = tid; a < K; a += BT_THREADS) z[a] = Z[(int64_t)a * ldz + t];
  __syncthreads();
  int rb = 0;
  for (int i = K - 3; i >= 0; --i) {
    const float bt = g_beta[i];
    if (bt == 0.f) continue;
    const int n = K - 1 - i;
    const float *v = Hv + (int64_t)i * K;
    float acc = 0.f;
    for (int a = tid; a < n; a += BT_THREADS) acc = fmaf(v[a], z[i + 1 + a], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) red[rb][wid] = acc;
    __syncthreads();
    float sdot = 0.f;
#pragma unroll
    for (int q = 0; q < BT_THREADS / 32; ++q) sdot += red[rb][q];
    rb ^= 1;
    const float h = bt * sdot;
    for (int a = tid; a < n; a += BT_THREADS) z[i + 1 + a] -= v[a] * h;
    __syncthreads();
  }
  for (int a = tid; a < K; a += BT_THREADS) W[(int64_t)a * ld_w + t] = z[a];
}

// ---- per-eigenvalue stages for 64 < K <= 256 --------------------------------
// Multisection for eigenvalue blockIdx.x (the t-th largest): one warp, 32
// Sturm counts per round (a lane per point) shrink the bracket 33-fold, from
// the Gershgorin interval to 2 ulp; the same counts and bracket rule as the
// one-CTA multisection.
__global__ void __launch_bounds__(32)
eig_bisect_kernel(int K, int kw, const float *__restrict__ g_d, const float *__restrict__ g_e,
                  float *__restrict__ lam_out) {
  pdl_wait();
  pdl_trigger();
  __shared__ float d[TR_K], e2[TR_K];
  const int lane = threadIdx.x, t = blockIdx.x;
  const unsigned full = 0xffffffffu;
  float glo = FLT_MAX, ghi = -FLT_MAX, emax = 0.f;
  for (int a = lane; a < K; a += 32) {
    const float ea = a + 1 < K ? g_e[a] : 0.f, eb = a > 0 ? g_e[a - 1] : 0.f;
    d[a] = g_d[a];
    e2[a] = ea * ea;
    const float r = fabsf(eb) + fabsf(ea);
    glo = fminf(glo, d[a] - r);
    ghi = fmaxf(ghi, d[a] + r);
    emax = fmaxf(emax, ea * ea);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(full, glo, off));
    ghi = fmaxf(ghi, __shfl_xor_sync(full, ghi, off));
    emax = fmaxf(emax, __shfl_xor_sync(full, emax, off));
  }
  __syncwarp();
  const float span = fmaxf(ghi - glo, fmaxf(fabsf(glo), fabsf(ghi)) * 1e-6f) + 1e-30f;
  float lo = glo - 1e-3f * span, hi = ghi + 1e-3f * span;
  const float pivmin = FLT_MIN * fmaxf(1.0f, emax);
  const int target = K - 1 - t;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.0f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + pivmin) break;  // uniform
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
    float qq = d[0] - x;
    int cnt = qq < 0.f;
    for (int a = 1; a < K; ++a) {
      if (fabsf(qq) < pivmin) qq = -pivmin;
      qq = d[a] - x - __fdividef(e2[a - 1], qq);
      cnt += qq < 0.f;
    }
    const unsigned below = __ballot_sync(full, cnt <= target);
    const unsigned above = __ballot_sync(full, cnt > target);
    const float xb = __shfl_sync(full, x, below ? 31 - __clz(below) : 0);
    const float xa = __shfl_sync(full, x, above ? __ffs(above) - 1 : 0);
    const float nl = below ? fmaxf(lo, xb) : lo;
    const float nh = above ? fminf(hi, xa) : hi;
    lo = nl;
    hi = fmaxf(nl, nh);
  }
  if (lane == 0) lam_out[t] = 0.5f * (lo + hi);
}

// Orthonormalisation of the inverse-iteration vectors Z (K x kw, kw <= 64):
// three CholeskyQR passes in shared memory (the first with a relative shift
// of 1e-6 of the mean diagonal), each Z <- Z R^{-1} with Z^T Z (+ shift) =
// R^T R.  Equal eigenvalues aside, the columns are already nearly orthogonal,
// so the Gram is well conditioned; a column whose pivot falls to the noise
// floor is zeroed.  256 threads: the Gram as eight warp partials (a warp per
// eighth of the rows, lanes along columns), the Cholesky factor in 16-column
// blocks (chol64_blocked, the unblocked loop's rounding), the solve a thread
// per row.
constexpr int EO_THREADS = 256, EO_KW = 64;
__global__ void __launch_bounds__(EO_THREADS, 1)
eig_orth_kernel(int K, int kw, float *__restrict__ Z, int ldz) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) float eo[];
  const int lz = kw | 1;                       // odd row stride
  float *Zs = eo;                              // K x lz
  float *P = Zs + (size_t)K * lz;              // 8 x kw x kw warp partials
  float *G = P + (size_t)8 * kw * kw;          // kw x (kw + 1)
  __shared__ float s_drop, s_pivok[EO_KW], rdg[EO_KW];
  __shared__ float Ls[64][65], linv[64], okf[64];  // the blocked Cholesky's R^T
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int lg = kw + 1;
  for (int f = tid; f < K * kw; f += EO_THREADS) {
    const int a = f / kw, c = f % kw;
    Zs[a * lz + c] = Z[(int64_t)a * ldz + c];
  }
  __syncthreads();
  for (int pass = 0; pass < 3; ++pass) {
    // partial Grams: warp wid over rows a = wid, wid + 8, ...; lane i (and i + 32)
    for (int j0 = 0; j0 < kw; j0 += 16) {
      float acc0[16], acc1[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc0[q] = acc1[q] = 0.f;
      for (int a = wid; a < K; a += 8) {
        const float *zr = Zs + a * lz;
        const float z0 = lane < kw ? zr[lane] : 0.f, z1 = lane + 32 < kw ? zr[lane + 32] : 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float zj = j0 + q < kw ? zr[j0 + q] : 0.f;
          acc0[q] = fmaf(z0, zj, acc0[q]);
          acc1[q] = fmaf(z1, zj, acc1[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (j0 + q >= kw) break;
        if (lane < kw) P[((size_t)wid * kw + lane) * kw + j0 + q] = acc0[q];
        if (lane + 32 < kw) P[((size_t)wid * kw + lane + 32) * kw + j0 + q] = acc1[q];
      }
    }
    __syncthreads();
    for (int f = tid; f < kw * kw; f += EO_THREADS) {
      const int i = f / kw, j = f % kw;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) s += P[((size_t)q * kw + i) * kw + j];
      G[i * lg + j] = s;
    }
    __syncthreads();
    if (tid == 0) {
      float tr = 0.f, mx = 0.f;
      for (int i = 0; i < kw; ++i) {
        tr += G[i * lg + i];
        mx = fmaxf(mx, G[i * lg + i]);
      }
      const float shift = pass == 0 ? 1e-6f * tr / (float)kw : 0.f;
      for (int i = 0; i < kw; ++i) G[i * lg + i] += shift;
      s_drop = fmaxf(1e-30f, 1e-12f * mx) + shift;
    }
    __syncthreads();
    // right-looking Cholesky G = R^T R: the strict upper triangle of G takes
    // R, its diagonal goes to rdg.  The blocked form (kw <= 64) on R^T, padded
    // with an identity block; its rounding is the unblocked loop's
    {
      for (int f = tid; f < 64 * 64; f += EO_THREADS) {
        const int a = f >> 6, b = f & 63;
        if (b <= a) Ls[a][b] = a < kw ? G[b * lg + a] : (a == b ? 1.f : 0.f);
      }
      if (tid < 64) okf[tid] = 1.f;
      __syncthreads();
      chol64_blocked(Ls, s_drop, linv, okf);
      for (int f = tid; f < kw * kw; f += EO_THREADS) {
        const int j = f / kw, c = f % kw;
        if (c > j) G[j * lg + c] = Ls[c][j];
      }
      if (tid < kw) {
        rdg[tid] = okf[tid] != 0.f ? Ls[tid][tid] * linv[tid] : 0.f;
        s_pivok[tid] = okf[tid];
      }
      __syncthreads();
    }
    // rows of Z: x R = z  (x_c = (z_c - sum_{k<c} x_k R[k][c]) / R[c][c]); dropped columns are zero
    for (int a = tid; a < K; a += EO_THREADS) {
      float *zr = Zs + a * lz;
      for (int c = 0; c < kw; ++c) {
        float s0 = zr[c], s1 = 0.f;
        int k = 0;
        for (; k + 1 < c; k += 2) {
          s0 = fmaf(-zr[k], G[k * lg + c], s0);
          s1 = fmaf(-zr[k + 1], G[(k + 1) * lg + c], s1);
        }
        if (k < c) s0 = fmaf(-zr[k], G[k * lg + c], s0);
        zr[c] = s_pivok[c] != 0.f ? (s0 + s1) / rdg[c] : 0.f;
      }
    }
    __syncthreads();
  }
  for (int f = tid; f < K * kw; f += EO_THREADS) {
    const int a = f / kw, c = f % kw;
    Z[(int64_t)a * ldz + c] = Zs[a * lz + c];
  }
}

size_t eig_orth_smem(int K, int kw) {
  return sizeof(float) * ((size_t)K * (kw | 1) + (size_t)8 * kw * kw + (size_t)kw * (kw + 1));
}

// Back-transformation W = H_0 H_1 ... H_{K-3} Z, a warp per vector: the
// vector lives in registers (K <= 256: 8 entries per lane), the reflectors of
// a chunk are staged in shared memory once for the CTA's eight warps, and each
// reflector costs the warp a dot product (shuffle reduction) and an update,
// without block barriers.
constexpr int BW_THREADS = 256, BW_CHUNK = 16;
__global__ void __launch_bounds__(BW_THREADS)
eig_backtr_warp_kernel(int K, int kw, const float *__restrict__ g_beta, const float *__restrict__ Hv,
                       const float *__restrict__ Z, int ldz, float *__restrict__ W, int ld_w) {
  pdl_wait();
  pdl_trigger();
  __shared__ __align__(16) float hv[BW_CHUNK][TR_K];
  __shared__ float bt[BW_CHUNK];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int t = blockIdx.x * (BW_THREADS / 32) + wid;
  const bool live = t < kw;
  const unsigned full = 0xffffffffu;
  float z[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int a = lane + 32 * q;
    z[q] = live && a < K ? Z[(int64_t)a * ldz + t] : 0.f;
  }
  for (int top = K - 3; top >= 0; top -= BW_CHUNK) {
    const int lowi = max(0, top - BW_CHUNK + 1);
    __syncthreads();
    // row i of the chunk: the reflector of step i aligned to global rows (zero at rows <= i)
    for (int f = tid; f < (top - lowi + 1) * TR_K; f += BW_THREADS) {
      const int r = f / TR_K, a = f % TR_K, i = lowi + r;
      hv[r][a] = (a > i && a < K) ? Hv[(int64_t)i * K + (a - i - 1)] : 0.f;
    }
    if (tid <= top - lowi) bt[tid] = g_beta[lowi + tid];
    __syncthreads();
    if (live) {
      for (int i = top; i >= lowi; --i) {
        const float b = bt[i - lowi];
        if (b == 0.f) continue;
        const float *v = hv[i - lowi];
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc = fmaf(v[lane + 32 * q], z[q], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(full, acc, off);
        const float h = b * acc;
#pragma unroll
        for (int q = 0; q < 8; ++q) z[q] = fmaf(-v[lane + 32 * q], h, z[q]);
      }
    }
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int a = lane + 32 * q;
      if (a < K) W[(int64_t)a * ld_w + t] = z[q];
    }
  }
}

// ------------------------------------------------------------------ plans --
// MC_EIG_TRI=packed keeps the packed shared-memory reduction for 64 < K <= 256.
bool tri_reg_on() {
  static const bool on = [] {
    const char *v = std::getenv("MC_EIG_TRI");
    return !(v && std::strcmp(v, "packed") == 0);
  }();
  return on;
}

// 64 < K <= 256 with at most 64 wanted pairs: multisection, inverse
// iteration and back-transformation on a CTA or warp per eigenvalue, the
// CholeskyQR orthonormalisation in one CTA (MC_EIG_MANY=0 keeps the one-CTA
// stages).
bool eig_many_cta(int K, int kw) {
  static const bool on = [] {
    const char *v = std::getenv("MC_EIG_MANY");
    return !(v && v[0] == '0');
  }();
  return on && K > TS_K && K <= TR_K && kw <= EO_KW;
}

// Matrices wider than this run the per-eigenvalue stages on many CTAs
// (MC_EIG_SPLIT_K overrides).
int split_k() {
  static const int v = [] {
    const char *e = std::getenv("MC_EIG_SPLIT_K");
    return e ? std::max(1, std::atoi(e)) : SPLIT_K;
  }();
  return v;
}

struct EigPlan {
  int coop;          // many-CTA reduction (K > 256, cooperative launch available)
  int64_t g_af, g_pv, g_part;
  int p_in_smem;
  size_t tri_smem;
  VecLayout vl;
  size_t vec_smem;
  int64_t g_d, g_e, g_beta, g_hv, g_p, g_total;  // float offsets in the work area
};

// Tridiagonalisation variant for K: registers per lane and threads.
struct TriCfg {
  int ppr, threads;
};
TriCfg tri_cfg(int K) {
  // the warp-per-row kernel serves K > 256 when the cooperative one cannot be
  // launched (K <= 256 has the row-per-thread kernels); rows of the trailing
  // matrix are at most K - 1 long: PPR x 32 >= K - 1
  if (K - 1 <= 256) return {8, 1024};
  if (K - 1 <= 512) return {16, 1024};
  return {32, 512};
}

EigPlan eig_plan(int K, int kw) {
  EigPlan pl{};
  const TriCfg tc = tri_cfg(K);
  const size_t tri_fixed = sizeof(float) * (4 * (size_t)K + (size_t)(tc.threads / 32) * 32 * tc.ppr);
  const size_t pbytes = sizeof(float) * ((size_t)K * (K + 1) / 2);
  pl.p_in_smem = tri_fixed + pbytes <= EIG_SMEM;
  pl.tri_smem = tri_fixed + (pl.p_in_smem ? pbytes : 0);
  int64_t off = 0;
  pl.g_d = off;
  off += round_up(K, 64);
  pl.g_e = off;
  off += round_up(K, 64);
  pl.g_beta = off;
  off += round_up(K, 64);
  pl.g_hv = off;
  off += round_up((int64_t)K * K, 64);
  pl.g_p = off;
  off += pl.p_in_smem ? 0 : round_up((int64_t)K * (K + 1) / 2, 64);
  pl.coop = K > 256;
  pl.g_af = off;
  off += pl.coop ? round_up((int64_t)K * K, 64) : 0;
  pl.g_pv = off;
  off += pl.coop ? round_up(K, 64) : 0;
  pl.g_part = off;
  off += pl.coop ? 1024 : 0;
  VecLayout vl{};
  vl.ldz = kw | 1;
  const bool split = K > split_k() || eig_many_cta(K, kw);
  const size_t vfixed =
      sizeof(float) * (3 * (size_t)K + 4 * (size_t)kw + NW * 32 + (size_t)HV_CHUNK * K + 2 * HV_CHUNK * HV_CHUNK +
                       (size_t)HV_CHUNK * kw) + 16;
  const size_t zbytes = sizeof(float) * (size_t)K * vl.ldz;
  vl.z_in_smem = !split && vfixed + zbytes <= EIG_SMEM;
  const size_t avail = EIG_SMEM - vfixed - (vl.z_in_smem ? zbytes : 0);
  int batch = static_cast<int>(std::min<size_t>(32, avail / (sizeof(float) * 4 * (size_t)K)));
  vl.f_in_smem = batch >= 8;
  if (!vl.f_in_smem) batch = 32;
  vl.batch = std::min(batch, std::max(kw, 1));
  vl.g_z = off;
  off += vl.z_in_smem ? 0 : round_up((int64_t)K * vl.ldz, 64);
  vl.g_f = off;
  off += vl.f_in_smem ? 0 : round_up((int64_t)4 * K * vl.batch, 64);
  pl.vl = vl;
  pl.vec_smem = vfixed + (vl.z_in_smem ? zbytes : 0) + (vl.f_in_smem ? sizeof(float) * 4 * (size_t)K * vl.batch : 0);
  pl.g_total = off;
  return pl;
}

}  // namespace

size_t eig_work_bytes(int K, int kw) { return sizeof(float) * (size_t)eig_plan(K, kw).g_total + 256; }

void eig_topk(cudaStream_t st, int K, int kw, const float *A, int lda, float *lam, float *W, int ld_w, void *work) {
  MC_REQUIRE(K >= 1 && K <= 1024 && kw >= 1 && kw <= K, "eig_topk: sizes out of range");
  const EigPlan pl = eig_plan(K, kw);
  MC_REQUIRE(pl.vec_smem <= EIG_SMEM && pl.tri_smem <= EIG_SMEM, "eig_topk: shared-memory plan does not fit");
  float *gw = static_cast<float *>(work);
  smem_attr(eig_vectors_kernel<256>, (int)EIG_SMEM);
  smem_attr(eig_vectors_kernel<1024>, (int)EIG_SMEM);
  const TriCfg tc = tri_cfg(K);
  bool done = false;
  if (pl.coop) {
    int dev = 0, sms = 0, coop = 0, occ = 0;
    MC_CUDA(cudaGetDevice(&dev));
    MC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    const size_t smem = sizeof(float) * 2 * (size_t)K;
    MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eig_tridiag_coop_kernel, CT_THREADS, smem));
    const int nb = std::min(std::min(sms, (K + 7) / 8), 1024);
    if (coop && occ >= 1 && nb >= 1) {
      float *Af = gw + pl.g_af, *gd = gw + pl.g_d, *ge = gw + pl.g_e, *gb = gw + pl.g_beta, *hv = gw + pl.g_hv;
      float *gp = gw + pl.g_pv, *gpart = gw + pl.g_part;
      int Kv = K, ldav = lda;
      const float *Av = A;
      void *args[] = {&Kv, &Av, &ldav, &Af, &gd, &ge, &gb, &hv, &gp, &gpart};
      MC_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(eig_tridiag_coop_kernel), dim3(nb),
                                          dim3(CT_THREADS), args, smem, st));
      count_launch();
      done = true;
    }
  }
#define MC_TRI_ARGS K, A, lda, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta, gw + pl.g_hv, gw + pl.g_p, pl.p_in_smem
  if (done) {
  } else if (K <= TS_K) {
    eig_tridiag_small_kernel<<<1, TS_THREADS, 0, st>>>(K, A, lda, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                       gw + pl.g_hv);
  } else if (K <= TR_K && tri_reg_on()) {
    launch_pdl(eig_tridiag_reg_kernel, dim3(1), dim3(TR_THREADS), 0, st, K, A, lda, gw + pl.g_d, gw + pl.g_e,
               gw + pl.g_beta, gw + pl.g_hv);
  } else if (K <= TM_K) {
    const size_t smem = sizeof(float) * ((size_t)K * (K + 1) / 2);
    smem_attr(eig_tridiag_mid_kernel, (int)(sizeof(float) * (TM_K * (TM_K + 1) / 2)));
    eig_tridiag_mid_kernel<<<1, TM_THREADS, smem, st>>>(K, A, lda, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                        gw + pl.g_hv);
  } else if (tc.ppr == 8) {
    smem_attr(eig_tridiag_kernel<8, 1024>, (int)EIG_SMEM);
    eig_tridiag_kernel<8, 1024><<<1, 1024, pl.tri_smem, st>>>(MC_TRI_ARGS);
  } else if (tc.ppr == 16) {
    smem_attr(eig_tridiag_kernel<16, 1024>, (int)EIG_SMEM);
    eig_tridiag_kernel<16, 1024><<<1, 1024, pl.tri_smem, st>>>(MC_TRI_ARGS);
  } else {
    smem_attr(eig_tridiag_kernel<32, 512>, (int)EIG_SMEM);
    eig_tridiag_kernel<32, 512><<<1, 512, pl.tri_smem, st>>>(MC_TRI_ARGS);
  }
#undef MC_TRI_ARGS
  MC_CHECK_LAUNCH();
  if (eig_many_cta(K, kw)) {
    float *Zg = gw + pl.vl.g_z;
    launch_pdl(eig_bisect_kernel, dim3(kw), dim3(32), 0, st, K, kw, gw + pl.g_d, gw + pl.g_e, lam);
    MC_CHECK_LAUNCH();
    const size_t ism = sizeof(float) * 7 * (size_t)K;
    smem_attr(eig_invit_kernel, (int)(7 * 4 * 1024));
    launch_pdl(eig_invit_kernel, dim3(kw), dim3(32), ism, st, K, kw, gw + pl.g_d, gw + pl.g_e, lam, Zg, pl.vl.ldz);
    MC_CHECK_LAUNCH();
    const size_t osm = eig_orth_smem(K, kw);
    smem_attr(eig_orth_kernel, (int)eig_orth_smem(TR_K, EO_KW));
    launch_pdl(eig_orth_kernel, dim3(1), dim3(EO_THREADS), osm, st, K, kw, Zg, pl.vl.ldz);
    MC_CHECK_LAUNCH();
    launch_pdl(eig_backtr_warp_kernel, dim3((kw + BW_THREADS / 32 - 1) / (BW_THREADS / 32)), dim3(BW_THREADS), 0, st, K,
               kw, gw + pl.g_beta, gw + pl.g_hv, Zg, pl.vl.ldz, W, ld_w);
    MC_CHECK_LAUNCH();
    return;
  }
  if (K <= split_k()) {
    // small matrices: 256 threads (cheaper barriers; 64 measured slower), else 1024
    if (K <= SMALL_K)
      eig_vectors_kernel<256><<<1, 256, pl.vec_smem, st>>>(K, kw, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                           gw + pl.g_hv, lam, W, ld_w, gw, pl.vl, ST_ALL);
    else
      eig_vectors_kernel<1024><<<1, 1024, pl.vec_smem, st>>>(K, kw, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                             gw + pl.g_hv, lam, W, ld_w, gw, pl.vl, ST_ALL);
    MC_CHECK_LAUNCH();
    return;
  }
  // wide: multisection (one CTA), inverse iteration (a CTA per eigenvalue),
  // Gram-Schmidt (one CTA), back-transformation (a CTA per vector)
  float *Zg = gw + pl.vl.g_z;
  eig_vectors_kernel<1024><<<1, 1024, pl.vec_smem, st>>>(K, kw, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                         gw + pl.g_hv, lam, W, ld_w, gw, pl.vl, ST_BISECT);
  MC_CHECK_LAUNCH();
  const size_t ism = sizeof(float) * 7 * (size_t)K;
  smem_attr(eig_invit_kernel, (int)(7 * 4 * 1024));
  eig_invit_kernel<<<kw, 32, ism, st>>>(K, kw, gw + pl.g_d, gw + pl.g_e, lam, Zg, pl.vl.ldz);
  MC_CHECK_LAUNCH();
  eig_vectors_kernel<1024><<<1, 1024, pl.vec_smem, st>>>(K, kw, gw + pl.g_d, gw + pl.g_e, gw + pl.g_beta,
                                                         gw + pl.g_hv, lam, W, ld_w, gw, pl.vl, ST_GS);
  MC_CHECK_LAUNCH();
  eig_backtr_kernel<<<kw, BT_THREADS, sizeof(float) * (size_t)K, st>>>(K, gw + pl.g_beta, gw + pl.g_hv, Zg,
                                                                       pl.vl.ldz, W, ld_w);
  MC_CHECK_LAUNCH();
}

}  // namespace mc
