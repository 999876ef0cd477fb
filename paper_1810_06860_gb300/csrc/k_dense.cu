// Dense kernels of the rSVD hot path:
//   gemm_tn   C = X^T Y over the long dimension (Gram B = A^T A of eigSVD,
//             Alg. 3 step 1, and the block projections Q^T H)
//   gemm_nn   Z = beta Z + X W diag(s) (U = A V S^-1 of Alg. 3 step 4, the
//             Ritz vectors U = Q W of Alg. 5 step 11, H R^-1)
//   chol_inv  R^-1 of the Cholesky factor of a small Gram (block normalisation
//             standing in for lu() and orth(), which Lemmas 2-3 allow)
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

// Sum of the per-split partial tiles, in split order: a block covers 32
// outputs with 8 lanes of split groups each, then adds the 8 group sums in order.
__global__ void __launch_bounds__(256)
gemm_tn_reduce_kernel(int K1, int K2, int nsplit, const float *__restrict__ partial, int K1p, int K2p, bool sym,
                      float *__restrict__ C, int ld_c) {
  __shared__ float sh[8][33];
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
      if (sym && (j / TN_T) < (i / TN_T)) {  // tile below the diagonal: read the mirrored tile
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

// ===================================================== chol_inv (one warp) ==
// K <= 64: the same factorisation and inverse by a single warp (no block
// barriers).  Lane l owns rows l and l + 32 of the working matrices.
__global__ void __launch_bounds__(32)
chol_inv_warp_kernel(int K, const float *__restrict__ G, int ld, float shift_rel, const float *__restrict__ ref_diag,
                     float ref_tol, float *__restrict__ Rinv) {
  __shared__ float L[64][65];
  __shared__ float X[64][65];
  __shared__ float keepf[64];
  const int lane = threadIdx.x;
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
  const float shift = shift_rel * tr / K;
  const float drop = fmaxf(1e-30f, 1e-12f * mx) + shift;
  for (int i = lane; i < K; i += 32)
    keepf[i] = (ref_diag && !(G[(int64_t)i * ld + i] > ref_tol * ref_diag[i])) ? 0.f : 1.f;
  __syncwarp();
  for (int i = 0; i < K; ++i)
    for (int j = lane; j < K; j += 32) {
      const bool live = keepf[i] != 0.f && keepf[j] != 0.f;
      L[i][j] = (j <= i && live) ? G[(int64_t)i * ld + j] + (i == j ? shift : 0.f) : 0.f;
    }
  __syncwarp();
  for (int j = 0; j < K; ++j) {
    const float d = L[j][j];
    const bool keep = d > drop;
    const float inv = keep ? rsqrtf(d) : 0.f;
    __syncwarp();
    for (int i = j + 1 + lane; i < K; i += 32) L[i][j] *= inv;
    if (lane == 0) {
      L[j][j] = keep ? d * inv : 1.0f;
      if (!keep) keepf[j] = 0.f;
    }
    __syncwarp();
    if (keep) {
      // trailing update, the lanes spread over the rows' entries
      for (int a = j + 1; a < K; ++a) {
        const float la = L[a][j];
        for (int b = j + 1 + lane; b <= a; b += 32) L[a][b] -= la * L[b][j];
      }
      __syncwarp();
    }
  }
  // forward substitution, lane l solves columns l and l + 32; four partial
  // sums shorten the dependency chain
  for (int c = lane; c < K; c += 32) {
    const bool kc = keepf[c] != 0.f;
    for (int i = 0; i < K; ++i) {
      float x = 0.f;
      if (kc && i >= c && keepf[i] != 0.f) {
        float a0 = (i == c) ? 1.0f : 0.0f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int l = c;
        for (; l + 3 < i; l += 4) {
          a0 -= L[i][l] * X[l][c];
          a1 -= L[i][l + 1] * X[l + 1][c];
          a2 -= L[i][l + 2] * X[l + 2][c];
          a3 -= L[i][l + 3] * X[l + 3][c];
        }
        for (; l < i; ++l) a0 -= L[i][l] * X[l][c];
        x = ((a0 + a1) + (a2 + a3)) / L[i][i];
      }
      X[i][c] = x;
    }
  }
  __syncwarp();
  for (int t = lane; t < K * K; t += 32) {
    const int i = t / K, j = t % K;
    Rinv[t] = X[j][i];
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

}  // namespace

// ================================================================ launchers ==
size_t colsumsq_scratch_floats(int K) { return (size_t)608 * K; }

void colsumsq(cudaStream_t st, int64_t R, int K, const float *X, int ld, float *out, float *scratch) {
  if (K <= 0) return;
  const int nchunk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(608, (R + 63) / 64)));
  const int64_t rows_per = (R + nchunk - 1) / nchunk;
  colsumsq_partial_kernel<<<nchunk, 128, 0, st>>>(R, K, X, ld, rows_per, scratch);
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

static int tn_splits(int64_t R, int tiles) {
  const int64_t want = std::max<int64_t>(1, (152 * 2 + tiles - 1) / std::max(tiles, 1));
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
  const int nb = static_cast<int>(std::min<int64_t>((total + 31) / 32, 152 * 8));
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
  if (K <= 64) {
    chol_inv_warp_kernel<<<1, 32, 0, st>>>(K, G, ld, shift_rel, ref_diag, ref_tol, Rinv);
    MC_CHECK_LAUNCH();
    return;
  }
  const size_t base = sizeof(float) * ((size_t)K * K + K);
  MC_REQUIRE(base <= 220 * 1024, "chol_inv: block too wide for shared memory");
  const bool x_sm = base + sizeof(float) * (size_t)K * K <= 220 * 1024;
  const size_t need = x_sm ? base + sizeof(float) * (size_t)K * K : base;
  MC_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(220 * 1024)));
  const int threads = K <= 128 ? 256 : 1024;
  chol_inv_kernel<<<1, threads, need, st>>>(K, G, ld, shift_rel, ref_diag, ref_tol, Rinv, x_sm ? 1 : 0);
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
