// Gaussian test matrix Omega (Alg. 1/4/5 step 1) from a counter-based RNG.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw (SC'11): ten
// rounds of two 32x32->64-bit multiplications whose high halves are xored
// with the remaining counter words and the key; the key advances by the two
// Weyl increments between rounds.  Element (i, j) of Omega uses counter
// (i, col0 + j, call_lo, call_hi) and key (seed_lo, seed_hi), and maps the
// first two output words to one normal deviate by Box-Muller:
//   u1 = (x0 + 1) 2^-32 in (0, 1],  u2 = x1 2^-32,  z = sqrt(-2 ln u1) cos(2 pi u2).
// ln u1 is taken through log1pf when u1 > 1/2 so that u1 close to 1 keeps its
// relative accuracy in float32.
#include "mc_common.cuh"

namespace mc {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ float box_muller(uint32_t x0, uint32_t x1) {
  const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
  float lg;
  if (x0 >= 0x80000000u) {
    lg = log1pf(-static_cast<float>(~x0) * two_m32);  // 1 - u1 = (2^32 - 1 - x0) 2^-32
  } else {
    lg = logf((static_cast<float>(x0) + 1.0f) * two_m32);
  }
  return sqrtf(-2.0f * lg) * cospif(static_cast<float>(x1) * (2.0f * two_m32));
}

__global__ void omega_kernel(int64_t n, int k, int ld, uint32_t s_lo, uint32_t s_hi, uint32_t c_lo,
                             uint32_t c_hi, int col0, float *__restrict__ out,
                             uint32_t *__restrict__ words) {
  const int64_t total = n * ld;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld;
    const int j = static_cast<int>(t - i * ld);
    if (j >= k) {
      out[t] = 0.0f;
      continue;
    }
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(col0 + j),
                                             c_lo, c_hi),
                                  s_lo, s_hi);
    out[t] = box_muller(x.x, x.y);
    if (words) {
      words[2 * (i * k + j)] = x.x;
      words[2 * (i * k + j) + 1] = x.y;
    }
  }
}

}  // namespace

void launch_omega(cudaStream_t st, int64_t n, int k, int ld, uint64_t seed, uint64_t call_id, int col0,
                  float *out, uint32_t *words) {
  if (n <= 0 || ld <= 0) return;
  const int64_t total = n * ld;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  const int grid = static_cast<int>(blocks < 152 * 32 ? blocks : 152 * 32);
  omega_kernel<<<grid, threads, 0, st>>>(n, k, ld, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                                         static_cast<uint32_t>(call_id), static_cast<uint32_t>(call_id >> 32),
                                         col0, out, words);
  MC_CHECK_LAUNCH();
}

}  // namespace mc
