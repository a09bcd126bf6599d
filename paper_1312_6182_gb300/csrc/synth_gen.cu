// gpspca_synth_spikes: seeded planted-spike matrices drawn on the device
// (the synthetic request inputs of the serving workload), so that no host
// RNG or host-to-device copy sits in a request's path.  Not part of the
// method: it produces inputs only.
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a
// counter-based generator: output = 10 rounds of multiply/xor mixing of a
// 4 x 32-bit counter under a 2 x 32-bit key, so every entry is computed
// independently from its own counter.  Normals by Box-Muller in float32.
// The counter assignment and the float32 arithmetic (no contractions) are the
// same as the host twin's (synth.counter_spikes), which regenerates any
// request's matrix; the two agree up to the last-ulp differences of the
// float32 log / sin / cos implementations.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "gpspca.h"
#include "plan.h"

namespace gpspca {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
constexpr int kSynthMaxK = 64;

struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1) {
  Philox4 c{{c0, c1, c2, c3}};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.v[0]), lo0 = kPhiloxM0 * c.v[0];
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.v[2]), lo1 = kPhiloxM1 * c.v[2];
    c = Philox4{{hi1 ^ c.v[1] ^ k0, lo1, hi0 ^ c.v[3] ^ k1, lo0}};
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// top 23 bits + 1/2, times 2^-23: a float32 in (0, 1), exact
__device__ __forceinline__ float uniform23(uint32_t w) {
  return __fmul_rn(__fadd_rn(static_cast<float>(w >> 9), 0.5f), 1.1920928955078125e-7f);
}

__device__ __forceinline__ void box_muller4(const Philox4& w, float z[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float u1 = uniform23(w.v[2 * h]), u2 = uniform23(w.v[2 * h + 1]);
    const float rad = sqrtf(__fmul_rn(-2.0f, logf(u1)));
    const float ang = __fmul_rn(6.2831855f, u2);
    z[2 * h] = __fmul_rn(rad, cosf(ang));
    z[2 * h + 1] = __fmul_rn(rad, sinf(ang));
  }
}

struct SynthArgs {
  void* At;
  int64_t p, n, ld;
  int k, bf16;
  float frac;
  uint32_t k0, k1;
  float coef[kSynthMaxK];
};

// One thread per (column i, row quad b): noise, plus the column's spike.
__global__ void synth_spikes_kernel(const SynthArgs a) {
  const int64_t P4 = (a.p + 3) / 4;
  const int64_t total = a.n * P4;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = q / P4;
    const uint32_t b = static_cast<uint32_t>(q - i * P4);
    const uint32_t ilo = static_cast<uint32_t>(i & 0xffffffff), ihi = static_cast<uint32_t>(i >> 32);
    float z[4];
    box_muller4(philox4x32_10(b, ilo, ihi, 0u, a.k0, a.k1), z);
    const Philox4 sw = philox4x32_10(ilo, ihi, 0u, 2u, a.k0, a.k1);
    int j = a.k;
    if (a.frac > 0.0f) {
      const float v = uniform23(sw.v[0]);
      j = static_cast<int>(floorf(__fdiv_rn(v, a.frac)));
    }
    if (j < a.k) {
      const float c = (sw.v[1] >> 31) ? -a.coef[j] : a.coef[j];
      float u[4];
      box_muller4(philox4x32_10(b, static_cast<uint32_t>(j), 0u, 1u, a.k0, a.k1), u);
#pragma unroll
      for (int e = 0; e < 4; ++e) z[e] = __fadd_rn(z[e], __fmul_rn(c, u[e]));
    }
    const int64_t r0 = 4 * static_cast<int64_t>(b);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (r0 + e < a.p) {
        const int64_t off = i * a.ld + r0 + e;
        if (a.bf16)
          static_cast<__nv_bfloat16*>(a.At)[off] = __float2bfloat16_rn(z[e]);
        else
          static_cast<float*>(a.At)[off] = z[e];
      }
    }
  }
}

}  // namespace gpspca

using namespace gpspca;

extern "C" int gpspca_synth_spikes(void* At, gpspca_dtype dtype, int64_t p, int64_t n, int64_t ld, int32_t k,
                                   const double* theta, double support_frac, uint64_t seed, void* cuda_stream) {
  if (!At && p * n > 0) return record_error(GPSPCA_EINVAL, "At is NULL");
  if (dtype != GPSPCA_F32 && dtype != GPSPCA_BF16)
    return record_error(GPSPCA_EINVAL, "gpspca_synth_spikes writes float32 or bfloat16");
  if (p < 0 || n < 0 || ld < p) return record_error(GPSPCA_EINVAL, "bad shape");
  if (k < 0 || k > kSynthMaxK || (k > 0 && !theta))
    return record_error(GPSPCA_EINVAL, "k must be in [0, 64] with k theta values");
  if (!(support_frac >= 0.0) || support_frac * k > 1.0 + 1e-12)
    return record_error(GPSPCA_EINVAL, "support_frac must be >= 0 with k * support_frac <= 1 (disjoint supports)");
  if (p == 0 || n == 0) return GPSPCA_OK;
  SynthArgs a{};
  a.At = At;
  a.p = p;
  a.n = n;
  a.ld = ld;
  a.k = k;
  a.bf16 = dtype == GPSPCA_BF16;
  a.frac = static_cast<float>(support_frac);
  a.k0 = static_cast<uint32_t>(seed & 0xffffffffu);
  a.k1 = static_cast<uint32_t>(seed >> 32);
  const double s = std::max(1.0, std::round(support_frac * static_cast<double>(n)));
  for (int j = 0; j < k; ++j) a.coef[j] = static_cast<float>(theta[j] / std::sqrt(s));
  const int64_t total = n * ((p + 3) / 4);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
  synth_spikes_kernel<<<static_cast<unsigned>(blocks), threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return record_error(GPSPCA_ECUDA, cudaGetErrorString(e));
  return GPSPCA_OK;
}
