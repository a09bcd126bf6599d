// Multi-component extraction by projection deflation (single-unit
// formulations of Table 1; the several components of Section 4.1, Fig. 3):
//
//   A_0 = A,   u_j = A_{j-1} z_j,   A_j = A_{j-1} - u_j z_j^T = A_{j-1} (I - z_j z_j^T),
//
// component j being the single-unit solve on A_{j-1} with unit loading z_j.
// The caller's A is never written: the library solves on a working copy W
// (float, or double for F64 storage) and deflates W in place.  Only the
// columns in the support of z_j change, so one deflation reads and writes
// |supp z_j| columns of W: a few MB against the hundreds of MB one sweep
// reads.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dd.cuh"
#include "deflate.cuh"
#include "gpspca.h"

namespace gpspca {

template <typename TA>
__device__ __forceinline__ float to_float(TA v);
template <>
__device__ __forceinline__ float to_float<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_float<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) {
  return static_cast<float>(v);
}

// W (ldw >= p, rows p..ldw-1 zero) = A in the working type; fp8 entries
// times their column scale.  Block (x: 1024 rows, y: columns, strided).
template <typename TA, typename TW>
__global__ void deflate_copy_kernel(const TA* __restrict__ A, int64_t ld, const float* __restrict__ scale,
                                    TW* __restrict__ W, int64_t ldw, int64_t p, int64_t n) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const float s = scale ? scale[i] : 1.0f;
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < ldw;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      TW v = TW(0);
      if (r < p) {
        if constexpr (sizeof(TW) == 8)
          v = static_cast<TW>(A[i * ld + r]);
        else
          v = scale ? to_float(A[i * ld + r]) * s : to_float(A[i * ld + r]);
      }
      W[i * ldw + r] = v;
    }
  }
}

// Accumulator of u_r = sum_i z_i W[r, i]: double-float for float W (the
// products and their sum to ~2^-48, on the float pipes), double for double W.
template <typename TW>
struct UAcc;
template <>
struct UAcc<float> {
  dd v{0.0f, 0.0f};
  __device__ void add(float z, float w) { v = dd_add(v, two_prod(z, w)); }
  __device__ float value() const { return v.hi + v.lo; }
};
template <>
struct UAcc<double> {
  double v = 0.0;
  __device__ void add(double z, double w) { v = fma(z, w, v); }
  __device__ double value() const { return v; }
};

// One deflation step on the rows of this block (one row per thread):
// u_r = sum_{z_i != 0} z_i W[r, i], then W[r, i] -= z_i u_r on the same
// columns.  Each warp finds the nonzeros of z 32 at a time by ballot, so
// zero entries cost one coalesced load per 32.  Rows are independent: no
// synchronisation between blocks; the sum runs in column order
// (deterministic).
template <typename TW>
__global__ void __launch_bounds__(256) deflate_kernel(TW* __restrict__ W, int64_t ldw, int64_t p, int64_t n,
                                                      const TW* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const bool row_ok = r < p;
  UAcc<TW> acc;
  for (int64_t c0 = 0; c0 < n; c0 += 32) {
    const TW zi = (c0 + lane < n) ? z[c0 + lane] : TW(0);
    uint32_t mask = __ballot_sync(0xffffffffu, zi != TW(0));
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const TW zb = __shfl_sync(0xffffffffu, zi, b);
      if (row_ok) acc.add(zb, W[(c0 + b) * ldw + r]);
    }
  }
  const TW u = acc.value();
  for (int64_t c0 = 0; c0 < n; c0 += 32) {
    const TW zi = (c0 + lane < n) ? z[c0 + lane] : TW(0);
    uint32_t mask = __ballot_sync(0xffffffffu, zi != TW(0));
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const TW zb = __shfl_sync(0xffffffffu, zi, b);
      if (row_ok) {
        TW* w = &W[(c0 + b) * ldw + r];
        *w = fma(-zb, u, *w);
      }
    }
  }
}

int64_t deflate_ld(int dtype, int64_t p) {
  const int64_t q = dtype == GPSPCA_F64 ? 2 : 4;  // 16-byte column stride
  return std::max<int64_t>(q, (p + q - 1) / q * q);
}

void launch_deflate_copy(int dtype, const void* A, int64_t ld, const float* scale, void* W, int64_t ldw, int64_t p,
                         int64_t n, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>(std::min<int64_t>((ldw + 1023) / 1024, 64)),
                  static_cast<unsigned>(std::min<int64_t>(n, 65535)));
  switch (dtype) {
    case GPSPCA_F32:
      deflate_copy_kernel<float, float><<<grid, 1024, 0, s>>>(static_cast<const float*>(A), ld, nullptr,
                                                              static_cast<float*>(W), ldw, p, n);
      break;
    case GPSPCA_BF16:
      deflate_copy_kernel<__nv_bfloat16, float><<<grid, 1024, 0, s>>>(static_cast<const __nv_bfloat16*>(A), ld,
                                                                      nullptr, static_cast<float*>(W), ldw, p, n);
      break;
    case GPSPCA_FP8_E4M3:
      deflate_copy_kernel<__nv_fp8_e4m3, float><<<grid, 1024, 0, s>>>(static_cast<const __nv_fp8_e4m3*>(A), ld,
                                                                      scale, static_cast<float*>(W), ldw, p, n);
      break;
    default:
      deflate_copy_kernel<double, double><<<grid, 1024, 0, s>>>(static_cast<const double*>(A), ld, nullptr,
                                                                static_cast<double*>(W), ldw, p, n);
      break;
  }
}

void launch_deflate(int dtype, void* W, int64_t ldw, int64_t p, int64_t n, const void* z, cudaStream_t s) {
  const unsigned blocks = static_cast<unsigned>((p + 255) / 256);
  if (dtype == GPSPCA_F64)
    deflate_kernel<double><<<blocks, 256, 0, s>>>(static_cast<double*>(W), ldw, p, n, static_cast<const double*>(z));
  else
    deflate_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float*>(W), ldw, p, n, static_cast<const float*>(z));
}

}  // namespace gpspca
