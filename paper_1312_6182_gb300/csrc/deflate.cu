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
  __device__ void store(float* hi, float* lo) const {
    *hi = v.hi;
    *lo = v.lo;
  }
  __device__ void merge(float hi, float lo) { v = dd_add(v, dd{hi, lo}); }
  __device__ float value() const { return v.hi + v.lo; }
};
template <>
struct UAcc<double> {
  double v = 0.0;
  __device__ void add(double z, double w) { v = fma(z, w, v); }
  __device__ void store(double* hi, float* lo) const {
    *hi = v;
    *lo = 0.0f;
  }
  __device__ void merge(double hi, float) { v += hi; }
  __device__ double value() const { return v; }
};

// ---- support compaction: the nonzero entries of z in index order
// (idx, val, count), two launches over contiguous ranges of z, one block per
// range: counts, then each block's offset (sum of the earlier counts) and an
// ordered write (ballot prefix within each 1024-entry window).
constexpr int kCompactThreads = 1024;

template <typename TW>
__global__ void __launch_bounds__(kCompactThreads) support_count_kernel(const TW* __restrict__ z, int64_t n,
                                                                         int64_t chunk, int32_t* __restrict__ cnt) {
  __shared__ int32_t red[kCompactThreads / 32];
  const int64_t b = blockIdx.x * chunk, e = min(n, b + chunk);
  int32_t c = 0;
  for (int64_t i = b + threadIdx.x; i < e; i += kCompactThreads) c += z[i] != TW(0);
  for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) t += red[w];
    cnt[blockIdx.x] = t;
  }
}

template <typename TW>
__global__ void __launch_bounds__(kCompactThreads) support_write_kernel(const TW* __restrict__ z, int64_t n,
                                                                         int64_t chunk, const int32_t* __restrict__ cnt,
                                                                         int32_t* __restrict__ idx,
                                                                         TW* __restrict__ val, int32_t* total) {
  __shared__ int32_t wcnt[kCompactThreads / 32];
  __shared__ int32_t base_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int32_t o = 0;
    for (int g = 0; g < static_cast<int>(blockIdx.x); ++g) o += cnt[g];
    base_s = o;
    if (blockIdx.x == gridDim.x - 1) *total = o + cnt[blockIdx.x];
  }
  __syncthreads();
  int32_t base = base_s;
  const int64_t b = blockIdx.x * chunk, e = min(n, b + chunk);
  for (int64_t w0 = b; w0 < e; w0 += kCompactThreads) {
    const int64_t i = w0 + threadIdx.x;
    const TW v = i < e ? z[i] : TW(0);
    const uint32_t bal = __ballot_sync(0xffffffffu, v != TW(0));
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int32_t before = 0, all = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) {
      before += w < warp ? wcnt[w] : 0;
      all += wcnt[w];
    }
    if (v != TW(0)) {
      const int32_t k = base + before + __popc(bal & ((1u << lane) - 1u));
      idx[k] = static_cast<int32_t>(i);
      val[k] = v;
    }
    base += all;
    __syncthreads();  // wcnt is rewritten by the next window
  }
}

// ---- one deflation step: 32 rows per block (lane = row), the support list
// split into 8 contiguous shares, one per warp.  u_r = sum_k val_k W[r, idx_k]
// (each warp's share, then the shares added in warp order: deterministic),
// then W[r, idx_k] -= val_k u_r over the same shares.
constexpr int kDeflateWarps = 8;
constexpr int kDeflateBatch = 8;  // support entries whose loads are in flight together

template <typename TW>
__global__ void __launch_bounds__(kDeflateWarps * 32) deflate_kernel(TW* __restrict__ W, int64_t ldw, int64_t p,
                                                                    const int32_t* __restrict__ idx,
                                                                    const TW* __restrict__ val,
                                                                    const int32_t* __restrict__ count) {
  __shared__ TW part_hi[kDeflateWarps][32];
  __shared__ float part_lo[kDeflateWarps][32];
  __shared__ TW u_s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r = blockIdx.x * 32ll + lane;
  const bool row_ok = r < p;
  const int32_t K = *count;
  const int32_t share = (K + kDeflateWarps - 1) / kDeflateWarps;
  const int32_t kb = min(K, warp * share), ke = min(K, kb + share);
  UAcc<TW> acc;
  for (int32_t k0 = kb; k0 < ke; k0 += kDeflateBatch) {
    TW w[kDeflateBatch], zv[kDeflateBatch];
#pragma unroll
    for (int q = 0; q < kDeflateBatch; ++q) {
      const bool ok = k0 + q < ke;
      zv[q] = ok ? val[k0 + q] : TW(0);
      w[q] = (ok && row_ok) ? W[static_cast<int64_t>(idx[k0 + q]) * ldw + r] : TW(0);
    }
#pragma unroll
    for (int q = 0; q < kDeflateBatch; ++q) acc.add(zv[q], w[q]);
  }
  acc.store(&part_hi[warp][lane], &part_lo[warp][lane]);
  __syncthreads();
  if (warp == 0) {
    UAcc<TW> t;
    for (int q = 0; q < kDeflateWarps; ++q) t.merge(part_hi[q][lane], part_lo[q][lane]);
    u_s[lane] = t.value();
  }
  __syncthreads();
  const TW u = u_s[lane];
  if (!row_ok) return;
  for (int32_t k0 = kb; k0 < ke; k0 += kDeflateBatch) {
#pragma unroll
    for (int q = 0; q < kDeflateBatch; ++q) {
      if (k0 + q < ke) {
        TW* wp = &W[static_cast<int64_t>(idx[k0 + q]) * ldw + r];
        *wp = fma(-val[k0 + q], u, *wp);
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

size_t deflate_list_bytes(int dtype, int64_t n) {
  const size_t tcs = dtype == GPSPCA_F64 ? sizeof(double) : sizeof(float);
  return static_cast<size_t>(n) * (sizeof(int32_t) + tcs) + sizeof(int32_t) * (kCompactThreads + 2) + 64;
}

template <typename TW>
static void deflate_typed(TW* W, int64_t ldw, int64_t p, int64_t n, const TW* z, void* list, cudaStream_t s) {
  // list layout: val (n), idx (n), count (1), per-range counts (<= 1024)
  TW* val = static_cast<TW*>(list);
  int32_t* idx = reinterpret_cast<int32_t*>(val + n);
  int32_t* count = idx + n;
  int32_t* cnt = count + 1;
  const int64_t ranges = std::min<int64_t>(kCompactThreads, (n + kCompactThreads - 1) / kCompactThreads);
  const int64_t chunk = (n + ranges - 1) / ranges;
  support_count_kernel<TW><<<static_cast<unsigned>(ranges), kCompactThreads, 0, s>>>(z, n, chunk, cnt);
  support_write_kernel<TW><<<static_cast<unsigned>(ranges), kCompactThreads, 0, s>>>(z, n, chunk, cnt, idx, val,
                                                                                     count);
  deflate_kernel<TW><<<static_cast<unsigned>((p + 31) / 32), kDeflateWarps * 32, 0, s>>>(W, ldw, p, idx, val, count);
}

void launch_deflate(int dtype, void* W, int64_t ldw, int64_t p, int64_t n, const void* z, void* list,
                    cudaStream_t s) {
  if (dtype == GPSPCA_F64)
    deflate_typed(static_cast<double*>(W), ldw, p, n, static_cast<const double*>(z), list, s);
  else
    deflate_typed(static_cast<float*>(W), ldw, p, n, static_cast<const float*>(z), list, s);
}

}  // namespace gpspca
