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
// range (blockIdx.y: the column of Z, each with its own list): counts, then
// each block's offset (sum of the earlier counts) and an ordered write
// (ballot prefix within each 1024-entry window).
constexpr int kCompactThreads = 1024;

struct SupportList {  // one column's list inside the scratch buffer
  int32_t *idx, *count, *cnt;
  void* val;
};
template <typename TW>
__host__ __device__ __forceinline__ SupportList support_list(void* list, size_t stride, int64_t n, int j) {
  SupportList L;
  char* b = static_cast<char*>(list) + stride * j;
  L.val = b;
  L.idx = reinterpret_cast<int32_t*>(b + sizeof(TW) * n);
  L.count = L.idx + n;
  L.cnt = L.count + 1;
  return L;
}

template <typename TW>
__global__ void __launch_bounds__(kCompactThreads) support_count_kernel(const TW* __restrict__ Z, int64_t n,
                                                                         int64_t chunk, void* list, size_t stride) {
  __shared__ int32_t red[kCompactThreads / 32];
  const TW* z = Z + n * blockIdx.y;
  const SupportList L = support_list<TW>(list, stride, n, blockIdx.y);
  const int64_t b = blockIdx.x * chunk, e = min(n, b + chunk);
  int32_t c = 0;
  for (int64_t i = b + threadIdx.x; i < e; i += kCompactThreads) c += z[i] != TW(0);
  for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) t += red[w];
    L.cnt[blockIdx.x] = t;
  }
}

template <typename TW>
__global__ void __launch_bounds__(kCompactThreads) support_write_kernel(const TW* __restrict__ Z, int64_t n,
                                                                         int64_t chunk, void* list, size_t stride) {
  __shared__ int32_t wcnt[kCompactThreads / 32];
  __shared__ int32_t base_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TW* z = Z + n * blockIdx.y;
  const SupportList L = support_list<TW>(list, stride, n, blockIdx.y);
  TW* val = static_cast<TW*>(L.val);
  if (threadIdx.x == 0) {
    int32_t o = 0;
    for (int g = 0; g < static_cast<int>(blockIdx.x); ++g) o += L.cnt[g];
    base_s = o;
    if (blockIdx.x == gridDim.x - 1) *L.count = o + L.cnt[blockIdx.x];
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
      L.idx[k] = static_cast<int32_t>(i);
      val[k] = v;
    }
    base += all;
    __syncthreads();  // wcnt is rewritten by the next window
  }
}

// ---- V consecutive rows of one column as the working type: 16-byte loads
// for float (4 rows) and double (2 rows), 8 / 4 bytes for bf16 / fp8 (4
// rows), or single elements (V = 1) for layouts without that alignment.
template <typename TA, typename TW, int V>
__device__ __forceinline__ void load_rows(const TA* p, TW (&v)[V]) {
  if constexpr (V == 1) {
    v[0] = static_cast<TW>(to_float(*p));
  } else if constexpr (sizeof(TA) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
  } else if constexpr (sizeof(TA) == 2) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(u.x << 16);
    v[1] = __uint_as_float(u.x & 0xffff0000u);
    v[2] = __uint_as_float(u.y << 16);
    v[3] = __uint_as_float(u.y & 0xffff0000u);
  } else {
    const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_fp8_e4m3 q;
      q.__x = static_cast<__nv_fp8_storage_t>((u >> (8 * e)) & 0xffu);
      v[e] = static_cast<float>(q);
    }
  }
}
template <>
__device__ __forceinline__ void load_rows<double, double, 1>(const double* p, double (&v)[1]) {
  v[0] = *p;
}
template <>
__device__ __forceinline__ void load_rows<double, double, 2>(const double* p, double (&v)[2]) {
  const double2 f = *reinterpret_cast<const double2*>(p);
  v[0] = f.x;
  v[1] = f.y;
}

// Rows per lane: 4 for float-type sums (2 for double) on aligned layouts.
template <typename TW>
constexpr int kRowsVec = sizeof(TW) == 8 ? 2 : 4;

// ---- u = B z (one column of Z per blockIdx.y), 32 V rows per block (V per
// lane), the support list split into kSupWarps contiguous shares, one per
// warp, the shares' sums added in warp order (deterministic).
constexpr int kSupWarps = 16;
constexpr int kSupBatch = 8;  // support entries whose loads are in flight together

template <typename TA, typename TW, int V>
__device__ __forceinline__ void support_dot(const TA* __restrict__ B, int64_t ld, const float* __restrict__ scale,
                                            int64_t r0, bool row_ok, const SupportList& L, TW (&u)[V],
                                            TW (*part_hi)[32 * V], float (*part_lo)[32 * V]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TW* val = static_cast<const TW*>(L.val);
  const int32_t K = *L.count;
  const int32_t share = (K + kSupWarps - 1) / kSupWarps;
  const int32_t kb = min(K, warp * share), ke = min(K, kb + share);
  UAcc<TW> acc[V];
  for (int32_t k0 = kb; k0 < ke; k0 += kSupBatch) {
    TW w[kSupBatch][V], zv[kSupBatch];
#pragma unroll
    for (int e = 0; e < kSupBatch; ++e) {
      const bool ok = k0 + e < ke;
      zv[e] = ok ? val[k0 + e] : TW(0);
#pragma unroll
      for (int v = 0; v < V; ++v) w[e][v] = TW(0);
      if (ok && row_ok) {
        const int32_t i = L.idx[k0 + e];
        load_rows<TA, TW, V>(B + static_cast<int64_t>(i) * ld + r0, w[e]);
        if (scale) {
#pragma unroll
          for (int v = 0; v < V; ++v) w[e][v] *= static_cast<TW>(scale[i]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < kSupBatch; ++e)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v].add(zv[e], w[e][v]);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v].store(&part_hi[warp][lane * V + v], &part_lo[warp][lane * V + v]);
  __syncthreads();
#pragma unroll
  for (int v = 0; v < V; ++v) {
    UAcc<TW> t;
    for (int q = 0; q < kSupWarps; ++q) t.merge(part_hi[q][lane * V + v], part_lo[q][lane * V + v]);
    u[v] = t.value();
  }
}

// S[:, j] = B z_j: grid (row blocks, m).
template <typename TA, typename TW, int V>
__global__ void __launch_bounds__(kSupWarps * 32) project_kernel(const TA* __restrict__ B, int64_t ld,
                                                                const float* __restrict__ scale, int64_t q, int64_t n,
                                                                void* list, size_t stride, TW* __restrict__ S) {
  __shared__ TW part_hi[kSupWarps][32 * V];
  __shared__ float part_lo[kSupWarps][32 * V];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (blockIdx.x * 32ll + lane) * V;
  const bool row_ok = r0 < q;
  const SupportList L = support_list<TW>(list, stride, n, blockIdx.y);
  TW u[V];
  support_dot<TA, TW, V>(B, ld, scale, r0, row_ok, L, u, part_hi, part_lo);
  if (warp == 0) {
    TW* Sj = S + q * blockIdx.y;
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (r0 + v < q) Sj[r0 + v] = u[v];
  }
}

// One deflation step, W <- W - (W z) z^T: u = W z on the block's rows (as
// above), then W[r, idx_k] -= val_k u_r over the same shares.  W's column
// stride is a multiple of V and its rows p..ldw-1 are zero (so u is zero
// there and they stay zero).
template <typename TW, int V>
__global__ void __launch_bounds__(kSupWarps * 32) deflate_kernel(TW* __restrict__ W, int64_t ldw, int64_t n,
                                                                void* list, size_t stride) {
  __shared__ TW part_hi[kSupWarps][32 * V];
  __shared__ float part_lo[kSupWarps][32 * V];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (blockIdx.x * 32ll + lane) * V;
  const bool row_ok = r0 < ldw;
  const SupportList L = support_list<TW>(list, stride, n, 0);
  TW u[V];
  support_dot<TW, TW, V>(W, ldw, nullptr, r0, row_ok, L, u, part_hi, part_lo);
  if (!row_ok) return;
  const TW* val = static_cast<const TW*>(L.val);
  const int32_t K = *L.count;
  const int32_t share = (K + kSupWarps - 1) / kSupWarps;
  const int32_t kb = min(K, warp * share), ke = min(K, kb + share);
  for (int32_t k = kb; k < ke; ++k) {
    TW* wp = W + static_cast<int64_t>(L.idx[k]) * ldw + r0;
    const TW z = val[k];
#pragma unroll
    for (int v = 0; v < V; ++v) wp[v] = fma(-z, u[v], wp[v]);
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
  const size_t b = static_cast<size_t>(n) * (sizeof(int32_t) + tcs) + sizeof(int32_t) * (kCompactThreads + 2) + 64;
  return (b + 255) / 256 * 256;
}

template <typename TW>
static void compact_supports(const TW* Z, int64_t n, int m, void* list, size_t stride, cudaStream_t s) {
  const int64_t ranges = std::min<int64_t>(kCompactThreads, (n + kCompactThreads - 1) / kCompactThreads);
  const int64_t chunk = (n + ranges - 1) / ranges;
  const dim3 grid(static_cast<unsigned>(ranges), static_cast<unsigned>(m));
  support_count_kernel<TW><<<grid, kCompactThreads, 0, s>>>(Z, n, chunk, list, stride);
  support_write_kernel<TW><<<grid, kCompactThreads, 0, s>>>(Z, n, chunk, list, stride);
}

template <typename TA, typename TW>
static void project_typed(const TA* B, int64_t ld, const float* scale, int64_t q, int64_t n, const TW* Z, int m,
                          TW* S, void* list, cudaStream_t s) {
  const size_t stride = deflate_list_bytes(sizeof(TW) == 8 ? GPSPCA_F64 : GPSPCA_F32, n);
  compact_supports(Z, n, m, list, stride, s);
  constexpr int V = kRowsVec<TW>;
  const bool vec = (reinterpret_cast<uintptr_t>(B) % (sizeof(TA) * V) == 0) && (ld % V == 0);
  if (vec) {
    const dim3 grid(static_cast<unsigned>((q + 32 * V - 1) / (32 * V)), static_cast<unsigned>(m));
    project_kernel<TA, TW, V><<<grid, kSupWarps * 32, 0, s>>>(B, ld, scale, q, n, list, stride, S);
  } else {
    const dim3 grid(static_cast<unsigned>((q + 31) / 32), static_cast<unsigned>(m));
    project_kernel<TA, TW, 1><<<grid, kSupWarps * 32, 0, s>>>(B, ld, scale, q, n, list, stride, S);
  }
}

void launch_project(int dtype, const void* B, int64_t ld, const float* scale, int64_t q, int64_t n, const void* Z,
                    int m, void* S, void* list, cudaStream_t s) {
  switch (dtype) {
    case GPSPCA_F32:
      project_typed(static_cast<const float*>(B), ld, nullptr, q, n, static_cast<const float*>(Z), m,
                    static_cast<float*>(S), list, s);
      break;
    case GPSPCA_BF16:
      project_typed(static_cast<const __nv_bfloat16*>(B), ld, nullptr, q, n, static_cast<const float*>(Z), m,
                    static_cast<float*>(S), list, s);
      break;
    case GPSPCA_FP8_E4M3:
      project_typed(static_cast<const __nv_fp8_e4m3*>(B), ld, scale, q, n, static_cast<const float*>(Z), m,
                    static_cast<float*>(S), list, s);
      break;
    default:
      project_typed(static_cast<const double*>(B), ld, nullptr, q, n, static_cast<const double*>(Z), m,
                    static_cast<double*>(S), list, s);
      break;
  }
}

template <typename TW>
static void deflate_typed(TW* W, int64_t ldw, int64_t n, const TW* z, void* list, cudaStream_t s) {
  const size_t stride = deflate_list_bytes(sizeof(TW) == 8 ? GPSPCA_F64 : GPSPCA_F32, n);
  compact_supports(z, n, 1, list, stride, s);
  constexpr int V = kRowsVec<TW>;
  deflate_kernel<TW, V><<<static_cast<unsigned>((ldw + 32 * V - 1) / (32 * V)), kSupWarps * 32, 0, s>>>(
      W, ldw, n, list, stride);
}

void launch_deflate(int dtype, void* W, int64_t ldw, int64_t p, int64_t n, const void* z, void* list,
                    cudaStream_t s) {
  (void)p;  // rows p..ldw-1 of W are zero and stay zero
  if (dtype == GPSPCA_F64)
    deflate_typed(static_cast<double*>(W), ldw, n, static_cast<const double*>(z), list, s);
  else
    deflate_typed(static_cast<float*>(W), ldw, n, static_cast<const float*>(z), list, s);
}

}  // namespace gpspca
