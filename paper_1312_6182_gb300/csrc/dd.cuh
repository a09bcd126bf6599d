// Double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 executes double precision at a small fraction of its float rate
// (about two FP64 lanes per clock per SM), so the serial m x m linear algebra
// of the polar step (Gram eigenproblem, Rayleigh-Ritz) runs on the float
// pipes in this representation instead: every operation below is a short
// chain of float adds and fused multiply-adds.
//
// The error-free transformations are the classical ones: Knuth's two-sum
// (TAOCP vol. 2, 4.2.2), Dekker's fast two-sum for |a| >= |b| and the
// product with its exact rounding error from one fused multiply-add
// (Dekker 1971, "A floating-point technique for extending the available
// precision").  Relative error of dd_add / dd_mul: a few units of 2^-48.
// Range: float's; callers scale their matrices by a power of two first.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace gpspca {

struct dd {
  float hi, lo;
};

__host__ __device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__host__ __device__ __forceinline__ dd fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}

__host__ __device__ __forceinline__ dd two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return {p, e};
}

__host__ __device__ __forceinline__ dd dd_from_double(double x) {
  const float h = static_cast<float>(x);
  return {h, static_cast<float>(x - static_cast<double>(h))};
}

__host__ __device__ __forceinline__ double dd_to_double(dd a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

__host__ __device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

// Accurate sum (both parts through two-sum): holds its error bound under
// cancellation, which the Jacobi updates rely on.
__host__ __device__ __forceinline__ dd dd_add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  dd u = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(u.hi, u.lo + t.lo);
}

__host__ __device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__host__ __device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const dd p = two_prod(a.hi, b.hi);
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, e);
}

__host__ __device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  const dd p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// a * b + c
__host__ __device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }

// 1/sqrt(x), x > 0: float estimate r, then one Newton step
// r + r (1 - x r^2) / 2 with the residual formed in dd (its relative error
// squares: ~1e-7 -> ~1e-14).
__host__ __device__ __forceinline__ dd dd_rsqrt(dd x) {
#ifdef __CUDA_ARCH__
  const float r = rsqrtf(x.hi);
#else
  const float r = 1.0f / std::sqrt(x.hi);
#endif
  const dd h = dd_sub(dd{1.0f, 0.0f}, dd_mul(x, two_prod(r, r)));
  return fast_two_sum(r, r * h.hi * 0.5f);
}

}  // namespace gpspca
