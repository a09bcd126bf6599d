// Kernels around the fused sweep (see aux.cuh).
#include <algorithm>

#include "aux.cuh"
#include "smalleig.cuh"

namespace gpspca {

// ---------------------------------------------------------------- helpers

// k-th output of the SplitMix64 stream seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int stop_rule(int k, double f, double f_prev, double tol, int maxit) {
  // Stopping test after sweep k (objective f_k): zero objective, relative
  // change below tol (from the second sweep on), or the sweep budget.
  if (f == 0.0) return GPSPCA_ZERO;
  if (k > 0 && fabs(f - f_prev) < tol * f_prev) return GPSPCA_CONVERGED;
  if (k == maxit - 1) return GPSPCA_MAXIT;
  return -1;
}

// 1/sqrt(x) for x > 0 in double: float estimate, two Newton steps (each
// squares the relative error: 1e-7 -> 1e-14 -> 1e-16).  Keeps the slow
// double-precision division and square root off the serial paths of the
// one-CTA kernels.
__device__ __forceinline__ double rsqrt_refined(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);  // outside float's comfortable range
  double r = static_cast<double>(rsqrtf(static_cast<float>(x)));
  r = r * (1.5 - 0.5 * x * r * r);
  r = r * (1.5 - 0.5 * x * r * r);
  return r;
}

// dst[q] = sum_{b < nb} src[b*stride + q] for q < nq, added in a fixed order
// (per q: strided over tpp lanes with the loads of four partials in flight,
// then a shuffle tree), so the result does not depend on scheduling.  dd
// partials are summed in double-float, double partials in double; dst is
// written as double.  All threads of the block must call it.
__device__ __forceinline__ dd sp_zero(const dd*) { return dd{0.0f, 0.0f}; }
__device__ __forceinline__ double sp_zero(const double*) { return 0.0; }
__device__ __forceinline__ dd sp_add(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ double sp_add(double a, double b) { return a + b; }
__device__ __forceinline__ double sp_out(dd a) { return dd_to_double(a); }
__device__ __forceinline__ double sp_out(double a) { return a; }
__device__ __forceinline__ dd sp_shfl(dd v, int off, int w) {
  return dd{__shfl_down_sync(0xffffffffu, v.hi, off, w), __shfl_down_sync(0xffffffffu, v.lo, off, w)};
}
__device__ __forceinline__ double sp_shfl(double v, int off, int w) { return __shfl_down_sync(0xffffffffu, v, off, w); }

template <typename P>
__device__ void sum_partials(const P* __restrict__ src, int nb, int stride, int nq, double* dst) {
  int tpp = 32;
  while (tpp > 1 && tpp * nq > static_cast<int>(blockDim.x)) tpp >>= 1;
  const int groups = blockDim.x / tpp;
  const int sub = threadIdx.x % tpp;
  for (int q0 = 0; q0 < nq; q0 += groups) {
    const int q = q0 + static_cast<int>(threadIdx.x) / tpp;
    P s0 = sp_zero(src), s1 = sp_zero(src);
    if (q < nq) {
      // sixteen partials' loads in flight per step (hundreds of partials
      // per entry: the sum is bound by the load latency), added in a fixed
      // order
      int b = sub;
      for (; b + 15 * tpp < nb; b += 16 * tpp) {
        P v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = src[static_cast<int64_t>(b + u * tpp) * stride + q];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          s0 = sp_add(s0, sp_add(v[u], v[u + 8]));
          s1 = sp_add(s1, sp_add(v[u + 1], v[u + 9]));
        }
      }
      for (; b + 3 * tpp < nb; b += 4 * tpp) {
        const P v0 = src[static_cast<int64_t>(b) * stride + q];
        const P v1 = src[static_cast<int64_t>(b + tpp) * stride + q];
        const P v2 = src[static_cast<int64_t>(b + 2 * tpp) * stride + q];
        const P v3 = src[static_cast<int64_t>(b + 3 * tpp) * stride + q];
        s0 = sp_add(s0, sp_add(v0, v2));
        s1 = sp_add(s1, sp_add(v1, v3));
      }
      for (; b < nb; b += tpp) s0 = sp_add(s0, src[static_cast<int64_t>(b) * stride + q]);
    }
    P s = sp_add(s0, s1);
    for (int off = tpp / 2; off > 0; off >>= 1) s = sp_add(s, sp_shfl(s, off, tpp));
    if (q < nq && sub == 0) dst[q] = sp_out(s);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ void reset_state_body(const IO* io, State* st, int m, int form) {
  const int j = threadIdx.x;
  if (j == 0) {
    st->k = -1;
    st->n_active = m;
    st->error = 0;
    st->any_degenerate = 0;
    st->cmax = 0.0;
    st->has_v = 0;
  }
  if (j < kMaxM) {
    const bool v = j < m;
    st->active[j] = v ? 1 : 0;
    st->status[j] = GPSPCA_MAXIT;
    st->iters[j] = 0;
    st->gamma[j] = v ? io->gamma_in[j] : 0.0;
    st->f_prev[j] = 0.0;
    st->f[j] = 0.0;
    st->znorm2[j] = 0.0;
    st->start_cols[j] = -1;
  }
}

// Load 16 bytes = Elem<TA>::ALIGN elements as float (or double for F64).
template <typename TA>
struct Wide;
template <>
struct Wide<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float (&v)[4]) { load_vec(p, v); }
};
template <>
struct Wide<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double (&v)[2]) { load_vec(p, v); }
};
template <>
struct Wide<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void load(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v[2 * i] = __uint_as_float(w[i] << 16);
      v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};
template <>
struct Wide<__nv_fp8_e4m3> {
  static constexpr int N = 16;
  __device__ static void load(const __nv_fp8_e4m3* p, float (&v)[16]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 a = fp8x2_to_float2(w[i] & 0xffffu);
      const float2 b = fp8x2_to_float2(w[i] >> 16);
      v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = b.x; v[4 * i + 3] = b.y;
    }
  }
};

// Column norms c_i = ||a_i||_2 (step a0).  Float storage: squares summed
// with Kahan compensation per lane in float, lanes combined in double; the
// accurate norms (double-float sums of exact products) of the leading
// candidates are recomputed by select_start_kernel before any decision is
// taken on them.  One warp per column.  A non-finite norm flags the solve.
template <typename TA>
__device__ __forceinline__ void colnorm_core(const TA* __restrict__ A, const float* col_scale, double* cnorm,
                                             int32_t* error, int64_t ld, int p, int n, int fast) {
  using TC = typename Elem<TA>::TC;
  constexpr int NW = Wide<TA>::N;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (int i = gw; i < n; i += nwarps) {
    const TA* col = A + static_cast<int64_t>(i) * ld;
    TC sum = 0, comp = 0;
    auto add = [&](TC v) {
      if constexpr (sizeof(TC) == 8) {
        sum += v * v;
      } else {
        const TC yk = v * v - comp;
        const TC tk = sum + yk;
        comp = (tk - sum) - yk;
        sum = tk;
      }
    };
    int r0 = 0;
    if (fast) {
      const int nvec = p / NW;
      for (int vi = lane; vi < nvec; vi += 32) {
        TC v[NW];
        Wide<TA>::load(col + vi * NW, v);
#pragma unroll
        for (int e = 0; e < NW; ++e) add(v[e]);
      }
      r0 = nvec * NW;
    }
    for (int r = r0 + lane; r < p; r += 32) add(to_tc<TA>(col[r]));
    double tot = static_cast<double>(sum) - static_cast<double>(comp);
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
    if (lane == 0) {
      double c = sqrt(tot);
      if (sizeof(TA) == 1) c *= static_cast<double>(col_scale[i]);
      if (!isfinite(c)) bad = true;
      cnorm[i] = c;
    }
  }
  if (bad) atomicOr(error, static_cast<int>(kErrNonFinite));
}
template <typename TA>
__device__ __forceinline__ void colnorm_body(const IO* io, State* st, int64_t ld, int p, int n, int fast) {
  colnorm_core<TA>(static_cast<const TA*>(io->A), io->col_scale, io->cnorm, &st->error, ld, p, n, fast);
}

// Squared norm of column i over the rows [r0, p) step `step`: float data in
// double-float (products of floats are exact, the sum is good to ~1e-14),
// double data in double.
template <typename TA>
__device__ __forceinline__ dd col_sumsq_part(const IO* io, int64_t ld, int p, int i, int r0, int step) {
  const TA* col = static_cast<const TA*>(io->A) + static_cast<int64_t>(i) * ld;
  if constexpr (sizeof(typename Elem<TA>::TC) == 8) {
    double s0 = 0.0, s1 = 0.0;
    int r = r0;
    for (; r + step < p; r += 2 * step) {
      const double v0 = static_cast<double>(to_tc<TA>(col[r]));
      const double v1 = static_cast<double>(to_tc<TA>(col[r + step]));
      s0 = fma(v0, v0, s0);
      s1 = fma(v1, v1, s1);
    }
    if (r < p) {
      const double v = static_cast<double>(to_tc<TA>(col[r]));
      s0 = fma(v, v, s0);
    }
    return dd_from_double(s0 + s1);
  } else {
    dd s0{0.0f, 0.0f}, s1{0.0f, 0.0f};
    int r = r0;
    for (; r + step < p; r += 2 * step) {
      const float v0 = to_tc<TA>(col[r]);
      const float v1 = to_tc<TA>(col[r + step]);
      s0 = dd_add(s0, two_prod(v0, v0));
      s1 = dd_add(s1, two_prod(v1, v1));
    }
    if (r < p) {
      const float v = to_tc<TA>(col[r]);
      s0 = dd_add(s0, two_prod(v, v));
    }
    return dd_add(s0, s1);
  }
}

__device__ __forceinline__ dd warp_sum_dd(dd v) {
  for (int off = 16; off > 0; off >>= 1)
    v = dd_add(v, dd{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)});
  return v;
}

// Accurate norm of column i by one warp (scaled by the FP8 column scale).
template <typename TA>
__device__ double exact_colnorm_warp(const IO* io, int64_t ld, int p, int i) {
  const dd s = warp_sum_dd(col_sumsq_part<TA>(io, ld, p, i, threadIdx.x & 31, 32));
  double c = sqrt(dd_to_double(s));
  if (sizeof(TA) == 1) c *= static_cast<double>(io->col_scale[i]);
  return c;
}

// Accurate norm of column i by the whole CTA (warp partials added in warp
// order); every thread gets the value.
template <typename TA>
__device__ double exact_colnorm_cta(const IO* io, int64_t ld, int p, int i, dd* red) {
  const dd s = warp_sum_dd(col_sumsq_part<TA>(io, ld, p, i, threadIdx.x, blockDim.x));
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = s;
  __syncthreads();
  dd t = red[0];
  for (int w = 1; w < nw; ++w) t = dd_add(t, red[w]);
  __syncthreads();
  double c = sqrt(dd_to_double(t));
  if (sizeof(TA) == 1) c *= static_cast<double>(io->col_scale[i]);
  return c;
}

// (value desc, index asc) ordering on non-negative doubles, compared through
// their bit patterns (which order like the values) on the integer pipes.
__device__ __forceinline__ bool better_bits(long long v, int i, long long bv, int bi) {
  return (v > bv) || (v == bv && i < bi);
}
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  return (v > bv) || (v == bv && i < bi);
}

// Start of the iteration (step a0): the largest-norm column (single-unit),
// ties to the lower index, decided on accurate norms; gamma scaled by
// max_i ||a_i|| when relative.  One CTA.
template <typename TA>
__device__ __forceinline__ void select_start_body(const StartArgs& a) {
  const IO* io = a.io;
  State* st = a.st;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  __shared__ long long sv[33];
  __shared__ int si[33];
  __shared__ dd red[32];
  __shared__ int cand[kMaxCandidates];
  __shared__ double cexact[kMaxCandidates];
  __shared__ int ncand;
  __shared__ int order0;
  if (st->error) {
    if (tid == 0) st->n_active = 0;
    return;
  }
  const bool block = a.form >= 2;
  // 1. arg-max of the compensated norms (the start column of single-unit
  //    forms; the largest norm also scales a relative gamma)
  const long long* cb = reinterpret_cast<const long long*>(io->cnorm);
  long long bv = -1;
  int bi = 0x7fffffff;
  for (int i = tid; i < a.n; i += nthr) {
    const long long v = cb[i];
    if (better_bits(v, i, bv, bi)) { bv = v; bi = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (better_bits(ov, oi, bv, bi)) { bv = ov; bi = oi; }
  }
  if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
  __syncthreads();
  if (tid == 0) {
    long long b = sv[0];
    int ib = si[0];
    for (int w = 1; w < nwarps; ++w)
      if (better_bits(sv[w], si[w], b, ib)) { b = sv[w]; ib = si[w]; }
    sv[32] = b;
    si[32] = ib;
    ncand = 0;
  }
  __syncthreads();
  const double vmax = __longlong_as_double(sv[32]);
  const int pick = si[32];
  // 2. candidates within 1e-5 (relative) of it; the compensated norms are
  //    accurate to ~1e-7, so the exact leading column is among them
  const long long thr = __double_as_longlong(vmax * (1.0 - 1e-5));
  for (int i = tid; i < a.n; i += nthr) {
    if (cb[i] >= thr) {
      const int slot = atomicAdd(&ncand, 1);
      if (slot < kMaxCandidates) cand[slot] = i;
    }
  }
  __syncthreads();
  const int nc = min(ncand, kMaxCandidates);
  const bool overflow = ncand > kMaxCandidates;
  // 3. accurate norms of the candidates: the whole CTA per candidate when
  //    there are few (the usual case), one warp each otherwise
  if (nc <= 4) {
    for (int c = 0; c < nc; ++c) {
      const double e = exact_colnorm_cta<TA>(io, a.ld, a.p, cand[c], red);
      if (tid == 0) cexact[c] = e;
    }
  } else {
    for (int c = warp; c < nc; c += nwarps) {
      const double e = exact_colnorm_warp<TA>(io, a.ld, a.p, cand[c]);
      if (lane == 0) cexact[c] = e;
    }
  }
  __syncthreads();
  // 4. the best candidate by (accurate norm desc, index asc); if more than
  //    kMaxCandidates columns tie within 1e-5, keep the approximate pick
  if (tid < nc && !overflow) {
    const double v = cexact[tid];
    const int i = cand[tid];
    int rank = 0;
    for (int c = 0; c < nc; ++c)
      if (better(cexact[c], cand[c], v, i)) ++rank;
    if (rank == 0) order0 = i;
  }
  if (overflow && tid == 0) order0 = pick;
  __syncthreads();
  double cmax0 = 0.0;
  if (overflow) cmax0 = exact_colnorm_cta<TA>(io, a.ld, a.p, order0, red);
  if (tid == 0) {
    double cmax = cmax0;
    if (!overflow)
      for (int c = 0; c < nc; ++c)
        if (cand[c] == order0) cmax = cexact[c];
    st->cmax = cmax;
    const bool l1 = (a.form & 1) == 0;
    for (int j = 0; j < a.m; ++j) {
      if (io->gamma_relative) {
        const double g = io->gamma_in[j] * cmax;
        st->gamma[j] = l1 ? g : g * g;
      }
      st->start_cols[j] = (io->has_x0 || block) ? -1 : order0;
    }
    if (!(cmax > 0.0)) {  // A == 0
      for (int j = 0; j < a.m; ++j) {
        st->status[j] = GPSPCA_ZERO;
        st->active[j] = 0;
      }
      st->n_active = 0;
    }
  }
}

// P[j][r] = start column (converted, scaled) or the caller's x0.
template <typename TA>
__device__ __forceinline__ void gather_start_body(const StartArgs& a) {
  using TC = typename Elem<TA>::TC;
  const IO* io = a.io;
  const State* st = a.st;
  if (st->n_active == 0) return;
  const int j = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.p) return;
  TC* P = static_cast<TC*>(io->P);
  TC v;
  if (io->has_x0) {
    v = static_cast<const TC*>(io->x0)[static_cast<int64_t>(j) * a.p + r];
  } else if (a.form >= 2) {  // block start: Rademacher sketch
    const uint64_t k = (static_cast<uint64_t>(j) << 32) + static_cast<uint64_t>(r) + 1ull;
    v = (splitmix64(kSketchSeed, k) >> 63) ? TC(-1) : TC(1);
  } else {
    const int col = st->start_cols[j];
    v = to_tc<TA>(static_cast<const TA*>(io->A)[static_cast<int64_t>(col) * a.ld + r]);
    if (sizeof(TA) == 1) v *= io->col_scale[col];
  }
  P[static_cast<int64_t>(j) * a.p + r] = v;
}

// Sum of partials along the split index: for float data a double-float sum
// on the float pipes, rounded to float once; for double data plain double.
template <typename TC>
struct YAcc;
template <>
struct YAcc<float> {
  dd v{0.0f, 0.0f};
  __device__ __forceinline__ void add(float x) {
    const dd s = two_sum(v.hi, x);
    v = fast_two_sum(s.hi, s.lo + v.lo);
  }
  __device__ __forceinline__ void add(const YAcc& o) { v = dd_add(v, o.v); }
  __device__ __forceinline__ float rounded() const { return v.hi + v.lo; }
};
template <>
struct YAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(const YAcc& o) { v += o.v; }
  __device__ __forceinline__ double rounded() const { return v; }
};

__device__ __forceinline__ dd shfl_xor_dd(dd v, int off) {
  return dd{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

// Whether entry t is active: the decision the sweep took for its gradient
// factor, in the same precision (float compute: float t against float gamma
// and mu), so that the objective, the loadings and the iterate's g agree on
// the active set even for t within rounding of the threshold (otherwise an
// entry could count in f while its g is zero, and an all-zero g with f > 0
// would look like a degenerate step).
__device__ __forceinline__ bool active_entry(int form, float t, double gam, double mu) {
  return grad_factor<float>(form, t, static_cast<float>(gam), static_cast<float>(mu)) != 0.0f;
}
__device__ __forceinline__ bool active_entry(int form, double t, double gam, double mu) {
  return grad_factor<double>(form, t, gam, mu) != 0.0;
}

// Table 1 summand and squared unnormalised loading of one entry t: the rule
// of threshold() on the active set of active_entry(), for float t evaluated
// in double-float against the double gamma and mu given as dd (no double
// arithmetic), for double t in double.  An active entry whose value rounds
// to the threshold contributes zero.
__device__ __forceinline__ void objective_terms(int form, float t, double gam_x, double mu_x, dd gam, dd mu,
                                                dd* term, dd* z2) {
  const bool act = active_entry(form, t, gam_x, mu_x);
  if ((form & 1) == 0) {  // L1: s = [mu |t| - gamma]_+, term = s^2 = z^2
    const dd s = dd_sub(dd_mul_f(mu, fabsf(t)), gam);
    const dd sq = dd_mul(s, s);
    *term = (act && s.hi > 0.0f) ? sq : dd{0.0f, 0.0f};
    *z2 = *term;
  } else {  // L0: u = mu t, active when u^2 > gamma: term = u^2 - gamma, z = u
    const dd u = dd_mul_f(mu, t);
    const dd u2 = dd_mul(u, u);
    const dd d = dd_sub(u2, gam);
    *term = (act && d.hi > 0.0f) ? d : dd{0.0f, 0.0f};
    *z2 = act ? u2 : dd{0.0f, 0.0f};
  }
}
__device__ __forceinline__ void objective_terms(int form, double t, double gam, double mu, dd, dd, dd* term,
                                                dd* z2) {
  const Thr th = threshold(form, t, gam, mu);
  *term = dd_from_double(th.term);
  *z2 = dd_from_double(th.zr * th.zr);
}

// The per-cluster partials of rows `row` of Y columns j0 .. j0+NJ-1 (those
// below m), splits g, g + G, g + 2G, ... (G = kReduceGroups) added in that
// order into s; the loads of KS splits x NJ columns are issued before any of
// their adds (the partials' latency, not their bytes, bounds small solves).
template <typename TC, int NJ, int KS, int JY>
__device__ __forceinline__ void sum_split_partials(const TC* __restrict__ yp, int nsplit, int64_t stride, int p,
                                                   int row, int g, int j0, int m, YAcc<TC> (&s)[JY]) {
  for (int sp0 = g; sp0 < nsplit; sp0 += KS * kReduceGroups) {
    TC v[KS][NJ];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int sp = sp0 + k * kReduceGroups;
#pragma unroll
      for (int u = 0; u < NJ; ++u) {
        const int j = j0 + u;
        v[k][u] = (sp < nsplit && j < m) ? yp[sp * stride + static_cast<int64_t>(j) * p + row] : TC(0);
      }
    }
#pragma unroll
    for (int k = 0; k < KS; ++k)
#pragma unroll
      for (int u = 0; u < NJ; ++u)
        if (sp0 + k * kReduceGroups < nsplit) s[u].add(v[k][u]);
  }
}

// One reduction launch after a sweep.  Blocks [0, nyb): Y = sum of the
// per-cluster partials (fixed order) for kReduceRows rows, and those rows'
// contribution to the Gram matrix Y^T Y (packed j <= l, or the diagonal), in
// double.  Blocks [nyb, nyb + nobj) (with `objective`): a share of the Table 1
// objective and of the loadings' squared norms from T, in double-float.
template <typename TC>
__device__ __forceinline__ void reduce_body(const ReduceArgs& a) {
  if (a.st->n_active == 0) return;
  const int tid = threadIdx.x;
  const int m = a.m, p = a.p;
  if (static_cast<int>(blockIdx.x) >= a.nyb) {
    // ---- objective share: entries [i0, i1) of every active column of T
    constexpr int JB = 8;  // columns per pass
    __shared__ dd red[kReduceGroups][2 * JB];
    const int b = blockIdx.x - a.nyb;
    const int chunk = (a.n + a.nobj - 1) / a.nobj;
    const int i0 = b * chunk, i1 = min(a.n, i0 + chunk);
    const TC* T = static_cast<const TC*>(a.io->T);
    const int lane = tid & 31, warp = tid >> 5;
    for (int j0 = 0; j0 < m; j0 += JB) {
      dd acc[2 * JB];
#pragma unroll
      for (int u = 0; u < 2 * JB; ++u) acc[u] = dd{0.0f, 0.0f};
#pragma unroll
      for (int u = 0; u < JB; ++u) {
        const int j = j0 + u;
        if (j >= m || !a.st->active[j]) continue;
        const double gam = a.st->gamma[j], mu = a.io->mu[j];
        const dd gam_d = dd_from_double(gam), mu_d = dd_from_double(mu);
        const TC* col = T + static_cast<int64_t>(j) * a.n;
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
          dd term, zz;
          objective_terms(a.form, col[i], gam, mu, gam_d, mu_d, &term, &zz);
          acc[u] = dd_add(acc[u], term);
          acc[JB + u] = dd_add(acc[JB + u], zz);
        }
      }
      // reduce-scatter over the warp: lane L ends with the warp total of acc[L % 16]
#pragma unroll
      for (int h = JB; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
          const dd send = up ? acc[q] : acc[q + h];
          const dd keep = up ? acc[q + h] : acc[q];
          acc[q] = dd_add(keep, shfl_xor_dd(send, h));
        }
      }
      acc[0] = dd_add(acc[0], shfl_xor_dd(acc[0], 16));
      if (lane < 2 * JB) red[warp][lane] = acc[0];
      __syncthreads();
      if (tid < 2 * JB) {
        dd t = red[0][tid];
        for (int w = 1; w < kReduceGroups; ++w) t = dd_add(t, red[w][tid]);
        const int u = tid % JB, which = tid / JB, j = j0 + u;
        if (j < m) a.io->fpart[(static_cast<int64_t>(b) * 2 + which) * m + j] = t;
      }
      __syncthreads();
    }
    return;
  }
  // ---- Y rows and their Gram contribution
  constexpr int JY = 4;  // columns whose partial loads are in flight together
  __shared__ YAcc<TC> part[kReduceGroups][JY][kReduceRows];
  __shared__ TC Ys[kMaxM][kReduceRows];
  __shared__ TC Yo[kMaxM][kReduceRows];  // cross mode: the previous Y
  const int rl = tid % kReduceRows, g = tid / kReduceRows;
  const int row = blockIdx.x * kReduceRows + rl;
  const TC* yp = static_cast<const TC*>(a.init ? a.io->P : a.io->ypart);
  TC* Y = static_cast<TC*>(a.io->Y);
  const int64_t stride = static_cast<int64_t>(m) * p;
  for (int j0 = 0; j0 < m; j0 += JY) {
    YAcc<TC> s[JY];
    if (row < p) {
      if (m == 1)
        sum_split_partials<TC, 1, 8>(yp, a.nsplit, stride, p, row, g, j0, m, s);
      else
        sum_split_partials<TC, JY, 2>(yp, a.nsplit, stride, p, row, g, j0, m, s);
    }
#pragma unroll
    for (int u = 0; u < JY; ++u) part[g][u][rl] = s[u];
    __syncthreads();
    if (tid < JY * kReduceRows) {
      const int u = tid / kReduceRows, j = j0 + u;
      const int r2 = blockIdx.x * kReduceRows + rl;
      if (j < m) {
        YAcc<TC> t = part[0][u][rl];
        for (int g2 = 1; g2 < kReduceGroups; ++g2) t.add(part[g2][u][rl]);
        const TC tc = t.rounded();
        Ys[j][rl] = (r2 < p) ? tc : TC(0);
        if (a.cross) {
          Yo[j][rl] = (r2 < p) ? Y[static_cast<int64_t>(j) * p + r2] : TC(0);
        } else if (r2 < p) {
          Y[static_cast<int64_t>(j) * p + r2] = tc;
        }
      }
    }
    __syncthreads();
  }
  if (a.cross) {  // C[j][l] = sum_r Yold[r][j] Ynew[r][l]
    for (int q = tid; q < a.npairs; q += blockDim.x) {
      const int j = q / m, l = q % m;
      double s = 0.0;
      for (int r = 0; r < kReduceRows; ++r)
        s = fma(static_cast<double>(Yo[j][r]), static_cast<double>(Ys[l][r]), s);
      a.io->gpart[static_cast<int64_t>(blockIdx.x) * a.npairs + q] = s;
    }
    return;
  }
  for (int q = tid; q < a.npairs; q += blockDim.x) {
    int j, l;
    if (a.full_gram) {
      j = 0;
      int rem = q;
      while (rem >= m - j) { rem -= m - j; ++j; }
      l = j + rem;
    } else {
      j = l = q;
    }
    double s = 0.0;
    for (int r = 0; r < kReduceRows; ++r) s = fma(static_cast<double>(Ys[j][r]), static_cast<double>(Ys[l][r]), s);
    a.io->gpart[static_cast<int64_t>(blockIdx.x) * a.npairs + q] = s;
  }
}

// Objective, stopping test and projection weights after a sweep, or one step
// of the start (projection of the start, Rayleigh-Ritz rotation).  One CTA:
// sums and stopping test in double, the m x m eigenproblems in double-float.
__device__ __forceinline__ void finish_body(const FinishArgs& a) {
  extern __shared__ double fsm[];
  State* st = a.st;
  const IO* io = a.io;
  const int tid = threadIdx.x;
  const int m = a.m;
  const bool block = a.form >= 2;
  __shared__ int s_stop;
  double* gsum = fsm;                    // npairs
  double* fz = gsum + a.npairs;          // 2m
  double* Wt = fz + 2 * m;               // m*m
  double* jac = Wt + m * m;              // Jacobi workspace (finish_smem_doubles)
  const bool proceed = st->n_active > 0;
  if (proceed) {
    sum_partials(io->gpart, a.nblk, a.npairs, a.npairs, gsum);
    if (a.mode == kFinishIterate) sum_partials(io->fpart, a.nsplit, 2 * m, 2 * m, fz);
  }
  if (proceed && (a.mode == kFinishRitz || a.mode == kFinishRitzT)) {
    ritz_weights(gsum, m, st->W, Wt, jac, a.mode == kFinishRitzT, a.mode == kFinishRitzT ? st->R : nullptr);
    for (int idx = tid; idx < m * m; idx += blockDim.x) st->W[idx] = Wt[idx];
  } else if (proceed && a.mode == kFinishPolar) {
    if (block) {
      const bool ok = polar_weights(gsum, m, st->W, jac, st->has_v ? st->V : nullptr, st->V);
      if (tid == 0) {
        if (ok) {
          st->has_v = 1;
        } else {
          for (int j = 0; j < m; ++j) { st->status[j] = GPSPCA_DEGENERATE; st->active[j] = 0; }
          st->n_active = 0;
          st->any_degenerate = 1;
        }
      }
    } else {  // one thread per component
      const int j = tid;
      bool live = false;
      if (j < m) {
        for (int l = 0; l < m; ++l) st->W[l * m + j] = 0.0;
        const double d = gsum[j];
        if (d > 0.0) {
          st->W[j * m + j] = rsqrt_refined(d);
          live = true;
        } else {
          st->status[j] = GPSPCA_DEGENERATE;
          st->active[j] = 0;
          st->any_degenerate = 1;
        }
      }
      const int na = __syncthreads_count(live);
      if (tid == 0) st->n_active = na;
    }
  } else if (proceed) {
    const int k = st->k;
    const double tol = io->tol;
    const int maxit = io->maxit;
    if (block) {
      if (tid == 0) {
        double f = 0.0;
        for (int j = 0; j < m; ++j) f += fz[j];
        int s = stop_rule(k, f, st->f_prev[0], tol, maxit);
        if (!isfinite(f)) {
          st->error |= kErrNonFinite;
          s = GPSPCA_MAXIT;
        }
        s_stop = s;
        if (s < 0) st->f_prev[0] = f;
      }
      __syncthreads();
      bool deg = false;
      if (s_stop < 0) {
        deg = !polar_weights(gsum, m, st->W, jac, st->has_v ? st->V : nullptr, st->V);
      }
      if (s_stop >= 0 || deg) {
        const int j = tid;
        if (j < m) {
          st->status[j] = deg ? GPSPCA_DEGENERATE : s_stop;
          st->iters[j] = k + 1;
          st->f[j] = fz[j];
          st->znorm2[j] = fz[m + j];
          st->active[j] = 0;
        }
        if (tid == 0) {
          if (deg) st->any_degenerate = 1;
          st->n_active = 0;
        }
      }
    } else {  // one thread per component (gamma path: independent solves)
      const int j = tid;
      bool live = false;
      if (j < m && st->active[j]) {
        const double f = fz[j];
        int s = stop_rule(k, f, st->f_prev[j], tol, maxit);
        if (!isfinite(f)) {
          atomicOr(&st->error, kErrNonFinite);
          s = GPSPCA_MAXIT;
        }
        bool deg = false;
        if (s < 0) {
          const double d = gsum[j];
          if (d > 0.0) {
            st->W[j * m + j] = rsqrt_refined(d);
            st->f_prev[j] = f;
            live = true;
          } else {
            deg = true;
          }
        }
        if (!live) {
          st->status[j] = deg ? GPSPCA_DEGENERATE : s;
          st->iters[j] = k + 1;
          st->f[j] = f;
          st->znorm2[j] = fz[m + j];
          st->active[j] = 0;
          st->W[j * m + j] = 0.0;
          if (deg) st->any_degenerate = 1;
        }
      } else if (j < m) {
        st->W[j * m + j] = 0.0;
      }
      const int na = __syncthreads_count(live);
      if (tid == 0) st->n_active = na;
    }
    if (tid == 0) st->k = k + 1;
  }
  __syncthreads();
  if (tid == 0 && a.mode != kFinishIterate && a.last) st->k = 0;
  if (tid == 0 && a.use_cond) cudaGraphSetConditional(a.cond, st->n_active > 0 ? 1u : 0u);
}

// Loadings from the last sweep's T (Table 1, original form): threshold,
// scale each column to unit norm, support bitmap; plus the scalar outputs.
template <typename TC>
__device__ __forceinline__ void finalize_body(const IO* io, const State* st, int p, int n, int m, int form) {
  const int j = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int it = st->iters[j];
  const double z2 = st->znorm2[j];
  const double inv = z2 > 0.0 ? 1.0 / sqrt(z2) : 0.0;
  const double gam = st->gamma[j];
  const double mu = io->mu[j];
  const TC* T = static_cast<const TC*>(io->T);
  TC z = 0;
  if (i < n && it > 0) {
    const TC t = T[static_cast<int64_t>(j) * n + i];
    if (active_entry(form, t, gam, mu)) {  // the active set of the objective and of g
      const Thr th = threshold(form, static_cast<double>(t), gam, mu);
      z = static_cast<TC>(th.zr * inv);
    }
  }
  if (i < n) static_cast<TC*>(io->Z)[static_cast<int64_t>(j) * n + i] = z;
  const unsigned bits = __ballot_sync(0xffffffffu, i < n && z != TC(0));
  if (io->support && (threadIdx.x & 31) == 0 && i < n) {
    const int nw = (n + 31) / 32;
    io->support[static_cast<int64_t>(j) * nw + i / 32] = bits;
  }
  if (i < p && it == 0) static_cast<TC*>(io->X)[static_cast<int64_t>(j) * p + i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    io->objective[j] = st->f[j];
    io->iters[j] = st->iters[j];
    io->status[j] = st->status[j];
    if (io->gamma_abs) io->gamma_abs[j] = st->gamma[j];
  }
}

// ---------------------------------------------------------------- launchers

// ---------------------------------------------------------------- entry kernels
//
// Each step as a kernel of one solve, and as a kernel of a group of
// same-shape solves (`*_grouped`): instance blockIdx.z of the group, its IO
// and State from the group's pointer arrays, the rest of the arguments shared.

__global__ void reset_state_kernel(const IO* io, State* st, int m, int form) { reset_state_body(io, st, m, form); }
__global__ void reset_state_grouped(GroupPtrs g, int m, int form) {
  reset_state_body(g.io[blockIdx.z], g.st[blockIdx.z], m, form);
}

template <typename TA>
__global__ void colnorm_kernel(const IO* io, State* st, int64_t ld, int p, int n, int fast) {
  colnorm_body<TA>(io, st, ld, p, n, fast);
}
template <typename TA>
__global__ void colnorm_grouped(GroupPtrs g, int64_t ld, int p, int n, int fast) {
  colnorm_body<TA>(g.io[blockIdx.z], g.st[blockIdx.z], ld, p, n, fast);
}
// column norms of a matrix that several solves of a batch share, into out
// (the same per-column arithmetic as colnorm_kernel, so the same values)
template <typename TA>
__global__ void colnorm_shared_kernel(const void* A, const float* col_scale, double* out, int32_t* error,
                                      int64_t ld, int p, int n, int fast) {
  colnorm_core<TA>(static_cast<const TA*>(A), col_scale, out, error, ld, p, n, fast);
}
// a solve's column norms taken from the batch's shared ones, with the
// non-finite check its own norm pass would have made
__global__ void copy_norms_kernel(const IO* io, State* st, int n) {
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double c = io->cnorm_src[i];
    if (!isfinite(c)) bad = true;
    io->cnorm[i] = c;
  }
  if (bad) atomicOr(&st->error, static_cast<int>(kErrNonFinite));
}

template <typename TA>
__global__ void __launch_bounds__(kStartThreads) select_start_kernel(const StartArgs a) { select_start_body<TA>(a); }
template <typename TA>
__global__ void __launch_bounds__(kStartThreads) select_start_grouped(StartArgs a, GroupPtrs g) {
  a.io = g.io[blockIdx.z];
  a.st = g.st[blockIdx.z];
  select_start_body<TA>(a);
}

template <typename TA>
__global__ void gather_start_kernel(const StartArgs a) { gather_start_body<TA>(a); }
template <typename TA>
__global__ void gather_start_grouped(StartArgs a, GroupPtrs g) {
  a.io = g.io[blockIdx.z];
  a.st = g.st[blockIdx.z];
  gather_start_body<TA>(a);
}

template <typename TC>
__global__ void __launch_bounds__(kReduceRows* kReduceGroups) reduce_kernel(const ReduceArgs a) { reduce_body<TC>(a); }
template <typename TC>
__global__ void __launch_bounds__(kReduceRows* kReduceGroups) reduce_grouped(ReduceArgs a, GroupPtrs g) {
  a.io = g.io[blockIdx.z];
  a.st = g.st[blockIdx.z];
  reduce_body<TC>(a);
}

__global__ void __launch_bounds__(kFinishThreads, 1) finish_kernel(const FinishArgs a) { finish_body(a); }
__global__ void __launch_bounds__(kFinishThreads, 1) finish_grouped(FinishArgs a, GroupPtrs g) {
  a.io = g.io[blockIdx.z];
  a.st = g.st[blockIdx.z];
  finish_body(a);
}

template <typename TC>
__global__ void finalize_kernel(const IO* io, const State* st, int p, int n, int m, int form) {
  finalize_body<TC>(io, st, p, n, m, form);
}
template <typename TC>
__global__ void finalize_grouped(GroupPtrs g, int p, int n, int m, int form) {
  finalize_body<TC>(g.io[blockIdx.z], g.st[blockIdx.z], p, n, m, form);
}

// The loop condition of a group: another sweep while any instance is active.
__global__ void group_cond_kernel(GroupPtrs g, int count, cudaGraphConditionalHandle h) {
  int any = 0;
  for (int i = threadIdx.x; i < count; i += 32) any |= g.st[i]->n_active > 0 ? 1 : 0;
  any = __any_sync(0xffffffffu, any);
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// ---------------------------------------------------------------- launchers

void launch_reset(const IO* io, State* st, int m, int form, cudaStream_t s) {
  reset_state_kernel<<<1, kMaxM, 0, s>>>(io, st, m, form);
}

template <typename TA>
static void colnorm_t(const IO* io, State* st, int64_t ld, int p, int n, int fast, cudaStream_t s) {
  const int blocks = std::max(1, std::min((n + 7) / 8, 4096));
  colnorm_kernel<TA><<<blocks, 256, 0, s>>>(io, st, ld, p, n, fast);
}

void launch_colnorm(int dtype, const IO* io, State* st, int64_t ld, int p, int n, int fast, cudaStream_t s) {
  switch (dtype) {
    case GPSPCA_F32: colnorm_t<float>(io, st, ld, p, n, fast, s); break;
    case GPSPCA_F64: colnorm_t<double>(io, st, ld, p, n, fast, s); break;
    case GPSPCA_BF16: colnorm_t<__nv_bfloat16>(io, st, ld, p, n, fast, s); break;
    default: colnorm_t<__nv_fp8_e4m3>(io, st, ld, p, n, fast, s); break;
  }
}

template <typename TA>
static void colnorm_shared_t(const void* A, const float* col_scale, double* out, int32_t* error, int64_t ld, int p,
                             int n, int fast, cudaStream_t s) {
  const int blocks = std::max(1, std::min((n + 7) / 8, 4096));
  colnorm_shared_kernel<TA><<<blocks, 256, 0, s>>>(A, col_scale, out, error, ld, p, n, fast);
}

void launch_colnorm_shared(int dtype, const void* A, const float* col_scale, double* out, int32_t* error,
                           int64_t ld, int p, int n, int fast, cudaStream_t s) {
  switch (dtype) {
    case GPSPCA_F32: colnorm_shared_t<float>(A, col_scale, out, error, ld, p, n, fast, s); break;
    case GPSPCA_F64: colnorm_shared_t<double>(A, col_scale, out, error, ld, p, n, fast, s); break;
    case GPSPCA_BF16: colnorm_shared_t<__nv_bfloat16>(A, col_scale, out, error, ld, p, n, fast, s); break;
    default: colnorm_shared_t<__nv_fp8_e4m3>(A, col_scale, out, error, ld, p, n, fast, s); break;
  }
}

void launch_copy_norms(const IO* io, State* st, int n, cudaStream_t s) {
  copy_norms_kernel<<<std::max(1, std::min((n + 255) / 256, 1024)), 256, 0, s>>>(io, st, n);
}

void launch_select_start(int dtype, const StartArgs& a, cudaStream_t s) {
  switch (dtype) {
    case GPSPCA_F32: select_start_kernel<float><<<1, kStartThreads, 0, s>>>(a); break;
    case GPSPCA_F64: select_start_kernel<double><<<1, kStartThreads, 0, s>>>(a); break;
    case GPSPCA_BF16: select_start_kernel<__nv_bfloat16><<<1, kStartThreads, 0, s>>>(a); break;
    default: select_start_kernel<__nv_fp8_e4m3><<<1, kStartThreads, 0, s>>>(a); break;
  }
}

void launch_gather_start(int dtype, const StartArgs& a, cudaStream_t s) {
  const dim3 grid((a.p + 255) / 256, a.m);
  switch (dtype) {
    case GPSPCA_F32: gather_start_kernel<float><<<grid, 256, 0, s>>>(a); break;
    case GPSPCA_F64: gather_start_kernel<double><<<grid, 256, 0, s>>>(a); break;
    case GPSPCA_BF16: gather_start_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(a); break;
    default: gather_start_kernel<__nv_fp8_e4m3><<<grid, 256, 0, s>>>(a); break;
  }
}

void launch_reduce(int tcsize, const ReduceArgs& a, cudaStream_t s) {
  const int nblk = a.nyb + (a.objective ? a.nobj : 0);
  if (tcsize == 8)
    reduce_kernel<double><<<nblk, kReduceRows * kReduceGroups, 0, s>>>(a);
  else
    reduce_kernel<float><<<nblk, kReduceRows * kReduceGroups, 0, s>>>(a);
}

void launch_finish(const FinishArgs& a, int smem, cudaStream_t s) {
  static bool once = [] {
    cudaFuncSetAttribute(finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinishMaxSmem);
    return true;
  }();
  (void)once;
  finish_kernel<<<1, kFinishThreads, smem, s>>>(a);
}

// Block forms on the CUDA cores: the iterate X = Y W of the next sweep (the
// projection of Section 2: Y (Y^T Y)^{-1/2} for the polar step, the
// Rayleigh-Ritz rotation after the start), one thread per (row, component).
// Float compute carries W as a high and a low float part and every
// product's and sum's rounding error in a second accumulator (Dekker's
// exact product by fma, Knuth's two-sum), so X is Y W rounded once to float
// even where W's entries (up to lambda_min(Y^T Y)^{-1/2}) make the sum
// cancel; double compute sums in double.
template <typename TC>
__global__ void form_x_kernel(const IO* io, const State* st, int p, int m) {
  __shared__ double wj[kMaxM];
  const int j = blockIdx.y;
  if (threadIdx.x < m) wj[threadIdx.x] = st->W[threadIdx.x * m + j];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p) return;
  const TC* Y = static_cast<const TC*>(io->Y);
  TC* X = static_cast<TC*>(io->Xf);
  if constexpr (sizeof(TC) == 8) {
    double x = 0.0;
    for (int l = 0; l < m; ++l) x += Y[static_cast<int64_t>(l) * p + r] * wj[l];
    X[static_cast<int64_t>(j) * p + r] = x;
  } else {
    float x = 0.0f, xe = 0.0f;
    for (int l = 0; l < m; ++l) {
      const float yv = Y[static_cast<int64_t>(l) * p + r];
      const float wh = static_cast<float>(wj[l]);
      const float wl = static_cast<float>(wj[l] - static_cast<double>(wh));
      const float pr = __fmul_rn(yv, wh);
      const float pe = fmaf(yv, wh, -pr);  // y w_hi = pr + pe exactly
      const float s2 = __fadd_rn(x, pr);
      const float bb = __fsub_rn(s2, x);
      const float se = __fadd_rn(__fsub_rn(x, __fsub_rn(s2, bb)), __fsub_rn(pr, bb));  // x + pr = s2 + se
      x = s2;
      xe += pe + se + yv * wl;
    }
    X[static_cast<int64_t>(j) * p + r] = __fadd_rn(x, xe);
  }
}

void launch_form_x(int tcsize, const IO* io, const State* st, int p, int m, cudaStream_t s) {
  const dim3 grid((p + 255) / 256, m);
  if (tcsize == 8)
    form_x_kernel<double><<<grid, 256, 0, s>>>(io, st, p, m);
  else
    form_x_kernel<float><<<grid, 256, 0, s>>>(io, st, p, m);
}

// T^T T, block b over columns [kGramTCols b, kGramTCols (b+1)) of T: the
// block's columns of every component in shared memory (rows padded by one
// float against bank conflicts), one (j, l >= j) pair per thread at a time,
// each product exact (Dekker) and the sum in double-float; written to both
// halves of the m x m partial.
__global__ void __launch_bounds__(256) gram_t_kernel(const IO* io, const State* st, int m, int n) {
  extern __shared__ float ts[];
  constexpr int W = kGramTCols, LD = kGramTCols + 1;
  if (st->n_active == 0) return;
  const int i0 = blockIdx.x * W, w = min(W, n - i0);
  const float* T = static_cast<const float*>(io->T);
  for (int idx = threadIdx.x; idx < m * W; idx += blockDim.x) {
    const int j = idx / W, i = idx - j * W;
    ts[j * LD + i] = i < w ? T[static_cast<int64_t>(j) * n + i0 + i] : 0.0f;
  }
  __syncthreads();
  const int npairs = m * (m + 1) / 2;
  double* out = io->gpart + static_cast<int64_t>(blockIdx.x) * m * m;
  for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
    int j = 0, rem = q;
    while (rem >= m - j) {
      rem -= m - j;
      ++j;
    }
    const int l = j + rem;
    const float* a = ts + j * LD;
    const float* b = ts + l * LD;
    dd s{0.0f, 0.0f};
    for (int i = 0; i < w; ++i) {
      const float pr = __fmul_rn(a[i], b[i]);
      s = dd_add(s, dd{pr, fmaf(a[i], b[i], -pr)});
    }
    const double v = dd_to_double(s);
    out[j * m + l] = v;
    out[l * m + j] = v;
  }
}

void launch_gram_t(const IO* io, const State* st, int m, int n, cudaStream_t s) {
  const int smem = static_cast<int>(sizeof(float)) * m * (kGramTCols + 1);
  static bool once = [] {
    cudaFuncSetAttribute(gram_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * (kGramTCols + 1) * 4);
    return true;
  }();
  (void)once;
  gram_t_kernel<<<gram_t_blocks(n), 256, smem, s>>>(io, st, m, n);
}

void launch_finalize(int tcsize, const IO* io, const State* st, int p, int n, int m, int form, cudaStream_t s) {
  const int len = std::max(n, p);
  const dim3 grid((len + 255) / 256, m);
  if (tcsize == 8)
    finalize_kernel<double><<<grid, 256, 0, s>>>(io, st, p, n, m, form);
  else
    finalize_kernel<float><<<grid, 256, 0, s>>>(io, st, p, n, m, form);
}

// ---- the same launches for a group of `count` same-shape solves

void launch_reset_g(GroupPtrs g, int count, int m, int form, cudaStream_t s) {
  reset_state_grouped<<<dim3(1, 1, count), kMaxM, 0, s>>>(g, m, form);
}

template <typename TA>
static void colnorm_g_t(GroupPtrs g, int count, int64_t ld, int p, int n, int fast, cudaStream_t s) {
  const int blocks = std::max(1, std::min((n + 7) / 8, 4096));
  colnorm_grouped<TA><<<dim3(blocks, 1, count), 256, 0, s>>>(g, ld, p, n, fast);
}

void launch_colnorm_g(int dtype, GroupPtrs g, int count, int64_t ld, int p, int n, int fast, cudaStream_t s) {
  switch (dtype) {
    case GPSPCA_F32: colnorm_g_t<float>(g, count, ld, p, n, fast, s); break;
    case GPSPCA_F64: colnorm_g_t<double>(g, count, ld, p, n, fast, s); break;
    case GPSPCA_BF16: colnorm_g_t<__nv_bfloat16>(g, count, ld, p, n, fast, s); break;
    default: colnorm_g_t<__nv_fp8_e4m3>(g, count, ld, p, n, fast, s); break;
  }
}

void launch_select_start_g(int dtype, const StartArgs& a, GroupPtrs g, int count, cudaStream_t s) {
  const dim3 grid(1, 1, count);
  switch (dtype) {
    case GPSPCA_F32: select_start_grouped<float><<<grid, kStartThreads, 0, s>>>(a, g); break;
    case GPSPCA_F64: select_start_grouped<double><<<grid, kStartThreads, 0, s>>>(a, g); break;
    case GPSPCA_BF16: select_start_grouped<__nv_bfloat16><<<grid, kStartThreads, 0, s>>>(a, g); break;
    default: select_start_grouped<__nv_fp8_e4m3><<<grid, kStartThreads, 0, s>>>(a, g); break;
  }
}

void launch_gather_start_g(int dtype, const StartArgs& a, GroupPtrs g, int count, cudaStream_t s) {
  const dim3 grid((a.p + 255) / 256, a.m, count);
  switch (dtype) {
    case GPSPCA_F32: gather_start_grouped<float><<<grid, 256, 0, s>>>(a, g); break;
    case GPSPCA_F64: gather_start_grouped<double><<<grid, 256, 0, s>>>(a, g); break;
    case GPSPCA_BF16: gather_start_grouped<__nv_bfloat16><<<grid, 256, 0, s>>>(a, g); break;
    default: gather_start_grouped<__nv_fp8_e4m3><<<grid, 256, 0, s>>>(a, g); break;
  }
}

void launch_reduce_g(int tcsize, const ReduceArgs& a, GroupPtrs g, int count, cudaStream_t s) {
  const dim3 grid(a.nyb + (a.objective ? a.nobj : 0), 1, count);
  if (tcsize == 8)
    reduce_grouped<double><<<grid, kReduceRows * kReduceGroups, 0, s>>>(a, g);
  else
    reduce_grouped<float><<<grid, kReduceRows * kReduceGroups, 0, s>>>(a, g);
}

void launch_finish_g(const FinishArgs& a, int smem, GroupPtrs g, int count, cudaStream_t s) {
  static bool once = [] {
    cudaFuncSetAttribute(finish_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinishMaxSmem);
    return true;
  }();
  (void)once;
  finish_grouped<<<dim3(1, 1, count), kFinishThreads, smem, s>>>(a, g);
}

void launch_finalize_g(int tcsize, GroupPtrs g, int count, int p, int n, int m, int form, cudaStream_t s) {
  const int len = std::max(n, p);
  const dim3 grid((len + 255) / 256, m, count);
  if (tcsize == 8)
    finalize_grouped<double><<<grid, 256, 0, s>>>(g, p, n, m, form);
  else
    finalize_grouped<float><<<grid, 256, 0, s>>>(g, p, n, m, form);
}

void launch_group_cond(GroupPtrs g, int count, cudaGraphConditionalHandle h, cudaStream_t s) {
  group_cond_kernel<<<1, 32, 0, s>>>(g, count, h);
}

}  // namespace gpspca
