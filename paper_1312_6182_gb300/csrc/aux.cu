// Kernels around the fused sweep (see aux.cuh).
#include <algorithm>

#include "aux.cuh"

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
// (per q: strided over tpp lanes, then a shuffle tree), so the result does not
// depend on scheduling.  All threads of the block must call it.
__device__ void sum_partials(const double* __restrict__ src, int nb, int stride, int nq, double* dst) {
  int tpp = 32;
  while (tpp > 1 && tpp * nq > static_cast<int>(blockDim.x)) tpp >>= 1;
  const int groups = blockDim.x / tpp;
  const int sub = threadIdx.x % tpp;
  for (int q0 = 0; q0 < nq; q0 += groups) {
    const int q = q0 + static_cast<int>(threadIdx.x) / tpp;
    double s = 0.0;
    if (q < nq)
      for (int b = sub; b < nb; b += tpp) s += src[static_cast<int64_t>(b) * stride + q];
    for (int off = tpp / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, tpp);
    if (q < nq && sub == 0) dst[q] = s;
  }
  __syncthreads();
}

__device__ double block_sum(double v, double* scratch) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += scratch[w];
    scratch[32] = t;
  }
  __syncthreads();
  t = scratch[32];
  __syncthreads();
  return t;
}

// Cyclic Jacobi eigensolver for a symmetric mm x mm matrix G (mm even) in
// shared memory, FP64.  Each round applies mm/2 disjoint rotations chosen by
// the round-robin (tournament) ordering, rows then columns, accumulating the
// eigenvectors in V.  On return diag(G) holds the eigenvalues.
__device__ void jacobi_eig(double* G, double* V, int mm, int* rp, int* rq, double* rc, double* rs,
                           double* scratch) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int idx = tid; idx < mm * mm; idx += nthr) V[idx] = (idx / mm == idx % mm) ? 1.0 : 0.0;
  __syncthreads();
  const int half = mm / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int idx = tid; idx < mm * mm; idx += nthr) {
      const int r = idx / mm, c = idx % mm;
      const double g = G[idx];
      if (r < c) off += g * g;
      if (r == c) dg += g * g;
    }
    off = block_sum(off, scratch);
    dg = block_sum(dg, scratch);
    if (!(off > 1e-32 * dg)) break;  // relative off-diagonal size below ~1e-16
    for (int round = 0; round < mm - 1; ++round) {
      if (tid < half) {
        const int k = tid;
        const int a = (k == 0) ? 0 : ((k - 1 + round) % (mm - 1)) + 1;
        const int b = ((mm - 2 - k + round) % (mm - 1)) + 1;
        const int pp = min(a, b), qq = max(a, b);
        const double apq = G[pp * mm + qq];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          // tan(theta) of the rotation that zeroes G_pq, in float (its
          // transcendentals are cheap; an angle good to 1e-7 still cuts G_pq
          // by 1e-7), then cos/sin refined in double so the rotation is
          // orthogonal to double rounding
          const double app = G[pp * mm + pp], aqq = G[qq * mm + qq];
          const double num = aqq - app, den = 2.0 * apq;
          float tau;
          if (fabs(den) > 1e-30 && fabs(den) < 1e30 && fabs(num) < 1e30) {
            tau = static_cast<float>(num) / static_cast<float>(den);  // may round to +-inf: no rotation
          } else {
            tau = static_cast<float>(fmax(fmin(num / den, 1e30), -1e30));
          }
          const float at = fabsf(tau);
          float t = (at > 1e18f) ? 0.5f / at : 1.0f / (at + sqrtf(1.0f + at * at));
          if (tau < 0.0f) t = -t;
          c = rsqrt_refined(1.0 + static_cast<double>(t) * t);
          s = static_cast<double>(t) * c;
        }
        rp[k] = pp; rq[k] = qq; rc[k] = c; rs[k] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < half * mm; idx += nthr) {  // rows: G <- J^T G
        const int k = idx / mm, l = idx % mm;
        const int pp = rp[k], qq = rq[k];
        const double c = rc[k], s = rs[k];
        const double gp = G[pp * mm + l], gq = G[qq * mm + l];
        G[pp * mm + l] = c * gp - s * gq;
        G[qq * mm + l] = s * gp + c * gq;
      }
      __syncthreads();
      for (int idx = tid; idx < half * mm; idx += nthr) {  // columns: G <- G J, V <- V J
        const int k = idx / mm, l = idx % mm;
        const int pp = rp[k], qq = rq[k];
        const double c = rc[k], s = rs[k];
        const double gp = G[l * mm + pp], gq = G[l * mm + qq];
        G[l * mm + pp] = c * gp - s * gq;
        G[l * mm + qq] = s * gp + c * gq;
        const double vp = V[l * mm + pp], vq = V[l * mm + qq];
        V[l * mm + pp] = c * vp - s * vq;
        V[l * mm + qq] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// Polar weights W = (Y^T Y)^{-1/2} from the Gram matrix (packed j <= l).
// With Vwarm (the eigenvectors of the previous iteration's Gram matrix) the
// Jacobi sweeps run on Vwarm^T G Vwarm, which is nearly diagonal near
// convergence; the eigenvectors found are written back to Vout.
// Returns false (degenerate) if lambda_min <= 1e-12 lambda_max.
__device__ bool polar_weights(const double* gsum, int m, double* W, double* sm, double* scratch,
                              const double* Vwarm, double* Vout) {
  const int mm = m + (m & 1);
  double* G = sm;
  double* V = sm + mm * mm;
  int* rp = reinterpret_cast<int*>(V + mm * mm);
  int* rq = rp + 32;
  double* rc = reinterpret_cast<double*>(rq + 32);
  double* rs = rc + 32;
  double* lam = rs + 32;
  double* Gf = lam + kMaxM;  // full G (m x m), for the warm start
  __shared__ int deg;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int r = idx / m, c = idx % m;
    const int j = min(r, c), l = max(r, c);
    Gf[idx] = gsum[j * m - j * (j - 1) / 2 + (l - j)];  // packed upper-triangle index
  }
  __syncthreads();
  if (Vwarm) {  // G <- Vwarm^T G Vwarm, via V as temporary for G Vwarm
    for (int idx = tid; idx < m * m; idx += nthr) {
      const int r = idx / m, c = idx % m;
      double t = 0.0;
      for (int k = 0; k < m; ++k) t += Gf[r * m + k] * Vwarm[k * m + c];
      V[idx] = t;
    }
    __syncthreads();
    for (int idx = tid; idx < mm * mm; idx += nthr) {
      const int r = idx / mm, c = idx % mm;
      double t = 0.0;
      if (r < m && c < m)
        for (int k = 0; k < m; ++k) t += Vwarm[k * m + r] * V[k * m + c];
      G[idx] = t;
    }
    __syncthreads();
    for (int idx = tid; idx < mm * mm; idx += nthr) {  // exact symmetry
      const int r = idx / mm, c = idx % mm;
      if (r < c) G[c * mm + r] = G[idx];
    }
  } else {
    for (int idx = tid; idx < mm * mm; idx += nthr) {
      const int r = idx / mm, c = idx % mm;
      G[idx] = (r < m && c < m) ? Gf[r * m + c] : 0.0;
    }
  }
  __syncthreads();
  jacobi_eig(G, V, mm, rp, rq, rc, rs, scratch);
  if (tid < m) lam[tid] = G[tid * mm + tid];
  __syncthreads();
  // eigenvectors of the Gram matrix: Vwarm * V (or V), kept in Gf
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int r = idx / m, c = idx % m;
    double t;
    if (Vwarm) {
      t = 0.0;
      for (int k = 0; k < m; ++k) t += Vwarm[r * m + k] * V[k * mm + c];
    } else {
      t = V[r * mm + c];
    }
    Gf[idx] = t;
  }
  if (tid == 0) {
    double lmax = 0.0, lmin = 1e308;
    for (int i = 0; i < m; ++i) {
      lmax = fmax(lmax, lam[i]);
      lmin = fmin(lmin, lam[i]);
    }
    deg = !(lmax > 0.0) || !(lmin > 1e-12 * lmax);
  }
  __syncthreads();
  if (deg) return false;
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int a = idx / m, b = idx % m;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += Gf[a * m + i] * Gf[b * m + i] * rsqrt_refined(lam[i]);
    W[a * m + b] = s;
    if (Vout) Vout[idx] = Gf[idx];
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------- kernels

__global__ void reset_state_kernel(const IO* io, State* st, int m, int form) {
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
// exact FP64 norms of the leading candidates are recomputed by
// select_start_kernel before any decision is taken on them.  One warp per
// column.  A non-finite norm flags the solve.
template <typename TA>
__global__ void colnorm_kernel(const IO* io, State* st, int64_t ld, int p, int n, int fast) {
  double* cnorm = io->cnorm;
  using TC = typename Elem<TA>::TC;
  constexpr int NW = Wide<TA>::N;
  const TA* __restrict__ A = static_cast<const TA*>(io->A);
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
      if (sizeof(TA) == 1) c *= static_cast<double>(io->col_scale[i]);
      if (!isfinite(c)) bad = true;
      cnorm[i] = c;
    }
  }
  if (bad) atomicOr(&st->error, static_cast<int>(kErrNonFinite));
}

// Exact FP64 norm of column i (used for the start decision and gamma scale).
template <typename TA>
__device__ double exact_colnorm_warp(const IO* io, int64_t ld, int p, int i) {
  const TA* col = static_cast<const TA*>(io->A) + static_cast<int64_t>(i) * ld;
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // independent chains
  int r = lane;
  for (; r + 96 < p; r += 128) {
    const double v0 = static_cast<double>(to_tc<TA>(col[r]));
    const double v1 = static_cast<double>(to_tc<TA>(col[r + 32]));
    const double v2 = static_cast<double>(to_tc<TA>(col[r + 64]));
    const double v3 = static_cast<double>(to_tc<TA>(col[r + 96]));
    s0 += v0 * v0;
    s1 += v1 * v1;
    s2 += v2 * v2;
    s3 += v3 * v3;
  }
  for (; r < p; r += 32) {
    const double v = static_cast<double>(to_tc<TA>(col[r]));
    s0 += v * v;
  }
  double s = (s0 + s1) + (s2 + s3);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  double c = sqrt(s);
  if (sizeof(TA) == 1) c *= static_cast<double>(io->col_scale[i]);
  return c;
}

// (value desc, index asc) ordering helpers for the block-wide argmax.
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  return (v > bv) || (v == bv && i < bi);
}

__device__ void block_argmax(double& v, int& i, double* sv, int* si) {
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, i, off);
    if (better(ov, oi, v, i)) { v = ov; i = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sv[warp] = v; si[warp] = i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = sv[0];
    int bi = si[0];
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w)
      if (better(sv[w], si[w], bv, bi)) { bv = sv[w]; bi = si[w]; }
    sv[32] = bv; si[32] = bi;
  }
  __syncthreads();
  v = sv[32];
  i = si[32];
  __syncthreads();
}

// Start of the iteration (step a0): the largest-norm column (single-unit) or
// the m largest-norm columns in decreasing order (block), ties to the lower
// index, decided on exact FP64 norms; gamma scaled by max_i ||a_i|| when
// relative.  One CTA.
template <typename TA>
__global__ void __launch_bounds__(kStartThreads) select_start_kernel(const StartArgs a) {
  const IO* io = a.io;
  State* st = a.st;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  __shared__ double sv[33];
  __shared__ int si[33];
  __shared__ int cand[kMaxCandidates];
  __shared__ double cexact[kMaxCandidates];
  __shared__ int ncand;
  __shared__ int order[kMaxM];
  __shared__ double vm;
  __shared__ int picks[kMaxM];
  if (st->error) {
    if (tid == 0) st->n_active = 0;
    return;
  }
  const bool block = a.form >= 2;
  // only the largest column is needed: it is the single-unit start, and
  // max_i ||a_i|| scales a relative gamma (block forms start from the sketch)
  const int mt = 1;
  // 1. the mt-th largest approximate norm, by mt rounds of arg-max below the previous pick
  double pv = 1e308;
  int pi = -1;
  for (int r = 0; r < mt; ++r) {
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int i = tid; i < a.n; i += nthr) {
      const double v = io->cnorm[i];
      const bool below = (v < pv) || (v == pv && i > pi);
      if (below && better(v, i, bv, bi)) { bv = v; bi = i; }
    }
    block_argmax(bv, bi, sv, si);
    pv = bv;
    pi = bi;
    if (tid == 0) picks[r] = bi;
  }
  if (tid == 0) { vm = pv; ncand = 0; }
  __syncthreads();
  // 2. candidates within 1e-5 (relative) of it; the compensated norms are
  //    accurate to ~1e-7, so the exact leading columns are all among them
  const double thr = vm * (1.0 - 1e-5);
  for (int i = tid; i < a.n; i += nthr) {
    if (io->cnorm[i] >= thr) {
      const int slot = atomicAdd(&ncand, 1);
      if (slot < kMaxCandidates) cand[slot] = i;
    }
  }
  __syncthreads();
  const int nc = min(ncand, kMaxCandidates);
  const bool overflow = ncand > kMaxCandidates;
  // 3. exact FP64 norms of the candidates (one warp each)
  for (int c = warp; c < nc; c += nwarps) {
    const double e = exact_colnorm_warp<TA>(io, a.ld, a.p, cand[c]);
    if (lane == 0) cexact[c] = e;
  }
  __syncthreads();
  // 4. rank candidates by (exact norm desc, index asc); if more than
  //    kMaxCandidates columns tie within 1e-5, keep the approximate order
  if (tid < nc && !overflow) {
    const double v = cexact[tid];
    const int i = cand[tid];
    int rank = 0;
    for (int c = 0; c < nc; ++c)
      if (better(cexact[c], cand[c], v, i)) ++rank;
    if (rank < mt) order[rank] = cand[tid];
  }
  if (overflow && tid < mt) order[tid] = picks[tid];
  __syncthreads();
  double cmax0 = 0.0;
  if (overflow && warp == 0) cmax0 = exact_colnorm_warp<TA>(io, a.ld, a.p, order[0]);
  if (tid == 0) {
    double cmax = cmax0;
    if (!overflow)
      for (int c = 0; c < nc; ++c)
        if (cand[c] == order[0]) cmax = cexact[c];
    st->cmax = cmax;
    const bool l1 = (a.form & 1) == 0;
    for (int j = 0; j < a.m; ++j) {
      if (io->gamma_relative) {
        const double g = io->gamma_in[j] * cmax;
        st->gamma[j] = l1 ? g : g * g;
      }
      st->start_cols[j] = (io->has_x0 || block) ? -1 : order[0];
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
__global__ void gather_start_kernel(const StartArgs a) {
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

// Y = sum of the per-cluster partials (fixed order), and this block's rows'
// contribution to the Gram matrix Y^T Y (packed j <= l, or the diagonal).
template <typename TC>
__global__ void __launch_bounds__(kReduceRows* kReduceGroups) reduce_kernel(const ReduceArgs a) {
  if (a.st->n_active == 0) return;
  __shared__ double part[kReduceGroups][kReduceRows];
  __shared__ double Ys[kMaxM][kReduceRows];
  __shared__ double Yo[kMaxM][kReduceRows];  // cross mode: the previous Y
  const int tid = threadIdx.x;
  const int rl = tid % kReduceRows, g = tid / kReduceRows;
  const int row = blockIdx.x * kReduceRows + rl;
  const TC* yp = static_cast<const TC*>(a.init ? a.io->P : a.io->ypart);
  TC* Y = static_cast<TC*>(a.io->Y);
  const int m = a.m, p = a.p;
  for (int j = 0; j < m; ++j) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // independent chains, fixed order
    if (row < p) {
      const int64_t stride = static_cast<int64_t>(m) * p;
      const TC* src = yp + static_cast<int64_t>(j) * p + row;
      int sp = g;
      for (; sp + 3 * kReduceGroups < a.nsplit; sp += 4 * kReduceGroups) {
        s0 += static_cast<double>(src[sp * stride]);
        s1 += static_cast<double>(src[(sp + kReduceGroups) * stride]);
        s2 += static_cast<double>(src[(sp + 2 * kReduceGroups) * stride]);
        s3 += static_cast<double>(src[(sp + 3 * kReduceGroups) * stride]);
      }
      for (; sp < a.nsplit; sp += kReduceGroups) s0 += static_cast<double>(src[sp * stride]);
    }
    part[g][rl] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (g == 0) {
      double t = 0.0;
      for (int g2 = 0; g2 < kReduceGroups; ++g2) t += part[g2][rl];
      const TC tc = static_cast<TC>(t);
      Ys[j][rl] = (row < p) ? static_cast<double>(tc) : 0.0;
      if (a.cross) {
        Yo[j][rl] = (row < p) ? static_cast<double>(Y[static_cast<int64_t>(j) * p + row]) : 0.0;
      } else if (row < p) {
        Y[static_cast<int64_t>(j) * p + row] = tc;
      }
    }
    __syncthreads();
  }
  if (a.objective) {
    // Table 1 objective f_j and the squared norm of the unnormalised
    // loadings, in double, over this block's share of T (active components)
    __shared__ double red2[2][kReduceGroups];
    const int nb = gridDim.x;
    const int chunk = (a.n + nb - 1) / nb;
    const int i0 = blockIdx.x * chunk, i1 = min(a.n, i0 + chunk);
    const TC* T = static_cast<const TC*>(a.io->T);
    for (int j = 0; j < m; ++j) {
      double f = 0.0, z2 = 0.0;
      if (a.st->active[j]) {
        const double gam = a.st->gamma[j], mu = a.io->mu[j];
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
          const Thr th = threshold(a.form, static_cast<double>(T[static_cast<int64_t>(j) * a.n + i]), gam, mu);
          f += th.term;
          z2 += th.zr * th.zr;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, off);
        z2 += __shfl_xor_sync(0xffffffffu, z2, off);
      }
      if ((tid & 31) == 0) {
        red2[0][tid >> 5] = f;
        red2[1][tid >> 5] = z2;
      }
      __syncthreads();
      if (tid == 0) {
        double F = 0.0, Z2 = 0.0;
        for (int w = 0; w < kReduceGroups; ++w) {
          F += red2[0][w];
          Z2 += red2[1][w];
        }
        a.io->fpart[(static_cast<int64_t>(blockIdx.x) * 2 + 0) * m + j] = F;
        a.io->fpart[(static_cast<int64_t>(blockIdx.x) * 2 + 1) * m + j] = Z2;
      }
      __syncthreads();
    }
  }
  if (a.cross) {  // C[j][l] = sum_r Yold[r][j] Ynew[r][l]
    for (int q = tid; q < a.npairs; q += blockDim.x) {
      const int j = q / m, l = q % m;
      double s = 0.0;
      for (int r = 0; r < kReduceRows; ++r) s += Yo[j][r] * Ys[l][r];
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
    for (int r = 0; r < kReduceRows; ++r) s += Ys[j][r] * Ys[l][r];
    a.io->gpart[static_cast<int64_t>(blockIdx.x) * a.npairs + q] = s;
  }
}

// Rayleigh-Ritz rotation of the block start.  The current start is
// Q = Y W (W the symmetric polar weights in the state) and the last sketch
// sweep gave C = Y^T (A A^T Q); B = Q^T A A^T Q = W C, symmetrised.  Its
// eigenvectors, by decreasing Ritz value, each signed so that its
// largest-magnitude entry (first on ties) is positive, rotate the start:
// new weights W V.  m x m work in FP64.
__device__ void ritz_weights(const double* C, int m, const double* Wcur, double* Wout, double* sm,
                             double* scratch) {
  const int mm = m + (m & 1);
  double* G = sm;
  double* V = sm + mm * mm;
  int* rp = reinterpret_cast<int*>(V + mm * mm);
  int* rq = rp + 32;
  double* rc = reinterpret_cast<double*>(rq + 32);
  double* rs = rc + 32;
  double* lam = rs + 32;
  __shared__ int ord[kMaxM];
  __shared__ double sgn[kMaxM];
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int idx = tid; idx < mm * mm; idx += nthr) {
    const int r = idx / mm, c = idx % mm;
    double v = 0.0;
    if (r < m && c < m) {
      double brc = 0.0, bcr = 0.0;
      for (int k = 0; k < m; ++k) {
        brc += Wcur[r * m + k] * C[k * m + c];
        bcr += Wcur[c * m + k] * C[k * m + r];
      }
      v = 0.5 * (brc + bcr);
    }
    G[idx] = v;
  }
  __syncthreads();
  jacobi_eig(G, V, mm, rp, rq, rc, rs, scratch);
  if (tid < m) lam[tid] = G[tid * mm + tid];
  __syncthreads();
  if (tid == 0) {  // order by decreasing Ritz value (ties: lower index first)
    for (int j = 0; j < m; ++j) ord[j] = j;
    for (int a = 0; a < m; ++a) {
      int best = a;
      for (int b = a + 1; b < m; ++b)
        if (lam[ord[b]] > lam[ord[best]]) best = b;
      const int t = ord[a];
      ord[a] = ord[best];
      ord[best] = t;
    }
    for (int j = 0; j < m; ++j) {
      const int c = ord[j];
      int imax = 0;
      for (int i = 1; i < m; ++i)
        if (fabs(V[i * mm + c]) > fabs(V[imax * mm + c])) imax = i;
      sgn[j] = V[imax * mm + c] < 0.0 ? -1.0 : 1.0;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int l = idx / m, j = idx % m;
    const int c = ord[j];
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += Wcur[l * m + k] * V[k * mm + c];
    Wout[l * m + j] = sgn[j] * s;
  }
  __syncthreads();
}

// Objective, stopping test and projection weights after a sweep, or one step
// of the start (projection of the start, Rayleigh-Ritz rotation).  One CTA;
// all FP64.
__global__ void __launch_bounds__(kFinishThreads) finish_kernel(const FinishArgs a) {
  extern __shared__ double fsm[];
  State* st = a.st;
  const IO* io = a.io;
  const int tid = threadIdx.x;
  const int m = a.m;
  const bool block = a.form >= 2;
  __shared__ double scratch[33];
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
  if (proceed && a.mode == kFinishRitz) {
    ritz_weights(gsum, m, st->W, Wt, jac, scratch);
    if (tid == 0)
      for (int idx = 0; idx < m * m; ++idx) st->W[idx] = Wt[idx];
  } else if (proceed && a.mode == kFinishPolar) {
    if (block) {
      const bool ok = polar_weights(gsum, m, Wt, jac, scratch, nullptr, st->V);
      if (tid == 0) {
        if (ok) {
          st->has_v = 1;
          for (int idx = 0; idx < m * m; ++idx) st->W[idx] = Wt[idx];
        } else {
          for (int j = 0; j < m; ++j) { st->status[j] = GPSPCA_DEGENERATE; st->active[j] = 0; }
          st->n_active = 0;
          st->any_degenerate = 1;
        }
      }
    } else if (tid == 0) {
      int na = 0;
      for (int j = 0; j < m; ++j) {
        for (int l = 0; l < m; ++l) st->W[l * m + j] = 0.0;
        const double d = gsum[j];
        if (d > 0.0) {
          st->W[j * m + j] = rsqrt_refined(d);
          ++na;
        } else {
          st->status[j] = GPSPCA_DEGENERATE;
          st->active[j] = 0;
          st->any_degenerate = 1;
        }
      }
      st->n_active = na;
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
        deg = !polar_weights(gsum, m, Wt, jac, scratch, st->has_v ? st->V : nullptr, st->V);
      }
      if (tid == 0) {
        if (s_stop >= 0 || deg) {
          for (int j = 0; j < m; ++j) {
            st->status[j] = deg ? GPSPCA_DEGENERATE : s_stop;
            st->iters[j] = k + 1;
            st->f[j] = fz[j];
            st->znorm2[j] = fz[m + j];
            st->active[j] = 0;
          }
          if (deg) st->any_degenerate = 1;
          st->n_active = 0;
        } else {
          for (int idx = 0; idx < m * m; ++idx) st->W[idx] = Wt[idx];
        }
      }
    } else if (tid == 0) {
      int na = 0;
      for (int j = 0; j < m; ++j) {
        if (!st->active[j]) {
          st->W[j * m + j] = 0.0;
          continue;
        }
        const double f = fz[j];
        int s = stop_rule(k, f, st->f_prev[j], tol, maxit);
        if (!isfinite(f)) {
          st->error |= kErrNonFinite;
          s = GPSPCA_MAXIT;
        }
        bool deg = false;
        if (s < 0) {
          const double d = gsum[j];
          if (d > 0.0) {
            st->W[j * m + j] = rsqrt_refined(d);
            st->f_prev[j] = f;
            ++na;
            continue;
          }
          deg = true;
        }
        st->status[j] = deg ? GPSPCA_DEGENERATE : s;
        st->iters[j] = k + 1;
        st->f[j] = f;
        st->znorm2[j] = fz[m + j];
        st->active[j] = 0;
        st->W[j * m + j] = 0.0;
        if (deg) st->any_degenerate = 1;
      }
      st->n_active = na;
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
__global__ void finalize_kernel(const IO* io, const State* st, int p, int n, int m, int form) {
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
    const Thr th = threshold(form, static_cast<double>(T[static_cast<int64_t>(j) * n + i]), gam, mu);
    z = static_cast<TC>(th.zr * inv);
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

void launch_reduce(int tcsize, const ReduceArgs& a, int nblk, cudaStream_t s) {
  if (tcsize == 8)
    reduce_kernel<double><<<nblk, kReduceRows * kReduceGroups, 0, s>>>(a);
  else
    reduce_kernel<float><<<nblk, kReduceRows * kReduceGroups, 0, s>>>(a);
}

void launch_finish(const FinishArgs& a, int smem, cudaStream_t s) {
  static bool once = [] {
    cudaFuncSetAttribute(finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)once;
  finish_kernel<<<1, kFinishThreads, smem, s>>>(a);
}

void launch_finalize(int tcsize, const IO* io, const State* st, int p, int n, int m, int form, cudaStream_t s) {
  const int len = std::max(n, p);
  const dim3 grid((len + 255) / 256, m);
  if (tcsize == 8)
    finalize_kernel<double><<<grid, 256, 0, s>>>(io, st, p, n, m, form);
  else
    finalize_kernel<float><<<grid, 256, 0, s>>>(io, st, p, n, m, form);
}

}  // namespace gpspca
