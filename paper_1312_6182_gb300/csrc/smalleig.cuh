// m x m symmetric eigenproblems of the polar step (Section 2: the block
// iterate is the polar factor of Y = A g(X)) and of the Rayleigh-Ritz
// rotation of the block start, in double-float arithmetic (dd.cuh) inside
// the one-CTA finish kernel.
//
// The Gram matrix G = Y^T Y arrives in double; it is scaled by an even power
// of two (max diagonal in [1/4, 1)), so that the float exponent range of the
// dd values is never approached, and W = G^{-1/2} is scaled back at the end.
// The eigensolver is the cyclic Jacobi method with the round-robin
// (tournament) ordering: each round applies mm/2 disjoint rotations in
// parallel.  A rotation's angle only needs float accuracy (an angle good to
// ~1e-7 still reduces its pivot by ~1e-7, and the next sweep finishes the
// job), but its cosine and sine are formed in dd so that every rotation is
// orthogonal to dd precision and so is the accumulated eigenvector matrix.
//
// Warm start: given the eigenvectors Vw of the previous Gram matrix, the
// sweeps run on Vw^T G Vw, which is close to diagonal once the iteration
// settles, and the eigenvectors are Vw times the accumulated rotations.  Any
// orthogonal Vw gives the same result (up to rounding); it only shortens the
// work.
#pragma once

#include "dd.cuh"
#include "internal.h"

namespace gpspca {

// Workspace of one solve, carved from the finish kernel's dynamic shared
// memory (8-byte slots; see eig_ws_slots).
struct EigWs {
  dd* H;      // mm x mm, the matrix being diagonalised
  dd* V;      // mm x mm, accumulated rotations
  dd* E;      // m x m, products / eigenvectors
  dd* T;      // m x m, the scaled input matrix (in V's space: dead before the sweeps start V)
  dd* Vs;     // m x m, shared copy of the warm-start eigenvectors
  dd* rc;     // 32 rotation cosines
  dd* rs;     // 32 rotation sines
  dd* lam;    // kMaxM eigenvalues (scaled)
  dd* w;      // kMaxM lambda^{-1/2} (scaled)
  int* rp;    // 32 rotation pivots p
  int* rq;    // 32 rotation pivots q
  float* red; // 32 floats: per-warp partial sums
};

__host__ __device__ inline int eig_ws_slots(int m) {
  const int mm = m + (m & 1);
  return 2 * mm * mm + 2 * m * m + 32 + 32 + 2 * kMaxM + 32 + 16;
}

__device__ inline EigWs eig_ws(double* base, int m) {
  const int mm = m + (m & 1);
  EigWs w;
  dd* d = reinterpret_cast<dd*>(base);
  w.H = d;
  w.V = w.H + mm * mm;
  w.E = w.V + mm * mm;
  w.T = w.V;
  w.Vs = w.E + m * m;
  w.rc = w.Vs + m * m;
  w.rs = w.rc + 32;
  w.lam = w.rs + 32;
  w.w = w.lam + kMaxM;
  w.rp = reinterpret_cast<int*>(w.w + kMaxM);
  w.rq = w.rp + 32;
  w.red = reinterpret_cast<float*>(w.rq + 32);
  return w;
}

// Sum of v over the CTA, the same value in every thread, added in a fixed
// order (xor tree within a warp, then the warps in index order).
__device__ __forceinline__ float cta_sum(float v, float* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.0f;
  for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Jacobi rotation (c, s) that zeroes the pivot H_pq of the 2 x 2 block
// [[app, apq], [apq, aqq]]: tan(theta) = t, the root of smaller magnitude of
// t^2 + 2 tau t - 1 = 0 with tau = (aqq - app) / (2 apq), to float accuracy
// (fast float intrinsics: an angle good to ~1e-6 still reduces the pivot by
// that factor), then cos = (1 + t^2)^{-1/2} and sin = t cos in dd, so that
// c^2 + s^2 = 1 to dd rounding.  Negligible pivots give the identity.
__device__ __forceinline__ void rotation(dd app, dd aqq, dd apq, dd* c, dd* s) {
  *c = dd{1.0f, 0.0f};
  *s = dd{0.0f, 0.0f};
  if (apq.hi == 0.0f) return;
  const dd num = dd_sub(aqq, app);
  const float den = 2.0f * apq.hi;
  if (!(fabsf(den) >= 1e-30f * fabsf(num.hi))) return;  // |tau| > 1e30: angle below 1e-30
  const float tau = __fdividef(num.hi, den);
  const float at = fabsf(tau);
  float t;
  if (at > 1e18f) {
    t = __fdividef(0.5f, at);
  } else {
    const float r = fmaf(at, at, 1.0f);
    t = __fdividef(1.0f, at + r * rsqrtf(r));
  }
  t = copysignf(t, tau);
  *c = dd_rsqrt(dd_add(dd{1.0f, 0.0f}, two_prod(t, t)));
  *s = dd_mul_f(*c, t);
}

// Stopping rule of the Jacobi sweeps: the off-diagonal Frobenius norm below
// 1e-12 of the diagonal's (far below the float data path's accuracy; dd
// rounding leaves ~1e-14 per entry, which larger matrices add up to), or a
// sweep that no longer halves it (the rounding floor has been reached).
__device__ __forceinline__ bool jacobi_done(float off, float dg, float off_prev) {
  return !(off > 1e-24f * dg) || (off_prev >= 0.0f && off > 0.25f * off_prev && off < 1e-20f * dg);
}

// Cyclic Jacobi for mm = MM <= 8 on warp 0 alone: every round's index
// arithmetic divides by constants, each lane owns (pair, index) slots of the
// row and column updates (up to four), and the rotation of each pair,
// computed by lane k, is broadcast by shuffles.  Same rotations, order and
// stopping rule as jacobi_dd_blocks.  The kernel runs once per launch with a cold
// instruction cache, so loops stay rolled: code size, not arithmetic, sets
// its time.
template <int MM>
__device__ void jacobi_small(dd* H, dd* V) {
  constexpr int HALF = MM / 2;
  constexpr int NE = MM * MM;
  constexpr int NSLOT = HALF * MM;            // (pair, index) slots of a round
  constexpr int NQ = (NSLOT + 31) / 32;       // slots per lane
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < NE; e += 32) V[e] = dd{(e / MM == e % MM) ? 1.0f : 0.0f, 0.0f};
  __syncwarp();
  float off_prev = -1.0f;
  for (int sweep = 0; sweep < 30; ++sweep) {
    float off = 0.0f, dg = 0.0f;
    for (int e = lane; e < NE; e += 32) {
      const int r = e / MM, c = e % MM;
      const float h = H[e].hi;
      if (r < c) off += h * h;
      if (r == c) dg += h * h;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(full, off, o);
      dg += __shfl_xor_sync(full, dg, o);
    }
    if (jacobi_done(off, dg, off_prev)) break;
    off_prev = off;
#pragma unroll 1
    for (int round = 0; round < MM - 1; ++round) {  // rolled: one copy of the body to fetch
      dd c{1.0f, 0.0f}, s{0.0f, 0.0f};
      if (lane < HALF) {
        const int a = (lane == 0) ? 0 : ((lane - 1 + round) % (MM - 1)) + 1;
        const int b = ((MM - 2 - lane + round) % (MM - 1)) + 1;
        const int pp = min(a, b), qq = max(a, b);
        rotation(H[pp * MM + pp], H[qq * MM + qq], H[pp * MM + qq], &c, &s);
      }
      dd ck[NQ], sk[NQ];
      int pq[NQ], qk[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {  // every lane joins every shuffle
        const int e = lane + 32 * q;
        const int k = (e < NSLOT) ? e / MM : 0;
        ck[q] = dd{__shfl_sync(full, c.hi, k), __shfl_sync(full, c.lo, k)};
        sk[q] = dd{__shfl_sync(full, s.hi, k), __shfl_sync(full, s.lo, k)};
        const int a = (k == 0) ? 0 : ((k - 1 + round) % (MM - 1)) + 1;
        const int b = ((MM - 2 - k + round) % (MM - 1)) + 1;
        pq[q] = min(a, b);
        qk[q] = max(a, b);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {  // rows: H <- J^T H
        const int e = lane + 32 * q;
        if (e < NSLOT) {
          const int l = e % MM, pp = pq[q], qq = qk[q];
          const dd hp = H[pp * MM + l], hq = H[qq * MM + l];
          H[pp * MM + l] = dd_sub(dd_mul(ck[q], hp), dd_mul(sk[q], hq));
          H[qq * MM + l] = dd_add(dd_mul(sk[q], hp), dd_mul(ck[q], hq));
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < NQ; ++q) {  // columns: H <- H J, V <- V J
        const int e = lane + 32 * q;
        if (e < NSLOT) {
          const int l = e % MM, pp = pq[q], qq = qk[q];
          const dd hp = H[l * MM + pp], hq = H[l * MM + qq];
          const dd vp = V[l * MM + pp], vq = V[l * MM + qq];
          H[l * MM + pp] = dd_sub(dd_mul(ck[q], hp), dd_mul(sk[q], hq));
          H[l * MM + qq] = dd_add(dd_mul(sk[q], hp), dd_mul(ck[q], hq));
          V[l * MM + pp] = dd_sub(dd_mul(ck[q], vp), dd_mul(sk[q], vq));
          V[l * MM + qq] = dd_add(dd_mul(sk[q], vp), dd_mul(ck[q], vq));
        }
      }
      __syncwarp();
    }
  }
}

// The same Jacobi for 8 < MM <= 16 on NSLOT / 32 rounded up warps (2-4):
// each thread owns one (pair, index) slot of a round's row and column
// updates, the rotations of the round's pairs (computed by the first HALF
// threads) pass through shared memory, and named barrier 1 joins the
// participating warps; the other threads of the CTA return at once.  Same
// rotations, order and updates as jacobi_small; the off-diagonal norm of
// the stopping rule is summed per warp, then over the warps in order.
template <int MM>
__device__ void jacobi_multi(const EigWs& ws) {
  constexpr int HALF = MM / 2;
  constexpr int NE = MM * MM;
  constexpr int NSLOT = HALF * MM;
  constexpr int NT = (NSLOT + 31) / 32 * 32;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x;
  if (tid >= NT) return;
  const unsigned full = 0xffffffffu;
  const int lane = tid & 31, warp = tid >> 5;
  dd* H = ws.H;
  dd* V = ws.V;
  auto bar = [] { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); };
  for (int e = tid; e < NE; e += NT) V[e] = dd{(e / MM == e % MM) ? 1.0f : 0.0f, 0.0f};
  float off_prev = -1.0f;
  for (int sweep = 0; sweep < 30; ++sweep) {
    bar();  // the previous sweep's updates (or V's start) are visible
    float off = 0.0f, dg = 0.0f;
    for (int e = tid; e < NE; e += NT) {
      const int r = e / MM, c = e % MM;
      const float h = H[e].hi;
      if (r < c) off += h * h;
      if (r == c) dg += h * h;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(full, off, o);
      dg += __shfl_xor_sync(full, dg, o);
    }
    if (lane == 0) {
      ws.red[warp] = off;
      ws.red[16 + warp] = dg;
    }
    bar();
    off = 0.0f;
    dg = 0.0f;
    for (int w = 0; w < NW; ++w) {
      off += ws.red[w];
      dg += ws.red[16 + w];
    }
    if (jacobi_done(off, dg, off_prev)) break;  // the same decision in every thread
    off_prev = off;
#pragma unroll 1
    for (int round = 0; round < MM - 1; ++round) {
      if (tid < HALF) {
        const int a = (tid == 0) ? 0 : ((tid - 1 + round) % (MM - 1)) + 1;
        const int b = ((MM - 2 - tid + round) % (MM - 1)) + 1;
        const int pp = min(a, b), qq = max(a, b);
        dd c, s;
        rotation(H[pp * MM + pp], H[qq * MM + qq], H[pp * MM + qq], &c, &s);
        ws.rc[tid] = c;
        ws.rs[tid] = s;
        ws.rp[tid] = pp;
        ws.rq[tid] = qq;
      }
      bar();
      const bool own = tid < NSLOT;
      const int k = own ? tid / MM : 0, l = tid % MM;
      const dd ck = ws.rc[k], sk = ws.rs[k];
      const int pp = ws.rp[k], qq = ws.rq[k];
      if (own) {  // rows: H <- J^T H
        const dd hp = H[pp * MM + l], hq = H[qq * MM + l];
        H[pp * MM + l] = dd_sub(dd_mul(ck, hp), dd_mul(sk, hq));
        H[qq * MM + l] = dd_add(dd_mul(sk, hp), dd_mul(ck, hq));
      }
      bar();
      if (own) {  // columns: H <- H J, V <- V J
        const dd hp = H[l * MM + pp], hq = H[l * MM + qq];
        const dd vp = V[l * MM + pp], vq = V[l * MM + qq];
        H[l * MM + pp] = dd_sub(dd_mul(ck, hp), dd_mul(sk, hq));
        H[l * MM + qq] = dd_add(dd_mul(sk, hp), dd_mul(ck, hq));
        V[l * MM + pp] = dd_sub(dd_mul(ck, vp), dd_mul(sk, vq));
        V[l * MM + qq] = dd_add(dd_mul(sk, vp), dd_mul(ck, vq));
      }
      bar();
    }
  }
}

// Cyclic Jacobi on the symmetric mm x mm dd matrix H (mm even) by the whole
// CTA; on return diag(H) holds the eigenvalues and V the eigenvectors
// (columns).  The mm - 1 rounds of a sweep rotate the mm / 2 disjoint pairs
// of a round-robin ordering at once; each round applies J^T H J as
// independent 2 x 2 block updates (rows p_i, q_i of the pair i rotation,
// columns p_j, q_j of pair j: one block per thread, the rows' update first,
// then the columns') together with V <- V J, so a round has two block
// barriers (rotations; updates).  Stops by jacobi_done, or after 30 sweeps.
__device__ inline void jacobi_dd_blocks(const EigWs& ws, int mm) {
  dd* H = ws.H;
  dd* V = ws.V;
  const int tid = static_cast<int>(threadIdx.x);
  const int nthr = static_cast<int>(blockDim.x);
  for (int idx = tid; idx < mm * mm; idx += nthr) V[idx] = dd{(idx / mm == idx % mm) ? 1.0f : 0.0f, 0.0f};
  __syncthreads();
  const int half = mm / 2;
  float off_prev = -1.0f;
  for (int sweep = 0; sweep < 30; ++sweep) {
    float off = 0.0f, dg = 0.0f;
    for (int idx = tid; idx < mm * mm; idx += nthr) {
      const int r = idx / mm, c = idx % mm;
      const float h = H[idx].hi;
      if (r < c) off += h * h;
      if (r == c) dg += h * h;
    }
    off = cta_sum(off, ws.red);
    dg = cta_sum(dg, ws.red);
    if (jacobi_done(off, dg, off_prev)) break;
    off_prev = off;
#pragma unroll 1
    for (int round = 0; round < mm - 1; ++round) {
      if (tid < half) {
        const int k = tid;
        const int a = (k == 0) ? 0 : ((k - 1 + round) % (mm - 1)) + 1;
        const int b = ((mm - 2 - k + round) % (mm - 1)) + 1;
        const int pp = min(a, b), qq = max(a, b);
        dd c, s;
        rotation(H[pp * mm + pp], H[qq * mm + qq], H[pp * mm + qq], &c, &s);
        ws.rp[k] = pp;
        ws.rq[k] = qq;
        ws.rc[k] = c;
        ws.rs[k] = s;
      }
      __syncthreads();
      for (int t = tid; t < half * half; t += nthr) {  // block (i, j): H <- J_i^T H J_j
        const int i = t / half, j = t % half;
        const int pi = ws.rp[i], qi = ws.rq[i], pj = ws.rp[j], qj = ws.rq[j];
        const dd ci = ws.rc[i], si = ws.rs[i], cj = ws.rc[j], sj = ws.rs[j];
        const dd h00 = H[pi * mm + pj], h01 = H[pi * mm + qj], h10 = H[qi * mm + pj], h11 = H[qi * mm + qj];
        // rows
        const dd r00 = dd_sub(dd_mul(ci, h00), dd_mul(si, h10)), r01 = dd_sub(dd_mul(ci, h01), dd_mul(si, h11));
        const dd r10 = dd_add(dd_mul(si, h00), dd_mul(ci, h10)), r11 = dd_add(dd_mul(si, h01), dd_mul(ci, h11));
        // columns
        H[pi * mm + pj] = dd_sub(dd_mul(cj, r00), dd_mul(sj, r01));
        H[pi * mm + qj] = dd_add(dd_mul(sj, r00), dd_mul(cj, r01));
        H[qi * mm + pj] = dd_sub(dd_mul(cj, r10), dd_mul(sj, r11));
        H[qi * mm + qj] = dd_add(dd_mul(sj, r10), dd_mul(cj, r11));
      }
      for (int t = tid; t < half * mm; t += nthr) {  // V <- V J
        const int k = t % half, l = t / half;
        const int pp = ws.rp[k], qq = ws.rq[k];
        const dd c = ws.rc[k], s = ws.rs[k];
        const dd vp = V[l * mm + pp], vq = V[l * mm + qq];
        V[l * mm + pp] = dd_sub(dd_mul(c, vp), dd_mul(s, vq));
        V[l * mm + qq] = dd_add(dd_mul(s, vp), dd_mul(c, vq));
      }
      __syncthreads();
    }
  }
}

// Runs the Jacobi sweeps on the group that suits mm; all threads of the CTA
// call it and leave it together.
__device__ inline void jacobi_dd_cta(const EigWs& ws, int mm) {
  if (mm <= 8) {
    if (threadIdx.x < 32) {
      switch (mm) {
        case 2: jacobi_small<2>(ws.H, ws.V); break;
        case 4: jacobi_small<4>(ws.H, ws.V); break;
        case 6: jacobi_small<6>(ws.H, ws.V); break;
        default: jacobi_small<8>(ws.H, ws.V); break;
      }
    }
  } else if (mm <= 16) {  // one thread per slot of a round: 2-4 warps
    switch (mm) {
      case 10: jacobi_multi<10>(ws); break;
      case 12: jacobi_multi<12>(ws); break;
      case 14: jacobi_multi<14>(ws); break;
      default: jacobi_multi<16>(ws); break;
    }
  } else {
    jacobi_dd_blocks(ws, mm);
  }
  __syncthreads();
}

// Even exponent e with x * 2^-e in [1/4, 1) for normal x > 0 (0 otherwise),
// read from the bits of x.
__device__ __forceinline__ int even_scale_exponent(double x) {
  const long long b = __double_as_longlong(x);
  const int be = static_cast<int>((b >> 52) & 0x7ff);
  if (b <= 0 || be == 0 || be == 0x7ff) return 0;
  const int e = max(-1000, min(1000, be - 1022));  // x = f 2^e, f in [1/2, 1) (clamped: no such Gram matrix)
  return (e & 1) ? e + 1 : e;
}

// 2^e as a double, |e| <= 1022, built from its bits.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double(static_cast<long long>(1023 + e) << 52); }

// Polar weights W = G^{-1/2} of the Gram matrix G = Y^T Y (packed upper
// triangle, row by row, in double), so that Y W is the polar factor of Y.
// Vw: dd eigenvectors of an earlier Gram matrix (m x m) or nullptr; Vout
// (may equal Vw) receives the eigenvectors of G.  Returns false (degenerate)
// if lambda_min <= 1e-12 lambda_max; W and Vout are then left unchanged.
// All threads of the CTA call it.
__device__ inline bool polar_weights(const double* gsum, int m, double* W, double* wsbase, const dd* Vw,
                                     dd* Vout) {
  const int mm = m + (m & 1);
  const EigWs ws = eig_ws(wsbase, m);
  __shared__ int s_e, s_deg;
  const int tid = threadIdx.x, nthr = blockDim.x;
  auto packed = [m](int r, int c) {
    const int j = min(r, c), l = max(r, c);
    return j * m - j * (j - 1) / 2 + (l - j);
  };
  if (tid == 0) {
    double dmax = 0.0;
    for (int j = 0; j < m; ++j) dmax = fmax(dmax, gsum[packed(j, j)]);
    s_e = even_scale_exponent(dmax);
  }
  __syncthreads();
  const double sc = pow2(-s_e);
  for (int idx = tid; idx < m * m; idx += nthr) {
    ws.T[idx] = dd_from_double(gsum[packed(idx / m, idx % m)] * sc);
    if (Vw) ws.Vs[idx] = Vw[idx];
  }
  __syncthreads();
  if (Vw) {
    Vw = ws.Vs;
    for (int idx = tid; idx < m * m; idx += nthr) {  // E = T Vw
      const int r = idx / m, c = idx % m;
      dd t{0.0f, 0.0f};
      for (int k = 0; k < m; ++k) t = dd_fma(ws.T[r * m + k], Vw[k * m + c], t);
      ws.E[idx] = t;
    }
    __syncthreads();
    for (int idx = tid; idx < mm * mm; idx += nthr) {  // H = Vw^T E, upper triangle
      const int r = idx / mm, c = idx % mm;
      dd t{0.0f, 0.0f};
      if (r < m && c < m && r <= c)
        for (int k = 0; k < m; ++k) t = dd_fma(Vw[k * m + r], ws.E[k * m + c], t);
      if (r <= c) ws.H[idx] = t;
    }
    __syncthreads();
    for (int idx = tid; idx < mm * mm; idx += nthr) {  // exact symmetry
      const int r = idx / mm, c = idx % mm;
      if (r > c) ws.H[idx] = ws.H[c * mm + r];
    }
  } else {
    for (int idx = tid; idx < mm * mm; idx += nthr) {
      const int r = idx / mm, c = idx % mm;
      ws.H[idx] = (r < m && c < m) ? ws.T[r * m + c] : dd{0.0f, 0.0f};
    }
  }
  __syncthreads();
  jacobi_dd_cta(ws, mm);
  for (int idx = tid; idx < m * m; idx += nthr) {  // eigenvectors of G: Vw V (or V)
    const int r = idx / m, c = idx % m;
    dd t;
    if (Vw) {
      t = dd{0.0f, 0.0f};
      for (int k = 0; k < m; ++k) t = dd_fma(Vw[r * m + k], ws.V[k * mm + c], t);
    } else {
      t = ws.V[r * mm + c];
    }
    ws.E[idx] = t;
  }
  if (tid < m) {
    const dd l = ws.H[tid * mm + tid];
    ws.lam[tid] = l;
    ws.w[tid] = (l.hi > 0.0f) ? dd_rsqrt(l) : dd{0.0f, 0.0f};
  }
  __syncthreads();
  if (tid == 0) {  // on the leading parts: the test's boundary is not resolved finer than dd rounding
    float lmax = 0.0f, lmin = 3.0e38f;
    for (int i = 0; i < m; ++i) {
      lmax = fmaxf(lmax, ws.lam[i].hi);
      lmin = fminf(lmin, ws.lam[i].hi);
    }
    s_deg = !(lmax > 0.0f) || !(lmin > 1e-12f * lmax);
  }
  __syncthreads();
  if (s_deg) return false;
  const double back = pow2(-s_e / 2);
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int a = idx / m, b = idx % m;
    dd s{0.0f, 0.0f};
    for (int i = 0; i < m; ++i) s = dd_fma(dd_mul(ws.E[a * m + i], ws.E[b * m + i]), ws.w[i], s);
    W[idx] = dd_to_double(s) * back;
  }
  __syncthreads();
  if (Vout)
    for (int idx = tid; idx < m * m; idx += nthr) Vout[idx] = ws.E[idx];
  __syncthreads();
  return true;
}

// Rayleigh-Ritz rotation of the block start.  The current start is
// Q = Y W (W the symmetric polar weights) and the last sketch sweep gave
// C = Y^T (A A^T Q); B = Q^T A A^T Q = W C, symmetrised.  Its eigenvectors,
// by decreasing Ritz value, each signed so that its largest-magnitude entry
// (first on ties) is positive, rotate the start: new weights W V.
// All threads of the CTA call it.
// direct: C is already the projected matrix Q^T A A^T Q (= T^T T for T = A^T
// Q) rather than the cross Gram of the two directions, and H = sym(C).
// Rout (optional): the rotation itself, ordered and signed (Wout = Wcur Rout).
__device__ inline void ritz_weights(const double* C, int m, const double* Wcur, double* Wout, double* wsbase,
                                    bool direct = false, double* Rout = nullptr) {
  const int mm = m + (m & 1);
  const EigWs ws = eig_ws(wsbase, m);
  __shared__ int ord[kMaxM];
  __shared__ float sgn[kMaxM];
  __shared__ int s_ec, s_ew;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    double cmax = 0.0, wmax = 0.0;
    for (int idx = 0; idx < m * m; ++idx) {
      cmax = fmax(cmax, fabs(C[idx]));
      wmax = fmax(wmax, fabs(Wcur[idx]));
    }
    s_ec = even_scale_exponent(cmax);
    s_ew = even_scale_exponent(wmax);
  }
  __syncthreads();
  const double sc = pow2(-s_ec), sw = pow2(-s_ew);
  for (int idx = tid; idx < m * m; idx += nthr) {  // T = scaled C, E = scaled W
    ws.T[idx] = dd_from_double(C[idx] * sc);
    ws.E[idx] = dd_from_double(Wcur[idx] * sw);
  }
  __syncthreads();
  for (int idx = tid; idx < mm * mm; idx += nthr) {  // H = sym(W C), or sym(C) when direct (scaled)
    const int r = idx / mm, c = idx % mm;
    dd v{0.0f, 0.0f};
    if (r < m && c < m) {
      dd brc{0.0f, 0.0f}, bcr{0.0f, 0.0f};
      if (direct) {
        brc = ws.T[r * m + c];
        bcr = ws.T[c * m + r];
      } else {
        for (int k = 0; k < m; ++k) {
          brc = dd_fma(ws.E[r * m + k], ws.T[k * m + c], brc);
          bcr = dd_fma(ws.E[c * m + k], ws.T[k * m + r], bcr);
        }
      }
      const dd sum = dd_add(brc, bcr);
      v = dd{sum.hi * 0.5f, sum.lo * 0.5f};
    }
    ws.H[idx] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < mm * mm; idx += nthr) {  // exact symmetry (round-off in the two products)
    const int r = idx / mm, c = idx % mm;
    if (r > c) ws.H[idx] = ws.H[c * mm + r];
  }
  __syncthreads();
  jacobi_dd_cta(ws, mm);
  if (tid == 0) {  // order by decreasing Ritz value (ties: lower index first)
    double lam[kMaxM];
    for (int j = 0; j < m; ++j) {
      ord[j] = j;
      lam[j] = dd_to_double(ws.H[j * mm + j]);
    }
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
      double vmax = fabs(dd_to_double(ws.V[c]));
      for (int i = 1; i < m; ++i) {
        const double v = fabs(dd_to_double(ws.V[i * mm + c]));
        if (v > vmax) {
          vmax = v;
          imax = i;
        }
      }
      sgn[j] = ws.V[imax * mm + c].hi < 0.0f ? -1.0f : 1.0f;
    }
  }
  __syncthreads();
  const double back = pow2(s_ew);
  for (int idx = tid; idx < m * m; idx += nthr) {
    const int l = idx / m, j = idx % m;
    const int c = ord[j];
    dd s{0.0f, 0.0f};
    for (int k = 0; k < m; ++k) s = dd_fma(ws.E[l * m + k], ws.V[k * mm + c], s);
    Wout[l * m + j] = sgn[j] * dd_to_double(s) * back;
    if (Rout) Rout[l * m + j] = sgn[j] * dd_to_double(ws.V[l * mm + c]);
  }
  __syncthreads();
}

}  // namespace gpspca
