// Tensor-core (tcgen05) wide sweep: see tc_sweep.cuh.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "plan.h"
#include "ptx.cuh"
#include "sweep.cuh"
#include "tc_sweep.cuh"

namespace gpspca {

constexpr uint32_t kTcA = 128 * 128;  // bytes of one A plane per stage: 128 x 64 bf16 (both passes)

// v = b0 + b1 + b2 exactly: each part is the bf16 rounding of what the
// previous ones left (the residuals are exact in float).
__device__ __forceinline__ void split3(float v, __nv_bfloat16& b0, __nv_bfloat16& b1, __nv_bfloat16& b2) {
  b0 = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(b0);
  b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  b2 = __float2bfloat16_rn(r2);
}

// X = Y W (the iterate this sweep evaluates, as the fused sweep forms it),
// written out for the active components and split into X3^T for the T pass;
// one thread per (row, component), blockIdx.y the component.
__global__ void tc_prep_kernel(const TcArgs a) {
  __shared__ float wj[kMaxM], wlo[kMaxM];
  const IO* io = a.io;
  const State* st = a.st;
  const int m = a.m, p = a.p, j = blockIdx.y;
  const bool block = a.form >= 2;
  // column j of W (its diagonal entry alone for the single-unit forms), as
  // a high and a low float part
  if (threadIdx.x < m) {
    const double w = j < m ? st->W[threadIdx.x * m + j] : 0.0;
    wj[threadIdx.x] = static_cast<float>(w);
    wlo[threadIdx.x] = static_cast<float>(w - static_cast<double>(wj[threadIdx.x]));
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= p) return;
  const float* Y = static_cast<const float*>(io->Y);
  float x = 0.0f;
  if (j < m) {
    if (block) {
      // Y W with every product's and sum's rounding error carried in a second
      // accumulator (Dekker's exact product by fma, Knuth's two-sum): X is Y W
      // rounded once to float even where W's large entries make the sum cancel
      float xe = 0.0f;
      for (int l = 0; l < m; ++l) {
        const float yv = Y[static_cast<int64_t>(l) * p + r];
        const float pr = __fmul_rn(yv, wj[l]);
        const float pe = fmaf(yv, wj[l], -pr);
        const float s2 = __fadd_rn(x, pr);
        const float bb = __fsub_rn(s2, x);
        const float se = __fadd_rn(__fsub_rn(x, __fsub_rn(s2, bb)), __fsub_rn(pr, bb));
        x = s2;
        xe += pe + se + yv * wlo[l];
      }
      x = __fadd_rn(x, xe);
    } else {
      x = Y[static_cast<int64_t>(j) * p + r] * wj[j];
    }
    if (!a.sketch && st->active[j]) static_cast<float*>(io->X)[static_cast<int64_t>(j) * p + r] = x;
  }
  __nv_bfloat16* X3 = static_cast<__nv_bfloat16*>(io->tc_x3);
  const int64_t rs = a.p_pad;
  __nv_bfloat16 b0, b1, b2;
  split3(x, b0, b1, b2);
  X3[(0 * a.mpad + j) * rs + r] = b0;
  X3[(1 * a.mpad + j) * rs + r] = b1;
  X3[(2 * a.mpad + j) * rs + r] = b2;
}

__host__ __device__ constexpr int tc_stages(int npad, int na) { return na == 3 ? 3 : (npad <= 48 ? 4 : (npad <= 96 ? 3 : 5)); }
__host__ __device__ constexpr int tc_ctas_per_sm(int npad, int na) { return na == 1 && npad <= 96 ? 2 : 1; }

template <int NPAD, int NA>
struct TcCfg {
  static constexpr int MPAD = NPAD / 3;
  static constexpr uint32_t kAll = NA * kTcA;  // A planes per stage
  static constexpr uint32_t kB = NPAD * 128;   // X3 / G3 bytes per stage: NPAD rows x 64 bf16
  static constexpr uint32_t kStage = kAll + kB;
  // ring depth: small N keeps two CTAs per SM (shared memory and tensor
  // memory both fit twice), which also absorbs the T pass's tile tail
  static constexpr int kStages = tc_stages(NPAD, NA);
  // two accumulators (ping-pong): the MMAs of one 64-deep chunk fill one while
  // the epilogue drains the other
  static constexpr uint32_t kCols = 2 * NPAD <= 128 ? 128 : (2 * NPAD <= 256 ? 256 : 512);
  static_assert(NPAD % 48 == 0 && NPAD <= 192, "N = 3 mpad, mpad a multiple of 16, at most 64");
  static_assert(NA == 1 || NA == 3, "one bf16 plane, or three for float A");
  static_assert(kStage % 1024 == 0, "stages keep the 1024-byte alignment of the swizzle atoms");
  static_assert(kStages * kStage + 1536 <= 227 * 1024, "stage ring fits the shared memory");
};

struct TcSmem {
  uint32_t base;         // 1024-aligned shared address of stage 0
  unsigned char* ptr;    // its generic pointer
  uint64_t* full;        // [kStages] TMA -> MMA
  uint64_t* empty;       // [kStages] MMA -> TMA
  uint64_t* accf;        // [2] MMA -> epilogue: a chunk's accumulator is complete
  uint64_t* acce;        // [2] epilogue -> MMA: it has been read
  uint32_t* tslot;
  int* abort_flag;
};

template <int NPAD, int NA>
__device__ __forceinline__ TcSmem tc_smem(unsigned char* raw) {
  TcSmem s;
  const uint32_t r = smem_u32(raw);
  s.base = (r + 1023u) & ~1023u;
  s.ptr = raw + (s.base - r);
  s.full = reinterpret_cast<uint64_t*>(s.ptr + TcCfg<NPAD, NA>::kStages * TcCfg<NPAD, NA>::kStage);
  s.empty = s.full + TcCfg<NPAD, NA>::kStages;
  s.accf = s.empty + TcCfg<NPAD, NA>::kStages;
  s.acce = s.accf + 2;
  s.tslot = reinterpret_cast<uint32_t*>(s.acce + 2);
  s.abort_flag = reinterpret_cast<int*>(s.tslot + 1);
  return s;
}

// Barriers, tensor memory; returns the accumulators' tensor-memory address.
template <int NPAD, int NA>
__device__ __forceinline__ uint32_t tc_setup(const TcSmem& S) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < TcCfg<NPAD, NA>::kStages; ++s) {
      mbar_init(smem_u32(&S.full[s]), 1);
      mbar_init(smem_u32(&S.empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&S.accf[b]), 1);
      mbar_init(smem_u32(&S.acce[b]), 128);
    }
    *S.abort_flag = 0;
    fence_mbar_init();
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(smem_u32(S.tslot), TcCfg<NPAD, NA>::kCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *S.tslot;
}

template <int NPAD, int NA>
__device__ __forceinline__ void tc_teardown(const TcSmem& S, uint32_t tmem, bool timed_out, State* st) {
  if (timed_out) atomicOr(&st->error, static_cast<int>(kErrTimeout));
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TcCfg<NPAD, NA>::kCols);
  }
}

__device__ __forceinline__ bool tc_aborted(const TcSmem& S) {
  return *reinterpret_cast<volatile int*>(S.abort_flag) != 0;
}

// TMA producer: chunk `it` of the launch goes to stage it % kStages once
// the MMAs of its previous use have completed.  load(c, sa, bar) issues the
// copies of chunk c; false on a timeout.
template <int NPAD, int NA, typename Load>
__device__ __forceinline__ bool tc_produce(const TcSmem& S, int it, int c, Load load) {
  constexpr int kS = TcCfg<NPAD, NA>::kStages;
  const int s = it % kS;
  const uint32_t u = static_cast<uint32_t>(it / kS);
  if (tc_aborted(S) || (u > 0 && !mbar_wait_bounded(smem_u32(&S.empty[s]), (u - 1) & 1))) {
    *S.abort_flag = 1;
    return false;
  }
  const uint32_t bar = smem_u32(&S.full[s]);
  mbar_arrive_expect_tx(bar, TcCfg<NPAD, NA>::kStage);
  load(c, S.base + s * TcCfg<NPAD, NA>::kStage, bar);
  return true;
}

// MMA issuer: the 4 MMAs (K = 16 each) of chunk `it` into accumulator it % 2,
// starting it afresh; then the stage is released and the accumulator handed
// to the epilogue.  false on a timeout.
template <int NPAD, int NA, typename Descs>
__device__ __forceinline__ bool tc_mma_chunk(const TcSmem& S, uint32_t tmem, int it, uint32_t idesc, Descs descs) {
  constexpr int kS = TcCfg<NPAD, NA>::kStages;
  const int s = it % kS, b = it & 1;
  const uint32_t u = static_cast<uint32_t>(it / kS), ub = static_cast<uint32_t>(it >> 1);
  if (ub > 0 && !mbar_wait_bounded(smem_u32(&S.acce[b]), (ub - 1) & 1)) return false;
  if (!mbar_wait_bounded(smem_u32(&S.full[s]), u & 1)) return false;
  tc_fence_after();
  const uint32_t sa = S.base + s * TcCfg<NPAD, NA>::kStage;
  const uint32_t d = tmem + static_cast<uint32_t>(b * NPAD);
  // smallest plane first, so the large terms are added last (the
  // accumulator's rounding is relative to its magnitude)
#pragma unroll
  for (int pl = NA - 1; pl >= 0; --pl) {
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      uint64_t ad, bd;
      descs(sa, pl, kk, &ad, &bd);
      umma_f16(d, ad, bd, idesc, (pl < NA - 1 || kk > 0) ? 1u : 0u);
    }
  }
  umma_commit(smem_u32(&S.empty[s]));
  umma_commit(smem_u32(&S.accf[b]));
  return true;
}

// Epilogue: adds chunk `it`'s accumulator (this thread's lane, the three split
// groups summed as x0 + (x1 + x2)) into acc[], then releases it.  IEEE float
// adds per chunk keep the sum at float accuracy however long the reduction
// dimension is.  false on a timeout.
template <int NPAD, int NA>
__device__ __forceinline__ bool tc_drain(const TcSmem& S, uint32_t tlane, int it, float (&acc)[TcCfg<NPAD, NA>::MPAD]) {
  constexpr int MPAD = TcCfg<NPAD, NA>::MPAD;
  const int b = it & 1;
  if (!mbar_wait_bounded(smem_u32(&S.accf[b]), static_cast<uint32_t>((it >> 1) & 1))) return false;
  tc_fence_after();
  const uint32_t col = tlane + static_cast<uint32_t>(b * NPAD);
#pragma unroll
  for (int c0 = 0; c0 < MPAD; c0 += 16) {
    uint32_t h[16], md[16], lo[16];
    tmem_ld16(col + c0, h);
    tmem_ld16(col + MPAD + c0, md);
    tmem_ld16(col + 2 * MPAD + c0, lo);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 16; ++e)
      acc[c0 + e] += __uint_as_float(h[e]) + (__uint_as_float(md[e]) + __uint_as_float(lo[e]));
  }
  tc_fence_before();
  mbar_arrive(smem_u32(&S.acce[b]));
  return true;
}

// ---- the T pass's work: items blockIdx.x, blockIdx.x + gridDim.x, ... of
// ntile1 * ksplit1, item = (column tile, range of kcs1 64-row chunks); with
// one range per tile the item is the whole tile.  Splitting the rows fills
// the last wave of CTAs when the tiles do not divide evenly among them.
struct TItem {
  int tile, ks, cb, ce;  // tile, range index, its chunks [cb, ce)
};
__device__ __forceinline__ TItem t_item(const TcArgs& a, int item) {
  TItem r;
  r.tile = item / a.ksplit1;
  r.ks = item - r.tile * a.ksplit1;
  r.cb = r.ks * a.kcs1;
  r.ce = min(a.kchunks1, r.cb + a.kcs1);
  return r;
}
// Walks this CTA's chunks in order (the TMA, MMA and converter roles).
struct TCursor {
  int item, c;
  TItem cur;
  __device__ void start(const TcArgs& a) {
    item = blockIdx.x;
    if (valid(a)) {
      cur = t_item(a, item);
      c = cur.cb;
    }
  }
  __device__ bool valid(const TcArgs& a) const { return item < a.ntile1 * a.ksplit1; }
  __device__ void next(const TcArgs& a) {
    if (++c >= cur.ce) {
      item += gridDim.x;
      if (valid(a)) {
        cur = t_item(a, item);
        c = cur.cb;
      }
    }
  }
};

// Entry (component j, column i) of the finished T (the sum of the column's
// products, before the fp8 column scale scl): the Table 1 threshold, T out,
// G split into bf16 thirds.
template <int MPAD>
__device__ __forceinline__ void tc_t_finish(const TcArgs& a, int i, int j, float t, float scl, int form,
                                            const float* gam_s, const float* mu_s, const int* act_s) {
  float g = 0.0f;
  if (j < a.m) {
    const float tj = t * scl;
    if ((!a.sketch && act_s[j]) || a.keep_t) static_cast<float*>(a.io->T)[static_cast<int64_t>(j) * a.n + i] = tj;
    g = grad_factor<float>(form, tj, gam_s[j], mu_s[j]) * scl;
    if (a.sparse && !a.sketch && g != 0.0f) a.io->tc_act[i] = 1;  // column i adds to Y = A G
  }
  __nv_bfloat16* G3 = static_cast<__nv_bfloat16*>(a.io->tc_g3);
  const int64_t gs = a.n_pad;
  __nv_bfloat16 b0, b1, b2;
  split3(g, b0, b1, b2);
  G3[(0 * MPAD + j) * gs + i] = b0;
  G3[(1 * MPAD + j) * gs + i] = b1;
  G3[(2 * MPAD + j) * gs + i] = b2;
}

// The epilogue of one T-pass item for column `col` of its tile: the column's
// finish, or, with several row ranges, its partial for tc_t_combine_kernel.
template <int MPAD>
__device__ __forceinline__ void tc_t_store(const TcArgs& a, const TItem& ti, int col, const float (&t)[MPAD],
                                           int form, const float* gam_s, const float* mu_s, const int* act_s) {
  const int i = ti.tile * kTcTile1 + col;
  if (i >= a.n) return;
  if (a.ksplit1 > 1) {
    float* tp = static_cast<float*>(a.io->tc_tpart);
#pragma unroll
    for (int j = 0; j < MPAD; ++j)
      if (j < a.m) tp[(static_cast<int64_t>(ti.ks) * MPAD + j) * a.n_pad + i] = t[j];
    return;
  }
  const float scl = a.scaled ? a.io->col_scale[i] : 1.0f;
#pragma unroll
  for (int j = 0; j < MPAD; ++j) tc_t_finish<MPAD>(a, i, j, t[j], scl, form, gam_s, mu_s, act_s);
}

// T from the row ranges' partials, summed in range order, and its finish:
// one thread per (column, component), blockIdx.y the component.
template <int MPAD>
__global__ void tc_t_combine_kernel(const TcArgs a) {
  __shared__ float gam_s[kMaxM], mu_s[kMaxM];
  __shared__ int act_s[kMaxM];
  const IO* io = a.io;
  const State* st = a.st;
  const bool sketch = a.sketch != 0;
  const int tid = threadIdx.x, j = blockIdx.y;
  if (tid < kMaxM) {
    const bool v = tid < a.m && !sketch;
    gam_s[tid] = v ? static_cast<float>(st->gamma[tid]) : 0.0f;
    mu_s[tid] = v ? static_cast<float>(io->mu[tid]) : 1.0f;
    act_s[tid] = tid < a.m ? st->active[tid] : 0;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + tid;
  if (i >= a.n) return;
  float sum = 0.0f;
  if (j < a.m) {
    const float* tp = static_cast<const float*>(io->tc_tpart) + static_cast<int64_t>(j) * a.n_pad + i;
    const int64_t ks_stride = static_cast<int64_t>(MPAD) * a.n_pad;
    float v[kTcMaxSplit1];
#pragma unroll
    for (int ks = 0; ks < kTcMaxSplit1; ++ks) v[ks] = ks < a.ksplit1 ? tp[ks * ks_stride] : 0.0f;
#pragma unroll
    for (int ks = 0; ks < kTcMaxSplit1; ++ks)
      if (ks < a.ksplit1) sum += v[ks];
  }
  const float scl = a.scaled ? io->col_scale[i] : 1.0f;
  tc_t_finish<MPAD>(a, i, j, sum, scl, sketch ? GPSPCA_SL0 : a.form, gam_s, mu_s, act_s);
}

// The first sweep after the block start: T = A^T X_0 for X_0 = Q R, the
// start's last iterate Q rotated by the Rayleigh-Ritz step, is (A^T Q) R,
// and the rotation step kept A^T Q in io->T; so this sweep forms T from it
// (double sums of m products per entry) instead of reading A, and finishes
// each entry as the T pass does.  One thread per column: its m entries of
// A^T Q are read before any entry of T is overwritten.  Unscaled storage
// only (the kept T already carries an fp8 column scale).
template <int MPAD>
__global__ void tc_t_from_ritz_kernel(const TcArgs a) {
  __shared__ float gam_s[kMaxM], mu_s[kMaxM];
  __shared__ int act_s[kMaxM];
  __shared__ double R[MPAD * MPAD];
  const IO* io = a.io;
  const State* st = a.st;
  if (st->n_active == 0) return;  // uniform across the grid
  const int tid = threadIdx.x, m = a.m;
  if (tid < kMaxM) {
    const bool v = tid < m;
    gam_s[tid] = v ? static_cast<float>(st->gamma[tid]) : 0.0f;
    mu_s[tid] = v ? static_cast<float>(io->mu[tid]) : 1.0f;
    act_s[tid] = v ? st->active[tid] : 0;
  }
  for (int idx = tid; idx < m * m; idx += blockDim.x) R[idx] = st->R[idx];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + tid;
  if (i >= a.n) return;
  float* T = static_cast<float*>(io->T);
  float q[MPAD];
#pragma unroll
  for (int k = 0; k < MPAD; ++k) q[k] = k < m ? T[static_cast<int64_t>(k) * a.n + i] : 0.0f;
#pragma unroll 4
  for (int j = 0; j < MPAD; ++j) {
    double t = 0.0;
    if (j < m)
      for (int k = 0; k < m; ++k) t = fma(static_cast<double>(q[k]), R[k * m + j], t);
    tc_t_finish<MPAD>(a, i, j, static_cast<float>(t), 1.0f, a.form, gam_s, mu_s, act_s);
  }
}

// ---- the active columns of a threshold sweep (some G_ij != 0), listed in
// increasing order for the Y pass, which then reads only those columns of A
// (the others multiply zeros).  Two launches over blocks of kTcCompactCols
// columns, one per thread: the counts, then each block's columns at its offset (the sum of
// the counts before it) with their G3 columns copied beside them; the flags
// are cleared as they are read.  Where the count exceeds the Y pass's sparse
// limit nothing but the count is written (the Y pass then reads every
// column).

__device__ __forceinline__ int tc_warp_sum(int v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) tc_count_kernel(const TcArgs a) {
  __shared__ int wsum[8];
  const uint8_t* act = a.io->tc_act;
  const int tid = threadIdx.x;
  const int i = blockIdx.x * kTcCompactCols + tid;
  int c = (i < a.n && act[i] != 0) ? 1 : 0;
  c = tc_warp_sum(c);
  if ((tid & 31) == 0) wsum[tid >> 5] = c;
  __syncthreads();
  if (tid == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    a.io->tc_cnt[blockIdx.x] = t;
  }
}

template <int MPAD>
__global__ void __launch_bounds__(256) tc_compact_kernel(const TcArgs a) {
  __shared__ int s_before[8], s_all[8], s_wtot[8], s_off, s_nl, s_tot;
  __shared__ int s_col[kTcCompactCols];
  const IO* io = a.io;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = gridDim.x;
  // counts of the blocks before this one, and of all blocks
  int before = 0, all = 0;
  for (int b = tid; b < nb; b += blockDim.x) {
    const int c = io->tc_cnt[b];
    all += c;
    if (b < static_cast<int>(blockIdx.x)) before += c;
  }
  before = tc_warp_sum(before);
  all = tc_warp_sum(all);
  const int i0 = blockIdx.x * kTcCompactCols + tid;  // this thread's column
  const int c = (i0 < a.n && io->tc_act[i0] != 0) ? 1 : 0;
  int inc = c;  // inclusive scan over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 0) {
    s_before[warp] = before;
    s_all[warp] = all;
  }
  if (lane == 31) s_wtot[warp] = inc;
  __syncthreads();
  if (tid == 0) {
    int off = 0, nl = 0, run = 0;
    for (int w = 0; w < 8; ++w) {
      off += s_before[w];
      nl += s_all[w];
      const int t = s_wtot[w];
      s_wtot[w] = run;
      run += t;
    }
    s_off = off;
    s_nl = nl;
    s_tot = run;
  }
  __syncthreads();
  const int nl = s_nl, tot = s_tot, off = s_off;
  const bool listed = static_cast<int64_t>(nl) * 10 <= static_cast<int64_t>(a.n) * kTcSparseTenths;
  // this block's active columns in order, then the flags cleared
  if (c) {
    s_col[s_wtot[warp] + inc - 1] = i0;
    io->tc_act[i0] = 0;
  }
  __syncthreads();
  if (listed) {  // the list, and the G3 columns beside it (consecutive threads: consecutive columns of a row)
    const int64_t gs = a.n_pad, cs = (static_cast<int64_t>(a.n) + 63) / 64 * 64;  // G3 / G3c row strides
    const __nv_bfloat16* G3 = static_cast<const __nv_bfloat16*>(io->tc_g3);
    __nv_bfloat16* G3c = static_cast<__nv_bfloat16*>(io->tc_g3c);
    for (int k = tid; k < tot; k += blockDim.x) io->tc_list[off + k] = s_col[k];
#pragma unroll 4
    for (int idx = tid; idx < 3 * MPAD * tot; idx += blockDim.x) {
      const int r = idx / tot, k = idx - r * tot;
      G3c[r * cs + off + k] = G3[r * gs + s_col[k]];
    }
    if (blockIdx.x == nb - 1) {  // the list padded to a multiple of 64
      const int end = (nl + 63) / 64 * 64;
      for (int k = nl + tid; k < end; k += blockDim.x) io->tc_list[k] = 0;
      for (int idx = tid; idx < 3 * MPAD * (end - nl); idx += blockDim.x) {
        const int r = idx / (end - nl), k = nl + idx % (end - nl);
        G3c[r * cs + k] = __float2bfloat16_rn(0.0f);
      }
    }
  }
  if (blockIdx.x == nb - 1 && tid == 0) *io->tc_nlist = nl;
}

// Column norms from the squared norms the first power step's T pass summed
// (the block start): ||a_i|| for the start selection and a relative gamma; a
// non-finite one (a NaN or infinity in A, or a square that overflowed)
// flags the solve.
__global__ void tc_norms_kernel(const TcArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < a.n) {
    const double c = sqrt(a.io->tc_nsq[i]);
    a.io->cnorm[i] = c;
    bad = !isfinite(c);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&a.st->error, static_cast<int>(kErrNonFinite));
}

// ---- pass 1: T = A^T X for 128-column tiles (persistent CTAs), threshold,
// G3^T for pass 2.  Tensor-memory lane = column of the tile.
template <int NPAD, int NA>
__global__ void __launch_bounds__(kTcThreads) tc_t_kernel(const TcArgs a) {
  using Cfg = TcCfg<NPAD, NA>;
  constexpr int MPAD = Cfg::MPAD;
  constexpr uint32_t kIdesc = idesc_bf16_f32(NPAD, 0, 0);
  extern __shared__ unsigned char smem_raw[];
  const TcSmem S = tc_smem<NPAD, NA>(smem_raw);
  __shared__ float gam_s[kMaxM], mu_s[kMaxM];
  __shared__ int act_s[kMaxM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const IO* io = a.io;
  State* st = a.st;
  const TcMaps* maps = static_cast<const TcMaps*>(io->tc_maps);
  const bool sketch = a.sketch != 0;
  const int form = sketch ? GPSPCA_SL0 : a.form;
  if (tid < kMaxM) {
    const bool v = tid < a.m && !sketch;
    gam_s[tid] = v ? static_cast<float>(st->gamma[tid]) : 0.0f;
    mu_s[tid] = v ? static_cast<float>(io->mu[tid]) : 1.0f;
    act_s[tid] = tid < a.m ? st->active[tid] : 0;
  }
  const uint32_t tmem = tc_setup<NPAD, NA>(S);
  bool timed_out = false;

  if (warp == 4) {  // TMA producer
    if (lane == 0) {
      for (int pl = 0; pl < NA; ++pl) tmap_acquire(&maps->a1[pl]);
      tmap_acquire(&maps->x3);
      TCursor cu;
      cu.start(a);
      for (int it = 0; cu.valid(a) && !timed_out; ++it, cu.next(a)) {
        const int tile = cu.cur.tile;
        const bool ok = tc_produce<NPAD, NA>(S, it, cu.c, [&](int cc, uint32_t sa, uint32_t bar) {
          for (int pl = 0; pl < NA; ++pl) tma_load_2d(sa + pl * kTcA, &maps->a1[pl], cc * kTcBK, tile * kTcTile1, bar);
          tma_load_2d(sa + Cfg::kAll, &maps->x3, cc * kTcBK, 0, bar);
        });
        if (!ok) timed_out = true;
      }
    }
  } else if (warp == 5) {  // MMA issuer
    if (lane == 0) {
      TCursor cu;
      cu.start(a);
      for (int it = 0; cu.valid(a) && !timed_out; ++it, cu.next(a)) {
        const bool ok =
            tc_mma_chunk<NPAD, NA>(S, tmem, it, kIdesc, [](uint32_t sa, int pl, int kk, uint64_t* ad, uint64_t* bd) {
              *ad = sdesc_sw128(sa + pl * kTcA + kk * 32, 16, 1024);
              *bd = sdesc_sw128(sa + Cfg::kAll + kk * 32, 16, 1024);
            });
        if (!ok) {
          timed_out = true;
          *S.abort_flag = 1;
        }
      }
    }
  } else {  // epilogue, warps 0-3: thread = tensor-memory lane = column of the tile
    const uint32_t tlane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    int it = 0;
    for (int item = blockIdx.x; item < a.ntile1 * a.ksplit1 && !timed_out; item += gridDim.x) {
      const TItem ti = t_item(a, item);
      float t[MPAD];
#pragma unroll
      for (int j = 0; j < MPAD; ++j) t[j] = 0.0f;
      for (int c = ti.cb; c < ti.ce; ++c, ++it) {
        if (!tc_drain<NPAD, NA>(S, tlane, it, t)) {
          timed_out = true;
          *S.abort_flag = 1;
          break;
        }
      }
      if (timed_out) break;
      tc_t_store<MPAD>(a, ti, warp * 32 + lane, t, form, gam_s, mu_s, act_s);
    }
  }
  tc_teardown<NPAD, NA>(S, tmem, timed_out, st);
}

// Producer of the Y pass over listed columns, bf16 planes (the whole warp):
// chunk c holds list entries 64c .. 64c+63 of this block's 128 rows.  Lanes
// 0-15 copy the sixteen 16-byte pieces of one listed column's rows, lanes
// 16-31 those of the next, by cp.async into the place a TMA tile load with
// the 128-byte swizzle would put them (half h = rows 64h .. 64h+63, column k
// of the chunk at byte 128 k, piece q at 16 (q xor k mod 8)), so the MMA
// reads the stage as in the dense pass; rows past p are zero-filled.  Lane 0
// copies the G3c tile by TMA.  A stage is handed to the MMA (one arrival,
// the G3c bytes expected) once the warp's copies into it have completed,
// kLag chunks later, after a proxy fence.  false on a timeout or an abort.
template <int NPAD, int NA>
__device__ __forceinline__ bool tc_list_producer(const TcSmem& S, const TcArgs& a, int rb, int cb, int ce,
                                                 const TcMaps* maps) {
  using Cfg = TcCfg<NPAD, NA>;
  constexpr int kS = Cfg::kStages;
  constexpr int kLag = kS >= 3 ? 2 : 1;  // chunks whose copies are in flight before their arrival
  static_assert(kLag < kS, "a stage's arrival precedes the wait for its next use");
  const int lane = threadIdx.x & 31;
  const int qp = lane & 15, half = qp >> 3, qq = qp & 7;
  const int32_t* list = a.io->tc_list;
  const __nv_bfloat16* base =
      static_cast<const __nv_bfloat16*>(a.io->tc_planes ? a.io->tc_planes : a.io->A);
  const int64_t ld = a.yld, plane = a.yld * a.n;
  const int r = rb * kTcRows2 + qp * 8;  // first row of this lane's pieces
  const uint32_t nbytes = static_cast<uint32_t>(max(0, min(8, a.p - r)) * 2);
  const int64_t roff = nbytes ? r : 0;
  int l0 = 0, l1 = 0;  // list entries 64c + lane and 64c + 32 + lane of the next chunk
  auto pull = [&](int c) {
    if (c < ce) {
      l0 = list[static_cast<int64_t>(c) * kTcBK + lane];
      l1 = list[static_cast<int64_t>(c) * kTcBK + 32 + lane];
    }
  };
  auto hand_over = [&](int it) {  // chunk it's copies are complete and visible to the MMA
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&S.full[it % kS]));
  };
  pull(cb);
  const int n_it = ce - cb;
  for (int it = 0; it < n_it; ++it) {
    const int c = cb + it;
    const int s = it % kS;
    const uint32_t u = static_cast<uint32_t>(it / kS);
    int ok = 1;
    if (lane == 0)
      ok = !tc_aborted(S) && (u == 0 || mbar_wait_bounded(smem_u32(&S.empty[s]), (u - 1) & 1)) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      cp_async_wait<0>();
      if (lane == 0) *S.abort_flag = 1;
      return false;
    }
    const uint32_t sa = S.base + s * Cfg::kStage;
    if (lane == 0) {
      const uint32_t bar = smem_u32(&S.full[s]);
      mbar_expect_tx(bar, Cfg::kB);
      tma_load_2d(sa + Cfg::kAll, &maps->g3c, c * kTcBK, 0, bar);
    }
    const int c0 = l0, c1 = l1;
    pull(c + 1);
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
      const int k = 2 * q + (lane >> 4);
      const int col = __shfl_sync(0xffffffffu, q < 16 ? c0 : c1, k & 31);
      const uint32_t dst = sa + half * (kTcA / 2) + k * 128 + ((qq ^ (k & 7)) << 4);
      const __nv_bfloat16* src = base + static_cast<int64_t>(col) * ld + roff;
#pragma unroll
      for (int pl = 0; pl < NA; ++pl) cp_async_16(dst + pl * kTcA, src + pl * plane, nbytes);
    }
    cp_async_commit();
    if (it >= kLag) {
      cp_async_wait<kLag>();
      hand_over(it - kLag);
    }
  }
  cp_async_wait<0>();
  for (int it = max(0, n_it - kLag); it < n_it; ++it) hand_over(it);
  return true;
}

// ---- pass 2: Y = A G for 128-row blocks, the columns split over gridDim.y;
// partial sums to ypart[split].  Tensor-memory lane = row of the block.  The
// A tile is the operand in MN-major form (64 rows contiguous per column).
// A threshold sweep with few active columns reads only those (listed by the
// compaction step, copied by tc_list_producer); otherwise every column.
template <int NPAD, int NA>
__global__ void __launch_bounds__(kTcThreads) tc_y_kernel(const TcArgs a) {
  using Cfg = TcCfg<NPAD, NA>;
  constexpr int MPAD = Cfg::MPAD;
  constexpr uint32_t kIdesc = idesc_bf16_f32(NPAD, 1, 0);
  extern __shared__ unsigned char smem_raw[];
  const TcSmem S = tc_smem<NPAD, NA>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const IO* io = a.io;
  State* st = a.st;
  const TcMaps* maps = static_cast<const TcMaps*>(io->tc_maps);
  const int rb = blockIdx.x, sp = blockIdx.y;
  const int nl = (a.sparse && !a.sketch) ? *io->tc_nlist : 0;
  const bool listed =
      a.sparse && !a.sketch && static_cast<int64_t>(nl) * 10 <= static_cast<int64_t>(a.n) * kTcSparseTenths;
  const int nch = listed ? (nl + kTcBK - 1) / kTcBK : a.nchunks2;
  const int kps = listed ? (nch + static_cast<int>(gridDim.y) - 1) / static_cast<int>(gridDim.y) : a.kps2;
  const int cb = sp * kps, ce = max(cb, min(nch, cb + kps));
  const uint32_t tmem = tc_setup<NPAD, NA>(S);
  bool timed_out = false;

  if (warp == 4 && listed) {  // copies of the listed columns
    if (lane == 0) tmap_acquire(&maps->g3c);
    __syncwarp();
    if (!tc_list_producer<NPAD, NA>(S, a, rb, cb, ce, maps)) timed_out = true;
  } else if (warp == 4) {  // TMA producer
    if (lane == 0) {
      for (int pl = 0; pl < NA; ++pl) tmap_acquire(&maps->a2[pl]);
      tmap_acquire(&maps->g3);
      for (int c = cb, it = 0; c < ce; ++c, ++it) {
        const bool ok = tc_produce<NPAD, NA>(S, it, c, [&](int cc, uint32_t sa, uint32_t bar) {
          for (int pl = 0; pl < NA; ++pl) {
            tma_load_2d(sa + pl * kTcA, &maps->a2[pl], rb * kTcRows2, cc * kTcBK, bar);
            tma_load_2d(sa + pl * kTcA + kTcA / 2, &maps->a2[pl], rb * kTcRows2 + 64, cc * kTcBK, bar);
          }
          tma_load_2d(sa + Cfg::kAll, &maps->g3, cc * kTcBK, 0, bar);
        });
        if (!ok) {
          timed_out = true;
          break;
        }
      }
    }
  } else if (warp == 5) {  // MMA issuer
    if (lane == 0) {
      for (int c = cb, it = 0; c < ce; ++c, ++it) {
        // A: rows 0-63 and 64-127 are the two MN atoms (LBO apart), 8 columns
        // per 1024-byte atom (SBO); B: K-major as in pass 1
        const bool ok =
            tc_mma_chunk<NPAD, NA>(S, tmem, it, kIdesc, [](uint32_t sa, int pl, int kk, uint64_t* ad, uint64_t* bd) {
              *ad = sdesc_sw128(sa + pl * kTcA + kk * 2048, kTcA / 2, 1024);
              *bd = sdesc_sw128(sa + Cfg::kAll + kk * 32, 16, 1024);
            });
        if (!ok) {
          timed_out = true;
          *S.abort_flag = 1;
          break;
        }
      }
    }
  } else {  // epilogue, warps 0-3
    const uint32_t tlane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    float y[MPAD];
#pragma unroll
    for (int j = 0; j < MPAD; ++j) y[j] = 0.0f;
    for (int c = cb, it = 0; c < ce; ++c, ++it) {
      if (!tc_drain<NPAD, NA>(S, tlane, it, y)) {
        timed_out = true;
        *S.abort_flag = 1;
        break;
      }
    }
    const int r = rb * kTcRows2 + warp * 32 + lane;
    if (!timed_out && r < a.p) {
      float* yp = static_cast<float*>(io->ypart);
#pragma unroll
      for (int j = 0; j < MPAD; ++j)
        if (j < a.m) yp[(static_cast<int64_t>(sp) * a.m + j) * a.p + r] = y[j];
    }
  }
  tc_teardown<NPAD, NA>(S, tmem, timed_out, st);
}

// ---------------------------------------------------------------- fused float passes
//
// Float A without a bf16 copy: TMA brings float tiles (128-byte swizzle, 32
// floats per row) into ring 1; eight converter warps split each float into
// its three bf16 parts (exact) and write them as the three planes of ring 2,
// in the layout TMA gives bf16 tiles (row = one column of A, 64 rows of A per
// 128 bytes, 16-byte chunks swizzled by row); after a proxy fence the MMA
// reads them like the planes of the copied path.  A is read once per pass at
// 4 bytes per element.
//
// Ring 1 stage: float A only (32 KB: two boxes of 32 x 128 for the T pass,
// four of 32 x 64 for the Y pass), released by the converters as soon as
// they have read it, so the float copies run ahead of the MMAs.
// Ring 2 stage: the three bf16 planes (48 KB) + the X3 / G3 tile (NPAD rows x
// 128 B), released by the MMAs' commit.

constexpr int kTcFusedThreads = 448;  // warps 0-3 epilogue, 4 TMA, 5 MMA, 6-13 converters
constexpr int kTcConverters = 256;
constexpr uint32_t kTcF = 32 * 1024;  // float A bytes per stage

__host__ __device__ constexpr int tc_fused_s1(int npad) { return npad <= 96 ? 3 : 2; }

__host__ __device__ constexpr int tc_fused_smem(int npad) {
  return tc_fused_s1(npad) * static_cast<int>(kTcF) + 2 * (3 * static_cast<int>(kTcA) + npad * 128) + 1024 + 512;
}

// Both passes with the bf16 planes in tensor memory (TM): the converters
// write the three planes of a chunk with tcgen05.st into one of S2
// tensor-memory buffers (lane = the MMA's M index: a column of the tile in
// the T pass, a row of the block in the Y pass; two K values per 32-bit
// column) and the MMAs read their A operand from there.  Ring 2 then holds
// only the X3 / G3 tile, and the shared memory the planes took (and the
// bandwidth of writing and reading them there: about half of the pass's
// shared-memory traffic) goes to float stages.  Tensor memory: NACC
// accumulators from column 0, the plane buffers (3 x 32 columns each) from
// the next multiple of 32 after them; up to NPAD = 96 this fits the 512
// columns of the SM.
constexpr uint32_t kTmABuf = 96;    // columns per plane buffer: 3 planes x 64 rows / 2
__host__ __device__ constexpr bool tc_fused_tm(int npad) { return npad <= 96; }
// accumulators: the MMAs of one chunk fill one while the epilogue drains the
// others; three where the tensor memory leaves room for three plane buffers
// next to them (NPAD = 48), else two.  Measured at 20000 x 100000, m = 16:
// block sweep 1.655 ms with two accumulators and four plane buffers, 1.607
// with three and three.
__host__ __device__ constexpr int tc_tm_nacc(int npad) { return npad <= 48 ? 3 : 2; }
// first tensor-memory column of the plane buffers: after the accumulators
__host__ __device__ constexpr uint32_t tc_tm_acol(int npad) {
  return static_cast<uint32_t>((tc_tm_nacc(npad) * npad + 31) / 32 * 32);
}
// plane buffers (and X3 stages): as many as the tensor memory holds next to
// the accumulators (3 for NPAD = 48 and 96); the converters run that many
// chunks ahead of the MMAs.  Measured at 20000 x 100000 with two
// accumulators: single-unit sweep 1.288 / 1.280 / 1.256 ms with 2 / 3 / 4
// buffers.
__host__ __device__ constexpr int tc_tm_s2(int npad) {
  return (512 - static_cast<int>(tc_tm_acol(npad))) / static_cast<int>(kTmABuf);
}
// float stages: as many as the shared memory holds next to the X3 stages, at most 6
__host__ __device__ constexpr int tc_tm_s1(int npad) {
  return (227 * 1024 - 1024 - 512 - tc_tm_s2(npad) * npad * 128) / static_cast<int>(kTcF) < 6
             ? (227 * 1024 - 1024 - 512 - tc_tm_s2(npad) * npad * 128) / static_cast<int>(kTcF)
             : 6;
}
__host__ __device__ constexpr int tc_fused_tm_smem(int npad) {
  return tc_tm_s1(npad) * static_cast<int>(kTcF) + tc_tm_s2(npad) * (npad * 128) + 1024 + 512;
}

template <int NPAD, bool TM = false>
struct TcFusedCfg {
  static constexpr int MPAD = NPAD / 3;
  static constexpr uint32_t kB = NPAD * 128;
  static constexpr uint32_t kStage1 = kTcF;
  static constexpr uint32_t kBOff = TM ? 0 : 3 * kTcA;  // X3 / G3 tile within a ring-2 stage
  static constexpr uint32_t kStage2 = kBOff + kB;
  static constexpr int S1 = TM ? tc_tm_s1(NPAD) : tc_fused_s1(NPAD);
  static constexpr int S2 = TM ? tc_tm_s2(NPAD) : 2;
  static constexpr uint32_t kCols = TM ? 512 : TcCfg<NPAD, 3>::kCols;
  static constexpr uint32_t kACol = tc_tm_acol(NPAD);
  static constexpr int NACC = TM ? tc_tm_nacc(NPAD) : 2;
  static_assert(kStage1 % 1024 == 0 && kStage2 % 1024 == 0, "1024-byte aligned stages");
  static_assert((TM ? tc_fused_tm_smem(NPAD) : tc_fused_smem(NPAD)) <= 227 * 1024, "rings fit the shared memory");
  static_assert(!TM || (S1 >= 3 && S2 >= 2 && kACol % 32 == 0 && kACol + S2 * kTmABuf <= 512),
                "float stages, accumulators and plane buffers fit");
};

struct TcFusedSmem {
  uint32_t base1, base2;  // shared addresses of ring 1 and ring 2
  unsigned char* ptr1;    // generic pointers of the same
  unsigned char* ptr2;
  uint64_t *full1, *empty1, *full2, *empty2;
  TcSmem acc;  // accf / acce / tensor-memory slot / abort flag (the drain uses these)
};

template <int NPAD, bool TM = false>
__device__ __forceinline__ TcFusedSmem tc_fused_smem(unsigned char* raw) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  TcFusedSmem s;
  const uint32_t r = smem_u32(raw);
  s.base1 = (r + 1023u) & ~1023u;
  s.ptr1 = raw + (s.base1 - r);
  s.base2 = s.base1 + Cfg::S1 * Cfg::kStage1;
  s.ptr2 = s.ptr1 + Cfg::S1 * Cfg::kStage1;
  uint64_t* b = reinterpret_cast<uint64_t*>(s.ptr2 + Cfg::S2 * Cfg::kStage2);
  s.full1 = b;
  s.empty1 = s.full1 + Cfg::S1;
  s.full2 = s.empty1 + Cfg::S1;
  s.empty2 = s.full2 + Cfg::S2;
  s.acc.accf = s.empty2 + Cfg::S2;
  s.acc.acce = s.acc.accf + Cfg::NACC;
  s.acc.tslot = reinterpret_cast<uint32_t*>(s.acc.acce + Cfg::NACC);
  s.acc.abort_flag = reinterpret_cast<int*>(s.acc.tslot + 1);
  s.acc.full = s.acc.empty = nullptr;
  s.acc.base = 0;
  s.acc.ptr = nullptr;
  return s;
}

template <int NPAD, bool TM = false>
__device__ __forceinline__ uint32_t tc_fused_setup(const TcFusedSmem& S) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int k = 0; k < Cfg::S1; ++k) {
      mbar_init(smem_u32(&S.full1[k]), 1);                   // the producer's expect_tx
      mbar_init(smem_u32(&S.empty1[k]), kTcConverters / 32);  // one arrival per converter warp
    }
    for (int k = 0; k < Cfg::S2; ++k) {
      mbar_init(smem_u32(&S.full2[k]), kTcConverters + 1);  // converters + the X3 / G3 copy
      mbar_init(smem_u32(&S.empty2[k]), 1);
    }
    for (int k = 0; k < Cfg::NACC; ++k) {
      mbar_init(smem_u32(&S.acc.accf[k]), 1);
      mbar_init(smem_u32(&S.acc.acce[k]), 128);
    }
    *S.acc.abort_flag = 0;
    fence_mbar_init();
  }
  if ((tid >> 5) == 0) {
    tmem_alloc(smem_u32(S.acc.tslot), Cfg::kCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *S.acc.tslot;
}

// Exact three-way split by truncation: a0 = a with its low 16 bits cleared,
// a1 the same of a - a0 (exact: at most 16 significant bits), a2 = what is
// left (at most 8 significant bits, exact in bf16); a = a0 + a1 + a2.  Each
// part's bf16 is the high half of its float.
__device__ __forceinline__ void split3_trunc(float x, uint32_t& h0, uint32_t& h1, uint32_t& h2) {
  const uint32_t b0 = __float_as_uint(x) & 0xFFFF0000u;
  const float r1 = x - __uint_as_float(b0);
  const uint32_t b1 = __float_as_uint(r1) & 0xFFFF0000u;
  const float r2 = r1 - __uint_as_float(b1);
  h0 = b0;
  h1 = b1;
  h2 = __float_as_uint(r2);
}

// One converter thread: rows [8 g0, 8 g0 + 8 ng) of the 64 rows of A held in
// one 128-byte row of a bf16 plane (row `prow` of the plane area), from the
// two float rows (32 rows of A each) at f0 / f1 in ring 1; all layouts
// swizzle the 16-byte chunks of a row by (row % 8), the float rows by their
// own index.
// NORM: also adds the squares of the converted values to ss (a share of the
// column's squared norm, for the block start's first power step).
template <bool NORM = false>
__device__ __forceinline__ void tc_convert_row(const unsigned char* f0, int frow0, const unsigned char* f1,
                                               int frow1, unsigned char* plane0, int prow, int g0, int ng,
                                               float* ss = nullptr) {
#pragma unroll 4
  for (int g = g0; g < g0 + ng; ++g) {  // 8 rows of A -> one 16-byte chunk per plane
    const unsigned char* src = g < 4 ? f0 : f1;
    const int fr = g < 4 ? frow0 : frow1;
    const int c0 = (g & 3) * 2;
    const uint4 v0 = *reinterpret_cast<const uint4*>(src + fr * 128 + ((c0 ^ (fr & 7)) * 16));
    const uint4 v1 = *reinterpret_cast<const uint4*>(src + fr * 128 + (((c0 + 1) ^ (fr & 7)) * 16));
    const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    if constexpr (NORM) {
#pragma unroll
      for (int e = 0; e < 8; ++e) *ss = fmaf(__uint_as_float(x[e]), __uint_as_float(x[e]), *ss);
    }
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t a0, a1, a2, b0, b1, b2;
      split3_trunc(__uint_as_float(x[e]), a0, a1, a2);
      split3_trunc(__uint_as_float(x[e + 1]), b0, b1, b2);
      // high halves of (even, odd) -> one bf16x2 word, even element in the low half
      w[0][e / 2] = __byte_perm(a0, b0, 0x7632);
      w[1][e / 2] = __byte_perm(a1, b1, 0x7632);
      w[2][e / 2] = __byte_perm(a2, b2, 0x7632);
    }
    const int off = prow * 128 + ((g ^ (prow & 7)) * 16);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
      *reinterpret_cast<uint4*>(plane0 + pl * kTcA + off) = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
  }
}

// The same for the gathered columns of the Y pass: col points at the 64
// rows of one MN atom of column i of the chunk (256 contiguous bytes, no
// swizzle).  At step gg the thread takes 8-row group (gg xor (i >> 1)) mod 4
// of its four, and that group's two 16-byte halves (i & 1) first: for the
// eight lanes of one 16-byte shared-memory phase (columns i .. i+7, 512
// bytes apart) both the loads and the stores into the swizzled plane rows
// (chunk g xor (i mod 8)) then touch eight different 16-byte bank slots.
__device__ __forceinline__ void tc_convert_row_plain(const unsigned char* col, int i, unsigned char* plane0, int g0) {
  const int hf = i & 1;
#pragma unroll
  for (int gg = 0; gg < 4; ++gg) {
    const int g = g0 + ((gg ^ (i >> 1)) & 3);
    const uint4 va = *reinterpret_cast<const uint4*>(col + g * 32 + hf * 16);
    const uint4 vb = *reinterpret_cast<const uint4*>(col + g * 32 + (hf ^ 1) * 16);
    const uint4 v0 = hf ? vb : va, v1 = hf ? va : vb;
    const uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t a0, a1, a2, b0, b1, b2;
      split3_trunc(__uint_as_float(x[e]), a0, a1, a2);
      split3_trunc(__uint_as_float(x[e + 1]), b0, b1, b2);
      w[0][e / 2] = __byte_perm(a0, b0, 0x7632);
      w[1][e / 2] = __byte_perm(a1, b1, 0x7632);
      w[2][e / 2] = __byte_perm(a2, b2, 0x7632);
    }
    const int off = i * 128 + ((g ^ (i & 7)) * 16);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
      *reinterpret_cast<uint4*>(plane0 + pl * kTcA + off) = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
  }
}

// Converter warps: chunk `it` from ring 1 into ring 2.  kY: Y-pass layout
// (two 64-row MN atoms of 64 columns) instead of the T pass's 128 columns.
template <int NPAD, bool kY, bool NORM = false>
__device__ __forceinline__ bool tc_convert_chunk(const TcFusedSmem& S, int it, bool plain = false,
                                                 float* ss = nullptr) {
  using Cfg = TcFusedCfg<NPAD>;
  const int s1 = it % Cfg::S1, s2 = it % Cfg::S2;
  const uint32_t u1 = static_cast<uint32_t>(it / Cfg::S1), u2 = static_cast<uint32_t>(it / Cfg::S2);
  if (!mbar_wait_bounded(smem_u32(&S.full1[s1]), u1 & 1)) return false;
  if (u2 > 0 && !mbar_wait_bounded(smem_u32(&S.empty2[s2]), (u2 - 1) & 1)) return false;
  const unsigned char* f = S.ptr1 + s1 * Cfg::kStage1;
  unsigned char* b = S.ptr2 + s2 * Cfg::kStage2;
  const int c = static_cast<int>(threadIdx.x) - 192;  // 0..255: (half of the 64 rows, plane row)
  const int h = c >> 7, q = c & 127;
  if (!kY) {  // row q = column q of the tile; float boxes: rows 0-31 | 32-63 of A
    tc_convert_row<NORM>(f, q, f + 16384, q, b, q, 4 * h, 4, ss);
  } else {    // atom a = rows 64a..64a+63 of A, row i = column i; float boxes of 32 rows x 64 columns
    const int a = q >> 6, i = q & 63;
    if (plain)  // gathered columns: column i's 128 rows at byte 512 i, not swizzled
      tc_convert_row_plain(f + i * 512 + a * 256, i, b + a * 8192, 4 * h);
    else
      tc_convert_row(f + (2 * a) * 8192, i, f + (2 * a + 1) * 8192, i, b + a * 8192, i, 4 * h, 4);
  }
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(&S.empty1[s1]));  // the float stage is read
  fence_async_smem();
  mbar_arrive(smem_u32(&S.full2[s2]));
  return true;
}

template <int NPAD, bool kY>
__device__ __forceinline__ bool tc_fused_mma(const TcFusedSmem& S, uint32_t tmem, int it, uint32_t idesc) {
  using Cfg = TcFusedCfg<NPAD>;
  const int s2 = it % Cfg::S2, b = it & 1;
  const uint32_t u2 = static_cast<uint32_t>(it / Cfg::S2);
  const uint32_t ub = static_cast<uint32_t>(it >> 1);
  if (ub > 0 && !mbar_wait_bounded(smem_u32(&S.acc.acce[b]), (ub - 1) & 1)) return false;
  if (!mbar_wait_bounded(smem_u32(&S.full2[s2]), u2 & 1)) return false;
  tc_fence_after();
  const uint32_t sa = S.base2 + s2 * Cfg::kStage2;
  const uint32_t sb = sa + 3 * kTcA;
  const uint32_t d = tmem + static_cast<uint32_t>(b * NPAD);
#pragma unroll
  for (int pl = 2; pl >= 0; --pl) {  // smallest plane first
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      const uint64_t ad = kY ? sdesc_sw128(sa + pl * kTcA + kk * 2048, kTcA / 2, 1024)
                             : sdesc_sw128(sa + pl * kTcA + kk * 32, 16, 1024);
      const uint64_t bd = sdesc_sw128(sb + kk * 32, 16, 1024);
      umma_f16(d, ad, bd, idesc, (pl < 2 || kk > 0) ? 1u : 0u);
    }
  }
  umma_commit(smem_u32(&S.empty2[s2]));
  umma_commit(smem_u32(&S.acc.accf[b]));
  return true;
}

// Converter warps of the TM T pass: chunk `it` from ring 1 into plane
// buffer it % S2 of tensor memory.  Warp w (6..13) may write the tensor-memory
// lanes 32 (w % 4) .. + 31, so its thread for lane L takes tile column
// q = 32 (w % 4) + L, and rows 32 h .. 32 h + 31 of the chunk with
// h = (w - 6) / 4: the 128-byte row q of float box h (16-byte chunks
// swizzled by q), split exactly into three bf16 parts, two rows per 32-bit
// column: plane pl, row r at column 2 NPAD + 96 (it % S2) + 32 pl + r / 2.
// NORM: also adds the squares of the values to ss (see tc_convert_row).
template <int NPAD, bool NORM = false>
__device__ __forceinline__ bool tc_convert_chunk_tm(const TcFusedSmem& S, uint32_t tmem, int it,
                                                    float* ss = nullptr) {
  using Cfg = TcFusedCfg<NPAD, true>;
  const int s1 = it % Cfg::S1, s2 = it % Cfg::S2;
  const uint32_t u1 = static_cast<uint32_t>(it / Cfg::S1), u2 = static_cast<uint32_t>(it / Cfg::S2);
  if (!mbar_wait_bounded(smem_u32(&S.full1[s1]), u1 & 1)) return false;
  // the MMAs that read this plane buffer (chunk it - 2) have completed
  if (u2 > 0 && !mbar_wait_bounded(smem_u32(&S.empty2[s2]), (u2 - 1) & 1)) return false;
  tc_fence_after();
  const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31);
  const int quad = warp & 3;
  const int q = 32 * quad + lane;
  const int h = (warp - 6) >> 2;
  const unsigned char* row = S.ptr1 + s1 * Cfg::kStage1 + h * 16384 + q * 128;
  const uint32_t tcol = tmem + (static_cast<uint32_t>(32 * quad) << 16) + Cfg::kACol +
                        static_cast<uint32_t>(s2) * kTmABuf + static_cast<uint32_t>(16 * h);
#pragma unroll
  for (int half = 0; half < 2; ++half) {  // rows 16 half .. + 15 of the thread's 32
    uint32_t w[3][8];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {  // 16-byte chunk j: rows 4 j .. 4 j + 3
      const uint4 v = *reinterpret_cast<const uint4*>(row + (((half * 4 + cc) ^ (q & 7)) * 16));
      const uint32_t x[4] = {v.x, v.y, v.z, v.w};
      if constexpr (NORM) {
#pragma unroll
        for (int e = 0; e < 4; ++e) *ss = fmaf(__uint_as_float(x[e]), __uint_as_float(x[e]), *ss);
      }
#pragma unroll
      for (int e = 0; e < 4; e += 2) {
        uint32_t a0, a1, a2, b0, b1, b2;
        split3_trunc(__uint_as_float(x[e]), a0, a1, a2);
        split3_trunc(__uint_as_float(x[e + 1]), b0, b1, b2);
        // high halves of (even row, odd row) -> one bf16x2 word, even row in the low half
        w[0][2 * cc + e / 2] = __byte_perm(a0, b0, 0x7632);
        w[1][2 * cc + e / 2] = __byte_perm(a1, b1, 0x7632);
        w[2][2 * cc + e / 2] = __byte_perm(a2, b2, 0x7632);
      }
    }
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) tmem_st8(tcol + static_cast<uint32_t>(32 * pl + 8 * half), w[pl]);
  }
  tmem_wait_st();
  // the float stage is released only now: releasing it as soon as its values
  // were in registers was measured 2% slower over the whole pass
  __syncwarp();
  if (lane == 0) mbar_arrive(smem_u32(&S.empty1[s1]));
  tc_fence_before();
  mbar_arrive(smem_u32(&S.full2[s2]));
  return true;
}

// Converter warps of the TM Y pass: chunk `it` (64 columns of A, 128 rows)
// from ring 1 into plane buffer it % S2.  The thread for tensor-memory lane
// r = 32 (w % 4) + L takes row r of the block and columns 32 h .. 32 h + 31
// of the chunk (h = (w - 6) / 4), one 4-byte load per column: in the stored
// layout (four boxes of 32 rows x 64 columns, 16-byte chunks swizzled by the
// column) or, for gathered columns (plain), column i's 128 rows at byte
// 512 i.  Two columns per 32-bit word, the even one in the low half.
template <int NPAD>
__device__ __forceinline__ bool tc_convert_chunk_tm_y(const TcFusedSmem& S, uint32_t tmem, int it, bool plain) {
  using Cfg = TcFusedCfg<NPAD, true>;
  const int s1 = it % Cfg::S1, s2 = it % Cfg::S2;
  const uint32_t u1 = static_cast<uint32_t>(it / Cfg::S1), u2 = static_cast<uint32_t>(it / Cfg::S2);
  if (!mbar_wait_bounded(smem_u32(&S.full1[s1]), u1 & 1)) return false;
  if (u2 > 0 && !mbar_wait_bounded(smem_u32(&S.empty2[s2]), (u2 - 1) & 1)) return false;
  tc_fence_after();
  const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31);
  const int quad = warp & 3;
  const int h = (warp - 6) >> 2;
  const unsigned char* f = S.ptr1 + s1 * Cfg::kStage1;
  // byte offset of (row r, column i): plain i * 512 + 4 r; stored box r / 32,
  // column row i, 16-byte chunk (r % 32) / 4 swizzled by i
  const unsigned char* rowp = plain ? f + 4 * (32 * quad + lane) : f + quad * 8192 + (lane & 3) * 4;
  const uint32_t tcol = tmem + (static_cast<uint32_t>(32 * quad) << 16) + Cfg::kACol +
                        static_cast<uint32_t>(s2) * kTmABuf + static_cast<uint32_t>(16 * h);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t w[3][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = 32 * h + 16 * half + 2 * e;
      float v0, v1;
      if (plain) {
        v0 = *reinterpret_cast<const float*>(rowp + i * 512);
        v1 = *reinterpret_cast<const float*>(rowp + (i + 1) * 512);
      } else {
        v0 = *reinterpret_cast<const float*>(rowp + i * 128 + (((lane >> 2) ^ (i & 7)) << 4));
        v1 = *reinterpret_cast<const float*>(rowp + (i + 1) * 128 + (((lane >> 2) ^ ((i + 1) & 7)) << 4));
      }
      uint32_t a0, a1, a2, b0, b1, b2;
      split3_trunc(v0, a0, a1, a2);
      split3_trunc(v1, b0, b1, b2);
      w[0][e] = __byte_perm(a0, b0, 0x7632);
      w[1][e] = __byte_perm(a1, b1, 0x7632);
      w[2][e] = __byte_perm(a2, b2, 0x7632);
    }
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) tmem_st8(tcol + static_cast<uint32_t>(32 * pl + 8 * half), w[pl]);
  }
  tmem_wait_st();
  __syncwarp();
  if (lane == 0) mbar_arrive(smem_u32(&S.empty1[s1]));
  tc_fence_before();
  mbar_arrive(smem_u32(&S.full2[s2]));
  return true;
}

// MMA issuer of the TM T pass: the 12 MMAs of chunk `it` (three planes, four
// K = 16 steps each, smallest plane first), A from plane buffer it % S2 of
// tensor memory, B the X3 tile of ring-2 stage it % S2.
template <int NPAD>
__device__ __forceinline__ bool tc_fused_mma_tm(const TcFusedSmem& S, uint32_t tmem, int it, uint32_t idesc) {
  using Cfg = TcFusedCfg<NPAD, true>;
  const int s2 = it % Cfg::S2, b = it % Cfg::NACC;
  const uint32_t u2 = static_cast<uint32_t>(it / Cfg::S2);
  const uint32_t ub = static_cast<uint32_t>(it / Cfg::NACC);
  if (ub > 0 && !mbar_wait_bounded(smem_u32(&S.acc.acce[b]), (ub - 1) & 1)) return false;
  if (!mbar_wait_bounded(smem_u32(&S.full2[s2]), u2 & 1)) return false;
  tc_fence_after();
  const uint32_t sb = S.base2 + s2 * Cfg::kStage2 + Cfg::kBOff;
  const uint32_t d = tmem + static_cast<uint32_t>(b * NPAD);
  const uint32_t at = tmem + Cfg::kACol + static_cast<uint32_t>(s2) * kTmABuf;
#pragma unroll
  for (int pl = 2; pl >= 0; --pl) {
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      const uint64_t bd = sdesc_sw128(sb + kk * 32, 16, 1024);
      umma_f16_ts(d, at + static_cast<uint32_t>(32 * pl + 8 * kk), bd, idesc, (pl < 2 || kk > 0) ? 1u : 0u);
    }
  }
  umma_commit(smem_u32(&S.empty2[s2]));
  umma_commit(smem_u32(&S.acc.accf[b]));
  return true;
}

// Epilogue of the TM T pass: as tc_drain, over the NACC accumulators.
template <int NPAD>
__device__ __forceinline__ bool tc_drain_tm(const TcSmem& S, uint32_t tlane, int it, float (&acc)[NPAD / 3]) {
  using Cfg = TcFusedCfg<NPAD, true>;
  constexpr int MPAD = NPAD / 3;
  const int b = it % Cfg::NACC;
  if (!mbar_wait_bounded(smem_u32(&S.accf[b]), static_cast<uint32_t>((it / Cfg::NACC) & 1))) return false;
  tc_fence_after();
  const uint32_t col = tlane + static_cast<uint32_t>(b * NPAD);
#pragma unroll
  for (int c0 = 0; c0 < MPAD; c0 += 16) {
    uint32_t h[16], md[16], lo[16];
    tmem_ld16(col + c0, h);
    tmem_ld16(col + MPAD + c0, md);
    tmem_ld16(col + 2 * MPAD + c0, lo);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 16; ++e)
      acc[c0 + e] += __uint_as_float(h[e]) + (__uint_as_float(md[e]) + __uint_as_float(lo[e]));
  }
  tc_fence_before();
  mbar_arrive(smem_u32(&S.acce[b]));
  return true;
}

// TMA producer of both rings: the float tile of chunk `it` once the
// converters have read the stage's previous tile, the X3 / G3 tile once the
// MMAs of the ring-2 stage's previous chunk have completed.  The two streams
// are polled without blocking, so neither waits behind the other.
// coordf / coordb(it, &c, &tr): the chunk's 64-deep index c and its tile (T
// pass) or 128-row block (Y pass), for the stored-tile and the X3 / G3
// streams; each is called with it = 0, 1, 2, ... in turn.  false on a
// timeout or an abort.
template <int NPAD, bool TM = false, typename CoordF, typename CoordB>
__device__ __forceinline__ bool tc_fused_producer(const TcFusedSmem& S, int total, CoordF coordf, CoordB coordb,
                                                  const TcMaps* maps, bool y_pass) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  int itf = 0, itb = 0;
  uint32_t idle = 0;
  while (itf < total || itb < total) {
    if (tc_aborted(S.acc)) return false;
    bool progressed = false;
    if (itf < total) {
      const int s1 = itf % Cfg::S1;
      const uint32_t u1 = static_cast<uint32_t>(itf / Cfg::S1);
      if (u1 == 0 || mbar_test(smem_u32(&S.empty1[s1]), (u1 - 1) & 1)) {
        int c, tr;
        coordf(itf, &c, &tr);
        const uint32_t sa = S.base1 + s1 * Cfg::kStage1;
        const uint32_t bar = smem_u32(&S.full1[s1]);
        mbar_arrive_expect_tx(bar, kTcF);
        if (!y_pass) {
          tma_load_2d(sa, &maps->a1f, c * kTcBK, tr * kTcTile1, bar);
          tma_load_2d(sa + 16384, &maps->a1f, c * kTcBK + 32, tr * kTcTile1, bar);
        } else {
          for (int q = 0; q < 4; ++q) tma_load_2d(sa + q * 8192, &maps->a2f, tr * kTcRows2 + 32 * q, c * kTcBK, bar);
        }
        ++itf;
        progressed = true;
      }
    }
    if (itb < total) {
      const int s2 = itb % Cfg::S2;
      const uint32_t u2 = static_cast<uint32_t>(itb / Cfg::S2);
      if (u2 == 0 || mbar_test(smem_u32(&S.empty2[s2]), (u2 - 1) & 1)) {
        int c, tr;
        coordb(itb, &c, &tr);
        const uint32_t bar = smem_u32(&S.full2[s2]);
        mbar_arrive_expect_tx(bar, Cfg::kB);
        tma_load_2d(S.base2 + s2 * Cfg::kStage2 + Cfg::kBOff, y_pass ? &maps->g3 : &maps->x3, c * kTcBK, 0, bar);
        ++itb;
        progressed = true;
      }
    }
    if (progressed) {
      idle = 0;
    } else {
      if (++idle > (1u << 25)) return false;
      __nanosleep(32);
    }
  }
  return true;
}

// ---- the fused Y pass's work: items k = blockIdx.x, blockIdx.x + gridDim.x,
// ... of nrow2 * nsplit2 (persistent CTAs), item k = (128-row block k mod
// nrow2, column split k / nrow2), a split = kps consecutive 64-column chunks
// (of all columns, or of the listed ones).  Walks the chunks of this CTA's
// items in order, skipping empty items.
struct YCursor {
  int item, c, cb, ce, rb, sp;
  int nrow2, nitems, nch, kps;
  __device__ void set(int k) {
    rb = k % nrow2;
    sp = k / nrow2;
    cb = sp * kps;
    ce = max(cb, min(nch, cb + kps));
    c = cb;
  }
  __device__ void seek(int k) {
    for (item = k; item < nitems; item += gridDim.x) {
      set(item);
      if (cb < ce) return;
    }
  }
  __device__ void start(int nrow2_, int nsplit, int nch_, int kps_) {
    nrow2 = nrow2_;
    nitems = nrow2_ * nsplit;
    nch = nch_;
    kps = kps_;
    seek(blockIdx.x);
  }
  __device__ bool valid() const { return item < nitems; }
  __device__ void next() {
    if (++c >= ce) seek(item + gridDim.x);
  }
};

// Producer of the fused Y pass over listed columns (the whole warp): chunk c
// holds list entries 64c .. 64c+63; lane g < 16 gathers the four columns 4g
// .. 4g+3, all 128 rows of the chunk's row block (tile::gather4, one
// 512-byte box row per column, no swizzle), so column k of the chunk lands
// at byte 512 k of the float stage.  The list entries of the next four
// chunks are loaded ahead into registers.  Lane 0 polls both rings and
// copies the G3c tile.  false on a timeout or an abort.
template <int NPAD, bool TM = false>
__device__ __forceinline__ bool tc_gather_producer(const TcFusedSmem& S, int total, YCursor ca, YCursor cg,
                                                   const int32_t* list, const TcMaps* maps) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  const int lane = threadIdx.x & 31;
  const int g = lane & 15;
  int itf = 0, itb = 0;
  uint32_t idle = 0;
  const int4 z = make_int4(0, 0, 0, 0);
  int4 q0 = z, q1 = z, q2 = z, q3 = z;
  int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
  auto pull = [&](int4& q, int& r) {
    if (ca.valid()) {
      q = *reinterpret_cast<const int4*>(list + static_cast<int64_t>(ca.c) * kTcBK + 4 * g);
      r = ca.rb;
      ca.next();
    }
  };
  pull(q0, r0);
  pull(q1, r1);
  pull(q2, r2);
  pull(q3, r3);
  while (itf < total || itb < total) {
    int want = 0;  // bit 0: the float stage is free, bit 1: the G3c stage, bit 2: abort
    if (lane == 0) {
      if (tc_aborted(S.acc)) {
        want = 4;
      } else {
        if (itf < total) {
          const uint32_t u1 = static_cast<uint32_t>(itf / Cfg::S1);
          if (u1 == 0 || mbar_test(smem_u32(&S.empty1[itf % Cfg::S1]), (u1 - 1) & 1)) want |= 1;
        }
        if (itb < total) {
          const uint32_t u2 = static_cast<uint32_t>(itb / Cfg::S2);
          if (u2 == 0 || mbar_test(smem_u32(&S.empty2[itb % Cfg::S2]), (u2 - 1) & 1)) want |= 2;
        }
      }
    }
    want = __shfl_sync(0xffffffffu, want, 0);
    if (want & 4) return false;
    if (want & 1) {
      const int s1 = itf % Cfg::S1;
      const uint32_t sa = S.base1 + s1 * Cfg::kStage1;
      const uint32_t bar = smem_u32(&S.full1[s1]);
      if (lane == 0) mbar_arrive_expect_tx(bar, kTcF);
      __syncwarp();
      if (lane < 16) tma_gather4(sa + g * 2048, &maps->a2g, r0 * kTcRows2, q0.x, q0.y, q0.z, q0.w, bar);
      ++itf;
      q0 = q1;
      r0 = r1;
      q1 = q2;
      r1 = r2;
      q2 = q3;
      r2 = r3;
      pull(q3, r3);
    }
    if (want & 2) {
      if (lane == 0) {
        const int s2 = itb % Cfg::S2;
        const uint32_t bar = smem_u32(&S.full2[s2]);
        mbar_arrive_expect_tx(bar, Cfg::kB);
        tma_load_2d(S.base2 + s2 * Cfg::kStage2 + Cfg::kBOff, &maps->g3c, cg.c * kTcBK, 0, bar);
      }
      ++itb;
      cg.next();
    }
    if (want & 3) {
      idle = 0;
    } else {
      if (++idle > (1u << 25)) return false;
      __nanosleep(32);
    }
  }
  return true;
}

// fused T pass (float A); TM: the bf16 planes in tensor memory
template <int NPAD, bool TM>
__global__ void __launch_bounds__(kTcFusedThreads, 1) tc_t_fused_kernel(const TcArgs a) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  constexpr int MPAD = Cfg::MPAD;
  constexpr uint32_t kIdesc = idesc_bf16_f32(NPAD, 0, 0);
  extern __shared__ unsigned char smem_raw[];
  const TcFusedSmem S = tc_fused_smem<NPAD, TM>(smem_raw);
  __shared__ float gam_s[kMaxM], mu_s[kMaxM];
  __shared__ int act_s[kMaxM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const IO* io = a.io;
  State* st = a.st;
  const TcMaps* maps = static_cast<const TcMaps*>(io->tc_maps);
  const bool sketch = a.sketch != 0;
  const int form = sketch ? GPSPCA_SL0 : a.form;
  if (tid < kMaxM) {
    const bool v = tid < a.m && !sketch;
    gam_s[tid] = v ? static_cast<float>(st->gamma[tid]) : 0.0f;
    mu_s[tid] = v ? static_cast<float>(io->mu[tid]) : 1.0f;
    act_s[tid] = tid < a.m ? st->active[tid] : 0;
  }
  const uint32_t tmem = tc_fused_setup<NPAD, TM>(S);
  bool timed_out = false;
  if (warp == 4) {
    if (lane == 0) {
      tmap_acquire(&maps->a1f);
      tmap_acquire(&maps->x3);
      int total = 0;
      for (int item = blockIdx.x; item < a.ntile1 * a.ksplit1; item += gridDim.x) {
        const TItem ti = t_item(a, item);
        total += ti.ce - ti.cb;
      }
      TCursor cf, cb;  // the stored-tile and the X3 streams, each called with consecutive indices
      cf.start(a);
      cb.start(a);
      if (!tc_fused_producer<NPAD, TM>(
              S, total,
              [&](int, int* c, int* tr) {
                *c = cf.c;
                *tr = cf.cur.tile;
                cf.next(a);
              },
              [&](int, int* c, int* tr) {
                *c = cb.c;
                *tr = cb.cur.tile;
                cb.next(a);
              },
              maps, false)) {
        timed_out = true;
        *S.acc.abort_flag = 1;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      TCursor cu;
      cu.start(a);
      for (int it = 0; cu.valid(a) && !timed_out; ++it, cu.next(a)) {
        bool ok;
        if constexpr (TM)
          ok = tc_fused_mma_tm<NPAD>(S, tmem, it, kIdesc);
        else
          ok = tc_fused_mma<NPAD, false>(S, tmem, it, kIdesc);
        if (!ok) {
          timed_out = true;
          *S.acc.abort_flag = 1;
        }
      }
    }
  } else if (warp >= 6) {  // converters
    TCursor cu;
    cu.start(a);
    // with a.norms (the block start's first power step): the squares of the
    // column's 32 rows each thread converts, summed per chunk in float, per
    // item in double, and added to the column's squared norm at the item's
    // end (two halves of the rows, and the row ranges, add up by atomics)
    const int q = TM ? 32 * (warp & 3) + lane : (tid - 192) & 127;  // the thread's column of the tile
    double nacc = 0.0;
    for (int it = 0; cu.valid(a) && !timed_out; ++it, cu.next(a)) {
      float ss = 0.0f;
      bool ok;
      if constexpr (TM)
        ok = a.norms ? tc_convert_chunk_tm<NPAD, true>(S, tmem, it, &ss) : tc_convert_chunk_tm<NPAD>(S, tmem, it);
      else
        ok = a.norms ? tc_convert_chunk<NPAD, false, true>(S, it, false, &ss) : tc_convert_chunk<NPAD, false>(S, it);
      if (tc_aborted(S.acc) || !ok) {
        timed_out = true;
        *S.acc.abort_flag = 1;
        break;
      }
      if (a.norms) {
        nacc += static_cast<double>(ss);
        if (cu.c + 1 >= cu.cur.ce) {
          const int col = cu.cur.tile * kTcTile1 + q;
          if (col < a.n) atomicAdd(&a.io->tc_nsq[col], nacc);
          nacc = 0.0;
        }
      }
    }
  } else {  // epilogue
    const uint32_t tlane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    int it = 0;
    for (int item = blockIdx.x; item < a.ntile1 * a.ksplit1 && !timed_out; item += gridDim.x) {
      const TItem ti = t_item(a, item);
      float t[MPAD];
#pragma unroll
      for (int j = 0; j < MPAD; ++j) t[j] = 0.0f;
      for (int c = ti.cb; c < ti.ce; ++c, ++it) {
        bool ok;
        if constexpr (TM)
          ok = tc_drain_tm<NPAD>(S.acc, tlane, it, t);
        else
          ok = tc_drain<NPAD, 3>(S.acc, tlane, it, t);
        if (!ok) {
          timed_out = true;
          *S.acc.abort_flag = 1;
          break;
        }
      }
      if (timed_out) break;
      tc_t_store<MPAD>(a, ti, warp * 32 + lane, t, form, gam_s, mu_s, act_s);
    }
  }
  if (timed_out) atomicOr(&st->error, static_cast<int>(kErrTimeout));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::kCols);
  }
}

// fused Y pass (float A), persistent CTAs over (row block, split) items; TM:
// the bf16 planes in tensor memory (rows in lanes, so the A operand is K-major)
template <int NPAD, bool TM>
__global__ void __launch_bounds__(kTcFusedThreads, 1) tc_y_fused_kernel(const TcArgs a) {
  using Cfg = TcFusedCfg<NPAD, TM>;
  constexpr int MPAD = Cfg::MPAD;
  constexpr uint32_t kIdesc = idesc_bf16_f32(NPAD, TM ? 0 : 1, 0);
  extern __shared__ unsigned char smem_raw[];
  const TcFusedSmem S = tc_fused_smem<NPAD, TM>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const IO* io = a.io;
  State* st = a.st;
  const TcMaps* maps = static_cast<const TcMaps*>(io->tc_maps);
  // a threshold sweep with few active columns reads only those (listed by
  // the compaction step); otherwise every column
  const int nl = (a.sparse && !a.sketch) ? *io->tc_nlist : 0;
  const bool listed =
      a.sparse && !a.sketch && static_cast<int64_t>(nl) * 10 <= static_cast<int64_t>(a.n) * kTcSparseTenths;
  const int nch = listed ? (nl + kTcBK - 1) / kTcBK : a.nchunks2;
  const int kps = listed ? (nch + a.nsplit2 - 1) / a.nsplit2 : a.kps2;
  YCursor cur;
  cur.start(a.nrow2, a.nsplit2, nch, kps);
  int total = 0;  // chunks of this CTA's items
  for (YCursor t = cur; t.valid(); t.seek(t.item + gridDim.x)) total += t.ce - t.cb;
  const uint32_t tmem = tc_fused_setup<NPAD, TM>(S);
  bool timed_out = false;
  if (warp == 4) {
    if (listed) {
      tmap_acquire(&maps->a2g);
      tmap_acquire(&maps->g3c);
      if (!tc_gather_producer<NPAD, TM>(S, total, cur, cur, io->tc_list, maps)) {
        timed_out = true;
        if (lane == 0) *S.acc.abort_flag = 1;
      }
    } else if (lane == 0) {
      tmap_acquire(&maps->a2f);
      tmap_acquire(&maps->g3);
      YCursor cf = cur, cb = cur;  // the stored-tile and the G3 streams
      if (!tc_fused_producer<NPAD, TM>(
              S, total,
              [&](int, int* c, int* tr) {
                *c = cf.c;
                *tr = cf.rb;
                cf.next();
              },
              [&](int, int* c, int* tr) {
                *c = cb.c;
                *tr = cb.rb;
                cb.next();
              },
              maps, true)) {
        timed_out = true;
        *S.acc.abort_flag = 1;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      for (int it = 0; it < total && !timed_out; ++it) {
        bool ok;
        if constexpr (TM)
          ok = tc_fused_mma_tm<NPAD>(S, tmem, it, kIdesc);
        else
          ok = tc_fused_mma<NPAD, true>(S, tmem, it, kIdesc);
        if (!ok) {
          timed_out = true;
          *S.acc.abort_flag = 1;
        }
      }
    }
  } else if (warp >= 6) {
    for (int it = 0; it < total && !timed_out; ++it) {
      bool ok = !tc_aborted(S.acc);
      if constexpr (TM)
        ok = ok && tc_convert_chunk_tm_y<NPAD>(S, tmem, it, listed);
      else
        ok = ok && tc_convert_chunk<NPAD, true>(S, it, listed);
      if (!ok) {
        timed_out = true;
        *S.acc.abort_flag = 1;
      }
    }
  } else {  // epilogue: every item of this CTA, empty ones included, writes its rows
    const uint32_t tlane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    float* yp = static_cast<float*>(io->ypart);
    YCursor t = cur;
    int it = 0;
    for (int k = blockIdx.x; k < t.nitems && !timed_out; k += gridDim.x) {
      t.set(k);
      float y[MPAD];
#pragma unroll
      for (int j = 0; j < MPAD; ++j) y[j] = 0.0f;
      for (int c = t.cb; c < t.ce; ++c, ++it) {
        bool ok;
        if constexpr (TM)
          ok = tc_drain_tm<NPAD>(S.acc, tlane, it, y);
        else
          ok = tc_drain<NPAD, 3>(S.acc, tlane, it, y);
        if (!ok) {
          timed_out = true;
          *S.acc.abort_flag = 1;
          break;
        }
      }
      const int r = t.rb * kTcRows2 + warp * 32 + lane;
      if (!timed_out && r < a.p) {
#pragma unroll
        for (int j = 0; j < MPAD; ++j)
          if (j < a.m) yp[(static_cast<int64_t>(t.sp) * a.m + j) * a.p + r] = y[j];
      }
    }
  }
  if (timed_out) atomicOr(&st->error, static_cast<int>(kErrTimeout));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::kCols);
  }
}

// ---------------------------------------------------------------- host

int tc_t_ctas_per_sm(int npad, int na, bool fused) { return fused ? 1 : tc_ctas_per_sm(npad, na); }

int tc_smem_bytes(int npad, int na) {
  return tc_stages(npad, na) * (na * static_cast<int>(kTcA) + npad * 128) + 1024 + 512;
}

bool tc_supported(int device) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  return major == 10 && minor == 3;  // built for sm_103a only
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// bf16 matrix with inner extent `inner` (contiguous) and `outer` rows of
// `stride_elems`; box 64 x box_outer, 128-byte swizzle, zero fill outside.
static bool encode_bf16(CUtensorMap* m, const void* base, int64_t inner, int64_t outer, int64_t stride_elems,
                        int box_outer) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(stride_elems) * 2};
  const cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(box_outer)};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encode_f32(CUtensorMap* m, const void* base, int64_t inner, int64_t outer, int64_t stride_elems,
                       int box_outer, bool swizzle = true, int box_inner = 32) {
  const EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(stride_elems) * 4};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_inner), static_cast<cuuint32_t>(box_outer)};
  const cuuint32_t estr[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_encode_maps_f32(TcMaps* maps, const void* A, int64_t p, int64_t n, int64_t ld, const void* x3, int p_pad,
                       const void* g3, int n_pad, int npad, const void* g3c) {
  if (!encode_bf16(&maps->x3, x3, p, npad, p_pad, npad) || !encode_bf16(&maps->g3, g3, n, npad, n_pad, npad) ||
      !encode_f32(&maps->a1f, A, p, n, ld, kTcTile1) || !encode_f32(&maps->a2f, A, p, n, ld, 64))
    return record_error(GPSPCA_ECUDA, "cuTensorMapEncodeTiled failed for the fused tensor-core sweep");
  if (g3c) {  // the Y pass over listed columns: A gathered a column at a time, G3c in rows of ceil(n / 64) * 64
    const int64_t n64 = (n + 63) / 64 * 64;
    if (!encode_f32(&maps->a2g, A, p, n, ld, 1, false, kTcRows2) ||
        !encode_bf16(&maps->g3c, g3c, n64, npad, n64, npad))
      return record_error(GPSPCA_ECUDA, "cuTensorMapEncodeTiled failed for the listed-column tensor-core sweep");
  }
  return GPSPCA_OK;
}

int tc_fused_smem_bytes(int npad) { return tc_fused_smem(npad); }

int tc_encode_maps(TcMaps* maps, const void* planes, int na, int64_t plane, int64_t p, int64_t n, int64_t ld,
                   const void* x3, int p_pad, const void* g3, int n_pad, int npad, const void* g3c) {
  bool ok = encode_bf16(&maps->x3, x3, p, npad, p_pad, npad) && encode_bf16(&maps->g3, g3, n, npad, n_pad, npad);
  for (int pl = 0; pl < na && ok; ++pl) {
    const void* base = static_cast<const __nv_bfloat16*>(planes) + pl * plane;
    ok = encode_bf16(&maps->a1[pl], base, p, n, ld, kTcTile1) && encode_bf16(&maps->a2[pl], base, p, n, ld, 64);
  }
  if (ok && g3c) {  // the Y pass over listed columns: G3c in rows of ceil(n / 64) * 64
    const int64_t n64 = (n + 63) / 64 * 64;
    ok = encode_bf16(&maps->g3c, g3c, n64, npad, n64, npad);
  }
  if (!ok) return record_error(GPSPCA_ECUDA, "cuTensorMapEncodeTiled failed for the tensor-core sweep");
  return GPSPCA_OK;
}

// float A -> three bf16 planes (a = a0 + a1 + a2 exactly); fp8 -> its values
// in bf16 (exact; the column scale stays separate); bf16 with a layout TMA
// cannot read -> a copy with the padded column stride.  Block (x, y): columns
// y, y + gridDim.y, ...; rows by the threads of x (coalesced along a column).
template <typename TA>
__global__ void tc_convert_kernel(const IO* io, int64_t p, int64_t n, int64_t ld, int64_t ldc) {
  const TA* A = static_cast<const TA*>(io->A);
  __nv_bfloat16* planes = static_cast<__nv_bfloat16*>(io->tc_planes);
  const int64_t plane = n * ldc;
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= p) return;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const float v = to_tc<TA>(A[i * ld + r]);
    if constexpr (sizeof(TA) == 4) {
      __nv_bfloat16 b0, b1, b2;
      split3(v, b0, b1, b2);
      planes[i * ldc + r] = b0;
      planes[plane + i * ldc + r] = b1;
      planes[2 * plane + i * ldc + r] = b2;
    } else {
      planes[i * ldc + r] = __float2bfloat16_rn(v);  // exact for fp8 and bf16 values
    }
  }
}

void launch_tc_convert(int dtype, const IO* io, int64_t p, int64_t n, int64_t ld, int64_t ldc, cudaStream_t s) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned bx = static_cast<unsigned>((p + 255) / 256);
  const unsigned by = static_cast<unsigned>(std::min<int64_t>(n, std::max<int64_t>(1, (nsm * 16) / bx)));
  const dim3 grid(bx, by);
  if (dtype == GPSPCA_F32)
    tc_convert_kernel<float><<<grid, 256, 0, s>>>(io, p, n, ld, ldc);
  else if (dtype == GPSPCA_FP8_E4M3)
    tc_convert_kernel<__nv_fp8_e4m3><<<grid, 256, 0, s>>>(io, p, n, ld, ldc);
  else if (dtype == GPSPCA_BF16)  // a layout TMA cannot read in place: padded copy
    tc_convert_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(io, p, n, ld, ldc);
}

template <int NPAD, int NA>
static void launch_tc_npad(const TcArgs& a, int nsm, cudaStream_t s, bool t_only) {
  static bool once = [] {
    cudaFuncSetAttribute(tc_t_kernel<NPAD, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(NPAD, NA));
    cudaFuncSetAttribute(tc_y_kernel<NPAD, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(NPAD, NA));
    return true;
  }();
  (void)once;
  const int smem = tc_smem_bytes(NPAD, NA);
  tc_prep_kernel<<<dim3((a.p + 255) / 256, a.mpad), 256, 0, s>>>(a);
  if (a.from_ritz) {
    tc_t_from_ritz_kernel<NPAD / 3><<<(a.n + 255) / 256, 256, 0, s>>>(a);
  } else {
    tc_t_kernel<NPAD, NA><<<std::max(1, std::min(a.ntile1 * a.ksplit1, tc_ctas_per_sm(NPAD, NA) * nsm)), kTcThreads,
                            smem, s>>>(a);
    if (a.ksplit1 > 1) tc_t_combine_kernel<NPAD / 3><<<dim3((a.n + 255) / 256, NPAD / 3), 256, 0, s>>>(a);
  }
  if (t_only) return;
  if (a.sparse && !a.sketch) {
    const int nb = (a.n + kTcCompactCols - 1) / kTcCompactCols;
    tc_count_kernel<<<nb, 256, 0, s>>>(a);
    tc_compact_kernel<NPAD / 3><<<nb, 256, 0, s>>>(a);
  }
  tc_y_kernel<NPAD, NA><<<dim3(a.nrow2, a.nsplit2), kTcThreads, smem, s>>>(a);
}

template <int NPAD>
static void launch_tc_fused_npad(const TcArgs& a, int nsm, cudaStream_t s, bool t_only) {
  constexpr bool kTM = tc_fused_tm(NPAD);  // planes in tensor memory where they fit
  const int smem_t = kTM ? tc_fused_tm_smem(NPAD) : tc_fused_smem(NPAD);
  static bool once = [smem_t] {
    cudaFuncSetAttribute(tc_t_fused_kernel<NPAD, kTM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_t);
    cudaFuncSetAttribute(tc_y_fused_kernel<NPAD, kTM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_t);
    return true;
  }();
  (void)once;
  tc_prep_kernel<<<dim3((a.p + 255) / 256, a.mpad), 256, 0, s>>>(a);
  if (a.from_ritz) {
    tc_t_from_ritz_kernel<NPAD / 3><<<(a.n + 255) / 256, 256, 0, s>>>(a);
  } else {
    tc_t_fused_kernel<NPAD, kTM>
        <<<std::max(1, std::min(a.ntile1 * a.ksplit1, nsm)), kTcFusedThreads, smem_t, s>>>(a);
    if (a.ksplit1 > 1) tc_t_combine_kernel<NPAD / 3><<<dim3((a.n + 255) / 256, NPAD / 3), 256, 0, s>>>(a);
  }
  if (a.norms) tc_norms_kernel<<<(a.n + 255) / 256, 256, 0, s>>>(a);
  if (t_only) return;
  if (a.sparse && !a.sketch) {
    const int nb = (a.n + kTcCompactCols - 1) / kTcCompactCols;
    tc_count_kernel<<<nb, 256, 0, s>>>(a);
    tc_compact_kernel<NPAD / 3><<<nb, 256, 0, s>>>(a);
  }
  tc_y_fused_kernel<NPAD, kTM><<<std::max(1, std::min(a.nrow2 * a.nsplit2, nsm)), kTcFusedThreads, smem_t, s>>>(a);
}

template <int NA>
static void launch_tc_na(const TcArgs& a, int npad, int nsm, cudaStream_t s, bool t_only) {
  switch (npad) {
    case 48: launch_tc_npad<48, NA>(a, nsm, s, t_only); break;
    case 96: launch_tc_npad<96, NA>(a, nsm, s, t_only); break;
    case 144: launch_tc_npad<144, NA>(a, nsm, s, t_only); break;
    default: launch_tc_npad<192, NA>(a, nsm, s, t_only); break;
  }
}

// t_only: the X3 preparation and the T pass (with its combine step) alone.
void launch_tc_sweep(const TcArgs& a, int npad, cudaStream_t s, bool t_only) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (a.fused) {
    switch (npad) {
      case 48: launch_tc_fused_npad<48>(a, nsm, s, t_only); break;
      case 96: launch_tc_fused_npad<96>(a, nsm, s, t_only); break;
      case 144: launch_tc_fused_npad<144>(a, nsm, s, t_only); break;
      default: launch_tc_fused_npad<192>(a, nsm, s, t_only); break;
    }
  } else if (a.na == 3) {
    launch_tc_na<3>(a, npad, nsm, s, t_only);
  } else {
    launch_tc_na<1>(a, npad, nsm, s, t_only);
  }
}

}  // namespace gpspca
