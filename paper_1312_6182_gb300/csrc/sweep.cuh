// Fused single-read sweep of the generalized power iteration (Section 2,
// Table 1): for a slab of columns a_i of A it forms t_ij = a_i^T x_j, applies
// the formulation's threshold, and accumulates y_j += g_ij a_i, reading each
// column from HBM once.
//
// Decomposition
//  * Thread-block clusters of C CTAs own a contiguous slab of columns; CTA r
//    of a cluster owns rows [r*ps, (r+1)*ps) of every column in the slab.
//  * One elected thread streams W-column tiles of the CTA's rows through an
//    S-stage shared-memory ring with 1-D bulk (TMA) copies on mbarriers.
//  * Each thread owns R = NCH*VEC fixed rows; the iterate x (MG components)
//    and the accumulated y for those rows live in registers.
//  * Per tile: per-thread partial dots -> warp reduce-scatter (31 shuffles
//    for 32 values) -> CTA sum -> partial sums of the C CTAs of the cluster
//    exchanged through distributed shared memory and added in rank order, so
//    every CTA holds the same t.  The threshold runs on one lane per
//    (column, component), then every thread applies g to its rows of the
//    tile still in shared memory (the second use of the tile costs no HBM
//    traffic).  The sweep stores t; the reduction forms the Table 1
//    objective from it in double, off this kernel's critical path.
//  * Epilogue: each cluster writes its partial y (all p rows); a separate
//    deterministic reduction adds them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.h"
#include "ptx.cuh"

namespace gpspca {

template <typename TA>
struct Elem;
template <>
struct Elem<float> {
  using TC = float;
  static constexpr int VEC = 4;    // elements per shared-memory vector load (16 B)
  static constexpr int ALIGN = 4;  // elements per 16 bytes
};
template <>
struct Elem<double> {
  using TC = double;
  static constexpr int VEC = 2;
  static constexpr int ALIGN = 2;
};
template <>
struct Elem<__nv_bfloat16> {
  using TC = float;
  static constexpr int VEC = 4;  // 8-byte loads
  static constexpr int ALIGN = 8;
};
template <>
struct Elem<__nv_fp8_e4m3> {
  using TC = float;
  static constexpr int VEC = 4;  // 4-byte loads
  static constexpr int ALIGN = 16;
};

__device__ __forceinline__ void load_vec(const float* p, float (&v)[4]) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void load_vec(const double* p, double (&v)[2]) {
  const double2 f = *reinterpret_cast<const double2*>(p);
  v[0] = f.x; v[1] = f.y;
}
__device__ __forceinline__ void load_vec(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(u.x << 16);
  v[1] = __uint_as_float(u.x & 0xffff0000u);
  v[2] = __uint_as_float(u.y << 16);
  v[3] = __uint_as_float(u.y & 0xffff0000u);
}
__device__ __forceinline__ float2 fp8x2_to_float2(uint32_t bits16) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(bits16), __NV_E4M3);
  return __half22float2(__half2(h));
}
__device__ __forceinline__ void load_vec(const __nv_fp8_e4m3* p, float (&v)[4]) {
  const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
  const float2 a = fp8x2_to_float2(u & 0xffffu);
  const float2 b = fp8x2_to_float2(u >> 16);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Packed float pairs for the float-compute sweeps: two rows' values in one
// 64-bit register, multiplied and accumulated by one fma.rn.f32x2 (two IEEE
// float fmas per instruction on sm_100-class SMs).  The block sweep is bound
// by instruction issue at the occupancy its register tiles allow; the pairs
// halve the FMA instructions of its dot products and rank update.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 f2unpack(uint64_t v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// Four consecutive elements as two float pairs (rows 0,1 and 2,3).
__device__ __forceinline__ void load_pairs(const float* p, uint64_t (&a)[2]) {
  const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(p);
  a[0] = u.x;
  a[1] = u.y;
}
template <typename TA>
__device__ __forceinline__ void load_pairs(const TA* p, uint64_t (&a)[2]) {
  float v[4];
  load_vec(p, v);
  a[0] = f2pack(v[0], v[1]);
  a[1] = f2pack(v[2], v[3]);
}

template <typename TA>
__device__ __forceinline__ typename Elem<TA>::TC to_tc(TA v);
template <>
__device__ __forceinline__ float to_tc<float>(float v) { return v; }
template <>
__device__ __forceinline__ double to_tc<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_tc<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_tc<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return static_cast<float>(v); }

// Threshold of Table 1 for one entry t = a_i^T x_j (already scaled), in
// double.  term: the summand of the reformulated objective; g: the gradient
// factor (the power step uses y_j = sum_i g_ij a_i); zr: the unnormalised
// original-form loading.  Ties are inactive; sign(0) = 0.
struct Thr {
  double term, g, zr;
};
__device__ __forceinline__ Thr threshold(int form, double t, double gam, double mu) {
  Thr r;
  if ((form & 1) == 0) {  // SL1 / BL1
    const double s = fmax(mu * fabs(t) - gam, 0.0);
    const double sg = (t > 0.0) ? 1.0 : ((t < 0.0) ? -1.0 : 0.0);
    r.term = s * s;
    r.g = mu * sg * s;
    r.zr = sg * s;
  } else {  // SL0 / BL0
    const double u = mu * t;
    const bool act = u * u > gam;
    r.term = act ? (u * u - gam) : 0.0;
    r.g = act ? mu * mu * t : 0.0;
    r.zr = act ? u : 0.0;
  }
  return r;
}

// Reduce K per-lane values over the warp (K a power of two <= 32): lane L
// returns the warp total of v[L % K].  K - 1 shuffles halve the vector over
// the low lane bits, then log2(32/K) more add the remaining lane groups.
template <int K, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[K], int lane) {
#pragma unroll
  for (int h = K / 2; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
#pragma unroll
  for (int o = K; o < 32; o <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

// Gradient factor of Table 1 in the compute type (the threshold decision on
// the critical path of a tile); the objective is recomputed in double off it.
template <typename TC>
__device__ __forceinline__ TC grad_factor(int form, TC t, TC gam, TC mu) {
  if ((form & 1) == 0) {
    const TC s = mu * (t < TC(0) ? -t : t) - gam;
    if (!(s > TC(0))) return TC(0);
    return t > TC(0) ? mu * s : -(mu * s);
  }
  const TC u = mu * t;
  return (u * u > gam) ? mu * mu * t : TC(0);
}

constexpr int kRingSlack = 33 * 4 * 4 * 8;  // 33 * NCHmax * VECmax * 8-byte elements

// Shared-memory layout of the sweep kernel (host and device agree on it).
struct SweepSmem {
  int stage_bytes, bars, xbars, red, xrecv, wsm, total;
};
constexpr int kMaxCluster = 8;
constexpr int kXSlots = 2;  // cluster-exchange slots, by tile parity (4 when tiles overlap, see the main loop)
__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }
__host__ __device__ inline SweepSmem sweep_smem_layout(int W, int S, int ps, int esize, int tcsize, int nwarps, int m,
                                                      int mg, int xslots = kXSlots) {
  SweepSmem L;
  L.stage_bytes = W * ps * esize;  // ps*esize is a multiple of 16
  // Threads own rows up to NCH*threads*VEC >= ps; rows past the CTA's slice
  // are read (and masked) but must stay inside the allocation: the slack
  // after the ring covers the largest overshoot (< 33 * NCH * VEC elements).
  int o = align_up(S * L.stage_bytes + kRingSlack, 128);
  L.bars = o; o += 8 * S;         // tile-copy mbarriers
  L.xbars = o; o += 8 * xslots;  // cluster-exchange mbarriers (tile mod xslots)
  o = align_up(o, 16);
  L.red = o; o += 2 * nwarps * 32 * tcsize;          // warp partials, by tile parity
  L.xrecv = o; o += xslots * kMaxCluster * 32 * tcsize;  // partials pushed by cluster peers
  L.wsm = o; o += m * mg * tcsize;
  L.total = align_up(o, 128);
  return L;
}

// (column, component) dot products reduced per tile, one per lane of a warp
// (single-unit tiles hold at most 8 columns; long columns leave room for 1-3
// anyway).  The host caps the tile width at sweep_kb(mg) / mg with the same
// function.
__host__ __device__ constexpr int sweep_kb(int mg) { return mg == 1 ? 8 : 32; }

// NRM: the sweep also forms each column's squared norm (one more reduction
// slot per column), for the block start's first power step, which reads A
// anyway: the column norms then need no pass of their own.
template <typename TA, int MG, int NCH, bool NRM = false, int FW = 0>
struct SweepCfg {
  using TC = typename Elem<TA>::TC;
  static constexpr int VEC = Elem<TA>::VEC;
  static constexpr int R = NCH * VEC;
  static constexpr int KB = sweep_kb(MG);
  static constexpr int SL = MG + (NRM ? 1 : 0);  // reduction slots per column
  static constexpr int WB = KB / SL;             // most columns one tile can hold
  // registers per thread: x and y tiles, the reduction slots, and a fixed
  // part (addresses, loop state, loads in flight) measured with -Xptxas -v
  static constexpr int REGS = static_cast<int>(sizeof(TC) / 4) * (2 * R * MG + KB + (MG == 1 ? 64 : (MG == 2 ? 60 : 40)));
  // register arrays of x and y beyond this spill; such variants are not built;
  // the fixed-width form exists for the float pairs only
  static constexpr bool kBuilt = static_cast<int>(sizeof(TC) / 4) * 2 * R * MG <= 160 &&
                                 (FW == 0 || (sizeof(TC) == 4 && VEC == 4 && FW >= 1 && FW <= WB));
  // each of the 4 SM sub-partitions holds a quarter of the CTA's warps in its
  // own 16K-register file: whole warps per sub-partition, times four
  static constexpr int WARPS_PER_SMSP = 16384 / (32 * REGS);
  static constexpr int MAXT_RAW = WARPS_PER_SMSP * 4 * 32;
  static constexpr int MAXT = MAXT_RAW >= 1024 ? 1024 : (MAXT_RAW < 128 ? 128 : MAXT_RAW);
};

// FW > 0: tiles are exactly FW columns wide (a.W == FW).  The dot products
// and the rank update then run every column slot of a tile without a test on
// the tile's width, so the columns' chains interleave; the last tile's empty
// slots hold zeros or earlier columns of A (the ring starts zeroed) and get
// g = 0.  FW = 0: any width up to WB, each slot tested.
template <typename TA, int MG, int NCH, bool NRM = false, int FW = 0>
__device__ __forceinline__ void sweep_body(const SweepArgs& a) {
  using Cfg = SweepCfg<TA, MG, NCH, NRM, FW>;
  constexpr int SL = Cfg::SL;
  using TC = typename Cfg::TC;
  constexpr int VEC = Cfg::VEC;
  constexpr int WB = Cfg::WB;
  constexpr int KB = Cfg::KB;
  constexpr bool kFP8 = (sizeof(TA) == 1);

  State* st = a.st;
  if (st->n_active == 0) return;  // uniform across the grid
  constexpr int WL = FW > 0 ? FW : WB;  // column slots a tile loop runs
  if (a.W > WB || a.W < 1 || (FW > 0 && a.W != FW)) {  // a tile width this variant does not run: refuse
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&st->error, static_cast<int>(kErrLaunch));
    return;
  }

  const IO* io = a.io;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = nthr >> 5;
  uint32_t C;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
  const uint32_t cr = cluster_ctarank();
  const int cl = blockIdx.x / static_cast<int>(C);
  const int m = a.m;
  const int p = a.p;
  const int n = a.n;
  const int ps = a.ps;
  const int row0 = static_cast<int>(cr) * ps;
  const int rows_valid = max(0, min(ps, p - row0));
  const int col_begin = cl * a.cols_per_cl;
  const int col_end = min(n, col_begin + a.cols_per_cl);
  const int ncols = max(0, col_end - col_begin);
  const int W = a.W;
  const int S = a.S;
  const int ntiles = (ncols + W - 1) / W;
  const bool block = a.form >= 2;
  // the block start's power steps use g = t (L0 threshold at gamma = 0, mu = 1)
  const bool sketch = a.sketch != 0;
  const int form = sketch ? GPSPCA_SL0 : a.form;
  const TA* __restrict__ A = static_cast<const TA*>(io->A);
  const int64_t ld = a.ld;

  // overlapped tiles (passes whose tile chain waits on a cluster exchange or
  // a single column): phase A of tile t+1 runs before phase B of tile t,
  // with four exchange slots
  const bool ov = a.overlap != 0;
  const int xsl = ov ? 4 : kXSlots;
  extern __shared__ __align__(128) unsigned char smem[];
  const SweepSmem L = sweep_smem_layout(W, S, ps, sizeof(TA), sizeof(TC), nwarps, m, MG, xsl);
  TA* stage = reinterpret_cast<TA*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* xbars = reinterpret_cast<uint64_t*>(smem + L.xbars);
  TC* red = reinterpret_cast<TC*>(smem + L.red);
  TC* xrecv = reinterpret_cast<TC*>(smem + L.xrecv);
  TC* wsm = reinterpret_cast<TC*>(smem + L.wsm);
  __shared__ TC gam_c[MG], mu_c[MG];
  __shared__ int act[MG];
  const int stage_elems = W * ps;

  // ---- prologue: parameters, weights, barriers, first tiles
  if (tid < MG) {
    const bool v = tid < a.mg_valid && !sketch;
    gam_c[tid] = v ? static_cast<TC>(st->gamma[a.j0 + tid]) : TC(0);
    mu_c[tid] = v ? static_cast<TC>(io->mu[a.j0 + tid]) : TC(1);
    act[tid] = (tid < a.mg_valid) ? st->active[a.j0 + tid] : 0;
  }
  for (int idx = tid; idx < m * MG; idx += nthr) {
    const int l = idx / MG, j = idx % MG;
    wsm[idx] = (j < a.mg_valid) ? static_cast<TC>(st->W[l * m + a.j0 + j]) : TC(0);
  }
  const uint32_t bytes_per_col = static_cast<uint32_t>(align_up(rows_valid * static_cast<int>(sizeof(TA)), 16));
  if constexpr (FW > 0) {  // zero the ring before the first bulk copy lands in it
    uint4* z = reinterpret_cast<uint4*>(smem);
    for (int i = tid; i < (S * L.stage_bytes + kRingSlack) / 16; i += nthr) z[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_async_smem();
  }
  if (tid == 0) {
    if (a.fast)
      for (int s = 0; s < S; ++s) mbar_init(smem_u32(&bars[s]), 1);
    for (int xs = 0; xs < xsl; ++xs) mbar_init(smem_u32(&xbars[xs]), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (C > 1) cluster_sync_all();  // peers' exchange barriers are initialised before any push
  auto issue_tile = [&](int tile, int buf) {
    const int c0 = col_begin + tile * W;
    const int wv = min(W, col_end - c0);
    const uint32_t bar = smem_u32(&bars[buf]);
    mbar_arrive_expect_tx(bar, bytes_per_col * static_cast<uint32_t>(wv));
    for (int w = 0; w < wv; ++w) {
      const TA* src = A + static_cast<int64_t>(c0 + w) * ld + row0;
      bulk_g2s(smem_u32(stage + buf * stage_elems + w * ps), src, bytes_per_col, bar);
    }
  };
  if (a.fast && tid == 0) {
    const int pre = min(S, ntiles);
    for (int s = 0; s < pre; ++s) issue_tile(s, s);
  }

  // ---- iterate rows in registers: X_k = Y_{k-1} W_{k-1}
  const TC* __restrict__ Yp = static_cast<const TC*>(io->Y);
  // float compute: x and y also as row pairs (packed, see ffma2)
  constexpr bool kPair = sizeof(TC) == 4 && VEC == 4;
  TC x[NCH][VEC][MG];
  TC y[NCH][VEC][MG];
  uint64_t xp[NCH][2][MG], yp[NCH][2][MG];
  uint32_t vmask = 0;  // bit (c*VEC+v): row is inside this CTA's valid rows
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if ((c * nthr + tid) * VEC + v < rows_valid) vmask |= 1u << (c * VEC + v);
#pragma unroll
      for (int j = 0; j < MG; ++j) {
        x[c][v][j] = 0;
        y[c][v][j] = 0;
      }
    }
  }
  // block: all m columns of Y contribute; single-unit: only column j0+j
  const int lbeg = block ? 0 : a.j0;
  const int lend = block ? m : a.j0 + a.mg_valid;
  if (block) {
    // block forms: X = Y W was formed before this launch (form_x_kernel,
    // float-accurate however large W's entries); its rows are loaded here
    const TC* xf = static_cast<const TC*>(io->Xf);
#pragma unroll
    for (int j = 0; j < MG; ++j) {
      if (j >= a.mg_valid) continue;
      const TC* xl = xf + static_cast<int64_t>(a.j0 + j) * p + row0;
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const int rl = (c * nthr + tid) * VEC + v;
          x[c][v][j] = (vmask & (1u << (c * VEC + v))) ? xl[rl] : TC(0);
        }
    }
  } else {
    // single-unit forms: column j0+j of Y times its own weight
    for (int l = lbeg; l < lend; ++l) {
      TC wl[MG];
#pragma unroll
      for (int j = 0; j < MG; ++j) wl[j] = (l == a.j0 + j) ? wsm[l * MG + j] : TC(0);
      const TC* yl = Yp + static_cast<int64_t>(l) * p + row0;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const int rl = (c * nthr + tid) * VEC + v;
          const TC yv = (vmask & (1u << (c * VEC + v))) ? yl[rl] : TC(0);
#pragma unroll
          for (int j = 0; j < MG; ++j) x[c][v][j] += yv * wl[j];
        }
      }
    }
  }
  if (cl == 0 && !sketch) {  // the iterate that this sweep evaluates is an output
    TC* Xo = static_cast<TC*>(io->X);
#pragma unroll
    for (int j = 0; j < MG; ++j) {
      if (j < a.mg_valid && act[j]) {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            if (vmask & (1u << (c * VEC + v)))
              Xo[static_cast<int64_t>(a.j0 + j) * p + row0 + (c * nthr + tid) * VEC + v] = x[c][v][j];
      }
    }
  }

  // pair masks: all ones for rows of this CTA's slice, zero outside (the
  // ring holds no data there); one AND per pair, in the one copy of the loop
  // (a second, unmasked copy for full tiles was measured 9% slower)
  uint64_t pmask[NCH][2];
  if constexpr (kPair) {
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        pmask[c][h] = ((vmask >> (c * VEC + 2 * h)) & 1u ? 0xffffffffull : 0ull) |
                      ((vmask >> (c * VEC + 2 * h + 1)) & 1u ? 0xffffffff00000000ull : 0ull);
#pragma unroll
        for (int j = 0; j < MG; ++j) {
          xp[c][h][j] = f2pack(static_cast<float>(x[c][2 * h][j]), static_cast<float>(x[c][2 * h + 1][j]));
          yp[c][h][j] = 0;
        }
      }
  }
  bool timed_out = false;
  TC* Tout = static_cast<TC*>(io->T);
  const float* cscale = io->col_scale;
  // lane L of every warp owns slot L = (column w = L / MG, component j = L % MG)
  const int wq = lane / SL, jq = lane % SL;

  // Tiles run in order: phase A (partial dots, CTA total, push to the
  // cluster peers), then phase B (the peers' totals, threshold, rank update).
  // Overlapping phase A of tile t+1 with phase B of tile t was measured
  // slower on GB300 (it costs a stage of prefetch or narrower tiles, and
  // full-width tiles with the deeper ring matter more).

  // phase A: returns this CTA's total for its lane's slot of tile `tile`
  auto phase_a = [&](int tile) -> TC {
    const int buf = tile % S;
    const TA* sb = stage + buf * stage_elems;
    const int c0 = col_begin + tile * W;
    const int wv = min(W, col_end - c0);
    if (a.fast) {
      if (!mbar_wait_bounded(smem_u32(&bars[buf]), static_cast<uint32_t>((tile / S) & 1))) timed_out = true;
    } else {
      __syncthreads();  // the buffer's previous tile (tile - S) is fully consumed
      TA* sbw = stage + buf * stage_elems;
      for (int w = 0; w < wv; ++w) {
        const TA* src = A + static_cast<int64_t>(c0 + w) * ld + row0;
        for (int r = tid; r < rows_valid; r += nthr) sbw[w * ps + r] = src[r];
      }
      __syncthreads();
    }
    // partial dots over this thread's rows
    TC pd[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) pd[i] = 0;
    if constexpr (kPair) {
#pragma unroll
      for (int w = 0; w < WL; ++w) {
        if (FW > 0 || w < wv) {
          const TA* colp = sb + w * ps;
          uint64_t acc[SL];
#pragma unroll
          for (int j = 0; j < SL; ++j) acc[j] = 0;
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            uint64_t a2[2];
            load_pairs(colp + (c * nthr + tid) * VEC, a2);
            a2[0] &= pmask[c][0];
            a2[1] &= pmask[c][1];
#pragma unroll
            for (int j = 0; j < MG; ++j) {
              acc[j] = ffma2(a2[0], xp[c][0][j], acc[j]);
              acc[j] = ffma2(a2[1], xp[c][1][j], acc[j]);
            }
            if constexpr (NRM) {  // the column's squared norm
              acc[MG] = ffma2(a2[0], a2[0], acc[MG]);
              acc[MG] = ffma2(a2[1], a2[1], acc[MG]);
            }
          }
#pragma unroll
          for (int j = 0; j < SL; ++j) {  // even + odd rows of column w
            const float2 f = f2unpack(acc[j]);
            pd[w * SL + j] = f.x + f.y;
          }
        }
      }
    } else {
#pragma unroll
    for (int w = 0; w < WB; ++w) {
      if (w < wv) {
        const TA* colp = sb + w * ps;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          TC av[VEC];
          load_vec(colp + (c * nthr + tid) * VEC, av);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const TC aval = (vmask & (1u << (c * VEC + v))) ? av[v] : TC(0);
#pragma unroll
            for (int j = 0; j < MG; ++j) pd[w * SL + j] += aval * x[c][v][j];
            if constexpr (NRM) pd[w * SL + MG] += aval * aval;
          }
        }
      }
    }
    }
    // Lane L holds the warp total of slot L % KB.  One block barrier per
    // tile: afterwards every warp adds the warp totals itself (partials are
    // double-buffered by tile parity).
    const TC mine = warp_reduce_scatter<KB>(pd, lane);
    TC* redp = red + (tile & 1) * nwarps * 32;
    redp[warp * 32 + lane] = mine;
    const int xs = tile % xsl;
    if (C > 1 && tid == 0)  // this tile's pushes from the C-1 peers
      mbar_arrive_expect_tx(smem_u32(&xbars[xs]), static_cast<uint32_t>((C - 1) * KB * sizeof(TC)));
    __syncthreads();  // (1) warp partials visible; phase B of the previous tile is done everywhere
    // refill the stage whose tile every thread has finished: tile - 1's
    // (tile - 2's when tiles overlap: phase B of tile - 1 comes after this)
    const int lag = ov ? 2 : 1;
    if (a.fast && tid == 0 && tile >= lag && tile - lag + S < ntiles) issue_tile(tile - lag + S, (tile - lag) % S);
    TC t = 0;
    for (int w2 = 0; w2 < nwarps; ++w2) t += redp[w2 * 32 + lane];
    if (C > 1 && warp == 0 && lane < KB) {  // push this CTA's total to every peer (one-way)
      TC* slot = xrecv + xs * kMaxCluster * 32;
      const uint32_t src = smem_u32(&slot[cr * 32 + lane]);
      const uint32_t bar = smem_u32(&xbars[xs]);
      for (uint32_t r = 0; r < C; ++r)
        if (r != cr) st_async_remote(dsmem_map(src, r), t, dsmem_map(bar, r));
    }
    return t;
  };

  // phase B: the cluster total, threshold, T, rank update of tile `tile`
  auto phase_b = [&](int tile, TC t) {
    const int buf = tile % S;
    const TA* sb = stage + buf * stage_elems;
    const int c0 = col_begin + tile * W;
    const int wv = min(W, col_end - c0);
    const bool norm_slot = NRM && jq == MG;  // this lane's slot is a column's squared norm
    const bool mine_valid = lane < WB * SL && wq < wv && !norm_slot && jq < a.mg_valid;
    if (C > 1) {  // wait for the peers' totals, add all C in rank order
      const int xs = tile % xsl;
      TC* slot = xrecv + xs * kMaxCluster * 32;
      if (!mbar_wait_bounded(smem_u32(&xbars[xs]), static_cast<uint32_t>((tile / xsl) & 1))) timed_out = true;
      TC tot = 0;
      for (uint32_t r = 0; r < C; ++r) tot += (r == cr) ? t : slot[r * 32 + lane];
      t = tot;
    }
    TC scl = TC(1);
    if (kFP8 && mine_valid) scl = static_cast<TC>(cscale[c0 + wq]);
    TC g = 0;
    if (mine_valid) {
      t *= scl;
      g = grad_factor<TC>(form, t, gam_c[jq], mu_c[jq]) * scl;
    }
    if constexpr (NRM) {  // ||a_i|| (the column-norm pass's output and its non-finite check)
      if (norm_slot && warp == 0 && cr == 0 && lane < WB * SL && wq < wv) {
        double c = sqrt(static_cast<double>(t));
        if (kFP8) c *= static_cast<double>(cscale[c0 + wq]);
        if (!isfinite(c)) atomicOr(&st->error, static_cast<int>(kErrNonFinite));
        io->cnorm[c0 + wq] = c;
      }
    }
    // T for the objective (formed by the reduction) and the loadings
    if (warp == 0 && mine_valid && cr == 0 && !sketch && act[jq])
      Tout[static_cast<int64_t>(a.j0 + jq) * n + c0 + wq] = t;
    // rank update y += g a over this thread's rows of the tile
#pragma unroll
    for (int w = 0; w < WL; ++w) {
      if (FW > 0 || w < wv) {
        TC gw[MG];
#pragma unroll
        for (int j = 0; j < MG; ++j) gw[j] = __shfl_sync(0xffffffffu, g, w * SL + j);
        const TA* colp = sb + w * ps;
        if constexpr (kPair) {
          uint64_t g2[MG];
#pragma unroll
          for (int j = 0; j < MG; ++j) g2[j] = f2pack(static_cast<float>(gw[j]), static_cast<float>(gw[j]));
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            uint64_t a2[2];
            load_pairs(colp + (c * nthr + tid) * VEC, a2);
#pragma unroll
            for (int j = 0; j < MG; ++j) {
              yp[c][0][j] = ffma2(a2[0], g2[j], yp[c][0][j]);
              yp[c][1][j] = ffma2(a2[1], g2[j], yp[c][1][j]);
            }
          }
        } else {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          TC av[VEC];
          load_vec(colp + (c * nthr + tid) * VEC, av);
#pragma unroll
          for (int v = 0; v < VEC; ++v)
#pragma unroll
            for (int j = 0; j < MG; ++j) y[c][v][j] += av[v] * gw[j];
        }
        }
      }
    }
  };

  if (ov) {
    // phase A of tile t+1 (its dot products) before phase B of tile t, so the
    // cluster exchange of tile t overlaps the next tile's arithmetic.  Safe
    // with four exchange slots: a push for tile t+1 into slot (t+1) mod 4
    // follows this CTA's phase B of tile t-1, which waited for every peer's
    // phase A of tile t-1, which each peer runs after its phase B of tile t-3,
    // the slot's previous reader.  The ring refill lags one more tile.
    TC t_cur = ntiles > 0 ? phase_a(0) : TC(0);
    for (int tile = 0; tile < ntiles; ++tile) {
      const TC t_next = tile + 1 < ntiles ? phase_a(tile + 1) : TC(0);
      phase_b(tile, t_cur);
      t_cur = t_next;
    }
  } else {
    for (int tile = 0; tile < ntiles; ++tile) phase_b(tile, phase_a(tile));
  }

  // ---- epilogue: this cluster's partial of Y = A G and of the objective
  if constexpr (kPair) {
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < MG; ++j) {
          const float2 f = f2unpack(yp[c][h][j]);
          y[c][2 * h][j] = f.x;
          y[c][2 * h + 1][j] = f.y;
        }
  }
  TC* yout = static_cast<TC*>(io->ypart);
#pragma unroll
  for (int j = 0; j < MG; ++j) {
    if (j < a.mg_valid) {
      TC* dst = yout + (static_cast<int64_t>(cl) * m + a.j0 + j) * p + row0;
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if (vmask & (1u << (c * VEC + v))) dst[(c * nthr + tid) * VEC + v] = y[c][v][j];
    }
  }
  if (timed_out) atomicOr(&st->error, static_cast<int>(kErrTimeout));
  if (C > 1) cluster_sync_all();  // no CTA leaves while a peer may read its shared memory
}

template <typename TA, int MG, int NCH, bool NRM = false, int FW = 0>
__global__ void __launch_bounds__(SweepCfg<TA, MG, NCH, NRM, FW>::MAXT, 1) sweep_kernel(const SweepArgs a) {
  sweep_body<TA, MG, NCH, NRM, FW>(a);
}

// The sweep of instance blockIdx.z of a group of same-shape solves (clusters
// of one CTA; the instance's IO and State from the group's arrays).
template <typename TA, int MG, int NCH>
__global__ void __launch_bounds__(SweepCfg<TA, MG, NCH>::MAXT, 1) sweep_kernel_grouped(SweepArgs a, GroupPtrs g) {
  a.io = g.io[blockIdx.z];
  a.st = g.st[blockIdx.z];
  sweep_body<TA, MG, NCH>(a);
}

template <typename TA, int MG, int NCH>
const void* sweep_kernel_grouped_ptr() {
  if constexpr (SweepCfg<TA, MG, NCH>::kBuilt) {
    return reinterpret_cast<const void*>(&sweep_kernel_grouped<TA, MG, NCH>);
  } else {
    return nullptr;
  }
}

template <typename TA, int MG, int NCH, bool NRM = false, int FW = 0>
const void* sweep_kernel_ptr() {
  if constexpr (SweepCfg<TA, MG, NCH, NRM, FW>::kBuilt) {
    return reinterpret_cast<const void*>(&sweep_kernel<TA, MG, NCH, NRM, FW>);
  } else {
    return nullptr;
  }
}

}  // namespace gpspca
