// Host engine of libgpspca: launch planning, workspace, CUDA-graph execution
// of the generalized power iteration with a device-driven loop, the
// request scheduler for gpspca_submit/gpspca_poll, and the C ABI.
//
// One solve is one CUDA graph:
//   reset -> column norms -> start selection -> gather start -> reduce(start)
//   -> finish(start)  -> WHILE(cond) { sweep pass(es) -> reduce -> finish }
//   -> finalize
// The finish kernel decides on the device whether another sweep is needed
// and sets the WHILE node's condition, so no host round trip happens per
// iteration.  Every pointer a kernel dereferences lives in a device-side IO
// record that is rewritten before each launch, so a graph is cached per
// launch geometry and replayed for new buffers and parameters.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aux.cuh"
#include "deflate.cuh"
#include "plan.h"
#include "tc_sweep.cuh"

namespace gpspca {

const void* sweep_kernel_f32(int mg, int nch);
const void* sweep_kernel_f64(int mg, int nch);
const void* sweep_kernel_bf16(int mg, int nch);
const void* sweep_kernel_fp8(int mg, int nch);
const void* sweep_kernel_f32_nrm(int mg, int nch);
const void* sweep_kernel_f32_full(int mg, int nch, int fw);
const void* sweep_kernel_f32_nrm_full(int mg, int nch, int fw);
const void* sweep_kernel_f64_nrm(int mg, int nch);
const void* sweep_kernel_bf16_nrm(int mg, int nch);
const void* sweep_kernel_fp8_nrm(int mg, int nch);
const void* sweep_kernel_grouped_su(int dtype, int nch);

// ---------------------------------------------------------------- errors

static thread_local std::string t_last_error;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

#define GP_CUDA(call)                                                                           \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(GPSPCA_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------- dtype facts

struct DInfo {
  int esize, tcsize, vec, align;
};
static DInfo dinfo(int dt) {
  switch (dt) {
    case GPSPCA_F32: return {4, 4, Elem<float>::VEC, Elem<float>::ALIGN};
    case GPSPCA_F64: return {8, 8, Elem<double>::VEC, Elem<double>::ALIGN};
    case GPSPCA_BF16: return {2, 4, Elem<__nv_bfloat16>::VEC, Elem<__nv_bfloat16>::ALIGN};
    default: return {1, 4, Elem<__nv_fp8_e4m3>::VEC, Elem<__nv_fp8_e4m3>::ALIGN};
  }
}

// nrm: the variant that also forms the column norms
static const void* sweep_ptr(int dt, int mg, int nch, bool nrm = false) {
  switch (dt) {
    case GPSPCA_F32: return nrm ? sweep_kernel_f32_nrm(mg, nch) : sweep_kernel_f32(mg, nch);
    case GPSPCA_F64: return nrm ? sweep_kernel_f64_nrm(mg, nch) : sweep_kernel_f64(mg, nch);
    case GPSPCA_BF16: return nrm ? sweep_kernel_bf16_nrm(mg, nch) : sweep_kernel_bf16(mg, nch);
    default: return nrm ? sweep_kernel_fp8_nrm(mg, nch) : sweep_kernel_fp8(mg, nch);
  }
}

struct KAttr {
  int max_threads = 0;
  size_t local = 0;
  int max_dyn_smem = 0;  // dynamic shared memory this kernel may use
  bool ok = false;
};

static std::mutex g_attr_mu;
static std::map<const void*, KAttr> g_attr;

static KAttr kattr(const void* f) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto it = g_attr.find(f);
  if (it != g_attr.end()) return it->second;
  KAttr k;
  cudaFuncAttributes a;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncGetAttributes(&a, f) == cudaSuccess) {
    // the opt-in limit covers static and dynamic shared memory together
    const int dyn = optin - static_cast<int>(a.sharedSizeBytes);
    if (dyn > 0 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess) {
      k.max_threads = a.maxThreadsPerBlock;
      k.local = a.localSizeBytes;
      k.max_dyn_smem = dyn;
      k.ok = true;
    }
  }
  cudaGetLastError();
  g_attr[f] = k;
  return k;
}

// ---------------------------------------------------------------- planning

constexpr int kSmemBudget = 200 * 1024;  // stage ring + bookkeeping, per CTA
constexpr int64_t kTcLongRows = 16384;    // float columns this long take the tensor-core sweep for any m

static const int kMGs[] = {1, 2, 4, 5, 8};

// Components per pass: passes of gmax (a built width), the last one the
// smallest built width that holds the rest.
static std::vector<std::pair<int, int>> split_components(int m, int gmax) {
  std::vector<std::pair<int, int>> out;  // (mg, valid)
  int rem = m;
  while (rem > 0) {
    int mg = gmax;
    if (rem < gmax)
      for (int c : kMGs)
        if (c >= rem) { mg = c; break; }
    const int v = std::min(rem, mg);
    out.push_back({mg, v});
    rem -= v;
  }
  return out;
}

// Threads / tile width / stages of kernel k (nch rows-per-thread chunks) for
// one pass with cluster size C; false if it does not fit.
static bool fit_variant(int dt, int mg, int nch, const void* k, int ps, int m, bool nrm, Pass* out) {
  const DInfo d = dinfo(dt);
  if (!k) return false;
  const KAttr at = kattr(k);
  if (!at.ok || at.local > 0) return false;  // spilling variants are not used
  int threads = (ps + nch * d.vec - 1) / (nch * d.vec);
  threads = std::max(64, (threads + 31) / 32 * 32);
  if (threads > at.max_threads) return false;
  const int colbytes = ps * d.esize;
  const int wb = sweep_kb(mg) / (mg + (nrm ? 1 : 0));  // the kernel's tile width limit
  const int nw = threads / 32;
  const SweepSmem base = sweep_smem_layout(0, 0, ps, d.esize, d.tcsize, nw, m, mg);
  const int room = kSmemBudget - base.total;
  int W = std::min(wb, std::max(1, 65536 / colbytes));
  int S = 0;
  while (W >= 1) {
    S = std::min(8, room / (W * colbytes));
    if (S >= 3 || (W == 1 && S >= 2)) break;
    --W;
  }
  if (W < 1 || S < 2) return false;
  // single-column tiles (long columns): the per-tile chain of dot products,
  // block barrier and cluster exchange is the latency, so tiles overlap
  // (phase A of the next before phase B of this one; four exchange slots,
  // one stage less of prefetch)
  const int ov = (W == 1 && S >= 3) ? 1 : 0;
  const SweepSmem L = sweep_smem_layout(W, S, ps, d.esize, d.tcsize, nw, m, mg, ov ? 4 : kXSlots);
  if (L.total > at.max_dyn_smem) return false;
  *out = Pass{0, 0, mg, nch, threads, W, S, L.total, k, ov};
  return true;
}

// Pick the kernel variant, threads, tile width and stages for one pass with
// cluster size C.  Float passes take the fixed-width form (no width test per
// tile slot; measured 8-14% faster on block sweeps, even with fewer threads
// where the 8-row form would spill) for the tile width the guarded form would
// use, fewest rows per thread that fit; the others, and every other storage
// type, the first guarded variant that fits, fewest rows per thread first.
// Returns false if this C does not fit.
static bool fit_pass(int dt, int mg, int C, int ps, int m, Pass* out, bool nrm = false) {
  static const int kNch[] = {1, 2, 3, 4};
  if (dt == GPSPCA_F32)
    for (int nch : kNch) {
      Pass g;  // the guarded form's geometry gives the tile width
      if (!fit_variant(dt, mg, nch, sweep_ptr(dt, mg, nch, nrm), ps, m, nrm, &g)) continue;
      const void* kf = nrm ? sweep_kernel_f32_nrm_full(mg, nch, g.W) : sweep_kernel_f32_full(mg, nch, g.W);
      Pass q;
      if (fit_variant(dt, mg, nch, kf, ps, m, nrm, &q) && q.W == g.W) {
        *out = q;
        return true;
      }
    }
  for (int nch : kNch)
    if (fit_variant(dt, mg, nch, sweep_ptr(dt, mg, nch, nrm), ps, m, nrm, out)) return true;
  return false;
}

// Tensor-core sweep geometry: T pass over 128-column tiles, Y pass over
// 128-row blocks with the columns split so that the grid fills whole waves.
static void plan_tc(Plan* pl, int m, int64_t p, int64_t n, int nsm) {
  pl->tc = 1;
  pl->mpad = (m + 15) / 16 * 16;
  pl->npad = 3 * pl->mpad;
  pl->p_pad = static_cast<int>((p + 7) / 8 * 8);
  pl->n_pad = static_cast<int>((n + 7) / 8 * 8);
  pl->ntile1 = static_cast<int>((n + kTcTile1 - 1) / kTcTile1);
  pl->kchunks1 = static_cast<int>((p + kTcBK - 1) / kTcBK);
  pl->nchunks2 = static_cast<int>((n + kTcBK - 1) / kTcBK);
  pl->nrow2 = static_cast<int>((p + kTcRows2 - 1) / kTcRows2);
  int best = 1;
  double best_eff = 0.0;
  for (int sp = 1; sp <= 16 && sp <= pl->nchunks2; ++sp) {
    const int ctas = pl->nrow2 * sp;
    const int waves = (ctas + nsm - 1) / nsm;
    const double eff = static_cast<double>(ctas) / (static_cast<double>(waves) * nsm);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
  }
  pl->kps2 = (pl->nchunks2 + best - 1) / best;
  pl->nsplit2 = (pl->nchunks2 + pl->kps2 - 1) / pl->kps2;
}

// Row ranges per column tile of the T pass.  With ntile1 tiles on one
// persistent CTA per SM the last wave runs only ntile1 mod nsm of them (157
// tiles on 152 SMs: two waves for 1.03 of work); splitting each tile's rows
// into s ranges evens the waves at the cost of the partial sums (s * mpad
// floats per column, written by the T pass and read back by the combine
// step).  Cost in units of one 64-row chunk streamed by every CTA: the
// largest CTA's chunks plus one per item (its pipeline fill and epilogue),
// the partials' traffic at twice that streaming rate (the combine step
// streams at the HBM rate), and two for the combine launch.  Geometries with
// two CTAs per SM already absorb the tail and stay unsplit.  Fitted on GB300
// over p x n in {5000 x 20000, 10000 x 50000, 20000 x 100000, 2000 x 60000,
// 8000 x 8000}, m in {16, 32, 64}, float and bf16 storage.
static void plan_tc_ksplit(Plan* pl, int nsm) {
  pl->ksplit1 = 1;
  pl->kcs1 = pl->kchunks1;
  if (tc_t_ctas_per_sm(pl->npad, pl->tc_na, pl->tc_fused != 0) > 1) return;
  const double chunk_bytes = static_cast<double>(kTcBK) * kTcTile1 * (pl->tc_fused ? 4 : 2 * pl->tc_na) * nsm;
  const double part_bytes = 2.0 * 4.0 * pl->mpad * pl->n_pad;
  int best = 1;
  double best_cost = 0.0;
  for (int sp = 1; sp <= kTcMaxSplit1; ++sp) {
    const int kcs = (pl->kchunks1 + sp - 1) / sp;
    if (sp > 1 && kcs < 4) break;
    const int items = pl->ntile1 * sp;
    const double cost = static_cast<double>((items + nsm - 1) / nsm) * (kcs + 1) +
                        (sp > 1 ? 0.5 * sp * part_bytes / chunk_bytes + 2.0 : 0.0);
    if (sp == 1 || cost < best_cost * 0.99) {
      best_cost = cost;
      best = sp;
    }
  }
  pl->kcs1 = (pl->kchunks1 + best - 1) / best;
  pl->ksplit1 = (pl->kchunks1 + pl->kcs1 - 1) / pl->kcs1;
}

// The CUDA-core passes of `m` components in groups of at most gmax, each
// pass in clusters of C CTAs; false if some pass does not fit.
// Passes of several components in clusters overlap their tiles too: the
// cluster exchange of a tile's dot products then hides behind the next
// tile's (block m = 5: 0.121 against 0.126 ms at 5000 x 20000 in clusters
// of two, 0.080 against 0.082 ms at 8000 x 8000, chosen by the autotuner).
static void overlap_in_clusters(int dt, int C, int ps, int m, Pass* q) {
  if (C < 2 || q->mg < 2 || q->S < 3 || q->ov) return;
  const DInfo d = dinfo(dt);
  const SweepSmem L = sweep_smem_layout(q->W, q->S, ps, d.esize, d.tcsize, q->threads / 32, m, q->mg, 4);
  if (L.total > kattr(q->k).max_dyn_smem) return;
  q->ov = 1;
  q->smem = L.total;
}

static bool cuda_layout(int dt, int m, int64_t p, int unit, int gmax, int C, int* ps_out, std::vector<Pass>* out) {
  const int ps = static_cast<int>(((p + C - 1) / C + unit - 1) / unit * unit);
  if (C > 1 && static_cast<int64_t>(C - 1) * ps >= p) return false;
  std::vector<Pass> passes;
  int j0 = 0;
  for (auto g : split_components(m, gmax)) {
    Pass q;
    if (!fit_pass(dt, g.first, C, ps, m, &q)) return false;
    overlap_in_clusters(dt, C, ps, m, &q);
    q.j0 = j0;
    q.mgv = g.second;
    j0 += g.second;
    passes.push_back(q);
  }
  *ps_out = ps;
  *out = passes;
  return true;
}

static bool same_passes(const std::vector<Pass>& a, const std::vector<Pass>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].mg != b[i].mg || a[i].mgv != b[i].mgv || a[i].k != b[i].k || a[i].threads != b[i].threads ||
        a[i].W != b[i].W || a[i].S != b[i].S || a[i].ov != b[i].ov)
      return false;
  return true;
}

int make_plan(int dt, int form, int m, int64_t p, int64_t n, int64_t ld, bool fast, int nsm, Plan* P,
              bool allow_tc, int cand, int* ncand) {
  const DInfo d = dinfo(dt);
  Plan pl;
  pl.dtype = dt;
  pl.form = form;
  pl.m = m;
  pl.p = static_cast<int>(p);
  pl.n = static_cast<int>(n);
  pl.ld = ld;
  pl.fast = fast ? 1 : 0;
  pl.tcsize = d.tcsize;
  pl.esize = d.esize;
  const int unit = std::max(d.align, d.vec);
  // Candidate layouts, the planner's default first: the tensor-core sweep
  // where the CUDA-core passes become compute-bound: bf16 storage from 6
  // components (or gamma values) on, read in place when its layout suits TMA
  // (16-byte aligned base and column stride) and copied once per solve into
  // a padded layout otherwise; float A that TMA can read (split into three
  // bf16 planes in shared memory) also from 6; other float layouts and fp8
  // (copied once per solve) from 9 (one CUDA-core pass covers up to 8).
  // Crossovers measured on GB300 over p x n in {5000 x 20000, 2000 x 60000,
  // 8000 x 8000}: at 6-8 float components the fused tensor-core sweep takes
  // 0.15 / 0.15 / 0.10 ms against 0.30 / 0.19 / 0.13 ms for one CUDA-core
  // pass; at 5 the CUDA-core pass is as fast or faster.  Float read in place
  // with columns of kTcLongRows rows or more takes the tensor-core sweep for
  // any m: a CUDA-core CTA holds at most 5000-8000 float rows in registers,
  // so such columns are split over clusters whose per-tile exchange (and
  // idle SMs) cost more than the tensor-core sweep's two passes (single-unit
  // sweeps at 10000 x 40000 / 12000 x 30000 / 20000 x 25000: 0.327 / 0.288 /
  // 0.392 ms against 0.363 / 0.318 / 0.441 ms; a tie at 16000 x 30000; block
  // m = 5 at 20000 x 25000: 0.71 ms on the CUDA cores).  Below 16384 rows
  // whole single-unit solves did not gain (64 solves at 10000 x 50000: 155
  // against 135 ms: the tensor-core sweep's extra launches and tensor maps
  // per solve).  Otherwise
  // the widest CUDA-core passes first (fewest reads of A) in the smallest
  // clusters that fit; long columns (large p) may only fit narrower passes,
  // whose per-thread register tiles are smaller.  The other candidates (the
  // autotuner times them all): the tensor-core sweep for any m, and
  // every pass grouping of at most 8, 5, 4, 2 or 1 components in clusters of
  // 1, 2, 4 or 8 that fits.
  struct Layout {
    bool tc;
    int C, ps;
    std::vector<Pass> passes;
  };
  std::vector<Layout> lay;
  const bool tc_type = dt == GPSPCA_BF16 || dt == GPSPCA_F32 || dt == GPSPCA_FP8_E4M3;
  const bool f32_in_place = dt == GPSPCA_F32 && fast && ld % 4 == 0;
  const int tc_min_m = (dt == GPSPCA_BF16 || f32_in_place) ? 6 : 9;
  const bool long_cols = f32_in_place && p >= kTcLongRows;
  const bool tc_default = allow_tc && tc_type && (m >= tc_min_m || long_cols) && p >= 1 && n >= 1;
  if (tc_default) lay.push_back({true, 1, static_cast<int>(p), {}});
  for (int gmax : {8, 4, 2, 1}) {
    if (!lay.empty()) break;
    for (int C : {1, 2, 4, 8}) {
      Layout L{false, C, 0, {}};
      if (cuda_layout(dt, m, p, unit, gmax, C, &L.ps, &L.passes)) {
        lay.push_back(L);
        break;
      }
    }
  }
  if (lay.empty())
    return fail(GPSPCA_EINVAL, "no sweep configuration fits p=%lld (rows too long for the on-chip tile ring)",
                (long long)p);
  if (cand > 0 || ncand) {  // the alternatives, only when asked for (they cost a fit per variant)
    if (!tc_default && allow_tc && tc_type && p >= 1 && n >= 1) lay.push_back({true, 1, static_cast<int>(p), {}});
    for (int gmax : {8, 5, 4, 2, 1})
      for (int C : {1, 2, 4, 8}) {
        Layout L{false, C, 0, {}};
        if (!cuda_layout(dt, m, p, unit, gmax, C, &L.ps, &L.passes)) continue;
        bool dup = false;
        for (const Layout& o : lay) dup = dup || (!o.tc && o.C == L.C && same_passes(o.passes, L.passes));
        if (!dup) lay.push_back(L);
      }
    // each CUDA-core layout also with its tiles overlapped the other way
    // (phase A of the next tile before phase B of this one, or not)
    const size_t base = lay.size();
    for (size_t li = 0; li < base; ++li) {
      if (lay[li].tc) continue;
      Layout L = lay[li];
      bool ok = true;
      for (Pass& q : L.passes) {
        if (q.S < 3) {
          ok = false;
          break;
        }
        q.ov = q.ov ? 0 : 1;
        const DInfo d = dinfo(dt);
        const SweepSmem S2 = sweep_smem_layout(q.W, q.S, L.ps, d.esize, d.tcsize, q.threads / 32, m, q.mg,
                                               q.ov ? 4 : kXSlots);
        if (S2.total > kattr(q.k).max_dyn_smem) {
          ok = false;
          break;
        }
        q.smem = S2.total;
      }
      if (ok) lay.push_back(L);
    }
  }
  if (ncand) *ncand = static_cast<int>(lay.size());
  const int pick = cand < 0 ? 0 : cand;
  if (pick >= static_cast<int>(lay.size()))
    return fail(GPSPCA_EINVAL, "plan candidate %d of %d", pick, static_cast<int>(lay.size()));
  const Layout& L = lay[pick];
  if (L.tc) {
    plan_tc(&pl, m, p, n, nsm);
    pl.tc_na = dt == GPSPCA_F32 ? 3 : 1;
    // float A that TMA can read (16-byte aligned base and column stride) is
    // split into its planes in shared memory; other float / fp8 / bf16
    // layouts are copied once per solve
    const bool native_bf16 = dt == GPSPCA_BF16 && fast && ld % 8 == 0;
    pl.tc_fused = f32_in_place ? 1 : 0;
    pl.tc_convert = (native_bf16 || pl.tc_fused) ? 0 : 1;
    pl.tc_sparse = 1;  // threshold sweeps' rank update over the listed active columns
    plan_tc_ksplit(&pl, nsm);
    pl.C = 1;
    pl.ps = static_cast<int>(p);
  } else {
    pl.C = L.C;
    pl.ps = L.ps;
    pl.passes = L.passes;
  }
  // clusters: as many as can be co-resident for the heaviest pass (the
  // tensor-core sweep's Y-pass splits play their part)
  int ncl = pl.tc ? pl.nsplit2 : nsm / pl.C;
  for (const Pass& q : pl.passes) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pl.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(pl.C * std::max(1, nsm / pl.C));
    cfg.blockDim = dim3(q.threads);
    cfg.dynamicSmemBytes = q.smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, q.k, &cfg) == cudaSuccess && nc > 0) ncl = std::min(ncl, nc);
  }
  if (!pl.tc) ncl = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ncl, n)));
  // block forms: the start's first power step reads A and can form the
  // column norms too (no pass of their own): the fused float tensor-core
  // sweep sums them in its T pass
  if (pl.tc && pl.tc_fused && form >= 2) pl.norms_in_sweep = 1;
  // on the CUDA cores, the first pass runs a variant that forms them
  if (!pl.tc && form >= 2 && !pl.passes.empty()) {
    Pass q;
    if (fit_pass(dt, pl.passes[0].mg, pl.C, pl.ps, m, &q, true)) {
      overlap_in_clusters(dt, pl.C, pl.ps, m, &q);
      q.j0 = pl.passes[0].j0;
      q.mgv = pl.passes[0].mgv;
      pl.norm_pass = q;
      pl.norms_in_sweep = 1;
    }
  }
  pl.ncl = ncl;
  pl.cols_per_cl = static_cast<int>((n + ncl - 1) / ncl);
  pl.nred = static_cast<int>((p + kReduceRows - 1) / kReduceRows);
  pl.nobj = static_cast<int>(std::min<int64_t>(std::max<int64_t>(1, (n + 1023) / 1024), 2 * nsm));
  pl.full_gram = form >= 2 ? 1 : 0;
  pl.npairs = pl.full_gram ? m * m : m;  // gpart capacity: the Ritz step's cross Gram is m x m
  pl.finish_smem = static_cast<int>(sizeof(double)) * finish_smem_doubles(m, pl.npairs);
  if (pl.finish_smem > kFinishMaxSmem)
    return fail(GPSPCA_EINVAL, "m = %d needs %d bytes of shared memory in the projection step (at most %d)", m,
                pl.finish_smem, kFinishMaxSmem);
  pl.ws_cnorm = sizeof(double) * n;
  pl.ws_P = static_cast<size_t>(d.tcsize) * m * p;
  if (!pl.tc && form >= 2) pl.ws_Xf = static_cast<size_t>(d.tcsize) * m * p;
  pl.ws_ypart = static_cast<size_t>(d.tcsize) * ncl * m * p;
  pl.ws_T = static_cast<size_t>(d.tcsize) * m * n;
  pl.ws_fpart = sizeof(dd) * static_cast<size_t>(pl.nobj) * 2 * m;
  // Gram partials: per reduction block, or per T^T T block of the tensor-core start
  pl.ws_gpart = sizeof(double) * static_cast<size_t>(std::max(pl.nred, pl.tc ? gram_t_blocks(n) : 0)) * pl.npairs;
  if (pl.tc) {
    pl.ws_x3 = 2 * static_cast<size_t>(pl.npad) * pl.p_pad;
    pl.ws_g3 = 2 * static_cast<size_t>(pl.npad) * pl.n_pad;
    if (pl.tc_convert) pl.ws_planes = 2 * static_cast<size_t>(pl.tc_na) * n * pl.p_pad;
    if (pl.ksplit1 > 1)
      pl.ws_tpart = sizeof(float) * static_cast<size_t>(pl.ksplit1) * pl.mpad * pl.n_pad;
    if (pl.tc_sparse) pl.ws_sparse = sparse_layout(n, pl.npad).total;
  }
  *P = pl;
  return GPSPCA_OK;
}

// ---------------------------------------------------------------- workspace

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Slot;

struct Budget {
  std::mutex mu;
  size_t limit = 0, used = 0;
};

// Autotuned sweep layouts of a context: problem shape (tune_shape) -> the
// key (Plan::key) of the candidate layout that timed fastest, and its time;
// and, once a solve has found that candidate among the planner's, its plan
// (so later solves of the shape skip the search).
struct TuneTable {
  std::mutex mu;
  std::unordered_map<std::string, std::pair<std::string, double>> best;
  std::unordered_map<std::string, Plan> resolved;
};

static std::string tune_shape(int dt, int form, int m, int64_t p, int64_t n, int64_t ld, bool fast, bool allow_tc,
                              int nsm) {
  char b[160];
  snprintf(b, sizeof(b), "d%d/%s/m%d/p%lld/n%lld/ld%lld/f%d/tc%d/sm%d", dt, form >= 2 ? "block" : "single", m,
           (long long)p, (long long)n, (long long)ld, fast ? 1 : 0, allow_tc ? 1 : 0, nsm);
  return b;
}

struct Slot {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  IO* io_dev = nullptr;
  State* st_dev = nullptr;
  IO* io_host = nullptr;     // pinned
  State* st_host = nullptr;  // pinned
  cudaEvent_t done = nullptr;
  Budget* budget = nullptr;
  TuneTable* tune = nullptr;  // the context's autotuned layouts
  // workspace buffers, grown on demand
  DevBuf b_cnorm, b_P, b_Y, b_Xf, b_ypart, b_T, b_fpart, b_gpart, b_x3, b_g3, b_maps, b_planes, b_tpart, b_sparse;
  TcMaps* maps_host = nullptr;  // pinned: the tensor maps copied to b_maps before a solve
  // staging for host-located inputs/outputs
  DevBuf s_A, s_scale, s_x0, s_X, s_Z, s_sup, s_obj, s_it, s_stat, s_gam;
  DevBuf d_W, d_list;  // deflation: the working copy of A, the support list of z_j
  struct GraphEntry {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  std::unordered_map<std::string, GraphEntry> graphs;

  size_t held() const {
    size_t s = 0;
    for (const DevBuf* b : {&b_cnorm, &b_P, &b_Y, &b_Xf, &b_ypart, &b_T, &b_fpart, &b_gpart, &b_x3, &b_g3, &b_maps,
                            &b_planes, &b_tpart, &b_sparse, &s_A,
                            &s_scale, &s_x0, &s_X,
                            &s_Z, &s_sup, &s_obj, &s_it, &s_stat, &s_gam, &d_W, &d_list})
      s += b->bytes;
    return s;
  }
};

static int ensure(Slot* s, DevBuf* b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  if (b->bytes >= bytes) return GPSPCA_OK;
  {
    std::lock_guard<std::mutex> lk(s->budget->mu);
    if (s->budget->used - b->bytes + bytes > s->budget->limit)
      return fail(GPSPCA_ENOMEM, "workspace of %zu bytes exceeds the context budget (%zu of %zu in use)", bytes,
                  s->budget->used, s->budget->limit);
    s->budget->used = s->budget->used - b->bytes + bytes;
  }
  // stream-ordered: the old buffer is released after the work queued on
  // this slot's stream, and no device-wide synchronisation happens
  if (b->p) cudaFreeAsync(b->p, s->stream);
  b->p = nullptr;
  b->bytes = 0;
  if (cudaMallocAsync(&b->p, bytes, s->stream) != cudaSuccess) {
    cudaGetLastError();
    b->p = nullptr;
    std::lock_guard<std::mutex> lk(s->budget->mu);
    s->budget->used -= bytes;
    return fail(GPSPCA_ENOMEM, "device allocation of %zu bytes failed", bytes);
  }
  b->bytes = bytes;
  return GPSPCA_OK;
}

static void release(Slot* s, DevBuf* b) {
  if (b->p) cudaFreeAsync(b->p, s->stream);
  std::lock_guard<std::mutex> lk(s->budget->mu);
  s->budget->used -= b->bytes;
  b->p = nullptr;
  b->bytes = 0;
}

static void release_workspace(Slot* s) {
  for (DevBuf* b : {&s->b_cnorm, &s->b_P, &s->b_Y, &s->b_Xf, &s->b_ypart, &s->b_T, &s->b_fpart, &s->b_gpart, &s->b_x3,
                    &s->b_g3, &s->b_maps, &s->b_planes, &s->b_tpart, &s->b_sparse, &s->s_A,
                    &s->s_scale, &s->s_x0, &s->s_X, &s->s_Z, &s->s_sup, &s->s_obj, &s->s_it, &s->s_stat, &s->s_gam,
                    &s->d_W, &s->d_list})
    release(s, b);
}

// graphs = false: a member of a group (its solve launched by the group's
// graph), so no capture streams.
static int slot_init(Slot* s, int device, cudaStream_t user_stream, Budget* budget, TuneTable* tune,
                     bool graphs = true) {
  s->device = device;
  s->budget = budget;
  s->tune = tune;
  if (user_stream) {
    s->stream = user_stream;
  } else {
    GP_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  if (graphs) {
    GP_CUDA(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
    GP_CUDA(cudaStreamCreateWithFlags(&s->cap2, cudaStreamNonBlocking));
  }
  GP_CUDA(cudaMalloc(&s->io_dev, sizeof(IO)));
  GP_CUDA(cudaMalloc(&s->st_dev, sizeof(State)));
  GP_CUDA(cudaMallocHost(&s->io_host, sizeof(IO)));
  GP_CUDA(cudaMallocHost(&s->st_host, sizeof(State)));
  GP_CUDA(cudaMallocHost(&s->maps_host, sizeof(TcMaps)));
  GP_CUDA(cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming));
  return GPSPCA_OK;
}

static void slot_free(Slot* s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  s->graphs.clear();
  release_workspace(s);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->io_dev) cudaFree(s->io_dev);
  if (s->st_dev) cudaFree(s->st_dev);
  if (s->io_host) cudaFreeHost(s->io_host);
  if (s->st_host) cudaFreeHost(s->st_host);
  if (s->maps_host) cudaFreeHost(s->maps_host);
  if (s->done) cudaEventDestroy(s->done);
  for (cudaStream_t c : {s->cap2, s->cap}) {  // never destroy a stream that is still capturing
    if (!c) continue;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c, &g);
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    cudaStreamDestroy(c);
  }
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  *s = Slot();
}

// ---------------------------------------------------------------- graph

static cudaError_t launch_sweeps(const Plan& pl, Slot* s, cudaStream_t cs, int sketch = 0, int norms = 0,
                                 int keep_t = 0, int from_ritz = 0);
static cudaError_t launch_body(const Plan& pl, Slot* s, cudaStream_t cs, cudaGraphConditionalHandle h,
                               int use_cond = 1, int from_ritz = 0);

// The first sweep after a block start on the tensor cores can form T from
// the T = A^T Q its Rayleigh-Ritz step kept (T = (A^T Q) R) instead of a T
// pass; unscaled storage (the kept T of fp8 storage carries the scales).
static bool first_sweep_from_ritz(const Plan& pl) { return pl.tc && pl.pca && pl.dtype != GPSPCA_FP8_E4M3; }

// Start of the solve: norms, gamma, the start directions and their
// projection.  Block forms without a caller start then take kPowerSteps
// power steps (A A^T Q, projected) and a Rayleigh-Ritz rotation; on the
// tensor cores the first sweep follows here (first_sweep), its T formed
// from the rotation step's.
static cudaError_t launch_prologue(const Plan& pl, Slot* s, cudaStream_t cs, cudaGraphConditionalHandle h, bool pca,
                                   int use_cond = 1, bool first_sweep = true) {
  if (pl.tc && pl.tc_convert)  // bf16 planes of a float / fp8 A for the tensor cores
    launch_tc_convert(pl.dtype, s->io_dev, pl.p, pl.n, pl.ld, pl.p_pad, cs);
  if (pl.tc_sparse) {  // no column is flagged active before the first threshold sweep
    const cudaError_t e0 =
        cudaMemsetAsync(static_cast<unsigned char*>(s->b_sparse.p) + sparse_layout(pl.n, pl.npad).act, 0,
                        static_cast<size_t>((pl.n + 63) / 64 * 64), cs);
    if (e0 != cudaSuccess) return e0;
  }
  if (pl.tc && pca && pl.norms_in_sweep) {  // the squared norms the first power step sums
    const cudaError_t e1 = cudaMemsetAsync(
        static_cast<unsigned char*>(s->b_sparse.p) + sparse_layout(pl.n, pl.npad).nsq, 0, sizeof(double) * pl.n, cs);
    if (e1 != cudaSuccess) return e1;
  }
  launch_reset(s->io_dev, s->st_dev, pl.m, pl.form, cs);
  // the block start's first power step forms the column norms itself; the
  // start selection (gamma scale, non-finite check) then follows that step
  const bool late_norms = pca && pl.norms_in_sweep;
  StartArgs sa{s->io_dev, s->st_dev, pl.ld, pl.p, pl.n, pl.m, pl.form};
  if (!late_norms) {
    if (pl.norms_given)  // computed once by the batch for its solves of this matrix
      launch_copy_norms(s->io_dev, s->st_dev, pl.n, cs);
    else
      launch_colnorm(pl.dtype, s->io_dev, s->st_dev, pl.ld, pl.p, pl.n, pl.fast, cs);
    launch_select_start(pl.dtype, sa, cs);
  }
  launch_gather_start(pl.dtype, sa, cs);
  const int gram_pairs = pl.full_gram ? pl.m * (pl.m + 1) / 2 : pl.m;
  ReduceArgs ra{s->io_dev, s->st_dev, 1, pl.m, pl.p, pl.full_gram, gram_pairs, 1, 0, 0, pl.n, pl.form, pl.nred, 0};
  launch_reduce(pl.tcsize, ra, cs);
  FinishArgs fa{s->io_dev, s->st_dev, pl.ncl, pl.nred, gram_pairs, pl.m, pl.form, kFinishPolar, pca ? 0 : 1, h,
                use_cond};
  launch_finish(fa, pl.finish_smem, cs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !pca) return e;
  for (int step = 0; step < kPowerSteps; ++step) {
    if ((e = launch_sweeps(pl, s, cs, 1, late_norms && step == 0)) != cudaSuccess) return e;
    ReduceArgs rp{s->io_dev, s->st_dev, pl.ncl, pl.m, pl.p, 1, gram_pairs, 0, 0, 0, pl.n, pl.form, pl.nred, 0};
    launch_reduce(pl.tcsize, rp, cs);
    FinishArgs fp{s->io_dev, s->st_dev, pl.ncl, pl.nred, gram_pairs, pl.m, pl.form, kFinishPolar, 0, h, use_cond};
    launch_finish(fp, pl.finish_smem, cs);
    if (late_norms && step == 0) launch_select_start(pl.dtype, sa, cs);
  }
  if (pl.tc) {
    // Rayleigh-Ritz from T = A^T Q alone: Q^T A A^T Q = T^T T, so this step
    // needs the T pass but no rank update (one read of A instead of two)
    if ((e = launch_sweeps(pl, s, cs, 1, 0, 1)) != cudaSuccess) return e;
    launch_gram_t(s->io_dev, s->st_dev, pl.m, pl.n, cs);
    FinishArgs fr{s->io_dev, s->st_dev, pl.ncl, gram_t_blocks(pl.n), pl.m * pl.m, pl.m, pl.form, kFinishRitzT, 1, h,
                  use_cond};
    launch_finish(fr, pl.finish_smem, cs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the first sweep, its T from the kept A^T Q and the rotation
    if (first_sweep && first_sweep_from_ritz(pl)) return launch_body(pl, s, cs, h, use_cond, 1);
    return cudaSuccess;
  }
  if ((e = launch_sweeps(pl, s, cs, 1)) != cudaSuccess) return e;
  ReduceArgs rc{s->io_dev, s->st_dev, pl.ncl, pl.m, pl.p, 1, pl.m * pl.m, 0, 1, 0, pl.n, pl.form, pl.nred, 0};
  launch_reduce(pl.tcsize, rc, cs);
  FinishArgs fr{s->io_dev, s->st_dev, pl.ncl, pl.nred, pl.m * pl.m, pl.m, pl.form, kFinishRitz, 1, h, use_cond};
  launch_finish(fr, pl.finish_smem, cs);
  return cudaGetLastError();
}

// keep_t (tensor-core sweep, start only): X3 and the T pass alone, T = A^T Q
// written to io->T for the Rayleigh-Ritz step's T^T T.  from_ritz
// (tensor-core sweep, the first sweep after the start): T from that kept T.
static cudaError_t launch_sweeps(const Plan& pl, Slot* s, cudaStream_t cs, int sketch, int norms, int keep_t,
                                 int from_ritz) {
  if (pl.tc) {
    TcArgs a{s->io_dev,  s->st_dev, pl.p,     pl.n,       pl.m,        pl.mpad,     pl.form,
             sketch,     pl.tc_na,  pl.tc_fused, pl.dtype == GPSPCA_FP8_E4M3 ? 1 : 0, pl.p_pad, pl.n_pad,
             pl.ntile1,  pl.kchunks1, pl.ksplit1, pl.kcs1, pl.nchunks2, pl.kps2, pl.nsplit2, pl.nrow2,
             pl.tc_sparse, norms, keep_t, pl.tc_convert ? static_cast<int64_t>(pl.p_pad) : pl.ld, from_ritz};
    launch_tc_sweep(a, pl.npad, cs, keep_t != 0);
    return cudaGetLastError();
  }
  if (pl.form >= 2) launch_form_x(pl.tcsize, s->io_dev, s->st_dev, pl.p, pl.m, cs);  // X = Y W for the passes
  for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
    const Pass& q = (norms && pi == 0) ? pl.norm_pass : pl.passes[pi];
    SweepArgs a{s->io_dev, s->st_dev, pl.ld, pl.p, pl.n, pl.m, pl.form, q.j0, q.mgv, pl.ps, q.W, q.S,
                pl.cols_per_cl, pl.fast, sketch, q.ov};
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pl.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(pl.ncl * pl.C);
    cfg.blockDim = dim3(q.threads);
    cfg.dynamicSmemBytes = q.smem;
    cfg.stream = cs;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, q.k, args);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_body(const Plan& pl, Slot* s, cudaStream_t cs, cudaGraphConditionalHandle h,
                               int use_cond, int from_ritz) {
  cudaError_t e = launch_sweeps(pl, s, cs, 0, 0, 0, from_ritz);
  if (e != cudaSuccess) return e;
  const int gram_pairs = pl.full_gram ? pl.m * (pl.m + 1) / 2 : pl.m;
  ReduceArgs ra{s->io_dev, s->st_dev, pl.ncl, pl.m, pl.p, pl.full_gram, gram_pairs, 0, 0, 1, pl.n, pl.form, pl.nred,
                pl.nobj};
  launch_reduce(pl.tcsize, ra, cs);
  FinishArgs fa{s->io_dev, s->st_dev, pl.nobj, pl.nred, gram_pairs, pl.m, pl.form, kFinishIterate, 0, h, use_cond};
  launch_finish(fa, pl.finish_smem, cs);
  return cudaGetLastError();
}

static cudaError_t launch_epilogue(const Plan& pl, Slot* s, cudaStream_t cs) {
  launch_finalize(pl.tcsize, s->io_dev, s->st_dev, pl.p, pl.n, pl.m, pl.form, cs);
  return cudaGetLastError();
}

// A graph of the start (pro), a conditional WHILE node over the loop body
// (body; the condition set by its kernels) and the end (epi), captured on
// the streams cap (outer) and cap2 (body).
template <typename Pro, typename Body, typename Epi>
static int capture_loop_graph(cudaStream_t cap, cudaStream_t cap2, Pro pro, Body body, Epi epi,
                              Slot::GraphEntry* out) {
  cudaGraph_t g = nullptr;
  GP_CUDA(cudaGraphCreate(&g, 0));
  bool outer = false, inner = false;
  cudaGraph_t tmp = nullptr;
  // on any failure: end the open captures (so the streams leave capture
  // mode), drop the partial graph and report the first error
  auto abort_with = [&](cudaError_t e, const char* what) {
    if (inner) cudaStreamEndCapture(cap2, &tmp);
    if (outer) cudaStreamEndCapture(cap, &tmp);
    cudaGetLastError();
    cudaGraphDestroy(g);
    return fail(GPSPCA_ECUDA, "graph build (%s): %s", what, cudaGetErrorString(e));
  };
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return abort_with(e, "conditional handle");
  if ((e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
    return abort_with(e, "begin capture");
  outer = true;
  if ((e = pro(cap, h))) return abort_with(e, "start kernels");
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if ((e = cudaStreamGetCaptureInfo(cap, &cst, nullptr, nullptr, &deps, nullptr, &ndeps)))
    return abort_with(e, "capture info");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if ((e = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp))) return abort_with(e, "while node");
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies)))
    return abort_with(e, "capture dependencies");
  if ((e = cudaStreamBeginCaptureToGraph(cap2, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
    return abort_with(e, "begin body capture");
  inner = true;
  if ((e = body(cap2, h))) return abort_with(e, "loop body kernels");
  inner = false;
  if ((e = cudaStreamEndCapture(cap2, &tmp))) return abort_with(e, "end body capture");
  if ((e = epi(cap))) return abort_with(e, "loadings kernel");
  outer = false;
  if ((e = cudaStreamEndCapture(cap, &tmp))) return abort_with(e, "end capture");
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaGraphInstantiate(&exec, g, 0))) return abort_with(e, "instantiate");
  out->g = g;
  out->exec = exec;
  return GPSPCA_OK;
}

static int build_graph(const Plan& pl, Slot* s, Slot::GraphEntry* out) {
  return capture_loop_graph(
      s->cap, s->cap2,
      [&](cudaStream_t cs, cudaGraphConditionalHandle h) { return launch_prologue(pl, s, cs, h, pl.pca != 0); },
      [&](cudaStream_t cs, cudaGraphConditionalHandle h) { return launch_body(pl, s, cs, h); },
      [&](cudaStream_t cs) { return launch_epilogue(pl, s, cs); }, out);
}

static int get_graph(const Plan& pl, Slot* s, cudaGraphExec_t* exec) {
  const std::string key = pl.key();
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    *exec = it->second.exec;
    return GPSPCA_OK;
  }
  Slot::GraphEntry e;
  const int rc = build_graph(pl, s, &e);
  if (rc != GPSPCA_OK) return rc;
  if (s->graphs.size() >= 64) {  // bound the cache
    for (auto& kv : s->graphs) {
      cudaGraphExecDestroy(kv.second.exec);
      cudaGraphDestroy(kv.second.g);
    }
    s->graphs.clear();
  }
  s->graphs[key] = e;
  *exec = e.exec;
  return GPSPCA_OK;
}

// ---------------------------------------------------------------- one solve

struct Request {
  gpspca_matrix A;
  gpspca_form form;
  std::vector<double> gamma, mu;
  int m = 0;
  double tol = 0;
  int maxit = 0;
  const void* x0 = nullptr;
  uint32_t flags = 0;
  gpspca_out out;
  // single-unit solves of a batch on one device matrix: the column norms the
  // batch computed once for them (device, n doubles), or null
  const double* cnorm_src = nullptr;
};

static int validate(const Request& r) {
  const gpspca_matrix& A = r.A;
  if (A.dtype < GPSPCA_F32 || A.dtype > GPSPCA_F64) return fail(GPSPCA_EINVAL, "unknown dtype %d", (int)A.dtype);
  if (A.location != GPSPCA_DEVICE && A.location != GPSPCA_HOST) return fail(GPSPCA_EINVAL, "bad A location");
  if (A.p < 0 || A.n < 0) return fail(GPSPCA_EINVAL, "negative shape");
  if (A.p > (1 << 30) || A.n > (1 << 30)) return fail(GPSPCA_EINVAL, "p and n must be below 2^30");
  if (A.p > 0 && A.n > 0) {
    if (!A.data) return fail(GPSPCA_EINVAL, "A.data is NULL");
    if (A.ld < A.p) return fail(GPSPCA_EINVAL, "ld (%lld) < p (%lld)", (long long)A.ld, (long long)A.p);
    if (A.dtype == GPSPCA_FP8_E4M3 && !A.col_scale) return fail(GPSPCA_EINVAL, "FP8 storage needs col_scale");
  }
  if (r.form < GPSPCA_SL1 || r.form > GPSPCA_BL0) return fail(GPSPCA_EINVAL, "unknown formulation %d", (int)r.form);
  if (r.m < 1 || r.m > kMaxM) return fail(GPSPCA_EINVAL, "m = %d outside [1, %d]", r.m, kMaxM);
  const bool block = r.form >= GPSPCA_BL1;
  for (int j = 0; j < r.m; ++j) {
    if (!(r.gamma[j] >= 0.0) || !std::isfinite(r.gamma[j])) return fail(GPSPCA_EINVAL, "gamma[%d] must be finite and >= 0", j);
    if (!(r.mu[j] > 0.0) || !std::isfinite(r.mu[j])) return fail(GPSPCA_EINVAL, "mu[%d] must be finite and > 0", j);
    if (!block && r.mu[j] != 1.0) return fail(GPSPCA_EINVAL, "single-unit formulations take no weights (mu = 1)");
  }
  if (block && A.p > 0 && r.m > A.p) return fail(GPSPCA_EINVAL, "block formulations need m <= p");
  if (block && !r.x0 && A.n > 0 && r.m > A.n) return fail(GPSPCA_EINVAL, "block start needs m <= n columns");
  if (!(r.tol >= 0.0) || !std::isfinite(r.tol)) return fail(GPSPCA_EINVAL, "tol must be finite and >= 0");
  if (r.maxit < 1) return fail(GPSPCA_EINVAL, "maxit must be >= 1");
  const gpspca_out& o = r.out;
  if (o.location != GPSPCA_DEVICE && o.location != GPSPCA_HOST) return fail(GPSPCA_EINVAL, "bad out location");
  if (!o.X || !o.Z || !o.objective || !o.iters || !o.status) return fail(GPSPCA_EINVAL, "an output pointer is NULL");
  return GPSPCA_OK;
}

// Empty A (p == 0 or n == 0): status ZERO, nothing to compute.
static int solve_empty(Slot* s, const Request& r) {
  std::vector<double> obj(r.m, 0.0);
  std::vector<int32_t> it(r.m, 0), stv(r.m, GPSPCA_ZERO);
  const cudaMemcpyKind k = r.out.location == GPSPCA_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  GP_CUDA(cudaMemcpyAsync(r.out.objective, obj.data(), sizeof(double) * r.m, k, s->stream));
  GP_CUDA(cudaMemcpyAsync(r.out.iters, it.data(), sizeof(int32_t) * r.m, k, s->stream));
  GP_CUDA(cudaMemcpyAsync(r.out.status, stv.data(), sizeof(int32_t) * r.m, k, s->stream));
  if (r.out.gamma_abs) GP_CUDA(cudaMemcpyAsync(r.out.gamma_abs, r.gamma.data(), sizeof(double) * r.m, k, s->stream));
  GP_CUDA(cudaStreamSynchronize(s->stream));
  return GPSPCA_OK;
}

// Validate, plan, size the workspace and write the IO record for one solve
// (asynchronous, on the slot's stream).  scratch_out: results go to library
// staging buffers and are not copied anywhere (used by the sweep timer).
// cand >= 0: candidate layout `cand` of the autotuner's list (*ncand its
// length); cand < 0: the tuned layout of this shape if the context has one,
// else the planner's default.  *shape (if given): the shape's tuning key.
// fixed: a plan made for the same shape and storage (a group's members
// share their first member's), used as it is.
static int prepare_solve(Slot* s, const Request& r, int nsm, bool scratch_out, Plan* plan, bool* empty,
                         int cand = -1, int* ncand = nullptr, std::string* shape = nullptr,
                         const Plan* fixed = nullptr) {
  *empty = false;
  int rc = validate(r);
  if (rc != GPSPCA_OK) return rc;
  if (r.A.p == 0 || r.A.n == 0) {
    *empty = true;
    return scratch_out ? GPSPCA_OK : solve_empty(s, r);
  }
  const DInfo d = dinfo(r.A.dtype);
  const bool host_in = r.A.location == GPSPCA_HOST;
  const bool staged_out = scratch_out || r.out.location == GPSPCA_HOST;
  const int64_t p = r.A.p, n = r.A.n, ld = r.A.ld;
  const int m = r.m;
  const size_t a_bytes = static_cast<size_t>(ld) * n * d.esize;
  const void* A_dev = r.A.data;
  const float* scale_dev = r.A.col_scale;
  const void* x0_dev = r.x0;
  if (host_in) {
    if ((rc = ensure(s, &s->s_A, a_bytes))) return rc;
    GP_CUDA(cudaMemcpyAsync(s->s_A.p, r.A.data, a_bytes, cudaMemcpyHostToDevice, s->stream));
    A_dev = s->s_A.p;
    if (r.A.dtype == GPSPCA_FP8_E4M3) {
      if ((rc = ensure(s, &s->s_scale, sizeof(float) * n))) return rc;
      GP_CUDA(cudaMemcpyAsync(s->s_scale.p, r.A.col_scale, sizeof(float) * n, cudaMemcpyHostToDevice, s->stream));
      scale_dev = static_cast<const float*>(s->s_scale.p);
    }
    if (r.x0) {
      if ((rc = ensure(s, &s->s_x0, static_cast<size_t>(d.tcsize) * p * m))) return rc;
      GP_CUDA(cudaMemcpyAsync(s->s_x0.p, r.x0, static_cast<size_t>(d.tcsize) * p * m, cudaMemcpyHostToDevice,
                              s->stream));
      x0_dev = s->s_x0.p;
    }
  }
  const bool fast = (reinterpret_cast<uintptr_t>(A_dev) % 16 == 0) && ((ld * d.esize) % 16 == 0);
  Plan& pl = *plan;
  const bool allow_tc = !(r.flags & GPSPCA_NO_TENSOR_CORES) && tc_supported(s->device);
  const int pca = (r.form >= GPSPCA_BL1 && !r.x0) ? 1 : 0;
  const std::string shape_key = tune_shape(r.A.dtype, r.form, m, p, n, ld, fast, allow_tc, nsm);
  if (shape) *shape = shape_key;
  std::string tuned;
  bool picked = false;
  if (fixed) {
    pl = *fixed;
    picked = true;
  }
  if (!picked && cand < 0 && s->tune) {
    std::lock_guard<std::mutex> lk(s->tune->mu);
    auto it = s->tune->best.find(shape_key);
    if (it != s->tune->best.end()) {
      tuned = it->second.first;
      auto rv = s->tune->resolved.find(shape_key);
      if (rv != s->tune->resolved.end() && rv->second.pca == pca && rv->second.key() == tuned) {
        pl = rv->second;
        picked = true;
      }
    }
  }
  if (!picked && !tuned.empty()) {  // the candidate whose plan key was stored (the default if none matches)
    int nc = 0;
    if (make_plan(r.A.dtype, r.form, m, p, n, ld, fast, nsm, &pl, allow_tc, 0, &nc) == GPSPCA_OK)
      for (int c = 0; c < nc && !picked; ++c) {
        Plan q;
        if (make_plan(r.A.dtype, r.form, m, p, n, ld, fast, nsm, &q, allow_tc, c) != GPSPCA_OK) continue;
        q.pca = pca;
        if (q.key() == tuned) {
          pl = q;
          picked = true;
        }
      }
    if (picked) {
      std::lock_guard<std::mutex> lk(s->tune->mu);
      s->tune->resolved[shape_key] = pl;
    }
  }
  if (!picked && (rc = make_plan(r.A.dtype, r.form, m, p, n, ld, fast, nsm, &pl, allow_tc, cand, ncand))) return rc;
  pl.pca = pca;
  pl.norms_given = (r.cnorm_src && r.form < GPSPCA_BL1 && !pl.norms_in_sweep) ? 1 : 0;
  if ((rc = ensure(s, &s->b_cnorm, pl.ws_cnorm))) return rc;
  if ((rc = ensure(s, &s->b_P, pl.ws_P))) return rc;
  if ((rc = ensure(s, &s->b_Y, pl.ws_P))) return rc;
  if (pl.ws_Xf && (rc = ensure(s, &s->b_Xf, pl.ws_Xf))) return rc;
  if ((rc = ensure(s, &s->b_ypart, pl.ws_ypart))) return rc;
  if ((rc = ensure(s, &s->b_T, pl.ws_T))) return rc;
  if ((rc = ensure(s, &s->b_fpart, pl.ws_fpart))) return rc;
  if ((rc = ensure(s, &s->b_gpart, pl.ws_gpart))) return rc;
  if (pl.tc) {
    if ((rc = ensure(s, &s->b_x3, pl.ws_x3))) return rc;
    if ((rc = ensure(s, &s->b_g3, pl.ws_g3))) return rc;
    if ((rc = ensure(s, &s->b_maps, sizeof(TcMaps)))) return rc;
    if (pl.tc_convert && (rc = ensure(s, &s->b_planes, pl.ws_planes))) return rc;
    if (pl.ksplit1 > 1 && (rc = ensure(s, &s->b_tpart, pl.ws_tpart))) return rc;
    if (pl.tc_sparse && (rc = ensure(s, &s->b_sparse, pl.ws_sparse))) return rc;
    // the host copy of the maps is reused only after this solve's copy has run
    GP_CUDA(cudaStreamSynchronize(s->stream));
    if (pl.tc_fused) {
      const void* g3c =
          pl.tc_sparse ? static_cast<unsigned char*>(s->b_sparse.p) + sparse_layout(n, pl.npad).g3c : nullptr;
      if ((rc = tc_encode_maps_f32(s->maps_host, A_dev, p, n, ld, s->b_x3.p, pl.p_pad, s->b_g3.p, pl.n_pad,
                                   pl.npad, g3c)))
        return rc;
    } else {
      const void* planes = pl.tc_convert ? s->b_planes.p : A_dev;
      const int64_t pld = pl.tc_convert ? pl.p_pad : ld;
      const void* g3c =
          pl.tc_sparse ? static_cast<unsigned char*>(s->b_sparse.p) + sparse_layout(n, pl.npad).g3c : nullptr;
      if ((rc = tc_encode_maps(s->maps_host, planes, pl.tc_na, pld * n, p, n, pld, s->b_x3.p, pl.p_pad, s->b_g3.p,
                               pl.n_pad, pl.npad, g3c)))
        return rc;
    }
    GP_CUDA(cudaMemcpyAsync(s->b_maps.p, s->maps_host, sizeof(TcMaps), cudaMemcpyHostToDevice, s->stream));
  }
  IO& io = *s->io_host;
  std::memset(&io, 0, sizeof(IO));
  io.A = A_dev;
  io.col_scale = scale_dev;
  io.x0 = x0_dev;
  if (staged_out) {
    const size_t nw = (n + 31) / 32;
    if ((rc = ensure(s, &s->s_X, static_cast<size_t>(d.tcsize) * p * m))) return rc;
    if ((rc = ensure(s, &s->s_Z, static_cast<size_t>(d.tcsize) * n * m))) return rc;
    if ((rc = ensure(s, &s->s_sup, sizeof(uint32_t) * nw * m))) return rc;
    if ((rc = ensure(s, &s->s_obj, sizeof(double) * m))) return rc;
    if ((rc = ensure(s, &s->s_it, sizeof(int32_t) * m))) return rc;
    if ((rc = ensure(s, &s->s_stat, sizeof(int32_t) * m))) return rc;
    if ((rc = ensure(s, &s->s_gam, sizeof(double) * m))) return rc;
    io.X = s->s_X.p;
    io.Z = s->s_Z.p;
    io.support = static_cast<uint32_t*>(s->s_sup.p);
    io.objective = static_cast<double*>(s->s_obj.p);
    io.iters = static_cast<int32_t*>(s->s_it.p);
    io.status = static_cast<int32_t*>(s->s_stat.p);
    io.gamma_abs = static_cast<double*>(s->s_gam.p);
  } else {
    io.X = r.out.X;
    io.Z = r.out.Z;
    io.support = r.out.support;
    io.objective = r.out.objective;
    io.iters = r.out.iters;
    io.status = r.out.status;
    io.gamma_abs = r.out.gamma_abs;
  }
  io.cnorm = static_cast<double*>(s->b_cnorm.p);
  io.cnorm_src = pl.norms_given ? r.cnorm_src : nullptr;
  io.P = s->b_P.p;
  io.Y = s->b_Y.p;
  io.Xf = pl.ws_Xf ? s->b_Xf.p : nullptr;
  io.ypart = s->b_ypart.p;
  io.T = s->b_T.p;
  io.fpart = static_cast<dd*>(s->b_fpart.p);
  io.gpart = static_cast<double*>(s->b_gpart.p);
  if (pl.tc) {
    io.tc_x3 = s->b_x3.p;
    io.tc_g3 = s->b_g3.p;
    io.tc_maps = s->b_maps.p;
    io.tc_planes = pl.tc_convert ? s->b_planes.p : nullptr;
    io.tc_tpart = pl.ksplit1 > 1 ? s->b_tpart.p : nullptr;
    if (pl.tc_sparse) {
      const SparseLayout L = sparse_layout(n, pl.npad);
      unsigned char* b = static_cast<unsigned char*>(s->b_sparse.p);
      io.tc_act = b + L.act;
      io.tc_list = reinterpret_cast<int32_t*>(b + L.list);
      io.tc_nlist = reinterpret_cast<int32_t*>(b + L.nlist);
      io.tc_cnt = reinterpret_cast<int32_t*>(b + L.cnt);
      io.tc_g3c = b + L.g3c;
      io.tc_nsq = reinterpret_cast<double*>(b + L.nsq);
    }
  }
  for (int j = 0; j < m; ++j) {
    io.gamma_in[j] = r.gamma[j];
    io.mu[j] = r.mu[j];
  }
  io.tol = r.tol;
  io.maxit = r.maxit;
  io.gamma_relative = (r.flags & GPSPCA_GAMMA_RELATIVE) ? 1 : 0;
  io.has_x0 = r.x0 ? 1 : 0;
  GP_CUDA(cudaMemcpyAsync(s->io_dev, s->io_host, sizeof(IO), cudaMemcpyHostToDevice, s->stream));
  return GPSPCA_OK;
}

// Enqueue one solve on the slot's stream (asynchronous).  *empty is set when
// nothing was launched.
// After a solve's kernels on stream cs: host outputs copied from the slot's
// staging, the state read back, the slot's done event recorded.
static int solve_tail(Slot* s, const Request& r, cudaStream_t cs) {
  const DInfo d = dinfo(r.A.dtype);
  const int64_t p = r.A.p, n = r.A.n;
  const int m = r.m;
  if (r.out.location == GPSPCA_HOST) {
    const size_t nw = (n + 31) / 32;
    GP_CUDA(cudaMemcpyAsync(r.out.X, s->s_X.p, static_cast<size_t>(d.tcsize) * p * m, cudaMemcpyDeviceToHost, cs));
    GP_CUDA(cudaMemcpyAsync(r.out.Z, s->s_Z.p, static_cast<size_t>(d.tcsize) * n * m, cudaMemcpyDeviceToHost, cs));
    if (r.out.support)
      GP_CUDA(cudaMemcpyAsync(r.out.support, s->s_sup.p, sizeof(uint32_t) * nw * m, cudaMemcpyDeviceToHost, cs));
    GP_CUDA(cudaMemcpyAsync(r.out.objective, s->s_obj.p, sizeof(double) * m, cudaMemcpyDeviceToHost, cs));
    GP_CUDA(cudaMemcpyAsync(r.out.iters, s->s_it.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, cs));
    GP_CUDA(cudaMemcpyAsync(r.out.status, s->s_stat.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, cs));
    if (r.out.gamma_abs)
      GP_CUDA(cudaMemcpyAsync(r.out.gamma_abs, s->s_gam.p, sizeof(double) * m, cudaMemcpyDeviceToHost, cs));
  }
  if (r.flags & GPSPCA_INJECT_TIMEOUT) {
    // the error word as a timed-out wait leaves it; the next solve's reset clears it
    static const int32_t kTimedOut = kErrTimeout;
    GP_CUDA(cudaMemcpyAsync(&s->st_dev->error, &kTimedOut, sizeof(int32_t), cudaMemcpyHostToDevice, cs));
  }
  // the host reads the state's leading words only (counter, active count,
  // error bits, degenerate flag): the rest stays on the device
  static_assert(offsetof(State, active) == 4 * sizeof(int32_t), "the state's host-read words lead it");
  GP_CUDA(cudaMemcpyAsync(s->st_host, s->st_dev, offsetof(State, active), cudaMemcpyDeviceToHost, cs));
  GP_CUDA(cudaEventRecord(s->done, cs));
  return GPSPCA_OK;
}

static int launch_solve(Slot* s, const Request& r, int nsm, bool* empty) {
  Plan pl;
  int rc = prepare_solve(s, r, nsm, false, &pl, empty);
  if (rc != GPSPCA_OK || *empty) return rc;
  if (r.flags & GPSPCA_EAGER) {
    // the graph's kernels, launched one by one; the host reads the active
    // count after each finish step in place of the WHILE node
    GP_CUDA(launch_prologue(pl, s, s->stream, 0, pl.pca != 0, 0));
    for (int k = 0; k <= r.maxit; ++k) {
      GP_CUDA(cudaMemcpyAsync(&s->st_host->n_active, &s->st_dev->n_active, sizeof(int32_t), cudaMemcpyDeviceToHost,
                              s->stream));
      GP_CUDA(cudaStreamSynchronize(s->stream));
      if (s->st_host->n_active <= 0) break;
      GP_CUDA(launch_body(pl, s, s->stream, 0, 0));
    }
    GP_CUDA(launch_epilogue(pl, s, s->stream));
  } else {
    cudaGraphExec_t exec = nullptr;
    if ((rc = get_graph(pl, s, &exec))) return rc;
    GP_CUDA(cudaGraphLaunch(exec, s->stream));
  }
  return solve_tail(s, r, s->stream);
}

// Result code of a finished solve from its device state.
static int solve_result(Slot* s) {
  GP_CUDA(cudaEventSynchronize(s->done));
  GP_CUDA(cudaGetLastError());
  const State& st = *s->st_host;
  if (st.error & kErrNonFinite) return fail(GPSPCA_ENONFINITE, "A has a non-finite entry (or an entry whose square overflows)");
  if (st.error & kErrTimeout) return fail(GPSPCA_ETIMEDOUT, "a device-side wait for a tile copy gave up");
  if (st.error & kErrLaunch) return fail(GPSPCA_ECUDA, "internal: sweep launched with a tile wider than it reduces");
  if (st.any_degenerate) return fail(GPSPCA_EDEGENERATE, "polar step met a rank-deficient Y (status DEGENERATE)");
  return GPSPCA_OK;
}

static int request_from(Request* r, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                        const double* mu, double tol, int32_t maxit, const void* x0, uint32_t flags,
                        gpspca_out* out) {
  if (!A || !out || !gamma) return fail(GPSPCA_EINVAL, "A, gamma and out must not be NULL");
  if (flags & ~(GPSPCA_GAMMA_RELATIVE | GPSPCA_EAGER | GPSPCA_NO_TENSOR_CORES | GPSPCA_INJECT_TIMEOUT |
                GPSPCA_TIME_T_PASS))
    return fail(GPSPCA_EINVAL, "unknown flag bits 0x%x", flags);
  if (m < 1 || m > kMaxM) return fail(GPSPCA_EINVAL, "m = %d outside [1, %d]", m, kMaxM);
  r->A = *A;
  r->form = form;
  r->m = m;
  r->gamma.assign(gamma, gamma + m);
  r->mu.assign(m, 1.0);
  if (mu) r->mu.assign(mu, mu + m);
  r->tol = tol;
  r->maxit = maxit;
  r->x0 = x0;
  r->flags = flags;
  r->out = *out;
  return GPSPCA_OK;
}

}  // namespace gpspca

// ---------------------------------------------------------------- context + serving

using namespace gpspca;

struct Ticket {
  Request req;
  std::string msg;
  int rc = GPSPCA_PENDING;
  bool done = false;
  std::chrono::steady_clock::time_point t_submit;
  size_t foot = 0;  // the request's own device bytes (A, its scales, the outputs), reserved while it runs
};

// Device bytes a submitted request holds while it is solved: its matrix (and
// fp8 scales) and its outputs; the solve's workspace comes on top.
static size_t request_footprint(const Request& r) {
  const DInfo d = dinfo(r.A.dtype);
  const size_t m = static_cast<size_t>(r.m), p = static_cast<size_t>(r.A.p), n = static_cast<size_t>(r.A.n);
  size_t f = static_cast<size_t>(r.A.ld) * n * d.esize;
  if (r.A.dtype == GPSPCA_FP8_E4M3) f += sizeof(float) * n;
  f += static_cast<size_t>(d.tcsize) * (p + n) * m + sizeof(uint32_t) * ((n + 31) / 32) * m +
       (2 * sizeof(double) + 2 * sizeof(int32_t)) * m;
  return f;
}

// Reserve (or return) bytes of the context budget; false if they do not fit.
static bool budget_take(Budget* b, size_t bytes) {
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->used + bytes > b->limit) return false;
  b->used += bytes;
  return true;
}
static void budget_give(Budget* b, size_t bytes) {
  std::lock_guard<std::mutex> lk(b->mu);
  b->used -= std::min(b->used, bytes);
}

struct gpspca_ctx {
  int device = 0;
  int nsm = 0;
  Budget budget;
  TuneTable tune;
  Slot sync_slot;
  std::mutex solve_mu;  // one synchronous solve at a time on sync_slot
  // serving
  std::vector<std::unique_ptr<Slot>> serve_slots;
  std::mutex q_mu;
  std::condition_variable q_cv;      // scheduler wakeup
  std::condition_variable done_cv;   // ticket completion
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread sched;
  bool sched_started = false;
  // batches (gpspca_solve_batch), under solve_mu
  std::vector<std::unique_ptr<Slot>> batch_slots;
  cudaEvent_t batch_start = nullptr;
  std::vector<DevBuf> batch_stage;  // host matrices shared by several requests, copied once
  std::vector<DevBuf> batch_norms;  // column norms of device matrices shared by single-unit requests
  // groups of same-shape single-unit solves (gpspca_solve_batch), under
  // solve_mu: member slots, the group's stream and capture streams, the
  // device arrays of the members' IO and State pointers, the group graphs
  std::vector<std::unique_ptr<Slot>> group_slots;
  cudaStream_t group_stream = nullptr, group_cap = nullptr, group_cap2 = nullptr;
  cudaEvent_t group_done = nullptr;
  void** group_ptrs = nullptr;       // device: kGroupMax IO pointers, then kGroupMax State pointers
  void** group_ptrs_host = nullptr;  // pinned
  std::unordered_map<std::string, Slot::GraphEntry> group_graphs;
  // uploads (gpspca_upload), under up_mu: copies on their own stream, each
  // destination with the event its copy recorded, oldest first
  std::mutex up_mu;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t up_tail = nullptr;
  struct Upload {
    const void* data;
    cudaEvent_t done;
  };
  std::vector<Upload> uploads;
};

static constexpr size_t kUploads = 16;

// Make stream s wait (on the device) for the copy of the latest upload whose
// destination is A's data, if there is one.
static int wait_upload(gpspca_ctx* ctx, cudaStream_t s, const gpspca_matrix& A) {
  if (A.location != GPSPCA_DEVICE || !A.data) return GPSPCA_OK;
  std::lock_guard<std::mutex> lk(ctx->up_mu);
  for (const gpspca_ctx::Upload& u : ctx->uploads)
    if (u.data == A.data) {
      GP_CUDA(cudaStreamWaitEvent(s, u.done, 0));
      break;
    }
  return GPSPCA_OK;
}

static constexpr int kServeSlots = 8;

// Scheduler: admits queued requests into free slots (each slot has its own
// stream and workspace), so solves that arrive while others run overlap on
// the device; completion is detected per slot with events and reported to
// gpspca_poll.  Admission is by HBM footprint: a request starts when its own
// device bytes (matrix, scales, outputs) and its solve's workspace fit in the
// context budget next to the running solves, and waits for one to finish
// otherwise; both are returned when it completes.
static void scheduler_main(gpspca_ctx* ctx) {
  cudaSetDevice(ctx->device);
  std::vector<uint64_t> running(ctx->serve_slots.size(), 0);
  for (;;) {
    bool progressed = false;
    // completions
    for (size_t i = 0; i < running.size(); ++i) {
      if (!running[i]) continue;
      Slot* s = ctx->serve_slots[i].get();
      if (cudaEventQuery(s->done) == cudaErrorNotReady) continue;
      const int rc = solve_result(s);
      release_workspace(s);  // the budget counts running solves only
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      auto it = ctx->tickets.find(running[i]);
      if (it != ctx->tickets.end()) {
        budget_give(&ctx->budget, it->second->foot);
        it->second->rc = rc;
        it->second->msg = rc == GPSPCA_OK ? "" : t_last_error;
        it->second->done = true;
      }
      running[i] = 0;
      progressed = true;
      ctx->done_cv.notify_all();
    }
    // admissions
    for (size_t i = 0; i < running.size(); ++i) {
      if (running[i]) continue;
      uint64_t id = 0;
      Ticket* t = nullptr;
      {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        if (ctx->queue.empty()) break;
        id = ctx->queue.front();
        t = ctx->tickets[id].get();
      }
      Slot* s = ctx->serve_slots[i].get();
      bool any = false;
      for (uint64_t r2 : running) any = any || r2;
      bool empty = false;
      int rc = GPSPCA_ENOMEM;
      if (budget_take(&ctx->budget, t->foot)) {
        rc = wait_upload(ctx, s->stream, t->req.A);
        if (rc == GPSPCA_OK) rc = launch_solve(s, t->req, ctx->nsm, &empty);
        if (rc != GPSPCA_OK || empty) budget_give(&ctx->budget, t->foot);
      }
      if (rc == GPSPCA_ENOMEM) {
        // does not fit next to the running solves: wait for one to finish,
        // unless nothing runs (then it can never fit)
        release_workspace(s);
        if (any) break;
        fail(GPSPCA_ENOMEM, "request of %zu bytes (matrix and outputs) and its workspace exceed the budget of %zu",
             t->foot, ctx->budget.limit);
      }
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      ctx->queue.pop_front();
      progressed = true;
      if (rc != GPSPCA_OK || empty) {
        if (rc != GPSPCA_OK) release_workspace(s);
        t->rc = rc;
        t->msg = rc == GPSPCA_OK ? "" : t_last_error;
        t->done = true;
        ctx->done_cv.notify_all();
      } else {
        running[i] = id;
      }
    }
    bool any_running = false;
    for (uint64_t r2 : running) any_running = any_running || r2;
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    if (ctx->stop && ctx->queue.empty() && !any_running) break;
    if (!progressed) {
      if (any_running)
        ctx->q_cv.wait_for(lk, std::chrono::microseconds(50));
      else
        ctx->q_cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return ctx->stop || !ctx->queue.empty(); });
    }
  }
}

extern "C" {

const char* gpspca_last_error(void) { return t_last_error.c_str(); }

int gpspca_create(gpspca_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return fail(GPSPCA_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  int ndev = 0;
  GP_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(GPSPCA_EINVAL, "device %d out of range (%d devices)", device, ndev);
  GP_CUDA(cudaSetDevice(device));
  auto* ctx = new gpspca_ctx();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  ctx->budget.limit = hbm_budget_bytes ? hbm_budget_bytes : static_cast<size_t>(0.9 * fr);
  int rc = slot_init(&ctx->sync_slot, device, static_cast<cudaStream_t>(cuda_stream), &ctx->budget, &ctx->tune);
  if (rc != GPSPCA_OK) {
    slot_free(&ctx->sync_slot);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return GPSPCA_OK;
}

static constexpr int kBatchSlots = 8;

// ---------------------------------------------------------------- groups
//
// Same-shape single-unit requests of a batch (one component; same storage
// type, form, shape, column stride and alignment; a CUDA-core plan of one
// pass in clusters of one CTA) run as a group: every step of the solve is
// one launch for all of them, the grid's z dimension the member, and the
// loop one WHILE node that continues while any member is active.  Each
// member keeps its own workspace, state, stopping test and outputs and runs
// the kernel bodies of a solo solve.  Its sweep is planned for about
// kGroupCols columns per CTA instead of one column slab per SM (the group
// fills the GPU, not the member), so its partial sums are grouped
// differently from a solo solve's: the results agree with it to float
// rounding and do not depend on the group's size or other members.  Many
// small solves then pay one launch per step, not one per solve per step.

static constexpr int kGroupMin = 4;      // fewer same-shape requests run as ordinary solves
static constexpr int kGroupMax = 256;    // members per group launch
static constexpr int64_t kGroupCols = 128;  // columns per CTA of a member's sweep

// The group a request may join ("" for none).
static std::string group_bucket(const Request& r) {
  if (r.form >= GPSPCA_BL1 || r.m != 1 || (r.flags & (GPSPCA_EAGER | GPSPCA_INJECT_TIMEOUT)) || r.A.p <= 0 ||
      r.A.n <= 0 || r.A.location != GPSPCA_DEVICE)
    return "";
  const DInfo d = dinfo(r.A.dtype);
  const bool fast = (reinterpret_cast<uintptr_t>(r.A.data) % 16 == 0) && ((r.A.ld * d.esize) % 16 == 0);
  char b[192];
  snprintf(b, sizeof(b), "%d/%d/%lld/%lld/%lld/%d/%u", static_cast<int>(r.A.dtype), static_cast<int>(r.form),
           (long long)r.A.p, (long long)r.A.n, (long long)r.A.ld, fast ? 1 : 0, r.flags & GPSPCA_NO_TENSOR_CORES);
  return b;
}

static bool group_plan_ok(const Plan& pl) {
  return !pl.tc && !pl.pca && !pl.norms_in_sweep && pl.C == 1 && pl.passes.size() == 1 && pl.passes[0].mg == 1 &&
         pl.passes[0].mgv == 1 && sweep_kernel_grouped_su(pl.dtype, pl.passes[0].nch) != nullptr;
}

// The start of a group's solves (as launch_prologue for a single-unit form).
static cudaError_t group_start(const Plan& pl, GroupPtrs g, int count, cudaStream_t cs,
                               cudaGraphConditionalHandle h) {
  launch_reset_g(g, count, pl.m, pl.form, cs);
  launch_colnorm_g(pl.dtype, g, count, pl.ld, pl.p, pl.n, pl.fast, cs);
  const StartArgs sa{nullptr, nullptr, pl.ld, pl.p, pl.n, pl.m, pl.form};
  launch_select_start_g(pl.dtype, sa, g, count, cs);
  launch_gather_start_g(pl.dtype, sa, g, count, cs);
  const int gram_pairs = pl.full_gram ? pl.m * (pl.m + 1) / 2 : pl.m;
  const ReduceArgs ra{nullptr, nullptr, 1, pl.m, pl.p, pl.full_gram, gram_pairs, 1, 0, 0, pl.n, pl.form, pl.nred, 0};
  launch_reduce_g(pl.tcsize, ra, g, count, cs);
  const FinishArgs fa{nullptr, nullptr, pl.ncl, pl.nred, gram_pairs, pl.m, pl.form, kFinishPolar, 1, h, 0};
  launch_finish_g(fa, pl.finish_smem, g, count, cs);
  launch_group_cond(g, count, h, cs);
  return cudaGetLastError();
}

// One sweep of a group (as launch_body for a single-unit form).
static cudaError_t group_sweep(const Plan& pl, GroupPtrs g, int count, cudaStream_t cs,
                               cudaGraphConditionalHandle h) {
  const Pass& q = pl.passes[0];
  SweepArgs a{nullptr, nullptr, pl.ld, pl.p, pl.n, pl.m, pl.form, q.j0, q.mgv, pl.ps, q.W, q.S, pl.cols_per_cl,
              pl.fast, 0, q.ov};
  void* args[] = {&a, &g};
  cudaError_t e = cudaLaunchKernel(sweep_kernel_grouped_su(pl.dtype, q.nch), dim3(pl.ncl, 1, count),
                                   dim3(q.threads), args, static_cast<size_t>(q.smem), cs);
  if (e != cudaSuccess) return e;
  const int gram_pairs = pl.full_gram ? pl.m * (pl.m + 1) / 2 : pl.m;
  const ReduceArgs ra{nullptr, nullptr, pl.ncl, pl.m, pl.p, pl.full_gram, gram_pairs, 0, 0, 1, pl.n, pl.form,
                      pl.nred, pl.nobj};
  launch_reduce_g(pl.tcsize, ra, g, count, cs);
  const FinishArgs fa{nullptr, nullptr, pl.nobj, pl.nred, gram_pairs, pl.m, pl.form, kFinishIterate, 0, h, 0};
  launch_finish_g(fa, pl.finish_smem, g, count, cs);
  launch_group_cond(g, count, h, cs);
  return cudaGetLastError();
}

static int group_init(gpspca_ctx* ctx) {
  if (ctx->group_stream) return GPSPCA_OK;
  GP_CUDA(cudaStreamCreateWithFlags(&ctx->group_stream, cudaStreamNonBlocking));
  GP_CUDA(cudaStreamCreateWithFlags(&ctx->group_cap, cudaStreamNonBlocking));
  GP_CUDA(cudaStreamCreateWithFlags(&ctx->group_cap2, cudaStreamNonBlocking));
  GP_CUDA(cudaEventCreateWithFlags(&ctx->group_done, cudaEventDisableTiming));
  GP_CUDA(cudaMalloc(&ctx->group_ptrs, 2 * kGroupMax * sizeof(void*)));
  GP_CUDA(cudaMallocHost(&ctx->group_ptrs_host, 2 * kGroupMax * sizeof(void*)));
  return GPSPCA_OK;
}

// Runs requests R[idx[k]] as one group, after the work on the context's
// stream recorded by ctx->batch_start, and collects each result into
// rcs[idx[k]].  *ran = false (nothing launched) when their plan cannot run
// as a group: the caller solves them one by one.
static int run_group(gpspca_ctx* ctx, const std::vector<Request>& R, const std::vector<int>& idx, int32_t* rcs,
                     bool* ran) {
  *ran = false;
  int rc = group_init(ctx);
  if (rc != GPSPCA_OK) return rc;
  const int count = static_cast<int>(idx.size());
  while (static_cast<int>(ctx->group_slots.size()) < count) {
    auto sl = std::make_unique<Slot>();
    rc = slot_init(sl.get(), ctx->device, ctx->group_stream, &ctx->budget, &ctx->tune, false);
    if (rc != GPSPCA_OK) {
      slot_free(sl.get());
      return rc;
    }
    ctx->group_slots.push_back(std::move(sl));
  }
  cudaStream_t gs = ctx->group_stream;
  GP_CUDA(cudaStreamWaitEvent(gs, ctx->batch_start, 0));
  // column slabs of a member's sweep: one per kGroupCols columns
  const int nsm_g = static_cast<int>(std::max<int64_t>(1, (R[idx[0]].A.n + kGroupCols - 1) / kGroupCols));
  Plan pl0;
  std::vector<int> member;  // indices into idx of the members that prepared
  for (int k = 0; k < count; ++k) {
    Plan pl;
    bool empty = false;
    const int r = prepare_solve(ctx->group_slots[k].get(), R[idx[k]], nsm_g, false, &pl, &empty, -1, nullptr,
                                nullptr, member.empty() ? nullptr : &pl0);
    if (r != GPSPCA_OK || empty) {
      rcs[idx[k]] = r;
      continue;
    }
    if (member.empty()) {
      if (!group_plan_ok(pl)) return GPSPCA_OK;  // not a group plan: solved one by one
      pl0 = pl;
    } else if (pl.key() != pl0.key()) {
      return GPSPCA_OK;
    }
    member.push_back(k);
  }
  *ran = true;
  const int nm = static_cast<int>(member.size());
  if (nm == 0) return GPSPCA_OK;
  for (int u = 0; u < nm; ++u) {
    ctx->group_ptrs_host[u] = ctx->group_slots[member[u]]->io_dev;
    ctx->group_ptrs_host[kGroupMax + u] = ctx->group_slots[member[u]]->st_dev;
  }
  GP_CUDA(cudaMemcpyAsync(ctx->group_ptrs, ctx->group_ptrs_host, 2 * kGroupMax * sizeof(void*),
                          cudaMemcpyHostToDevice, gs));
  const GroupPtrs g{reinterpret_cast<const IO* const*>(ctx->group_ptrs),
                    reinterpret_cast<State* const*>(ctx->group_ptrs + kGroupMax)};
  kattr(sweep_kernel_grouped_su(pl0.dtype, pl0.passes[0].nch));  // its dynamic shared memory limit
  const std::string key = pl0.key() + "|group" + std::to_string(nm);
  auto it = ctx->group_graphs.find(key);
  if (it == ctx->group_graphs.end()) {
    Slot::GraphEntry ge;
    rc = capture_loop_graph(
        ctx->group_cap, ctx->group_cap2,
        [&](cudaStream_t cs, cudaGraphConditionalHandle h) { return group_start(pl0, g, nm, cs, h); },
        [&](cudaStream_t cs, cudaGraphConditionalHandle h) { return group_sweep(pl0, g, nm, cs, h); },
        [&](cudaStream_t cs) {
          launch_finalize_g(pl0.tcsize, g, nm, pl0.p, pl0.n, pl0.m, pl0.form, cs);
          return cudaGetLastError();
        },
        &ge);
    if (rc != GPSPCA_OK) return rc;
    if (ctx->group_graphs.size() >= 64) {  // bound the cache
      for (auto& kv : ctx->group_graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.g);
      }
      ctx->group_graphs.clear();
    }
    it = ctx->group_graphs.emplace(key, ge).first;
  }
  GP_CUDA(cudaGraphLaunch(it->second.exec, gs));
  for (int u = 0; u < nm; ++u)
    if ((rc = solve_tail(ctx->group_slots[member[u]].get(), R[idx[member[u]]], gs)) != GPSPCA_OK) return rc;
  GP_CUDA(cudaEventRecord(ctx->group_done, gs));
  for (int u = 0; u < nm; ++u) rcs[idx[member[u]]] = solve_result(ctx->group_slots[member[u]].get());
  return GPSPCA_OK;
}

int gpspca_solve_batch(gpspca_ctx* ctx, int32_t count, const gpspca_request* reqs, int32_t* rcs) {
  if (!ctx) return fail(GPSPCA_EINVAL, "ctx is NULL");
  if (count < 0 || (count > 0 && (!reqs || !rcs))) return fail(GPSPCA_EINVAL, "bad batch arguments");
  std::vector<Request> R(static_cast<size_t>(count));
  for (int i = 0; i < count; ++i) {
    gpspca_out o = reqs[i].out;
    const int rc = request_from(&R[i], &reqs[i].A, reqs[i].form, reqs[i].gamma, reqs[i].m, reqs[i].mu, reqs[i].tol,
                                reqs[i].maxit, reqs[i].x0, reqs[i].flags, &o);
    if (rc != GPSPCA_OK) return fail(rc, "batch request %d: %s", i, t_last_error.c_str());
  }
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  if (!ctx->batch_start) GP_CUDA(cudaEventCreateWithFlags(&ctx->batch_start, cudaEventDisableTiming));
  const int nb = std::min(count, kBatchSlots);
  while (static_cast<int>(ctx->batch_slots.size()) < nb) {
    auto s = std::make_unique<Slot>();
    const int rc = slot_init(s.get(), ctx->device, nullptr, &ctx->budget, &ctx->tune);
    if (rc != GPSPCA_OK) {
      slot_free(s.get());
      return rc;
    }
    ctx->batch_slots.push_back(std::move(s));
  }
  cudaStream_t cs = ctx->sync_slot.stream;
  // A host matrix that several requests share (same buffer, type, shape,
  // stride and scales) is copied to the device once, on the context's stream
  // before the batch starts, and those requests read the device copy.
  {
    size_t nstage = 0;
    for (int i = 0; i < count; ++i) {
      const gpspca_matrix& Ai = R[i].A;
      if (Ai.location != GPSPCA_HOST || Ai.p <= 0 || Ai.n <= 0 || !Ai.data) continue;
      int users = 0;
      for (int k = i; k < count; ++k) {
        const gpspca_matrix& Ak = R[k].A;
        users += Ak.location == GPSPCA_HOST && Ak.data == Ai.data && Ak.dtype == Ai.dtype && Ak.p == Ai.p &&
                 Ak.n == Ai.n && Ak.ld == Ai.ld && Ak.col_scale == Ai.col_scale;
      }
      if (users < 2) continue;
      const gpspca_matrix host = Ai;
      const size_t a_bytes = static_cast<size_t>(host.ld) * host.n * dinfo(host.dtype).esize;
      const size_t s_bytes = host.dtype == GPSPCA_FP8_E4M3 ? sizeof(float) * host.n : 0;
      if (ctx->batch_stage.size() <= nstage) ctx->batch_stage.resize(nstage + 1);
      DevBuf* buf = &ctx->batch_stage[nstage++];
      int rc = ensure(&ctx->sync_slot, buf, a_bytes + s_bytes + 256);
      if (rc != GPSPCA_OK) return rc;
      GP_CUDA(cudaMemcpyAsync(buf->p, host.data, a_bytes, cudaMemcpyHostToDevice, cs));
      float* scale = nullptr;
      if (s_bytes) {
        scale = reinterpret_cast<float*>(static_cast<char*>(buf->p) + (a_bytes + 255) / 256 * 256);
        GP_CUDA(cudaMemcpyAsync(scale, host.col_scale, s_bytes, cudaMemcpyHostToDevice, cs));
      }
      for (int k = i; k < count; ++k) {
        gpspca_matrix& Ak = R[k].A;
        if (Ak.location == GPSPCA_HOST && Ak.data == host.data && Ak.dtype == host.dtype && Ak.p == host.p &&
            Ak.n == host.n && Ak.ld == host.ld && Ak.col_scale == host.col_scale) {
          Ak.location = GPSPCA_DEVICE;
          Ak.data = buf->p;
          Ak.col_scale = scale;
        }
      }
    }
  }
  for (int i = 0; i < count; ++i) {
    const int rc = wait_upload(ctx, cs, R[i].A);
    if (rc != GPSPCA_OK) return rc;
  }
  // kGroupMin or more same-shape single-unit requests: grouped launches
  std::vector<std::vector<int>> groups;
  std::vector<char> grouped(static_cast<size_t>(count), 0);
  {
    std::map<std::string, std::vector<int>> buckets;
    for (int i = 0; i < count; ++i) {
      const std::string b = group_bucket(R[i]);
      if (!b.empty()) buckets[b].push_back(i);
    }
    for (auto& kv : buckets)
      for (size_t o = 0; o < kv.second.size(); o += kGroupMax) {
        const size_t e = std::min(kv.second.size(), o + kGroupMax);
        if (e - o < static_cast<size_t>(kGroupMin)) continue;
        groups.emplace_back(kv.second.begin() + static_cast<std::ptrdiff_t>(o),
                            kv.second.begin() + static_cast<std::ptrdiff_t>(e));
        for (size_t q = o; q < e; ++q) grouped[kv.second[q]] = 1;
      }
  }
  std::vector<int> solo;
  for (int i = 0; i < count; ++i)
    if (!grouped[i]) solo.push_back(i);
  // Single-unit solo requests that share a device matrix (two or more of
  // them: same buffer, type, shape, stride and scales) take its column norms
  // from one pass made here, on the context's stream before the batch
  // starts, instead of one pass each: the norm of a column does not depend on
  // the launch, so every solve sees the values its own pass would have made
  // (block solves keep theirs: they form them in their first power step).
  {
    auto same = [](const gpspca_matrix& a, const gpspca_matrix& b) {
      return a.location == b.location && a.data == b.data && a.dtype == b.dtype && a.p == b.p && a.n == b.n &&
             a.ld == b.ld && a.col_scale == b.col_scale;
    };
    auto shares = [](const Request& r) {
      return r.form < GPSPCA_BL1 && r.A.location == GPSPCA_DEVICE && r.A.p > 0 && r.A.n > 0 && r.A.data &&
             r.A.ld >= r.A.p && !(r.flags & GPSPCA_INJECT_TIMEOUT);
    };
    std::vector<char> taken(static_cast<size_t>(count), 0);
    size_t nsh = 0;
    for (size_t a = 0; a < solo.size(); ++a) {
      const int i = solo[a];
      if (taken[i] || !shares(R[i])) continue;
      std::vector<int> users;
      for (size_t b = a; b < solo.size(); ++b)
        if (!taken[solo[b]] && shares(R[solo[b]]) && same(R[solo[b]].A, R[i].A)) users.push_back(solo[b]);
      if (users.size() < 2) continue;
      const gpspca_matrix& A = R[i].A;
      const DInfo d = dinfo(A.dtype);
      const size_t nbytes = (sizeof(double) * static_cast<size_t>(A.n) + 255) / 256 * 256;
      if (ctx->batch_norms.size() <= nsh) ctx->batch_norms.resize(nsh + 1);
      DevBuf* nb = &ctx->batch_norms[nsh++];
      const int rc = ensure(&ctx->sync_slot, nb, nbytes + 256);
      if (rc != GPSPCA_OK) return rc;
      double* norms = static_cast<double*>(nb->p);
      int32_t* err = reinterpret_cast<int32_t*>(static_cast<char*>(nb->p) + nbytes);  // not read: each solve checks
      const bool fast = (reinterpret_cast<uintptr_t>(A.data) % 16 == 0) && ((A.ld * d.esize) % 16 == 0);
      launch_colnorm_shared(A.dtype, A.data, A.col_scale, norms, err, A.ld, static_cast<int>(A.p),
                            static_cast<int>(A.n), fast ? 1 : 0, cs);
      GP_CUDA(cudaGetLastError());
      for (int k : users) {
        taken[k] = 1;
        R[k].cnorm_src = norms;
      }
    }
  }
  GP_CUDA(cudaEventRecord(ctx->batch_start, cs));
  std::vector<char> running(static_cast<size_t>(count), 0);
  auto collect = [&](int k) {  // the solo solve at position k
    rcs[solo[k]] = solve_result(ctx->batch_slots[k % kBatchSlots].get());
    running[solo[k]] = 0;
  };
  for (int k = 0; k < static_cast<int>(solo.size()); ++k) {
    const int i = solo[k];
    Slot* s = ctx->batch_slots[k % kBatchSlots].get();
    if (k >= kBatchSlots && running[solo[k - kBatchSlots]]) collect(k - kBatchSlots);  // the slot's previous solve
    GP_CUDA(cudaStreamWaitEvent(s->stream, ctx->batch_start, 0));
    bool empty = false;
    const int rc = launch_solve(s, R[i], ctx->nsm, &empty);
    rcs[i] = rc;
    running[i] = (rc == GPSPCA_OK && !empty) ? 1 : 0;
  }
  // the groups, one after the other on the group stream, while the solo
  // solves run; a group whose plan cannot run grouped is solved one by one
  // on the context's stream
  for (const std::vector<int>& gv : groups) {
    bool ran = false;
    const int rc = run_group(ctx, R, gv, rcs, &ran);
    if (rc != GPSPCA_OK) {
      for (int i : gv) rcs[i] = rc;
      continue;
    }
    if (ran) continue;
    for (int i : gv) {
      bool empty = false;
      rcs[i] = launch_solve(&ctx->sync_slot, R[i], ctx->nsm, &empty);
      if (rcs[i] == GPSPCA_OK && !empty) rcs[i] = solve_result(&ctx->sync_slot);
    }
  }
  if (!groups.empty() && ctx->group_done) GP_CUDA(cudaStreamWaitEvent(cs, ctx->group_done, 0));
  for (int k = 0; k < nb; ++k) GP_CUDA(cudaStreamWaitEvent(cs, ctx->batch_slots[k]->done, 0));
  for (int k = 0; k < static_cast<int>(solo.size()); ++k)
    if (running[solo[k]]) collect(k);
  for (int i = 0; i < count; ++i)
    if (rcs[i] != GPSPCA_OK && rcs[i] != GPSPCA_EDEGENERATE) return fail(rcs[i], "batch request %d failed", i);
  return GPSPCA_OK;
}

int gpspca_upload(gpspca_ctx* ctx, const gpspca_matrix* host, const gpspca_matrix* dst) {
  if (!ctx || !host || !dst) return fail(GPSPCA_EINVAL, "ctx, host and dst must not be NULL");
  const gpspca_matrix& H = *host;
  const gpspca_matrix& D = *dst;
  if (H.location != GPSPCA_HOST) return fail(GPSPCA_EINVAL, "upload source must be a host matrix");
  if (D.location != GPSPCA_DEVICE) return fail(GPSPCA_EINVAL, "upload destination must be a device matrix");
  if (H.dtype < GPSPCA_F32 || H.dtype > GPSPCA_F64) return fail(GPSPCA_EINVAL, "unknown dtype %d", (int)H.dtype);
  if (H.dtype != D.dtype || H.p != D.p || H.n != D.n)
    return fail(GPSPCA_EINVAL, "upload source and destination differ in dtype or shape");
  const int64_t p = H.p, n = H.n;
  if (p < 0 || n < 0 || p > (1 << 30) || n > (1 << 30)) return fail(GPSPCA_EINVAL, "bad shape");
  if (p == 0 || n == 0) return GPSPCA_OK;
  if (!H.data || !D.data) return fail(GPSPCA_EINVAL, "upload data pointer is NULL");
  if (H.ld < p || D.ld < p) return fail(GPSPCA_EINVAL, "ld < rows");
  const bool fp8 = H.dtype == GPSPCA_FP8_E4M3;
  if (fp8 && (!H.col_scale || !D.col_scale)) return fail(GPSPCA_EINVAL, "FP8 storage needs col_scale on both sides");
  std::lock_guard<std::mutex> lk(ctx->up_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  if (!ctx->copy_stream) GP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->up_tail) GP_CUDA(cudaEventCreateWithFlags(&ctx->up_tail, cudaEventDisableTiming));
  // after the work already enqueued on the context's stream
  GP_CUDA(cudaEventRecord(ctx->up_tail, ctx->sync_slot.stream));
  GP_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->up_tail, 0));
  const size_t es = dinfo(H.dtype).esize;
  void* dd = const_cast<void*>(D.data);  // the descriptor's pointer is const for the solves' reads
  if (H.ld == D.ld) {
    const size_t bytes = (static_cast<size_t>(n - 1) * H.ld + p) * es;
    GP_CUDA(cudaMemcpyAsync(dd, H.data, bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
  } else {
    GP_CUDA(cudaMemcpy2DAsync(dd, D.ld * es, H.data, H.ld * es, p * es, n, cudaMemcpyHostToDevice,
                              ctx->copy_stream));
  }
  if (fp8)
    GP_CUDA(cudaMemcpyAsync(const_cast<float*>(D.col_scale), H.col_scale, sizeof(float) * n, cudaMemcpyHostToDevice,
                            ctx->copy_stream));
  // the destination's entry (moved to the back), or a new one; the oldest
  // is dropped when the table is full, once its copy has finished (later
  // solves of that destination need not wait for it)
  std::vector<gpspca_ctx::Upload>& U = ctx->uploads;
  gpspca_ctx::Upload e{D.data, nullptr};
  for (size_t i = 0; i < U.size(); ++i)
    if (U[i].data == D.data) {
      e = U[i];
      U.erase(U.begin() + static_cast<std::ptrdiff_t>(i));
      break;
    }
  if (!e.done) {
    if (U.size() >= kUploads) {
      GP_CUDA(cudaEventSynchronize(U.front().done));
      e.done = U.front().done;
      U.erase(U.begin());
    } else {
      GP_CUDA(cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming));
    }
  }
  U.push_back(e);
  GP_CUDA(cudaEventRecord(e.done, ctx->copy_stream));
  return GPSPCA_OK;
}

int gpspca_solve(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                 const double* mu, double tol, int32_t maxit, const void* x0, uint32_t flags, gpspca_out* out) {
  if (!ctx) return fail(GPSPCA_EINVAL, "ctx is NULL");
  Request r;
  int rc = request_from(&r, A, form, gamma, m, mu, tol, maxit, x0, flags, out);
  if (rc != GPSPCA_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  if ((rc = wait_upload(ctx, ctx->sync_slot.stream, r.A)) != GPSPCA_OK) return rc;
  bool empty = false;
  rc = launch_solve(&ctx->sync_slot, r, ctx->nsm, &empty);
  if (rc != GPSPCA_OK || empty) return rc;
  return solve_result(&ctx->sync_slot);
}

int gpspca_solve_deflated(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                          double tol, int32_t maxit, uint32_t flags, gpspca_out* out) {
  if (!ctx) return fail(GPSPCA_EINVAL, "ctx is NULL");
  if (form != GPSPCA_SL1 && form != GPSPCA_SL0)
    return fail(GPSPCA_EINVAL, "deflation extracts single-unit components (SL1 or SL0)");
  Request r;
  int rc = request_from(&r, A, form, gamma, m, nullptr, tol, maxit, nullptr, flags, out);
  if (rc != GPSPCA_OK) return rc;
  if ((rc = validate(r)) != GPSPCA_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  Slot* s = &ctx->sync_slot;
  if (r.A.p == 0 || r.A.n == 0) return solve_empty(s, r);
  if ((rc = wait_upload(ctx, s->stream, r.A)) != GPSPCA_OK) return rc;
  const int64_t p = r.A.p, n = r.A.n;
  const int wdt = r.A.dtype == GPSPCA_F64 ? GPSPCA_F64 : GPSPCA_F32;
  const size_t tcs = wdt == GPSPCA_F64 ? sizeof(double) : sizeof(float);
  const int64_t ldw = deflate_ld(wdt, p);
  const size_t nw = static_cast<size_t>((n + 31) / 32);
  // A on the device (host input staged), then the working copy
  const DInfo d = dinfo(r.A.dtype);
  const void* A_dev = r.A.data;
  const float* scale_dev = r.A.col_scale;
  if (r.A.location == GPSPCA_HOST) {
    const size_t a_bytes = static_cast<size_t>(r.A.ld) * n * d.esize;
    if ((rc = ensure(s, &s->s_A, a_bytes))) return rc;
    GP_CUDA(cudaMemcpyAsync(s->s_A.p, r.A.data, a_bytes, cudaMemcpyHostToDevice, s->stream));
    A_dev = s->s_A.p;
    if (r.A.dtype == GPSPCA_FP8_E4M3) {
      if ((rc = ensure(s, &s->s_scale, sizeof(float) * n))) return rc;
      GP_CUDA(cudaMemcpyAsync(s->s_scale.p, r.A.col_scale, sizeof(float) * n, cudaMemcpyHostToDevice, s->stream));
      scale_dev = static_cast<const float*>(s->s_scale.p);
    }
  }
  // workspace like the solves' own (kept for the next call, counted against the budget)
  if ((rc = ensure(s, &s->d_W, tcs * static_cast<size_t>(ldw) * n))) return rc;
  if ((rc = ensure(s, &s->d_list, deflate_list_bytes(wdt, n)))) return rc;
  launch_deflate_copy(r.A.dtype, A_dev, r.A.ld, r.A.dtype == GPSPCA_FP8_E4M3 ? scale_dev : nullptr, s->d_W.p, ldw, p, n,
                      s->stream);
  GP_CUDA(cudaGetLastError());
  if (r.A.location == GPSPCA_HOST) release(s, &s->s_A);  // only the working copy is read from here on
  // results on the device: the caller's buffers, or staging for host outputs
  const bool staged = r.out.location == GPSPCA_HOST;
  gpspca_out o = r.out;
  if (staged) {
    if ((rc = ensure(s, &s->s_X, tcs * p * m))) return rc;
    if ((rc = ensure(s, &s->s_Z, tcs * n * m))) return rc;
    if ((rc = ensure(s, &s->s_sup, sizeof(uint32_t) * nw * m))) return rc;
    if ((rc = ensure(s, &s->s_obj, sizeof(double) * m))) return rc;
    if ((rc = ensure(s, &s->s_it, sizeof(int32_t) * m))) return rc;
    if ((rc = ensure(s, &s->s_stat, sizeof(int32_t) * m))) return rc;
    if ((rc = ensure(s, &s->s_gam, sizeof(double) * m))) return rc;
    o.location = GPSPCA_DEVICE;
    o.X = s->s_X.p;
    o.Z = s->s_Z.p;
    o.support = r.out.support ? static_cast<uint32_t*>(s->s_sup.p) : nullptr;
    o.objective = static_cast<double*>(s->s_obj.p);
    o.iters = static_cast<int32_t*>(s->s_it.p);
    o.status = static_cast<int32_t*>(s->s_stat.p);
    o.gamma_abs = r.out.gamma_abs ? static_cast<double*>(s->s_gam.p) : nullptr;
  }
  int first_err = GPSPCA_OK;
  for (int j = 0; j < m; ++j) {
    Request rj;
    rj.A = gpspca_matrix{s->d_W.p, static_cast<gpspca_dtype>(wdt), GPSPCA_DEVICE, p, n, ldw, nullptr};
    rj.form = r.form;
    rj.m = 1;
    rj.gamma.assign(1, r.gamma[j]);
    rj.mu.assign(1, 1.0);
    rj.tol = r.tol;
    rj.maxit = r.maxit;
    rj.flags = r.flags;
    rj.out = o;
    rj.out.X = static_cast<char*>(o.X) + tcs * p * j;
    rj.out.Z = static_cast<char*>(o.Z) + tcs * n * j;
    rj.out.support = o.support ? o.support + nw * j : nullptr;
    rj.out.objective = o.objective + j;
    rj.out.iters = o.iters + j;
    rj.out.status = o.status + j;
    rj.out.gamma_abs = o.gamma_abs ? o.gamma_abs + j : nullptr;
    bool empty = false;
    rc = launch_solve(s, rj, ctx->nsm, &empty);
    if (rc == GPSPCA_OK && !empty) rc = solve_result(s);
    if (rc != GPSPCA_OK && rc != GPSPCA_EDEGENERATE) return rc;
    if (first_err == GPSPCA_OK) first_err = rc;
    // A_j = A_{j-1} - (A_{j-1} z_j) z_j^T (z_j = 0 leaves it unchanged)
    if (j + 1 < m) {
      launch_deflate(wdt, s->d_W.p, ldw, p, n, rj.out.Z, s->d_list.p, s->stream);
      GP_CUDA(cudaGetLastError());
    }
  }
  if (staged) {
    GP_CUDA(cudaMemcpyAsync(r.out.X, o.X, tcs * p * m, cudaMemcpyDeviceToHost, s->stream));
    GP_CUDA(cudaMemcpyAsync(r.out.Z, o.Z, tcs * n * m, cudaMemcpyDeviceToHost, s->stream));
    if (r.out.support)
      GP_CUDA(cudaMemcpyAsync(r.out.support, o.support, sizeof(uint32_t) * nw * m, cudaMemcpyDeviceToHost, s->stream));
    GP_CUDA(cudaMemcpyAsync(r.out.objective, o.objective, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
    GP_CUDA(cudaMemcpyAsync(r.out.iters, o.iters, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s->stream));
    GP_CUDA(cudaMemcpyAsync(r.out.status, o.status, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s->stream));
    if (r.out.gamma_abs)
      GP_CUDA(cudaMemcpyAsync(r.out.gamma_abs, o.gamma_abs, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream));
  }
  GP_CUDA(cudaStreamSynchronize(s->stream));
  if (first_err != GPSPCA_OK) return fail(first_err, "a component's polar step was degenerate (status DEGENERATE)");
  return GPSPCA_OK;
}

int gpspca_project(gpspca_ctx* ctx, const gpspca_matrix* B, const void* Z, int32_t m, void* S) {
  if (!ctx || !B || !Z || !S) return fail(GPSPCA_EINVAL, "ctx, B, Z and S must not be NULL");
  if (m < 1 || m > kMaxM) return fail(GPSPCA_EINVAL, "m = %d outside [1, %d]", m, kMaxM);
  if (B->dtype < GPSPCA_F32 || B->dtype > GPSPCA_F64) return fail(GPSPCA_EINVAL, "unknown dtype %d", (int)B->dtype);
  if (B->location != GPSPCA_DEVICE && B->location != GPSPCA_HOST) return fail(GPSPCA_EINVAL, "bad B location");
  const int64_t q = B->p, n = B->n;
  if (q < 0 || n < 0 || q > (1 << 30) || n > (1 << 30)) return fail(GPSPCA_EINVAL, "bad shape");
  if (q > 0 && n > 0) {
    if (!B->data) return fail(GPSPCA_EINVAL, "B.data is NULL");
    if (B->ld < q) return fail(GPSPCA_EINVAL, "ld (%lld) < rows (%lld)", (long long)B->ld, (long long)q);
    if (B->dtype == GPSPCA_FP8_E4M3 && !B->col_scale) return fail(GPSPCA_EINVAL, "FP8 storage needs col_scale");
  }
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  Slot* s = &ctx->sync_slot;
  const int wdt = B->dtype == GPSPCA_F64 ? GPSPCA_F64 : GPSPCA_F32;
  const size_t tcs = wdt == GPSPCA_F64 ? sizeof(double) : sizeof(float);
  const bool host = B->location == GPSPCA_HOST;
  if (q == 0) return GPSPCA_OK;
  if (n == 0) {  // no variables: every score is zero
    if (host) {
      std::memset(S, 0, tcs * q * m);
      return GPSPCA_OK;
    }
    GP_CUDA(cudaMemsetAsync(S, 0, tcs * q * m, s->stream));
    GP_CUDA(cudaStreamSynchronize(s->stream));
    return GPSPCA_OK;
  }
  int rc;
  if ((rc = wait_upload(ctx, s->stream, *B)) != GPSPCA_OK) return rc;
  const void* Bd = B->data;
  const float* scale = B->col_scale;
  const void* Zd = Z;
  void* Sd = S;
  if (host) {
    const size_t b_bytes = static_cast<size_t>(B->ld) * n * dinfo(B->dtype).esize;
    if ((rc = ensure(s, &s->s_A, b_bytes))) return rc;
    GP_CUDA(cudaMemcpyAsync(s->s_A.p, B->data, b_bytes, cudaMemcpyHostToDevice, s->stream));
    Bd = s->s_A.p;
    if (B->dtype == GPSPCA_FP8_E4M3) {
      if ((rc = ensure(s, &s->s_scale, sizeof(float) * n))) return rc;
      GP_CUDA(cudaMemcpyAsync(s->s_scale.p, B->col_scale, sizeof(float) * n, cudaMemcpyHostToDevice, s->stream));
      scale = static_cast<const float*>(s->s_scale.p);
    }
    if ((rc = ensure(s, &s->s_Z, tcs * n * m))) return rc;
    GP_CUDA(cudaMemcpyAsync(s->s_Z.p, Z, tcs * n * m, cudaMemcpyHostToDevice, s->stream));
    Zd = s->s_Z.p;
    if ((rc = ensure(s, &s->s_X, tcs * q * m))) return rc;
    Sd = s->s_X.p;
  }
  if ((rc = ensure(s, &s->d_list, deflate_list_bytes(wdt, n) * m))) return rc;
  launch_project(B->dtype, Bd, B->ld, B->dtype == GPSPCA_FP8_E4M3 ? scale : nullptr, q, n, Zd, m, Sd, s->d_list.p,
                 s->stream);
  GP_CUDA(cudaGetLastError());
  if (host) GP_CUDA(cudaMemcpyAsync(S, Sd, tcs * q * m, cudaMemcpyDeviceToHost, s->stream));
  GP_CUDA(cudaStreamSynchronize(s->stream));
  return GPSPCA_OK;
}

int gpspca_time_sweep(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                      const double* mu, uint32_t flags, int32_t reps, double* ms_per_sweep) {
  if (!ctx || !ms_per_sweep) return fail(GPSPCA_EINVAL, "ctx and ms_per_sweep must not be NULL");
  if (reps < 1) return fail(GPSPCA_EINVAL, "reps must be >= 1");
  gpspca_out dummy = {};
  dummy.location = GPSPCA_DEVICE;
  double one = 0.0;
  dummy.X = dummy.Z = dummy.objective = &one;  // replaced by staging buffers
  dummy.iters = dummy.status = reinterpret_cast<int32_t*>(&one);
  Request r;
  int rc = request_from(&r, A, form, gamma, m, mu, 0.0, 1 << 30, nullptr, flags, &dummy);
  if (rc != GPSPCA_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  Slot* s = &ctx->sync_slot;
  if ((rc = wait_upload(ctx, s->stream, r.A)) != GPSPCA_OK) return rc;
  Plan pl;
  bool empty = false;
  rc = prepare_solve(s, r, ctx->nsm, true, &pl, &empty);
  if (rc != GPSPCA_OK) return rc;
  if (empty) return fail(GPSPCA_EINVAL, "empty matrix");
  const int t_only = (flags & GPSPCA_TIME_T_PASS) ? 1 : 0;
  if (t_only && !pl.tc) return fail(GPSPCA_EINVAL, "GPSPCA_TIME_T_PASS: this problem runs the CUDA-core sweep");
  // the start alone (the sweeps timed are the loop's; its first one stays out)
  GP_CUDA(launch_prologue(pl, s, s->stream, cudaGraphConditionalHandle{}, pl.pca != 0, 0, false));
  cudaEvent_t e0, e1;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  GP_CUDA(launch_sweeps(pl, s, s->stream, 0, 0, t_only));  // warm-up
  GP_CUDA(cudaEventRecord(e0, s->stream));
  for (int i = 0; i < reps; ++i) GP_CUDA(launch_sweeps(pl, s, s->stream, 0, 0, t_only));
  GP_CUDA(cudaEventRecord(e1, s->stream));
  GP_CUDA(cudaEventSynchronize(e1));
  GP_CUDA(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GP_CUDA(cudaMemcpy(s->st_host, s->st_dev, sizeof(State), cudaMemcpyDeviceToHost));
  if (s->st_host->error & kErrTimeout) return fail(GPSPCA_ETIMEDOUT, "a device-side wait for a tile copy gave up");
  if (s->st_host->n_active == 0) return fail(GPSPCA_EINVAL, "the start is degenerate or A is zero: nothing to time");
  *ms_per_sweep = static_cast<double>(ms) / reps;
  return GPSPCA_OK;
}

// Kernel launches of one plan: before the iterations, per iteration, after
// (mirrors launch_prologue / launch_body / launch_epilogue).
static void plan_launch_counts(const Plan& pl, int32_t c[3]) {
  // the start's power steps launch no active-column list (two kernels in a threshold sweep)
  const int sweeps = pl.tc ? 3 + (pl.ksplit1 > 1 ? 1 : 0)
                          : static_cast<int>(pl.passes.size()) + (pl.form >= 2 ? 1 : 0);  // + form_x
  const bool late_norms = pl.pca && pl.norms_in_sweep;
  int pro = (pl.tc && pl.tc_convert ? 1 : 0) + 1 + (late_norms ? 0 : 2) + 1 + 2;
  // the Rayleigh-Ritz step: a sweep, its reduction and finish; on the tensor
  // cores X3 and the T pass (+ combine), T^T T and the finish
  const int ritz = pl.tc ? 2 + (pl.ksplit1 > 1 ? 1 : 0) + 2 : sweeps + 2;
  if (pl.pca) pro += kPowerSteps * (sweeps + 2) + (late_norms ? 1 : 0) + (late_norms && pl.tc ? 1 : 0) + ritz;
  // the first sweep runs with the start, its T pass (and combine) replaced
  // by one kernel: counted as an iteration, less the difference
  if (first_sweep_from_ritz(pl)) pro -= (pl.ksplit1 > 1 ? 1 : 0);
  c[0] = pro;
  c[1] = sweeps + (pl.tc_sparse ? 2 : 0) + 2;
  c[2] = 1;
}

int gpspca_plan_launches(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                         const double* mu, uint32_t flags, int32_t counts[3]) {
  if (!ctx || !counts) return fail(GPSPCA_EINVAL, "ctx and counts must not be NULL");
  gpspca_out dummy = {};
  dummy.location = GPSPCA_DEVICE;
  double one = 0.0;
  dummy.X = dummy.Z = dummy.objective = &one;  // replaced by staging buffers
  dummy.iters = dummy.status = reinterpret_cast<int32_t*>(&one);
  Request r;
  int rc = request_from(&r, A, form, gamma, m, mu, 0.0, 1, nullptr, flags, &dummy);
  if (rc != GPSPCA_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  Plan pl;
  bool empty = false;
  rc = prepare_solve(&ctx->sync_slot, r, ctx->nsm, true, &pl, &empty);
  if (rc != GPSPCA_OK) return rc;
  if (empty) {
    counts[0] = counts[1] = counts[2] = 0;
    return GPSPCA_OK;
  }
  plan_launch_counts(pl, counts);
  return GPSPCA_OK;
}

// Time one prepared plan's sweep: start and projection as a solve does,
// one warm-up sweep, then `reps` sweeps between CUDA events.
static int time_plan(Slot* s, const Plan& pl, int reps, double* ms_per_sweep) {
  // the start alone (the sweeps timed are the loop's; its first one stays out)
  GP_CUDA(launch_prologue(pl, s, s->stream, cudaGraphConditionalHandle{}, pl.pca != 0, 0, false));
  cudaEvent_t e0, e1;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  GP_CUDA(launch_sweeps(pl, s, s->stream));  // warm-up
  GP_CUDA(cudaEventRecord(e0, s->stream));
  for (int i = 0; i < reps; ++i) GP_CUDA(launch_sweeps(pl, s, s->stream));
  GP_CUDA(cudaEventRecord(e1, s->stream));
  GP_CUDA(cudaEventSynchronize(e1));
  GP_CUDA(cudaGetLastError());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GP_CUDA(cudaMemcpy(s->st_host, s->st_dev, sizeof(State), cudaMemcpyDeviceToHost));
  if (s->st_host->error & kErrTimeout) return fail(GPSPCA_ETIMEDOUT, "a device-side wait for a tile copy gave up");
  if (s->st_host->error & kErrLaunch) return fail(GPSPCA_ECUDA, "a sweep refused its launch geometry");
  if (s->st_host->n_active == 0) return fail(GPSPCA_EINVAL, "the start is degenerate or A is zero: nothing to time");
  *ms_per_sweep = static_cast<double>(ms) / reps;
  return GPSPCA_OK;
}

int gpspca_tune(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                const double* mu, uint32_t flags, int32_t reps, int32_t* n_candidates, double* ms_best,
                double* ms_default) {
  if (!ctx || !n_candidates || !ms_best || !ms_default)
    return fail(GPSPCA_EINVAL, "ctx and the result pointers must not be NULL");
  if (reps < 1) return fail(GPSPCA_EINVAL, "reps must be >= 1");
  gpspca_out dummy = {};
  dummy.location = GPSPCA_DEVICE;
  double one = 0.0;
  dummy.X = dummy.Z = dummy.objective = &one;  // replaced by staging buffers
  dummy.iters = dummy.status = reinterpret_cast<int32_t*>(&one);
  Request r;
  int rc = request_from(&r, A, form, gamma, m, mu, 0.0, 1 << 30, nullptr, flags, &dummy);
  if (rc != GPSPCA_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->solve_mu);
  GP_CUDA(cudaSetDevice(ctx->device));
  Slot* s = &ctx->sync_slot;
  if ((rc = wait_upload(ctx, s->stream, r.A)) != GPSPCA_OK) return rc;
  int nc = 0;
  double best = 0.0, def = 0.0;
  std::string best_key, shape;
  for (int c = 0; c == 0 || c < nc; ++c) {
    Plan pl;
    bool empty = false;
    rc = prepare_solve(s, r, ctx->nsm, true, &pl, &empty, c, c == 0 ? &nc : nullptr, c == 0 ? &shape : nullptr);
    if (rc == GPSPCA_ENOMEM && c > 0) continue;  // a candidate whose workspace does not fit the budget
    if (rc != GPSPCA_OK) return rc;
    if (empty) return fail(GPSPCA_EINVAL, "empty matrix");
    double ms = 0.0;
    if ((rc = time_plan(s, pl, reps, &ms)) != GPSPCA_OK) return rc;
    if (c == 0) def = ms;
    if (c == 0 || ms < best) {
      best = ms;
      best_key = pl.key();
    }
  }
  {
    std::lock_guard<std::mutex> tl(ctx->tune.mu);
    ctx->tune.best[shape] = {best_key, best};
    ctx->tune.resolved.erase(shape);
  }
  *n_candidates = nc;
  *ms_best = best;
  *ms_default = def;
  return GPSPCA_OK;
}

int gpspca_tune_save(gpspca_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(GPSPCA_EINVAL, "ctx and path must not be NULL");
  FILE* f = fopen(path, "w");
  if (!f) return fail(GPSPCA_EINVAL, "cannot write %s", path);
  fprintf(f, "gpspca-tune 1\n");
  {
    std::lock_guard<std::mutex> tl(ctx->tune.mu);
    for (const auto& kv : ctx->tune.best)
      fprintf(f, "%s\t%s\t%.6f\n", kv.first.c_str(), kv.second.first.c_str(), kv.second.second);
  }
  const bool ok = fclose(f) == 0;
  return ok ? GPSPCA_OK : fail(GPSPCA_EINVAL, "cannot write %s", path);
}

int gpspca_tune_load(gpspca_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(GPSPCA_EINVAL, "ctx and path must not be NULL");
  FILE* f = fopen(path, "r");
  if (!f) return fail(GPSPCA_ENOTFOUND, "cannot read %s", path);
  std::vector<std::pair<std::string, std::pair<std::string, double>>> rows;
  char line[4096];
  bool header = false, bad = false;
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    if (!header) {
      header = true;
      if (l != "gpspca-tune 1") {
        bad = true;
        break;
      }
      continue;
    }
    if (l.empty()) continue;
    const size_t t1 = l.find('\t'), t2 = t1 == std::string::npos ? t1 : l.find('\t', t1 + 1);
    if (t1 == std::string::npos || t2 == std::string::npos || t1 == 0 || t2 == t1 + 1) {
      bad = true;
      break;
    }
    char* end = nullptr;
    const double ms = strtod(l.c_str() + t2 + 1, &end);
    if (end == l.c_str() + t2 + 1) {
      bad = true;
      break;
    }
    rows.push_back({l.substr(0, t1), {l.substr(t1 + 1, t2 - t1 - 1), ms}});
  }
  fclose(f);
  if (bad || !header) return fail(GPSPCA_EINVAL, "%s is not a tuned-layout table", path);
  std::lock_guard<std::mutex> tl(ctx->tune.mu);
  for (auto& row : rows) {
    ctx->tune.best[row.first] = row.second;
    ctx->tune.resolved.erase(row.first);
  }
  return GPSPCA_OK;
}

int gpspca_submit(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                  const double* mu, double tol, int32_t maxit, uint32_t flags, gpspca_out* out, uint64_t* ticket) {
  if (!ctx || !ticket) return fail(GPSPCA_EINVAL, "ctx and ticket must not be NULL");
  auto t = std::make_unique<Ticket>();
  int rc = request_from(&t->req, A, form, gamma, m, mu, tol, maxit, nullptr, flags, out);
  if (rc != GPSPCA_OK) return rc;
  if ((rc = validate(t->req)) != GPSPCA_OK) return rc;
  if (A->location != GPSPCA_DEVICE || out->location != GPSPCA_DEVICE)
    return fail(GPSPCA_EINVAL, "gpspca_submit takes device buffers only");
  t->foot = request_footprint(t->req);
  if (t->foot > ctx->budget.limit)
    return fail(GPSPCA_ENOMEM, "request of %zu bytes (matrix and outputs) exceeds the context budget of %zu", t->foot,
                ctx->budget.limit);
  t->t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(ctx->q_mu);
  if (!ctx->sched_started) {
    cudaSetDevice(ctx->device);
    for (int i = 0; i < kServeSlots; ++i) {
      auto s = std::make_unique<Slot>();
      rc = slot_init(s.get(), ctx->device, nullptr, &ctx->budget, &ctx->tune);
      if (rc != GPSPCA_OK) return rc;
      ctx->serve_slots.push_back(std::move(s));
    }
    ctx->sched = std::thread(scheduler_main, ctx);
    ctx->sched_started = true;
  }
  const uint64_t id = ctx->next_ticket++;
  ctx->tickets[id] = std::move(t);
  ctx->queue.push_back(id);
  *ticket = id;
  ctx->q_cv.notify_all();
  return GPSPCA_OK;
}

int gpspca_poll(gpspca_ctx* ctx, uint64_t ticket, int32_t wait_us) {
  if (!ctx) return fail(GPSPCA_EINVAL, "ctx is NULL");
  std::unique_lock<std::mutex> lk(ctx->q_mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return fail(GPSPCA_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Ticket* t = it->second.get();
  auto ready = [&] { return t->done; };
  if (!t->done) {
    if (wait_us < 0)
      ctx->done_cv.wait(lk, ready);
    else if (wait_us > 0)
      ctx->done_cv.wait_for(lk, std::chrono::microseconds(wait_us), ready);
  }
  if (!t->done) return GPSPCA_PENDING;
  const int rc = t->rc;
  if (rc != GPSPCA_OK) t_last_error = t->msg;
  ctx->tickets.erase(it);
  return rc;
}

int gpspca_destroy(gpspca_ctx* ctx) {
  if (!ctx) return GPSPCA_OK;
  if (ctx->sched_started) {
    {
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      ctx->stop = true;
    }
    ctx->q_cv.notify_all();
    ctx->sched.join();
  }
  cudaSetDevice(ctx->device);
  for (auto& s : ctx->serve_slots) slot_free(s.get());
  for (auto& s : ctx->batch_slots) slot_free(s.get());
  for (auto& s : ctx->group_slots) slot_free(s.get());
  for (auto& kv : ctx->group_graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.g);
  }
  if (ctx->group_done) cudaEventDestroy(ctx->group_done);
  if (ctx->group_ptrs) cudaFree(ctx->group_ptrs);
  if (ctx->group_ptrs_host) cudaFreeHost(ctx->group_ptrs_host);
  for (cudaStream_t c : {ctx->group_cap2, ctx->group_cap, ctx->group_stream})
    if (c) cudaStreamDestroy(c);
  if (ctx->batch_start) cudaEventDestroy(ctx->batch_start);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  for (gpspca_ctx::Upload& u : ctx->uploads) cudaEventDestroy(u.done);
  if (ctx->up_tail) cudaEventDestroy(ctx->up_tail);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (DevBuf& b : ctx->batch_stage) release(&ctx->sync_slot, &b);
  for (DevBuf& b : ctx->batch_norms) release(&ctx->sync_slot, &b);
  slot_free(&ctx->sync_slot);
  delete ctx;
  return GPSPCA_OK;
}

}  // extern "C"
