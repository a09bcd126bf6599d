// Launch plan of one solve (chosen by the engine from the kernels' register
// and shared-memory needs); shared by the entry points of the library.
#pragma once

#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

namespace gpspca {

struct Pass {
  int j0, mgv, mg, nch, threads, W, S, smem;
  const void* k;
  int ov = 0;  // overlapped tiles (phase A of tile t+1 before phase B of tile t)
};

struct Plan {
  int dtype = 0, form = 0, m = 0, p = 0, n = 0;
  int64_t ld = 0;
  int fast = 0;
  int pca = 0;  // block start by power steps + Rayleigh-Ritz (no caller x0)
  int C = 1, ps = 0, ncl = 0, cols_per_cl = 0;
  std::vector<Pass> passes;
  // block start: the first power step's pass with the column norms (its
  // first pass of components; the others as in `passes`)
  Pass norm_pass{};
  int norms_in_sweep = 0;
  // the column norms come from a pass the batch made once for several
  // solves of this matrix (copied in the prologue instead of computed)
  int norms_given = 0;
  int nred = 0, nobj = 0, npairs = 0, full_gram = 0;
  int finish_smem = 0;
  int tcsize = 4, esize = 4;
  // tensor-core wide sweep (tc_sweep.cuh) instead of the CUDA-core passes
  int tc = 0, mpad = 0, npad = 0, p_pad = 0, n_pad = 0, ntile1 = 0, kchunks1 = 0, nchunks2 = 0, kps2 = 0,
      nsplit2 = 0, nrow2 = 0;
  int tc_na = 1;       // bf16 planes of A the contractions read (3 for float A)
  int tc_convert = 0;  // the planes are a workspace copy made once per solve (float / fp8 A)
  int tc_fused = 0;    // float A read in place, split into planes in shared memory
  int tc_sparse = 0;   // fused Y pass of threshold sweeps over the active columns only
  int ksplit1 = 1, kcs1 = 0;  // T pass: row ranges per column tile, 64-row chunks per range
  size_t ws_cnorm = 0, ws_P = 0, ws_ypart = 0, ws_T = 0, ws_fpart = 0, ws_gpart = 0, ws_x3 = 0, ws_g3 = 0,
         ws_planes = 0, ws_tpart = 0, ws_sparse = 0, ws_Xf = 0;

  std::string key() const {
    char b[256];
    snprintf(b, sizeof(b), "%d/%d/%d/%d/%d/%lld/%d/%d/%d/%d/%d/%d", dtype, form, m, p, n, (long long)ld, fast, pca, C,
             ps, ncl, cols_per_cl);
    std::string s(b);
    if (tc) {
      snprintf(b, sizeof(b), "|tc%d,%d,%d,%d,%d,%d,%d", npad, kps2, nsplit2, tc_na, tc_convert, tc_fused, ksplit1);
      s += b;
    }
    for (const Pass& q : passes) {
      snprintf(b, sizeof(b), "|%d,%d,%d,%d,%d,%d,%d%s", q.j0, q.mgv, q.mg, q.nch, q.threads, q.W, q.S,
               q.ov ? "o" : "");
      s += b;
    }
    if (norms_in_sweep) {
      snprintf(b, sizeof(b), "|n%d,%d,%d,%d", norm_pass.nch, norm_pass.threads, norm_pass.W, norm_pass.S);
      s += b;
    }
    if (norms_given) s += "|ng";
    return s;
  }
  size_t workspace_bytes() const {
    return ws_cnorm + 2 * ws_P + ws_Xf + ws_ypart + ws_T + ws_fpart + ws_gpart + ws_x3 + ws_g3 + ws_planes +
           ws_tpart + ws_sparse + 14 * 256 + 1024;
  }
};

// Layout of the buffers of the fused float tensor-core sweep (one
// allocation): the listed-column rank update's flags [n64] bytes | list
// [n64] int32 | count | per-block counts [ceil(n / 256)] int32 | G3c
// [npad][n64] bf16, and the start's squared column norms [n] double, each
// 256-aligned.
struct SparseLayout {
  size_t act, list, nlist, cnt, g3c, nsq, total;
};
inline SparseLayout sparse_layout(int64_t n, int npad) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t n64 = static_cast<size_t>((n + 63) / 64 * 64);
  SparseLayout L;
  L.act = 0;
  L.list = up(n64);
  L.nlist = L.list + up(4 * n64);
  L.cnt = L.nlist + 256;
  L.g3c = L.cnt + up(4 * static_cast<size_t>((n + 255) / 256));
  L.nsq = L.g3c + up(2 * static_cast<size_t>(npad) * n64);
  L.total = L.nsq + up(8 * static_cast<size_t>(n));
  return L;
}

// Plan a solve: cluster size, per-pass kernel variant, threads, tile ring;
// or, with allow_tc and a wide problem, the tensor-core sweep.  cand < 0:
// the planner's default; cand >= 0: candidate layout `cand` of the list the
// autotuner times (0 is the default; *ncand receives the list's length).
int make_plan(int dt, int form, int m, int64_t p, int64_t n, int64_t ld, bool fast, int nsm, Plan* P,
              bool allow_tc = false, int cand = -1, int* ncand = nullptr);

// Record `msg` as the calling thread's last error (gpspca_last_error) and return code.
int record_error(int code, const char* msg);

}  // namespace gpspca
