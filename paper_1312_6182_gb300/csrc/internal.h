// Internal types shared by the kernels and the host engine of libgpspca.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dd.cuh"
#include "gpspca.h"

namespace gpspca {

constexpr int kMaxM = GPSPCA_MAX_M;

// Per-call inputs that change between calls with the same launch geometry.
// The host writes one IO record into device memory before each graph launch,
// so a cached CUDA graph can be replayed for new buffers and parameters.
struct IO {
  const void* A;           // device pointer to A (p x n, column-major, ld)
  const float* col_scale;  // FP8: per-column scale
  const void* x0;          // optional start (device), p x m
  void* X;                 // outputs (device)
  void* Z;
  uint32_t* support;
  double* objective;
  int32_t* iters;
  int32_t* status;
  double* gamma_abs;
  // library workspace (device)
  double* cnorm;  // n approximate column norms
  const double* cnorm_src;  // the same, computed once for the batch's solves of this matrix (or null)
  void* P;        // [m][p] start directions
  void* Y;        // [m][p] last unnormalised direction
  void* Xf;       // [m][p] block forms on the CUDA cores: the iterate X = Y W the next sweep evaluates
  void* ypart;    // [nsplit][m][p] per-cluster partials of Y = A G
  void* T;        // [m][n] dot products of the last sweep
  dd* fpart;      // [nobj][2][m] objective / loading-norm partials (double-float)
  double* gpart;  // [nred][npairs] Gram partials
  void* tc_x3;    // tensor-core path: [3 mpad][p_pad] bf16 split of the iterate X (transposed)
  void* tc_g3;    // tensor-core path: [3 mpad][n_pad] bf16 split of the gradient factors G (transposed)
  const void* tc_maps;  // tensor-core path: the TMA tensor maps of A, X3 and G3 (TcMaps)
  void* tc_planes;      // tensor-core path: bf16 planes of a float / fp8 A ([na][n][p_pad])
  void* tc_tpart;       // tensor-core path: T partials of the row ranges ([ksplit][mpad][n_pad] float)
  // tensor-core path, rank update over the active columns only (columns i
  // with some G_ij != 0; the others add nothing to Y = A G)
  uint8_t* tc_act;      // [n_pad] 1 where column i is active in this sweep (cleared once listed)
  int32_t* tc_list;     // [n64] the active columns in increasing order, padded to a multiple of 64
  int32_t* tc_nlist;    // their count
  int32_t* tc_cnt;      // [ceil(n / 256)] active columns per block of 256
  void* tc_g3c;         // [3 mpad][n_pad] bf16: the G3 columns of the listed columns, zero past the count
  double* tc_nsq;       // [n] squared column norms summed by the block start's first T pass
  double gamma_in[kMaxM];  // as passed (absolute, or relative with the flag)
  double mu[kMaxM];
  double tol;
  int32_t maxit;
  int32_t gamma_relative;
  int32_t has_x0;
  int32_t pad_;
};

// Error bits in State::error.
enum : int32_t { kErrNonFinite = 1, kErrTimeout = 2, kErrLaunch = 4 };

// Device-resident state of one solve.
struct State {
  int32_t k;       // sweeps completed (-1 before the start is projected)
  int32_t n_active;
  int32_t error;   // kErr* bits
  int32_t any_degenerate;
  int32_t active[kMaxM];
  int32_t status[kMaxM];
  int32_t iters[kMaxM];
  double gamma[kMaxM];  // absolute gamma used on the device
  double f_prev[kMaxM];
  double f[kMaxM];
  double znorm2[kMaxM];  // squared norm of the unnormalised loading column of the last sweep
  double W[kMaxM * kMaxM];  // projection weights: X_k = Y_{k-1} W, [l * m + j]
  double R[kMaxM * kMaxM];  // the block start's Rayleigh-Ritz rotation: X_0 = Q R, [k * m + j]
  dd V[kMaxM * kMaxM];      // eigenvectors of the last Gram matrix, double-float (warm start of the next eigensolve)
  int32_t has_v;
  double cmax;              // max_i ||a_i||
  int32_t start_cols[kMaxM];
};

// A group of same-shape solves launched together (grid z = instance): the
// device arrays of the instances' IO and State.
struct GroupPtrs {
  const IO* const* io;
  State* const* st;
};

// Launch geometry of the fused sweep (host-chosen).
struct SweepGeom {
  int C;       // cluster size: CTAs splitting the rows of a column slab
  int ncl;     // clusters (column slabs)
  int threads; // per CTA
  int nch;     // row chunks per thread (template)
  int mg;      // components per pass (template)
  int ps;      // rows per CTA (multiple of the vector and TMA alignment)
  int W;       // columns per pipeline stage
  int S;       // pipeline stages
  int cols_per_cl;
  int smem;    // dynamic shared memory bytes
  int fast;    // 1: bulk-copy (TMA) loads; 0: element-wise loads
};

// Arguments of one sweep pass (components j0 .. j0+mg_valid-1).
struct SweepArgs {
  const IO* io;
  State* st;
  int64_t ld;
  int p, n, m;
  int form;
  int j0, mg_valid;
  int ps, W, S, cols_per_cl, fast;
  int sketch;  // 1: power step of the block start (no threshold, no outputs)
  int overlap; // 1: phase A of tile t+1 before phase B of tile t
};

}  // namespace gpspca
