// Per-solve kernels around the fused sweep: state reset, column norms and the
// start (step a0), deterministic reduction of the sweep partials with the
// Gram matrix of Y, the FP64 finish step (objective, stopping test, polar
// weights via a Jacobi eigensolve), and the recovery of the loadings.
#pragma once

#include "sweep.cuh"

namespace gpspca {

struct ReduceArgs {
  const IO* io;
  State* st;
  int nsplit;         // partials in io->ypart (or the start io->P when init)
  int m, p;
  int full_gram;      // 1: all j <= l pairs (block forms); 0: diagonal only
  int npairs;
  int init;           // 1: reducing the start (runs even before the state is active)
};

struct FinishArgs {
  const IO* io;
  State* st;
  int nsplit;  // objective partials in io->fpart
  int nblk;    // Gram partials in io->gpart
  int npairs;
  int m, form, init;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

struct StartArgs {
  const IO* io;
  State* st;
  int64_t ld;
  int p, n, m, form;
};

constexpr int kReduceRows = 32;   // rows per reduction block
constexpr int kReduceGroups = 8;  // partial groups per reduction block
constexpr int kFinishThreads = 256;
constexpr int kStartThreads = 1024;
constexpr int kMaxCandidates = 256;

// Host-side launchers (each kernel is launched from the file that defines it).
void launch_reset(const IO* io, State* st, int m, int form, cudaStream_t s);
void launch_colnorm(int dtype, const IO* io, State* st, int64_t ld, int p, int n, int fast, cudaStream_t s);
void launch_select_start(int dtype, const StartArgs& a, cudaStream_t s);
void launch_gather_start(int dtype, const StartArgs& a, cudaStream_t s);
void launch_reduce(int tcsize, const ReduceArgs& a, int nblk, cudaStream_t s);
void launch_finish(const FinishArgs& a, int smem, cudaStream_t s);
void launch_finalize(int tcsize, const IO* io, const State* st, int p, int n, int m, int form, cudaStream_t s);

}  // namespace gpspca
