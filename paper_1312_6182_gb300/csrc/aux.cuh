// Per-solve kernels around the fused sweep: state reset, column norms and the
// start (step a0), deterministic reduction of the sweep partials with the
// Gram matrix of Y, the FP64 finish step (objective, stopping test, polar
// weights via a Jacobi eigensolve), and the recovery of the loadings.
#pragma once

#include "smalleig.cuh"
#include "sweep.cuh"

namespace gpspca {

struct ReduceArgs {
  const IO* io;
  State* st;
  int nsplit;         // partials in io->ypart (or the start io->P when init)
  int m, p;
  int full_gram;      // 1: all j <= l pairs (block forms); 0: diagonal only
  int npairs;
  int init;           // 1: the partials are the start directions io->P (nsplit = 1)
  int cross;          // 1: no Y update; Gram partials of (old Y, new Y) pairs, m*m
  int objective;      // 1: also the Table 1 objective partials from io->T (n entries, form)
  int n, form;
  int nyb;            // blocks summing Y rows (kReduceRows each)
  int nobj;           // blocks forming objective partials (after the Y blocks), when objective
};

struct FinishArgs {
  const IO* io;
  State* st;
  int nsplit;  // objective partial sets in io->fpart (one per objective block)
  int nblk;    // Gram partials in io->gpart
  int npairs;
  int m, form;
  int mode;  // kFinishIterate, kFinishPolar (project the start), kFinishRitz / kFinishRitzT (rotate the start)
  int last;  // 1: the start is complete after this step (sweep counter k = 0)
  cudaGraphConditionalHandle cond;
  int use_cond;
};

enum : int { kFinishIterate = 0, kFinishPolar = 1, kFinishRitz = 2, kFinishRitzT = 3 };

// Fixed sketch of the block start: SplitMix64 (Steele, Lea & Flood 2014),
// entry (r, j) = sign from the top bit of output k = j * 2^32 + r + 1 of the
// stream seeded with kSketchSeed.
constexpr unsigned long long kSketchSeed = 0x5EED5EED5EED5EEDull;
constexpr int kPowerSteps = 2;

struct StartArgs {
  const IO* io;
  State* st;
  int64_t ld;
  int p, n, m, form;
};

constexpr int kReduceRows = 32;   // rows per reduction block
constexpr int kReduceGroups = 8;  // partial groups per reduction block
constexpr int kFinishThreads = 256;
constexpr int kFinishMaxSmem = 220 * 1024;  // dynamic shared memory of finish_kernel (m = 64 needs ~195 KB)
constexpr int kStartThreads = 1024;
constexpr int kMaxCandidates = 256;

// Shared memory (in 8-byte slots) of finish_kernel for m components and
// npairs Gram entries: partial sums, objective parts, weights, eigensolver
// workspace.
inline int finish_smem_doubles(int m, int npairs) { return npairs + 2 * m + m * m + eig_ws_slots(m); }

// Host-side launchers (each kernel is launched from the file that defines it).
void launch_reset(const IO* io, State* st, int m, int form, cudaStream_t s);
void launch_colnorm(int dtype, const IO* io, State* st, int64_t ld, int p, int n, int fast, cudaStream_t s);
// the column norms of a matrix that several solves of a batch share, once,
// into out (n doubles; error collects kErrNonFinite)
void launch_colnorm_shared(int dtype, const void* A, const float* col_scale, double* out, int32_t* error,
                           int64_t ld, int p, int n, int fast, cudaStream_t s);
// a solve's column norms copied from io->cnorm_src, with the non-finite check
void launch_copy_norms(const IO* io, State* st, int n, cudaStream_t s);
void launch_select_start(int dtype, const StartArgs& a, cudaStream_t s);
void launch_gather_start(int dtype, const StartArgs& a, cudaStream_t s);
void launch_reduce(int tcsize, const ReduceArgs& a, cudaStream_t s);
void launch_finish(const FinishArgs& a, int smem, cudaStream_t s);
void launch_finalize(int tcsize, const IO* io, const State* st, int p, int n, int m, int form, cudaStream_t s);
void launch_form_x(int tcsize, const IO* io, const State* st, int p, int m, cudaStream_t s);
// T^T T of the float T = A^T Q in io->T ([m][n]) as Gram partials (gpart,
// [blocks][m*m], full), for the start's Rayleigh-Ritz rotation.
constexpr int kGramTCols = 256;  // columns of T per block
inline int gram_t_blocks(int64_t n) { return static_cast<int>((n + kGramTCols - 1) / kGramTCols); }
void launch_gram_t(const IO* io, const State* st, int m, int n, cudaStream_t s);

// The same steps for a group of `count` same-shape solves, one launch each
// (grid z = instance; the IO and State pointers of `a` are replaced by the
// group's); the loop condition of a group: any instance still active.
void launch_reset_g(GroupPtrs g, int count, int m, int form, cudaStream_t s);
void launch_colnorm_g(int dtype, GroupPtrs g, int count, int64_t ld, int p, int n, int fast, cudaStream_t s);
void launch_select_start_g(int dtype, const StartArgs& a, GroupPtrs g, int count, cudaStream_t s);
void launch_gather_start_g(int dtype, const StartArgs& a, GroupPtrs g, int count, cudaStream_t s);
void launch_reduce_g(int tcsize, const ReduceArgs& a, GroupPtrs g, int count, cudaStream_t s);
void launch_finish_g(const FinishArgs& a, int smem, GroupPtrs g, int count, cudaStream_t s);
void launch_finalize_g(int tcsize, GroupPtrs g, int count, int p, int n, int m, int form, cudaStream_t s);
void launch_group_cond(GroupPtrs g, int count, cudaGraphConditionalHandle h, cudaStream_t s);

}  // namespace gpspca
