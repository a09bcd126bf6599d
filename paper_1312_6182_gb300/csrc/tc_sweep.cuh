// The wide sweep on the 5th-generation tensor cores (tcgen05): for many
// components (or gamma values; the planner's crossover is m >= 6 for bf16
// storage and for float storage read in place, m >= 9 otherwise), one power
// iteration is two tall-skinny
// contractions over A,
//
//   T = A^T X   (n x m; then the Table 1 threshold gives G, per entry)
//   Y = A G     (p x m),
//
// the same three steps as the fused CUDA-core sweep (column sweep,
// threshold, rank update), with the dot products and the rank update on the
// tensor cores.  A (bf16) streams through shared memory by TMA in 128-byte
// swizzled tiles; one thread issues tcgen05.mma, accumulators live in tensor
// memory and are read back with tcgen05.ld.
//
// Accuracy: X and G are float; each is split into three bf16 parts
// (x = x0 + x1 + x2 exactly, 24 significant bits), laid side by side as the
// N = 3 mpad columns of one MMA, so the tensor cores form A x0, A x1, A x2 in
// float accumulators and the epilogue adds them (x0 + (x1 + x2)): the
// products are those of float X against the stored A.  A float A is split
// the same way once per solve into three bf16 planes (a0 + a1 + a2 = a
// exactly), whose MMAs go into the same accumulator smallest plane first;
// fp8 values are exact in bf16 (one plane) with the column scale applied in
// the epilogue.  Each 64-deep chunk's accumulator is drained into registers
// (IEEE float adds), so the sum keeps float accuracy for any p or n.
//
// Why two passes and not one: the rank update's accumulator Y (p x 3 mpad
// floats) must stay in tensor memory (256 KB per SM) across every column
// tile of a CTA's share of A; for the shapes that need this path (many
// components, p in the thousands) it does not fit, while T's accumulator (128 columns x
// 3 mpad) always does.  Each pass reads A once, at tensor-core rate instead
// of CUDA-core rate.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace gpspca {

constexpr int kTcThreads = 192;  // warps 0-3: epilogue (tensor-memory lanes 0-127), 4: TMA, 5: MMA
constexpr int kTcBK = 64;        // elements of the reduction dimension per stage (one 128-byte row)
constexpr int kTcTile1 = 128;    // columns of A per T-pass tile (the MMA's M)
constexpr int kTcRows2 = 128;    // rows of A per Y-pass block (the MMA's M)

// TMA descriptors of one solve (device memory, refreshed by the host before
// each solve).
struct TcMaps {
  CUtensorMap a1[3];  // bf16 planes of A, box 64 rows x 128 columns (T pass)
  CUtensorMap x3;     // X3^T, box 64 x N
  CUtensorMap a2[3];  // bf16 planes of A, box 64 rows x 64 columns (Y pass)
  CUtensorMap g3;     // G3^T, box 64 x N
  CUtensorMap a1f;    // float A, box 32 rows x 128 columns (fused T pass)
  CUtensorMap a2f;    // float A, box 32 rows x 64 columns (fused Y pass)
  CUtensorMap a2g;    // float A, box 128 rows x 1 column, no swizzle (fused Y pass, gathered columns: tile::gather4)
  CUtensorMap g3c;    // G3c^T (the active columns' G3), box 64 x N
};

constexpr int kTcMaxSplit1 = 8;  // T pass: at most this many row ranges per column tile
constexpr int kTcCompactCols = 256;  // columns per block of the active-column list kernels (one per thread)
// the Y pass runs over the listed columns while they are at most this
// fraction (in tenths) of n, and over all columns otherwise
constexpr int kTcSparseTenths = 6;

struct TcArgs {
  const IO* io;
  State* st;
  int p, n, m, mpad, form, sketch;
  int na;             // bf16 planes of A: 1 (bf16 storage, or the fp8 values), 3 (float A = a0 + a1 + a2)
  int fused;          // float A read as float by TMA and split into its 3 planes in shared memory
  int scaled;         // fp8 storage: a_i = s_i q_i, the column scale applied to t and g
  int p_pad, n_pad;   // row strides (elements) of X3^T and G3^T
  int ntile1;         // ceil(n / 128)
  int kchunks1;       // ceil(p / 64)
  int ksplit1;        // T pass: row ranges per column tile (partial T summed by a combine step when > 1)
  int kcs1;           // 64-row chunks per row range
  int nchunks2;       // ceil(n / 64)
  int kps2;           // 64-column chunks per Y-pass split
  int nsplit2;        // Y-pass splits of the columns
  int nrow2;          // ceil(p / 128)
  int sparse;         // Y pass over the active columns only (threshold sweeps, not the start)
  int norms;          // fused float T pass also sums the columns' squared norms (the start's first step)
  int keep_t;         // start: the T pass writes T = A^T Q to io->T (the Rayleigh-Ritz step's T^T T)
  int64_t yld;        // bf16 planes: column stride (elements) of the planes the Y pass reads
  int from_ritz;      // first sweep after the block start: T = (A^T Q) R from the kept T, no T pass
};

// Host side (tc_sweep.cu).
int tc_smem_bytes(int npad, int na);
bool tc_supported(int device);
// planes: na bf16 matrices (p x n, column stride ld elements, `plane` elements apart)
int tc_encode_maps(TcMaps* maps, const void* planes, int na, int64_t plane, int64_t p, int64_t n, int64_t ld,
                   const void* x3, int p_pad, const void* g3, int n_pad, int npad, const void* g3c);
// float A read in place by the fused passes (16-byte aligned base, ld % 4 == 0)
int tc_encode_maps_f32(TcMaps* maps, const void* A, int64_t p, int64_t n, int64_t ld, const void* x3, int p_pad,
                       const void* g3, int n_pad, int npad, const void* g3c);
int tc_fused_smem_bytes(int npad);
// float / fp8 / unaligned bf16 A -> bf16 planes in the workspace (once per
// solve); ldc = p_pad
void launch_tc_convert(int dtype, const IO* io, int64_t p, int64_t n, int64_t ld, int64_t ldc, cudaStream_t s);
void launch_tc_sweep(const TcArgs& a, int npad, cudaStream_t s, bool t_only = false);
// CTAs of the T pass resident per SM (1 or 2) for a geometry.
int tc_t_ctas_per_sm(int npad, int na, bool fused);

}  // namespace gpspca
