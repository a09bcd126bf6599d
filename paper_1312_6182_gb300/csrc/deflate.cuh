// Host launchers of the deflation kernels (deflate.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpspca {

// Column stride of the working copy: p rounded up to 16 bytes.
int64_t deflate_ld(int dtype, int64_t p);
// W (working type: double for GPSPCA_F64, float otherwise; ldw x n) = A,
// fp8 entries times their column scale; rows p..ldw-1 zero.
void launch_deflate_copy(int dtype, const void* A, int64_t ld, const float* scale, void* W, int64_t ldw, int64_t p,
                         int64_t n, cudaStream_t s);
// Device bytes of the support list launch_deflate needs for n entries.
size_t deflate_list_bytes(int dtype, int64_t n);
// W <- W - (W z) z^T, touching only the columns where z (n entries, the
// working type) is nonzero; list: deflate_list_bytes of device scratch.
// dtype: GPSPCA_F64 (double W, z) or any other (float).
void launch_deflate(int dtype, void* W, int64_t ldw, int64_t p, int64_t n, const void* z, void* list,
                    cudaStream_t s);

// S[:, j] = B z_j for j < m: B (q x n, column-major, ld; dtype as the
// matrix descriptor, fp8 with its column scales), Z (n x m, ld n) and S
// (q x m, ld q) in the working type (double for GPSPCA_F64, float
// otherwise), all device memory; reads only the support columns of each z_j.
// list: m * deflate_list_bytes(dtype, n) of device scratch (one support
// list per column).
void launch_project(int dtype, const void* B, int64_t ld, const float* scale, int64_t q, int64_t n, const void* Z,
                    int m, void* S, void* list, cudaStream_t s);

}  // namespace gpspca
