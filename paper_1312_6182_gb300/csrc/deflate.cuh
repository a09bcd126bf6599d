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

}  // namespace gpspca
