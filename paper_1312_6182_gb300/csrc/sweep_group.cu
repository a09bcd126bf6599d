// Instantiations of the grouped single-unit sweep (one pass, one component
// per instance, clusters of one CTA) for every storage type.
#include "sweep.cuh"

namespace gpspca {

// nch: rows-per-thread chunks of the pass; nullptr where no such variant exists
const void* sweep_kernel_grouped_su(int dtype, int nch) {
  switch (dtype * 10 + nch) {
    case GPSPCA_F32 * 10 + 1: return sweep_kernel_grouped_ptr<float, 1, 1>();
    case GPSPCA_F32 * 10 + 2: return sweep_kernel_grouped_ptr<float, 1, 2>();
    case GPSPCA_F32 * 10 + 3: return sweep_kernel_grouped_ptr<float, 1, 3>();
    case GPSPCA_F32 * 10 + 4: return sweep_kernel_grouped_ptr<float, 1, 4>();
    case GPSPCA_F64 * 10 + 1: return sweep_kernel_grouped_ptr<double, 1, 1>();
    case GPSPCA_F64 * 10 + 2: return sweep_kernel_grouped_ptr<double, 1, 2>();
    case GPSPCA_F64 * 10 + 3: return sweep_kernel_grouped_ptr<double, 1, 3>();
    case GPSPCA_F64 * 10 + 4: return sweep_kernel_grouped_ptr<double, 1, 4>();
    case GPSPCA_BF16 * 10 + 1: return sweep_kernel_grouped_ptr<__nv_bfloat16, 1, 1>();
    case GPSPCA_BF16 * 10 + 2: return sweep_kernel_grouped_ptr<__nv_bfloat16, 1, 2>();
    case GPSPCA_BF16 * 10 + 3: return sweep_kernel_grouped_ptr<__nv_bfloat16, 1, 3>();
    case GPSPCA_BF16 * 10 + 4: return sweep_kernel_grouped_ptr<__nv_bfloat16, 1, 4>();
    case GPSPCA_FP8_E4M3 * 10 + 1: return sweep_kernel_grouped_ptr<__nv_fp8_e4m3, 1, 1>();
    case GPSPCA_FP8_E4M3 * 10 + 2: return sweep_kernel_grouped_ptr<__nv_fp8_e4m3, 1, 2>();
    case GPSPCA_FP8_E4M3 * 10 + 3: return sweep_kernel_grouped_ptr<__nv_fp8_e4m3, 1, 3>();
    case GPSPCA_FP8_E4M3 * 10 + 4: return sweep_kernel_grouped_ptr<__nv_fp8_e4m3, 1, 4>();
    default: return nullptr;
  }
}

}  // namespace gpspca
