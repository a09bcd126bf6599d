// Instantiations of the fused sweep for A stored as float with fixed-width
// tiles (every tile slot run without a width test): for two or more
// components the variant's full width; one component at any width (in
// sweep_f32_full1.cu).
#include "sweep.cuh"

namespace gpspca {

const void* sweep_kernel_f32_full1(int nch, int fw);

#define GPSPCA_K(MG, NCH) \
  case MG * 10 + NCH:     \
    return sweep_kernel_ptr<float, MG, NCH, false, sweep_kb(MG) / MG>();

// fw: the tile width the pass runs; nullptr where no such variant exists
const void* sweep_kernel_f32_full(int mg, int nch, int fw) {
  if (mg == 1) return sweep_kernel_f32_full1(nch, fw);
  if (fw != sweep_kb(mg) / mg) return nullptr;
  switch (mg * 10 + nch) {
    GPSPCA_K(2, 1) GPSPCA_K(2, 2) GPSPCA_K(2, 3) GPSPCA_K(2, 4)
    GPSPCA_K(4, 1) GPSPCA_K(4, 2) GPSPCA_K(4, 3) GPSPCA_K(4, 4)
    GPSPCA_K(5, 1) GPSPCA_K(5, 2) GPSPCA_K(5, 3) GPSPCA_K(5, 4)
    GPSPCA_K(8, 1) GPSPCA_K(8, 2) GPSPCA_K(8, 3) GPSPCA_K(8, 4)
    default:
      return nullptr;
  }
}

#undef GPSPCA_K

}  // namespace gpspca
