// Instantiations of the fused sweep that also forms the column norms (the
// block start's first power step), for A stored as float, full-width tiles
// (every tile slot run without a width test).
#include "sweep.cuh"

namespace gpspca {

#define GPSPCA_K(MG, NCH) \
  case MG * 10 + NCH:     \
    return sweep_kernel_ptr<float, MG, NCH, true, sweep_kb(MG) / (MG + 1)>();

// fw: the tile width the pass runs; nullptr unless it is the variant's width
const void* sweep_kernel_f32_nrm_full(int mg, int nch, int fw) {
  if (fw != sweep_kb(mg) / (mg + 1)) return nullptr;
  switch (mg * 10 + nch) {
    GPSPCA_K(1, 1) GPSPCA_K(1, 2) GPSPCA_K(1, 3) GPSPCA_K(1, 4)
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
