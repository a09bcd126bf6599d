// Instantiations of the fused sweep for A stored as float with fixed-width
// tiles (every tile slot run without a width test), one component, tile widths 1-8 (a single-unit
// pass's width follows the column length).
#include "sweep.cuh"

namespace gpspca {

#define GPSPCA_K(NCH, FW) \
  case NCH * 100 + FW:    \
    return sweep_kernel_ptr<float, 1, NCH, false, FW>();

const void* sweep_kernel_f32_full1(int nch, int fw) {
  switch (nch * 100 + fw) {
    GPSPCA_K(1, 1) GPSPCA_K(1, 2) GPSPCA_K(1, 3) GPSPCA_K(1, 4) GPSPCA_K(1, 5) GPSPCA_K(1, 6) GPSPCA_K(1, 7) GPSPCA_K(1, 8)
    GPSPCA_K(2, 1) GPSPCA_K(2, 2) GPSPCA_K(2, 3) GPSPCA_K(2, 4) GPSPCA_K(2, 5) GPSPCA_K(2, 6) GPSPCA_K(2, 7) GPSPCA_K(2, 8)
    GPSPCA_K(3, 1) GPSPCA_K(3, 2) GPSPCA_K(3, 3) GPSPCA_K(3, 4) GPSPCA_K(3, 5) GPSPCA_K(3, 6) GPSPCA_K(3, 7) GPSPCA_K(3, 8)
    GPSPCA_K(4, 1) GPSPCA_K(4, 2) GPSPCA_K(4, 3) GPSPCA_K(4, 4) GPSPCA_K(4, 5) GPSPCA_K(4, 6) GPSPCA_K(4, 7) GPSPCA_K(4, 8)
    default:
      return nullptr;
  }
}

#undef GPSPCA_K

}  // namespace gpspca
