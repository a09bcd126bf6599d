// Instantiations of the fused sweep for A stored as float with fixed-width
// tiles (every tile slot run without a width test), two components, tile widths 9-16.
#include "sweep.cuh"

namespace gpspca {

#define GPSPCA_K(NCH, FW) \
  case NCH * 100 + FW:    \
    return sweep_kernel_ptr<float, 2, NCH, false, FW>();

const void* sweep_kernel_f32_full2b(int nch, int fw) {
  switch (nch * 100 + fw) {
    GPSPCA_K(1, 9) GPSPCA_K(1, 10) GPSPCA_K(1, 11) GPSPCA_K(1, 12) GPSPCA_K(1, 13) GPSPCA_K(1, 14) GPSPCA_K(1, 15) GPSPCA_K(1, 16)
    GPSPCA_K(2, 9) GPSPCA_K(2, 10) GPSPCA_K(2, 11) GPSPCA_K(2, 12) GPSPCA_K(2, 13) GPSPCA_K(2, 14) GPSPCA_K(2, 15) GPSPCA_K(2, 16)
    GPSPCA_K(3, 9) GPSPCA_K(3, 10) GPSPCA_K(3, 11) GPSPCA_K(3, 12) GPSPCA_K(3, 13) GPSPCA_K(3, 14) GPSPCA_K(3, 15) GPSPCA_K(3, 16)
    GPSPCA_K(4, 9) GPSPCA_K(4, 10) GPSPCA_K(4, 11) GPSPCA_K(4, 12) GPSPCA_K(4, 13) GPSPCA_K(4, 14) GPSPCA_K(4, 15) GPSPCA_K(4, 16)
    default:
      return nullptr;
  }
}

#undef GPSPCA_K

}  // namespace gpspca
