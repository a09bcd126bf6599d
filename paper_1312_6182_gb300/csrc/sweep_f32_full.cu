// The fixed-width float sweeps (every tile slot run without a width test):
// dispatch by component count and tile width to the instantiation files.
#include "sweep.cuh"

namespace gpspca {

const void* sweep_kernel_f32_full1(int nch, int fw);
const void* sweep_kernel_f32_full2a(int nch, int fw);
const void* sweep_kernel_f32_full2b(int nch, int fw);
const void* sweep_kernel_f32_full4(int nch, int fw);
const void* sweep_kernel_f32_full5(int nch, int fw);
const void* sweep_kernel_f32_full8(int nch, int fw);

// fw: the tile width the pass runs; nullptr where no such variant exists
const void* sweep_kernel_f32_full(int mg, int nch, int fw) {
  if (fw < 1 || fw > sweep_kb(mg) / mg) return nullptr;
  switch (mg) {
    case 1: return sweep_kernel_f32_full1(nch, fw);
    case 2: return fw <= 8 ? sweep_kernel_f32_full2a(nch, fw) : sweep_kernel_f32_full2b(nch, fw);
    case 4: return sweep_kernel_f32_full4(nch, fw);
    case 5: return sweep_kernel_f32_full5(nch, fw);
    case 8: return sweep_kernel_f32_full8(nch, fw);
    default: return nullptr;
  }
}

}  // namespace gpspca
