// Instantiations of the tiled spread kernel for float (one translation unit per
// kernel and precision so the build compiles them in parallel).
#include "points_tiled.cuh"

namespace gbnfft {

#define GBNFFT_CASE(D, W, R) \
  case (D) * 100 + (W):      \
    return reinterpret_cast<const void*>(&k_spread_tiled<D, W, R>);

const void* spread_tiled_kernel_f32(int d, int taps) {
  switch (d * 100 + taps) {
    GBNFFT_TAPS_1_2(GBNFFT_CASE, 1, float)
    GBNFFT_TAPS_1_2(GBNFFT_CASE, 2, float)
    GBNFFT_TAPS_3(GBNFFT_CASE, 3, float)
    default:
      return nullptr;
  }
}

}  // namespace gbnfft
