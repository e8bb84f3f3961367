// Instantiations of the warp-per-point kernels for float.
#include "points_wpp.cuh"

namespace gbnfft {

#define GBNFFT_WPP_SPREAD(D, W, R) \
  case (D) * 100 + (W):            \
    return reinterpret_cast<const void*>(&k_spread_wpp<D, W, R>);
#define GBNFFT_WPP_INTERP(D, W, R) \
  case (D) * 100 + (W):            \
    return reinterpret_cast<const void*>(&k_interp_wpp<D, W, R>);

const void* wpp_kernel_f32(int d, int taps, bool spread) {
  if (spread) {
    switch (d * 100 + taps) {
      GBNFFT_WPP_TAPS(GBNFFT_WPP_SPREAD, 2, float)
      GBNFFT_WPP_TAPS(GBNFFT_WPP_SPREAD, 3, float)
      default:
        return nullptr;
    }
  }
  switch (d * 100 + taps) {
    GBNFFT_WPP_TAPS(GBNFFT_WPP_INTERP, 2, float)
    GBNFFT_WPP_TAPS(GBNFFT_WPP_INTERP, 3, float)
    default:
      return nullptr;
  }
}

}  // namespace gbnfft
