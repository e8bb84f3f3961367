// Instantiations of the warp-per-point grid kernels for double.
#include "points_gm.cuh"

namespace gbnfft {

#define GBNFFT_GM_CASE(D, W, R)                                                  \
  case (D) * 100 + (W):                                                          \
    return spread ? reinterpret_cast<const void*>(&k_spread_gm<D, W, R>)         \
                  : reinterpret_cast<const void*>(&k_interp_gm<D, W, R>);

const void* gm_kernel_f64(int d, int taps, bool spread) {
  switch (d * 100 + taps) {
    GBNFFT_GM_TAPS(GBNFFT_GM_CASE, 1, double)
    GBNFFT_GM_TAPS(GBNFFT_GM_CASE, 2, double)
    GBNFFT_GM_TAPS(GBNFFT_GM_CASE, 3, double)
    default:
      return nullptr;
  }
}

}  // namespace gbnfft
