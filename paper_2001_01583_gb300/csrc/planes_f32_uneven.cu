// Instantiations of the 3-D plane-owner spreading kernel for float with more
// warps than divide the taps (warps take ceil or floor of taps / warps planes).
#include "points_planes.cuh"

namespace gbnfft {

#define GBNFFT_PLANE_SPREAD(W, NW, R) \
  case (W) * 100 + (NW):              \
    return reinterpret_cast<const void*>(&k_spread_planes<W, NW, R>);

const void* planes_spread_f32_uneven(int taps, int warps) {
  switch (taps * 100 + warps) {
    GBNFFT_PLANE_SPREAD_CASES_UNEVEN(GBNFFT_PLANE_SPREAD, float)
    default:
      return nullptr;
  }
}

}  // namespace gbnfft
