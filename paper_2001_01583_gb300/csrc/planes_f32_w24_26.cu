// Instantiations of the 3-D shared-tile kernels for float, windows of 24 and 26 taps.
#include "points_planes.cuh"

namespace gbnfft {

#define GBNFFT_PLANE_SPREAD(W, NW, R) \
  case (W) * 100 + (NW):              \
    return reinterpret_cast<const void*>(&k_spread_planes<W, NW, R>);
#define GBNFFT_PLANE_INTERP(W, R) \
  case W:                         \
    return reinterpret_cast<const void*>(&k_interp_groups<W, R>);
#define GBNFFT_PLANE_BYTES(W, R) \
  case W:                        \
    return plane_table_bytes<W, R>(bp, np, nw, tile, spread);

const void* planes_kernel_f32_w24_26(int taps, int warps, bool spread) {
  if (spread) {
    switch (taps * 100 + warps) {
      GBNFFT_PLANE_SPREAD_CASES_W24_26(GBNFFT_PLANE_SPREAD, float)
      default:
        return nullptr;
    }
  }
  switch (taps) {
    GBNFFT_PLANE_TAPS_W24_26(GBNFFT_PLANE_INTERP, float)
    default:
      return nullptr;
  }
}

size_t planes_table_bytes_f32_w24_26(int taps, int bp, int np, int nw, const int* tile, bool spread) {
  switch (taps) {
    GBNFFT_PLANE_TAPS_W24_26(GBNFFT_PLANE_BYTES, float)
    default:
      return 0;
  }
}

}  // namespace gbnfft
