// Instantiations of the 3-D shared-tile kernels for double, windows of 18 and 20 taps.
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

const void* planes_kernel_f64_w18_20(int taps, int warps, bool spread) {
  if (spread) {
    switch (taps * 100 + warps) {
      GBNFFT_PLANE_SPREAD_CASES_W18_20(GBNFFT_PLANE_SPREAD, double)
      default:
        return nullptr;
    }
  }
  switch (taps) {
    GBNFFT_PLANE_TAPS_W18_20(GBNFFT_PLANE_INTERP, double)
    default:
      return nullptr;
  }
}

size_t planes_table_bytes_f64_w18_20(int taps, int bp, int np, int nw, const int* tile, bool spread) {
  switch (taps) {
    GBNFFT_PLANE_TAPS_W18_20(GBNFFT_PLANE_BYTES, double)
    default:
      return 0;
  }
}

}  // namespace gbnfft
