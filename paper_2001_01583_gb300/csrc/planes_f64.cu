// Instantiations of the 3-D shared-tile kernels for double, windows of up to 16 taps (18 and 20: planes_f64_w18_20.cu).
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

const void* planes_kernel_f64_w18_20(int taps, int warps, bool spread);
size_t planes_table_bytes_f64_w18_20(int taps, int bp, int np, int nw, const int* tile, bool spread);

const void* planes_spread_f64_uneven(int taps, int warps);

const void* planes_kernel_f64(int taps, int warps, bool spread) {
  if (taps >= 18) return planes_kernel_f64_w18_20(taps, warps, spread);
  if (spread) {
    switch (taps * 100 + warps) {
      GBNFFT_PLANE_SPREAD_CASES_NARROW(GBNFFT_PLANE_SPREAD, double)
      default:
        return planes_spread_f64_uneven(taps, warps);
    }
  }
  switch (taps) {
    GBNFFT_PLANE_TAPS_NARROW(GBNFFT_PLANE_INTERP, double)
    default:
      return nullptr;
  }
}

size_t planes_table_bytes_f64(int taps, int bp, int np, int nw, const int* tile, bool spread) {
  if (taps >= 18) return planes_table_bytes_f64_w18_20(taps, bp, np, nw, tile, spread);
  switch (taps) {
    GBNFFT_PLANE_TAPS_NARROW(GBNFFT_PLANE_BYTES, double)
    default:
      return 0;
  }
}

}  // namespace gbnfft
