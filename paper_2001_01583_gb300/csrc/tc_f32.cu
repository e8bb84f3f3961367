// Instantiations of the tensor-core 3-D spreading and interpolation kernels
// (points_tc.cuh): FP32 plans, windows of 4, 6 or 8 taps.
#include "points_tc.cuh"

namespace gbnfft {

const void* tc_spread_kernel_f32(int taps) {
  switch (taps) {
    case 4:
      return reinterpret_cast<const void*>(&k_spread_tc<4>);
    case 6:
      return reinterpret_cast<const void*>(&k_spread_tc<6>);
    case 8:
      return reinterpret_cast<const void*>(&k_spread_tc<8>);
    default:
      return nullptr;
  }
}

size_t tc_spread_smem_bytes(int taps, int ncols, const int* tile) { return tc_smem_bytes(taps, ncols, tile); }

const void* tc_interp_kernel_f32(int taps) {
  switch (taps) {
    case 4:
      return reinterpret_cast<const void*>(&k_interp_tc<4>);
    case 6:
      return reinterpret_cast<const void*>(&k_interp_tc<6>);
    case 8:
      return reinterpret_cast<const void*>(&k_interp_tc<8>);
    default:
      return nullptr;
  }
}

size_t tc_interp_smem_bytes_host(int taps, int ncols, const int* tile) { return tc_interp_smem_bytes(taps, ncols, tile); }

}  // namespace gbnfft
