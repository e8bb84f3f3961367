// Instantiations of the 3-D owner spreading kernel for float.
#include "points_owner.cuh"

namespace gbnfft {

#define GBNFFT_OWNER_CASE(W) \
  case W:                    \
    return reinterpret_cast<const void*>(&k_spread_owner<W, float>);

const void* owner_kernel_f32(int taps) {
  switch (taps) {
    GBNFFT_OWNER_CASE(2) GBNFFT_OWNER_CASE(4) GBNFFT_OWNER_CASE(6) GBNFFT_OWNER_CASE(8) GBNFFT_OWNER_CASE(10)
    GBNFFT_OWNER_CASE(12) GBNFFT_OWNER_CASE(14) GBNFFT_OWNER_CASE(16) GBNFFT_OWNER_CASE(18)
    GBNFFT_OWNER_CASE(20) GBNFFT_OWNER_CASE(22) GBNFFT_OWNER_CASE(24) GBNFFT_OWNER_CASE(26)
    default:
      return nullptr;
  }
}

}  // namespace gbnfft
