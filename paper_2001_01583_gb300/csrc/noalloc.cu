// nfft_ewald_reciprocal_sum_noalloc: the reciprocal-sum reduction of
// nfft_ewald_reciprocal_sum without a plan and without any device allocation.
//
// Who needs it: code that may not call cudaMalloc at the point where it wants
// this sum -- for example a caller running inside a framework whose caching
// allocator owns all device memory (a raw cudaMalloc there can fail or
// synchronise the device), a caller in a steady-state loop that forbids
// allocation, or a caller without any plan at hand.  Such a caller passes its
// own input and output buffers; the only scratch memory, the per-tile FP64
// partial sums, lives in the file-scope array below.
//
// The array is part of the library image: every GPU that loads the library
// holds it (kNoallocMaxPartials doubles = 32 KiB) until the process exits.
// Host code must not use the symbol itself as a device address (in host code
// it names a host-side stand-in); the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
#include <cmath>
#include <mutex>

#include "ewald.h"
#include "gbnfft.h"

namespace gbnfft {
namespace {

constexpr int64_t kNoallocMaxPartials = NFFT_NOALLOC_MAX_MODES / kEwaldTile;
static_assert(kNoallocMaxPartials * kEwaldTile == NFFT_NOALLOC_MAX_MODES, "max modes must be whole tiles");

static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device (looked up on
// the first call per device).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NFFT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return NFFT_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return NFFT_OK;
}

}  // namespace
}  // namespace gbnfft

extern "C" int nfft_ewald_reciprocal_sum_noalloc(int d, const int64_t* N, int precision, const void* S_dev, double L,
                                                 double alpha, double* sum_dev, void* cuda_stream) {
  using namespace gbnfft;
  if (d < 1 || d > 3 || !N || !S_dev || !sum_dev) return NFFT_ERR_INVALID_ARG;
  if (precision != NFFT_FP64 && precision != NFFT_FP32_MIXED) return NFFT_ERR_INVALID_ARG;
  if (!(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha)) return NFFT_ERR_INVALID_ARG;
  EwaldGeom g{};
  g.d = d;
  g.NN = 1;
  for (int t = 0; t < kMaxDim; ++t) {
    g.N[t] = 1;
    g.n[t] = 1;
    g.inv_c[t] = nullptr;
  }
  for (int t = 0; t < d; ++t) {
    if (N[t] < 2 || (N[t] & 1) || N[t] > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
    g.N[t] = (int)N[t];
    g.n[t] = (int)N[t];
    if (g.NN > NFFT_NOALLOC_MAX_MODES / N[t]) return NFFT_ERR_UNSUPPORTED;  // before any overflow
    g.NN *= N[t];
  }
  if (g.NN > NFFT_NOALLOC_MAX_MODES) return NFFT_ERR_UNSUPPORTED;
  const double al = alpha * L;
  g.coef = M_PI * M_PI / (al * al);
  double* scratch = nullptr;
  const int s = scratch_for_current_device(&scratch);
  if (s != NFFT_OK) return s;
  // every partial is written by the first kernel before the second reads it,
  // so the shared array needs no clearing between calls
  const double scale = 1.0 / (2.0 * M_PI * L);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const cudaError_t e =
      precision == NFFT_FP64
          ? launch_ewald_sum<double>(static_cast<const double2*>(S_dev), false, g, scratch, scale, 0.0, sum_dev, st)
          : launch_ewald_sum<float>(static_cast<const float2*>(S_dev), false, g, scratch, scale, 0.0, sum_dev, st);
  return e == cudaSuccess ? NFFT_OK : NFFT_ERR_CUDA;
}
