// C ABI of batches (include/gbnfft.h): many independent transforms of
// uneven sizes, set up once and run as one CUDA-graph launch per call.
#include <new>
#include <vector>

#include "engine.h"

using namespace gbnfft;

struct nfft_batch {
  Engine eng;
};

extern "C" {

int nfft_batch_create(nfft_batch** out, int count, const nfft_batch_item* items, int precision, void* cuda_stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > 65535 || !items) return NFFT_ERR_INVALID_ARG;
  std::vector<ItemSpec> specs((size_t)count);
  for (int i = 0; i < count; ++i) {
    const nfft_batch_item& b = items[i];
    if (b.d < 1 || b.d > 3) return NFFT_ERR_INVALID_ARG;
    ItemSpec& s = specs[(size_t)i];
    s.d = b.d;
    for (int t = 0; t < 3; ++t) s.N[t] = t < b.d ? b.N[t] : 1;
    s.M = b.M;
    s.sigma = b.sigma;
    s.m = b.m;
    s.window = b.window;
    s.nrhs = b.nrhs;
    const int st = validate_spec(s, precision);
    if (st != NFFT_OK) return st;
  }
  // the sort indexes every point of the batch with 32-bit integers (bin
  // starts, ranks, scatter positions): checked before any device work
  if (total_points_exceed_int32(specs)) return NFFT_ERR_UNSUPPORTED;
  nfft_batch* p = new (std::nothrow) nfft_batch();
  if (!p) return NFFT_ERR_OOM;
  const int st = p->eng.init(specs, precision, static_cast<cudaStream_t>(cuda_stream), false);
  if (st != NFFT_OK) {
    delete p;
    return st;
  }
  *out = p;
  return NFFT_OK;
}

int nfft_batch_destroy(nfft_batch* p) {
  delete p;
  return NFFT_OK;
}

int nfft_batch_set_points(nfft_batch* p, const double* const* x_dev) {
  if (!p || !x_dev) return NFFT_ERR_INVALID_ARG;
  return p->eng.set_points_batch(x_dev);
}

int nfft_batch_adjoint(nfft_batch* p, const void* const* f_dev, void* const* fhat_dev) {
  if (!p || !f_dev || !fhat_dev) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  for (size_t i = 0; i < p->eng.specs.size(); ++i)
    if (!fhat_dev[i] || (!f_dev[i] && p->eng.specs[i].M > 0)) return NFFT_ERR_INVALID_ARG;
  return p->eng.adjoint_batch(f_dev, fhat_dev);
}

int nfft_batch_forward(nfft_batch* p, const void* const* fhat_dev, void* const* f_dev) {
  if (!p || !f_dev || !fhat_dev) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  for (size_t i = 0; i < p->eng.specs.size(); ++i)
    if (!fhat_dev[i] || (!f_dev[i] && p->eng.specs[i].M > 0)) return NFFT_ERR_INVALID_ARG;
  return p->eng.forward_batch(fhat_dev, f_dev);
}

int nfft_batch_autotune(nfft_batch* p, int reps, double* best_ms) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.autotune(reps, best_ms);
}

int nfft_batch_sync(nfft_batch* p) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.sync();
}

int nfft_batch_set_option(nfft_batch* p, int option, int64_t value) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.set_option(option, value);
}

int nfft_batch_stage_times(nfft_batch* p, double* ms, int64_t* launches, int reset) {
  if (!p || !ms) return NFFT_ERR_INVALID_ARG;
  return p->eng.stage_times(ms, launches, reset);
}

int nfft_batch_kernel_launches(const nfft_batch* p, int64_t* count) {
  if (!p || !count) return NFFT_ERR_INVALID_ARG;
  *count = p->eng.launched();
  return NFFT_OK;
}

}  // extern "C"
