// C ABI of single plans (include/gbnfft.h): a plan is an engine holding one
// item whose data pointers come with every call.
#include <cmath>
#include <new>
#include <vector>

#include "engine.h"

using namespace gbnfft;

struct nfft_plan {
  Engine eng;
};

namespace {
constexpr int kVersion = 10100;  // 1.1.0
}

extern "C" {

int nfft_version(void) { return kVersion; }

const char* nfft_status_string(int s) {
  switch (s) {
    case NFFT_OK: return "ok";
    case NFFT_ERR_INVALID_ARG: return "invalid argument";
    case NFFT_ERR_DOMAIN: return "non-finite point coordinate";
    case NFFT_ERR_OOM: return "out of device memory";
    case NFFT_ERR_CUDA: return "CUDA runtime error";
    case NFFT_ERR_CUFFT: return "cuFFT error";
    case NFFT_ERR_NOT_READY: return "points not set";
    case NFFT_ERR_TIMEOUT: return "device wait timed out";
    case NFFT_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

int nfft_plan_params(int d, const int64_t* N, double sigma, int m, int window, int64_t* n_out, int* taps_out) {
  if (d < 1 || d > 3 || !N) return NFFT_ERR_INVALID_ARG;
  ItemSpec s{};
  s.d = d;
  for (int t = 0; t < d; ++t) s.N[t] = N[t];
  s.M = 0;
  s.sigma = sigma;
  s.m = m;
  s.window = window;
  s.nrhs = 1;
  const int st = validate_spec(s, NFFT_FP64);
  if (st != NFFT_OK) return st;
  for (int t = 0; t < d; ++t)
    if (n_out) n_out[t] = oversampled_size(N[t], sigma);
  if (taps_out) *taps_out = window_taps(window, m);
  return NFFT_OK;
}

int nfft_deconv_amplification(int d, const int64_t* N, double sigma, int m, int window, double* rms, double* peak) {
  int64_t n[3] = {1, 1, 1};
  int taps = 0;
  const int st = nfft_plan_params(d, N, sigma, m, window, n, &taps);
  if (st != NFFT_OK) return st;
  double r = 1.0, x = 1.0;
  for (int t = 0; t < d; ++t) {
    const double b = shape_param(window, m, (double)n[t] / (double)N[t]);
    const double c0 = inv_c_at(window, m, n[t], b, 0.0);
    // at most 4097 frequencies per dimension (all of them up to N_t = 4096)
    const int64_t step = N[t] > 4096 ? (N[t] + 4095) / 4096 : 1;
    double s2 = 0.0, mx = 0.0;
    int64_t cnt = 0;
    for (int64_t a = 0; a < N[t]; a += step) {
      const double v = inv_c_at(window, m, n[t], b, (double)(a - N[t] / 2)) / c0;
      s2 += v * v;
      mx = v > mx ? v : mx;
      ++cnt;
    }
    // the edge frequency -N_t/2 carries the maximum
    const double edge = inv_c_at(window, m, n[t], b, (double)(-N[t] / 2)) / c0;
    mx = edge > mx ? edge : mx;
    r *= std::sqrt(s2 / (double)cnt);
    x *= mx;
  }
  if (rms) *rms = r;
  if (peak) *peak = x;
  return NFFT_OK;
}

int nfft_plan_create(nfft_plan** out, int d, const int64_t* N, int64_t M, double sigma, int m, int window,
                     int precision, void* cuda_stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (d < 1 || d > 3 || !N) return NFFT_ERR_INVALID_ARG;
  ItemSpec s{};
  s.d = d;
  for (int t = 0; t < 3; ++t) s.N[t] = t < d ? N[t] : 1;
  s.M = M;
  s.sigma = sigma;
  s.m = m;
  s.window = window;
  s.nrhs = 1;
  const int st0 = validate_spec(s, precision);
  if (st0 != NFFT_OK) return st0;
  nfft_plan* p = new (std::nothrow) nfft_plan();
  if (!p) return NFFT_ERR_OOM;
  const int st = p->eng.init(std::vector<ItemSpec>{s}, precision, static_cast<cudaStream_t>(cuda_stream), true);
  if (st != NFFT_OK) {
    delete p;
    return st;
  }
  *out = p;
  return NFFT_OK;
}

int nfft_plan_destroy(nfft_plan* p) {
  delete p;
  return NFFT_OK;
}

int nfft_set_points(nfft_plan* p, const double* x_dev) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  if (!x_dev && p->eng.specs[0].M > 0) return NFFT_ERR_INVALID_ARG;
  return p->eng.set_points_single(x_dev);
}

int nfft_adjoint(nfft_plan* p, const void* f_dev, void* fhat_dev, int R) {
  if (!p || R < 0) return NFFT_ERR_INVALID_ARG;
  if (R == 0) return NFFT_OK;
  if (!fhat_dev || (!f_dev && p->eng.specs[0].M > 0)) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  return p->eng.adjoint_single(f_dev, fhat_dev, R);
}

int nfft_forward(nfft_plan* p, const void* fhat_dev, void* f_dev, int R) {
  if (!p || R < 0) return NFFT_ERR_INVALID_ARG;
  if (R == 0) return NFFT_OK;
  if (!fhat_dev || (!f_dev && p->eng.specs[0].M > 0)) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  return p->eng.forward_single(fhat_dev, f_dev, R);
}

int nfft_ewald_reciprocal(nfft_plan* p, const void* q_dev, double L, double alpha, double* out) {
  if (!p || !out || !(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  if (!q_dev && p->eng.specs[0].M > 0) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  return p->eng.ewald(q_dev, L, alpha, out);
}

int nfft_ewald_reciprocal_forces(nfft_plan* p, const void* q_dev, double L, double alpha, double* F_dev) {
  if (!p || !F_dev || !(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  if (!q_dev && p->eng.specs[0].M > 0) return NFFT_ERR_INVALID_ARG;
  if (!p->eng.points_set) return NFFT_ERR_NOT_READY;
  return p->eng.ewald_forces(q_dev, L, alpha, F_dev);
}

int nfft_ewald_reciprocal_sum(nfft_plan* p, const void* S_dev, double L, double alpha, double* sum_dev) {
  if (!p || !S_dev || !sum_dev || !(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  return p->eng.ewald_sum(S_dev, L, alpha, sum_dev);
}

int nfft_autotune(nfft_plan* p, int reps, double* best_ms) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.autotune(reps, best_ms);
}

int nfft_sync(nfft_plan* p) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.sync();
}

int nfft_set_stream(nfft_plan* p, void* cuda_stream) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.set_stream(static_cast<cudaStream_t>(cuda_stream));
}

int nfft_set_option(nfft_plan* p, int option, int64_t value) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  return p->eng.set_option(option, value);
}

int nfft_get_info(const nfft_plan* p, nfft_plan_info* info) {
  if (!p || !info) return NFFT_ERR_INVALID_ARG;
  return p->eng.info(info);
}

int nfft_stage_times(nfft_plan* p, double* ms, int64_t* launches, int reset) {
  if (!p || !ms) return NFFT_ERR_INVALID_ARG;
  return p->eng.stage_times(ms, launches, reset);
}

}  // extern "C"
