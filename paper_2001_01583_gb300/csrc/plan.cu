// Host side of the gbnfft C ABI (declared in include/gbnfft.h): plans,
// nfft_set_points, and the two transforms of Section 2 as sequences of
// kernels and cuFFT calls queued on the plan's stream.
#include <cufft.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <climits>
#include <map>
#include <new>
#include <vector>

#include "gbnfft.h"
#include "ewald.h"
#include "kernels.h"

using namespace gbnfft;

namespace {

constexpr int kVersion = 10000;  // 1.0.0
constexpr size_t kSmemBudget = 200 * 1024;     // per block, tiled kernels (opt-in limit is 227 KB)
constexpr size_t kSmemTarget = 100 * 1024;     // aim: two blocks per SM

struct EventPair {
  int stage;
  cudaEvent_t start, stop;
};

}  // namespace

struct nfft_plan {
  int d = 0;
  int64_t N[3] = {1, 1, 1};
  int64_t n[3] = {1, 1, 1};
  int64_t M = 0;
  int m = 0;
  int window = 0;
  int precision = 0;
  double sigma = 2.0;
  size_t csize = 16;  // bytes per complex value
  WindowDev win{};
  GridGeom geom{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 1;
  size_t smem_optin = 48 * 1024;
  size_t smem_per_sm = 100 * 1024;
  int wpp_pitch = 0;   // row pitch of the warp-per-point tiles
  std::map<std::pair<const void*, std::pair<int, size_t>>, int> occupancy;  // (kernel, threads, smem) -> blocks/SM

  // options
  int method_opt = NFFT_METHOD_AUTO;
  int method = NFFT_METHOD_TILED;
  int bin_opt[3] = {0, 0, 0};
  int max_sub = 0;      // points per subproblem in use
  int max_sub_opt = 0;
  int rhs_cap = 1;
  int threads = 256;
  int threads_opt = 0;   // explicit threads per block for the 3-D warp kernels (0 = chosen per launch)
  bool profile = false;

  // device memory
  void* grid = nullptr;
  double* inv_c[3] = {nullptr, nullptr, nullptr};
  int* bin_count = nullptr;
  int* bin_start = nullptr;
  int* sub_count = nullptr;
  int* sub_start = nullptr;
  int* num_subs = nullptr;
  SubProblem* subs = nullptr;
  int64_t max_subs = 0;
  int2* bin_rank = nullptr;
  int* perm = nullptr;
  uint32_t* local = nullptr;
  void* delta[3] = {nullptr, nullptr, nullptr};
  int* err_flag = nullptr;
  double* ewald_partials = nullptr;   // reduction scratch (Eq. 12)
  double* ewald_out = nullptr;        // [reciprocal sum, self term]
  int64_t device_bytes = 0;
  int64_t sort_capacity_bins = 0;

  std::map<int, cufftHandle> ffts;  // batch size -> plan
  bool points_set = false;

  std::vector<EventPair> events;
  std::vector<EventPair> free_events;
  double stage_ms[NFFT_STAGE_COUNT] = {0};
  int64_t stage_calls[NFFT_STAGE_COUNT] = {0};
};

namespace {

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      return e_ == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA; \
    }                                              \
  } while (0)

bool is_fft_friendly(int64_t n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// n_t: smallest even 2,3,5,7-smooth integer >= sigma N_t (sigma = 2 gives 2N_t).
int64_t oversampled(int64_t N, double sigma) {
  int64_t n = (int64_t)std::ceil(sigma * (double)N - 1e-9);
  if (n < 2) n = 2;
  while (n % 2 != 0 || !is_fft_friendly(n)) ++n;
  return n;
}

int taps_for(int window, int m) { return window == NFFT_KAISER_BESSEL ? 2 * m : 2 * m + 2; }

// Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2
// (all terms positive, so it is accurate to rounding for the x used here).
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

double shape_param(int window, int m, double sigma) {
  if (window == NFFT_GAUSSIAN) return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * M_PI);
  return M_PI * (2.0 - 1.0 / sigma);
}

// 1 / c_k for k = -N/2 .. N/2-1 of one dimension, with the kernels' window
// normalisation psi = phi / phi(0):  inv_c(k) = phi(0) / (n phihat(k)).
//   Gaussian:       phi(0) = (pi b)^(-1/2),        n phihat(k) = exp(-b (pi k / n)^2)
//   Kaiser-Bessel:  phi(0) = sinh(b m) / (pi m),   n phihat(k) = I0(m sqrt(b^2 - (2 pi k / n)^2))
std::vector<double> scaling_table(int window, int m, int64_t N, int64_t n, double b) {
  std::vector<double> out((size_t)N);
  for (int64_t a = 0; a < N; ++a) {
    const double k = (double)(a - N / 2);
    if (window == NFFT_GAUSSIAN) {
      const double t = M_PI * k / (double)n;
      out[(size_t)a] = std::exp(b * t * t) / std::sqrt(M_PI * b);
    } else {
      const double w = 2.0 * M_PI * k / (double)n;
      const double arg = m * std::sqrt(b * b - w * w);
      out[(size_t)a] = std::sinh(b * m) / (M_PI * m * bessel_i0(arg));
    }
  }
  return out;
}

void free_dev(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
int alloc_dev(T*& p, size_t bytes, int64_t& total) {
  void* q = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA;
  }
  p = static_cast<T*>(q);
  total += (int64_t)bytes;
  return NFFT_OK;
}

#define TRY(x)               \
  do {                       \
    int s_ = (x);            \
    if (s_ != NFFT_OK) return s_; \
  } while (0)

void release_sort(nfft_plan* p) {
  void* v;
  v = p->bin_count; free_dev(v); p->bin_count = nullptr;
  v = p->bin_start; free_dev(v); p->bin_start = nullptr;
  v = p->sub_count; free_dev(v); p->sub_count = nullptr;
  v = p->sub_start; free_dev(v); p->sub_start = nullptr;
  v = p->subs; free_dev(v); p->subs = nullptr;
}

void release_all(nfft_plan* p) {
  release_sort(p);
  void* v;
  free_dev(p->grid);
  for (int t = 0; t < 3; ++t) {
    v = p->inv_c[t]; free_dev(v); p->inv_c[t] = nullptr;
    free_dev(p->delta[t]);
  }
  v = p->num_subs; free_dev(v); p->num_subs = nullptr;
  v = p->bin_rank; free_dev(v); p->bin_rank = nullptr;
  v = p->perm; free_dev(v); p->perm = nullptr;
  v = p->local; free_dev(v); p->local = nullptr;
  v = p->err_flag; free_dev(v); p->err_flag = nullptr;
  v = p->ewald_partials; free_dev(v); p->ewald_partials = nullptr;
  v = p->ewald_out; free_dev(v); p->ewald_out = nullptr;
  for (auto& kv : p->ffts) cufftDestroy(kv.second);
  p->ffts.clear();
  for (auto& e : p->events) { cudaEventDestroy(e.start); cudaEventDestroy(e.stop); }
  for (auto& e : p->free_events) { cudaEventDestroy(e.start); cudaEventDestroy(e.stop); }
  p->events.clear();
  p->free_events.clear();
}

size_t tile_bytes(const nfft_plan* p, const int* bin) {
  size_t cells = 1;
  for (int t = 0; t < p->d; ++t) cells *= (size_t)(bin[t] + p->win.taps - 1);
  return cells * p->csize;
}

// Row pitch for the warp-per-point tiles: a warp instruction touches Q rows
// of W consecutive elements; the pitch (>= the row length `last`) that needs
// the fewest shared-memory wavefronts -- the largest number of 4-byte words
// one bank must serve, averaged over the row's start -- wins, the smallest on
// ties.
int choose_pitch(int last, int W, int csize) {
  const int Q = 32 / W > 0 ? 32 / W : 1;
  const int words = csize / 4;
  int best = last, best_cost = INT_MAX;
  for (int pitch = last; pitch < last + 32; ++pitch) {
    int cost = 0;
    for (int x0 = 0; x0 < 32; ++x0) {
      int bank[32] = {0};
      for (int q = 0; q < Q; ++q)
        for (int ix = 0; ix < W; ++ix)
          for (int w = 0; w < words; ++w) ++bank[((q * pitch + x0 + ix) * words + w) % 32];
      int mx = 0;
      for (int b = 0; b < 32; ++b) mx = bank[b] > mx ? bank[b] : mx;
      cost += mx;
    }
    if (cost < best_cost) {
      best_cost = cost;
      best = pitch;
    }
  }
  return best;
}

size_t wpp_tile_bytes(const nfft_plan* p, const int* bin, int pitch) {
  size_t rows = 1;
  for (int t = 0; t + 1 < p->d; ++t) rows *= (size_t)(bin[t] + p->win.taps - 1);
  return rows * (size_t)pitch * p->csize;
}

// Choose bins and the method.  Default bins: 1-D 1024, 2-D 32 x 32,
// 3-D 8 x 8 x 16 (the fastest dimension longest: fewer tile rows to flush),
// clamped to the grid and halved while the tile exceeds the per-block
// shared-memory budget; the global method if nothing fits.
int configure_bins(nfft_plan* p) {
  const int defaults[3][3] = {{1024, 1, 1}, {32, 32, 1}, {8, 8, 16}};
  int bin[3] = {1, 1, 1};
  for (int t = 0; t < p->d; ++t) {
    int b = p->bin_opt[t] > 0 ? p->bin_opt[t] : defaults[p->d - 1][t];
    if (b > p->n[t]) b = (int)p->n[t];
    const int maxb = p->d == 1 ? (1 << 30) : (1 << local_bits(p->d)) - 1;
    if (b > maxb) b = maxb;
    bin[t] = b;
  }
  const size_t budget = p->smem_optin < kSmemBudget ? p->smem_optin : kSmemBudget;
  bool explicit_bins = p->bin_opt[0] > 0 || p->bin_opt[1] > 0 || p->bin_opt[2] > 0;
  while (tile_bytes(p, bin) > budget && !explicit_bins) {
    int tmax = 0;
    for (int t = 1; t < p->d; ++t)
      if (bin[t] > bin[tmax]) tmax = t;
    if (bin[tmax] <= 2) break;
    bin[tmax] /= 2;
  }
  bool tiled_ok = tile_bytes(p, bin) <= budget;
  const bool have_kernel = (p->win.taps <= (p->d == 3 ? 26 : 32));
  const int last = bin[p->d - 1] + p->win.taps - 1;
  p->wpp_pitch = choose_pitch(last, p->win.taps, (int)p->csize);
  // the warp-per-point form needs at least two private tiles per block
  const size_t wtile = wpp_tile_bytes(p, bin, p->wpp_pitch);
  const bool warp_ok = p->d >= 2 && p->win.taps <= 16 &&
                       (p->d == 3 ? wtile + 32768 <= budget : 2 * wtile + 4096 <= budget);
  int method = p->method_opt;
  if (method == NFFT_METHOD_AUTO)
    method = warp_ok ? NFFT_METHOD_WARP : ((tiled_ok && have_kernel) ? NFFT_METHOD_TILED : NFFT_METHOD_GLOBAL);
  if (method == NFFT_METHOD_TILED && (!tiled_ok || !have_kernel)) return NFFT_ERR_UNSUPPORTED;
  if (method == NFFT_METHOD_WARP && !warp_ok) return NFFT_ERR_UNSUPPORTED;
  p->method = method;
  GridGeom& g = p->geom;
  g.d = p->d;
  g.grid_cells = 1;
  g.tile_cells = 1;
  for (int t = 0; t < 3; ++t) {
    g.n[t] = t < p->d ? (int)p->n[t] : 1;
    g.bin[t] = t < p->d ? bin[t] : 1;
    g.nbins[t] = t < p->d ? (int)((p->n[t] + bin[t] - 1) / bin[t]) : 1;
    g.tile[t] = t < p->d ? bin[t] + p->win.taps - 1 : 1;
  }
  for (int t = 0; t < p->d; ++t) {
    g.grid_cells *= g.n[t];
    g.tile_cells *= g.tile[t];
  }
  return NFFT_OK;
}

int64_t n_bins(const nfft_plan* p) {
  int64_t nb = 1;
  for (int t = 0; t < p->d; ++t) nb *= p->geom.nbins[t];
  return nb;
}

// (Re)allocate the per-bin and subproblem arrays for the current bins.
int alloc_sort(nfft_plan* p) {
  const int defaults_P[3] = {1024, 1024, 1024};
  p->max_sub = p->max_sub_opt > 0 ? p->max_sub_opt : defaults_P[p->d - 1];
  const int64_t nb = n_bins(p);
  if (nb > (int64_t)1 << 30) return NFFT_ERR_UNSUPPORTED;
  const int64_t max_subs = nb + p->M / p->max_sub + 1;
  if (nb == p->sort_capacity_bins && max_subs <= p->max_subs && p->bin_count) return NFFT_OK;
  int64_t dummy = 0;
  if (p->bin_count) {
    p->device_bytes -= (int64_t)(4 * 4 * p->sort_capacity_bins + sizeof(SubProblem) * p->max_subs);
    release_sort(p);
  }
  TRY(alloc_dev(p->bin_count, sizeof(int) * nb, dummy));
  TRY(alloc_dev(p->bin_start, sizeof(int) * nb, dummy));
  TRY(alloc_dev(p->sub_count, sizeof(int) * nb, dummy));
  TRY(alloc_dev(p->sub_start, sizeof(int) * nb, dummy));
  TRY(alloc_dev(p->subs, sizeof(SubProblem) * max_subs, dummy));
  p->sort_capacity_bins = nb;
  p->max_subs = max_subs;
  p->device_bytes += (int64_t)(4 * 4 * nb + sizeof(SubProblem) * max_subs);
  return NFFT_OK;
}

int alloc_grid(nfft_plan* p, int cap) {
  const size_t bytes = (size_t)cap * (size_t)p->geom.grid_cells * p->csize;
  void* g = nullptr;
  cudaError_t e = cudaMalloc(&g, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA;
  }
  if (p->grid) {
    p->device_bytes -= (int64_t)p->rhs_cap * p->geom.grid_cells * (int64_t)p->csize;
    cudaFree(p->grid);
  }
  p->grid = g;
  p->rhs_cap = cap;
  p->device_bytes += (int64_t)bytes;
  return NFFT_OK;
}

int fft_handle(nfft_plan* p, int batch, cufftHandle* out) {
  auto it = p->ffts.find(batch);
  if (it != p->ffts.end()) {
    *out = it->second;
    return cufftSetStream(it->second, p->stream) == CUFFT_SUCCESS ? NFFT_OK : NFFT_ERR_CUFFT;
  }
  cufftHandle h;
  if (cufftCreate(&h) != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
  long long dims[3];
  for (int t = 0; t < p->d; ++t) dims[t] = p->n[t];
  size_t work = 0;
  const cufftType type = p->precision == NFFT_FP64 ? CUFFT_Z2Z : CUFFT_C2C;
  const long long dist = p->geom.grid_cells;
  cufftResult r = cufftMakePlanMany64(h, p->d, dims, nullptr, 1, dist, nullptr, 1, dist, type, batch, &work);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return r == CUFFT_ALLOC_FAILED ? NFFT_ERR_OOM : NFFT_ERR_CUFFT;
  }
  if (cufftSetStream(h, p->stream) != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return NFFT_ERR_CUFFT;
  }
  p->ffts[batch] = h;
  *out = h;
  return NFFT_OK;
}

int run_fft(nfft_plan* p, int batch, int direction) {
  cufftHandle h;
  TRY(fft_handle(p, batch, &h));
  cufftResult r;
  if (p->precision == NFFT_FP64) {
    cufftDoubleComplex* g = static_cast<cufftDoubleComplex*>(p->grid);
    r = cufftExecZ2Z(h, g, g, direction);
  } else {
    cufftComplex* g = static_cast<cufftComplex*>(p->grid);
    r = cufftExecC2C(h, g, g, direction);
  }
  return r == CUFFT_SUCCESS ? NFFT_OK : NFFT_ERR_CUFFT;
}

// ---- profiling ----------------------------------------------------------
int stage_begin(nfft_plan* p, int stage, EventPair* ev) {
  if (!p->profile) return NFFT_OK;
  if (!p->free_events.empty()) {
    *ev = p->free_events.back();
    p->free_events.pop_back();
  } else {
    CK(cudaEventCreate(&ev->start));
    CK(cudaEventCreate(&ev->stop));
  }
  ev->stage = stage;
  CK(cudaEventRecord(ev->start, p->stream));
  return NFFT_OK;
}

int stage_end(nfft_plan* p, EventPair* ev) {
  if (!p->profile) return NFFT_OK;
  CK(cudaEventRecord(ev->stop, p->stream));
  p->events.push_back(*ev);
  return NFFT_OK;
}

// ---- point kernels --------------------------------------------------------
template <typename Real>
PointKernelArgs<Real> point_args(nfft_plan* p) {
  PointKernelArgs<Real> a{};
  a.pts.perm = p->perm;
  a.pts.local = p->local;
  for (int t = 0; t < 3; ++t) a.pts.delta[t] = static_cast<const Real*>(p->delta[t]);
  a.pts.subs = p->subs;
  a.pts.num_subs = p->num_subs;
  a.geom = p->geom;
  a.win = p->win;
  a.M = p->M;
  return a;
}

template <typename Real>
const void* wpp_kernel(int d, int taps, bool spread);
template <>
const void* wpp_kernel<float>(int d, int taps, bool spread) { return wpp_kernel_f32(d, taps, spread); }
template <>
const void* wpp_kernel<double>(int d, int taps, bool spread) { return wpp_kernel_f64(d, taps, spread); }

int blocks_per_sm(nfft_plan* p, const void* fn, int threads, size_t smem) {
  const auto key = std::make_pair(fn, std::make_pair(threads, smem));
  auto it = p->occupancy.find(key);
  if (it != p->occupancy.end()) return it->second;
  int nb = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess)
    nb = 0;
  p->occupancy[key] = nb;
  return nb;
}

template <typename Real>
const void* planes_kernel(int taps, int warps, bool spread);
template <>
const void* planes_kernel<float>(int taps, int warps, bool spread) { return planes_kernel_f32(taps, warps, spread); }
template <>
const void* planes_kernel<double>(int taps, int warps, bool spread) { return planes_kernel_f64(taps, warps, spread); }
template <typename Real>
size_t planes_table_bytes(int taps, int bp, int np, int nw, const int* tile);
template <>
size_t planes_table_bytes<float>(int taps, int bp, int np, int nw, const int* tile) {
  return planes_table_bytes_f32(taps, bp, np, nw, tile);
}
template <>
size_t planes_table_bytes<double>(int taps, int bp, int np, int nw, const int* tile) {
  return planes_table_bytes_f64(taps, bp, np, nw, tile);
}

// 3-D: one shared tile per block.  Spreading splits the tile's planes among
// the block's warps (a power of two dividing the taps); interpolation gives
// each warp groups of points.  Warps per block: the option if set, else the
// most resident warps (ties: fewer warps per block, which share the per-point
// work among fewer warps).  Right-hand sides per pass fit two blocks per SM.
template <typename Real>
int run_planes(nfft_plan* p, PointKernelArgs<Real>& a, bool spread) {
  const int W = p->win.taps;
  const size_t rows = (size_t)p->geom.tile[0] * p->geom.tile[1];
  const size_t tbytes = rows * (size_t)p->wpp_pitch * p->csize;
  auto smem_of = [&](int nw, int np) {
    return (size_t)np * tbytes + planes_table_bytes<Real>(W, 32 * nw, np, nw, p->geom.tile);
  };
  int np = 1;
  while (np < a.nrhs && smem_of(8, np + 1) <= p->smem_per_sm / 2) ++np;
  int best_nw = 0, best_warps = 0;
  size_t best_smem = 0;
  const void* best_fn = nullptr;
  for (int nw = 1; nw <= 8; nw *= 2) {
    if (p->threads_opt > 0 && 32 * nw != p->threads_opt) continue;
    const void* fn = planes_kernel<Real>(W, nw, spread);
    if (!fn) continue;
    const size_t smem = smem_of(nw, np);
    if (smem > p->smem_optin) continue;
    const int per_sm = blocks_per_sm(p, fn, 32 * nw, smem);
    if (per_sm * nw > best_warps) {
      best_warps = per_sm * nw;
      best_nw = nw;
      best_smem = smem;
      best_fn = fn;
    }
  }
  if (!best_fn || best_warps == 0) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = np;
  WppLayout lay{p->wpp_pitch, (int)(rows * p->wpp_pitch), best_nw};
  int64_t blocks = (int64_t)(best_warps / best_nw) * p->num_sms;
  if (blocks > p->max_subs) blocks = p->max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a, &lay};
  CK(cudaFuncSetAttribute(best_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_smem));
  CK(cudaLaunchKernel(best_fn, dim3((unsigned)blocks), dim3(32 * best_nw), args, best_smem, p->stream));
  return NFFT_OK;
}

// Warp per point: private tiles for spreading, one shared tile for
// interpolation.  Right-hand sides per pass and warps per block are chosen
// for the most resident warps within the shared-memory budget.
template <typename Real>
int run_wpp(nfft_plan* p, PointKernelArgs<Real>& a, bool spread) {
  const int D = p->d, W = p->win.taps;
  const void* fn = wpp_kernel<Real>(D, W, spread);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  const int last = p->geom.tile[D - 1];
  const int rows = p->geom.tile_cells / last;
  const size_t elems = (size_t)rows * p->wpp_pitch;
  const size_t tbytes = elems * p->csize;
  const size_t scratch = (size_t)(32 * D * W + (D == 3 ? W * W : W)) * sizeof(Real);  // weight table + row weights
  const size_t sm = p->smem_per_sm;
  int np = 1;
  if (spread) {
    while (np < a.nrhs && 4 * (size_t)(np + 1) * tbytes + 4 * scratch <= sm) ++np;
  } else {
    while (np < a.nrhs && (size_t)(np + 1) * tbytes + 8 * scratch <= sm / 2) ++np;
  }
  int best_nw = 0, best_warps = 0;
  size_t best_smem = 0;
  for (int nw = 1; nw <= 8; ++nw) {
    // spread: per warp its tiles, weight table and the batch's values ([np][32] complex)
    const size_t smem = spread ? (size_t)nw * ((size_t)np * tbytes + scratch + (size_t)np * 32 * p->csize)
                               : (size_t)np * tbytes + nw * scratch;
    if (smem > p->smem_optin) break;
    const int per_sm = blocks_per_sm(p, fn, 32 * nw, smem);
    if (per_sm * nw > best_warps) {
      best_warps = per_sm * nw;
      best_nw = nw;
      best_smem = smem;
    }
  }
  if (best_nw == 0) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = np;
  WppLayout lay{p->wpp_pitch, (int)elems, best_nw};
  int64_t blocks = (int64_t)(best_warps / best_nw) * p->num_sms;
  if (blocks > p->max_subs) blocks = p->max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a, &lay};
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_smem));
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(32 * best_nw), args, best_smem, p->stream));
  return NFFT_OK;
}

template <typename Real>
int run_points(nfft_plan* p, PointKernelArgs<Real>& a, bool spread) {
  if (p->method == NFFT_METHOD_WARP) return p->d == 3 ? run_planes<Real>(p, a, spread) : run_wpp<Real>(p, a, spread);
  const int threads = p->threads;
  if (p->method == NFFT_METHOD_TILED) {
    const size_t one = (size_t)p->geom.tile_cells * p->csize;
    size_t budget = p->smem_optin < kSmemBudget ? p->smem_optin : kSmemBudget;
    if (budget > kSmemTarget && one <= kSmemTarget) budget = kSmemTarget;
    int pass = (int)(budget / one);
    if (pass < 1) pass = 1;
    if (pass > a.nrhs) pass = a.nrhs;
    a.rhs_per_pass = pass;
    const size_t smem = one * (size_t)pass;
    CK(tiled_set_smem_limit<Real>(p->d, p->win.taps, spread, smem));
    int per_sm = tiled_blocks_per_sm<Real>(p->d, p->win.taps, spread, threads, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)per_sm * p->num_sms;
    if (blocks > p->max_subs) blocks = p->max_subs;
    if (blocks < 1) blocks = 1;
    cudaError_t err = cudaSuccess;
    const bool ok = spread ? launch_spread_tiled<Real>(a, (int)blocks, threads, smem, p->stream, &err)
                           : launch_interp_tiled<Real>(a, (int)blocks, threads, smem, p->stream, &err);
    if (!ok) return NFFT_ERR_UNSUPPORTED;
    CK(err);
    return NFFT_OK;
  }
  a.rhs_per_pass = a.nrhs;
  int64_t blocks = (int64_t)8 * p->num_sms;
  if (blocks > p->max_subs) blocks = p->max_subs;
  if (blocks < 1) blocks = 1;
  CK(spread ? launch_spread_global<Real>(a, (int)blocks, threads, p->stream)
            : launch_interp_global<Real>(a, (int)blocks, threads, p->stream));
  return NFFT_OK;
}

int64_t NN_of(const nfft_plan* p) {
  int64_t nn = 1;
  for (int t = 0; t < p->d; ++t) nn *= p->N[t];
  return nn;
}

template <typename Real>
int adjoint_impl(nfft_plan* p, const void* f, void* fhat, int R) {
  using C = typename Cplx<Real>::type;
  const C* fin = static_cast<const C*>(f);
  C* out = static_cast<C*>(fhat);
  const int64_t NN = NN_of(p);
  int Nint[3];
  for (int t = 0; t < 3; ++t) Nint[t] = (int)p->N[t];
  for (int r0 = 0; r0 < R; r0 += p->rhs_cap) {
    const int nr = (R - r0) < p->rhs_cap ? (R - r0) : p->rhs_cap;
    EventPair ev{};
    TRY(stage_begin(p, NFFT_STAGE_SPREAD, &ev));
    CK(cudaMemsetAsync(p->grid, 0, (size_t)nr * p->geom.grid_cells * p->csize, p->stream));
    if (p->M > 0) {
      PointKernelArgs<Real> a = point_args<Real>(p);
      a.f_in = fin + (int64_t)r0 * p->M;
      a.grid = static_cast<C*>(p->grid);
      a.nrhs = nr;
      TRY(run_points<Real>(p, a, true));
    }
    TRY(stage_end(p, &ev));
    TRY(stage_begin(p, NFFT_STAGE_FFT, &ev));
    TRY(run_fft(p, nr, CUFFT_FORWARD));
    TRY(stage_end(p, &ev));
    TRY(stage_begin(p, NFFT_STAGE_DECONV, &ev));
    CK(launch_deconv_crop<Real>(static_cast<const C*>(p->grid), out + (int64_t)r0 * NN, p->inv_c, p->geom, Nint, nr,
                                p->stream));
    TRY(stage_end(p, &ev));
  }
  return NFFT_OK;
}

template <typename Real>
int forward_impl(nfft_plan* p, const void* fhat, void* f, int R) {
  using C = typename Cplx<Real>::type;
  const C* hin = static_cast<const C*>(fhat);
  C* out = static_cast<C*>(f);
  const int64_t NN = NN_of(p);
  int Nint[3];
  for (int t = 0; t < 3; ++t) Nint[t] = (int)p->N[t];
  for (int r0 = 0; r0 < R; r0 += p->rhs_cap) {
    const int nr = (R - r0) < p->rhs_cap ? (R - r0) : p->rhs_cap;
    EventPair ev{};
    TRY(stage_begin(p, NFFT_STAGE_PAD, &ev));
    CK(launch_pad_deconv<Real>(hin + (int64_t)r0 * NN, static_cast<C*>(p->grid), p->inv_c, p->geom, Nint, nr,
                               p->stream));
    TRY(stage_end(p, &ev));
    TRY(stage_begin(p, NFFT_STAGE_IFFT, &ev));
    TRY(run_fft(p, nr, CUFFT_INVERSE));
    TRY(stage_end(p, &ev));
    TRY(stage_begin(p, NFFT_STAGE_INTERP, &ev));
    if (p->M > 0) {
      PointKernelArgs<Real> a = point_args<Real>(p);
      a.grid_in = static_cast<const C*>(p->grid);
      a.f_out = out + (int64_t)r0 * p->M;
      a.nrhs = nr;
      TRY(run_points<Real>(p, a, false));
    }
    TRY(stage_end(p, &ev));
  }
  return NFFT_OK;
}

template <typename Real>
int set_points_impl(nfft_plan* p, const double* x) {
  const int nb = (int)n_bins(p);
  EventPair ev{};
  TRY(stage_begin(p, NFFT_STAGE_SORT, &ev));
  CK(cudaMemsetAsync(p->bin_count, 0, sizeof(int) * (size_t)nb, p->stream));
  CK(launch_bin_count<Real>(x, p->M, p->geom, p->bin_count, p->bin_rank, p->err_flag, p->stream));
  CK(launch_scan(p->bin_count, p->bin_start, nb, nullptr, p->stream));
  Real* d[3] = {static_cast<Real*>(p->delta[0]), static_cast<Real*>(p->delta[1]), static_cast<Real*>(p->delta[2])};
  CK(launch_scatter<Real>(x, p->M, p->geom, p->bin_start, p->bin_rank, p->perm, p->local, d, p->stream));
  CK(launch_subproblem_count(p->bin_count, nb, p->max_sub, p->sub_count, p->stream));
  CK(launch_scan(p->sub_count, p->sub_start, nb, p->num_subs, p->stream));
  CK(launch_subproblem_fill(p->bin_count, p->bin_start, p->sub_start, nb, p->max_sub, p->subs, p->stream));
  TRY(stage_end(p, &ev));
  return NFFT_OK;
}

EwaldGeom ewald_geom(const nfft_plan* p, double L, double alpha) {
  EwaldGeom g{};
  g.d = p->d;
  g.NN = 1;
  for (int t = 0; t < kMaxDim; ++t) {
    g.N[t] = t < p->d ? (int)p->N[t] : 1;
    g.n[t] = t < p->d ? (int)p->n[t] : 1;
    g.inv_c[t] = t < p->d ? p->inv_c[t] : nullptr;
  }
  for (int t = 0; t < p->d; ++t) g.NN *= p->N[t];
  const double al = alpha * L;
  g.coef = M_PI * M_PI / (al * al);
  return g;
}

// Eq. 12 from the charges: spread + FFT (adjoint steps 1-2), then the scaled
// spectrum is weighted and reduced without forming fhat; the self term is a
// second reduction over the charges.
template <typename Real>
int ewald_impl(nfft_plan* p, const void* q, double L, double alpha) {
  using C = typename Cplx<Real>::type;
  EventPair ev{};
  TRY(stage_begin(p, NFFT_STAGE_SPREAD, &ev));
  CK(cudaMemsetAsync(p->grid, 0, (size_t)p->geom.grid_cells * p->csize, p->stream));
  if (p->M > 0) {
    PointKernelArgs<Real> a = point_args<Real>(p);
    a.f_in = static_cast<const C*>(q);
    a.grid = static_cast<C*>(p->grid);
    a.nrhs = 1;
    TRY(run_points<Real>(p, a, true));
  }
  TRY(stage_end(p, &ev));
  TRY(stage_begin(p, NFFT_STAGE_FFT, &ev));
  TRY(run_fft(p, 1, CUFFT_FORWARD));
  TRY(stage_end(p, &ev));
  TRY(stage_begin(p, NFFT_STAGE_DECONV, &ev));
  const EwaldGeom g = ewald_geom(p, L, alpha);
  CK(launch_ewald_sum<Real>(static_cast<const C*>(p->grid), true, g, p->ewald_partials, 1.0 / (2.0 * M_PI * L), 0.0,
                            p->ewald_out, p->stream));
  CK(launch_sumsq<Real>(static_cast<const C*>(q), p->M, p->ewald_partials, -alpha / std::sqrt(M_PI), 0.0,
                        p->ewald_out + 1, p->stream));
  TRY(stage_end(p, &ev));
  return NFFT_OK;
}

int validate_params(int d, const int64_t* N, int64_t M, double sigma, int m, int window, int precision) {
  if (d < 1 || d > 3 || !N) return NFFT_ERR_INVALID_ARG;
  if (M < 0 || M > (int64_t)INT32_MAX) return NFFT_ERR_INVALID_ARG;
  if (!(sigma >= 1.0) || !std::isfinite(sigma) || sigma > 16.0) return NFFT_ERR_INVALID_ARG;
  if (m < 1) return NFFT_ERR_INVALID_ARG;
  if (window != NFFT_GAUSSIAN && window != NFFT_KAISER_BESSEL) return NFFT_ERR_INVALID_ARG;
  if (precision != NFFT_FP64 && precision != NFFT_FP32_MIXED) return NFFT_ERR_INVALID_ARG;
  if (taps_for(window, m) > kMaxTaps) return NFFT_ERR_UNSUPPORTED;
  for (int t = 0; t < d; ++t)
    if (N[t] < 2 || (N[t] & 1) || N[t] > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
  return NFFT_OK;
}

}  // namespace

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
  const int s = validate_params(d, N, 0, sigma, m, window, NFFT_FP64);
  if (s != NFFT_OK) return s;
  for (int t = 0; t < d; ++t) {
    const int64_t n = oversampled(N[t], sigma);
    if (n < 2 * m + 2 || n < N[t]) return NFFT_ERR_INVALID_ARG;
    if (n_out) n_out[t] = n;
  }
  if (taps_out) *taps_out = taps_for(window, m);
  return NFFT_OK;
}

int nfft_plan_create(nfft_plan** out, int d, const int64_t* N, int64_t M, double sigma, int m, int window,
                     int precision, void* cuda_stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  int64_t n[3] = {1, 1, 1};
  int taps = 0;
  int s = validate_params(d, N, M, sigma, m, window, precision);
  if (s != NFFT_OK) return s;
  s = nfft_plan_params(d, N, sigma, m, window, n, &taps);
  if (s != NFFT_OK) return s;
  int64_t cells = 1;
  for (int t = 0; t < d; ++t) cells *= n[t];
  if (cells > (int64_t)INT32_MAX) return NFFT_ERR_UNSUPPORTED;

  nfft_plan* p = new (std::nothrow) nfft_plan();
  if (!p) return NFFT_ERR_OOM;
  p->d = d;
  p->M = M;
  p->m = m;
  p->window = window;
  p->precision = precision;
  p->sigma = sigma;
  p->csize = precision == NFFT_FP64 ? 16 : 8;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  for (int t = 0; t < d; ++t) {
    p->N[t] = N[t];
    p->n[t] = n[t];
  }
  auto fail = [&](int st) {
    release_all(p);
    delete p;
    return st;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(NFFT_ERR_CUDA);
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    return fail(NFFT_ERR_CUDA);
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess)
    return fail(NFFT_ERR_CUDA);
  p->smem_optin = (size_t)optin;
  int per_sm = 0;
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device) != cudaSuccess)
    return fail(NFFT_ERR_CUDA);
  p->smem_per_sm = (size_t)per_sm;

  p->win.kind = window;
  p->win.m = m;
  p->win.shift = window == NFFT_KAISER_BESSEL ? 1 : 0;
  p->win.taps = taps;
  for (int t = 0; t < 3; ++t) {
    const double sig = t < d ? (double)n[t] / (double)N[t] : 2.0;
    const double b = shape_param(window, m, sig);
    p->win.b[t] = b;
    p->win.kb_norm[t] = 1.0 / (1.0 - std::exp(-2.0 * b * m));
  }
  s = configure_bins(p);
  if (s != NFFT_OK) return fail(s);

  int64_t& tot = p->device_bytes;
  for (int t = 0; t < d; ++t) {
    std::vector<double> tab = scaling_table(window, m, N[t], n[t], p->win.b[t]);
    s = alloc_dev(p->inv_c[t], sizeof(double) * tab.size(), tot);
    if (s != NFFT_OK) return fail(s);
    if (cudaMemcpy(p->inv_c[t], tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(NFFT_ERR_CUDA);
  }
  const size_t real_size = precision == NFFT_FP64 ? 8 : 4;
  const size_t Mz = (size_t)(M > 0 ? M : 1);
  if ((s = alloc_dev(p->num_subs, sizeof(int), tot)) != NFFT_OK) return fail(s);
  if ((s = alloc_dev(p->err_flag, sizeof(int), tot)) != NFFT_OK) return fail(s);
  if ((s = alloc_dev(p->bin_rank, sizeof(int2) * Mz, tot)) != NFFT_OK) return fail(s);
  if ((s = alloc_dev(p->perm, sizeof(int) * Mz, tot)) != NFFT_OK) return fail(s);
  if ((s = alloc_dev(p->local, sizeof(uint32_t) * Mz, tot)) != NFFT_OK) return fail(s);
  for (int t = 0; t < d; ++t) {
    void* q = nullptr;
    if ((s = alloc_dev(q, real_size * Mz, tot)) != NFFT_OK) return fail(s);
    p->delta[t] = q;
  }
  {
    int64_t NN = 1;
    for (int t = 0; t < d; ++t) NN *= N[t];
    const int64_t np = std::max(ewald_partials_needed(NN), ewald_partials_needed(M)) + 1;
    if ((s = alloc_dev(p->ewald_partials, sizeof(double) * (size_t)np, tot)) != NFFT_OK) return fail(s);
    if ((s = alloc_dev(p->ewald_out, sizeof(double) * 2, tot)) != NFFT_OK) return fail(s);
  }
  if (cudaMemset(p->err_flag, 0, sizeof(int)) != cudaSuccess) return fail(NFFT_ERR_CUDA);
  if (cudaMemset(p->num_subs, 0, sizeof(int)) != cudaSuccess) return fail(NFFT_ERR_CUDA);
  if ((s = alloc_sort(p)) != NFFT_OK) return fail(s);
  if ((s = alloc_grid(p, 1)) != NFFT_OK) return fail(s);
  cufftHandle h;
  if ((s = fft_handle(p, 1, &h)) != NFFT_OK) return fail(s);
  *out = p;
  return NFFT_OK;
}

int nfft_plan_destroy(nfft_plan* p) {
  if (!p) return NFFT_OK;
  cudaStreamSynchronize(p->stream);
  release_all(p);
  delete p;
  return NFFT_OK;
}

int nfft_set_points(nfft_plan* p, const double* x_dev) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  if (!x_dev && p->M > 0) return NFFT_ERR_INVALID_ARG;
  p->points_set = false;
  TRY(alloc_sort(p));
  const int s = p->precision == NFFT_FP64 ? set_points_impl<double>(p, x_dev) : set_points_impl<float>(p, x_dev);
  if (s == NFFT_OK) p->points_set = true;
  return s;
}

int nfft_adjoint(nfft_plan* p, const void* f_dev, void* fhat_dev, int R) {
  if (!p || R < 0) return NFFT_ERR_INVALID_ARG;
  if (R == 0) return NFFT_OK;
  if (!fhat_dev || (!f_dev && p->M > 0)) return NFFT_ERR_INVALID_ARG;
  if (!p->points_set) return NFFT_ERR_NOT_READY;
  return p->precision == NFFT_FP64 ? adjoint_impl<double>(p, f_dev, fhat_dev, R)
                                   : adjoint_impl<float>(p, f_dev, fhat_dev, R);
}

int nfft_forward(nfft_plan* p, const void* fhat_dev, void* f_dev, int R) {
  if (!p || R < 0) return NFFT_ERR_INVALID_ARG;
  if (R == 0) return NFFT_OK;
  if (!fhat_dev || (!f_dev && p->M > 0)) return NFFT_ERR_INVALID_ARG;
  if (!p->points_set) return NFFT_ERR_NOT_READY;
  return p->precision == NFFT_FP64 ? forward_impl<double>(p, fhat_dev, f_dev, R)
                                   : forward_impl<float>(p, fhat_dev, f_dev, R);
}

int nfft_ewald_reciprocal(nfft_plan* p, const void* q_dev, double L, double alpha, double* out) {
  if (!p || !out || !(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  if (!q_dev && p->M > 0) return NFFT_ERR_INVALID_ARG;
  if (!p->points_set) return NFFT_ERR_NOT_READY;
  TRY(p->precision == NFFT_FP64 ? ewald_impl<double>(p, q_dev, L, alpha) : ewald_impl<float>(p, q_dev, L, alpha));
  double parts[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(parts, p->ewald_out, sizeof(parts), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  out[0] = parts[0] + parts[1];
  out[1] = parts[0];
  out[2] = parts[1];
  return NFFT_OK;
}

int nfft_ewald_reciprocal_sum(nfft_plan* p, const void* S_dev, double L, double alpha, double* sum_dev) {
  if (!p || !S_dev || !sum_dev || !(L > 0.0) || !(alpha > 0.0) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  const EwaldGeom g = ewald_geom(p, L, alpha);
  const double scale = 1.0 / (2.0 * M_PI * L);
  if (p->precision == NFFT_FP64)
    CK(launch_ewald_sum<double>(static_cast<const double2*>(S_dev), false, g, p->ewald_partials, scale, 0.0, sum_dev,
                                p->stream));
  else
    CK(launch_ewald_sum<float>(static_cast<const float2*>(S_dev), false, g, p->ewald_partials, scale, 0.0, sum_dev,
                               p->stream));
  return NFFT_OK;
}

int nfft_sync(nfft_plan* p) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(p->stream));
  int flag = 0;
  CK(cudaMemcpy(&flag, p->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemset(p->err_flag, 0, sizeof(int)));
    if (flag & 2) return NFFT_ERR_TIMEOUT;
    if (flag & 1) return NFFT_ERR_DOMAIN;
  }
  return NFFT_OK;
}

int nfft_set_stream(nfft_plan* p, void* cuda_stream) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  return NFFT_OK;
}

int nfft_set_option(nfft_plan* p, int option, int64_t value) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  switch (option) {
    case NFFT_OPT_METHOD:
      if (value < NFFT_METHOD_AUTO || value > NFFT_METHOD_WARP) return NFFT_ERR_INVALID_ARG;
      p->method_opt = (int)value;
      break;
    case NFFT_OPT_BIN_0:
    case NFFT_OPT_BIN_1:
    case NFFT_OPT_BIN_2: {
      const int t = option - NFFT_OPT_BIN_0;
      if (value < 0 || t >= p->d || value > 65535) return NFFT_ERR_INVALID_ARG;
      p->bin_opt[t] = (int)value;
      break;
    }
    case NFFT_OPT_MAX_SUBPROBLEM:
      if (value < 0 || value > (1 << 20)) return NFFT_ERR_INVALID_ARG;
      p->max_sub_opt = (int)value;
      break;
    case NFFT_OPT_RHS_CAPACITY: {
      if (value < 1 || value > 4096) return NFFT_ERR_INVALID_ARG;
      CK(cudaStreamSynchronize(p->stream));
      TRY(alloc_grid(p, (int)value));
      cufftHandle h;
      TRY(fft_handle(p, (int)value, &h));
      return NFFT_OK;
    }
    case NFFT_OPT_PROFILE:
      p->profile = value != 0;
      return NFFT_OK;
    case NFFT_OPT_THREADS:
      if (value != 0 && (value < 32 || value > 256 || value % 32 != 0)) return NFFT_ERR_INVALID_ARG;
      p->threads = value == 0 ? 256 : (int)value;
      p->threads_opt = (int)value;
      return NFFT_OK;
    default:
      return NFFT_ERR_INVALID_ARG;
  }
  // bins, method or subproblem size changed: reconfigure; points must be set again
  const int s = configure_bins(p);
  p->points_set = false;
  if (s != NFFT_OK) return s;
  CK(cudaStreamSynchronize(p->stream));
  return alloc_sort(p);
}

int nfft_get_info(const nfft_plan* p, nfft_plan_info* info) {
  if (!p || !info) return NFFT_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->d = p->d;
  info->M = p->M;
  info->m = p->m;
  info->taps = p->win.taps;
  info->window = p->window;
  info->precision = p->precision;
  info->method = p->method;
  info->n_bins = 1;
  for (int t = 0; t < 3; ++t) {
    info->N[t] = p->N[t];
    info->n[t] = p->n[t];
    info->bin[t] = p->geom.bin[t];
    info->sigma[t] = t < p->d ? (double)p->n[t] / (double)p->N[t] : 1.0;
    if (t < p->d) info->n_bins *= p->geom.nbins[t];
  }
  info->rhs_capacity = p->rhs_cap;
  info->threads = p->threads;
  info->device_bytes = p->device_bytes;
  return NFFT_OK;
}

int nfft_stage_times(nfft_plan* p, double* ms, int64_t* launches, int reset) {
  if (!p || !ms) return NFFT_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(p->stream));
  for (auto& e : p->events) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e.start, e.stop));
    p->stage_ms[e.stage] += t;
    p->stage_calls[e.stage] += 1;
    p->free_events.push_back(e);
  }
  p->events.clear();
  for (int s = 0; s < NFFT_STAGE_COUNT; ++s) {
    ms[s] = p->stage_ms[s];
    if (launches) launches[s] = p->stage_calls[s];
    if (reset) {
      p->stage_ms[s] = 0;
      p->stage_calls[s] = 0;
    }
  }
  return NFFT_OK;
}

}  // extern "C"
