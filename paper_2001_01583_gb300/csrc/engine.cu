// Host engine: layout, sort, transforms and batch graphs (see engine.h).
#include "engine.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <utility>

namespace gbnfft {

namespace {

constexpr size_t kSmemBudget = 200 * 1024;   // per block (the opt-in limit is 227 KB)
constexpr size_t kSmemTarget = 100 * 1024;   // thread-per-point tiles: aim at two blocks per SM

#define CK(call)                                                             \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      cudaGetLastError();                                                    \
      return e_ == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA; \
    }                                                                        \
  } while (0)

#define TRY(x)                    \
  do {                            \
    int s_ = (x);                 \
    if (s_ != NFFT_OK) return s_; \
  } while (0)

bool is_fft_friendly(int64_t n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

int taps_for(int window, int m) { return window == NFFT_GAUSSIAN ? 2 * m + 2 : 2 * m; }

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

// The table of 1 / c_k (inv_c_at below) over k = -N/2 .. N/2-1.
std::vector<double> scaling_table(int window, int m, int64_t N, int64_t n, double b) {
  std::vector<double> out((size_t)N);
  for (int64_t a = 0; a < N; ++a) out[(size_t)a] = inv_c_at(window, m, n, b, (double)(a - N / 2));
  return out;
}

// Row pitch for the warp kernels' tiles: a warp instruction touches Q rows of
// W consecutive elements; the pitch (>= the row length) needing the fewest
// shared-memory wavefronts -- the most 4-byte words one bank must serve,
// averaged over the row's start -- wins, the smallest on ties.
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

template <typename T>
void free_dev(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <typename Real>
const void* tiled_kernel(int d, int taps, bool spread);
template <>
const void* tiled_kernel<float>(int d, int taps, bool spread) {
  return spread ? spread_tiled_kernel_f32(d, taps) : interp_tiled_kernel_f32(d, taps);
}
template <>
const void* tiled_kernel<double>(int d, int taps, bool spread) {
  return spread ? spread_tiled_kernel_f64(d, taps) : interp_tiled_kernel_f64(d, taps);
}
template <typename Real>
const void* global_kernel(bool spread);
template <>
const void* global_kernel<float>(bool spread) { return global_kernel_f32(spread); }
template <>
const void* global_kernel<double>(bool spread) { return global_kernel_f64(spread); }
template <typename Real>
const void* wpp_kernel(int d, int taps, bool spread);
template <>
const void* wpp_kernel<float>(int d, int taps, bool spread) { return wpp_kernel_f32(d, taps, spread); }
template <>
const void* wpp_kernel<double>(int d, int taps, bool spread) { return wpp_kernel_f64(d, taps, spread); }
template <typename Real>
const void* planes_kernel(int taps, int warps, bool spread);
template <>
const void* planes_kernel<float>(int taps, int warps, bool spread) { return planes_kernel_f32(taps, warps, spread); }
template <>
const void* planes_kernel<double>(int taps, int warps, bool spread) { return planes_kernel_f64(taps, warps, spread); }
template <typename Real>
size_t planes_table_bytes(int taps, int bp, int np, int nw, const int* tile, bool spread);
template <>
size_t planes_table_bytes<float>(int taps, int bp, int np, int nw, const int* tile, bool spread) {
  return planes_table_bytes_f32(taps, bp, np, nw, tile, spread);
}
template <>
size_t planes_table_bytes<double>(int taps, int bp, int np, int nw, const int* tile, bool spread) {
  return planes_table_bytes_f64(taps, bp, np, nw, tile, spread);
}

}  // namespace

double shape_param(int window, int m, double sigma) {
  if (window == NFFT_GAUSSIAN) return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * M_PI);
  if (window == NFFT_B_SPLINE) return 0.0;
  // sinc-power: sinc(pi b u) in the cell variable u
  if (window == NFFT_SINC_POWER) return (2.0 * sigma - 1.0) / (2.0 * m * sigma);
  return M_PI * (2.0 - 1.0 / sigma);
}

// 1 / c_k for k = -N/2 .. N/2-1 of one dimension, with the kernels' window
// normalisation psi = phi / phi(0):  inv_c(k) = phi(0) / (n phihat(k)).
//   Gaussian:       phi(0) = (pi b)^(-1/2),        n phihat(k) = exp(-b (pi k / n)^2)
//   Kaiser-Bessel:  phi(0) = sinh(b m) / (pi m),   n phihat(k) = I0(m sqrt(b^2 - (2 pi k / n)^2))
double cardinal_bspline(int order, double u) {
  const double s = u + 0.5 * order;
  if (!(s > 0.0 && s < (double)order)) return 0.0;
  // v[i] = N_j(s - i) of the uniform B-spline N_j (support [0, j]), raised
  // from N_1 (the indicator of [0, 1)) by N_j(s) = (s N_(j-1)(s) +
  // (j - s) N_(j-1)(s - 1)) / (j - 1): nonnegative terms only
  double v[2 * kMaxTaps + 2] = {0.0};
  const int f = (int)std::floor(s);
  v[f] = 1.0;
  for (int j = 2; j <= order; ++j)
    for (int i = 0; i <= order - j; ++i) {
      const double si = s - i;
      v[i] = (si * v[i] + (j - si) * v[i + 1]) / (j - 1);
    }
  return v[0];
}

double inv_c_at(int window, int m, int64_t n, double b, double k) {
  if (window == NFFT_GAUSSIAN) {
    const double t = M_PI * k / (double)n;
    return std::exp(b * t * t) / std::sqrt(M_PI * b);
  }
  if (window == NFFT_B_SPLINE) {
    // phi(0) = M_2m(0), n phihat(k) = sinc(pi k / n)^(2m)
    const double t = M_PI * k / (double)n;
    const double sc = t == 0.0 ? 1.0 : std::sin(t) / t;
    return cardinal_bspline(2 * m, 0.0) / std::pow(sc, 2 * m);
  }
  if (window == NFFT_SINC_POWER) {
    // phi(x) = a sinc(pi a x)^(2m) with a = n b: phi(0) = a,
    // n phihat(k) = n M_2m(k / a)
    const double a = (double)n * b;
    return a / ((double)n * cardinal_bspline(2 * m, k / a));
  }
  const double w = 2.0 * M_PI * k / (double)n;
  const double arg = m * std::sqrt(b * b - w * w);
  return std::sinh(b * m) / (M_PI * m * bessel_i0(arg));
}


// ===========================================================================
// parameters shared with nfft_plan_params

int64_t oversampled_size(int64_t N, double sigma) {
  int64_t n = (int64_t)std::ceil(sigma * (double)N - 1e-9);
  if (n < 2) n = 2;
  while (n % 2 != 0 || !is_fft_friendly(n)) ++n;
  return n;
}

int window_taps(int window, int m) { return taps_for(window, m); }

int validate_spec(const ItemSpec& s, int precision) {
  if (s.d < 1 || s.d > 3) return NFFT_ERR_INVALID_ARG;
  if (s.M < 0 || s.M > (int64_t)INT32_MAX) return NFFT_ERR_INVALID_ARG;
  if (!(s.sigma >= 1.0) || !std::isfinite(s.sigma) || s.sigma > 16.0) return NFFT_ERR_INVALID_ARG;
  if (s.m < 1) return NFFT_ERR_INVALID_ARG;
  if (s.window < NFFT_GAUSSIAN || s.window > NFFT_SINC_POWER) return NFFT_ERR_INVALID_ARG;
  if (precision != NFFT_FP64 && precision != NFFT_FP32_MIXED) return NFFT_ERR_INVALID_ARG;
  if (s.nrhs < 1 || s.nrhs > 4096) return NFFT_ERR_INVALID_ARG;
  if (taps_for(s.window, s.m) > kMaxTaps) return NFFT_ERR_UNSUPPORTED;
  int64_t cells = 1;
  for (int t = 0; t < s.d; ++t) {
    if (s.N[t] < 2 || (s.N[t] & 1) || s.N[t] > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
    const int64_t n = oversampled_size(s.N[t], s.sigma);
    if (n < 2 * s.m + 2 || n < s.N[t]) return NFFT_ERR_INVALID_ARG;
    cells *= n;
  }
  if (cells > (int64_t)INT32_MAX) return NFFT_ERR_UNSUPPORTED;
  return NFFT_OK;
}

// ===========================================================================
// lifetime

Engine::~Engine() {
  if (stream) cudaStreamSynchronize(stream);
  drop_graphs();
  if (capture_stream) cudaStreamDestroy(capture_stream);
  release_layout();
  for (auto& fc : fclasses) {
    destroy_fft_plans(fc);
    free_dev(fc.buf);
  }
  for (double* t : tables) cudaFree(t);
  free_dev(err_flag);
  free_dev(ewald_partials);
  free_dev(ewald_out);
  free_dev(force_modes);
  free_dev(force_vals);
  free_dev(d_items);
  for (int k = 0; k < 2; ++k) {
    if (h_table[k]) cudaFreeHost(h_table[k]);
    if (slot_done[k]) cudaEventDestroy(slot_done[k]);
  }
  for (auto& e : events) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
  for (auto& e : free_events) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
}

bool total_points_exceed_int32(const std::vector<ItemSpec>& specs) {
  int64_t total = 0;
  for (const auto& s : specs) {
    total += s.M;
    if (total > (int64_t)INT32_MAX) return true;
  }
  return false;
}

int Engine::init(const std::vector<ItemSpec>& in_specs, int prec, cudaStream_t st, bool is_single) {
  if (in_specs.empty()) return NFFT_ERR_INVALID_ARG;
  for (const auto& s : in_specs) TRY(validate_spec(s, prec));
  if (total_points_exceed_int32(in_specs)) return NFFT_ERR_UNSUPPORTED;
  specs = in_specs;
  precision = prec;
  csize = prec == NFFT_FP64 ? 16 : 8;
  stream = st;
  single = is_single;
  CK(cudaGetDevice(&device));
  CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  int v = 0;
  CK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  smem_optin = (size_t)v;
  CK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  smem_per_sm = (size_t)v;
  TRY(alloc_dev(err_flag, sizeof(int), device_bytes));
  CK(cudaMemset(err_flag, 0, sizeof(int)));
  TRY(alloc_dev(ewald_out, 2 * sizeof(double), device_bytes));
  if (single) {
    int64_t NN = 1;
    for (int t = 0; t < specs[0].d; ++t) NN *= specs[0].N[t];
    const int64_t np = std::max(ewald_partials_needed(NN), ewald_partials_needed(specs[0].M)) + 1;
    TRY(alloc_dev(ewald_partials, sizeof(double) * (size_t)np, device_bytes));
  }
  TRY(alloc_dev(d_items, sizeof(ItemDev) * specs.size(), device_bytes));
  if (!single) {
    for (int k = 0; k < 2; ++k) {
      CK(cudaMallocHost((void**)&h_table[k], sizeof(ItemDev) * specs.size()));
      CK(cudaEventCreateWithFlags(&slot_done[k], cudaEventDisableTiming));
    }
  }
  TRY(build_fft());
  TRY(build_layout());
  return NFFT_OK;
}

// FFT classes: items with the same (d, n); every item owns spec.nrhs grids
// (a plan: rhs_cap grids) in its class buffer.
int Engine::build_fft() {
  const int nitems = (int)specs.size();
  item_fclass.assign(nitems, -1);
  item_grid_offset.assign(nitems, 0);
  for (int i = 0; i < nitems; ++i) {
    const ItemSpec& s = specs[i];
    int64_t n[3] = {1, 1, 1};
    for (int t = 0; t < s.d; ++t) n[t] = oversampled_size(s.N[t], s.sigma);
    int found = -1;
    for (size_t c = 0; c < fclasses.size(); ++c)
      if (fclasses[c].d == s.d && fclasses[c].n[0] == n[0] && fclasses[c].n[1] == n[1] && fclasses[c].n[2] == n[2])
        found = (int)c;
    if (found < 0) {
      FClass fc;
      fc.d = s.d;
      fc.cells = 1;
      for (int t = 0; t < 3; ++t) {
        fc.n[t] = n[t];
        fc.cells *= n[t];
      }
      fc.grids = 0;
      fclasses.push_back(fc);
      found = (int)fclasses.size() - 1;
    }
    FClass& fc = fclasses[found];
    item_fclass[i] = found;
    item_grid_offset[i] = (int64_t)fc.grids * fc.cells;
    fc.grids += single ? rhs_cap : s.nrhs;
  }
  for (auto& fc : fclasses) {
    TRY(alloc_dev(fc.buf, (size_t)fc.grids * (size_t)fc.cells * csize, device_bytes));
    cufftHandle h;
    TRY(fft_handle(fc, single ? 1 : fc.grids, &h));
  }
  return NFFT_OK;
}

int Engine::release_layout() {
  free_dev(d_point_offsets);
  free_dev(d_bin_offsets);
  free_dev(d_crop_blocks);
  free_dev(d_pad_blocks);
  free_dev(bin_count);
  free_dev(bin_start);
  free_dev(sub_count);
  free_dev(sub_start);
  free_dev(scan_partials);
  free_dev(num_subs);
  free_dev(subs);
  free_dev(bin_rank);
  free_dev(perm);
  free_dev(local);
  for (int t = 0; t < 3; ++t) free_dev(delta[t]);
  device_bytes -= layout_bytes;
  layout_bytes = 0;
  return NFFT_OK;
}

// Bins, kernel classes, the internal item order, the item table and the
// sort buffers.  Re-run when the method, a bin edge or the subproblem size
// changes; points must then be set again.
int Engine::build_layout() {
  drop_graphs();
  release_layout();
  points_set = false;
  const int nitems = (int)specs.size();
  max_sub = max_sub_opt > 0 ? max_sub_opt : 1024;
  const size_t budget = smem_optin < kSmemBudget ? smem_optin : kSmemBudget;

  struct Choice {
    int bin[3], tile[3], pitch, method, taps, sparse, sparse_interp;
    bool owner, tensor, tensor_interp;
  };
  std::vector<Choice> ch(nitems);
  for (int i = 0; i < nitems; ++i) {
    const ItemSpec& s = specs[i];
    Choice& c = ch[i];
    c.taps = taps_for(s.window, s.m);
    const int defaults[3][3] = {{1024, 1, 1}, {32, 32, 1}, {8, 8, 16}};
    int64_t n[3] = {1, 1, 1};
    for (int t = 0; t < s.d; ++t) n[t] = oversampled_size(s.N[t], s.sigma);
    for (int t = 0; t < 3; ++t) c.bin[t] = 1;
    for (int t = 0; t < s.d; ++t) {
      int b = bin_opt[t] > 0 ? bin_opt[t] : defaults[s.d - 1][t];
      if (b > n[t]) b = (int)n[t];
      const int maxb = s.d == 1 ? (1 << 30) : (1 << local_bits(s.d)) - 1;
      if (b > maxb) b = maxb;
      c.bin[t] = b;
    }
    auto tile_bytes = [&](const int* bin) {
      size_t cells = 1;
      for (int t = 0; t < s.d; ++t) cells *= (size_t)(bin[t] + c.taps - 1);
      return cells * csize;
    };
    const bool explicit_bins = bin_opt[0] > 0 || bin_opt[1] > 0 || bin_opt[2] > 0;
    auto halve_largest = [&](int* bin) {
      int tmax = 0;
      for (int t = 1; t < s.d; ++t)
        if (bin[t] > bin[tmax]) tmax = t;
      if (bin[tmax] <= 2) return false;
      bin[tmax] /= 2;
      return true;
    };
    // 3-D shared-tile kernels: the padded tile plus the kernel's tables must
    // fit one block (wide windows: one block of two warps per SM at least)
    auto planes_fit = [&](const int* bin) {
      int tile[3];
      for (int t = 0; t < 3; ++t) tile[t] = bin[t] + c.taps - 1;
      const size_t wt = (size_t)tile[0] * tile[1] * choose_pitch(tile[2], c.taps, (int)csize) * csize;
      if (c.taps <= 16) return wt + 32768 <= budget;
      const size_t tables = precision == NFFT_FP64 ? planes_table_bytes_f64(c.taps, 64, 1, 2, tile, true)
                                                   : planes_table_bytes_f32(c.taps, 64, 1, 2, tile, true);
      return wt + tables <= smem_optin;
    };
    bool planes = false;
    const bool planes_built = (precision == NFFT_FP64 ? planes_kernel_f64(c.taps, 2, true)
                                                      : planes_kernel_f32(c.taps, 2, true)) != nullptr;
    if (s.d == 3 && c.taps <= kMaxPlaneTaps && planes_built) {
      int pb[3] = {c.bin[0], c.bin[1], c.bin[2]};
      while (!planes_fit(pb) && !explicit_bins && halve_largest(pb)) {
      }
      if (planes_fit(pb)) {
        planes = true;
        for (int t = 0; t < 3; ++t) c.bin[t] = pb[t];
      }
    }
    // tensor-core spreading: the tile's (z, y) rows are the MMA's M = 128
    // rows and its x columns (complex) its N <= 112 columns
    c.tensor = c.tensor_interp = false;
    if ((tensor_enabled || tensor_interp_enabled) && planes && precision == NFFT_FP32_MIXED &&
        s.window != NFFT_B_SPLINE && (method_opt == NFFT_METHOD_AUTO || method_opt == NFFT_METHOD_WARP) &&
        tc_spread_kernel_f32(c.taps)) {
      if (!explicit_bins) {
        const int want[3] = {12 - c.taps, 12 - c.taps, 16};
        for (int t = 0; t < 3; ++t) c.bin[t] = (int)std::min<int64_t>(want[t], n[t]);
      }
      const int t0 = c.bin[0] + c.taps - 1, t1 = c.bin[1] + c.taps - 1, t2 = c.bin[2] + c.taps - 1;
      if (t0 * t1 > kTcRowsHost || 2 * t2 > kTcMaxColsHost) return NFFT_ERR_UNSUPPORTED;
      c.tensor = tensor_enabled;
      c.tensor_interp = tensor_interp_enabled;
    }
    if (!planes)
      while (tile_bytes(c.bin) > budget && !explicit_bins && halve_largest(c.bin)) {
      }
    for (int t = 0; t < 3; ++t) c.tile[t] = t < s.d ? c.bin[t] + c.taps - 1 : 1;
    c.pitch = choose_pitch(c.tile[s.d - 1], c.taps, (int)csize);
    size_t rows = 1;
    for (int t = 0; t + 1 < s.d; ++t) rows *= (size_t)c.tile[t];
    const size_t wtile = rows * (size_t)c.pitch * csize;
    const bool tiled_ok = tile_bytes(c.bin) <= budget && c.taps <= (s.d == 3 ? 26 : 32);
    const bool warp_ok = s.d == 3 ? planes : (s.d == 2 && c.taps <= 16 && 2 * wtile + 4096 <= budget);
    const bool gm_ok = (precision == NFFT_FP64 ? gm_kernel_f64(s.d, c.taps, true) : gm_kernel_f32(s.d, c.taps, true)) !=
                       nullptr;
    int method = method_opt;
    // no tile fits (wide FP64 windows): a warp per point straight on the grid
    // (vector atomics along grid rows) before the thread-per-point global kernel
    if (method == NFFT_METHOD_AUTO)
      method = warp_ok ? NFFT_METHOD_WARP
                       : (tiled_ok ? NFFT_METHOD_TILED : (gm_ok ? NFFT_METHOD_GRID_WARP : NFFT_METHOD_GLOBAL));
    // B-spline windows run on the global kernels only (the others keep their
    // registers free of its evaluation)
    if (s.window == NFFT_B_SPLINE) {
      if (method_opt != NFFT_METHOD_AUTO && method_opt != NFFT_METHOD_GLOBAL) return NFFT_ERR_UNSUPPORTED;
      method = NFFT_METHOD_GLOBAL;
    }
    if (method == NFFT_METHOD_TILED && !tiled_ok) return NFFT_ERR_UNSUPPORTED;
    if (method == NFFT_METHOD_WARP && !warp_ok) return NFFT_ERR_UNSUPPORTED;
    if (method == NFFT_METHOD_GRID_WARP && !gm_ok) return NFFT_ERR_UNSUPPORTED;
    c.method = method;
    // with AUTO, subproblems too small to pay for a tile go to the grid-warp
    // kernels: spreading below one point per W^d / 2 tile cells (the grid-warp
    // spread is bound by its atomics), interpolation below one point per
    // W^d / 5 tile cells (its gathers are cheaper than a tile load)
    c.sparse = c.sparse_interp = 0;
    if (method_opt == NFFT_METHOD_AUTO && gm_ok && (method == NFFT_METHOD_WARP || method == NFFT_METHOD_TILED)) {
      double cells = 1.0, foot = 1.0;
      for (int t = 0; t < s.d; ++t) {
        cells *= c.tile[t];
        foot *= c.taps;
      }
      auto pick = [&](int opt, double per_cell) {
        if (opt < 0) return 0;
        if (opt > 0) return opt;
        return std::max(1, std::min((int)std::ceil(per_cell * cells / foot), max_sub));
      };
      c.sparse = pick(sparse_opt, 2.0);
      c.sparse_interp = pick(sparse_interp_opt, 5.0);
    }
    // 3-D sparse bins spread by their cells' owners (no atomics): needs one
    // periodic image per footprint (n_t >= bin_t + W - 1) and the warps'
    // tiles in shared memory
    c.owner = false;
    if (s.d == 3 && c.sparse > 0 && owner_enabled) {
      const bool built = (precision == NFFT_FP64 ? owner_kernel_f64(c.taps) : owner_kernel_f32(c.taps)) != nullptr;
      bool fits = built;
      for (int t = 0; t < 3; ++t) {
        fits = fits && n[t] >= (int64_t)c.bin[t] + c.taps - 1;
        // bins within the reach (bin + W - 1 cells, possibly split in two by the wrap)
        fits = fits && (c.bin[t] + c.taps - 2) / c.bin[t] + 3 <= kOwnerReachHost;
      }
      const size_t osmem = (size_t)kOwnerWarpsHost *
                           ((size_t)c.bin[0] * c.bin[1] * c.bin[2] * csize + (size_t)3 * c.taps * (csize / 2));
      c.owner = fits && osmem <= smem_optin;
    }
  }
  // group items into kernel classes (stable by first appearance)
  // (items with different right-hand-side counts get their own launch: the
  // right-hand sides per pass size the shared memory of the whole launch)
  auto same = [&](int a, int b) {
    return specs[a].d == specs[b].d && ch[a].taps == ch[b].taps && specs[a].window == specs[b].window &&
           (single || specs[a].nrhs == specs[b].nrhs) &&
           ch[a].method == ch[b].method && ch[a].sparse == ch[b].sparse &&
           ch[a].sparse_interp == ch[b].sparse_interp && ch[a].owner == ch[b].owner && ch[a].bin[0] == ch[b].bin[0] &&
           ch[a].bin[1] == ch[b].bin[1] &&
           ch[a].bin[2] == ch[b].bin[2];
  };
  std::vector<int> rep;
  std::vector<int> cls(nitems);
  for (int i = 0; i < nitems; ++i) {
    int found = -1;
    for (size_t r = 0; r < rep.size(); ++r)
      if (same(i, rep[r])) found = (int)r;
    if (found < 0) {
      rep.push_back(i);
      found = (int)rep.size() - 1;
    }
    cls[i] = found;
  }
  order.clear();
  for (size_t r = 0; r < rep.size(); ++r)
    for (int i = 0; i < nitems; ++i)
      if (cls[i] == (int)r) order.push_back(i);

  // items in internal order
  items.assign(nitems, ItemDev{});
  kclasses.clear();
  std::vector<int64_t> pts_off(nitems + 1, 0);
  std::vector<int> bin_off(nitems + 1, 0);
  max_subs_total = 0;
  for (int k = 0; k < nitems; ++k) {
    const int u = order[k];
    const ItemSpec& s = specs[u];
    const Choice& c = ch[u];
    ItemDev& it = items[k];
    std::memset(&it, 0, sizeof(it));
    GridGeom& g = it.geom;
    g.d = s.d;
    g.grid_cells = 1;
    g.tile_cells = 1;
    int nb_total = 1;
    for (int t = 0; t < 3; ++t) {
      const int64_t n = t < s.d ? oversampled_size(s.N[t], s.sigma) : 1;
      g.n[t] = (int)n;
      g.bin[t] = c.bin[t];
      g.nbins[t] = (int)((n + c.bin[t] - 1) / c.bin[t]);
      g.tile[t] = c.tile[t];
      g.grid_cells *= n;
      g.tile_cells *= c.tile[t];
      nb_total *= g.nbins[t];
      it.N[t] = t < s.d ? (int)s.N[t] : 1;
    }
    it.NN = 1;
    for (int t = 0; t < s.d; ++t) it.NN *= s.N[t];
    it.M = s.M;
    it.nrhs = single ? 1 : s.nrhs;
    WindowDev& w = it.win;
    w.kind = s.window;
    w.m = s.m;
    w.shift = s.window == NFFT_GAUSSIAN ? 0 : 1;
    w.taps = c.taps;
    for (int t = 0; t < 3; ++t) {
      const double sig = t < s.d ? (double)g.n[t] / (double)s.N[t] : 2.0;
      const double b = shape_param(s.window, s.m, sig);
      w.b[t] = b;
      w.kb_norm[t] = s.window == NFFT_KAISER_BESSEL ? 1.0 / (1.0 - std::exp(-2.0 * b * s.m))
                     : (s.window == NFFT_B_SPLINE ? 1.0 / cardinal_bspline(2 * s.m, 0.0) : 1.0);
      w.bf[t] = (float)w.b[t];
      w.kb_normf[t] = (float)w.kb_norm[t];
      w.binvf[t] = w.b[t] != 0.0 ? (float)(1.0 / w.b[t]) : 0.0f;
      if (t < s.d) {
        const auto key = std::make_tuple(s.window, s.N[t], (int64_t)g.n[t], s.m, 0);
        auto f = table_cache.find(key);
        if (f == table_cache.end()) {
          std::vector<double> tab = scaling_table(s.window, s.m, s.N[t], g.n[t], b);
          double* dtab = nullptr;
          TRY(alloc_dev(dtab, sizeof(double) * tab.size(), device_bytes));
          CK(cudaMemcpy(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
          tables.push_back(dtab);
          f = table_cache.emplace(key, dtab).first;
        }
        it.inv_c[t] = f->second;
      }
    }
    FClass& fc = fclasses[item_fclass[u]];
    it.grid = static_cast<char*>(fc.buf) + item_grid_offset[u] * (int64_t)csize;
    it.point_offset = pts_off[k];
    it.bin_offset = bin_off[k];
    pts_off[k + 1] = pts_off[k] + s.M;
    bin_off[k + 1] = bin_off[k] + nb_total;
    max_subs_total += nb_total + s.M / max_sub + 1;
    if ((int64_t)bin_off[k + 1] > ((int64_t)1 << 30)) return NFFT_ERR_UNSUPPORTED;
    // kernel class bookkeeping
    if (kclasses.empty() || cls[u] != cls[order[kclasses.back().item_begin]]) {
      KClass kc{};
      kc.d = s.d;
      kc.taps = c.taps;
      kc.window = s.window;
      kc.method = c.method;
      for (int t = 0; t < 3; ++t) {
        kc.bin[t] = c.bin[t];
        kc.tile[t] = c.tile[t];
      }
      kc.pitch = c.pitch;
      kc.sparse_points = c.sparse;
      kc.sparse_points_interp = c.sparse_interp;
      kc.owner = c.owner;
      kc.tensor = c.tensor;
      kc.tensor_interp = c.tensor_interp;
      kc.item_begin = k;
      kc.bin_begin = bin_off[k];
      kc.max_nrhs = 0;
      kc.max_subs = 0;
      kclasses.push_back(kc);
    }
    KClass& kc = kclasses.back();
    kc.item_end = k + 1;
    kc.bin_end = bin_off[k + 1];
    kc.max_nrhs = std::max(kc.max_nrhs, it.nrhs);
    kc.max_subs += nb_total + s.M / max_sub + 1;
  }
  total_points = pts_off[nitems];
  if (total_points > (int64_t)INT32_MAX) return NFFT_ERR_UNSUPPORTED;   // 32-bit sort indices
  // an FFT class needs no clearing before spreading when the owner kernel
  // writes every grid in it
  for (auto& fc : fclasses) fc.owner_written = true;
  for (const auto& kc : kclasses)
    for (int k = kc.item_begin; k < kc.item_end; ++k)
      if (!kc.owner) fclasses[item_fclass[order[k]]].owner_written = false;
  total_bins = bin_off[nitems];
  // device buffers
  int64_t before = device_bytes;
  const size_t P = (size_t)std::max<int64_t>(total_points, 1);
  const size_t B = (size_t)std::max(total_bins, 1);
  TRY(alloc_dev(d_point_offsets, sizeof(int64_t) * (nitems + 1), device_bytes));
  TRY(alloc_dev(d_bin_offsets, sizeof(int) * (nitems + 1), device_bytes));
  TRY(alloc_dev(bin_count, sizeof(int) * B, device_bytes));
  TRY(alloc_dev(bin_start, sizeof(int) * B, device_bytes));
  TRY(alloc_dev(sub_count, sizeof(int) * B, device_bytes));
  TRY(alloc_dev(sub_start, sizeof(int) * B, device_bytes));
  TRY(alloc_dev(scan_partials, sizeof(int) * (size_t)scan_partials_needed((int)B), device_bytes));
  TRY(alloc_dev(num_subs, sizeof(int), device_bytes));
  TRY(alloc_dev(subs, sizeof(SubProblem) * (size_t)max_subs_total, device_bytes));
  TRY(alloc_dev(bin_rank, sizeof(int2) * P, device_bytes));
  TRY(alloc_dev(perm, sizeof(int) * P, device_bytes));
  TRY(alloc_dev(local, sizeof(uint32_t) * P, device_bytes));
  const int dmax = [&] {
    int m = 1;
    for (const auto& s : specs) m = std::max(m, s.d);
    return m;
  }();
  const size_t rsize = precision == NFFT_FP64 ? 8 : 4;
  for (int t = 0; t < dmax; ++t) TRY(alloc_dev(delta[t], rsize * P, device_bytes));
  layout_bytes = device_bytes - before;
  {
    std::vector<int> cb(nitems + 1, 0), pb(nitems + 1, 0);
    for (int k = 0; k < nitems; ++k) {
      const ItemDev& it = items[k];
      const int dl = it.geom.d - 1;
      cb[k + 1] = cb[k] + (int)scale_blocks(it.NN / it.N[dl] * it.nrhs, it.N[dl], true);
      pb[k + 1] = pb[k] + (int)scale_blocks(it.geom.grid_cells / it.geom.n[dl] * it.nrhs, it.geom.n[dl], true);
    }
    crop_blocks = cb[nitems];
    pad_blocks = pb[nitems];
    // [prefix sums (nitems + 1) | item of every block], for crop and for pad
    auto table = [&](const std::vector<int>& pre, int64_t blocks) {
      std::vector<int> t(pre);
      t.reserve((size_t)(nitems + 1 + blocks));
      for (int k = 0; k < nitems; ++k)
        for (int b = pre[k]; b < pre[k + 1]; ++b) t.push_back(k);
      return t;
    };
    const std::vector<int> ct = table(cb, crop_blocks), pt = table(pb, pad_blocks);
    TRY(alloc_dev(d_crop_blocks, sizeof(int) * ct.size(), device_bytes));
    TRY(alloc_dev(d_pad_blocks, sizeof(int) * pt.size(), device_bytes));
    layout_bytes += (int64_t)(sizeof(int) * (ct.size() + pt.size()));
    CK(cudaMemcpy(d_crop_blocks, ct.data(), sizeof(int) * ct.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_pad_blocks, pt.data(), sizeof(int) * pt.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(d_point_offsets, pts_off.data(), sizeof(int64_t) * (nitems + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_bin_offsets, bin_off.data(), sizeof(int) * (nitems + 1), cudaMemcpyHostToDevice));
  CK(cudaMemset(num_subs, 0, sizeof(int)));
  CK(cudaMemset(sub_start, 0, sizeof(int) * B));
  CK(cudaMemcpy(d_items, items.data(), sizeof(ItemDev) * nitems, cudaMemcpyHostToDevice));
  if (!single)
    for (int k = 0; k < 2; ++k) std::memcpy(h_table[k], items.data(), sizeof(ItemDev) * nitems);
  return NFFT_OK;
}

int Engine::fft_handle(FClass& fc, int batch, cufftHandle* out) {
  auto it = fc.plans.find(batch);
  if (it != fc.plans.end()) {
    *out = it->second;
    return cufftSetStream(it->second, stream) == CUFFT_SUCCESS ? NFFT_OK : NFFT_ERR_CUFFT;
  }
  cufftHandle h;
  if (cufftCreate(&h) != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
  long long dims[3];
  for (int t = 0; t < fc.d; ++t) dims[t] = fc.n[t];
  size_t work = 0;
  const cufftType type = precision == NFFT_FP64 ? CUFFT_Z2Z : CUFFT_C2C;
  const cufftResult r =
      cufftMakePlanMany64(h, fc.d, dims, nullptr, 1, fc.cells, nullptr, 1, fc.cells, type, batch, &work);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return r == CUFFT_ALLOC_FAILED ? NFFT_ERR_OOM : NFFT_ERR_CUFFT;
  }
  if (cufftSetStream(h, stream) != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return NFFT_ERR_CUFFT;
  }
  fc.plans[batch] = h;
  *out = h;
  return NFFT_OK;
}

void Engine::destroy_fft_plans(FClass& fc) {
  for (auto& kv : fc.plans) cufftDestroy(kv.second);
  fc.plans.clear();
  if (fc.prune_z) cufftDestroy(fc.prune_z);
  if (fc.prune_yx) cufftDestroy(fc.prune_yx);
  fc.prune_z = fc.prune_yx = 0;
  fc.prune_built = false;
}

// The FFT of a single 3-D item split by dimension (NFFT_OPT_PRUNED_FFT): the
// frequencies of I_N sit in the planes 0 .. N_0 / 2 - 1 and
// n_0 - N_0 / 2 .. n_0 - 1 of dimension 0 (k < 0 wraps to k + n_0).
// Automatic choice: grids of at least 128 MiB (larger than the L2 cache);
// a smaller grid's single 3-D cuFFT runs from L2 and beats three launches.
constexpr double kPruneMinBytes = 134217728.0;

bool Engine::fft_pruned(const FClass& fc) const {
  if (!(single && fc.d == 3 && !items.empty() && items[0].N[0] < fc.n[0])) return false;
  if (pruned_fft_mode >= 0) return pruned_fft_mode == 1;
  return (double)fc.cells * (double)csize >= kPruneMinBytes;
}

int Engine::build_pruned(FClass& fc) {
  if (fc.prune_built) return NFFT_OK;
  const cufftType type = precision == NFFT_FP64 ? CUFFT_Z2Z : CUFFT_C2C;
  const long long plane = fc.n[1] * fc.n[2];
  long long nz[1] = {fc.n[0]};
  long long nyx[2] = {fc.n[1], fc.n[2]};
  size_t work = 0;
  cufftHandle hz = 0, hyx = 0;
  if (cufftCreate(&hz) != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
  // lines along dimension 0: element stride n_1 n_2, one line per (y, x)
  cufftResult r = cufftMakePlanMany64(hz, 1, nz, nz, plane, 1, nz, plane, 1, type, plane, &work);
  if (r == CUFFT_SUCCESS && cufftCreate(&hyx) != CUFFT_SUCCESS) r = CUFFT_INTERNAL_ERROR;
  // N_0 / 2 contiguous planes of n_1 x n_2
  if (r == CUFFT_SUCCESS)
    r = cufftMakePlanMany64(hyx, 2, nyx, nyx, 1, plane, nyx, 1, plane, type, items[0].N[0] / 2, &work);
  if (r == CUFFT_SUCCESS && (cufftSetStream(hz, stream) != CUFFT_SUCCESS || cufftSetStream(hyx, stream) != CUFFT_SUCCESS))
    r = CUFFT_INTERNAL_ERROR;
  if (r != CUFFT_SUCCESS) {
    if (hz) cufftDestroy(hz);
    if (hyx) cufftDestroy(hyx);
    return r == CUFFT_ALLOC_FAILED ? NFFT_ERR_OOM : NFFT_ERR_CUFFT;
  }
  fc.prune_z = hz;
  fc.prune_yx = hyx;
  fc.prune_built = true;
  return NFFT_OK;
}

int Engine::run_fft(FClass& fc, int batch, int64_t grid_offset, int direction) {
  if (fft_pruned(fc)) {
    TRY(build_pruned(fc));
    if (cufftSetStream(fc.prune_z, stream) != CUFFT_SUCCESS || cufftSetStream(fc.prune_yx, stream) != CUFFT_SUCCESS)
      return NFFT_ERR_CUFFT;
    const int64_t plane = fc.n[1] * fc.n[2];
    const int64_t upper = (fc.n[0] - items[0].N[0] / 2) * plane;   // first plane of the k < 0 run
    for (int b = 0; b < batch; ++b) {
      const int64_t g0 = grid_offset + (int64_t)b * fc.cells;
      cufftResult r = CUFFT_SUCCESS;
      auto exec = [&](cufftHandle h, int64_t off) {
        if (r != CUFFT_SUCCESS) return;
        if (precision == NFFT_FP64) {
          cufftDoubleComplex* g = static_cast<cufftDoubleComplex*>(fc.buf) + off;
          r = cufftExecZ2Z(h, g, g, direction);
        } else {
          cufftComplex* g = static_cast<cufftComplex*>(fc.buf) + off;
          r = cufftExecC2C(h, g, g, direction);
        }
      };
      if (direction == CUFFT_FORWARD) {   // adjoint: every line along 0, then the kept planes
        exec(fc.prune_z, g0);
        exec(fc.prune_yx, g0);
        exec(fc.prune_yx, g0 + upper);
      } else {                            // forward: the filled planes, then every line along 0
        exec(fc.prune_yx, g0);
        exec(fc.prune_yx, g0 + upper);
        exec(fc.prune_z, g0);
      }
      if (r != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
    }
    return NFFT_OK;
  }
  cufftHandle h;
  TRY(fft_handle(fc, batch, &h));
  cufftResult r;
  if (precision == NFFT_FP64) {
    cufftDoubleComplex* g = static_cast<cufftDoubleComplex*>(fc.buf) + grid_offset;
    r = cufftExecZ2Z(h, g, g, direction);
  } else {
    cufftComplex* g = static_cast<cufftComplex*>(fc.buf) + grid_offset;
    r = cufftExecC2C(h, g, g, direction);
  }
  return r == CUFFT_SUCCESS ? NFFT_OK : NFFT_ERR_CUFFT;
}

// ===========================================================================
// profiling

int Engine::stage_begin(int stage, EventPair* ev) {
  if (!profile) return NFFT_OK;
  if (!free_events.empty()) {
    *ev = free_events.back();
    free_events.pop_back();
  } else {
    CK(cudaEventCreate(&ev->start));
    CK(cudaEventCreate(&ev->stop));
  }
  ev->stage = stage;
  CK(cudaEventRecord(ev->start, stream));
  return NFFT_OK;
}

int Engine::stage_end(EventPair* ev) {
  if (!profile) return NFFT_OK;
  CK(cudaEventRecord(ev->stop, stream));
  events.push_back(*ev);
  return NFFT_OK;
}

int Engine::stage_times(double* ms, int64_t* launches, int reset) {
  CK(cudaStreamSynchronize(stream));
  for (auto& e : events) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e.start, e.stop));
    stage_ms[e.stage] += t;
    stage_calls[e.stage] += 1;
    free_events.push_back(e);
  }
  events.clear();
  for (int s = 0; s < NFFT_STAGE_COUNT; ++s) {
    ms[s] = stage_ms[s];
    if (launches) launches[s] = stage_calls[s];
    if (reset) {
      stage_ms[s] = 0;
      stage_calls[s] = 0;
    }
  }
  return NFFT_OK;
}

int Engine::blocks_per_sm(const void* fn, int threads, size_t smem) {
  const auto key = std::make_tuple(fn, threads, smem);
  auto it = occupancy.find(key);
  if (it != occupancy.end()) return it->second;
  int nb = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 0;
  }
  occupancy[key] = nb;
  return nb;
}

// ===========================================================================
// point kernels

template <typename Real>
int Engine::run_points(const KClass& kc, bool spread, const void* in, void* out, int nrhs) {
  PointKernelArgs<Real> a{};
  a.pts.perm = perm;
  a.pts.local = local;
  for (int t = 0; t < 3; ++t) a.pts.delta[t] = static_cast<const Real*>(delta[t]);
  a.pts.subs = subs;
  a.pts.sub_start = sub_start;
  a.pts.num_subs = num_subs;
  a.pts.bin_count = bin_count;
  a.pts.bin_start = bin_start;
  a.items = d_items;
  a.item_begin = kc.item_begin;
  a.item_end = kc.item_end;
  a.bin_begin = kc.bin_begin;
  a.bin_end = kc.bin_end;
  a.total_bins = total_bins;
  a.in = in;
  a.out = out;
  a.nrhs = nrhs;
  const int max_nrhs = in ? nrhs : kc.max_nrhs;
  a.sub_min_count = 0;
  a.sub_max_count = INT_MAX;
  a.err = err_flag;
  if (kc.method == NFFT_METHOD_GRID_WARP) return run_gm<Real>(kc, a, spread);
  if (kc.method == NFFT_METHOD_GLOBAL) return run_global<Real>(kc, a, spread);
  // tiled kernels take the bins of at least `split` points, the owner
  // kernel (3-D spreading, first: it writes every cell) or the grid-warp
  // kernels the rest
  const int split = spread ? kc.sparse_points : kc.sparse_points_interp;
  if (spread && kc.owner) {
    TRY(run_owner<Real>(kc, a));
    a.sub_min_count = split;
    return kc.method == NFFT_METHOD_WARP ? run_planes<Real>(kc, a, spread, max_nrhs)
                                         : run_tiled<Real>(kc, a, spread, max_nrhs);
  }
  a.sub_min_count = split;
  int st;
  if constexpr (sizeof(Real) == 4) {
    if (spread ? kc.tensor : kc.tensor_interp) {
      st = run_tc(kc, a, spread);
    } else {
      st = kc.method == NFFT_METHOD_WARP
               ? (kc.d == 3 ? run_planes<Real>(kc, a, spread, max_nrhs) : run_wpp<Real>(kc, a, spread, max_nrhs))
               : run_tiled<Real>(kc, a, spread, max_nrhs);
    }
  } else {
    st = kc.method == NFFT_METHOD_WARP
             ? (kc.d == 3 ? run_planes<Real>(kc, a, spread, max_nrhs) : run_wpp<Real>(kc, a, spread, max_nrhs))
             : run_tiled<Real>(kc, a, spread, max_nrhs);
  }
  if (st != NFFT_OK || split <= 0) return st;
  a.sub_min_count = 0;
  a.sub_max_count = split;
  return run_gm<Real>(kc, a, spread);
}

// A warp per owner bin; the launch covers every bin of the class.
template <typename Real>
int Engine::run_owner(const KClass& kc, PointKernelArgs<Real>& a) {
  const void* fn = precision == NFFT_FP64 ? owner_kernel_f64(kc.taps) : owner_kernel_f32(kc.taps);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  const int threads = 32 * kOwnerWarpsHost;
  const size_t smem = (size_t)kOwnerWarpsHost *
                      ((size_t)kc.bin[0] * kc.bin[1] * kc.bin[2] * csize + (size_t)3 * kc.taps * (csize / 2));
  const int per_sm = std::max(1, blocks_per_sm(fn, threads, smem));
  int64_t blocks = (int64_t)per_sm * num_sms;
  const int64_t need = ((int64_t)(kc.bin_end - kc.bin_begin) + kOwnerWarpsHost - 1) / kOwnerWarpsHost;
  if (blocks > need) blocks = need;
  if (blocks < 1) return NFFT_OK;
  const int sparse_below = kc.sparse_points;
  void* args[] = {&a, (void*)&sparse_below};
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(threads), args, smem, stream));
  ++kernel_launches;
  return NFFT_OK;
}

// One warp per point straight on the grid; kGmSplitHost warps share a subproblem.
template <typename Real>
int Engine::run_gm(const KClass& kc, PointKernelArgs<Real>& a, bool spread) {
  const void* fn = precision == NFFT_FP64 ? gm_kernel_f64(kc.d, kc.taps, spread) : gm_kernel_f32(kc.d, kc.taps, spread);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = 1;
  const int threads = 32 * kGmWarpsHost;
  const int per_sm = std::max(1, blocks_per_sm(fn, threads, 0));
  int64_t blocks = (int64_t)per_sm * num_sms;
  const int64_t need = (kc.max_subs * kGmSplitHost + kGmWarpsHost - 1) / kGmWarpsHost;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(threads), args, 0, stream));
  ++kernel_launches;
  return NFFT_OK;
}

// 3-D: one shared tile per block.  Spreading splits the tile's planes among
// the block's warps (a power of two dividing the taps); interpolation gives
// each warp groups of points.  Warps per block: the option if set, else the
// most resident warps (ties: fewer warps per block).  Right-hand sides per
// pass fit two blocks per SM.
template <typename Real>
int Engine::run_planes(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs) {
  const int W = kc.taps;
  const size_t rows = (size_t)kc.tile[0] * kc.tile[1];
  const size_t tbytes = rows * (size_t)kc.pitch * csize;
  auto smem_of = [&](int nw, int np) {
    return (size_t)np * tbytes + planes_table_bytes<Real>(W, 32 * nw, np, nw, kc.tile, spread);
  };
  int np = 1;
  while (np < max_nrhs && smem_of(8, np + 1) <= smem_per_sm / 2) ++np;
  int best_nw = 0, best_warps = 0;
  size_t best_smem = 0;
  const void* best_fn = nullptr;
  const int topt = (spread ? spread_threads_opt : interp_threads_opt) > 0
                       ? (spread ? spread_threads_opt : interp_threads_opt)
                       : threads_opt;
  for (int nw = 1; nw <= 8; nw *= 2) {
    if (topt > 0 && 32 * nw != topt) continue;
    const void* fn = planes_kernel<Real>(W, nw, spread);
    if (!fn) continue;
    const size_t smem = smem_of(nw, np);
    if (smem > smem_optin) continue;
    const int per_sm = blocks_per_sm(fn, 32 * nw, smem);
    if (per_sm * nw > best_warps) {
      best_warps = per_sm * nw;
      best_nw = nw;
      best_smem = smem;
      best_fn = fn;
    }
  }
  if (!best_fn || best_warps == 0) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = np;
  WppLayout lay{kc.pitch, (int)(rows * kc.pitch), best_nw};
  int64_t blocks = (int64_t)(best_warps / best_nw) * num_sms;
  if (blocks > kc.max_subs) blocks = kc.max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a, &lay};
  CK(cudaFuncSetAttribute(best_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_smem));
  CK(cudaLaunchKernel(best_fn, dim3((unsigned)blocks), dim3(32 * best_nw), args, best_smem, stream));
  ++kernel_launches;
  (spread ? last_spread_threads : last_interp_threads) = 32 * best_nw;
  return NFFT_OK;
}

// 3-D dense bins spread on the tensor cores: a block of kTcThreadsHost
// threads per subproblem, the tile in tensor memory (points_tc.cuh).
int Engine::run_tc(const KClass& kc, PointKernelArgs<float>& a, bool spread) {
  const void* fn = spread ? tc_spread_kernel_f32(kc.taps) : tc_interp_kernel_f32(kc.taps);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  TcLaunch lay{};
  lay.ncols = (2 * kc.tile[2] + 15) / 16 * 16;
  int part = 32;   // columns of one accumulator: spreading holds two chunk partials and the tile (four)
  while (part < lay.ncols) part *= 2;
  lay.tmem_cols = spread ? 4 * part : part;
  if (kc.tile[0] * kc.tile[1] > kTcRowsHost || lay.ncols > kTcMaxColsHost) return NFFT_ERR_UNSUPPORTED;
  size_t smem = spread ? tc_spread_smem_bytes(kc.taps, lay.ncols, kc.tile)
                       : tc_interp_smem_bytes_host(kc.taps, lay.ncols, kc.tile);
  // blocks resident on an SM must not ask for more than its 512 tensor-memory
  // columns (an allocation that does not fit waits for another block to
  // free its columns): pad the shared memory so that at most 512 / tmem_cols
  // blocks fit
  const size_t max_blocks = (size_t)(512 / lay.tmem_cols);
  if (max_blocks >= 1 && smem * (max_blocks + 1) <= smem_per_sm) smem = smem_per_sm / (max_blocks + 1) + 1024;
  if (smem > smem_optin) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = 1;
  // blocks that fit an SM's shared memory (each also holds 1 KB for the
  // system) and its 512 tensor-memory columns
  int per_sm = std::max(1, (int)(smem_per_sm / (smem + 1024)));
  per_sm = std::min(per_sm, 512 / lay.tmem_cols);
  int64_t blocks = (int64_t)per_sm * num_sms;
  if (blocks > kc.max_subs) blocks = kc.max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a, &lay};
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kTcThreadsHost), args, smem, stream));
  ++kernel_launches;
  (spread ? last_spread_threads : last_interp_threads) = kTcThreadsHost;
  return NFFT_OK;
}

// 2-D warp per point: private tiles for spreading, one shared tile for
// interpolation.
template <typename Real>
int Engine::run_wpp(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs) {
  const int D = kc.d, W = kc.taps;
  const void* fn = wpp_kernel<Real>(D, W, spread);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  size_t rows = 1;
  for (int t = 0; t + 1 < D; ++t) rows *= (size_t)kc.tile[t];
  const size_t elems = rows * (size_t)kc.pitch;
  const size_t tbytes = elems * csize;
  const size_t scratch = (size_t)(32 * D * W + (D == 3 ? W * W : W)) * (csize / 2);
  int np = 1;
  if (spread) {
    while (np < max_nrhs && 4 * (size_t)(np + 1) * tbytes + 4 * scratch <= smem_per_sm) ++np;
  } else {
    while (np < max_nrhs && (size_t)(np + 1) * tbytes + 8 * scratch <= smem_per_sm / 2) ++np;
  }
  int best_nw = 0, best_warps = 0;
  size_t best_smem = 0;
  for (int nw = 1; nw <= 8; ++nw) {
    const size_t smem = spread ? (size_t)nw * ((size_t)np * tbytes + scratch + (size_t)np * 32 * csize)
                               : (size_t)np * tbytes + nw * scratch;
    if (smem > smem_optin) break;
    const int per_sm = blocks_per_sm(fn, 32 * nw, smem);
    if (per_sm * nw > best_warps) {
      best_warps = per_sm * nw;
      best_nw = nw;
      best_smem = smem;
    }
  }
  if (best_nw == 0) return NFFT_ERR_UNSUPPORTED;
  a.rhs_per_pass = np;
  WppLayout lay{kc.pitch, (int)elems, best_nw};
  int64_t blocks = (int64_t)(best_warps / best_nw) * num_sms;
  if (blocks > kc.max_subs) blocks = kc.max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a, &lay};
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)best_smem));
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(32 * best_nw), args, best_smem, stream));
  ++kernel_launches;
  (spread ? last_spread_threads : last_interp_threads) = 32 * best_nw;
  return NFFT_OK;
}

// Thread per point with a shared tile (shared-memory atomics for spreading).
template <typename Real>
int Engine::run_tiled(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs) {
  const void* fn = tiled_kernel<Real>(kc.d, kc.taps, spread);
  if (!fn) return NFFT_ERR_UNSUPPORTED;
  size_t cells = 1;
  for (int t = 0; t < kc.d; ++t) cells *= (size_t)kc.tile[t];
  const size_t one = cells * csize;
  size_t budget = smem_optin < kSmemBudget ? smem_optin : kSmemBudget;
  if (budget > kSmemTarget && one <= kSmemTarget) budget = kSmemTarget;
  int pass = (int)(budget / one);
  if (pass < 1) pass = 1;
  if (pass > max_nrhs) pass = max_nrhs;
  a.rhs_per_pass = pass;
  const size_t smem = one * (size_t)pass;
  const int topt = (spread ? spread_threads_opt : interp_threads_opt) > 0
                       ? (spread ? spread_threads_opt : interp_threads_opt)
                       : threads_opt;
  const int threads = topt > 0 ? topt : 256;
  int per_sm = blocks_per_sm(fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = (int64_t)per_sm * num_sms;
  if (blocks > kc.max_subs) blocks = kc.max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(threads), args, smem, stream));
  ++kernel_launches;
  (spread ? last_spread_threads : last_interp_threads) = threads;
  return NFFT_OK;
}

template <typename Real>
int Engine::run_global(const KClass& kc, PointKernelArgs<Real>& a, bool spread) {
  const void* fn = global_kernel<Real>(spread);
  a.rhs_per_pass = 1;
  int64_t blocks = (int64_t)8 * num_sms;
  if (blocks > kc.max_subs) blocks = kc.max_subs;
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  const int threads = threads_opt > 0 ? threads_opt : 256;
  CK(cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(threads), args, 0, stream));
  ++kernel_launches;
  return NFFT_OK;
}

// ===========================================================================
// set_points

template <typename Real>
int Engine::set_points_impl(const double* x_override) {
  SortArgs s{};
  s.items = d_items;
  s.n_items = (int)items.size();
  s.point_offsets = d_point_offsets;
  s.bin_offsets = d_bin_offsets;
  s.total_points = total_points;
  s.total_bins = total_bins;
  s.x_override = x_override;
  s.err = err_flag;
  s.single_d = items.size() == 1 ? items[0].geom.d : 0;
  EventPair ev{};
  TRY(stage_begin(NFFT_STAGE_SORT, &ev));
  CK(cudaMemsetAsync(bin_count, 0, sizeof(int) * (size_t)std::max(total_bins, 1), stream));
  CK(launch_bin_count<Real>(s, bin_count, bin_rank, stream));
  // bin count, scatter, subproblem count and fill, two scans
  kernel_launches += (s.total_points > 0 ? 4 : 2) + 2 * scan_launches(total_bins);
  CK(launch_scan(bin_count, bin_start, total_bins, nullptr, scan_partials, stream));
  Real* d[3] = {static_cast<Real*>(delta[0]), static_cast<Real*>(delta[1]), static_cast<Real*>(delta[2])};
  CK(launch_scatter<Real>(s, bin_start, bin_rank, perm, local, d, stream));
  CK(launch_subproblem_count(bin_count, total_bins, max_sub, sub_count, stream));
  CK(launch_scan(sub_count, sub_start, total_bins, num_subs, scan_partials, stream));
  CK(launch_subproblem_fill(s, bin_count, bin_start, sub_start, max_sub, subs, stream));
  TRY(stage_end(&ev));
  return NFFT_OK;
}

int Engine::set_points_single(const double* x) {
  points_set = false;
  last_x = x;
  const int s = precision == NFFT_FP64 ? set_points_impl<double>(x) : set_points_impl<float>(x);
  if (s == NFFT_OK) points_set = true;
  return s;
}

int Engine::set_points_batch(const double* const* x) {
  points_set = false;
  batch_x.assign(x, x + specs.size());
  for (size_t k = 0; k < items.size(); ++k) {
    items[k].x = x[order[k]];
    if (!items[k].x && items[k].M > 0) return NFFT_ERR_INVALID_ARG;
  }
  // the points pointers ride in both graph tables too
  for (int k = 0; k < 2; ++k) {
    CK(cudaEventSynchronize(slot_done[k]));
    for (size_t i = 0; i < items.size(); ++i) h_table[k][i].x = items[i].x;
  }
  CK(cudaMemcpyAsync(d_items, items.data(), sizeof(ItemDev) * items.size(), cudaMemcpyHostToDevice, stream));
  const int s = precision == NFFT_FP64 ? set_points_impl<double>(nullptr) : set_points_impl<float>(nullptr);
  // the host copy must outlive the async copy above
  CK(cudaStreamSynchronize(stream));
  if (s == NFFT_OK) points_set = true;
  return s;
}

// ===========================================================================
// transforms of a single item (per-call pointers as overrides)

int Engine::adjoint_single(const void* f, void* fhat, int R) {
  FClass& fc = fclasses[item_fclass[0]];
  const ItemDev& it = items[0];
  for (int r0 = 0; r0 < R; r0 += rhs_cap) {
    const int nr = (R - r0) < rhs_cap ? (R - r0) : rhs_cap;
    EventPair ev{};
    TRY(stage_begin(NFFT_STAGE_SPREAD, &ev));
    if (!kclasses[0].owner || it.M == 0) CK(cudaMemsetAsync(it.grid, 0, (size_t)nr * fc.cells * csize, stream));
    if (it.M > 0) {
      const void* fin = static_cast<const char*>(f) + (int64_t)r0 * it.M * (int64_t)csize;
      TRY(precision == NFFT_FP64 ? run_points<double>(kclasses[0], true, fin, nullptr, nr)
                                 : run_points<float>(kclasses[0], true, fin, nullptr, nr));
    }
    TRY(stage_end(&ev));
    TRY(stage_begin(NFFT_STAGE_FFT, &ev));
    TRY(run_fft(fc, nr, item_grid_offset[0], CUFFT_FORWARD));
    TRY(stage_end(&ev));
    TRY(stage_begin(NFFT_STAGE_DECONV, &ev));
    void* out = static_cast<char*>(fhat) + (int64_t)r0 * it.NN * (int64_t)csize;
    const int64_t cblocks = scale_blocks(it.NN / it.N[it.geom.d - 1] * nr, it.N[it.geom.d - 1], false);
    CK(precision == NFFT_FP64 ? launch_deconv_crop<double>(d_items, nullptr, nullptr, cblocks, out, nr, stream)
                              : launch_deconv_crop<float>(d_items, nullptr, nullptr, cblocks, out, nr, stream));
    kernel_launches += cblocks > 0 ? 1 : 0;
    TRY(stage_end(&ev));
  }
  return NFFT_OK;
}

int Engine::forward_single(const void* fhat, void* f, int R) {
  FClass& fc = fclasses[item_fclass[0]];
  const ItemDev& it = items[0];
  for (int r0 = 0; r0 < R; r0 += rhs_cap) {
    const int nr = (R - r0) < rhs_cap ? (R - r0) : rhs_cap;
    EventPair ev{};
    TRY(stage_begin(NFFT_STAGE_PAD, &ev));
    const void* hin = static_cast<const char*>(fhat) + (int64_t)r0 * it.NN * (int64_t)csize;
    const int64_t pblocks = scale_blocks(fc.cells / fc.n[fc.d - 1] * nr, fc.n[fc.d - 1], false);
    CK(precision == NFFT_FP64 ? launch_pad_deconv<double>(d_items, nullptr, nullptr, pblocks, hin, nr, stream)
                              : launch_pad_deconv<float>(d_items, nullptr, nullptr, pblocks, hin, nr, stream));
    kernel_launches += pblocks > 0 ? 1 : 0;
    TRY(stage_end(&ev));
    TRY(stage_begin(NFFT_STAGE_IFFT, &ev));
    TRY(run_fft(fc, nr, item_grid_offset[0], CUFFT_INVERSE));
    TRY(stage_end(&ev));
    TRY(stage_begin(NFFT_STAGE_INTERP, &ev));
    if (it.M > 0) {
      void* fout = static_cast<char*>(f) + (int64_t)r0 * it.M * (int64_t)csize;
      // interpolation reads `in` only through the override flag; the values come from the grid
      TRY(precision == NFFT_FP64 ? run_points<double>(kclasses[0], false, fout, fout, nr)
                                 : run_points<float>(kclasses[0], false, fout, fout, nr));
    }
    TRY(stage_end(&ev));
  }
  return NFFT_OK;
}

// ===========================================================================
// transforms of a batch (pointers from the item table)

template <typename Real>
int Engine::adjoint_table(bool in_graph) {
  EventPair ev{};
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_SPREAD, &ev));
  for (auto& fc : fclasses)
    if (!fc.owner_written) CK(cudaMemsetAsync(fc.buf, 0, (size_t)fc.grids * fc.cells * csize, stream));
  for (const auto& kc : kclasses) TRY(run_points<Real>(kc, true, nullptr, nullptr, 0));
  if (!in_graph) TRY(stage_end(&ev));
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_FFT, &ev));
  for (auto& fc : fclasses) TRY(run_fft(fc, fc.grids, 0, CUFFT_FORWARD));
  if (!in_graph) TRY(stage_end(&ev));
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_DECONV, &ev));
  CK(launch_deconv_crop<Real>(d_items, d_crop_blocks, d_crop_blocks + items.size() + 1, crop_blocks, nullptr, 0,
                              stream));
  kernel_launches += crop_blocks > 0 ? 1 : 0;
  if (!in_graph) TRY(stage_end(&ev));
  return NFFT_OK;
}

template <typename Real>
int Engine::forward_table(bool in_graph) {
  EventPair ev{};
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_PAD, &ev));
  CK(launch_pad_deconv<Real>(d_items, d_pad_blocks, d_pad_blocks + items.size() + 1, pad_blocks, nullptr, 0,
                             stream));
  kernel_launches += pad_blocks > 0 ? 1 : 0;
  if (!in_graph) TRY(stage_end(&ev));
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_IFFT, &ev));
  for (auto& fc : fclasses) TRY(run_fft(fc, fc.grids, 0, CUFFT_INVERSE));
  if (!in_graph) TRY(stage_end(&ev));
  if (!in_graph) TRY(stage_begin(NFFT_STAGE_INTERP, &ev));
  for (const auto& kc : kclasses) TRY(run_points<Real>(kc, false, nullptr, nullptr, 0));
  if (!in_graph) TRY(stage_end(&ev));
  return NFFT_OK;
}

void Engine::drop_graphs() {
  for (int k = 0; k < 2; ++k) {
    if (graph_adj[k]) cudaGraphExecDestroy(graph_adj[k]);
    if (graph_fwd[k]) cudaGraphExecDestroy(graph_fwd[k]);
    graph_adj[k] = graph_fwd[k] = nullptr;
  }
}

// One graph per direction and table slot: the table upload (pinned host ->
// device), then every launch of the transform.
int Engine::capture_graphs() {
  // capture on a private stream (the legacy default stream cannot be
  // captured); the graphs are launched on the caller's stream
  if (!capture_stream) CK(cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
  struct Restore {
    Engine* e;
    cudaStream_t s;
    ~Restore() { e->stream = s; }
  } restore{this, stream};
  stream = capture_stream;
  for (int k = 0; k < 2; ++k) {
    for (int dir = 0; dir < 2; ++dir) {
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      int s = NFFT_OK;
      cudaError_t e = cudaMemcpyAsync(d_items, h_table[k], sizeof(ItemDev) * items.size(), cudaMemcpyHostToDevice,
                                      stream);
      if (e != cudaSuccess) s = NFFT_ERR_CUDA;
      const int64_t before = kernel_launches;
      if (s == NFFT_OK) {
        if (dir == 0)
          s = precision == NFFT_FP64 ? adjoint_table<double>(true) : adjoint_table<float>(true);
        else
          s = precision == NFFT_FP64 ? forward_table<double>(true) : forward_table<float>(true);
      }
      graph_launches[dir] = kernel_launches - before;   // kernels per replay
      kernel_launches = before;
      const cudaError_t ee = cudaStreamEndCapture(stream, &g);
      if (s != NFFT_OK || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s != NFFT_OK ? s : NFFT_ERR_CUDA;
      }
      cudaGraphExec_t ex = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        cudaGetLastError();
        return NFFT_ERR_CUDA;
      }
      (dir == 0 ? graph_adj : graph_fwd)[k] = ex;
    }
  }
  return NFFT_OK;
}

int Engine::adjoint_batch(const void* const* f, void* const* fhat) {
  if (!graph_adj[0]) TRY(capture_graphs());
  const int k = slot;
  slot ^= 1;
  CK(cudaEventSynchronize(slot_done[k]));   // the launch that last read this table is done
  for (size_t i = 0; i < items.size(); ++i) {
    h_table[k][i].in = f[order[i]];
    h_table[k][i].out = fhat[order[i]];
  }
  EventPair ev{};
  TRY(stage_begin(NFFT_STAGE_SPREAD, &ev));   // whole-graph time is booked as the spread stage
  CK(cudaGraphLaunch(graph_adj[k], stream));
  kernel_launches += graph_launches[0];
  TRY(stage_end(&ev));
  CK(cudaEventRecord(slot_done[k], stream));
  return NFFT_OK;
}

int Engine::forward_batch(const void* const* fhat, void* const* f) {
  if (!graph_fwd[0]) TRY(capture_graphs());
  const int k = slot;
  slot ^= 1;
  CK(cudaEventSynchronize(slot_done[k]));
  for (size_t i = 0; i < items.size(); ++i) {
    h_table[k][i].in = fhat[order[i]];
    h_table[k][i].out = f[order[i]];
  }
  EventPair ev{};
  TRY(stage_begin(NFFT_STAGE_INTERP, &ev));
  CK(cudaGraphLaunch(graph_fwd[k], stream));
  kernel_launches += graph_launches[1];
  TRY(stage_end(&ev));
  CK(cudaEventRecord(slot_done[k], stream));
  return NFFT_OK;
}

// ===========================================================================
// Ewald reciprocal energy (single item)

template <typename Real>
int Engine::ewald_impl(const void* q, double L, double alpha) {
  using C = typename Cplx<Real>::type;
  FClass& fc = fclasses[item_fclass[0]];
  const ItemDev& it = items[0];
  EventPair ev{};
  TRY(stage_begin(NFFT_STAGE_SPREAD, &ev));
  if (!kclasses[0].owner || it.M == 0) CK(cudaMemsetAsync(it.grid, 0, (size_t)fc.cells * csize, stream));
  if (it.M > 0) TRY(run_points<Real>(kclasses[0], true, q, nullptr, 1));
  TRY(stage_end(&ev));
  TRY(stage_begin(NFFT_STAGE_FFT, &ev));
  TRY(run_fft(fc, 1, item_grid_offset[0], CUFFT_FORWARD));
  TRY(stage_end(&ev));
  TRY(stage_begin(NFFT_STAGE_DECONV, &ev));
  EwaldGeom g{};
  g.d = it.geom.d;
  g.NN = it.NN;
  for (int t = 0; t < kMaxDim; ++t) {
    g.N[t] = it.N[t];
    g.n[t] = it.geom.n[t];
    g.inv_c[t] = t < it.geom.d ? it.inv_c[t] : nullptr;
  }
  const double al = alpha * L;
  g.coef = M_PI * M_PI / (al * al);
  CK(launch_ewald_sum<Real>(static_cast<const C*>(it.grid), true, g, ewald_partials, 1.0 / (2.0 * M_PI * L), 0.0,
                            ewald_out, stream));
  kernel_launches += 2;
  CK(launch_sumsq<Real>(static_cast<const C*>(q), it.M, ewald_partials, -alpha / std::sqrt(M_PI), 0.0,
                        ewald_out + 1, stream));
  kernel_launches += 2;
  TRY(stage_end(&ev));
  return NFFT_OK;
}

int Engine::ewald(const void* q, double L, double alpha, double* out) {
  TRY(precision == NFFT_FP64 ? ewald_impl<double>(q, L, alpha) : ewald_impl<float>(q, L, alpha));
  double parts[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(parts, ewald_out, sizeof(parts), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  out[0] = parts[0] + parts[1];
  out[1] = parts[0];
  out[2] = parts[1];
  return NFFT_OK;
}

template <typename Real>
int Engine::ewald_forces_impl(const void* q, double L, double alpha, double* F) {
  using C = typename Cplx<Real>::type;
  const ItemDev& it = items[0];
  if (!force_modes) TRY(alloc_dev(force_modes, (size_t)3 * (size_t)it.NN * csize, device_bytes));
  if (!force_vals && it.M > 0) TRY(alloc_dev(force_vals, (size_t)3 * (size_t)it.M * csize, device_bytes));
  // S(n): the adjoint NFFT (Eq. 5) of the charges, into the first block
  TRY(adjoint_single(q, force_modes, 1));
  EwaldGeom g{};
  g.d = it.geom.d;
  g.NN = it.NN;
  for (int t = 0; t < kMaxDim; ++t) {
    g.N[t] = it.N[t];
    g.n[t] = it.geom.n[t];
    g.inv_c[t] = nullptr;
  }
  const double al = alpha * L;
  g.coef = M_PI * M_PI / (al * al);
  CK(launch_force_modes<Real>(static_cast<C*>(force_modes), g, stream));
  kernel_launches += it.NN > 0 ? 1 : 0;
  if (it.M == 0) return NFFT_OK;
  // sum_n w(n) n_t S(n) exp(+2 pi i n.x_i): the forward NFFT (Eq. 6), three right-hand sides
  TRY(forward_single(force_modes, force_vals, 3));
  CK(launch_force_finish<Real>(static_cast<const C*>(force_vals), static_cast<const C*>(q), it.M, 2.0 / (L * L), F,
                               stream));
  kernel_launches += 1;
  return NFFT_OK;
}

int Engine::ewald_forces(const void* q, double L, double alpha, double* F) {
  if (specs[0].d != 3) return NFFT_ERR_UNSUPPORTED;
  return precision == NFFT_FP64 ? ewald_forces_impl<double>(q, L, alpha, F)
                                : ewald_forces_impl<float>(q, L, alpha, F);
}

int Engine::ewald_sum(const void* S, double L, double alpha, double* sum_dev) {
  const ItemDev& it = items[0];
  EwaldGeom g{};
  g.d = it.geom.d;
  g.NN = it.NN;
  for (int t = 0; t < kMaxDim; ++t) {
    g.N[t] = it.N[t];
    g.n[t] = it.geom.n[t];
    g.inv_c[t] = nullptr;
  }
  const double al = alpha * L;
  g.coef = M_PI * M_PI / (al * al);
  const double scale = 1.0 / (2.0 * M_PI * L);
  if (precision == NFFT_FP64)
    CK(launch_ewald_sum<double>(static_cast<const double2*>(S), false, g, ewald_partials, scale, 0.0, sum_dev,
                                stream));
  else
    CK(launch_ewald_sum<float>(static_cast<const float2*>(S), false, g, ewald_partials, scale, 0.0, sum_dev,
                               stream));
  kernel_launches += 2;
  return NFFT_OK;
}

// ===========================================================================
// options, info, sync

int Engine::sync() {
  CK(cudaStreamSynchronize(stream));
  int flag = 0;
  CK(cudaMemcpy(&flag, err_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemset(err_flag, 0, sizeof(int)));
    if (flag & 2) return NFFT_ERR_TIMEOUT;
    if (flag & 1) return NFFT_ERR_DOMAIN;
  }
  return NFFT_OK;
}

int Engine::set_stream(cudaStream_t s) {
  stream = s;
  drop_graphs();   // graphs are replayed on any stream, but the cuFFT plans follow the stream
  return NFFT_OK;
}

int Engine::set_option(int option, int64_t value) {
  switch (option) {
    case NFFT_OPT_METHOD:
      if (value < NFFT_METHOD_AUTO || value > NFFT_METHOD_GRID_WARP) return NFFT_ERR_INVALID_ARG;
      method_opt = (int)value;
      break;
    case NFFT_OPT_OWNER_SPREAD:
      if (value != 0 && value != 1) return NFFT_ERR_INVALID_ARG;
      owner_enabled = value != 0;
      break;
    case NFFT_OPT_TENSOR_SPREAD:
    case NFFT_OPT_TENSOR_INTERP:
      if (value != 0 && value != 1) return NFFT_ERR_INVALID_ARG;
      (option == NFFT_OPT_TENSOR_SPREAD ? tensor_enabled : tensor_interp_enabled) = value != 0;
      break;
    case NFFT_OPT_PRUNED_FFT:
      if (value < -1 || value > 1) return NFFT_ERR_INVALID_ARG;
      pruned_fft_mode = (int)value;
      break;
    case NFFT_OPT_SPARSE_POINTS:
    case NFFT_OPT_SPARSE_POINTS_INTERP:
      if (value < -1 || value > (1 << 20)) return NFFT_ERR_INVALID_ARG;
      (option == NFFT_OPT_SPARSE_POINTS ? sparse_opt : sparse_interp_opt) = (int)value;
      break;
    case NFFT_OPT_BIN_0:
    case NFFT_OPT_BIN_1:
    case NFFT_OPT_BIN_2: {
      const int t = option - NFFT_OPT_BIN_0;
      int dmax = 1;
      for (const auto& s : specs) dmax = std::max(dmax, s.d);
      if (value < 0 || t >= dmax || value > 65535) return NFFT_ERR_INVALID_ARG;
      bin_opt[t] = (int)value;
      break;
    }
    case NFFT_OPT_MAX_SUBPROBLEM:
      if (value < 0 || value > (1 << 20)) return NFFT_ERR_INVALID_ARG;
      max_sub_opt = (int)value;
      break;
    case NFFT_OPT_RHS_CAPACITY: {
      if (value < 1 || value > 4096) return NFFT_ERR_INVALID_ARG;
      if (!single) return NFFT_ERR_UNSUPPORTED;   // a batch fixes its right-hand sides per item
      CK(cudaStreamSynchronize(stream));
      for (auto& fc : fclasses) {
        destroy_fft_plans(fc);
        device_bytes -= (int64_t)fc.grids * fc.cells * (int64_t)csize;
        free_dev(fc.buf);
      }
      fclasses.clear();
      rhs_cap = (int)value;
      TRY(build_fft());
      const bool had = points_set;
      TRY(build_layout());   // item grid pointers moved
      (void)had;
      return NFFT_OK;
    }
    case NFFT_OPT_PROFILE:
      profile = value != 0;
      return NFFT_OK;
    case NFFT_OPT_THREADS:
    case NFFT_OPT_SPREAD_THREADS:
    case NFFT_OPT_INTERP_THREADS:
      if (value != 0 && (value < 32 || value > 256 || value % 32 != 0)) return NFFT_ERR_INVALID_ARG;
      (option == NFFT_OPT_THREADS ? threads_opt
                                  : (option == NFFT_OPT_SPREAD_THREADS ? spread_threads_opt : interp_threads_opt)) =
          (int)value;
      return NFFT_OK;
    default:
      return NFFT_ERR_INVALID_ARG;
  }
  CK(cudaStreamSynchronize(stream));
  return build_layout();
}

int Engine::info(nfft_plan_info* out) const {
  std::memset(out, 0, sizeof(*out));
  const ItemSpec& s = specs[0];
  const ItemDev& it = items[0];
  out->d = s.d;
  out->M = s.M;
  out->m = s.m;
  out->taps = it.win.taps;
  out->window = s.window;
  out->precision = precision;
  out->method = kclasses.empty() ? 0 : kclasses[0].method;
  out->n_bins = 1;
  for (int t = 0; t < 3; ++t) {
    out->N[t] = t < s.d ? s.N[t] : 1;
    out->n[t] = it.geom.n[t];
    out->bin[t] = it.geom.bin[t];
    out->sigma[t] = t < s.d ? (double)it.geom.n[t] / (double)s.N[t] : 1.0;
    if (t < s.d) out->n_bins *= it.geom.nbins[t];
  }
  out->rhs_capacity = single ? rhs_cap : s.nrhs;
  out->threads = threads_opt;
  out->device_bytes = device_bytes;
  out->max_subproblem = max_sub;
  out->spread_threads = spread_threads_opt;
  out->sparse_points = kclasses.empty() ? 0 : kclasses[0].sparse_points;
  out->sparse_points_interp = kclasses.empty() ? 0 : kclasses[0].sparse_points_interp;
  out->owner_spread = kclasses.empty() ? 0 : (kclasses[0].owner ? 1 : 0);
  out->kernel_launches = kernel_launches;
  out->interp_threads = interp_threads_opt;
  out->tensor_spread = kclasses.empty() ? 0 : (kclasses[0].tensor ? 1 : 0);
  out->tensor_interp = kclasses.empty() ? 0 : (kclasses[0].tensor_interp ? 1 : 0);
  out->pruned_fft = (!fclasses.empty() && fft_pruned(fclasses[0])) ? 1 : 0;
  out->spread_block_threads = last_spread_threads;
  out->interp_block_threads = last_interp_threads;
  return NFFT_OK;
}

// ===========================================================================
// autotuner

namespace {
// Deterministic complex test values (a hash of the index): the timings do not
// depend on the values, but zeros would skip work.
template <typename Real>
__global__ void k_fill_values(typename Cplx<Real>::type* v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = (uint32_t)(i * 2654435761u) ^ (uint32_t)(i >> 32);
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  const Real re = (Real)((h & 0xffff) / 32768.0 - 1.0);
  const Real im = (Real)(((h >> 16) & 0xffff) / 32768.0 - 1.0);
  v[i].x = re;
  v[i].y = im;
}
}  // namespace

int Engine::reset_points() {
  if (single) return set_points_single(last_x);
  const std::vector<const double*> xs = batch_x;
  return set_points_batch(xs.data());
}

int Engine::time_transforms(int reps, const std::vector<void*>& fin, const std::vector<void*>& fout,
                            const std::vector<void*>& hin, const std::vector<void*>& hout, double* ms) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  std::vector<float> t;
  for (int r = 0; r < reps + 1; ++r) {   // the first run warms up (and captures the graphs)
    CK(cudaEventRecord(a, stream));
    if (single) {
      TRY(adjoint_single(fin[0], hout[0], 1));
      TRY(forward_single(hin[0], fout[0], 1));
    } else {
      TRY(adjoint_batch(const_cast<const void* const*>(fin.data()), hout.data()));
      TRY(forward_batch(const_cast<const void* const*>(hin.data()), fout.data()));
    }
    CK(cudaEventRecord(b, stream));
    CK(cudaEventSynchronize(b));
    float e = 0.f;
    CK(cudaEventElapsedTime(&e, a, b));
    if (r > 0) t.push_back(e);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(t.begin(), t.end());
  *ms = t.empty() ? 0.0 : (double)t[t.size() / 2];
  return NFFT_OK;
}

int Engine::autotune(int reps, double* best_ms) {
  if (!points_set) return NFFT_ERR_NOT_READY;
  if (reps < 1) reps = 3;
  const bool was_profiling = profile;
  profile = false;
  // test buffers per item (user order): values in, results out
  std::vector<void*> fin(specs.size()), fout(specs.size()), hin(specs.size()), hout(specs.size());
  std::vector<void*> owned;
  int st = NFFT_OK;
  int64_t dummy = 0;
  for (size_t i = 0; i < specs.size() && st == NFFT_OK; ++i) {
    const ItemSpec& s = specs[i];
    int64_t NN = 1;
    for (int t = 0; t < s.d; ++t) NN *= s.N[t];
    const int64_t R = single ? 1 : s.nrhs;
    void* p[4] = {nullptr, nullptr, nullptr, nullptr};
    const int64_t sizes[4] = {R * std::max<int64_t>(s.M, 1), R * std::max<int64_t>(s.M, 1), R * NN, R * NN};
    for (int k = 0; k < 4 && st == NFFT_OK; ++k) {
      st = alloc_dev(p[k], (size_t)sizes[k] * csize, dummy);
      if (st == NFFT_OK) owned.push_back(p[k]);
    }
    if (st != NFFT_OK) break;
    for (int k = 0; k < 4; k += 2) {
      const int64_t n = sizes[k];
      if (precision == NFFT_FP64)
        k_fill_values<double><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(static_cast<double2*>(p[k]), n);
      else
        k_fill_values<float><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(static_cast<float2*>(p[k]), n);
    }
    fin[i] = p[0];
    fout[i] = p[1];
    hin[i] = p[2];
    hout[i] = p[3];
  }
  int dmax = 1;
  for (const auto& s : specs) dmax = std::max(dmax, s.d);
  struct Cand {
    int bin[3];
    int P;
  };
  std::vector<Cand> cands;
  const int Ps[3] = {1024, 256, 4096};
  if (dmax == 3 && (tensor_enabled || tensor_interp_enabled) && precision == NFFT_FP32_MIXED) {
    // tensor-core spreading: (z, y) rows of the tile within the MMA's 128,
    // x columns along the N dimension
    const int b = std::max(1, 12 - taps_for(specs[0].window, specs[0].m));
    const int bins[][3] = {{b, b, 16}, {b, b, 32}, {b, b, 8}, {b, b, 24}};
    for (const auto& bb : bins)
      for (int P : Ps) cands.push_back(Cand{{bb[0], bb[1], bb[2]}, P});
  } else if (dmax == 3) {
    const int bins[][3] = {{8, 8, 16}, {8, 8, 8}, {4, 8, 16}, {8, 16, 16}, {8, 8, 32}, {4, 4, 32}};
    for (const auto& b : bins)
      for (int P : Ps) cands.push_back(Cand{{b[0], b[1], b[2]}, P});
  } else if (dmax == 2) {
    const int bins[][2] = {{32, 32}, {16, 32}, {32, 64}, {64, 64}, {16, 16}};
    for (const auto& b : bins)
      for (int P : Ps) cands.push_back(Cand{{b[0], b[1], 0}, P});
  } else {
    for (int b : {1024, 256, 4096})
      for (int P : Ps) cands.push_back(Cand{{b, 0, 0}, P});
  }
  // layouts (bin edges, subproblem size) at the default block sizes
  std::vector<std::pair<double, int>> ranked;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    const Cand& c = cands[ci];
    if (st != NFFT_OK) break;
    for (int t = 0; t < 3; ++t) bin_opt[t] = t < dmax ? c.bin[t] : 0;
    max_sub_opt = c.P;
    spread_threads_opt = interp_threads_opt = 0;
    CK(cudaStreamSynchronize(stream));
    if (build_layout() != NFFT_OK) continue;   // e.g. a tile that does not fit
    if (reset_points() != NFFT_OK) continue;
    double ms = 0;
    if (time_transforms(reps, fin, fout, hin, hout, &ms) != NFFT_OK) continue;
    ranked.emplace_back(ms, (int)ci);
  }
  std::sort(ranked.begin(), ranked.end());
  // threads per block for spreading and for interpolation, on each of the
  // fastest layouts (a layout's rank can change with its block sizes)
  double best = ranked.empty() ? 1e30 : ranked[0].first;
  Cand best_c = ranked.empty() ? cands[0] : cands[ranked[0].second];
  int best_sth = 0, best_ith = 0;
  const size_t top = dmax >= 2 ? std::min<size_t>(ranked.size(), 3) : 0;
  for (size_t k = 0; k < top && st == NFFT_OK; ++k) {
    const Cand& c = cands[ranked[k].second];
    for (int t = 0; t < 3; ++t) bin_opt[t] = t < dmax ? c.bin[t] : 0;
    max_sub_opt = c.P;
    spread_threads_opt = interp_threads_opt = 0;
    CK(cudaStreamSynchronize(stream));
    if (build_layout() != NFFT_OK || reset_points() != NFFT_OK) {
      cudaGetLastError();
      continue;
    }
    double here = ranked[k].first;
    for (int pass = 0; pass < 2; ++pass) {
      int& opt = pass == 0 ? spread_threads_opt : interp_threads_opt;
      int keep = 0;
      for (int th : {64, 128, 256}) {
        opt = th;
        drop_graphs();
        double ms = 0;
        if (time_transforms(reps, fin, fout, hin, hout, &ms) != NFFT_OK) {
          cudaGetLastError();
          continue;
        }
        if (ms < here) {
          here = ms;
          keep = th;
        }
      }
      opt = keep;
    }
    if (here < best || k == 0) {
      best = here;
      best_c = c;
      best_sth = spread_threads_opt;
      best_ith = interp_threads_opt;
    }
  }
  drop_graphs();
  for (int t = 0; t < 3; ++t) bin_opt[t] = t < dmax ? best_c.bin[t] : 0;
  max_sub_opt = best_c.P;
  spread_threads_opt = best_sth;
  interp_threads_opt = best_ith;
  if (st == NFFT_OK) {
    CK(cudaStreamSynchronize(stream));
    st = build_layout();
    if (st == NFFT_OK) st = reset_points();
  }
  // the sparse/dense split, for spreading and for interpolation: points of a
  // bin below which the grid-warp kernels take it (the automatic threshold
  // is a rule of thumb; the crossover moves with the window and the point
  // density)
  if (st == NFFT_OK && method_opt == NFFT_METHOD_AUTO) {
    for (int pass = 0; pass < 2 && st == NFFT_OK; ++pass) {
      int& opt = pass == 0 ? sparse_opt : sparse_interp_opt;
      const int base = opt;
      int keep = base;
      for (int th : {-1, 32, 128, 512, 1 << 20}) {
        if (th == base) continue;
        opt = th;
        CK(cudaStreamSynchronize(stream));
        double ms = 0;
        if (build_layout() != NFFT_OK || reset_points() != NFFT_OK ||
            time_transforms(reps, fin, fout, hin, hout, &ms) != NFFT_OK) {
          cudaGetLastError();
          continue;
        }
        if (ms < best) {
          best = ms;
          keep = th;
        }
      }
      opt = keep;
      CK(cudaStreamSynchronize(stream));
      st = build_layout();
      if (st == NFFT_OK) st = reset_points();
    }
    drop_graphs();
  }
  // the pruned against the full 3-D FFT (automatic mode only): the faster
  // stays, and the other form's cuFFT plans are released
  if (st == NFFT_OK && pruned_fft_mode < 0 && single && !fclasses.empty()) {
    FClass& fc = fclasses[item_fclass[0]];
    const int auto_mode = fft_pruned(fc) ? 1 : 0;
    pruned_fft_mode = 1;
    if (fft_pruned(fc)) {
      double t[2] = {1e30, 1e30};
      for (int mode = 0; mode < 2; ++mode) {
        pruned_fft_mode = mode;
        if (time_transforms(reps, fin, fout, hin, hout, &t[mode]) != NFFT_OK) {
          cudaGetLastError();
          t[mode] = 1e30;
        }
      }
      pruned_fft_mode = t[1] <= t[0] ? 1 : 0;
      if (t[pruned_fft_mode] >= 1e30) pruned_fft_mode = auto_mode;
      best = std::min(best, t[pruned_fft_mode]);
      CK(cudaStreamSynchronize(stream));
      if (pruned_fft_mode == 1) {
        for (auto& kv : fc.plans) cufftDestroy(kv.second);
        fc.plans.clear();
      } else {
        if (fc.prune_z) cufftDestroy(fc.prune_z);
        if (fc.prune_yx) cufftDestroy(fc.prune_yx);
        fc.prune_z = fc.prune_yx = 0;
        fc.prune_built = false;
      }
    } else {
      pruned_fft_mode = -1;   // not applicable (sigma = 1 along dimension 0)
    }
  }
  CK(cudaStreamSynchronize(stream));
  for (void* p : owned) cudaFree(p);
  profile = was_profiling;
  if (best_ms) *best_ms = best;
  return st;
}

}  // namespace gbnfft
