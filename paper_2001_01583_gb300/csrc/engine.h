// The host engine behind the C ABI: a set of NFFT items (one for a plan, many
// for a batch) with their sort buffers, grids, cuFFT plans and kernel
// launches.
//
//   kernel class: items with the same d, taps, window and bin edges (hence
//                 tile shape); their points are spread / interpolated by one
//                 persistent launch over the class's subproblems;
//   FFT class:    items with the same oversampled grid; their grids are
//                 contiguous and transformed by one cuFFT plan-many.
#pragma once

#include <cufft.h>

#include <map>
#include <tuple>
#include <vector>

#include "ewald.h"
#include "gbnfft.h"
#include "kernels.h"

namespace gbnfft {

struct ItemSpec {
  int d;
  int64_t N[3];
  int64_t M;
  double sigma;
  int m;
  int window;
  int nrhs;     // grids kept for the item (batch: its right-hand sides)
};

struct KClass {
  int d, taps, window, method;
  int bin[3], tile[3], nbins_total;
  int pitch;
  int item_begin, item_end;   // internal item range
  int bin_begin, bin_end;     // global bin range
  int max_nrhs;
  int64_t max_subs;           // bound on the class's subproblems
  int sparse_points;          // spreading subproblems below this many points: grid-warp kernel (0: none)
  int sparse_points_interp;   // the same for interpolation
  bool owner;                 // spreading of sparse bins by the owner kernel (3-D)
  bool tensor;                // dense bins spread on the tensor cores (3-D, FP32)
  bool tensor_interp;         // dense bins interpolated on the tensor cores (3-D, FP32)
};

struct FClass {
  int d;
  int64_t n[3];
  int64_t cells;
  int grids;                  // grids in the buffer
  void* buf = nullptr;
  std::map<int, cufftHandle> plans;
  bool owner_written = false;   // every grid of the class is written whole by the owner kernel
  // pruned 3-D FFT (one item): 1-D along dimension 0 over the grid, 2-D over
  // N_0 / 2 contiguous planes (applied to the two runs of planes holding I_N)
  cufftHandle prune_z = 0, prune_yx = 0;
  bool prune_built = false;
};

struct EventPair {
  int stage;
  cudaEvent_t start, stop;
};

// Shared parameter rules (engine.cu).
int64_t oversampled_size(int64_t N, double sigma);
int window_taps(int window, int m);
int validate_spec(const ItemSpec& s, int precision);
// true when the items' point counts add up to more than INT32_MAX (the sort's
// bin starts, ranks and scatter positions are 32-bit)
bool total_points_exceed_int32(const std::vector<ItemSpec>& specs);
double shape_param(int window, int m, double sigma);
// centred cardinal B-spline M_order(u) (support |u| < order / 2), host FP64
double cardinal_bspline(int order, double u);
// 1 / c_k of one dimension at frequency k (kernels' normalisation psi = phi / phi(0)).
double inv_c_at(int window, int m, int64_t n, double b, double k);

class Engine {
 public:
  ~Engine();
  // Validate, allocate everything, build the layout.  single = one item whose
  // pointers come with every call (a plan); else a batch (pointer table).
  int init(const std::vector<ItemSpec>& specs, int precision, cudaStream_t stream, bool single);

  int set_option(int option, int64_t value);
  int set_stream(cudaStream_t s);
  int set_points_single(const double* x);
  int set_points_batch(const double* const* x);
  int adjoint_single(const void* f, void* fhat, int R);
  int forward_single(const void* fhat, void* f, int R);
  int adjoint_batch(const void* const* f, void* const* fhat);
  int forward_batch(const void* const* fhat, void* const* f);
  int sync();
  int stage_times(double* ms, int64_t* launches, int reset);
  int ewald(const void* q, double L, double alpha, double* out3);
  int ewald_sum(const void* S, double L, double alpha, double* sum_dev);
  // Reciprocal-space forces (negative gradient of Eq. 12) at the points set:
  // F (device, M x 3 doubles).  Allocates its mode and value buffers on the
  // first call.
  int ewald_forces(const void* q, double L, double alpha, double* F);
  int info(nfft_plan_info* out) const;
  int64_t launched() const { return kernel_launches; }
  // Time candidate layouts on the points already set and keep the fastest
  // (see nfft_autotune).  best_ms: adjoint + forward time of the winner.
  int autotune(int reps, double* best_ms);

  // exposed for the C ABI
  int precision = 0;
  cudaStream_t stream = nullptr;
  std::vector<ItemSpec> specs;        // user order
  bool points_set = false;

 private:
  int build_layout();
  int release_layout();
  int build_fft();
  template <typename Real> int set_points_impl(const double* x_override);
  template <typename Real> int run_points(const KClass& kc, bool spread, const void* in, void* out, int nrhs);
  template <typename Real> int run_planes(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs);
  template <typename Real> int run_wpp(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs);
  template <typename Real> int run_tiled(const KClass& kc, PointKernelArgs<Real>& a, bool spread, int max_nrhs);
  template <typename Real> int run_gm(const KClass& kc, PointKernelArgs<Real>& a, bool spread);
  template <typename Real> int run_owner(const KClass& kc, PointKernelArgs<Real>& a);
  template <typename Real> int run_global(const KClass& kc, PointKernelArgs<Real>& a, bool spread);
  int run_tc(const KClass& kc, PointKernelArgs<float>& a, bool spread);
  template <typename Real> int adjoint_table(bool in_graph);
  template <typename Real> int forward_table(bool in_graph);
  template <typename Real> int ewald_impl(const void* q, double L, double alpha);
  template <typename Real> int ewald_forces_impl(const void* q, double L, double alpha, double* F);
  int run_fft(FClass& fc, int batch, int64_t grid_offset, int direction);
  bool fft_pruned(const FClass& fc) const;
  int build_pruned(FClass& fc);
  void destroy_fft_plans(FClass& fc);
  int fft_handle(FClass& fc, int batch, cufftHandle* out);
  int blocks_per_sm(const void* fn, int threads, size_t smem);
  int stage_begin(int stage, EventPair* ev);
  int stage_end(EventPair* ev);
  int capture_graphs();
  void drop_graphs();
  int reset_points();
  int time_transforms(int reps, const std::vector<void*>& fin, const std::vector<void*>& fout,
                      const std::vector<void*>& hin, const std::vector<void*>& hout, double* ms);

  size_t csize = 16;
  int device = 0, num_sms = 1;
  size_t smem_optin = 48 * 1024, smem_per_sm = 100 * 1024;
  bool single = true;

  // options
  int method_opt = NFFT_METHOD_AUTO;
  int bin_opt[3] = {0, 0, 0};
  int max_sub_opt = 0;
  int sparse_opt = 0;          // NFFT_OPT_SPARSE_POINTS
  bool owner_enabled = false;  // NFFT_OPT_OWNER_SPREAD
  bool tensor_enabled = false; // NFFT_OPT_TENSOR_SPREAD
  bool tensor_interp_enabled = false;  // NFFT_OPT_TENSOR_INTERP
  int pruned_fft_mode = -1;             // NFFT_OPT_PRUNED_FFT: -1 automatic, 0 never, 1 always
  int64_t kernel_launches = 0;   // this library's kernels launched so far (graph replays included)
  int64_t graph_launches[2] = {0, 0};
  int sparse_interp_opt = 0;   // NFFT_OPT_SPARSE_POINTS_INTERP
  int max_sub = 1024;
  int threads_opt = 0;
  int spread_threads_opt = 0;
  int interp_threads_opt = 0;
  // block threads of the last tiled spreading / interpolation launch (reported by get_info)
  int last_spread_threads = 0;
  int last_interp_threads = 0;
  int rhs_cap = 1;
  const double* last_x = nullptr;      // single item: the points of the last set_points
  std::vector<const double*> batch_x;  // batch: the points of the last set_points (user order)
  bool profile = false;

  // items (internal order: grouped by kernel class)
  std::vector<int> order;             // internal -> user
  std::vector<ItemDev> items;         // internal order, host copy
  ItemDev* d_items = nullptr;
  ItemDev* h_table[2] = {nullptr, nullptr};   // pinned copies the batch graphs upload
  std::vector<int> item_fclass;       // user order
  std::vector<int64_t> item_grid_offset;   // user order, elements into the FFT class buffer
  std::vector<KClass> kclasses;
  std::vector<FClass> fclasses;
  std::vector<double*> tables;        // scaling tables (owned)
  std::map<std::tuple<int, int64_t, int64_t, int, int>, double*> table_cache;

  // sort buffers
  int64_t total_points = 0;
  int total_bins = 0;
  int64_t max_subs_total = 0;
  int64_t* d_point_offsets = nullptr;
  int* d_bin_offsets = nullptr;
  int* d_crop_blocks = nullptr;        // scaling launches: per-item block prefix sums, then each block's item
  int* d_pad_blocks = nullptr;
  int64_t crop_blocks = 0, pad_blocks = 0;
  int* bin_count = nullptr;
  int* bin_start = nullptr;
  int* sub_count = nullptr;
  int* scan_partials = nullptr;   // scratch of the multi-block scans
  int* sub_start = nullptr;
  int* num_subs = nullptr;
  SubProblem* subs = nullptr;
  int2* bin_rank = nullptr;
  int* perm = nullptr;
  uint32_t* local = nullptr;
  void* delta[3] = {nullptr, nullptr, nullptr};
  int* err_flag = nullptr;
  double* ewald_partials = nullptr;
  double* ewald_out = nullptr;
  void* force_modes = nullptr;   // 3 |I_N| complex (forces)
  void* force_vals = nullptr;    // 3 M complex (forces)
  int64_t device_bytes = 0;
  int64_t layout_bytes = 0;

  // batch graphs (two slots: the host fills one table while the other runs)
  cudaGraphExec_t graph_adj[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_fwd[2] = {nullptr, nullptr};
  cudaEvent_t slot_done[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  int slot = 0;

  // profiling
  std::vector<EventPair> events, free_events;
  double stage_ms[NFFT_STAGE_COUNT] = {0};
  int64_t stage_calls[NFFT_STAGE_COUNT] = {0};
  std::map<std::tuple<const void*, int, size_t>, int> occupancy;
};

}  // namespace gbnfft
