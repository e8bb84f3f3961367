// Internal launch interface between the host engine and the kernels.
//
// Every launch works on a table of items (ItemDev): a single plan is a
// batch of one item.  Per-call pointers can be passed as overrides in the
// launch arguments (single-item launches) or read from the table (batched
// launches, where a CUDA graph refreshes the table before the kernels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbnfft {

// ---- set_points (sort.cu) -------------------------------------------------
struct SortArgs {
  const ItemDev* items;
  int n_items;
  const int64_t* point_offsets;   // n_items + 1 prefix sums of M (device)
  const int* bin_offsets;         // n_items + 1 prefix sums of bins (device)
  int64_t total_points;
  int total_bins;
  const double* x_override;       // single item: points of this call (else items[i].x)
  int* err;                       // bit 0: non-finite coordinate
  int single_d;                   // one item: its dimension (the kernels' one-item form); 0 otherwise
};
// Cell and global bin of every point, and its rank inside its bin.
template <typename Real>
cudaError_t launch_bin_count(const SortArgs& s, int* bin_count, int2* bin_rank, cudaStream_t st);
// Exclusive prefix sum of n ints; *total = sum (may be null).  partials:
// scan_partials_needed(n) ints of device scratch.  scan_launches(n) kernels.
int scan_partials_needed(int n);
int scan_launches(int n);
cudaError_t launch_scan(const int* in, int* out, int n, int* total, int* partials, cudaStream_t st);
// Write every point to its sorted slot: perm (index within its item), packed in-bin offsets, deltas.
template <typename Real>
cudaError_t launch_scatter(const SortArgs& s, const int* bin_start, const int2* bin_rank, int* perm, uint32_t* local,
                           Real* const* delta, cudaStream_t st);
// Subproblems per global bin (ceil(count / P)), then their records.
cudaError_t launch_subproblem_count(const int* bin_count, int nbins, int P, int* sub_count, cudaStream_t st);
cudaError_t launch_subproblem_fill(const SortArgs& s, const int* bin_count, const int* bin_start, const int* sub_start,
                                   int P, SubProblem* subs, cudaStream_t st);

// ---- spreading / interpolation ---------------------------------------------
template <typename Real>
struct PointKernelArgs {
  SortedPoints<Real> pts;
  const ItemDev* items;
  int bin_begin, bin_end;   // the global bins of this launch's items
  int total_bins;
  int rhs_per_pass;         // tiles held in shared memory at once
  // single-item overrides (in == nullptr: read the item table)
  const void* in;
  void* out;
  int nrhs;
  // subproblems whose bin holds sub_min_count <= points < sub_max_count are this launch's
  int sub_min_count, sub_max_count;
  int item_begin, item_end;   // the launch's items (internal order)
  int* err;                   // device error flag: kernels that give up a wait set bit 1
};

// Points of the subproblem's whole bin (the sparse / dense split is per bin).
template <typename Real>
__device__ __forceinline__ bool sub_selected(const PointKernelArgs<Real>& a, const SubProblem& s) {
  const int total = a.pts.bin_count[a.items[s.item].bin_offset + s.bin];
  return total >= a.sub_min_count && total < a.sub_max_count;
}

// The launch's subproblems: [lo, hi).
template <typename Real>
__device__ __forceinline__ void launch_subs(const PointKernelArgs<Real>& a, int& lo, int& hi) {
  lo = a.pts.sub_start[a.bin_begin];
  hi = a.bin_end < a.total_bins ? a.pts.sub_start[a.bin_end] : *a.pts.num_subs;
}

// Per-call view of an item.
struct ItemCall {
  const void* in;
  void* out;
  int nrhs;
};
template <typename Real>
__device__ __forceinline__ ItemCall item_call(const PointKernelArgs<Real>& a, const ItemDev& it) {
  ItemCall c;
  c.in = a.in ? a.in : it.in;
  c.out = a.in ? a.out : it.out;
  c.nrhs = a.in ? a.nrhs : it.nrhs;
  return c;
}

// Tiled thread-per-point kernels (any d, taps <= 32; d = 3 up to 26).
const void* spread_tiled_kernel_f32(int d, int taps);
const void* spread_tiled_kernel_f64(int d, int taps);
const void* interp_tiled_kernel_f32(int d, int taps);
const void* interp_tiled_kernel_f64(int d, int taps);
// Global-memory kernels (any d, taps <= 32).
const void* global_kernel_f32(bool spread);
const void* global_kernel_f64(bool spread);

// Warp-per-point kernels straight on the grid (points_gm.cuh), any d, taps 2..26 even;
// blocks of kGmWarpsHost warps.
constexpr int kGmWarpsHost = 8;
constexpr int kGmSplitHost = 4;   // warps sharing one subproblem
const void* gm_kernel_f32(int d, int taps, bool spread);
const void* gm_kernel_f64(int d, int taps, bool spread);

// 3-D owner spreading of sparse bins (points_owner.cuh): a warp per bin's
// cells, plain stores, no atomics; blocks of kOwnerWarpsHost warps, dynamic
// shared memory kOwnerWarpsHost * (bin cells * complex + 3 taps * real).
constexpr int kOwnerWarpsHost = 4;
constexpr int kOwnerReachHost = 16;   // bins per dimension within a window's reach of a bin, at most
const void* owner_kernel_f32(int taps);
const void* owner_kernel_f64(int taps);

// Warp-per-point (d = 2) and shared-tile (d = 3) kernels, taps <= 16.
struct WppLayout {
  int pitch;        // row pitch of a tile, in complex elements
  int warp_cells;   // elements of one tile (rows * pitch)
  int warps;        // warps per block
};
const void* wpp_kernel_f32(int d, int taps, bool spread);
const void* wpp_kernel_f64(int d, int taps, bool spread);
// 3-D shared-tile kernels (points_planes.cuh): plane-owner spreading (warps
// a power of two dividing the taps) and point-group interpolation.
constexpr int kMaxPlaneTaps = 26;   // widest window of the 3-D shared-tile kernels
const void* planes_kernel_f32(int taps, int warps, bool spread);
const void* planes_kernel_f64(int taps, int warps, bool spread);
size_t planes_table_bytes_f32(int taps, int bp, int np, int nw, const int* tile, bool spread);
size_t planes_table_bytes_f64(int taps, int bp, int np, int nw, const int* tile, bool spread);

// 3-D spreading on the tensor cores (points_tc.cuh): FP32, taps 4, 6 or 8,
// tiles of at most 128 (z, y) rows and 2 T2 <= kTcMaxColsHost real columns;
// blocks of kTcThreadsHost threads.
constexpr int kTcThreadsHost = 256;
constexpr int kTcRowsHost = 128;
constexpr int kTcMaxColsHost = 112;
struct TcLaunch {
  int ncols;       // N of the MMAs: 2 T2 rounded up to 16
  int tmem_cols;   // tensor-memory columns per block: 4 x a power of two >= max(32, ncols)
};
const void* tc_spread_kernel_f32(int taps);
size_t tc_spread_smem_bytes(int taps, int ncols, const int* tile);
// Interpolation on the tensor cores (the same tiles): one block per SM.
const void* tc_interp_kernel_f32(int taps);
size_t tc_interp_smem_bytes_host(int taps, int ncols, const int* tile);

// ---- scaling (deconv.cu) --------------------------------------------------
// Adjoint step 3 for every item: fhat[r][k] = grid[r][k mod n] * inv_c(k), k in I_N.
// Forward step 1 for every item: grid[r][l] = fhat[r][k] * inv_c(k) if l = k mod n, else 0.
// Work is cut into segments: rows of the last dimension, rows longer than
// kSegment elements cut into pieces of kSegment; a warp takes a segment at a
// time.  A block of kScaleWarps warps takes kSegsPerBlock consecutive
// segments of one item of a batch (kScaleWarps segments of a single item:
// block_offsets null).  An item has nrhs * |I_N| / N_last rows of length
// N_last to crop and nrhs * |I_n| / n_last rows of length n_last to pad.
// The blocks of all items form one flat range of `blocks` blocks;
// block_offsets (device, n_items + 1) are the prefix sums of each item's
// blocks and block_items (device, `blocks`) each block's item (both null for
// a single item).  out / in and nrhs override the item table when non-null.
constexpr int kScaleWarps = 8;
constexpr int kSegsPerBlock = 32;
constexpr int kSegment = 4096;
int64_t scale_blocks(int64_t rows, int64_t row_length, bool batched);
template <typename Real>
cudaError_t launch_deconv_crop(const ItemDev* items, const int* block_offsets, const int* block_items, int64_t blocks,
                               void* out, int nrhs, cudaStream_t st);
template <typename Real>
cudaError_t launch_pad_deconv(const ItemDev* items, const int* block_offsets, const int* block_items, int64_t blocks,
                              const void* in, int nrhs, cudaStream_t st);

}  // namespace gbnfft
