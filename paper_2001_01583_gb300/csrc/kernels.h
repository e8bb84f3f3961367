// Internal launch interface between the host plan code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gbnfft {

// ---- set_points (sort.cu) -------------------------------------------------
// Cell and bin of every point, and its rank inside its bin (warp-aggregated
// atomics on bin_count).  err gets bit 0 for a non-finite coordinate.
template <typename Real>
cudaError_t launch_bin_count(const double* x, int64_t M, const GridGeom& g, int* bin_count, int2* bin_rank,
                             int* err, cudaStream_t st);
// Exclusive prefix sum of n ints (one block); *total = sum (may be null).
cudaError_t launch_scan(const int* in, int* out, int n, int* total, cudaStream_t st);
// Write every point to its sorted slot: perm, packed in-bin offsets, deltas.
template <typename Real>
cudaError_t launch_scatter(const double* x, int64_t M, const GridGeom& g, const int* bin_start, const int2* bin_rank,
                           int* perm, uint32_t* local, Real* const* delta, cudaStream_t st);
// Subproblems per bin (ceil(count / P)), then their records after a scan.
cudaError_t launch_subproblem_count(const int* bin_count, int nbins, int P, int* sub_count, cudaStream_t st);
cudaError_t launch_subproblem_fill(const int* bin_count, const int* bin_start, const int* sub_start, int nbins,
                                   int P, SubProblem* subs, cudaStream_t st);

// ---- spreading / interpolation (spread_*.cu, interp_*.cu) -----------------
template <typename Real>
struct PointKernelArgs {
  SortedPoints<Real> pts;
  GridGeom geom;
  WindowDev win;
  int64_t M;
  const typename Cplx<Real>::type* f_in;   // spread: R x M values
  typename Cplx<Real>::type* f_out;        // interp: R x M values
  typename Cplx<Real>::type* grid;         // R grids of geom.grid_cells
  const typename Cplx<Real>::type* grid_in;
  int nrhs;                                // right-hand sides in this call
  int rhs_per_pass;                        // tiles held in shared memory at once
};

// Tiled (shared-memory) kernels; false if (d, taps) has no instantiation.
template <typename Real>
bool launch_spread_tiled(const PointKernelArgs<Real>& a, int blocks, int threads, size_t smem, cudaStream_t st,
                         cudaError_t* err);
template <typename Real>
bool launch_interp_tiled(const PointKernelArgs<Real>& a, int blocks, int threads, size_t smem, cudaStream_t st,
                         cudaError_t* err);
// Global-memory kernels (any d, any taps <= kMaxTaps).
template <typename Real>
cudaError_t launch_spread_global(const PointKernelArgs<Real>& a, int blocks, int threads, cudaStream_t st);
template <typename Real>
cudaError_t launch_interp_global(const PointKernelArgs<Real>& a, int blocks, int threads, cudaStream_t st);
// Occupancy query for the tiled kernels (blocks per SM, 0 if unsupported).
template <typename Real>
int tiled_blocks_per_sm(int d, int taps, bool spread, int threads, size_t smem);
template <typename Real>
cudaError_t tiled_set_smem_limit(int d, int taps, bool spread, size_t smem);

// Warp-per-point kernels (points_wpp.cuh, d = 2, 3, taps <= 16): the block
// layout the host chooses.
struct WppLayout {
  int pitch;        // row pitch of a tile, in complex elements
  int warp_cells;   // elements of one private tile (rows * pitch), spread only
  int warps;        // warps per block
};
const void* wpp_kernel_f32(int d, int taps, bool spread);
const void* wpp_kernel_f64(int d, int taps, bool spread);
// 3-D shared-tile kernels (points_planes.cuh): plane-owner spreading and
// point-group interpolation, taps <= 16, same WppLayout (warps divides taps
// for spreading).
const void* planes_kernel_f32(int taps, int warps, bool spread);
const void* planes_kernel_f64(int taps, int warps, bool spread);
size_t planes_table_bytes_f32(int taps, int bp, int np, int nw, const int* tile);
size_t planes_table_bytes_f64(int taps, int bp, int np, int nw, const int* tile);

// ---- scaling (deconv.cu) --------------------------------------------------
// Adjoint step 3: fhat[r][k] = grid[r][k mod n] * inv_c(k), k in I_N.
template <typename Real>
cudaError_t launch_deconv_crop(const typename Cplx<Real>::type* grid, typename Cplx<Real>::type* fhat,
                               const double* const* inv_c, const GridGeom& g, const int* N, int R, cudaStream_t st);
// Forward step 1: grid[r][l] = fhat[r][k] * inv_c(k) if l = k mod n, k in I_N, else 0.
template <typename Real>
cudaError_t launch_pad_deconv(const typename Cplx<Real>::type* fhat, typename Cplx<Real>::type* grid,
                              const double* const* inv_c, const GridGeom& g, const int* N, int R, cudaStream_t st);

}  // namespace gbnfft
