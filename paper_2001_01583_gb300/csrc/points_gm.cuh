// Warp-per-point spreading and interpolation straight on the grid, for
// subproblems holding few points (sparse point sets, the thin bins of a
// clustered set).
//
// A shared tile pays for zeroing, loading and flushing (b + W - 1)^d cells
// per subproblem; with a few points per bin that costs more than the points'
// own W^d cell updates.  Here kGmSplit warps share a subproblem, each taking
// every kGmSplit-th point, with no tile and no block barrier:
//   - lanes split the point's d * W window weights into a per-warp table;
//   - lanes cover one plane of the point's footprint (W x W cells, the last
//     two dimensions; W cells in 1-D) in ceil(W^2 / 32) passes, lanes along
//     the contiguous dimension, so every instruction touches whole grid rows;
//   - spreading adds into the grid with vector atomics (plane by plane over
//     the first dimension in 3-D); interpolation gathers, sums per lane and
//     reduces across the warp.
// Weights and wrapped offsets are computed once per point and reused for
// every right-hand side.
#pragma once

#include "points_tiled.cuh"

namespace gbnfft {

template <int D, int W>
struct GmShape {
  static constexpr int PLANE = D == 1 ? W : W * W;   // footprint cells of one plane
  static constexpr int P = (PLANE + 31) / 32;        // lane passes over a plane
  static constexpr int PLANES = D == 3 ? W : 1;      // planes of the footprint
};

constexpr int kGmWarps = kGmWarpsHost;   // warps per block
constexpr int kGmSplit = kGmSplitHost;   // warps sharing one subproblem's points
// resident blocks asked of the compiler: the kernels wait on global loads,
// so narrow windows trade registers (at most 64) for more warps
template <int W>
constexpr int gm_min_blocks() { return W <= 6 ? 4 : (W <= 8 ? 3 : 1); }

// Per-lane footprint of one point: offsets inside a plane and the product of
// the in-plane weights; the point's first plane index (3-D).
template <int D, int W, typename Real>
struct GmPoint {
  int64_t off[GmShape<D, W>::P];
  Real w[GmShape<D, W>::P];
  int first0;
};

template <int D, int W, typename Real>
__device__ __forceinline__ void gm_point(const SortedPoints<Real>& pts, const ItemDev& it, const int* bc, int idx,
                                         Real* wt, int lane, GmPoint<D, W, Real>& q) {
  using S = GmShape<D, W>;
  const GridGeom& g = it.geom;
  const uint32_t loc = pts.local[idx];
  __syncwarp();
  for (int i = lane; i < D * W; i += 32) {
    const int t = i / W, k = i - t * W;
    const Real base = pts.delta[t][idx] + (Real)(it.win.m - it.win.shift);
    wt[i] = window_psi<Real>(it.win, t, base - (Real)k);
  }
  __syncwarp();
  int first[kMaxDim];
  for (int t = 0; t < D; ++t) first[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift + unpack_local(loc, D, t);
  q.first0 = first[0];
#pragma unroll
  for (int p = 0; p < S::P; ++p) {
    const int c = lane + 32 * p;
    q.off[p] = 0;
    q.w[p] = (Real)0;
    if (c < S::PLANE) {
      if (D == 1) {
        q.off[p] = wrap_near(first[0] + c, g.n[0]);
        q.w[p] = wt[c];
      } else {
        const int iy = c / W, ix = c - iy * W;
        q.off[p] = (int64_t)wrap_near(first[D - 2] + iy, g.n[D - 2]) * g.n[D - 1] +
                   wrap_near(first[D - 1] + ix, g.n[D - 1]);
        q.w[p] = wt[(D - 2) * W + iy] * wt[(D - 1) * W + ix];
      }
    }
  }
}

// sub_selected (points of the subproblem's bin) selects the subproblems of this launch.
template <int D, int W, typename Real>
__global__ void __launch_bounds__(32 * kGmWarps, gm_min_blocks<W>()) k_spread_gm(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  using S = GmShape<D, W>;
  __shared__ Real wt_all[kGmWarps][D * W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* wt = wt_all[warp];
  int lo, hi;
  launch_subs(a, lo, hi);
  const int64_t stride = (int64_t)gridDim.x * kGmWarps;
  const int64_t work = (int64_t)(hi - lo) * kGmSplit;
  for (int64_t wi = (int64_t)blockIdx.x * kGmWarps + warp; wi < work; wi += stride) {
    const int sp = lo + (int)(wi / kGmSplit), part = (int)(wi % kGmSplit);
    const SubProblem sub = a.pts.subs[sp];
    if (part >= sub.count || !sub_selected(a, sub)) continue;
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    const C* f_in = static_cast<const C*>(call.in);
    C* grid = static_cast<C*>(it.grid);
    int bc[kMaxDim];
    bin_coords(sub.bin, g, bc);
    const int64_t plane_cells = D == 3 ? (int64_t)g.n[1] * g.n[2] : 0;
    for (int pp = part; pp < sub.count; pp += kGmSplit) {
      const int idx = sub.start + pp;
      const int j = a.pts.perm[idx];
      GmPoint<D, W, Real> q;
      gm_point<D, W, Real>(a.pts, it, bc, idx, wt, lane, q);
      for (int r = 0; r < call.nrhs; ++r) {
        const C v = f_in[(int64_t)r * it.M + j];
        C* gr = grid + (int64_t)r * g.grid_cells;
        for (int iz = 0; iz < S::PLANES; ++iz) {
          int64_t zoff = 0;
          Real wz = (Real)1;
          if (D == 3) {
            zoff = (int64_t)wrap_near(q.first0 + iz, g.n[0]) * plane_cells;
            wz = wt[iz];
          }
#pragma unroll
          for (int p = 0; p < S::P; ++p) {
            if (lane + 32 * p < S::PLANE) {
              const Real w = wz * q.w[p];
              C val;
              val.x = v.x * w;
              val.y = v.y * w;
              grid_add(gr + zoff + q.off[p], val);
            }
          }
        }
      }
    }
  }
}

template <int D, int W, typename Real>
__global__ void __launch_bounds__(32 * kGmWarps, gm_min_blocks<W>()) k_interp_gm(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  using S = GmShape<D, W>;
  __shared__ Real wt_all[kGmWarps][D * W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* wt = wt_all[warp];
  int lo, hi;
  launch_subs(a, lo, hi);
  const int64_t stride = (int64_t)gridDim.x * kGmWarps;
  const int64_t work = (int64_t)(hi - lo) * kGmSplit;
  for (int64_t wi = (int64_t)blockIdx.x * kGmWarps + warp; wi < work; wi += stride) {
    const int sp = lo + (int)(wi / kGmSplit), part = (int)(wi % kGmSplit);
    const SubProblem sub = a.pts.subs[sp];
    if (part >= sub.count || !sub_selected(a, sub)) continue;
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    C* f_out = static_cast<C*>(call.out);
    const C* grid = static_cast<const C*>(it.grid);
    int bc[kMaxDim];
    bin_coords(sub.bin, g, bc);
    const int64_t plane_cells = D == 3 ? (int64_t)g.n[1] * g.n[2] : 0;
    for (int pp = part; pp < sub.count; pp += kGmSplit) {
      const int idx = sub.start + pp;
      const int j = a.pts.perm[idx];
      GmPoint<D, W, Real> q;
      gm_point<D, W, Real>(a.pts, it, bc, idx, wt, lane, q);
      for (int r = 0; r < call.nrhs; ++r) {
        const C* gr = grid + (int64_t)r * g.grid_cells;
        Real ar = 0, ai = 0;
        for (int iz = 0; iz < S::PLANES; ++iz) {
          int64_t zoff = 0;
          Real wz = (Real)1;
          if (D == 3) {
            zoff = (int64_t)wrap_near(q.first0 + iz, g.n[0]) * plane_cells;
            wz = wt[iz];
          }
          Real pr = 0, pi = 0;
#pragma unroll
          for (int p = 0; p < S::P; ++p) {
            if (lane + 32 * p < S::PLANE) {
              const C c = gr[zoff + q.off[p]];
              pr += c.x * q.w[p];
              pi += c.y * q.w[p];
            }
          }
          ar += wz * pr;
          ai += wz * pi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          ar += __shfl_xor_sync(0xffffffffu, ar, o);
          ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) f_out[(int64_t)r * it.M + j] = cmake<C>(ar, ai);
      }
    }
  }
}

// Taps instantiated (every window of the library: 2 .. 26, even).
#define GBNFFT_GM_TAPS(X, D, R) \
  X(D, 2, R) X(D, 4, R) X(D, 6, R) X(D, 8, R) X(D, 10, R) X(D, 12, R) X(D, 14, R) X(D, 16, R) X(D, 18, R) \
      X(D, 20, R) X(D, 22, R) X(D, 24, R) X(D, 26, R)

}  // namespace gbnfft
