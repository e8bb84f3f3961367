// Warp-per-point spreading and interpolation (d = 2, 3).
//
// One warp handles one point at a time.  The point's W^d cells form rows of
// W cells along the fastest dimension; lane (ix, q) = (lane % W, lane / W)
// takes cell ix of rows q, q + Q, q + 2Q, ... (Q = 32 / W rows per pass), so
// the lanes of a warp never touch the same cell for one point.
//
//   spread: every warp owns a private tile (the bin plus halo) in shared
//           memory and updates it with plain loads and stores -- no atomics;
//           after the subproblem the block adds its warps' tiles and adds the
//           sum to the grid once (vector atomics, since halos overlap);
//   interp: the block shares one tile loaded from the grid; lanes gather
//           their cells and a shuffle tree sums the warp's partial sums.
//
// A warp takes its points in batches of 32 consecutive sorted points: lane L
// loads point L's record and value (coalesced) and evaluates its d*W window
// weights once into a per-warp table; the warp then walks the batch, forming
// each point's W^(d-1) row weights in shared memory and reusing the weights
// for every right-hand side of the pass.  The row pitch of a tile (`pitch`, >= the tile's
// fastest extent) is chosen on the host to spread a warp's rows over the
// shared-memory banks.
#pragma once

#include "points_tiled.cuh"

namespace gbnfft {

template <int D, int W>
struct WppShape {
  static constexpr int Q = (32 / W) > 0 ? (32 / W) : 1;          // rows per pass
  static constexpr int ROWS = D == 3 ? W * W : W;                 // rows of a footprint
  static constexpr int ITERS = (ROWS + Q - 1) / Q;                // passes per point
  static constexpr int BATCH = ITERS < 8 ? ITERS : 8;             // cells in flight per lane
};

// Shared memory per warp after the tiles: the weights of a batch of 32
// points (d*W each) and the row weights of the current point.
template <int D, int W, typename Real>
__host__ __device__ constexpr int wpp_scratch_reals() {
  return 32 * D * W + WppShape<D, W>::ROWS;
}

// A warp's batch of up to 32 consecutive sorted points: lane L loads point
// L's record (coalesced) and its window weights into wtab[L][t*W + i].
template <int D, int W, typename Real>
struct WppBatch {
  int j;           // original index of this lane's point
  uint32_t loc;    // packed in-bin cell of this lane's point
};

template <int D, int W, typename Real>
__device__ __forceinline__ WppBatch<D, W, Real> wpp_load_batch(const PointKernelArgs<Real>& a, const WindowDev& win,
                                                               int first, int nb, Real* wtab, int lane) {
  WppBatch<D, W, Real> b{0, 0u};
  if (lane < nb) {
    const int idx = first + lane;
    b.j = a.pts.perm[idx];
    b.loc = a.pts.local[idx];
    Real* w = wtab + lane * (D * W);
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const Real base = a.pts.delta[t][idx] + (Real)(win.m - win.shift);
#pragma unroll
      for (int i = 0; i < W; ++i) w[t * W + i] = window_psi<Real>(win, t, base - (Real)i);
    }
  }
  __syncwarp();
  return b;
}

// Row weights of point pp of the batch: wrow[row] = w_0(z) w_1(y) (d = 3) or w_0(row) (d = 2).
template <int D, int W, typename Real>
__device__ __forceinline__ void wpp_rows(const Real* wt, Real* wrow, int lane) {
  if (D == 3) {
    for (int e = lane; e < W * W; e += 32) wrow[e] = wt[e / W] * wt[W + (e - (e / W) * W)];
  } else {
    for (int e = lane; e < W; e += 32) wrow[e] = wt[e];
  }
  __syncwarp();
}

template <int D, int W, typename Real>
__global__ void __launch_bounds__(256) k_spread_wpp(PointKernelArgs<Real> a, WppLayout lay) {
  using C = typename Cplx<Real>::type;
  using S = WppShape<D, W>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = lay.warps;
  const int np_max = a.rhs_per_pass;
  C* tiles = reinterpret_cast<C*>(smem_raw);                                   // [nw][np][warp_cells]
  Real* scratch = reinterpret_cast<Real*>(tiles + (size_t)nw * np_max * lay.warp_cells);
  Real* wtab = scratch + warp * wpp_scratch_reals<D, W, Real>();
  Real* wrow = wtab + 32 * D * W;
  // the batch's values, [np][32] per warp, after all warps' weight tables
  C* vtab = reinterpret_cast<C*>(scratch + nw * wpp_scratch_reals<D, W, Real>()) + (size_t)warp * np_max * 32;
  C* mine = tiles + (size_t)warp * np_max * lay.warp_cells;
  const int ix = lane % W, q = lane / W;
  const bool active = q < S::Q;
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    if (!sub_selected(a, s)) continue;   // block-uniform
    const ItemDev& it = a.items[s.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    const C* f_in = static_cast<const C*>(call.in);
    C* grid = static_cast<C*>(it.grid);
    const int T1 = D == 3 ? g.tile[1] : 1;                                     // rows of a 3-D tile plane
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < D; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      for (int e = lane; e < np * lay.warp_cells; e += 32) mine[e] = cmake<C>(0.0, 0.0);
      __syncwarp();
      for (int pb = warp * 32; pb < s.count; pb += nw * 32) {
        const int nb = min(32, s.count - pb);
        const WppBatch<D, W, Real> bt = wpp_load_batch<D, W, Real>(a, it.win, s.start + pb, nb, wtab, lane);
        for (int r = 0; r < np; ++r)
          if (lane < nb) vtab[r * 32 + lane] = f_in[(int64_t)(r0 + r) * it.M + bt.j];
        __syncwarp();
        for (int pp = 0; pp < nb; ++pp) {
          const uint32_t loc = __shfl_sync(0xffffffffu, bt.loc, pp);
          const Real* wt = wtab + pp * (D * W);
          wpp_rows<D, W, Real>(wt, wrow, lane);
          const Real wx = wt[(D - 1) * W + ix];
          const int l0 = unpack_local(loc, D, 0);
          const int l1 = unpack_local(loc, D, 1);
          const int l2 = D == 3 ? unpack_local(loc, D, 2) : 0;
          const int base = D == 3 ? ((l0 * T1 + l1) * lay.pitch + l2 + ix) : (l0 * lay.pitch + l1 + ix);
          for (int r = 0; r < np; ++r) {
            const C v = vtab[r * 32 + pp];
            const Real vr = v.x * wx, vi = v.y * wx;
            C* tr = mine + r * lay.warp_cells;
#pragma unroll
            for (int k0 = 0; k0 < S::ITERS; k0 += S::BATCH) {
              C cell[S::BATCH];
              int addr[S::BATCH];
#pragma unroll
              for (int b = 0; b < S::BATCH; ++b) {
                const int row = (k0 + b) * S::Q + q;
                const int zr = D == 3 ? row / W : row;
                const int yr = D == 3 ? row - zr * W : 0;
                addr[b] = base + (D == 3 ? (zr * T1 + yr) * lay.pitch : zr * lay.pitch);
                if (active && k0 + b < S::ITERS && row < S::ROWS) cell[b] = tr[addr[b]];
              }
#pragma unroll
              for (int b = 0; b < S::BATCH; ++b) {
                const int row = (k0 + b) * S::Q + q;
                if (active && k0 + b < S::ITERS && row < S::ROWS) {
                  const Real w = wrow[row];
                  cell[b].x += vr * w;
                  cell[b].y += vi * w;
                  tr[addr[b]] = cell[b];
                }
              }
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // add the warps' tiles and flush the sum into the grid once
      for (int e = threadIdx.x; e < np * g.tile_cells; e += blockDim.x) {
        const int r = e / g.tile_cells;
        const int ee = e - r * g.tile_cells;
        const int last = g.tile[D - 1];
        const int row = ee / last, col = ee - row * last;
        const int off = r * lay.warp_cells + row * lay.pitch + col;
        Real sx = 0, sy = 0;
        for (int w = 0; w < nw; ++w) {
          const C c = tiles[(size_t)w * np_max * lay.warp_cells + off];
          sx += c.x;
          sy += c.y;
        }
        if (sx != (Real)0 || sy != (Real)0)
          grid_add(grid + (int64_t)(r0 + r) * g.grid_cells + tile_to_grid(ee, g, origin), cmake<C>(sx, sy));
      }
      __syncthreads();
    }
  }
}

template <int D, int W, typename Real>
__global__ void __launch_bounds__(256) k_interp_wpp(PointKernelArgs<Real> a, WppLayout lay) {
  using C = typename Cplx<Real>::type;
  using S = WppShape<D, W>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = lay.warps;
  const int tile_elems = lay.warp_cells;
  C* tile = reinterpret_cast<C*>(smem_raw);                                    // [np][rows][pitch]
  Real* scratch = reinterpret_cast<Real*>(tile + (size_t)a.rhs_per_pass * tile_elems);
  Real* wtab = scratch + warp * wpp_scratch_reals<D, W, Real>();
  Real* wrow = wtab + 32 * D * W;
  const int ix = lane % W, q = lane / W;
  const bool active = q < S::Q;
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    if (!sub_selected(a, s)) continue;   // block-uniform
    const ItemDev& it = a.items[s.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    C* f_out = static_cast<C*>(call.out);
    const C* grid_in = static_cast<const C*>(it.grid);
    const int T1 = D == 3 ? g.tile[1] : 1;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < D; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      __syncthreads();
      for (int e = threadIdx.x; e < np * g.tile_cells; e += blockDim.x) {
        const int r = e / g.tile_cells;
        const int ee = e - r * g.tile_cells;
        const int last = g.tile[D - 1];
        const int row = ee / last, col = ee - row * last;
        tile[r * tile_elems + row * lay.pitch + col] =
            grid_in[(int64_t)(r0 + r) * g.grid_cells + tile_to_grid(ee, g, origin)];
      }
      __syncthreads();
      for (int pb = warp * 32; pb < s.count; pb += nw * 32) {
        const int nb = min(32, s.count - pb);
        const WppBatch<D, W, Real> bt = wpp_load_batch<D, W, Real>(a, it.win, s.start + pb, nb, wtab, lane);
        for (int r = 0; r < np; ++r) {
          const C* tr = tile + r * tile_elems;
          // lane L keeps the finished value of point L of the batch
          Real outr = 0, outi = 0;
          for (int pp = 0; pp < nb; ++pp) {
            const uint32_t loc = __shfl_sync(0xffffffffu, bt.loc, pp);
            const Real* wt = wtab + pp * (D * W);
            wpp_rows<D, W, Real>(wt, wrow, lane);
            const Real wx = wt[(D - 1) * W + ix];
            const int l0 = unpack_local(loc, D, 0);
            const int l1 = unpack_local(loc, D, 1);
            const int l2 = D == 3 ? unpack_local(loc, D, 2) : 0;
            const int base = D == 3 ? ((l0 * T1 + l1) * lay.pitch + l2 + ix) : (l0 * lay.pitch + l1 + ix);
            Real ar = 0, ai = 0;
#pragma unroll
            for (int k = 0; k < S::ITERS; ++k) {
              const int row = k * S::Q + q;
              if (active && row < S::ROWS) {
                const int zr = D == 3 ? row / W : row;
                const int yr = D == 3 ? row - zr * W : 0;
                const C c = tr[base + (D == 3 ? (zr * T1 + yr) * lay.pitch : zr * lay.pitch)];
                const Real w = wrow[row];
                ar += c.x * w;
                ai += c.y * w;
              }
            }
            ar *= wx;
            ai *= wx;
            for (int o = 16; o > 0; o >>= 1) {
              ar += __shfl_xor_sync(0xffffffffu, ar, o);
              ai += __shfl_xor_sync(0xffffffffu, ai, o);
            }
            if (lane == pp) {
              outr = ar;
              outi = ai;
            }
            __syncwarp();
          }
          if (lane < nb) f_out[(int64_t)(r0 + r) * it.M + bt.j] = cmake<C>(outr, outi);
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
}

#define GBNFFT_WPP_TAPS(X, D, R) \
  X(D, 2, R) X(D, 4, R) X(D, 6, R) X(D, 8, R) X(D, 10, R) X(D, 12, R) X(D, 14, R) X(D, 16, R)

}  // namespace gbnfft
