// Global-memory point kernels: one thread per point adding straight into the
// grid with atomics (the paper's spread kernel, Section 3) and gathering
// straight from it (its interpolate kernel, Section 3), for any dimension
// and tap count; and the kernel-pointer accessors of the tiled kernels.
#include "points_tiled.cuh"

namespace gbnfft {

namespace {

// Per point and dimension: weights and wrapped grid indices of the W taps.
template <typename Real>
__device__ __forceinline__ void global_taps(const SortedPoints<Real>& pts, const ItemDev& it, int idx,
                                            const int* origin, Real (*w)[kMaxTaps], int (*gi)[kMaxTaps]) {
  const GridGeom& g = it.geom;
  const int W = it.win.taps;
  const uint32_t loc = pts.local[idx];
  for (int t = 0; t < g.d; ++t) {
    const Real base = pts.delta[t][idx] + (Real)(it.win.m - it.win.shift);
    const int c0 = origin[t] + unpack_local(loc, g.d, t);
    for (int i = 0; i < W; ++i) {
      w[t][i] = window_psi_any<Real>(it.win, t, base - (Real)i);
      gi[t][i] = wrap_mod(c0 + i, g.n[t]);
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_spread_global(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
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
    const int W = it.win.taps;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < g.d; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
      const int idx = s.start + p;
      const int j = a.pts.perm[idx];
      Real w[kMaxDim][kMaxTaps];
      int gi[kMaxDim][kMaxTaps];
      global_taps<Real>(a.pts, it, idx, origin, w, gi);
      for (int r = 0; r < call.nrhs; ++r) {
        const C v = f_in[(int64_t)r * it.M + j];
        C* gr = grid + (int64_t)r * g.grid_cells;
        if (g.d == 1) {
          for (int i0 = 0; i0 < W; ++i0) grid_add(gr + gi[0][i0], cmake<C>(v.x * w[0][i0], v.y * w[0][i0]));
        } else if (g.d == 2) {
          for (int i0 = 0; i0 < W; ++i0)
            for (int i1 = 0; i1 < W; ++i1) {
              const Real ww = w[0][i0] * w[1][i1];
              grid_add(gr + (int64_t)gi[0][i0] * g.n[1] + gi[1][i1], cmake<C>(v.x * ww, v.y * ww));
            }
        } else {
          for (int i0 = 0; i0 < W; ++i0)
            for (int i1 = 0; i1 < W; ++i1) {
              const Real w01 = w[0][i0] * w[1][i1];
              const int64_t row = ((int64_t)gi[0][i0] * g.n[1] + gi[1][i1]) * g.n[2];
              for (int i2 = 0; i2 < W; ++i2) {
                const Real ww = w01 * w[2][i2];
                grid_add(gr + row + gi[2][i2], cmake<C>(v.x * ww, v.y * ww));
              }
            }
        }
      }
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_interp_global(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    if (!sub_selected(a, s)) continue;   // block-uniform
    const ItemDev& it = a.items[s.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    C* f_out = static_cast<C*>(call.out);
    const C* grid = static_cast<const C*>(it.grid);
    const int W = it.win.taps;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < g.d; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
      const int idx = s.start + p;
      const int j = a.pts.perm[idx];
      Real w[kMaxDim][kMaxTaps];
      int gi[kMaxDim][kMaxTaps];
      global_taps<Real>(a.pts, it, idx, origin, w, gi);
      for (int r = 0; r < call.nrhs; ++r) {
        const C* gr = grid + (int64_t)r * g.grid_cells;
        Real ar = 0, ai = 0;
        if (g.d == 1) {
          for (int i0 = 0; i0 < W; ++i0) {
            const C c = gr[gi[0][i0]];
            ar += c.x * w[0][i0];
            ai += c.y * w[0][i0];
          }
        } else if (g.d == 2) {
          for (int i0 = 0; i0 < W; ++i0) {
            Real rr = 0, ri = 0;
            for (int i1 = 0; i1 < W; ++i1) {
              const C c = gr[(int64_t)gi[0][i0] * g.n[1] + gi[1][i1]];
              rr += c.x * w[1][i1];
              ri += c.y * w[1][i1];
            }
            ar += rr * w[0][i0];
            ai += ri * w[0][i0];
          }
        } else {
          for (int i0 = 0; i0 < W; ++i0) {
            Real pr = 0, pi = 0;
            for (int i1 = 0; i1 < W; ++i1) {
              const int64_t row = ((int64_t)gi[0][i0] * g.n[1] + gi[1][i1]) * g.n[2];
              Real rr = 0, ri = 0;
              for (int i2 = 0; i2 < W; ++i2) {
                const C c = gr[row + gi[2][i2]];
                rr += c.x * w[2][i2];
                ri += c.y * w[2][i2];
              }
              pr += rr * w[1][i1];
              pi += ri * w[1][i1];
            }
            ar += pr * w[0][i0];
            ai += pi * w[0][i0];
          }
        }
        f_out[(int64_t)r * it.M + j] = cmake<C>(ar, ai);
      }
    }
  }
}

}  // namespace

const void* global_kernel_f32(bool spread) {
  return spread ? reinterpret_cast<const void*>(&k_spread_global<float>)
                : reinterpret_cast<const void*>(&k_interp_global<float>);
}
const void* global_kernel_f64(bool spread) {
  return spread ? reinterpret_cast<const void*>(&k_spread_global<double>)
                : reinterpret_cast<const void*>(&k_interp_global<double>);
}

}  // namespace gbnfft
