// Tiled spreading (adjoint step 1, Fig. 1) and interpolation (forward step 3,
// Fig. 2) over bin-sorted points.
//
// A block takes subproblems (runs of at most P points of one bin) in turn.
// For a bin of b_0 x ... x b_{d-1} cells the tile holds the bin plus the
// window halo, (b_t + W - 1) cells per dimension, for rhs_per_pass right-hand
// sides at once.
//   spread: zero the tile, every thread adds its points' W^d weighted values
//           with shared-memory atomics, then the tile is added to the global
//           grid once (vector atomics, since halos of neighbouring bins and
//           several subproblems of one bin overlap).
//   interp: load the tile from the grid once, every thread gathers its
//           points' W^d cells from shared memory, no atomics.
// The window weights of a point are computed once per point (W per
// dimension) and reused for every right-hand side.
#pragma once

#include "kernels.h"

namespace gbnfft {

template <typename Real>
__device__ __forceinline__ void smem_add(Real* p, Real v) {
  atomicAdd(p, v);
}

__device__ __forceinline__ void grid_add(float2* p, float2 v) { atomicAdd(p, v); }
__device__ __forceinline__ void grid_add(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// v mod n for v in [-n, 2n).
__device__ __forceinline__ int wrap_near(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Bin coordinates of a bin id (C order over the d used dimensions).
__device__ __forceinline__ void bin_coords(int bin, const GridGeom& g, int* bc) {
  for (int t = g.d - 1; t >= 0; --t) {
    bc[t] = bin % g.nbins[t];
    bin /= g.nbins[t];
  }
}

// Tile element e (C order over the tile) -> flat grid index, with the
// periodic wrap of the oversampled grid.
__device__ __forceinline__ int64_t tile_to_grid(int e, const GridGeom& g, const int* origin) {
  int64_t flat = 0;
  int rem = e;
  int coord[kMaxDim];
  for (int t = g.d - 1; t >= 0; --t) {
    coord[t] = rem % g.tile[t];
    rem /= g.tile[t];
  }
  for (int t = 0; t < g.d; ++t) flat = flat * g.n[t] + wrap_mod(origin[t] + coord[t], g.n[t]);
  return flat;
}

template <int W, typename Real>
__device__ __forceinline__ void taps_of(const WindowDev& win, int t, Real delta, Real* w) {
  const Real base = delta + (Real)(win.m - win.shift);
#pragma unroll
  for (int i = 0; i < W; ++i) w[i] = window_psi<Real>(win, t, base - (Real)i);
}

template <int D, int W, typename Real>
__global__ void __launch_bounds__(256) k_spread_tiled(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* tile = reinterpret_cast<Real*>(smem_raw);  // interleaved (re, im)
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    if (!sub_selected(a, s)) continue;   // block-uniform
    const ItemDev& it = a.items[s.item];
    const GridGeom& g = it.geom;
    const WindowDev& win = it.win;
    const ItemCall call = item_call(a, it);
    const C* f_in = static_cast<const C*>(call.in);
    C* grid = static_cast<C*>(it.grid);
    const int64_t M = it.M;
    const int tc = g.tile_cells;
    const int T1 = D >= 2 ? g.tile[1] : 1;
    const int T2 = D >= 3 ? g.tile[2] : 1;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < D; ++t) origin[t] = bc[t] * g.bin[t] - win.m + win.shift;
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      for (int e = threadIdx.x; e < 2 * tc * np; e += blockDim.x) tile[e] = (Real)0;
      __syncthreads();
      for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
        const int idx = s.start + p;
        const int j = a.pts.perm[idx];
        const uint32_t loc = a.pts.local[idx];
        Real w0[W], w1[W], w2[W];
        taps_of<W, Real>(win, 0, a.pts.delta[0][idx], w0);
        if (D >= 2) taps_of<W, Real>(win, 1, a.pts.delta[1][idx], w1);
        if (D >= 3) taps_of<W, Real>(win, 2, a.pts.delta[2][idx], w2);
        const int l0 = unpack_local(loc, D, 0);
        const int l1 = D >= 2 ? unpack_local(loc, D, 1) : 0;
        const int l2 = D >= 3 ? unpack_local(loc, D, 2) : 0;
        for (int r = 0; r < np; ++r) {
          const C v = f_in[(int64_t)(r0 + r) * M + j];
          Real* tr = tile + 2 * r * tc;
          if (D == 1) {
#pragma unroll
            for (int i0 = 0; i0 < W; ++i0) {
              Real* c = tr + 2 * (l0 + i0);
              smem_add(c, v.x * w0[i0]);
              smem_add(c + 1, v.y * w0[i0]);
            }
          } else if (D == 2) {
            for (int i0 = 0; i0 < W; ++i0) {
              const Real vr = v.x * w0[i0], vi = v.y * w0[i0];
              Real* row = tr + 2 * ((l0 + i0) * T1 + l1);
#pragma unroll
              for (int i1 = 0; i1 < W; ++i1) {
                smem_add(row + 2 * i1, vr * w1[i1]);
                smem_add(row + 2 * i1 + 1, vi * w1[i1]);
              }
            }
          } else {
            for (int i0 = 0; i0 < W; ++i0) {
              for (int i1 = 0; i1 < W; ++i1) {
                const Real w01 = w0[i0] * w1[i1];
                const Real vr = v.x * w01, vi = v.y * w01;
                Real* row = tr + 2 * (((l0 + i0) * T1 + l1 + i1) * T2 + l2);
#pragma unroll
                for (int i2 = 0; i2 < W; ++i2) {
                  smem_add(row + 2 * i2, vr * w2[i2]);
                  smem_add(row + 2 * i2 + 1, vi * w2[i2]);
                }
              }
            }
          }
        }
      }
      __syncthreads();
      // flush the tile into the grid once
      for (int e = threadIdx.x; e < tc * np; e += blockDim.x) {
        const int r = e / tc;
        const int ee = e - r * tc;
        C val;
        val.x = tile[2 * e];
        val.y = tile[2 * e + 1];
        if (val.x != (Real)0 || val.y != (Real)0)
          grid_add(grid + (int64_t)(r0 + r) * g.grid_cells + tile_to_grid(ee, g, origin), val);
      }
      __syncthreads();
    }
  }
}

template <int D, int W, typename Real>
__global__ void __launch_bounds__(256) k_interp_tiled(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    if (!sub_selected(a, s)) continue;   // block-uniform
    const ItemDev& it = a.items[s.item];
    const GridGeom& g = it.geom;
    const WindowDev& win = it.win;
    const ItemCall call = item_call(a, it);
    C* f_out = static_cast<C*>(call.out);
    const C* grid_in = static_cast<const C*>(it.grid);
    const int64_t M = it.M;
    const int tc = g.tile_cells;
    const int T1 = D >= 2 ? g.tile[1] : 1;
    const int T2 = D >= 3 ? g.tile[2] : 1;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < D; ++t) origin[t] = bc[t] * g.bin[t] - win.m + win.shift;
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      __syncthreads();
      for (int e = threadIdx.x; e < tc * np; e += blockDim.x) {
        const int r = e / tc;
        const int ee = e - r * tc;
        tile[e] = grid_in[(int64_t)(r0 + r) * g.grid_cells + tile_to_grid(ee, g, origin)];
      }
      __syncthreads();
      for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
        const int idx = s.start + p;
        const int j = a.pts.perm[idx];
        const uint32_t loc = a.pts.local[idx];
        Real w0[W], w1[W], w2[W];
        taps_of<W, Real>(win, 0, a.pts.delta[0][idx], w0);
        if (D >= 2) taps_of<W, Real>(win, 1, a.pts.delta[1][idx], w1);
        if (D >= 3) taps_of<W, Real>(win, 2, a.pts.delta[2][idx], w2);
        const int l0 = unpack_local(loc, D, 0);
        const int l1 = D >= 2 ? unpack_local(loc, D, 1) : 0;
        const int l2 = D >= 3 ? unpack_local(loc, D, 2) : 0;
        for (int r = 0; r < np; ++r) {
          const C* tr = tile + r * tc;
          Real ar = 0, ai = 0;
          if (D == 1) {
#pragma unroll
            for (int i0 = 0; i0 < W; ++i0) {
              const C c = tr[l0 + i0];
              ar += c.x * w0[i0];
              ai += c.y * w0[i0];
            }
          } else if (D == 2) {
            for (int i0 = 0; i0 < W; ++i0) {
              const C* row = tr + (l0 + i0) * T1 + l1;
              Real rr = 0, ri = 0;
#pragma unroll
              for (int i1 = 0; i1 < W; ++i1) {
                const C c = row[i1];
                rr += c.x * w1[i1];
                ri += c.y * w1[i1];
              }
              ar += rr * w0[i0];
              ai += ri * w0[i0];
            }
          } else {
            for (int i0 = 0; i0 < W; ++i0) {
              Real pr = 0, pi = 0;
              for (int i1 = 0; i1 < W; ++i1) {
                const C* row = tr + ((l0 + i0) * T1 + l1 + i1) * T2 + l2;
                Real rr = 0, ri = 0;
#pragma unroll
                for (int i2 = 0; i2 < W; ++i2) {
                  const C c = row[i2];
                  rr += c.x * w2[i2];
                  ri += c.y * w2[i2];
                }
                pr += rr * w1[i1];
                pi += ri * w1[i1];
              }
              ar += pr * w0[i0];
              ai += pi * w0[i0];
            }
          }
          C out;
          out.x = ar;
          out.y = ai;
          f_out[(int64_t)(r0 + r) * M + j] = out;
        }
      }
      __syncthreads();
    }
  }
}

// Kernel pointer tables: (d, W) -> instantiation, W even in [2, kMaxTaps]
// (d = 3 up to 26).  Unsupported combinations give nullptr.
#define GBNFFT_TAPS_1_2(X, D, R)                                                                           \
  X(D, 2, R) X(D, 4, R) X(D, 6, R) X(D, 8, R) X(D, 10, R) X(D, 12, R) X(D, 14, R) X(D, 16, R) X(D, 18, R) \
      X(D, 20, R) X(D, 22, R) X(D, 24, R) X(D, 26, R) X(D, 28, R) X(D, 30, R) X(D, 32, R)
#define GBNFFT_TAPS_3(X, D, R) \
  X(D, 2, R) X(D, 4, R) X(D, 6, R) X(D, 8, R) X(D, 10, R) X(D, 12, R) X(D, 14, R) X(D, 16, R) X(D, 18, R) \
      X(D, 20, R) X(D, 22, R) X(D, 24, R) X(D, 26, R)

}  // namespace gbnfft
