// 3-D spreading of sparse bins by the cells' owners, without atomics.
//
// A warp owns one bin's cells at a time (an owner region R of
// bin_0 x bin_1 x bin_2 cells, ragged at the grid's edge) and holds them in
// its own shared-memory tile.  It visits the bins within the window's reach
// of R, skips the dense ones (their points are spread by the tiled kernel
// afterwards) and, for every point of a sparse bin whose footprint meets R,
// adds the footprint's part inside R: lanes cover a W x W plane of the
// footprint, masked to R, plane by plane along the first dimension.  Then it
// writes R into the grid with plain stores, every cell exactly once, so the
// sparse part of the grid costs no atomics and needs no prior clearing.
//
// Eq. 8: the adjoint is a sum over points, so splitting the points into the
// sparse bins' (gathered here by owners) and the dense bins' (added by the
// tiled kernel after this one) changes nothing but the order of additions.
//
// Requires n_t >= bin_t + W - 1 in every dimension (then at most one
// periodic image of a footprint meets R) and at most kOwnerReach bins per
// dimension within the window's reach of R (both checked on the host).
#pragma once

#include "points_tiled.cuh"

namespace gbnfft {

constexpr int kOwnerWarps = kOwnerWarpsHost;
constexpr int kOwnerReach = kOwnerReachHost;   // neighbour bins per dimension, at most

template <int W, typename Real>
__global__ void __launch_bounds__(32 * kOwnerWarps) k_spread_owner(PointKernelArgs<Real> a, int sparse_below) {
  using C = typename Cplx<Real>::type;
  constexpr int P = (W * W + 31) / 32;   // lane passes over a footprint plane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nbins = a.bin_end - a.bin_begin;
  if (nbins <= 0) return;
  // this launch's bins share their shape: tile = one bin
  const GridGeom& g0 = a.items[a.item_begin].geom;
  const int b0 = g0.bin[0], b1 = g0.bin[1], b2 = g0.bin[2];
  const int cells = b0 * b1 * b2;
  C* tile = reinterpret_cast<C*>(smem_raw) + (size_t)warp * cells;
  Real* wt = reinterpret_cast<Real*>(reinterpret_cast<C*>(smem_raw) + (size_t)kOwnerWarps * cells) + warp * 3 * W;
  // per-lane footprint plane slots (compile-time W: cheap divisions)
  int sy[P], sx[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int s = lane + 32 * p;
    sy[p] = s < W * W ? s / W : -1;
    sx[p] = s < W * W ? s - (s / W) * W : -1;
  }
  const int stride = gridDim.x * kOwnerWarps;
  for (int ob = blockIdx.x * kOwnerWarps + warp; ob < nbins; ob += stride) {
    const int gbin = a.bin_begin + ob;
    // the item holding this bin: last item with bin_offset <= gbin
    int lo = a.item_begin, hi = a.item_end;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.items[mid].bin_offset <= gbin) lo = mid;
      else hi = mid;
    }
    const ItemDev& it = a.items[lo];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    const C* f_in = static_cast<const C*>(call.in);
    C* grid = static_cast<C*>(it.grid);
    int bc[kMaxDim];
    bin_coords(gbin - it.bin_offset, g, bc);
    int olo[3], olen[3], nlist[3][kOwnerReach], ncount[3];
    const int left = it.win.m - it.win.shift;   // cells left of a point's cell
    const int right = W - 1 - left;             // cells right of it
    for (int t = 0; t < 3; ++t) {
      olo[t] = bc[t] * g.bin[t];
      olen[t] = min(g.bin[t], g.n[t] - olo[t]);
      // bins holding the cells whose points reach R: the cells
      // [olo - right, olo + olen - 1 + left], wrapped into one or two
      // segments of [0, n) (no cell twice: the span is <= n); last bins may
      // be ragged, so bins come from wrapped cells, each listed once
      const int lo_c = olo[t] - right, hi_c = olo[t] + olen[t] - 1 + left;
      int seg[2][2], nseg = 1;
      if (lo_c < 0) {
        seg[0][0] = lo_c + g.n[t], seg[0][1] = g.n[t] - 1, seg[1][0] = 0, seg[1][1] = hi_c, nseg = 2;
      } else if (hi_c >= g.n[t]) {
        seg[0][0] = lo_c, seg[0][1] = g.n[t] - 1, seg[1][0] = 0, seg[1][1] = hi_c - g.n[t], nseg = 2;
      } else {
        seg[0][0] = lo_c, seg[0][1] = hi_c;
      }
      ncount[t] = 0;
      for (int sg = 0; sg < nseg; ++sg)
        for (int k = seg[sg][0] / g.bin[t]; k <= seg[sg][1] / g.bin[t]; ++k) {
          bool seen = false;
          for (int j = 0; j < ncount[t]; ++j) seen = seen || nlist[t][j] == k;
          if (!seen && ncount[t] < kOwnerReach) nlist[t][ncount[t]++] = k;
        }
    }
    const int nn = ncount[0] * ncount[1] * ncount[2];   // neighbour bins
    for (int r = 0; r < call.nrhs; ++r) {
      for (int c = lane; c < cells; c += 32) tile[c] = cmake<C>(0.0, 0.0);
      __syncwarp();
      // neighbour bins 32 at a time: lane j reads bin j's count and start at
      // once (sparse bins only), a warp scan lays their points out flat, and
      // each lane then loads one candidate point, so every round of global
      // loads is issued in parallel
      for (int j0 = 0; j0 < nn; j0 += 32) {
        const int j = j0 + lane;
        int cnt = 0, start = 0, nbc0 = 0, nbc1 = 0, nbc2 = 0;
        if (j < nn) {
          const int i2 = j % ncount[2], i1 = (j / ncount[2]) % ncount[1], i0 = j / (ncount[2] * ncount[1]);
          nbc0 = nlist[0][i0], nbc1 = nlist[1][i1], nbc2 = nlist[2][i2];
          const int gnb = it.bin_offset + (nbc0 * g.nbins[1] + nbc1) * g.nbins[2] + nbc2;
          cnt = a.pts.bin_count[gnb];
          if (cnt >= sparse_below) cnt = 0;   // dense: the tiled kernel's
          start = a.pts.bin_start[gnb];
        }
        // inclusive scan of the counts across the warp
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int base = 0; base < total; base += 32) {
          const int k = base + lane;
          // this lane's candidate: the neighbour whose range holds k
          int owner_lane = 0;
          for (int l = 0; l < 32; ++l) owner_lane += (__shfl_sync(0xffffffffu, incl, l) <= k) ? 1 : 0;
          const int ol = min(owner_lane, 31);
          const int n_start = __shfl_sync(0xffffffffu, start, ol);
          const int n_excl = __shfl_sync(0xffffffffu, incl - cnt, ol);
          const int nb[3] = {__shfl_sync(0xffffffffu, nbc0, ol), __shfl_sync(0xffffffffu, nbc1, ol),
                             __shfl_sync(0xffffffffu, nbc2, ol)};
          int rel[3] = {0, 0, 0};
          Real dl[3] = {0, 0, 0};
          C v = cmake<C>(0.0, 0.0);
          bool hit = k < total;
          if (hit) {
            const int idx = n_start + (k - n_excl);
            const uint32_t loc = a.pts.local[idx];
            for (int t = 0; t < 3; ++t) {
              // the footprint's first tap relative to R, on the image that meets R
              int q = nb[t] * g.bin[t] + unpack_local(loc, 3, t) - left - olo[t];
              if (q + W - 1 < 0) q += g.n[t];
              else if (q >= olen[t]) q -= g.n[t];
              rel[t] = q;
              hit = hit && q < olen[t] && q + W - 1 >= 0;
            }
            if (hit) {
              for (int t = 0; t < 3; ++t) dl[t] = a.pts.delta[t][idx];
              v = f_in[(int64_t)r * it.M + a.pts.perm[idx]];
            }
          }
          unsigned mask = __ballot_sync(0xffffffffu, hit);
          while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const int rz = __shfl_sync(0xffffffffu, rel[0], src);
            const int ry = __shfl_sync(0xffffffffu, rel[1], src);
            const int rx = __shfl_sync(0xffffffffu, rel[2], src);
            Real d3[3];
            for (int t = 0; t < 3; ++t) d3[t] = __shfl_sync(0xffffffffu, dl[t], src);
            C vv;
            vv.x = __shfl_sync(0xffffffffu, v.x, src);
            vv.y = __shfl_sync(0xffffffffu, v.y, src);
            for (int i = lane; i < 3 * W; i += 32) {
              const int t = i / W, tap = i - t * W;
              const Real u = (t == 0 ? d3[0] : (t == 1 ? d3[1] : d3[2])) + (Real)(it.win.m - it.win.shift) -
                             (Real)tap;
              wt[i] = window_psi<Real>(it.win, t, u);
            }
            __syncwarp();
            // in-plane slots of this lane inside R, with their weights
            int off[P];
            Real wyx[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const int yy = ry + sy[p], xx = rx + sx[p];
              const bool in = sy[p] >= 0 && yy >= 0 && yy < olen[1] && xx >= 0 && xx < olen[2];
              off[p] = in ? yy * b2 + xx : -1;
              wyx[p] = in ? wt[W + sy[p]] * wt[2 * W + sx[p]] : (Real)0;
            }
            const int z0 = max(0, -rz), z1 = min(W, olen[0] - rz);
            for (int iz = z0; iz < z1; ++iz) {
              C* plane = tile + (rz + iz) * b1 * b2;
              const Real wz = wt[iz];
#pragma unroll
              for (int p = 0; p < P; ++p) {
                if (off[p] >= 0) {
                  const Real w = wz * wyx[p];
                  C c = plane[off[p]];
                  c.x += vv.x * w;
                  c.y += vv.y * w;
                  plane[off[p]] = c;
                }
              }
            }
            __syncwarp();
          }
        }
      }
      // R into the grid, every cell once
      C* gr = grid + (int64_t)r * g.grid_cells;
      for (int row = 0; row < olen[0] * olen[1]; ++row) {
        const int zz = row / olen[1], yy = row - zz * olen[1];
        const int64_t gbase = ((int64_t)(olo[0] + zz) * g.n[1] + (olo[1] + yy)) * g.n[2] + olo[2];
        for (int xx = lane; xx < olen[2]; xx += 32) gr[gbase + xx] = tile[(zz * b1 + yy) * b2 + xx];
      }
      __syncwarp();
    }
  }
}

}  // namespace gbnfft
