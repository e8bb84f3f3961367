// 3-D spreading and interpolation with one shared tile per block.
//
// A block takes a subproblem (a run of bin-sorted points of one bin) and
// stages its points in batches of blockDim.x: thread t loads point t's
// record (value, tile offset, first plane) and evaluates its 3*W window
// weights into a shared table, so the per-point work of every warp is table
// lookups.  The wrapped grid index of every tile row and column is
// tabulated once per subproblem for the tile load / flush.
//
// spread ("plane owner"): warp w of NW (a power of two) owns the tile planes
//   z = w (mod NW), so for every point each warp updates ceil(W/NW) or
//   floor(W/NW) of the point's W planes, and no two warps ever write the
//   same cell: plain shared-memory loads and stores, no atomics, one tile
//   per block.
//   Inside a plane, lane (ix, q) = (lane % W, lane / W) takes cell ix of rows
//   q, q + Q, ... (Q = 32 / W).  After the subproblem the tile is added to
//   the grid once (vector atomics: halos of neighbouring bins overlap).
//   In FP32 with every lane busy and one right-hand side, the point loop
//   runs on 32-bit shared addresses with the next point's parameters loaded
//   ahead (spread_points_fast).
// interp: the tile arrives by cp.async copies.  In FP32 with up to 8 taps a
//   warp reads one point at a time in the spreading lane layout and reduces
//   four points at once (interp_points_fast); otherwise ("point groups") a
//   warp works on 32/W points at once, W lanes per point: lane ix of a group
//   sums column ix of its point's W x W rows with the weights held in
//   registers, then the group adds its W partial sums.
#pragma once

#include "points_tiled.cuh"

namespace gbnfft {


template <int W>
struct PlaneShape {
  static constexpr int Q = (32 / W) > 0 ? (32 / W) : 1;   // rows of a plane per pass
  static constexpr int PASSES = (W + Q - 1) / Q;           // passes over a plane
  static constexpr bool FULL = (Q * PASSES == W) && (32 % W == 0);  // every lane busy on every pass
  static constexpr int PPW = (32 / W) > 0 ? (32 / W) : 1;  // interp: points per warp
  static constexpr bool POW2 = (W & (W - 1)) == 0;
};

// Per-point record of a staged batch: the value of the first right-hand
// side, the tile offset of the point's first tap and its first-tap plane.
// One 16-byte shared load in FP32.
template <typename Real>
struct PlaneRec;
template <>
struct __align__(16) PlaneRec<float> {
  float vx, vy;
  int off, z;
};
template <>
struct __align__(8) PlaneRec<double> {
  double vx, vy;
  int off, z;
};

// Window weights of a staged point, one row of 3W per point.
//   interpolation: wz[W] | wy[W] | wx[W]
//   spreading (NW warps): wz | wy | wx, where wz is rotated when NW divides
//     W, so that warp w finds the weight of the u-th plane it owns at slot
//     u * NW + w without knowing the point's plane, and wy is permuted when
//     the lane rows cover the W rows exactly (Q * PASSES == W), so that lane
//     row q finds its PASSES weights (rows q, q + Q, ...) side by side.
template <int W, int NW>
struct SpreadRow {
  using S = PlaneShape<W>;
  static constexpr int TAPS = (W + NW - 1) / NW;
  static constexpr bool ROT = W % NW == 0;
  static constexpr bool PERM = S::Q * S::PASSES == W;
  static constexpr int WZ = 0;
  static constexpr int WY = W;
  static constexpr int WX = 2 * W;
  static constexpr int STRIDE = 3 * W;   // W is even: 8-byte aligned rows
};

// FP32 spreading with 6 taps, where 32 / W = 5 rows of W lanes fill no
// plane's 6 rows evenly (per plane a pass of 5 rows and one of 1: 56% of the
// lanes busy), and warps that divide the taps: each warp walks its planes'
// rows as one list (the flat layout), so a pass can finish one plane and
// start the next (90% busy).  Wider windows would need too many per-lane
// pass offsets in registers.
template <int W, typename Real>
__host__ __device__ constexpr bool plane_flat_ok() {
  return sizeof(Real) == 4 && W == 6;
}

// The flat layout's shape for NW warps: lane (ix, q) takes rows q, q + Q, ...
// of the warp's R rows in KP passes.  A lane with no row in pass k (q = Q, or
// past R) shadows the pass's last row, min(Q k + Q - 1, R - 1).  Staged per
// point: for each warp and lane row q, the KP products wz(plane) wy(row) of
// its passes side by side (one 16-byte load per lane per point), then wx.
template <int W, int NW>
struct FlatShape {
  static constexpr int TAPS = W / NW;
  static constexpr int Q = 32 / W;
  static constexpr int R = TAPS * W;
  static constexpr int KP = (R + Q - 1) / Q;
  static constexpr int PW = Q * KP;                 // products per warp
  static constexpr int WX = NW * PW;                // where wx starts
  // row stride: a multiple of 4 floats, and an odd number of 16-byte units,
  // so that 8 consecutive rows' 16-byte stores fall in distinct banks
  static constexpr int S4 = (WX + W + 3) / 4;
  static constexpr int STRIDE = 4 * (S4 % 2 ? S4 : S4 + 1);
  __host__ __device__ static constexpr int row(int q, int k) {
    return (q < Q && q + Q * k < R) ? q + Q * k : (Q * k + Q - 1 < R - 1 ? Q * k + Q - 1 : R - 1);
  }
};

// Weight-row stride (the flat spreading layout: FlatShape's, for 1 or 2
// warps; interpolation keeps 3W).
template <int W, typename Real>
__host__ __device__ inline int plane_wt_stride(bool spread) {
  if (spread && plane_flat_ok<W, Real>()) {
    constexpr int a = FlatShape<W, 1>::STRIDE, b = FlatShape<W, 2>::STRIDE;
    constexpr int f = a > b ? a : b;
    return f > 3 * W ? f : 3 * W;
  }
  return 3 * W;
}

// Shared layout after the tiles (bp points per batch, np right-hand sides):
//   (16-byte aligned) rec[bp] PlaneRec | wt[bp][stride] Real |
//   vt[np - 1][bp] complex (right-hand sides after the first) | jt[bp] int |
//   gz[T0] gy[T1] gx[T2] int64
template <int W, typename Real>
__host__ __device__ inline size_t plane_table_bytes(int bp, int np, int nw, const int* tile, bool spread) {
  return 16 + (size_t)bp * sizeof(PlaneRec<Real>) + (size_t)bp * plane_wt_stride<W, Real>(spread) * sizeof(Real) +
         (size_t)(np - 1) * bp * 2 * sizeof(Real) + (size_t)(bp + 1) * sizeof(int) +
         (size_t)(tile[0] + tile[1] + tile[2]) * sizeof(int64_t);
}

template <int W, typename Real>
struct PlaneSmem {
  typename Cplx<Real>::type* tile;   // [np][rows][pitch]
  PlaneRec<Real>* rec;
  Real* wt;
  typename Cplx<Real>::type* vt;
  int* jt;
  int64_t* gz;
  int64_t* gy;
  int64_t* gx;
};

template <int W, typename Real>
__device__ __forceinline__ PlaneSmem<W, Real> plane_smem(unsigned char* raw, int np_max, int tile_elems, int bp,
                                                         int nw, const GridGeom& g, bool spread) {
  using C = typename Cplx<Real>::type;
  PlaneSmem<W, Real> s;
  s.tile = reinterpret_cast<C*>(raw);
  const size_t rec_at = ((size_t)np_max * tile_elems * sizeof(C) + 15) & ~(size_t)15;
  s.rec = reinterpret_cast<PlaneRec<Real>*>(raw + rec_at);
  s.wt = reinterpret_cast<Real*>(s.rec + bp);
  s.vt = reinterpret_cast<C*>(s.wt + (size_t)bp * plane_wt_stride<W, Real>(spread));
  s.jt = reinterpret_cast<int*>(s.vt + (size_t)(np_max - 1) * bp);
  s.gz = reinterpret_cast<int64_t*>(s.jt + bp + (bp & 1));   // keep 8-byte alignment
  s.gy = s.gz + g.tile[0];
  s.gx = s.gy + g.tile[1];
  return s;
}

// Wrapped grid offsets of the tile's planes, rows and columns.
template <int W, typename Real>
__device__ __forceinline__ void plane_index_tables(const PlaneSmem<W, Real>& s, const GridGeom& g,
                                                   const int* origin) {
  for (int i = threadIdx.x; i < g.tile[0] + g.tile[1] + g.tile[2]; i += blockDim.x) {
    if (i < g.tile[0]) {
      s.gz[i] = (int64_t)wrap_mod(origin[0] + i, g.n[0]) * g.n[1] * g.n[2];
    } else if (i < g.tile[0] + g.tile[1]) {
      const int y = i - g.tile[0];
      s.gy[y] = (int64_t)wrap_mod(origin[1] + y, g.n[1]) * g.n[2];
    } else {
      const int x = i - g.tile[0] - g.tile[1];
      s.gx[x] = wrap_mod(origin[2] + x, g.n[2]);
    }
  }
}

// The tile rows a warp takes, e = first, first + step, ... over np tiles of
// T0 x T1 rows: tile r, plane z and row y advanced by additions (no
// divisions per row).
struct TileRowWalk {
  int r, z, y;
  __device__ __forceinline__ TileRowWalk(int first, int T0, int T1) : r(0), z(0), y(first) { norm(T0, T1); }
  __device__ __forceinline__ void norm(int T0, int T1) {
    while (y >= T1) {
      y -= T1;
      if (++z == T0) {
        z = 0;
        ++r;
      }
    }
  }
  __device__ __forceinline__ void next(int step, int T0, int T1) {
    y += step;
    norm(T0, T1);
  }
};

// Stage a batch: thread t handles point first + t.  NW > 0: the spreading
// layout for NW warps (values of every right-hand side of the pass);
// NW == 0: the interpolation layout (no values, the point's index instead);
// NW < 0: the interpolation layout with wy permuted as for spreading.
template <int W, int NW, typename Real>
__device__ __forceinline__ void plane_stage_batch(const PointKernelArgs<Real>& a, const PlaneSmem<W, Real>& s,
                                                  const WindowDev& win, const typename Cplx<Real>::type* f_in,
                                                  int64_t M, int first, int nb, int r0, int np, int bp, int T1,
                                                  int pitch, int stride) {
  using S = PlaneShape<W>;
  const int t = threadIdx.x;
  if (t >= nb) return;
  const int idx = first + t;
  const int j = a.pts.perm[idx];
  const uint32_t loc = a.pts.local[idx];
  const int l0 = unpack_local(loc, 3, 0), l1 = unpack_local(loc, 3, 1), l2 = unpack_local(loc, 3, 2);
  PlaneRec<Real> rec;
  rec.off = (l0 * T1 + l1) * pitch + l2;
  rec.z = l0;
  rec.vx = 0;
  rec.vy = 0;
  Real* w = s.wt + (size_t)t * stride;
  Real base[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) base[d] = a.pts.delta[d][idx] + (Real)(win.m - win.shift);
  if (NW == 0) {
    s.jt[t] = j;
    if constexpr (sizeof(Real) == 4 && W % 2 == 0) {
      // 8-byte stores (row stride 3W even, table 16-byte aligned)
      float2* w2 = reinterpret_cast<float2*>(w);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int i = 0; i < W; i += 2)
          w2[(d * W + i) / 2] = make_float2(window_psi<float>(win, d, base[d] - (float)i),
                                            window_psi<float>(win, d, base[d] - (float)(i + 1)));
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int i = 0; i < W; ++i) w[d * W + i] = window_psi<Real>(win, d, base[d] - (Real)i);
    }
  } else {
    using R = SpreadRow<W, (NW > 0 ? NW : 1)>;
    constexpr int NWs = NW > 0 ? NW : 1;
#pragma unroll
    for (int u = 0; u < R::TAPS; ++u)
#pragma unroll
      for (int ww = 0; ww < NWs; ++ww) {
        const int slot = u * NWs + ww;
        const int i = R::ROT ? ((ww - l0) & (NWs - 1)) + u * NWs : slot;
        if (slot < W) w[R::WZ + slot] = window_psi<Real>(win, 0, base[0] - (Real)i);
      }
#pragma unroll
    for (int q = 0; q < S::Q; ++q)
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) {
        const int slot = R::PERM ? q * S::PASSES + k : k * S::Q + q;
        const int i = k * S::Q + q;
        if (i < W) w[R::WY + slot] = window_psi<Real>(win, 1, base[1] - (Real)i);
      }
#pragma unroll
    for (int i = 0; i < W; ++i) w[R::WX + i] = window_psi<Real>(win, 2, base[2] - (Real)i);
    if (NW < 0) {
      s.jt[t] = j;
    } else {
      if (np > 0) {
        const auto v0 = f_in[(int64_t)r0 * M + j];
        rec.vx = v0.x;
        rec.vy = v0.y;
      }
      for (int r = 1; r < np; ++r) s.vt[(r - 1) * bp + t] = f_in[(int64_t)(r0 + r) * M + j];
    }
  }
  s.rec[t] = rec;
}

// PASSES consecutive weights of a spreading row (8-byte aligned pairs).
template <int N, typename Real>
__device__ __forceinline__ void load_row(const Real* p, Real* out) {
  if (sizeof(Real) == 4 && N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 2) {
      const float2 v = *reinterpret_cast<const float2*>(p + k);
      out[k] = v.x;
      out[k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = p[k];
  }
}

// 32-bit shared-memory accesses (the spreading loop's addresses are byte
// offsets in the block's shared window).
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f1(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
// One grid cell copied from global to shared memory without passing through
// registers (8 bytes in FP32, 16 in FP64); completed by cp_async_wait_all.
__device__ __forceinline__ void cp_async_cell(uint32_t dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_cell(uint32_t dst, const double2* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int lds_i1(uint32_t a) {
  int v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_f2(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

// The weights a spreading lane needs for one point: those of the planes its
// warp owns (u-th: tap (warp - z) mod NW + u NW), of its rows (q + k Q) and
// of its column ix.  Zero where a tap is past the window.
template <int W, int NW, typename Real>
__device__ __forceinline__ void spread_point_weights(const Real* w, int z, int warp, int q, int ix, bool active,
                                                     Real* wz, Real* wy, Real& wx) {
  using S = PlaneShape<W>;
  using R = SpreadRow<W, NW>;
  const int i0 = (warp - z) & (NW - 1);
#pragma unroll
  for (int u = 0; u < R::TAPS; ++u) {
    if (R::ROT) {
      wz[u] = w[R::WZ + u * NW + warp];
    } else {
      const int i = i0 + u * NW;
      wz[u] = i < W ? w[R::WZ + i] : (Real)0;
    }
  }
  if (R::PERM) {
    if (active) {
      load_row<S::PASSES>(w + R::WY + q * S::PASSES, wy);
    } else {
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) wy[k] = 0;
    }
  } else {
#pragma unroll
    for (int k = 0; k < S::PASSES; ++k) {
      const int i = k * S::Q + q;
      wy[k] = (active && i < W) ? w[R::WY + i] : (Real)0;
    }
  }
  wx = w[R::WX + ix];
}

// The plane-owner loop over a staged batch for one right-hand side in FP32
// (see k_spread_planes): each point's record and weights are loaded one
// point ahead; the warp adds the point into the cells of its planes.
template <int W, int NW, typename Real>
__device__ __forceinline__ void spread_points_fast(const PlaneSmem<W, Real>& s, int nb, int warp, int lane_off,
                                                   int q, int ix, int pstride, int qstride) {
  using S = PlaneShape<W>;
  using R = SpreadRow<W, NW>;
  constexpr uint32_t ROW = 4u * R::STRIDE;   // bytes per weight row
  const uint32_t tile_a = (uint32_t)__cvta_generic_to_shared(s.tile) + 8u * (uint32_t)lane_off;
  const uint32_t rec_a = (uint32_t)__cvta_generic_to_shared(s.rec);
  const uint32_t wt_a = (uint32_t)__cvta_generic_to_shared(s.wt);
  const uint32_t wz_a = wt_a + 4u * (uint32_t)(R::WZ + warp);
  const uint32_t wy_a = wt_a + 4u * (uint32_t)(R::WY + q * S::PASSES);
  const uint32_t wx_a = wt_a + 4u * (uint32_t)(R::WX + ix);
  const uint32_t pb = 8u * (uint32_t)pstride;
  uint32_t qoff[S::PASSES], uoff[R::TAPS];
#pragma unroll
  for (int k = 0; k < S::PASSES; ++k) qoff[k] = 8u * (uint32_t)(k * qstride);
#pragma unroll
  for (int u = 0; u < R::TAPS; ++u) uoff[u] = (uint32_t)(u * NW) * pb;
  float4 nrec = lds_f4(rec_a);
  float nwz[R::TAPS], nwy[S::PASSES], nwx;
#pragma unroll
  for (int u = 0; u < R::TAPS; ++u) nwz[u] = lds_f1(wz_a + 4u * (uint32_t)(u * NW));
#pragma unroll
  for (int k = 0; k < S::PASSES; k += 2) {
    const float2 t = lds_f2(wy_a + 4u * k);
    nwy[k] = t.x;
    nwy[k + 1] = t.y;
  }
  nwx = lds_f1(wx_a);
#pragma unroll 2
  for (int pp = 0; pp < nb; ++pp) {
    const float4 rc = nrec;
    float wz[R::TAPS], wy[S::PASSES];
    const float wx = nwx;
#pragma unroll
    for (int u = 0; u < R::TAPS; ++u) wz[u] = nwz[u];
#pragma unroll
    for (int k = 0; k < S::PASSES; ++k) wy[k] = nwy[k];
    const uint32_t pn = (uint32_t)min(pp + 1, nb - 1);
    nrec = lds_f4(rec_a + 16u * pn);
#pragma unroll
    for (int u = 0; u < R::TAPS; ++u) nwz[u] = lds_f1(wz_a + ROW * pn + 4u * (uint32_t)(u * NW));
#pragma unroll
    for (int k = 0; k < S::PASSES; k += 2) {
      const float2 t = lds_f2(wy_a + ROW * pn + 4u * k);
      nwy[k] = t.x;
      nwy[k + 1] = t.y;
    }
    nwx = lds_f1(wx_a + ROW * pn);
    const int i0 = (warp - __float_as_int(rc.w)) & (NW - 1);   // first tap whose plane this warp owns
    const uint32_t a0 = tile_a + 8u * (uint32_t)__float_as_int(rc.z) + (uint32_t)i0 * pb;
#pragma unroll
    for (int u = 0; u < R::TAPS; ++u) {
      const float wzx = wz[u] * wx;
      const float2 v = cscale(make_float2(rc.x, rc.y), wzx);
      const uint32_t au = a0 + uoff[u];
      float2 c[S::PASSES];
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) c[k] = lds_f2(au + qoff[k]);
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) {
        c[k] = cmad(v, wy[k], c[k]);
        sts_f2(au + qoff[k], c[k]);
      }
    }
    __syncwarp();
  }
}

// Stage a batch in the flat layout (FP32, one right-hand side): thread t
// handles point first + t; its row holds FlatShape's products, then wx.
template <int W, int NW>
__device__ __forceinline__ void plane_stage_flat(const PointKernelArgs<float>& a, const PlaneSmem<W, float>& s,
                                                 const WindowDev& win, const float2* f_in, int64_t M, int first,
                                                 int nb, int r0, int T1, int pitch, int stride) {
  static_assert(NW <= 2, "the flat record holds one tile offset per warp");
  static_assert(FlatShape<W, NW>::KP % 4 == 0, "a lane's products are whole 16-byte units");
  const int t = threadIdx.x;
  if (t >= nb) return;
  const int idx = first + t;
  const int j = a.pts.perm[idx];
  const uint32_t loc = a.pts.local[idx];
  const int l0 = unpack_local(loc, 3, 0), l1 = unpack_local(loc, 3, 1), l2 = unpack_local(loc, 3, 2);
  // the record's two offsets: the tile cell of the first plane warp 0 and
  // warp 1 own (tap (w - l0) mod NW)
  PlaneRec<float> rec;
  const int off = (l0 * T1 + l1) * pitch + l2;
  rec.off = off + ((0 - l0) & (NW - 1)) * T1 * pitch;
  rec.z = off + ((1 - l0) & (NW - 1)) * T1 * pitch;
  const float2 v0 = f_in[(int64_t)r0 * M + j];
  rec.vx = v0.x;
  rec.vy = v0.y;
  float base[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) base[d] = a.pts.delta[d][idx] + (float)(win.m - win.shift);
  float wz[W], wy[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    wz[i] = window_psi<float>(win, 0, base[0] - (float)i);
    wy[i] = window_psi<float>(win, 1, base[1] - (float)i);
  }
  // products first (16-byte stores: the row stride is an odd number of
  // 16-byte units and the table 16-byte aligned), then wx
  using F = FlatShape<W, NW>;
  float* w = s.wt + (size_t)t * stride;
#pragma unroll
  for (int ww = 0; ww < NW; ++ww) {
    const int i0 = (ww - l0) & (NW - 1);
#pragma unroll
    for (int q = 0; q < F::Q; ++q) {
      float pk[F::KP];
#pragma unroll
      for (int k = 0; k < F::KP; ++k) {
        const int r = F::row(q, k), u = r / W, y = r % W;
        // wz[i0 + u NW] by selects (a runtime index would put wz in local memory)
        float z = wz[u * NW];
#pragma unroll
        for (int c = 1; c < NW; ++c)
          if (i0 == c) z = wz[c + u * NW];
        pk[k] = z * wy[y];
      }
#pragma unroll
      for (int k = 0; k < F::KP; k += 4)
        *reinterpret_cast<float4*>(w + ww * F::PW + q * F::KP + k) = make_float4(pk[k], pk[k + 1], pk[k + 2], pk[k + 3]);
    }
  }
#pragma unroll
  for (int i = 0; i < W; i += 2)
    *reinterpret_cast<float2*>(w + F::WX + i) = make_float2(window_psi<float>(win, 2, base[2] - (float)i),
                                                            window_psi<float>(win, 2, base[2] - (float)(i + 1)));
  s.rec[t] = rec;
}

// The plane-owner loop over a batch staged in the flat layout: lane (ix, q)
// takes the rows q, q + Q, ... (Q = 32 / W) of the warp's W / NW planes
// walked as one list of rows, column ix.
template <int W, int NW>
__device__ __forceinline__ void spread_points_flat(const PlaneSmem<W, float>& s, int nb, int warp, int lane,
                                                   int pitch, int pstride, int stride) {
  using F = FlatShape<W, NW>;
  constexpr int Q = F::Q, KP = F::KP;
  const int ix = lane % W, q = lane / W;
  const uint32_t tile_a = (uint32_t)__cvta_generic_to_shared(s.tile);
  const uint32_t rec_a = (uint32_t)__cvta_generic_to_shared(s.rec);
  const uint32_t wt_a = (uint32_t)__cvta_generic_to_shared(s.wt);
  const uint32_t rowb = 4u * (uint32_t)stride;
  // Every lane loads and stores unconditionally: one with no row in pass k
  // shadows the pass's last row (FlatShape::row), which a lane of the same
  // pass updates, so it loads the same cell and weights and stores the same
  // value.  The last row's lanes sit in the upper half of the warp with the
  // idle ones, so a pass touches no more distinct addresses per half warp
  // than the rows themselves.
  uint32_t coff[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int r = F::row(q, k);
    const int u = r / W, y = r % W;
    coff[k] = 8u * (uint32_t)(u * NW * pstride + y * pitch + ix);
  }
  // this lane's KP products (lanes q = Q read row q = Q - 1's, whose shadow
  // rows are theirs) and its column weight
  const uint32_t poff = 4u * (uint32_t)(warp * F::PW + (q < Q ? q : Q - 1) * KP);
  const uint32_t wx_off = 4u * (uint32_t)(F::WX + ix);
  // the next point's record, column weight and products are loaded one point
  // ahead; a point's cells are all loaded before any is written back (the
  // passes touch distinct cells)
  float4 nrc = lds_f4(rec_a);
  float nwx = lds_f1(wt_a + wx_off);
  float npw[KP];
#pragma unroll
  for (int k = 0; k < KP; k += 4) {
    const float4 t4 = lds_f4(wt_a + poff + 4u * k);
    npw[k] = t4.x;
    npw[k + 1] = t4.y;
    npw[k + 2] = t4.z;
    npw[k + 3] = t4.w;
  }
#pragma unroll 2
  for (int pp = 0; pp < nb; ++pp) {
    const float4 rc = nrc;
    const float wx = nwx;
    float pw[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) pw[k] = npw[k];
    {
      const uint32_t pn = (uint32_t)min(pp + 1, nb - 1);
      const uint32_t row = wt_a + rowb * pn;
      nrc = lds_f4(rec_a + 16u * pn);
      nwx = lds_f1(row + wx_off);
#pragma unroll
      for (int k = 0; k < KP; k += 4) {
        const float4 t4 = lds_f4(row + poff + 4u * k);
        npw[k] = t4.x;
        npw[k + 1] = t4.y;
        npw[k + 2] = t4.z;
        npw[k + 3] = t4.w;
      }
    }
    const float2 v = cscale(make_float2(rc.x, rc.y), wx);
    const uint32_t base = tile_a + 8u * (uint32_t)(warp == 0 ? __float_as_int(rc.z) : __float_as_int(rc.w));
    float2 c[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) c[k] = lds_f2(base + coff[k]);
#pragma unroll
    for (int k = 0; k < KP; ++k) sts_f2(base + coff[k], cmad(v, pw[k], c[k]));
    __syncwarp();
  }
}

template <int W, int NW, typename Real>
__global__ void __launch_bounds__(32 * NW) k_spread_planes(PointKernelArgs<Real> a, WppLayout lay) {
  using C = typename Cplx<Real>::type;
  using S = PlaneShape<W>;
  static_assert((NW & (NW - 1)) == 0 && NW <= 8, "warps per block must be a power of two, at most 8");
  using R = SpreadRow<W, NW>;                // R::TAPS: at most this many planes of a point per warp
  constexpr bool EVEN = W % NW == 0;        // every warp takes exactly R::TAPS planes
  // FP32, every lane busy on every pass, rotated and permuted weight rows:
  // the single-right-hand-side loop runs on 32-bit shared addresses
  constexpr bool FAST = sizeof(Real) == 4 && EVEN && S::FULL && R::ROT && R::PERM && S::PASSES % 2 == 0;
  // FP32, warps dividing the taps, rows that do not fill a warp: the flat layout
  constexpr bool FLAT = EVEN && plane_flat_ok<W, Real>();
  constexpr int BP = 32 * NW;    // points per batch
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int np_max = a.rhs_per_pass;
  const int pitch = lay.pitch;
  const int tile_elems = lay.warp_cells;
  const int ix = lane % W, q = lane / W;
  const bool active = S::FULL || q < S::Q;
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem sub = a.pts.subs[sp];
    if (!sub_selected(a, sub)) continue;   // block-uniform
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    const C* f_in = static_cast<const C*>(call.in);
    C* grid = static_cast<C*>(it.grid);
    const int T1 = g.tile[1], T2 = g.tile[2];
    const PlaneSmem<W, Real> s = plane_smem<W, Real>(smem_raw, np_max, tile_elems, BP, NW, g, true);
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(sub.bin, g, bc);
    for (int t = 0; t < 3; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    plane_index_tables<W, Real>(s, g, origin);
    const int lane_off = ix + q * pitch;   // this lane's first cell in a plane of the footprint
    const int pstride = T1 * pitch;        // tile plane
    const int qstride = S::Q * pitch;      // rows between a lane's passes
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      for (int e = threadIdx.x; e < np * tile_elems; e += BP) s.tile[e] = cmake<C>(0.0, 0.0);
      for (int pb = 0; pb < sub.count; pb += BP) {
        const int nb = min(BP, sub.count - pb);
        __syncthreads();   // tile zeroed / previous batch no longer read
        if constexpr (FLAT) {
          if (np == 1) {
            const int fstride = plane_wt_stride<W, Real>(true);
            plane_stage_flat<W, NW>(a, s, it.win, f_in, it.M, sub.start + pb, nb, r0, T1, pitch, fstride);
            __syncthreads();
            spread_points_flat<W, NW>(s, nb, warp, lane, pitch, pstride, fstride);
            continue;
          }
        }
        plane_stage_batch<W, NW, Real>(a, s, it.win, f_in, it.M, sub.start + pb, nb, r0, np, BP, T1, pitch,
                                       R::STRIDE);
        __syncthreads();
        if constexpr (FAST) {
          if (np == 1) {
            spread_points_fast<W, NW>(s, nb, warp, lane_off, q, ix, pstride, qstride);
            continue;
          }
        }
        // a point's parameters, loaded one point ahead (the tables are
        // read-only here): the record, the weights of this warp's planes,
        // of this lane's rows and of its column
        PlaneRec<Real> nrec = s.rec[0];
        Real nwz[R::TAPS], nwy[S::PASSES], nwx;
        spread_point_weights<W, NW, Real>(s.wt, nrec.z, warp, q, ix, active, nwz, nwy, nwx);
#pragma unroll 2
        for (int pp = 0; pp < nb; ++pp) {
          const PlaneRec<Real> rec = nrec;
          Real wz[R::TAPS], wy[S::PASSES];
          const Real wx = nwx;
#pragma unroll
          for (int u = 0; u < R::TAPS; ++u) wz[u] = nwz[u];
#pragma unroll
          for (int k = 0; k < S::PASSES; ++k) wy[k] = nwy[k];
          {
            const int pn = min(pp + 1, nb - 1);
            nrec = s.rec[pn];
            spread_point_weights<W, NW, Real>(s.wt + pn * R::STRIDE, nrec.z, warp, q, ix, active, nwz, nwy, nwx);
          }
          const int i0 = (warp - rec.z) & (NW - 1);   // first tap whose plane this warp owns
          const int cell0 = rec.off + lane_off + i0 * pstride;
          for (int r = 0; r < np; ++r) {
            Real vx = rec.vx, vy = rec.vy;
            if (r > 0) {
              const C v = s.vt[(r - 1) * BP + pp];
              vx = v.x;
              vy = v.y;
            }
            C* tr = s.tile + r * tile_elems + cell0;
#pragma unroll
            for (int u = 0; u < R::TAPS; ++u) {
              if (!EVEN && i0 + u * NW >= W) break;
              C v;
              v.x = vx;
              v.y = vy;
              v = cscale(v, wz[u] * wx);
              C* plane = tr + u * NW * pstride;
              C cell[S::PASSES];
#pragma unroll
              for (int k = 0; k < S::PASSES; ++k)
                if (active && k * S::Q + q < W) cell[k] = plane[k * qstride];
#pragma unroll
              for (int k = 0; k < S::PASSES; ++k) {
                if (active && k * S::Q + q < W) {
                  cell[k] = cmad(v, wy[k], cell[k]);
                  plane[k * qstride] = cell[k];
                }
              }
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // flush the tile into the grid once: a warp per row, lanes along the row
      for (TileRowWalk w(warp, g.tile[0], T1); w.r < np; w.next(NW, g.tile[0], T1)) {
        const int r = w.r, z = w.z, y = w.y;
        const int row = z * T1 + y;
        const int64_t gb = (int64_t)(r0 + r) * g.grid_cells + s.gz[z] + s.gy[y];
        const C* src = s.tile + r * tile_elems + row * pitch;
        for (int x = lane; x < T2; x += 32) {
          const C c = src[x];
          if (c.x != (Real)0 || c.y != (Real)0) grid_add(grid + gb + s.gx[x], c);
        }
      }
      __syncthreads();
    }
  }
}

// The 4 points' 8 real values of a warp pass (v[2g], v[2g + 1]: this lane's
// share of point p0 + g), reduced over the warp at once by a transposed
// butterfly (10 shuffles): after the exchanges over lane bits 4, 3 and 2 each
// lane keeps one value, and bits 1 and 0 finish its sum; lane 8g then
// writes point p0 + g to its place in the caller's order.
__device__ __forceinline__ void butterfly4_store(const float* v, int lane, int p0, int nb, uint32_t jt_a,
                                                 float2* out) {
  const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
  float a4[4], a2[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = b4 ? v[j] : v[4 + j];
    const float keep = b4 ? v[4 + j] : v[j];
    a4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = b3 ? a4[j] : a4[2 + j];
    const float keep = b3 ? a4[2 + j] : a4[j];
    a2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float a1;
  {
    const float send = b2 ? a2[0] : a2[1];
    const float keep = b2 ? a2[1] : a2[0];
    a1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
  a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  // lane l now holds value l >> 2: point l >> 3, real part when bit 2 is 0
  const float im = __shfl_down_sync(0xffffffffu, a1, 4);
  const int g = lane >> 3;
  if ((lane & 7) == 0 && p0 + g < nb) {
    const int j = lds_i1(jt_a + 4u * (uint32_t)(p0 + g));
    out[j] = make_float2(a1, im);
  }
}

// Interpolation of a staged batch for one right-hand side in FP32.  A warp
// takes 4 points at a time, one after another: lane (ix, q) reads cell ix
// of rows q, q + Q, ... of every plane of the point's footprint, with the
// spreading layout's conflict-free rows, and sums them with the plane and
// row weights; times the column weight, that is the lane's share of the
// point's value.  A transposed butterfly then reduces the 4 points' 8 real
// values over the warp at once (10 shuffles): after the exchanges over
// lane bits 4, 3 and 2 each lane keeps one value, and bits 1 and 0 finish
// its sum.
template <int W, typename Real>
__device__ __forceinline__ void interp_points_fast(const PlaneSmem<W, Real>& s, int nb, int warp, int nw, int lane,
                                                   int pitch, int pstride, typename Cplx<Real>::type* out) {
  using S = PlaneShape<W>;
  constexpr int PG = 4;                      // points per warp pass
  constexpr uint32_t ROW = 4u * 3 * W;       // bytes per weight row (16-byte multiple)
  const int ix = lane % W, q = lane / W;
  const uint32_t tile_a = (uint32_t)__cvta_generic_to_shared(s.tile) + 8u * (uint32_t)(ix + q * pitch);
  const uint32_t off_a = (uint32_t)__cvta_generic_to_shared(s.rec) + 8u;   // PlaneRec<float>::off
  const uint32_t jt_a = (uint32_t)__cvta_generic_to_shared(s.jt);
  const uint32_t wz_a = (uint32_t)__cvta_generic_to_shared(s.wt);
  const uint32_t wy_a = wz_a + 4u * (uint32_t)(W + q * S::PASSES);
  const uint32_t wx_a = wz_a + 4u * (uint32_t)(2 * W + ix);
  const uint32_t pb = 8u * (uint32_t)pstride;
  uint32_t qoff[S::PASSES];
#pragma unroll
  for (int k = 0; k < S::PASSES; ++k) qoff[k] = 8u * (uint32_t)(k * S::Q * pitch);
  for (int p0 = warp * PG; p0 < nb; p0 += nw * PG) {
    float v[2 * PG];
#pragma unroll
    for (int g = 0; g < PG; ++g) {
      const uint32_t pp = (uint32_t)min(p0 + g, nb - 1);   // past the batch: recomputed, not written
      const int off = lds_i1(off_a + 16u * pp);
      float wz[W], wy[S::PASSES];
#pragma unroll
      for (int i = 0; i < W; i += 4) {
        const float4 t = lds_f4(wz_a + ROW * pp + 4u * i);
        wz[i] = t.x;
        wz[i + 1] = t.y;
        wz[i + 2] = t.z;
        wz[i + 3] = t.w;
      }
#pragma unroll
      for (int k = 0; k < S::PASSES; k += 2) {
        const float2 t = lds_f2(wy_a + ROW * pp + 4u * k);
        wy[k] = t.x;
        wy[k + 1] = t.y;
      }
      const float wx = lds_f1(wx_a + ROW * pp);
      float2 u[S::PASSES];
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) u[k] = make_float2(0.0f, 0.0f);
      uint32_t ad = tile_a + 8u * (uint32_t)off;
#pragma unroll
      for (int iz = 0; iz < W; ++iz) {
#pragma unroll
        for (int k = 0; k < S::PASSES; ++k) u[k] = cmad(lds_f2(ad + qoff[k]), wz[iz], u[k]);
        ad += pb;
      }
      float2 sum = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < S::PASSES; ++k) sum = cmad(u[k], wy[k], sum);
      const float2 sw = cscale(sum, wx);
      v[2 * g] = sw.x;
      v[2 * g + 1] = sw.y;
    }
    butterfly4_store(v, lane, p0, nb, jt_a, out);
  }
}

// FP32 narrow windows: three blocks of 256 threads per SM (at most 85 registers)
template <int W, typename Real>
__global__ void __launch_bounds__(256, (W <= 8 && sizeof(Real) == 4) ? 3 : 1) k_interp_groups(PointKernelArgs<Real> a, WppLayout lay) {
  using C = typename Cplx<Real>::type;
  using S = PlaneShape<W>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = lay.warps;
  const int bp = blockDim.x;
  const int np_max = a.rhs_per_pass;
  const int pitch = lay.pitch;
  const int tile_elems = lay.warp_cells;
  const int grp = lane / W, ix = lane % W;
  const bool active = grp < S::PPW;
  // FP32 with every lane busy (8 taps or fewer: the registers of wider
  // windows would halve the resident blocks): one point at a time per warp
  // in the spreading lane layout (conflict-free rows at the chosen pitch)
  constexpr bool FAST = sizeof(Real) == 4 && S::FULL && S::PASSES % 2 == 0 && W <= 8;
  int lo, hi;
  launch_subs(a, lo, hi);
  for (int sp = lo + blockIdx.x; sp < hi; sp += gridDim.x) {
    const SubProblem sub = a.pts.subs[sp];
    if (!sub_selected(a, sub)) continue;   // block-uniform
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    C* f_out = static_cast<C*>(call.out);
    const C* grid_in = static_cast<const C*>(it.grid);
    const int T1 = g.tile[1], T2 = g.tile[2];
    const int plane_stride = T1 * pitch;
    const PlaneSmem<W, Real> s = plane_smem<W, Real>(smem_raw, np_max, tile_elems, bp, nw, g, false);
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(sub.bin, g, bc);
    for (int t = 0; t < 3; ++t) origin[t] = bc[t] * g.bin[t] - it.win.m + it.win.shift;
    __syncthreads();   // the previous subproblem's readers are done
    plane_index_tables<W, Real>(s, g, origin);
    for (int r0 = 0; r0 < call.nrhs; r0 += a.rhs_per_pass) {
      const int np = min(a.rhs_per_pass, call.nrhs - r0);
      __syncthreads();
      // load the tile with asynchronous global-to-shared copies: a warp per
      // row, lanes along it; every copy of the tile is in flight before the
      // block waits for them
      for (TileRowWalk w(warp, g.tile[0], T1); w.r < np; w.next(nw, g.tile[0], T1)) {
        const int r = w.r, z = w.z, y = w.y;
        const int row = z * T1 + y;
        const C* src = grid_in + (int64_t)(r0 + r) * g.grid_cells + s.gz[z] + s.gy[y];
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s.tile + r * tile_elems + row * pitch);
        for (int x = lane; x < T2; x += 32) cp_async_cell(dst + (uint32_t)(x * sizeof(C)), src + s.gx[x]);
      }
      cp_async_wait_all();
      for (int pb = 0; pb < sub.count; pb += bp) {
        const int nb = min(bp, sub.count - pb);
        __syncthreads();
        if constexpr (FAST) {
          if (np == 1) {
            plane_stage_batch<W, -1, Real>(a, s, it.win, nullptr, it.M, sub.start + pb, nb, r0, 0, bp, T1,
                                           pitch, 3 * W);
            __syncthreads();
            interp_points_fast<W, Real>(s, nb, warp, nw, lane, pitch, plane_stride,
                                        f_out + (int64_t)r0 * it.M);
            continue;
          }
        }
        plane_stage_batch<W, 0, Real>(a, s, it.win, nullptr, it.M, sub.start + pb, nb, r0, 0, bp, T1, pitch, 3 * W);
        __syncthreads();
        for (int p0 = warp * S::PPW; p0 < nb; p0 += nw * S::PPW) {
          const int pp = p0 + grp;
          const bool mine = active && pp < nb;
          Real wz[W], wy[W];
          Real wx = 0;
          int base = 0;
          if (mine) {
            const Real* w = s.wt + pp * (3 * W);
#pragma unroll
            for (int i = 0; i < W; ++i) {
              wz[i] = w[i];
              wy[i] = w[W + i];
            }
            wx = w[2 * W + ix];
            base = s.rec[pp].off + ix;
          }
          for (int r = 0; r < np; ++r) {
            Real ar = 0, ai = 0;
            if (mine) {
              const C* tr = s.tile + r * tile_elems + base;
              C acc = cmake<C>(0.0, 0.0);
#pragma unroll
              for (int iz = 0; iz < W; ++iz) {
                C p = cmake<C>(0.0, 0.0);
                const C* pl = tr + iz * plane_stride;
#pragma unroll
                for (int iy = 0; iy < W; ++iy) p = cmad(pl[iy * pitch], wy[iy], p);
                acc = cmad(p, wz[iz], acc);
              }
              acc = cscale(acc, wx);
              ar = acc.x;
              ai = acc.y;
            }
            if (S::POW2) {
#pragma unroll
              for (int o = W / 2; o > 0; o >>= 1) {
                ar += __shfl_xor_sync(0xffffffffu, ar, o);
                ai += __shfl_xor_sync(0xffffffffu, ai, o);
              }
            } else {
              // segmented sum over the group's W lanes: after the step of
              // offset o lane ix holds the sum of lanes ix .. min(ix + 2o, W) - 1
              // of its group, so lane ix = 0 ends with the whole group's
#pragma unroll
              for (int o = 1; o < W; o <<= 1) {
                const Real tr = __shfl_down_sync(0xffffffffu, ar, o);
                const Real ti = __shfl_down_sync(0xffffffffu, ai, o);
                if (ix + o < W) {
                  ar += tr;
                  ai += ti;
                }
              }
            }
            if (mine && ix == 0) f_out[(int64_t)(r0 + r) * it.M + s.jt[pp]] = cmake<C>(ar, ai);
          }
        }
      }
    }
  }
}

// (taps, warps) pairs instantiated for spreading: up to 16 taps the warps
// divide the taps; wider windows take 2, 4 or 8 warps (one block per SM);
// in FP64 only 18 and 20 taps (wider tiles do not fit shared memory).
#define GBNFFT_PLANE_SPREAD_CASES_NARROW(X, R)                                                             \
  X(2, 1, R) X(2, 2, R) X(4, 1, R) X(4, 2, R) X(4, 4, R) X(6, 1, R) X(6, 2, R) X(8, 1, R) X(8, 2, R)      \
      X(8, 4, R) X(8, 8, R) X(10, 1, R) X(10, 2, R) X(12, 1, R) X(12, 2, R) X(12, 4, R) X(14, 1, R)       \
          X(14, 2, R) X(16, 1, R) X(16, 2, R) X(16, 4, R) X(16, 8, R)
#define GBNFFT_PLANE_TAPS_NARROW(X, R) X(2, R) X(4, R) X(6, R) X(8, R) X(10, R) X(12, R) X(14, R) X(16, R)
// narrow windows with more warps than divide the taps (more warps per SM)
#define GBNFFT_PLANE_SPREAD_CASES_UNEVEN(X, R) \
  X(6, 4, R) X(10, 4, R) X(10, 8, R) X(12, 8, R) X(14, 4, R) X(14, 8, R)
// wide windows, split over translation units to keep each compile short
#define GBNFFT_PLANE_SPREAD_CASES_W18_22(X, R) \
  X(18, 2, R) X(18, 4, R) X(18, 8, R) X(20, 2, R) X(20, 4, R) X(20, 8, R) X(22, 2, R) X(22, 4, R)
#define GBNFFT_PLANE_TAPS_W18_22(X, R) X(18, R) X(20, R) X(22, R)
#define GBNFFT_PLANE_SPREAD_CASES_W24_26(X, R) X(24, 2, R) X(24, 4, R) X(26, 2, R) X(26, 4, R)
#define GBNFFT_PLANE_TAPS_W24_26(X, R) X(24, R) X(26, R)
#define GBNFFT_PLANE_SPREAD_CASES_W18_20(X, R) X(18, 2, R) X(18, 4, R) X(20, 2, R) X(20, 4, R)
#define GBNFFT_PLANE_TAPS_W18_20(X, R) X(18, R) X(20, R)

}  // namespace gbnfft
