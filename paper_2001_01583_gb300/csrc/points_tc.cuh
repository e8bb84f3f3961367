// 3-D spreading on the tensor cores (tcgen05), one tile per block.
//
// The spreading step of Section 2 (Fig. 1, Algorithm 2) adds, for every
// point j of a bin, f_j wz_j(z) wy_j(y) wx_j(x) into the bin's tile of
// T0 x T1 x T2 cells.  Taking the tile's (z, y) rows as the M dimension
// (T0 T1 <= 128) and its x columns, real and imaginary part side by side, as
// the N dimension (2 T2, rounded up to a multiple of 16), a chunk of K points
// adds the product of two dense matrices:
//   D[(z,y), (x,c)] += sum_k A[(z,y), k] B[k, (x,c)],
//   A[(z,y), k] = wz_k(z - z0_k) wy_k(y - y0_k),  B[k, (x,c)] = (f_k)_c wx_k(x - x0_k),
// both zero outside the point's W x W x W footprint (z0, y0, x0: its first
// tap in tile coordinates).  D is the tile itself; it stays in tensor memory
// (TMEM) for the whole subproblem and is added to the grid once, like the
// shared tile of the plane kernels (halos of neighbouring bins overlap).
//
// FP32 accuracy from TF32 products: each operand is split as v = hi + lo with
// hi = tf32(v) and lo = tf32(v - hi) (round to nearest), and the MMAs add
// hi*hi + hi*lo + lo*hi.  The split represents v to 2^-24 relative and the
// dropped lo*lo term is below 2^-24 of the product, so a product carries
// about three FP32 roundings, as the plane kernels' weight products do.  The
// MMAs' own FP32 accumulation does not round to nearest: its error grows
// with the number of MMAs adding into a value (measured: 2e-5 of the rms
// for dense clusters, against 2e-6 for the plane kernels).  So each pair of
// chunks accumulates in a fresh TMEM partial (two, alternating) and the
// block adds the completed partial into a third TMEM region, the tile, with
// ordinary FP32 adds (round to nearest): the MMA accumulation error is that
// of 24 MMAs, whatever the subproblem's size.
//
// Block of 256 threads, chunks of kTcChunk = 32 points (four K = 8 steps,
// three products each = 12 MMAs per chunk), operands double-buffered in
// shared memory in the canonical K-major layout without swizzle: 8 x 16-byte
// core matrices, 8-row groups kTcSbo = 128 bytes apart, 4-column (K) groups
// LBO bytes apart.  Per chunk: all threads stage the points' window weights
// (thread (p, i): tap i of point p in each dimension); then all threads build
// A and B (16-byte stores of 4 consecutive points of one row: a warp covers
// 32 consecutive rows, conflict-free) into the buffer whose previous MMAs
// have completed (mbarrier, bounded wait); one thread issues the MMAs and a
// commit to that buffer's mbarrier, so the tensor cores work on chunk c
// while the threads build chunk c + 1.  After the subproblem the block reads
// D from TMEM (tcgen05.ld, warp w reads lanes 32w..32w+31), stages it in
// shared memory and adds it to the grid with a warp per tile row.
//
// Every wait on an mbarrier gives up after kTcMaxWaits polls: the block then
// sets bit 1 of the error flag (NFFT_ERR_TIMEOUT at the next nfft_sync),
// waits once more (bounded) for its MMAs in flight, frees its TMEM and
// returns.
#pragma once

#include "points_tiled.cuh"

namespace gbnfft {

constexpr int kTcChunk = 32;            // points per chunk
constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;            // M of every MMA
constexpr uint32_t kTcSbo = 128;        // bytes between 8-row core-matrix groups
constexpr uint32_t kTcLboA = (kTcRows / 8) * 128;              // bytes between 4-column groups of A
constexpr uint32_t kTcABytes = (kTcChunk / 4) * kTcLboA;        // one split of one A buffer (16 KB)
constexpr int kTcMaxWaits = 1 << 22;

// ncols: N of the MMAs (2 T2 rounded up to 16, at most kTcMaxCols);
// tmem_cols: TMEM columns allocated, 4 x a power of two >= max(32, ncols):
// the chunk partials at columns 0 and tmem_cols / 4, the tile at tmem_cols / 2.
constexpr int kTcMaxCols = 112;         // the epilogue stages D (128 x (N + 1) floats) in the A buffers
static_assert(kTcMaxCols == kTcMaxColsHost && kTcThreads == kTcThreadsHost && kTcRows == kTcRowsHost,
              "host and device limits of the tensor-core kernel");
static_assert(kTcRows * (kTcMaxCols + 1) * 4 <= 4 * kTcABytes, "the epilogue's staging fits the A buffers");
using TcLayout = TcLaunch;

__host__ __device__ inline uint32_t tc_b_bytes(int ncols) { return (uint32_t)(kTcChunk / 4) * (uint32_t)(ncols / 8) * 128u; }

// Dynamic shared memory of k_spread_tc: A (2 buffers x hi/lo), B likewise,
// kTcChunk point records and weight rows, the tile's index tables, two
// mbarriers and the TMEM address slot.
__host__ __device__ inline size_t tc_smem_bytes(int taps, int ncols, const int* tile) {
  return 4 * (size_t)kTcABytes + 4 * (size_t)tc_b_bytes(ncols) + (size_t)kTcChunk * (16 + 8) +
         (size_t)kTcChunk * 3 * taps * 4 + (size_t)kTcRows * 8 + (size_t)(tile[0] + tile[1] + tile[2]) * 8 + 16 + 16;
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (8-row) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// M = 128, N = ncols.
__device__ __forceinline__ uint32_t tc_idesc(int ncols) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(ncols >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ float tc_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_sts4(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}

// Split four values and store hi at `hi`, lo at `lo` (16 bytes each).
__device__ __forceinline__ void tc_store_split(uint32_t hi, uint32_t lo, const float* v) {
  float h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = tc_tf32(v[q]);
    l[q] = tc_tf32(v[q] - h[q]);
  }
  tc_sts4(hi, h[0], h[1], h[2], h[3]);
  tc_sts4(lo, l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kTcMaxWaits; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// Warps 0-3: tile (TMEM columns sum_col..) += partial (src_col..), or = when
// `copy`; lane 32 w + l of TMEM is row 32 w + l of both.
__device__ __forceinline__ void tc_fold(uint32_t tmem, int warp, int ncols, uint32_t src_col, uint32_t sum_col,
                                        bool copy) {
  if (warp >= 4) return;
  const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < ncols; c0 += 16) {
    float v[16];
    tc_ld16(base + src_col + (uint32_t)c0, v);
    if (!copy) {
      float t[16];
      tc_ld16(base + sum_col + (uint32_t)c0, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += t[j];
    }
    tc_st16(base + sum_col + (uint32_t)c0, v);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int W>
__global__ void __launch_bounds__(kTcThreads, 1) k_spread_tc(PointKernelArgs<float> a, TcLayout lay) {
  static_assert(W >= 2 && W <= 8 && W % 2 == 0, "8 threads stage one point, one tap each");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int S = 3 * W;   // weight row of a staged point: wz | wy | wx
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = lay.ncols;
  const uint32_t lboB = (uint32_t)(N / 8) * 128u;
  const uint32_t bBytes = tc_b_bytes(N);
  unsigned char* const sA = smem_raw;
  unsigned char* const sB = smem_raw + 4 * kTcABytes;
  int4* const pos = reinterpret_cast<int4*>(sB + 4 * bBytes);          // z0, y0, x0 of a point's first tap
  float2* const fv = reinterpret_cast<float2*>(pos + kTcChunk);          // its value
  float* const wts = reinterpret_cast<float*>(fv + kTcChunk);            // [kTcChunk][S]
  int2* const zyt = reinterpret_cast<int2*>(wts + kTcChunk * S);         // (z, y) of tile row m (8-byte aligned)
  int64_t* const gz = reinterpret_cast<int64_t*>(zyt + kTcRows);
  const uint32_t sA_a = tc_smem_u32(sA), sB_a = tc_smem_u32(sB);
  int lo, hi;
  launch_subs(a, lo, hi);
  // the index tables and the barriers follow the largest tile of the launch
  const int T0m = a.items[a.item_begin].geom.tile[0], T1m = a.items[a.item_begin].geom.tile[1],
            T2m = a.items[a.item_begin].geom.tile[2];
  int64_t* const gy = gz + T0m;
  int64_t* const gx = gy + T1m;
  uint64_t* const bars = reinterpret_cast<uint64_t*>(gx + T2m);
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const uint32_t bar_a[2] = {tc_smem_u32(&bars[0]), tc_smem_u32(&bars[1])};

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tmem_slot)),
                 "r"(lay.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a[0]));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a[1]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc_idesc(N);
  const uint32_t part_cols = (uint32_t)lay.tmem_cols / 4;   // chunk partials at 0 and part_cols
  const uint32_t sum_col = 2 * part_cols;                    // the tile

  uint32_t cc = 0;       // chunks committed by this block (uniform)
  bool failed = false;   // a wait gave up (uniform)
  for (int sp = lo + blockIdx.x; sp < hi && !failed; sp += gridDim.x) {
    const SubProblem sub = a.pts.subs[sp];
    if (!sub_selected(a, sub)) continue;   // block-uniform
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    const float2* f_in = static_cast<const float2*>(call.in);
    float2* grid = static_cast<float2*>(it.grid);
    const int T1 = g.tile[1], T2 = g.tile[2];
    const int rows = g.tile[0] * T1;
    const WindowDev& win = it.win;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(sub.bin, g, bc);
    for (int t = 0; t < 3; ++t) origin[t] = bc[t] * g.bin[t] - win.m + win.shift;
    __syncthreads();   // the previous subproblem's flush no longer reads the tables
    for (int i = tid; i < g.tile[0] + T1 + T2; i += kTcThreads) {
      if (i < g.tile[0]) {
        gz[i] = (int64_t)wrap_mod(origin[0] + i, g.n[0]) * g.n[1] * g.n[2];
      } else if (i < g.tile[0] + T1) {
        gy[i - g.tile[0]] = (int64_t)wrap_mod(origin[1] + i - g.tile[0], g.n[1]) * g.n[2];
      } else {
        const int x = i - g.tile[0] - T1;
        gx[x] = wrap_mod(origin[2] + x, g.n[2]);
      }
    }
    // (z, y) of every MMA row; rows past the tile get a position no footprint reaches
    for (int m = tid; m < kTcRows; m += kTcThreads)
      zyt[m] = m < rows ? make_int2(m / T1, m % T1) : make_int2(-4096, -4096);
    for (int r = 0; r < call.nrhs && !failed; ++r) {
      int k = 0;          // chunks of this subproblem so far
      bool copy = true;   // the next fold starts the tile
      // thread (p, i) stages tap i of point p of every chunk; its point's
      // offsets, cell and index are loaded one chunk ahead (while the block
      // builds the current chunk) and its value after the build, so the
      // staging reads registers instead of waiting on global memory
      const int sp_p = tid >> 3, sp_i = tid & 7;
      const float sh = (float)(win.m - win.shift);
      float pd[3] = {0.0f, 0.0f, 0.0f};
      uint32_t ploc = 0;
      int pperm = 0;
      float2 pf = make_float2(0.0f, 0.0f);
      auto fetch = [&](int start) {
        if (start < sub.count && sp_p < sub.count - start) {
          const int idx = sub.start + start + sp_p;
#pragma unroll
          for (int d = 0; d < 3; ++d) pd[d] = a.pts.delta[d][idx];
          ploc = a.pts.local[idx];
          pperm = a.pts.perm[idx];
        }
      };
      auto fetch_value = [&](int start) {
        if (sp_i == 0 && start < sub.count && sp_p < sub.count - start) pf = f_in[(int64_t)r * it.M + pperm];
      };
      fetch(0);
      fetch_value(0);
      for (int pb = 0; pb < sub.count; pb += kTcChunk, ++k) {
        const int nb = min(kTcChunk, sub.count - pb);
        const int buf = (int)(cc & 1u);
        // the MMAs that last read this buffer and this partial (chunk cc - 2)
        // must be done; chunks 2p and 2p + 1 accumulate into partial p & 1, so
        // the wait completes pair (k - 3) / 2 at odd k >= 3, whose partial
        // pair (k + 1) / 2 reuses from chunk k + 1 on: it is added to the tile
        // now (the previous chunk's build is over: every thread passed its
        // barrier, so the staging tables below are free as well)
        bool ok = true;
        if (cc >= 2) ok = tc_wait(bar_a[buf], ((cc - 2) >> 1) & 1u);
        ok = __all_sync(0xffffffffu, ok);   // the fold's tensor-memory accesses are warp-wide
        if (ok && k >= 3 && (k & 1)) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          tc_fold(tmem, warp, N, (uint32_t)(((k - 3) >> 1) & 1) * part_cols, sum_col, copy);
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        if (k >= 3 && (k & 1)) copy = false;
        // stage: thread (p, i) evaluates tap i of point p in each dimension
        if (sp_p < nb) {
          if (sp_i < W) {
#pragma unroll
            for (int d = 0; d < 3; ++d) wts[sp_p * S + d * W + sp_i] = window_psi<float>(win, d, pd[d] + sh - (float)sp_i);
          }
          if (sp_i == 0) {
            pos[sp_p] = make_int4(unpack_local(ploc, 3, 0), unpack_local(ploc, 3, 1), unpack_local(ploc, 3, 2), 0);
            fv[sp_p] = pf;
          }
        } else if (sp_i == 0) {
          pos[sp_p] = make_int4(-1024, -1024, -1024, 0);   // past the chunk: a zero column of A and row of B
          fv[sp_p] = make_float2(0.0f, 0.0f);
        }
        fetch(pb + kTcChunk);
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
        // build A (rows of (z, y)) and B (rows of (x, re / im)) of the chunk:
        // item e < 1024: A row e & 127, points 4 (e >> 7) ..; then B
        const uint32_t aHi = sA_a + (uint32_t)(2 * buf) * kTcABytes, aLo = aHi + kTcABytes;
        const uint32_t bHi = sB_a + (uint32_t)(2 * buf) * bBytes, bLo = bHi + bBytes;
        const int nA = kTcRows * (kTcChunk / 4), nItems = nA + N * (kTcChunk / 4);
        for (int e = tid; e < nItems; e += kTcThreads) {
          float v[4];
          if (e < nA) {
            const int m = e & (kTcRows - 1), k4 = (e >> 7) * 4;
            const int2 zy = zyt[m];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int kk = k4 + q;
              const int4 ps = pos[kk];
              const int dz = zy.x - ps.x, dy = zy.y - ps.y;
              const bool in = (unsigned)dz < (unsigned)W && (unsigned)dy < (unsigned)W;
              const float wz = wts[kk * S + (in ? dz : 0)];
              const float wy = wts[kk * S + W + (in ? dy : 0)];
              v[q] = in ? wz * wy : 0.0f;
            }
            const uint32_t off = (uint32_t)m * 16u + (uint32_t)(k4 >> 2) * kTcLboA;
            tc_store_split(aHi + off, aLo + off, v);
          } else {
            const int eb = e - nA;
            const int n = eb % N, k4 = (eb / N) * 4;
            const int x = n >> 1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int kk = k4 + q;
              const int dx = x - pos[kk].z;
              const bool in = x < T2 && (unsigned)dx < (unsigned)W;
              const float wx = wts[kk * S + 2 * W + (in ? dx : 0)];
              const float2 f = fv[kk];
              v[q] = in ? wx * ((n & 1) ? f.y : f.x) : 0.0f;
            }
            const uint32_t off = (uint32_t)n * 16u + (uint32_t)(k4 >> 2) * lboB;
            tc_store_split(bHi + off, bLo + off, v);
          }
        }
        fetch_value(pb + kTcChunk);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int ks = 0; ks < kTcChunk / 8; ++ks) {
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
              const uint32_t ad = (pr == 2 ? aLo : aHi) + (uint32_t)(2 * ks) * kTcLboA;
              const uint32_t bd = (pr == 1 ? bLo : bHi) + (uint32_t)(2 * ks) * lboB;
              tc_mma(tmem + (uint32_t)((k >> 1) & 1) * part_cols, tc_desc(ad, kTcLboA, kTcSbo),
                     tc_desc(bd, lboB, kTcSbo), idesc, ((k & 1) || ks > 0 || pr > 0) ? 1u : 0u);
            }
          }
          tc_commit(bar_a[buf]);
        }
        ++cc;
      }
      if (failed || k == 0) continue;   // k == 0: the subproblem had no points
      // the subproblem's last commit covers every MMA before it; its last
      // one or two partials are still to be added
      const uint32_t last = cc - 1;
      const bool ok = tc_wait(bar_a[last & 1u], (last >> 1) & 1u);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      {
        // pairs folded in the loop: one per odd k in [3, K - 1]; the rest (one or two) now
        const int pairs = (k + 1) >> 1;
        const int folded = k >= 4 ? ((k - 4) >> 1) + 1 : 0;
        for (int pp = folded; pp < pairs; ++pp) {
          tc_fold(tmem, warp, N, (uint32_t)(pp & 1) * part_cols, sum_col, copy);
          copy = false;
        }
      }
      // the tile -> shared (the A buffers: every MMA reading them is done), row m at pitch N + 1
      float* const scratch = reinterpret_cast<float*>(sA);
      const int pitch = N + 1;
      if (warp < 4) {
        const int m = warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + sum_col + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) scratch[m * pitch + c0 + j] = v[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      // add the tile to the grid: a warp per (z, y) row, lanes along x
      for (int row = warp; row < rows; row += kTcThreads / 32) {
        const int z = row / T1, y = row - z * T1;
        const int64_t gb = (int64_t)r * g.grid_cells + gz[z] + gy[y];
        for (int x = lane; x < T2; x += 32) {
          const float2 c = make_float2(scratch[row * pitch + 2 * x], scratch[row * pitch + 2 * x + 1]);
          if (c.x != 0.0f || c.y != 0.0f) grid_add(grid + gb + gx[x], c);
        }
      }
      __syncthreads();   // scratch read before the next chunk's operands overwrite it
    }
  }
  if (failed) {
    if (tid == 0) atomicOr(a.err, 2);
    // one more bounded wait for the MMAs in flight before the memory goes away
    if (cc > 0) tc_wait(bar_a[(cc - 1) & 1u], ((cc - 1) >> 1) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}


// ---------------------------------------------------------------------------
// Interpolation on the tensor cores (the interpolating step of Section 2,
// Fig. 2, Algorithm 5): f_j = sum_{z,y,x} G[z,y,x] wz_j(z - z0_j) wy_j(y - y0_j)
// wx_j(x - x0_j).  With the chunk's points as the M dimension (128 points),
// the tile's (z, y) rows as K (128) and the tile's x columns, real and
// imaginary part side by side, as N:
//   D[j, (x,c)] = sum_m A[j, m] B[(x,c), m],  A[j, (z,y)] = wz_j(z - z0_j) wy_j(y - y0_j),
//   B[(x,c), (z,y)] = the tile's component c at (z, y, x),
// and f_j = sum_x wx_j(x - x0_j) (D[j, (x,0)] + i D[j, (x,1)]): TMEM lane j
// holds point j's row, so each thread finishes its own point's sum over x.
// B (the tile) is loaded and split once per subproblem; A is built per chunk
// of 128 points (hi and lo, 64 KB each); 16 K steps x 3 products = 48 MMAs
// (M = 128, N = 2 T2 rounded to 16, K = 8) per chunk, whose FP32 accumulation
// error is that of 48 MMAs.  One block per SM (about 190 KB of shared
// memory); the chunk steps run in sequence: stage, build A, MMAs, wait
// (bounded), read D.
constexpr int kTcIChunk = 128;                                  // points per chunk (M)
constexpr uint32_t kTcILboA = (kTcIChunk / 8) * 128;            // K groups of A 2048 bytes apart
constexpr uint32_t kTcIABytes = (kTcRows / 4) * kTcILboA;       // one split of A: 128 x 128 floats (64 KB)
__host__ __device__ inline uint32_t tc_ib_bytes(int ncols) { return (uint32_t)(kTcRows / 4) * (uint32_t)(ncols / 8) * 128u; }

// Dynamic shared memory of k_interp_tc: A hi/lo, B hi/lo, kTcIChunk point
// records (position, output index) and weight rows, index tables, one
// mbarrier and the TMEM slot.
__host__ __device__ inline size_t tc_interp_smem_bytes(int taps, int ncols, const int* tile) {
  return 2 * (size_t)kTcIABytes + 2 * (size_t)tc_ib_bytes(ncols) + (size_t)kTcIChunk * (16 + 8) +
         (size_t)kTcIChunk * 3 * taps * 4 + (size_t)kTcRows * 8 + (size_t)(tile[0] + tile[1] + tile[2]) * 8 + 16 +
         16;
}

template <int W>
__global__ void __launch_bounds__(kTcThreads, 1) k_interp_tc(PointKernelArgs<float> a, TcLayout lay) {
  static_assert(W >= 2 && W <= 8 && W % 2 == 0, "windows of 2 to 8 taps");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int S = 3 * W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = lay.ncols;
  const uint32_t lboB = (uint32_t)(N / 8) * 128u;
  const uint32_t bBytes = tc_ib_bytes(N);
  unsigned char* const sA = smem_raw;
  unsigned char* const sB = smem_raw + 2 * kTcIABytes;
  int4* const pos = reinterpret_cast<int4*>(sB + 2 * bBytes);         // z0, y0, x0 of a point's first tap
  int* const jt = reinterpret_cast<int*>(pos + kTcIChunk);              // its index in the output
  float* const wts = reinterpret_cast<float*>(jt + 2 * kTcIChunk);      // [kTcIChunk][S] (8-byte aligned)
  int2* const zyt = reinterpret_cast<int2*>(wts + kTcIChunk * S);        // (z, y) of tile row m
  int64_t* const gz = reinterpret_cast<int64_t*>(zyt + kTcRows);
  const uint32_t sA_a = tc_smem_u32(sA), sB_a = tc_smem_u32(sB);
  int lo, hi;
  launch_subs(a, lo, hi);
  const int T0m = a.items[a.item_begin].geom.tile[0], T1m = a.items[a.item_begin].geom.tile[1],
            T2m = a.items[a.item_begin].geom.tile[2];
  int64_t* const gy = gz + T0m;
  int64_t* const gx = gy + T1m;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(gx + T2m);
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t bar_a = tc_smem_u32(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tmem_slot)),
                 "r"(lay.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc_idesc(N);
  const uint32_t aHi = sA_a, aLo = sA_a + kTcIABytes, bHi = sB_a, bLo = sB_a + bBytes;

  uint32_t cc = 0;   // chunks committed (uniform): the mbarrier's phase
  bool failed = false;
  for (int sp = lo + blockIdx.x; sp < hi && !failed; sp += gridDim.x) {
    const SubProblem sub = a.pts.subs[sp];
    if (!sub_selected(a, sub)) continue;   // block-uniform
    const ItemDev& it = a.items[sub.item];
    const GridGeom& g = it.geom;
    const ItemCall call = item_call(a, it);
    float2* f_out = static_cast<float2*>(call.out);
    const float2* grid_in = static_cast<const float2*>(it.grid);
    const int T1 = g.tile[1], T2 = g.tile[2];
    const int rows = g.tile[0] * T1;
    const WindowDev& win = it.win;
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(sub.bin, g, bc);
    for (int t = 0; t < 3; ++t) origin[t] = bc[t] * g.bin[t] - win.m + win.shift;
    __syncthreads();   // the previous subproblem's readers of B and the tables are done
    for (int i = tid; i < g.tile[0] + T1 + T2; i += kTcThreads) {
      if (i < g.tile[0]) {
        gz[i] = (int64_t)wrap_mod(origin[0] + i, g.n[0]) * g.n[1] * g.n[2];
      } else if (i < g.tile[0] + T1) {
        gy[i - g.tile[0]] = (int64_t)wrap_mod(origin[1] + i - g.tile[0], g.n[1]) * g.n[2];
      } else {
        const int x = i - g.tile[0] - T1;
        gx[x] = wrap_mod(origin[2] + x, g.n[2]);
      }
    }
    for (int m = tid; m < kTcRows; m += kTcThreads)
      zyt[m] = m < rows ? make_int2(m / T1, m % T1) : make_int2(-4096, -4096);
    __syncthreads();
    for (int r = 0; r < call.nrhs && !failed; ++r) {
      // B: the tile of right-hand side r, B[(x, c), m] at rows n = 2x + c,
      // K = the tile row m = (z, y); zero outside the tile
      for (int e = tid; e < N * (kTcRows / 4); e += kTcThreads) {
        const int n = e % N, m4 = (e / N) * 4;
        const int x = n >> 1;
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int m = m4 + q;
          v[q] = 0.0f;
          if (m < rows && x < T2) {
            const int2 zy = zyt[m];
            const float2 c = grid_in[(int64_t)r * g.grid_cells + gz[zy.x] + gy[zy.y] + gx[x]];
            v[q] = (n & 1) ? c.y : c.x;
          }
        }
        const uint32_t off = (uint32_t)n * 16u + (uint32_t)(m4 >> 2) * lboB;
        tc_store_split(bHi + off, bLo + off, v);
      }
      for (int pb = 0; pb < sub.count; pb += kTcIChunk) {
        const int nb = min(kTcIChunk, sub.count - pb);
        // stage: the chunk's window weights, positions and output indices
        for (int e = tid; e < kTcIChunk * W; e += kTcThreads) {
          const int p = e / W, i = e - p * W;
          if (p < nb) {
            const int idx = sub.start + pb + p;
            const float sh = (float)(win.m - win.shift);
#pragma unroll
            for (int d = 0; d < 3; ++d)
              wts[p * S + d * W + i] = window_psi<float>(win, d, a.pts.delta[d][idx] + sh - (float)i);
            if (i == 0) {
              const uint32_t loc = a.pts.local[idx];
              pos[p] = make_int4(unpack_local(loc, 3, 0), unpack_local(loc, 3, 1), unpack_local(loc, 3, 2), 0);
              jt[p] = a.pts.perm[idx];
            }
          } else if (i == 0) {
            pos[p] = make_int4(-1024, -1024, -1024, 0);   // a zero row of A
          }
        }
        __syncthreads();
        // A[j, m] = wz_j(z - z0_j) wy_j(y - y0_j); item e: point e & 127, rows 4 (e >> 7) ..
        for (int e = tid; e < kTcIChunk * (kTcRows / 4); e += kTcThreads) {
          const int j = e & (kTcIChunk - 1), m4 = (e >> 7) * 4;
          const int4 ps = pos[j];
          float v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int2 zy = zyt[m4 + q];
            const int dz = zy.x - ps.x, dy = zy.y - ps.y;
            const bool in = (unsigned)dz < (unsigned)W && (unsigned)dy < (unsigned)W;
            const float wz = wts[j * S + (in ? dz : 0)];
            const float wy = wts[j * S + W + (in ? dy : 0)];
            v[q] = in ? wz * wy : 0.0f;
          }
          const uint32_t off = (uint32_t)j * 16u + (uint32_t)(m4 >> 2) * kTcILboA;
          tc_store_split(aHi + off, aLo + off, v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int ks = 0; ks < kTcRows / 8; ++ks) {
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
              const uint32_t ad = (pr == 2 ? aLo : aHi) + (uint32_t)(2 * ks) * kTcILboA;
              const uint32_t bd = (pr == 1 ? bLo : bHi) + (uint32_t)(2 * ks) * lboB;
              tc_mma(tmem, tc_desc(ad, kTcILboA, kTcSbo), tc_desc(bd, lboB, kTcSbo), idesc,
                     (ks == 0 && pr == 0) ? 0u : 1u);
            }
          }
          tc_commit(bar_a);
        }
        const bool ok = tc_wait(bar_a, cc & 1u);
        ++cc;
        if (__syncthreads_or(!ok)) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // point j = 32 warp + lane: its row of D, summed over x with its x weights
        if (warp < 4) {
          const int j = warp * 32 + lane;
          float sr = 0.0f, si = 0.0f;
          const int x0 = pos[j].z;
          for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int h = 0; h < 8; ++h) {
              const int dx = (c0 >> 1) + h - x0;
              const bool in = (unsigned)dx < (unsigned)W;
              const float wx = wts[j * S + 2 * W + (in ? dx : 0)];
              sr = fmaf(in ? wx : 0.0f, v[2 * h], sr);
              si = fmaf(in ? wx : 0.0f, v[2 * h + 1], si);
            }
          }
          if (j < nb) f_out[(int64_t)r * it.M + jt[j]] = make_float2(sr, si);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // D read and the chunk's tables used before the next chunk overwrites them
      }
    }
  }
  if (failed) {
    if (tid == 0) atomicOr(a.err, 2);
    if (cc > 0) tc_wait(bar_a, (cc - 1) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}

}  // namespace gbnfft
