// nfft_set_points kernels: argument reduction and counting sort of the points
// by spatial bin.  The bins are the on-device form of the paper's subcells
// (Section 3, Eqs. 7-8): a transform is the sum of the sub-transforms of any
// partition of the points, so every bin can be spread independently.
//
// All items of a batch are sorted in one pass: item i's points are global
// points [point_offsets[i], point_offsets[i+1]) and its bins are global bins
// [bin_offsets[i], bin_offsets[i+1]).
#include "kernels.h"

namespace gbnfft {

namespace {

// Largest i with offs[i] <= v (offs ascending, offs[0] = 0 <= v < offs[n]).
template <typename T>
__device__ __forceinline__ int find_item(const T* offs, int n, T v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Reduce one coordinate to a cell c in [0, n) and the offset u - c of the
// cell coordinate u (Eq. 5 is 1-periodic in x, so any integer shift of x
// changes no exact sum), rounded once to Real.  An offset that rounds up to 1
// moves to the next cell with offset 0 (the same position).
//
// FP32 offsets: integer arithmetic throughout (FP64 is a slow pipe here).
// The fraction of |x| is taken from its mantissa bits as a 64-bit binary
// fraction F (exact for |x| >= 2^-12; below that the bits under 2^-64 are
// dropped), the fraction of x is F or 1 - F, and the 96-bit product n F
// splits into the cell (its bits 64 and up) and the offset (the 64 below),
// whose top 32 bits are rounded to float.
// FP64 offsets: the paper's reduction written out in FP64: x is brought into
// the torus [-1/2, 1/2) of Section 1 as x - floor(x + 1/2), u = n times
// that, c = floor(u) (then taken mod n) and the offset u - floor(u), so the
// offset carries only the rounding of that product, at most n/2 2^-53 cells
// (a reduction to [0, 1) would add the rounding of x + 1 for negative x, up
// to n 2^-53 cells).
__device__ __forceinline__ unsigned long long frac64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1075 - e;   // |x| = mant * 2^-sh
  unsigned long long f;
  if (e == 0 || sh <= 0) f = 0;           // zero, subnormal (taken as 0) or an integer
  else if (sh <= 64) f = mant << (64 - sh);
  else if (sh < 64 + 53) f = mant >> (sh - 64);
  else f = 0;
  if ((b >> 63) && f) f = 0ull - f;       // frac(-y) = 1 - frac(y)
  return f;
}

template <typename Real>
__device__ __forceinline__ void reduce_cell(double x, int n, int& c, Real& delta);
template <>
__device__ __forceinline__ void reduce_cell<float>(double x, int n, int& c, float& delta) {
  const unsigned long long f = frac64(x);
  const unsigned long long nn = (unsigned long long)n;
  c = (int)__umul64hi(f, nn);
  delta = __uint2float_rn((unsigned)((f * nn) >> 32)) * 2.3283064365386963e-10f;   // 2^-32
}
template <>
__device__ __forceinline__ void reduce_cell<double>(double x, int n, int& c, double& delta) {
  const double xw = x - floor(x + 0.5);
  const double u = (double)n * xw;
  const double cf = floor(u);
  c = (int)cf;
  if (c < 0) c += n;   // u >= -n/2 - 1 (x + 1/2 may round up to the next integer)
  delta = u - cf;
}

template <typename Real>
__device__ __forceinline__ void reduce_coord(double x, int n, int& c, Real& delta) {
  int ci;
  Real dr;
  reduce_cell<Real>(x, n, ci, dr);
  if (dr >= (Real)1) {
    dr = (Real)0;
    ci += 1;
  }
  if (ci >= n) ci -= n;
  c = ci;
  delta = dr;
}

__device__ __forceinline__ double load_coord(const double* x, int64_t j, int d, int t, bool& bad) {
  const double v = x[j * d + t];
  if (!isfinite(v)) {
    bad = true;
    return 0.0;
  }
  return v;
}

// Points per thread of the two point passes: a thread's points are kSortThreads
// apart (coalesced per slot) and every load and atomic of its points is
// issued before any result is used, so each thread keeps kSortPer memory
// requests in flight (the passes are bound by memory latency).
constexpr int kSortThreads = 256;
constexpr int kSortPer = 4;

template <typename Real>
__global__ void __launch_bounds__(kSortThreads) k_bin_count(SortArgs s, int* __restrict__ bin_count,
                                                            int2* __restrict__ bin_rank) {
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * kSortPer) + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int bin[kSortPer];
  bool any_bad = false;
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    bin[k] = -1;
    if (gidx < s.total_points) {
      const int item = find_item<int64_t>(s.point_offsets, s.n_items, gidx);
      const ItemDev& it = s.items[item];
      const int64_t j = gidx - it.point_offset;
      const double* x = s.x_override ? s.x_override : it.x;
      const GridGeom& g = it.geom;
      bool bad = false;
      int local = 0;
      for (int t = 0; t < g.d; ++t) {
        int c;
        Real dl;
        reduce_coord<Real>(load_coord(x, j, g.d, t, bad), g.n[t], c, dl);
        local = local * g.nbins[t] + c / g.bin[t];
      }
      any_bad |= bad;
      bin[k] = it.bin_offset + local;
    }
  }
  if (any_bad) atomicOr(s.err, 1);
  // warp-aggregated ranks: lanes with the same bin share one atomic; the
  // atomics of all slots are in flight before their results are read
  unsigned peers[kSortPer];
  int got[kSortPer];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    peers[k] = __match_any_sync(0xffffffffu, bin[k]);
    got[k] = 0;
    if (bin[k] >= 0 && lane == __ffs(peers[k]) - 1) got[k] = atomicAdd(&bin_count[bin[k]], __popc(peers[k]));
  }
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int first = __shfl_sync(peers[k], got[k], __ffs(peers[k]) - 1);
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    if (bin[k] >= 0) bin_rank[gidx] = make_int2(bin[k], first + __popc(peers[k] & ((1u << lane) - 1u)));
  }
}

template <typename Real>
__global__ void __launch_bounds__(kSortThreads) k_scatter(SortArgs s, const int* __restrict__ bin_start,
                                                          const int2* __restrict__ bin_rank, int* __restrict__ perm,
                                                          uint32_t* __restrict__ local, Real* d0, Real* d1, Real* d2) {
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * kSortPer) + threadIdx.x;
  Real* dst[3] = {d0, d1, d2};
  int2 br[kSortPer];
  int pos[kSortPer];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    br[k] = gidx < s.total_points ? bin_rank[gidx] : make_int2(-1, 0);
  }
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) pos[k] = br[k].x >= 0 ? bin_start[br[k].x] + br[k].y : -1;
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    if (pos[k] < 0) continue;
    const int item = find_item<int64_t>(s.point_offsets, s.n_items, gidx);
    const ItemDev& it = s.items[item];
    const int64_t j = gidx - it.point_offset;
    const double* x = s.x_override ? s.x_override : it.x;
    const GridGeom& g = it.geom;
    bool bad = false;
    uint32_t packed = 0;
    const int bits = local_bits(g.d);
    for (int t = 0; t < g.d; ++t) {
      int c;
      Real dl;
      reduce_coord<Real>(load_coord(x, j, g.d, t, bad), g.n[t], c, dl);
      const uint32_t lc = (uint32_t)(c % g.bin[t]);
      packed |= (g.d == 1) ? lc : (lc << (bits * t));
      dst[t][pos[k]] = dl;
    }
    perm[pos[k]] = (int)j;
    local[pos[k]] = packed;
  }
}

// The two point passes for one item of dimension D (single plans): the
// item's geometry is held in registers, and every coordinate of a thread's
// points is loaded before any is reduced (no item search, no reload of the
// item's fields per point).
template <int D>
struct OneItem {
  const double* x;
  int64_t poff;
  int boff;
  int n[D], bw[D], nb[D];
  __device__ __forceinline__ explicit OneItem(const SortArgs& s) {
    const ItemDev& it = s.items[0];
    x = s.x_override ? s.x_override : it.x;
    poff = it.point_offset;
    boff = it.bin_offset;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      n[t] = it.geom.n[t];
      bw[t] = it.geom.bin[t];
      nb[t] = it.geom.nbins[t];
    }
  }
};

template <typename Real, int D>
__global__ void __launch_bounds__(kSortThreads) k_bin_count_one(SortArgs s, int* __restrict__ bin_count,
                                                                int2* __restrict__ bin_rank) {
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * kSortPer) + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const OneItem<D> one(s);
  double v[kSortPer][D];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
#pragma unroll
    for (int t = 0; t < D; ++t) v[k][t] = gidx < s.total_points ? one.x[(gidx - one.poff) * D + t] : 0.0;
  }
  int bin[kSortPer];
  bool any_bad = false;
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    int local = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      double c0 = v[k][t];
      if (!isfinite(c0)) {
        any_bad = true;
        c0 = 0.0;
      }
      int c;
      Real dl;
      reduce_coord<Real>(c0, one.n[t], c, dl);
      local = local * one.nb[t] + c / one.bw[t];
    }
    bin[k] = gidx < s.total_points ? one.boff + local : -1;
  }
  if (any_bad) atomicOr(s.err, 1);
  unsigned peers[kSortPer];
  int got[kSortPer];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    peers[k] = __match_any_sync(0xffffffffu, bin[k]);
    got[k] = 0;
    if (bin[k] >= 0 && lane == __ffs(peers[k]) - 1) got[k] = atomicAdd(&bin_count[bin[k]], __popc(peers[k]));
  }
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int first = __shfl_sync(peers[k], got[k], __ffs(peers[k]) - 1);
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    if (bin[k] >= 0) bin_rank[gidx] = make_int2(bin[k], first + __popc(peers[k] & ((1u << lane) - 1u)));
  }
}

template <typename Real, int D>
__global__ void __launch_bounds__(kSortThreads) k_scatter_one(SortArgs s, const int* __restrict__ bin_start,
                                                              const int2* __restrict__ bin_rank, int* __restrict__ perm,
                                                              uint32_t* __restrict__ local, Real* d0, Real* d1, Real* d2) {
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * kSortPer) + threadIdx.x;
  Real* dst[3] = {d0, d1, d2};
  const OneItem<D> one(s);
  int2 br[kSortPer];
  double v[kSortPer][D];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    const bool in = gidx < s.total_points;
    br[k] = in ? bin_rank[gidx] : make_int2(-1, 0);
#pragma unroll
    for (int t = 0; t < D; ++t) v[k][t] = in ? one.x[(gidx - one.poff) * D + t] : 0.0;
  }
  int pos[kSortPer];
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) pos[k] = br[k].x >= 0 ? bin_start[br[k].x] + br[k].y : -1;
  constexpr int bits = D == 1 ? 32 : (D == 2 ? 16 : 10);
#pragma unroll
  for (int k = 0; k < kSortPer; ++k) {
    if (pos[k] < 0) continue;
    const int64_t gidx = base + (int64_t)k * kSortThreads;
    uint32_t packed = 0;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const double c0 = isfinite(v[k][t]) ? v[k][t] : 0.0;
      int c;
      Real dl;
      reduce_coord<Real>(c0, one.n[t], c, dl);
      const uint32_t lc = (uint32_t)(c % one.bw[t]);
      packed |= (D == 1) ? lc : (lc << (bits * t));
      dst[t][pos[k]] = dl;
    }
    perm[pos[k]] = (int)(gidx - one.poff);
    local[pos[k]] = packed;
  }
}

// Exclusive scan of n ints with one block of 1024 threads: each thread scans a
// contiguous chunk sequentially, the chunk totals are scanned in shared memory.
// Used for the per-tile partial sums of the multi-block scan below.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int* __restrict__ out, int n,
                                                int* __restrict__ total) {
  __shared__ int part[1024];
  const int T = blockDim.x;
  const int chunk = (n + T - 1) / T;
  const int lo = min(n, threadIdx.x * chunk);
  const int hi = min(n, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the chunk totals
  for (int off = 1; off < T; off <<= 1) {
    const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = lo; i < hi; ++i) {
    const int v = in[i];
    out[i] = run;
    run += v;
  }
  if (total && threadIdx.x == T - 1) *total = part[T - 1];
}

// Multi-block exclusive scan: tiles of kScanTile ints.  k_scan_reduce sums
// each tile (coalesced), k_scan scans the tile sums, k_scan_apply scans each
// tile (16 consecutive ints per thread, then the block's thread totals) and
// adds its tile's offset.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive prefix of v over the block's threads (in thread order).
__device__ __forceinline__ int block_exclusive(int v) {
  __shared__ int wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += wsum[k];
  return before + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ in, int n,
                                                               int* __restrict__ partials) {
  __shared__ int wsum[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
    if (base + i < n) s += in[base + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < kScanThreads / 32; ++k) t += wsum[k];
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ in, int* __restrict__ out, int n,
                                                              const int* __restrict__ offsets) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = base + q < n ? in[base + q] : 0;
    s += v[q];
  }
  int run = block_exclusive(s) + offsets[blockIdx.x];
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
}

__global__ void k_sub_count(const int* __restrict__ bin_count, int nbins, int P, int* __restrict__ sub_count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbins) sub_count[b] = (bin_count[b] + P - 1) / P;
}

__global__ void k_sub_fill(SortArgs s, const int* __restrict__ bin_count, const int* __restrict__ bin_start,
                           const int* __restrict__ sub_start, int P, SubProblem* __restrict__ subs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= s.total_bins) return;
  const int cnt = bin_count[b];
  if (cnt == 0) return;
  const int item = find_item<int>(s.bin_offsets, s.n_items, b);
  const int local_bin = b - s.bin_offsets[item];
  const int s0 = sub_start[b];
  for (int k = 0, off = 0; off < cnt; ++k, off += P) {
    SubProblem sp;
    sp.bin = local_bin;
    sp.start = bin_start[b] + off;
    sp.count = min(P, cnt - off);
    sp.item = item;
    subs[s0 + k] = sp;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename Real>
cudaError_t launch_bin_count(const SortArgs& s, int* bin_count, int2* bin_rank, cudaStream_t st) {
  if (s.total_points == 0) return cudaSuccess;
  const unsigned blocks = blocks_for(s.total_points, kSortThreads * kSortPer);
  switch (s.single_d) {
    case 1: k_bin_count_one<Real, 1><<<blocks, kSortThreads, 0, st>>>(s, bin_count, bin_rank); break;
    case 2: k_bin_count_one<Real, 2><<<blocks, kSortThreads, 0, st>>>(s, bin_count, bin_rank); break;
    case 3: k_bin_count_one<Real, 3><<<blocks, kSortThreads, 0, st>>>(s, bin_count, bin_rank); break;
    default: k_bin_count<Real><<<blocks, kSortThreads, 0, st>>>(s, bin_count, bin_rank);
  }
  return cudaGetLastError();
}

int scan_partials_needed(int n) { return 2 * ((n + kScanTile - 1) / kScanTile) + 1; }

// Up to kScanSingle ints one block scans them in one launch (a few per
// thread); longer arrays take the three tiled launches.
constexpr int kScanSingle = 4 * kScanTile;

int scan_launches(int n) { return n <= kScanSingle ? 1 : 3; }

cudaError_t launch_scan(const int* in, int* out, int n, int* total, int* partials, cudaStream_t st) {
  if (n <= kScanSingle) {
    k_scan<<<1, 1024, 0, st>>>(in, out, n, total);
    return cudaGetLastError();
  }
  const int tiles = (n + kScanTile - 1) / kScanTile;
  int* const offsets = partials + tiles;   // the scanned tile sums
  if (tiles > 0) k_scan_reduce<<<tiles, kScanThreads, 0, st>>>(in, n, partials);
  k_scan<<<1, 1024, 0, st>>>(partials, offsets, tiles, total);
  if (tiles > 0) k_scan_apply<<<tiles, kScanThreads, 0, st>>>(in, out, n, offsets);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_scatter(const SortArgs& s, const int* bin_start, const int2* bin_rank, int* perm, uint32_t* local,
                           Real* const* delta, cudaStream_t st) {
  if (s.total_points == 0) return cudaSuccess;
  const unsigned blocks = blocks_for(s.total_points, kSortThreads * kSortPer);
  switch (s.single_d) {
    case 1:
      k_scatter_one<Real, 1><<<blocks, kSortThreads, 0, st>>>(s, bin_start, bin_rank, perm, local, delta[0], delta[1],
                                                              delta[2]);
      break;
    case 2:
      k_scatter_one<Real, 2><<<blocks, kSortThreads, 0, st>>>(s, bin_start, bin_rank, perm, local, delta[0], delta[1],
                                                              delta[2]);
      break;
    case 3:
      k_scatter_one<Real, 3><<<blocks, kSortThreads, 0, st>>>(s, bin_start, bin_rank, perm, local, delta[0], delta[1],
                                                              delta[2]);
      break;
    default:
      k_scatter<Real><<<blocks, kSortThreads, 0, st>>>(s, bin_start, bin_rank, perm, local, delta[0], delta[1],
                                                       delta[2]);
  }
  return cudaGetLastError();
}

cudaError_t launch_subproblem_count(const int* bin_count, int nbins, int P, int* sub_count, cudaStream_t st) {
  k_sub_count<<<blocks_for(nbins, 256), 256, 0, st>>>(bin_count, nbins, P, sub_count);
  return cudaGetLastError();
}

cudaError_t launch_subproblem_fill(const SortArgs& s, const int* bin_count, const int* bin_start, const int* sub_start,
                                   int P, SubProblem* subs, cudaStream_t st) {
  k_sub_fill<<<blocks_for(s.total_bins, 256), 256, 0, st>>>(s, bin_count, bin_start, sub_start, P, subs);
  return cudaGetLastError();
}

template cudaError_t launch_bin_count<float>(const SortArgs&, int*, int2*, cudaStream_t);
template cudaError_t launch_bin_count<double>(const SortArgs&, int*, int2*, cudaStream_t);
template cudaError_t launch_scatter<float>(const SortArgs&, const int*, const int2*, int*, uint32_t*, float* const*,
                                           cudaStream_t);
template cudaError_t launch_scatter<double>(const SortArgs&, const int*, const int2*, int*, uint32_t*,
                                            double* const*, cudaStream_t);

}  // namespace gbnfft
