// Reciprocal-space Ewald energy of Section 5 (Eq. 12):
//   U^K = 1/(2 pi L) sum_{n in I_N, n != 0} exp(-pi^2 |n|^2 / (alpha L)^2) / |n|^2 |S(n)|^2
//         - alpha / sqrt(pi) sum_j q_j^2,
// with S(n) = sum_j q_j exp(-2 pi i n.r_j / L), the adjoint NFFT (Eq. 5) of the
// charges at x_j = r_j / L (S(n) S(-n) = |S(n)|^2 for real charges).
//
// Reductions are deterministic: block b always sums the fixed tile
// [b * kEwaldTile, (b + 1) * kEwaldTile) of the index range in FP64 (a fixed
// per-thread stride, then a fixed shuffle tree), and a second single-block
// kernel adds the per-tile partials in a fixed tree.  The partials are the
// only scratch memory; ewald_partials_needed() gives their count.
#include <algorithm>

#include "ewald.h"

namespace gbnfft {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_sums[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_sums[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kThreads / 32 ? warp_sums[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// The Gaussian factor is separable, exp(-c |n|^2) = prod_t exp(-c n_t^2): a
// block tabulates exp(-c k^2), k = -N_t/2 .. N_t/2 - 1, per dimension in
// shared memory (dimension t at offset N_0 + .. + N_(t-1)) when the tables
// fit kEwaldTabMax doubles, so an element costs two FP64 products instead of
// an FP64 exponential (a slow pipe on this GPU).
constexpr int kEwaldTabMax = 3072;

// Fills tab (block-wide; every thread must call) and returns whether it was used.
__device__ __forceinline__ bool ewald_tables(const EwaldGeom& g, double* tab) {
  int total = 0;
  for (int t = 0; t < g.d; ++t) total += g.N[t];
  if (total > kEwaldTabMax) return false;
  int off = 0;
  for (int t = 0; t < g.d; ++t) {
    for (int i = threadIdx.x; i < g.N[t]; i += blockDim.x) {
      const double k = (double)(i - g.N[t] / 2);
      tab[off + i] = exp(-g.coef * k * k);
    }
    off += g.N[t];
  }
  __syncthreads();
  return true;
}

// Ewald weight exp(-c |n|^2) / |n|^2 of the flat C-order index e of I_N (0 at
// n = 0); a[t] gets the digit of dimension t.  tab: the tables of
// ewald_tables, or null for the exponential itself.
__device__ __forceinline__ double ewald_weight(int64_t e, const EwaldGeom& g, int* a, const double* tab) {
  if (g.NN <= (int64_t)INT32_MAX) {
    unsigned rem = (unsigned)e;
    for (int t = g.d - 1; t >= 0; --t) {
      a[t] = (int)(rem % (unsigned)g.N[t]);
      rem /= (unsigned)g.N[t];
    }
  } else {
    int64_t rem = e;
    for (int t = g.d - 1; t >= 0; --t) {
      a[t] = (int)(rem % g.N[t]);
      rem /= g.N[t];
    }
  }
  int64_t n2 = 0;
  for (int t = 0; t < g.d; ++t) {
    const int64_t k = a[t] - g.N[t] / 2;
    n2 += k * k;
  }
  if (n2 == 0) return 0.0;
  if (!tab) return exp(-g.coef * (double)n2) / (double)n2;
  double E = 1.0;
  int off = 0;
  for (int t = 0; t < g.d; ++t) {
    E *= tab[off + a[t]];
    off += g.N[t];
  }
  return E / (double)n2;
}

// Partial sums of w(n) |S(n)|^2 with S read from an fhat array (C order over I_N).
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_ewald_partial_fhat(const typename Cplx<Real>::type* __restrict__ S,
                                                                EwaldGeom g, double* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * kEwaldTile;
  const int64_t hi = lo + kEwaldTile < g.NN ? lo + kEwaldTile : g.NN;
  __shared__ double tab[kEwaldTabMax];
  const double* tp = ewald_tables(g, tab) ? tab : nullptr;
  double acc = 0.0;
  int a[kMaxDim];
  for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
    const double w = ewald_weight(e, g, a, tp);
    const double sr = (double)S[e].x, si = (double)S[e].y;
    acc += w * (sr * sr + si * si);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// The same sum with S(n) = ghat(n mod n) * inv_c(n) read straight from the
// oversampled spectrum after the FFT (the scaling step fused in; no fhat).
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_ewald_partial_grid(const typename Cplx<Real>::type* __restrict__ grid,
                                                                EwaldGeom g, double* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * kEwaldTile;
  const int64_t hi = lo + kEwaldTile < g.NN ? lo + kEwaldTile : g.NN;
  __shared__ double tab[kEwaldTabMax];
  const double* tp = ewald_tables(g, tab) ? tab : nullptr;
  double acc = 0.0;
  int a[kMaxDim];
  for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
    const double w = ewald_weight(e, g, a, tp);
    int64_t flat = 0;
    double factor = 1.0;
    for (int t = 0; t < g.d; ++t) {
      const int k = a[t] - g.N[t] / 2;
      flat = flat * g.n[t] + (k < 0 ? k + g.n[t] : k);
      factor *= g.inv_c[t][a[t]];
    }
    const typename Cplx<Real>::type v = grid[flat];
    const Real f = (Real)factor;   // the same once-rounded factor the scaling kernel applies
    const double sr = (double)(v.x * f), si = (double)(v.y * f);
    acc += w * (sr * sr + si * si);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Partial sums of |q_j|^2.
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_sumsq_partial(const typename Cplx<Real>::type* __restrict__ q, int64_t M,
                                                           double* __restrict__ partials) {
  const int64_t lo = (int64_t)blockIdx.x * kEwaldTile;
  const int64_t hi = lo + kEwaldTile < M ? lo + kEwaldTile : M;
  double acc = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += kThreads) {
    const double qr = (double)q[e].x, qi = (double)q[e].y;
    acc += qr * qr + qi * qi;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out = scale * sum(partials) + add, summed in a fixed order by one block.
__global__ void __launch_bounds__(kThreads) k_finish(const double* __restrict__ partials, int np, double scale,
                                                     double add, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += kThreads) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = scale * acc + add;
}

// w(n) n_t S(n) for t = 0, 1, 2 from S in block 0 (each thread reads its
// S(n) before writing the three blocks at the same index).
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_force_modes(typename Cplx<Real>::type* __restrict__ modes, EwaldGeom g) {
  using C = typename Cplx<Real>::type;
  __shared__ double tab[kEwaldTabMax];
  const double* tp = ewald_tables(g, tab) ? tab : nullptr;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < g.NN; e += (int64_t)gridDim.x * kThreads) {
    int a[kMaxDim];
    const double w = ewald_weight(e, g, a, tp);
    const C S = modes[e];
    const double sr = (double)S.x, si = (double)S.y;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const double f = w * (double)(a[t] - g.N[t] / 2);
      modes[t * g.NN + e] = cmake<C>(f * sr, f * si);
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(kThreads) k_force_finish(const typename Cplx<Real>::type* __restrict__ vals,
                                                          const typename Cplx<Real>::type* __restrict__ q, int64_t M,
                                                          double scale, double* __restrict__ F) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < M; i += (int64_t)gridDim.x * kThreads) {
    const double qi = (double)q[i].x;
#pragma unroll
    for (int t = 0; t < 3; ++t) F[i * 3 + t] = scale * qi * (double)vals[t * M + i].y;
  }
}

}  // namespace

template <typename Real>
cudaError_t launch_force_modes(typename Cplx<Real>::type* modes, const EwaldGeom& g, cudaStream_t st) {
  if (g.NN == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((g.NN + kThreads - 1) / kThreads, 65535);
  k_force_modes<Real><<<(unsigned)blocks, kThreads, 0, st>>>(modes, g);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_force_finish(const typename Cplx<Real>::type* vals, const typename Cplx<Real>::type* q, int64_t M,
                                double scale, double* F, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((M + kThreads - 1) / kThreads, 65535);
  k_force_finish<Real><<<(unsigned)blocks, kThreads, 0, st>>>(vals, q, M, scale, F);
  return cudaGetLastError();
}

template cudaError_t launch_force_modes<float>(float2*, const EwaldGeom&, cudaStream_t);
template cudaError_t launch_force_modes<double>(double2*, const EwaldGeom&, cudaStream_t);
template cudaError_t launch_force_finish<float>(const float2*, const float2*, int64_t, double, double*, cudaStream_t);
template cudaError_t launch_force_finish<double>(const double2*, const double2*, int64_t, double, double*,
                                                 cudaStream_t);

int64_t ewald_partials_needed(int64_t count) { return (count + kEwaldTile - 1) / kEwaldTile; }

template <typename Real>
cudaError_t launch_ewald_sum(const typename Cplx<Real>::type* src, bool from_grid, const EwaldGeom& g,
                             double* partials, double scale, double add, double* out, cudaStream_t st) {
  const int64_t np = ewald_partials_needed(g.NN);
  if (np > 0) {
    if (from_grid)
      k_ewald_partial_grid<Real><<<(unsigned)np, kThreads, 0, st>>>(src, g, partials);
    else
      k_ewald_partial_fhat<Real><<<(unsigned)np, kThreads, 0, st>>>(src, g, partials);
  }
  k_finish<<<1, kThreads, 0, st>>>(partials, (int)np, scale, add, out);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_sumsq(const typename Cplx<Real>::type* q, int64_t M, double* partials, double scale, double add,
                         double* out, cudaStream_t st) {
  const int64_t np = ewald_partials_needed(M);
  if (np > 0) k_sumsq_partial<Real><<<(unsigned)np, kThreads, 0, st>>>(q, M, partials);
  k_finish<<<1, kThreads, 0, st>>>(partials, (int)np, scale, add, out);
  return cudaGetLastError();
}

template cudaError_t launch_ewald_sum<float>(const float2*, bool, const EwaldGeom&, double*, double, double, double*,
                                             cudaStream_t);
template cudaError_t launch_ewald_sum<double>(const double2*, bool, const EwaldGeom&, double*, double, double, double*,
                                              cudaStream_t);
template cudaError_t launch_sumsq<float>(const float2*, int64_t, double*, double, double, double*, cudaStream_t);
template cudaError_t launch_sumsq<double>(const double2*, int64_t, double*, double, double, double*, cudaStream_t);

}  // namespace gbnfft
