// Scaling kernels of Section 2.
//   adjoint step 3 ("scale", Algorithm 2): fhat(k) = ghat(k) / c_k(phi~), k in I_N,
//     read from the oversampled spectrum at array index k mod n (crop);
//   forward step 1 ("subdivide", Algorithm 5): ghat(k) = fhat(k) / c_k(phi~)
//     on I_N and 0 on I_n \ I_N, written over the whole grid.
// 1 / c_k is a product of per-dimension FP64 tables; the product is formed in
// FP64 and rounded once to the data precision.
#include "kernels.h"

namespace gbnfft {

namespace {

struct ScaleGeom {
  int d;
  int N[kMaxDim];
  int n[kMaxDim];
  int64_t NN;      // |I_N|
  int64_t cells;   // |I_n|
  const double* inv_c[kMaxDim];
};

template <typename Real>
__global__ void k_deconv_crop(const typename Cplx<Real>::type* __restrict__ grid,
                              typename Cplx<Real>::type* __restrict__ fhat, ScaleGeom s, int R) {
  using C = typename Cplx<Real>::type;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.NN * R) return;
  const int r = (int)(e / s.NN);
  int64_t rem = e - (int64_t)r * s.NN;
  int a[kMaxDim];
  for (int t = s.d - 1; t >= 0; --t) {
    a[t] = (int)(rem % s.N[t]);
    rem /= s.N[t];
  }
  int64_t flat = 0;
  double factor = 1.0;
  for (int t = 0; t < s.d; ++t) {
    const int k = a[t] - s.N[t] / 2;          // k_t in [-N_t/2, N_t/2)
    flat = flat * s.n[t] + (k < 0 ? k + s.n[t] : k);
    factor *= s.inv_c[t][a[t]];
  }
  const C g = grid[(int64_t)r * s.cells + flat];
  const Real f = (Real)factor;
  C out;
  out.x = g.x * f;
  out.y = g.y * f;
  fhat[e] = out;
}

template <typename Real>
__global__ void k_pad_deconv(const typename Cplx<Real>::type* __restrict__ fhat,
                             typename Cplx<Real>::type* __restrict__ grid, ScaleGeom s, int R) {
  using C = typename Cplx<Real>::type;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s.cells * R) return;
  const int r = (int)(e / s.cells);
  int64_t rem = e - (int64_t)r * s.cells;
  int l[kMaxDim];
  for (int t = s.d - 1; t >= 0; --t) {
    l[t] = (int)(rem % s.n[t]);
    rem /= s.n[t];
  }
  bool inside = true;
  int64_t flat = 0;
  double factor = 1.0;
  for (int t = 0; t < s.d; ++t) {
    const int half = s.N[t] / 2;
    int k;
    if (l[t] < half) k = l[t];
    else if (l[t] >= s.n[t] - half) k = l[t] - s.n[t];
    else { inside = false; break; }
    const int a = k + half;
    flat = flat * s.N[t] + a;
    factor *= s.inv_c[t][a];
  }
  C out;
  if (inside) {
    const C h = fhat[(int64_t)r * s.NN + flat];
    const Real f = (Real)factor;
    out.x = h.x * f;
    out.y = h.y * f;
  } else {
    out.x = (Real)0;
    out.y = (Real)0;
  }
  grid[e] = out;
}

ScaleGeom make_geom(const double* const* inv_c, const GridGeom& g, const int* N) {
  ScaleGeom s;
  s.d = g.d;
  s.NN = 1;
  s.cells = 1;
  for (int t = 0; t < kMaxDim; ++t) {
    s.N[t] = t < g.d ? N[t] : 1;
    s.n[t] = t < g.d ? g.n[t] : 1;
    s.inv_c[t] = t < g.d ? inv_c[t] : nullptr;
  }
  for (int t = 0; t < g.d; ++t) {
    s.NN *= s.N[t];
    s.cells *= s.n[t];
  }
  return s;
}

}  // namespace

template <typename Real>
cudaError_t launch_deconv_crop(const typename Cplx<Real>::type* grid, typename Cplx<Real>::type* fhat,
                               const double* const* inv_c, const GridGeom& g, const int* N, int R, cudaStream_t st) {
  const ScaleGeom s = make_geom(inv_c, g, N);
  const int64_t total = s.NN * R;
  if (total == 0) return cudaSuccess;
  k_deconv_crop<Real><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(grid, fhat, s, R);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_pad_deconv(const typename Cplx<Real>::type* fhat, typename Cplx<Real>::type* grid,
                              const double* const* inv_c, const GridGeom& g, const int* N, int R, cudaStream_t st) {
  const ScaleGeom s = make_geom(inv_c, g, N);
  const int64_t total = s.cells * R;
  if (total == 0) return cudaSuccess;
  k_pad_deconv<Real><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(fhat, grid, s, R);
  return cudaGetLastError();
}

template cudaError_t launch_deconv_crop<float>(const float2*, float2*, const double* const*, const GridGeom&,
                                               const int*, int, cudaStream_t);
template cudaError_t launch_deconv_crop<double>(const double2*, double2*, const double* const*, const GridGeom&,
                                                const int*, int, cudaStream_t);
template cudaError_t launch_pad_deconv<float>(const float2*, float2*, const double* const*, const GridGeom&,
                                              const int*, int, cudaStream_t);
template cudaError_t launch_pad_deconv<double>(const double2*, double2*, const double* const*, const GridGeom&,
                                               const int*, int, cudaStream_t);

}  // namespace gbnfft
