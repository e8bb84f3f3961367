// Scaling kernels of Section 2, for every item of a batch in one launch
// (blockIdx.y = item).
//   adjoint step 3 ("scale", Algorithm 2): fhat(k) = ghat(k) / c_k(phi~), k in I_N,
//     read from the oversampled spectrum at array index k mod n (crop);
//   forward step 1 ("subdivide", Algorithm 5): ghat(k) = fhat(k) / c_k(phi~)
//     on I_N and 0 on I_n \ I_N, written over the whole grid.
// 1 / c_k is a product of per-dimension FP64 tables; the product is formed in
// FP64 and rounded once to the data precision.
#include "kernels.h"

namespace gbnfft {

namespace {

template <typename Real>
__global__ void k_deconv_crop(const ItemDev* __restrict__ items, void* out_override, int nrhs_override) {
  using C = typename Cplx<Real>::type;
  const ItemDev& it = items[blockIdx.y];
  const int nrhs = out_override ? nrhs_override : it.nrhs;
  C* fhat = static_cast<C*>(out_override ? out_override : it.out);
  const C* grid = static_cast<const C*>(it.grid);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= it.NN * nrhs) return;
  const int d = it.geom.d;
  const int r = (int)(e / it.NN);
  int64_t rem = e - (int64_t)r * it.NN;
  int a[kMaxDim];
  for (int t = d - 1; t >= 0; --t) {
    a[t] = (int)(rem % it.N[t]);
    rem /= it.N[t];
  }
  int64_t flat = 0;
  double factor = 1.0;
  for (int t = 0; t < d; ++t) {
    const int k = a[t] - it.N[t] / 2;          // k_t in [-N_t/2, N_t/2)
    flat = flat * it.geom.n[t] + (k < 0 ? k + it.geom.n[t] : k);
    factor *= it.inv_c[t][a[t]];
  }
  const C g = grid[(int64_t)r * it.geom.grid_cells + flat];
  const Real f = (Real)factor;
  C o;
  o.x = g.x * f;
  o.y = g.y * f;
  fhat[e] = o;
}

template <typename Real>
__global__ void k_pad_deconv(const ItemDev* __restrict__ items, const void* in_override, int nrhs_override) {
  using C = typename Cplx<Real>::type;
  const ItemDev& it = items[blockIdx.y];
  const int nrhs = in_override ? nrhs_override : it.nrhs;
  const C* fhat = static_cast<const C*>(in_override ? in_override : it.in);
  C* grid = static_cast<C*>(it.grid);
  const int64_t cells = it.geom.grid_cells;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cells * nrhs) return;
  const int d = it.geom.d;
  const int r = (int)(e / cells);
  int64_t rem = e - (int64_t)r * cells;
  int l[kMaxDim];
  for (int t = d - 1; t >= 0; --t) {
    l[t] = (int)(rem % it.geom.n[t]);
    rem /= it.geom.n[t];
  }
  bool inside = true;
  int64_t flat = 0;
  double factor = 1.0;
  for (int t = 0; t < d; ++t) {
    const int half = it.N[t] / 2;
    int k;
    if (l[t] < half) k = l[t];
    else if (l[t] >= it.geom.n[t] - half) k = l[t] - it.geom.n[t];
    else { inside = false; break; }
    const int a = k + half;
    flat = flat * it.N[t] + a;
    factor *= it.inv_c[t][a];
  }
  C o;
  if (inside) {
    const C h = fhat[(int64_t)r * it.NN + flat];
    const Real f = (Real)factor;
    o.x = h.x * f;
    o.y = h.y * f;
  } else {
    o.x = (Real)0;
    o.y = (Real)0;
  }
  grid[e] = o;
}

}  // namespace

template <typename Real>
cudaError_t launch_deconv_crop(const ItemDev* items, int n_items, int64_t max_elems, const void* in, void* out,
                               int nrhs, cudaStream_t st) {
  (void)in;
  if (max_elems <= 0 || n_items <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((max_elems + 255) / 256), (unsigned)n_items);
  k_deconv_crop<Real><<<grid, 256, 0, st>>>(items, out, nrhs);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_pad_deconv(const ItemDev* items, int n_items, int64_t max_elems, const void* in, void* out,
                              int nrhs, cudaStream_t st) {
  (void)out;
  if (max_elems <= 0 || n_items <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((max_elems + 255) / 256), (unsigned)n_items);
  k_pad_deconv<Real><<<grid, 256, 0, st>>>(items, in, nrhs);
  return cudaGetLastError();
}

template cudaError_t launch_deconv_crop<float>(const ItemDev*, int, int64_t, const void*, void*, int, cudaStream_t);
template cudaError_t launch_deconv_crop<double>(const ItemDev*, int, int64_t, const void*, void*, int, cudaStream_t);
template cudaError_t launch_pad_deconv<float>(const ItemDev*, int, int64_t, const void*, void*, int, cudaStream_t);
template cudaError_t launch_pad_deconv<double>(const ItemDev*, int, int64_t, const void*, void*, int, cudaStream_t);

}  // namespace gbnfft
