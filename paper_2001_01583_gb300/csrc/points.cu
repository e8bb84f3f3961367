// Launch wrappers for the point kernels, and the global-memory variants:
// one thread per point adding straight into the grid with atomics (the
// paper's spread kernel, Section 3) and gathering straight from it (its
// interpolate kernel, Section 3), for any dimension and tap count.
#include "points_tiled.cuh"

namespace gbnfft {

const void* spread_tiled_kernel_f32(int d, int taps);
const void* spread_tiled_kernel_f64(int d, int taps);
const void* interp_tiled_kernel_f32(int d, int taps);
const void* interp_tiled_kernel_f64(int d, int taps);

namespace {

template <typename Real>
const void* tiled_kernel(int d, int taps, bool spread);
template <>
const void* tiled_kernel<float>(int d, int taps, bool spread) {
  return spread ? spread_tiled_kernel_f32(d, taps) : interp_tiled_kernel_f32(d, taps);
}
template <>
const void* tiled_kernel<double>(int d, int taps, bool spread) {
  return spread ? spread_tiled_kernel_f64(d, taps) : interp_tiled_kernel_f64(d, taps);
}

// Per point and dimension: weights and wrapped grid indices of the W taps.
template <typename Real>
__device__ __forceinline__ void global_taps(const PointKernelArgs<Real>& a, int idx, const int* origin,
                                            Real (*w)[kMaxTaps], int (*gi)[kMaxTaps]) {
  const GridGeom& g = a.geom;
  const int W = a.win.taps;
  const uint32_t loc = a.pts.local[idx];
  for (int t = 0; t < g.d; ++t) {
    const Real base = a.pts.delta[t][idx] + (Real)(a.win.m - a.win.shift);
    const int c0 = origin[t] + unpack_local(loc, g.d, t);
    for (int i = 0; i < W; ++i) {
      w[t][i] = window_psi<Real>(a.win, t, base - (Real)i);
      gi[t][i] = wrap_mod(c0 + i, g.n[t]);
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_spread_global(PointKernelArgs<Real> a) {
  using C = typename Cplx<Real>::type;
  const GridGeom& g = a.geom;
  const int W = a.win.taps;
  const int nsub = *a.pts.num_subs;
  for (int sp = blockIdx.x; sp < nsub; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < g.d; ++t) origin[t] = bc[t] * g.bin[t] - a.win.m + a.win.shift;
    for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
      const int idx = s.start + p;
      const int j = a.pts.perm[idx];
      Real w[kMaxDim][kMaxTaps];
      int gi[kMaxDim][kMaxTaps];
      global_taps<Real>(a, idx, origin, w, gi);
      for (int r = 0; r < a.nrhs; ++r) {
        const C v = a.f_in[(int64_t)r * a.M + j];
        C* gr = a.grid + (int64_t)r * g.grid_cells;
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
  const GridGeom& g = a.geom;
  const int W = a.win.taps;
  const int nsub = *a.pts.num_subs;
  for (int sp = blockIdx.x; sp < nsub; sp += gridDim.x) {
    const SubProblem s = a.pts.subs[sp];
    int bc[kMaxDim], origin[kMaxDim];
    bin_coords(s.bin, g, bc);
    for (int t = 0; t < g.d; ++t) origin[t] = bc[t] * g.bin[t] - a.win.m + a.win.shift;
    for (int p = threadIdx.x; p < s.count; p += blockDim.x) {
      const int idx = s.start + p;
      const int j = a.pts.perm[idx];
      Real w[kMaxDim][kMaxTaps];
      int gi[kMaxDim][kMaxTaps];
      global_taps<Real>(a, idx, origin, w, gi);
      for (int r = 0; r < a.nrhs; ++r) {
        const C* gr = a.grid_in + (int64_t)r * g.grid_cells;
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
        a.f_out[(int64_t)r * a.M + j] = cmake<C>(ar, ai);
      }
    }
  }
}

}  // namespace

template <typename Real>
bool launch_spread_tiled(const PointKernelArgs<Real>& a, int blocks, int threads, size_t smem, cudaStream_t st,
                         cudaError_t* err) {
  const void* fn = tiled_kernel<Real>(a.geom.d, a.win.taps, true);
  if (!fn) return false;
  void* args[] = {const_cast<PointKernelArgs<Real>*>(&a)};
  *err = cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st);
  return true;
}

template <typename Real>
bool launch_interp_tiled(const PointKernelArgs<Real>& a, int blocks, int threads, size_t smem, cudaStream_t st,
                         cudaError_t* err) {
  const void* fn = tiled_kernel<Real>(a.geom.d, a.win.taps, false);
  if (!fn) return false;
  void* args[] = {const_cast<PointKernelArgs<Real>*>(&a)};
  *err = cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, st);
  return true;
}

template <typename Real>
cudaError_t launch_spread_global(const PointKernelArgs<Real>& a, int blocks, int threads, cudaStream_t st) {
  k_spread_global<Real><<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_interp_global(const PointKernelArgs<Real>& a, int blocks, int threads, cudaStream_t st) {
  k_interp_global<Real><<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename Real>
int tiled_blocks_per_sm(int d, int taps, bool spread, int threads, size_t smem) {
  const void* fn = tiled_kernel<Real>(d, taps, spread);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

template <typename Real>
cudaError_t tiled_set_smem_limit(int d, int taps, bool spread, size_t smem) {
  const void* fn = tiled_kernel<Real>(d, taps, spread);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#define GBNFFT_POINTS_INST(R)                                                                                    \
  template bool launch_spread_tiled<R>(const PointKernelArgs<R>&, int, int, size_t, cudaStream_t, cudaError_t*); \
  template bool launch_interp_tiled<R>(const PointKernelArgs<R>&, int, int, size_t, cudaStream_t, cudaError_t*); \
  template cudaError_t launch_spread_global<R>(const PointKernelArgs<R>&, int, int, cudaStream_t);              \
  template cudaError_t launch_interp_global<R>(const PointKernelArgs<R>&, int, int, cudaStream_t);              \
  template int tiled_blocks_per_sm<R>(int, int, bool, int, size_t);                                             \
  template cudaError_t tiled_set_smem_limit<R>(int, int, bool, size_t);
GBNFFT_POINTS_INST(float)
GBNFFT_POINTS_INST(double)

}  // namespace gbnfft
