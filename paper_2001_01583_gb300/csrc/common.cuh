// Shared device definitions of the gbnfft CUDA library.
//
// Grid storage: the oversampled grid I_n is stored with cell l_t at array
// index l_t mod n_t, C order (dimension d-1 fastest).  With that layout the
// centred DFTs of Section 2 are plain cuFFT transforms.
//
// Points: after nfft_set_points every point j is described, in sorted order,
// by its original index perm[p], its in-bin cell offsets (packed) and its
// in-cell offsets delta_t = u_t - floor(u_t), u_t = n_t (x_t mod 1).  The
// subproblem list cuts every non-empty bin into runs of at most P points.
//
// Window taps: a point in cell c reaches cells c - m + s + i, i = 0..W-1,
// where (s, W) = (0, 2m+2) for the Gaussian and (1, 2m) for the Kaiser-Bessel
// window (whose weight is exactly zero at the two outer cells of the 2m + 2
// the method defines).  The distance u - l of tap i is delta + (m - s) - i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbnfft {

constexpr int kMaxDim = 3;
constexpr int kMaxTaps = 32;

template <typename Real> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmake(double re, double im);
template <> __device__ __forceinline__ float2 cmake<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 cmake<double2>(double re, double im) { return make_double2(re, im); }

// c + v w for a complex v and a real w: per component one round-to-nearest
// fma (as fmaf / fma); in FP32 both components in one paired instruction
// (FFMA2, sm_100 and later).
__device__ __forceinline__ float2 cmad(float2 v, float w, float2 c) { return __ffma2_rn(v, make_float2(w, w), c); }
__device__ __forceinline__ double2 cmad(double2 v, double w, double2 c) {
  return make_double2(fma(v.x, w, c.x), fma(v.y, w, c.y));
}
// v w, per component one round-to-nearest product (FP32: FMUL2).
__device__ __forceinline__ float2 cscale(float2 v, float w) { return __fmul2_rn(v, make_float2(w, w)); }
__device__ __forceinline__ double2 cscale(double2 v, double w) { return make_double2(v.x * w, v.y * w); }

// Window parameters, normalised so that psi(0) = 1 (the constant phi(0) is
// moved into the FP64 scaling factors on the host).  The shape parameter
// depends on sigma_t = n_t / N_t, so it is kept per dimension.
struct WindowDev {
  int kind;                 // 0 Gaussian, 1 Kaiser-Bessel, 2 B-spline, 3 sinc-power
  int m;                    // cut-off
  int shift;                // s: first tap is c - m + s
  int taps;                 // W
  double b[kMaxDim];        // shape parameter per dimension
  double kb_norm[kMaxDim];  // Kaiser-Bessel: 1 / (1 - exp(-2 b m)); B-spline: 1 / M_2m(0)
  float bf[kMaxDim];        // the same two, rounded to float once (FP32 kernels)
  float kb_normf[kMaxDim];
  float binvf[kMaxDim];     // 1 / b in float (FP32 Gaussian)
};

// psi(u) = phi(u / n) / phi(0) for the distance u (in cells).
//   Gaussian:       exp(-u^2 / b)
//   Kaiser-Bessel:  sinh(b z) / z * m / sinh(b m),  z = sqrt(m^2 - u^2), |u| < m
//   B-spline:       M_2m(u) / M_2m(0)           (window_psi_any only)
//   sinc-power:     sinc(pi b u)^(2m),  |u| < m
// The Kaiser-Bessel form is evaluated as
//   exp(-b u^2 / (z + m)) * m * ((1 - exp(-2 b z)) / z) * kb_norm
// so the large exponent b m cancels exactly instead of in floating point.
template <typename Real>
__device__ __forceinline__ Real window_psi(const WindowDev& w, int t, Real u);

// Centred cardinal B-spline M_order(u), |u| < order / 2, raised from the
// indicator of [0, 1) by the two-term recurrence of uniform B-splines
// (nonnegative terms only).  Only window_psi_any (the global kernels, which
// run every B-spline plan) calls it: the other kernels keep their registers.
template <typename Real>
__device__ __noinline__ Real cardinal_bspline_dev(int order, Real u) {
  const Real s = u + (Real)(order / 2);
  if (!(s > (Real)0 && s < (Real)order)) return (Real)0;
  Real v[kMaxTaps + 1];
  const int f = (int)floor(s);
  for (int i = 0; i <= order; ++i) v[i] = (Real)0;
  v[f] = (Real)1;
  for (int j = 2; j <= order; ++j) {
    const Real inv = (Real)1 / (Real)(j - 1);
    const int i0 = f - j + 1 > 0 ? f - j + 1 : 0, i1 = f < order - j ? f : order - j;
    for (int i = i0; i <= i1; ++i) {
      const Real si = s - (Real)i;
      v[i] = (si * v[i] + ((Real)j - si) * v[i + 1]) * inv;
    }
  }
  return v[0];
}

// FP32: the hardware reciprocal square root, reciprocal and exponential
// (a few ulp each) in place of correctly rounded division, sqrt and expm1.
// At the window's peak the result is exp(0) = 1 times 1/z, within 2 ulp;
// the exponentials' argument-proportional error and the cancellation in
// 1 - exp(-2 b z) for small z act only where the weight is far below one
// (at |u| = m it is about 2 b m exp(-b m)), so every weight stays within a
// few 1e-8 of psi(u) in absolute terms, the size of its FP32 rounding.
template <>
__device__ __forceinline__ float window_psi<float>(const WindowDev& w, int t, float u) {
  if (w.kind == 0) return expf(-(u * u) * w.binvf[t]);
  const float b = w.bf[t];
  const float m = (float)w.m;
  const float u2 = u * u;
  const float m2 = m * m;
  if (!(u2 < m2)) return 0.0f;
  if (w.kind == 3) {
    // sinc(pi c u) with c = b: sinpi needs no large-argument reduction
    const float zz = b * u;
    const float sc = zz != 0.0f ? __fdividef(sinpif(zz), 3.14159265358979f * zz) : 1.0f;
    const float r = sc * sc;
    float p = 1.0f;
    for (int i = 0; i < w.m; ++i) p *= r;
    return p;
  }
  const float z2 = m2 - u2;
  const float rz = rsqrtf(z2);   // 1 / z
  const float z = z2 * rz;
  const float e = __expf(__fdividef(-b * u2, z + m));
  const float s = (1.0f - __expf(-2.0f * b * z)) * rz;
  return e * m * s * w.kb_normf[t];
}

template <>
__device__ __forceinline__ double window_psi<double>(const WindowDev& w, int t, double u) {
  const double b = w.b[t];
  if (w.kind == 0) return exp(-(u * u) / b);
  const double m = (double)w.m;
  const double u2 = u * u;
  const double m2 = m * m;
  if (!(u2 < m2)) return 0.0;
  if (w.kind == 3) {
    const double zz = b * u;
    const double sc = zz != 0.0 ? sinpi(zz) / (3.141592653589793 * zz) : 1.0;
    const double r = sc * sc;
    double p = 1.0;
    for (int i = 0; i < w.m; ++i) p *= r;
    return p;
  }
  const double z = sqrt(m2 - u2);
  const double e = exp(-b * u2 / (z + m));
  const double s = -expm1(-2.0 * b * z) / z;
  return e * m * s * w.kb_norm[t];
}

// Every window, the B-spline included (global kernels only).
template <typename Real>
__device__ __forceinline__ Real window_psi_any(const WindowDev& w, int t, Real u) {
  if (w.kind == 2) return cardinal_bspline_dev<Real>(2 * w.m, u) * (Real)w.kb_norm[t];
  return window_psi<Real>(w, t, u);
}

// One subproblem: a run of sorted points inside one bin of one item.
struct SubProblem {
  int bin;     // bin id within the item
  int start;   // first sorted position
  int count;
  int item;
};

struct GridGeom {
  int d;
  int n[kMaxDim];            // oversampled sizes (unused dims = 1)
  int bin[kMaxDim];          // bin edges (unused dims = 1)
  int nbins[kMaxDim];        // bins per dimension
  int tile[kMaxDim];         // bin + W - 1 (unused dims = 1)
  int64_t grid_cells;        // prod n
  int tile_cells;            // prod tile
};

// One transform of a batch (a single plan is a batch of one), as the
// kernels see it.  Items of one kernel launch share d, the taps and the bin
// edges (so the tile shape); n, M, the window shape and the pointers may
// differ.
struct ItemDev {
  GridGeom geom;
  WindowDev win;
  int N[kMaxDim];
  int64_t NN;                  // |I_N|
  int64_t M;
  int nrhs;
  int bin_offset;              // first global bin id of the item
  int64_t point_offset;        // first point of the item in the unsorted concatenation
  const double* x;             // M x d points (read by nfft_set_points only)
  void* grid;                  // nrhs grids of geom.grid_cells
  const double* inv_c[kMaxDim];
  const void* in;              // per call: f (adjoint) or fhat (forward), nrhs blocks
  void* out;                   // per call: fhat (adjoint) or f (forward)
};

// Point data after sorting (all arrays indexed by sorted position).
template <typename Real>
struct SortedPoints {
  const int* perm;           // sorted position -> point index within its item
  const uint32_t* local;     // packed in-bin cell offsets
  const Real* delta[kMaxDim];
  const SubProblem* subs;
  const int* sub_start;      // exclusive scan of subproblems per global bin
  const int* num_subs;       // device scalar: all subproblems
  const int* bin_count;      // points per global bin
  const int* bin_start;      // first sorted position per global bin
};

// Pack / unpack of in-bin offsets: 32 bits split evenly over d dimensions.
__host__ __device__ __forceinline__ int local_bits(int d) { return d == 1 ? 32 : (d == 2 ? 16 : 10); }

__device__ __forceinline__ int unpack_local(uint32_t v, int d, int t) {
  if (d == 1) return (int)v;
  const int bits = local_bits(d);
  return (int)((v >> (bits * t)) & ((1u << bits) - 1u));
}

__device__ __forceinline__ int wrap_mod(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

}  // namespace gbnfft
