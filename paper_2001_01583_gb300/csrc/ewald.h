// Internal interface of the Ewald reciprocal-energy reductions (ewald.cu).
#pragma once

#include "kernels.h"

namespace gbnfft {

// Elements of the index range one block sums (a fixed tile: the summation
// order never depends on the launch or the GPU).
constexpr int64_t kEwaldTile = 8192;

struct EwaldGeom {
  int d;
  int N[kMaxDim];
  int n[kMaxDim];
  int64_t NN;                     // |I_N|
  const double* inv_c[kMaxDim];   // scaling tables (grid form only)
  double coef;                    // pi^2 / (alpha L)^2
};

// Number of FP64 partials a reduction over `count` elements needs.
int64_t ewald_partials_needed(int64_t count);

// out = scale * sum_{n in I_N, n != 0} exp(-coef |n|^2) / |n|^2 |S(n)|^2 + add.
// from_grid: S(n) = src[n mod n_t] * inv_c(n) (the oversampled spectrum);
// otherwise src is S on I_N in C order.
template <typename Real>
cudaError_t launch_ewald_sum(const typename Cplx<Real>::type* src, bool from_grid, const EwaldGeom& g,
                             double* partials, double scale, double add, double* out, cudaStream_t st);

// Forces (Section 5, the negative gradient of Eq. 12): modes holds S on I_N
// (C order) in its first |I_N| complex values; afterwards its three blocks of
// |I_N| hold w(n) n_t S(n), t = 0, 1, 2, w(n) = exp(-coef |n|^2) / |n|^2
// (0 at n = 0), the right-hand sides of a forward NFFT (Eq. 6).  Requires d = 3.
template <typename Real>
cudaError_t launch_force_modes(typename Cplx<Real>::type* modes, const EwaldGeom& g, cudaStream_t st);
// F[i][t] = scale * Re(q_i) * Im(vals[t][i]) for i < M, t < 3 (vals: three
// blocks of M complex, the forward NFFT of the force modes at the points).
template <typename Real>
cudaError_t launch_force_finish(const typename Cplx<Real>::type* vals, const typename Cplx<Real>::type* q, int64_t M,
                                double scale, double* F, cudaStream_t st);

// out = scale * sum_j |q_j|^2 + add.
template <typename Real>
cudaError_t launch_sumsq(const typename Cplx<Real>::type* q, int64_t M, double* partials, double scale, double add,
                         double* out, cudaStream_t st);

}  // namespace gbnfft
