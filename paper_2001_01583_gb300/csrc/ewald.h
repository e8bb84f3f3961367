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

// out = scale * sum_j |q_j|^2 + add.
template <typename Real>
cudaError_t launch_sumsq(const typename Cplx<Real>::type* q, int64_t M, double* partials, double scale, double add,
                         double* out, cudaStream_t st);

}  // namespace gbnfft
