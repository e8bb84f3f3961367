// Real-space part of the Ewald energy, Eq. 11 (Section 5):
//   U^R = 1/2 sum'_n sum_{i,j} q_i q_j erfc(alpha |r_ij + n L|) / |r_ij + n L|
// over the pairs (and periodic images) closer than a cut-off r_c; the primed
// sum omits n = 0 for i = j.
//
// Two forms, chosen by the box:
//   - cell list (L / r_c >= 3): the box is cut into nc^3 cells of edge
//     h = L / nc >= r_c / 2, the ions are counting-sorted by cell, and each
//     ion visits the 5^3 cells around its own (a partner within r_c is at
//     most two cells away).  That is 125 h^3 ~ 15.6 r_c^3 of candidates
//     instead of 27 r_c^3 with cells of edge r_c: the kernel issues one pair
//     term per candidate and warp (every lane takes the same candidate, so
//     erfc runs whenever one lane of the 32 accepts), which made the kernel
//     issue-bound.  With r_c <= L / 3 only the minimum image of a pair can be
//     within r_c, and it is found exactly once.  Each ion is stored as its
//     offset from its cell's centre in FP32 (|offset| <= h / 2), so a
//     separation (d h + o_j - o_i, |d| <= 2) carries about 1e-6 of absolute
//     error instead of FP32's 1e-5 on box coordinates; the pair term
//     erfc(alpha r) / r is FP32, each neighbour cell's sum is added to the
//     ion's FP64 potential;
//   - all pairs (smaller boxes): the minimum image of every pair plus the 26
//     shifts by L, all in FP64, which is the definition itself (r_c < L).
// The energy 1/2 sum_i q_i phi_i is reduced in FP64 in a fixed order (block
// partials, then one block over the partials), so it is the same run to run.
//
// Forces (the negative gradient of Eq. 11; the paper names MD as the use but
// prints no force formula): F_i = q_i sum_j q_j g(d) (r_i - r_j + n L) with
// g(d) = (erfc(alpha d) / d + 2 alpha / sqrt(pi) exp(-alpha^2 d^2)) / d^2,
// summed by the same two forms (each ion sums its own force, no atomics).
#include <cmath>
#include <cstdint>

#include "gbnfft.h"
#include "kernels.h"

namespace gbnfft {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsReach = 2;   // neighbour cells per side (cell edge >= r_c / kRsReach)

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v into partial[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_partial(double v, double* partial) {
  __shared__ double ws[kRsThreads / 32];
  v = warp_sum_f64(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    s = warp_sum_f64(s);
    if (lane == 0) partial[blockIdx.x] = s;
  }
}

// Cell of each ion (coordinates reduced into [0, L)) and its rank in the cell.
__global__ void k_rs_count(int64_t n, const double* __restrict__ r, double L, int nc, int* __restrict__ count,
                           int2* __restrict__ cell_rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
  for (int t = 0; t < 3; ++t) {
    const double u = r[i * 3 + t] / L;
    const double s = (u - floor(u)) * nc;
    int ct = (int)floor(s);
    c[t] = ct < 0 ? 0 : (ct >= nc ? nc - 1 : ct);
  }
  const int cell = (c[0] * nc + c[1]) * nc + c[2];
  cell_rank[i] = make_int2(cell, atomicAdd(&count[cell], 1));
}

// Sorted record: offset from the cell centre (FP32) and the charge.
__global__ void k_rs_scatter(int64_t n, const double* __restrict__ r, const double* __restrict__ q, double L, int nc,
                             const int* __restrict__ start, const int2* __restrict__ cell_rank,
                             float4* __restrict__ rec, int* __restrict__ rec_cell, int* __restrict__ rec_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int2 cr = cell_rank[i];
  const int cz = cr.x % nc, cy = (cr.x / nc) % nc, cx = cr.x / (nc * nc);
  const int cc[3] = {cx, cy, cz};
  const double h = L / nc;
  float o[3];
  for (int t = 0; t < 3; ++t) {
    const double u = r[i * 3 + t] / L;
    const double pos = (u - floor(u)) * L;   // in [0, L]
    o[t] = (float)(pos - (cc[t] + 0.5) * h);
  }
  const int p = start[cr.x] + cr.y;
  rec[p] = make_float4(o[0], o[1], o[2], (float)q[i]);
  rec_cell[p] = cr.x;
  if (rec_idx) rec_idx[p] = (int)i;
}

constexpr float kTwoOverSqrtPiF = 1.1283791670955126f;
constexpr double kTwoOverSqrtPi = 1.1283791670955126;

// Potential of each sorted ion from the 27 cells around its own; block
// partials of q_i phi_i.  FORCES: also the ion's force, written to its
// original index (F: n x 3 doubles).
template <bool FORCES>
__global__ void __launch_bounds__(kRsThreads) k_rs_cells(int n, int nc, float h, float rc2, float alpha,
                                                         const float4* __restrict__ rec,
                                                         const int* __restrict__ rec_cell,
                                                         const int* __restrict__ start, double* __restrict__ partial,
                                                         const int* __restrict__ rec_idx, double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n) {
    const float4 pi = rec[i];
    const int cell = rec_cell[i];
    const int cz = cell % nc, cy = (cell / nc) % nc, cx = cell / (nc * nc);
    double phi = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    const float c2 = kTwoOverSqrtPiF * alpha, a2 = alpha * alpha;
    for (int dx = -kRsReach; dx <= kRsReach; ++dx) {
      const int x = cx + dx < 0 ? cx + dx + nc : (cx + dx >= nc ? cx + dx - nc : cx + dx);
      for (int dy = -kRsReach; dy <= kRsReach; ++dy) {
        const int y = cy + dy < 0 ? cy + dy + nc : (cy + dy >= nc ? cy + dy - nc : cy + dy);
        for (int dz = -kRsReach; dz <= kRsReach; ++dz) {
          const int z = cz + dz < 0 ? cz + dz + nc : (cz + dz >= nc ? cz + dz - nc : cz + dz);
          const int nb = (x * nc + y) * nc + z;
          const float sx = dx * h - pi.x, sy = dy * h - pi.y, sz = dz * h - pi.z;
          float acc = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
          for (int j = start[nb]; j < start[nb + 1]; ++j) {
            const float4 pj = rec[j];
            const float rx = pj.x + sx, ry = pj.y + sy, rz = pj.z + sz;   // r_j - r_i
            const float d2 = rx * rx + ry * ry + rz * rz;
            if (d2 < rc2 && d2 > 0.0f) {
              const float rinv = rsqrtf(d2);
              const float ec = erfcf(alpha * d2 * rinv) * rinv;
              acc += pj.w * ec;
              if (FORCES) {
                const float g = pj.w * (ec + c2 * __expf(-a2 * d2)) * rinv * rinv;
                ax -= g * rx;
                ay -= g * ry;
                az -= g * rz;
              }
            }
          }
          phi += (double)acc;
          if (FORCES) {
            fx += (double)ax;
            fy += (double)ay;
            fz += (double)az;
          }
        }
      }
    }
    e = (double)pi.w * phi;
    if (FORCES) {
      const int64_t o = (int64_t)rec_idx[i] * 3;
      F[o] = (double)pi.w * fx;
      F[o + 1] = (double)pi.w * fy;
      F[o + 2] = (double)pi.w * fz;
    }
  }
  block_partial(e, partial);
}

// All pairs with the minimum image and the 26 shifts by L, FP64.  FORCES:
// also each ion's force (F: n x 3 doubles, input order).
template <bool FORCES>
__global__ void __launch_bounds__(kRsThreads) k_rs_pairs(int n, const double* __restrict__ r,
                                                         const double* __restrict__ q, double L, double rc,
                                                         double alpha, double* __restrict__ partial,
                                                         double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n) {
    const double xi = r[3 * i], yi = r[3 * i + 1], zi = r[3 * i + 2];
    double phi = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int j = 0; j < n; ++j) {
      double d[3] = {xi - r[3 * j], yi - r[3 * j + 1], zi - r[3 * j + 2]};
      for (int t = 0; t < 3; ++t) d[t] -= L * rint(d[t] / L);
      for (int s = 0; s < 27; ++s) {
        const double ax = d[0] + (s / 9 - 1) * L, ay = d[1] + ((s / 3) % 3 - 1) * L, az = d[2] + (s % 3 - 1) * L;
        const double dist = sqrt(ax * ax + ay * ay + az * az);
        if (dist > 0.0 && dist < rc) {
          const double ec = erfc(alpha * dist) / dist;
          phi += q[j] * ec;
          if (FORCES) {
            const double g = q[j] * (ec + kTwoOverSqrtPi * alpha * exp(-alpha * alpha * dist * dist)) / (dist * dist);
            fx += g * ax;   // (r_i - r_j + n L)
            fy += g * ay;
            fz += g * az;
          }
        }
      }
    }
    e = q[i] * phi;
    if (FORCES) {
      F[3 * i] = q[i] * fx;
      F[3 * i + 1] = q[i] * fy;
      F[3 * i + 2] = q[i] * fz;
    }
  }
  block_partial(e, partial);
}

// Fixed-order sum of the block partials; out = scale * sum.
__global__ void __launch_bounds__(kRsThreads) k_rs_total(const double* __restrict__ partial, int count, double scale,
                                                         double* __restrict__ out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) s += partial[k];
  block_partial(s, out);                    // thread 0 writes out[0]
  if (threadIdx.x == 0) out[0] *= scale;
}

}  // namespace
}  // namespace gbnfft

namespace gbnfft {
namespace {

// The energy (and with F the forces) of Eq. 11: shared by both entry points.
int real_space_impl(int64_t n, const double* r_dev, const double* q_dev, double L, double alpha, double rcut,
                    double* energy, double* F_dev, void* cuda_stream) {
  if (n < 0 || !energy || (n > 0 && (!r_dev || !q_dev))) return NFFT_ERR_INVALID_ARG;
  if (!(L > 0.0) || !(alpha > 0.0) || !(rcut > 0.0) || !(rcut < L) || !std::isfinite(L) || !std::isfinite(alpha))
    return NFFT_ERR_INVALID_ARG;
  if (n > ((int64_t)1 << 30)) return NFFT_ERR_UNSUPPORTED;
  *energy = 0.0;
  if (n == 0) return NFFT_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // cells of edge L / nc >= rcut / kRsReach (at least 2 kRsReach + 1 of them
  // per side, so the neighbour cells are distinct); L / rcut < 3: all pairs
  const int nc = (int)std::floor(L / rcut) < 3 ? 1 : std::min((int)std::floor(kRsReach * L / rcut), 256);
  if (nc == 1 && n > 65536) return NFFT_ERR_UNSUPPORTED;   // the all-pairs form is O(n^2)
  const int ni = (int)n;
  const int blocks = (ni + kRsThreads - 1) / kRsThreads;
  const int cells = nc * nc * nc;
  // scratch: partials (blocks + 1), and for the cell list counts, starts,
  // scan scratch, (cell, rank), records, record cells and record indices
  size_t bytes = sizeof(double) * (size_t)(blocks + 1);
  if (nc > 1) {
    bytes += sizeof(int) * (size_t)(2 * cells + 2) + sizeof(int2) * (size_t)n + sizeof(float4) * (size_t)n +
             sizeof(int) * (size_t)n + sizeof(int) * (size_t)scan_partials_needed(cells + 1) +
             (F_dev ? sizeof(int) * (size_t)n : 0) + 64;
  }
  char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return NFFT_ERR_OOM;
  }
  int status = NFFT_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && status == NFFT_OK) status = NFFT_ERR_CUDA;
  };
  double* partial = reinterpret_cast<double*>(buf);
  double* total = partial + blocks;
  if (nc > 1) {
    char* p = buf + sizeof(double) * (size_t)(blocks + 1);
    float4* rec = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
    int* rec_cell = reinterpret_cast<int*>(rec + n);
    int2* cell_rank = reinterpret_cast<int2*>(rec_cell + n + (n & 1));
    int* count = reinterpret_cast<int*>(cell_rank + n);
    int* start = count + cells + 1;
    int* scan_scratch = start + cells + 1;
    int* rec_idx = F_dev ? scan_scratch + scan_partials_needed(cells + 1) : nullptr;
    ck(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(cells + 1), st));
    k_rs_count<<<blocks, kRsThreads, 0, st>>>(n, r_dev, L, nc, count, cell_rank);
    ck(cudaGetLastError());
    ck(launch_scan(count, start, cells + 1, nullptr, scan_scratch, st));   // start[cells] = n
    k_rs_scatter<<<blocks, kRsThreads, 0, st>>>(n, r_dev, q_dev, L, nc, start, cell_rank, rec, rec_cell, rec_idx);
    ck(cudaGetLastError());
    const double h = L / nc;
    if (F_dev)
      k_rs_cells<true><<<blocks, kRsThreads, 0, st>>>(ni, nc, (float)h, (float)(rcut * rcut), (float)alpha, rec,
                                                      rec_cell, start, partial, rec_idx, F_dev);
    else
      k_rs_cells<false><<<blocks, kRsThreads, 0, st>>>(ni, nc, (float)h, (float)(rcut * rcut), (float)alpha, rec,
                                                       rec_cell, start, partial, nullptr, nullptr);
    ck(cudaGetLastError());
  } else {
    if (F_dev)
      k_rs_pairs<true><<<blocks, kRsThreads, 0, st>>>(ni, r_dev, q_dev, L, rcut, alpha, partial, F_dev);
    else
      k_rs_pairs<false><<<blocks, kRsThreads, 0, st>>>(ni, r_dev, q_dev, L, rcut, alpha, partial, nullptr);
    ck(cudaGetLastError());
  }
  k_rs_total<<<1, kRsThreads, 0, st>>>(partial, blocks, 0.5, total);
  ck(cudaGetLastError());
  double host = 0.0;
  ck(cudaMemcpyAsync(&host, total, sizeof(double), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  cudaFree(buf);
  if (status == NFFT_OK) *energy = host;
  return status;
}

}  // namespace
}  // namespace gbnfft

extern "C" int nfft_ewald_real_space(int64_t n, const double* r_dev, const double* q_dev, double L, double alpha,
                                     double rcut, double* energy, void* cuda_stream) {
  return gbnfft::real_space_impl(n, r_dev, q_dev, L, alpha, rcut, energy, nullptr, cuda_stream);
}

extern "C" int nfft_ewald_real_space_forces(int64_t n, const double* r_dev, const double* q_dev, double L,
                                            double alpha, double rcut, double* F_dev, double* energy,
                                            void* cuda_stream) {
  if (n > 0 && !F_dev) return NFFT_ERR_INVALID_ARG;
  return gbnfft::real_space_impl(n, r_dev, q_dev, L, alpha, rcut, energy, n > 0 ? F_dev : nullptr, cuda_stream);
}
