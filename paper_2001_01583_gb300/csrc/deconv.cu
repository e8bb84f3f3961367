// Scaling kernels of Section 2, for every item of a batch in one launch.
//   adjoint step 3 ("scale", Algorithm 2): fhat(k) = ghat(k) / c_k(phi~), k in I_N,
//     read from the oversampled spectrum at array index k mod n (crop);
//   forward step 1 ("subdivide", Algorithm 5): ghat(k) = fhat(k) / c_k(phi~)
//     on I_N and 0 on I_n \ I_N, written over the whole grid.
// Work is cut into segments of rows of the last (contiguous) dimension (a
// row longer than kSegment is cut into pieces); a warp takes one segment at
// a time: it decodes the row's leading indices once and forms the product of
// their FP64 scaling factors once, then the lanes walk the segment.  A block
// of kScaleWarps warps takes kSegsPerBlock consecutive segments of one item
// of a batch (kScaleWarps of a single item).  The blocks of all items form
// one flat range (block_offsets: prefix sums of each item's blocks;
// block_items: each block's item, built on the host, so a block finds its
// item with one load).  1 / c_k is a product of per-dimension FP64 tables,
// formed in FP64 and rounded once to the data precision.
#include "kernels.h"

namespace gbnfft {

namespace {

// This block's item and its first segment: blocks of a batch map to items
// through block_items (host-built), single items have no tables.
__device__ __forceinline__ int block_item(const int* offs, const int* block_items, int64_t& first_seg) {
  if (!offs) {
    first_seg = (int64_t)blockIdx.x * kScaleWarps;
    return 0;
  }
  const int item = block_items[blockIdx.x];
  first_seg = (int64_t)(blockIdx.x - offs[item]) * kSegsPerBlock;
  return item;
}

// Leading indices of a row: row = (r * R0 + i0) * R1 + i1 over (rhs, dims < d-1)
// (rows of one launch item stay below 2^31: 32-bit arithmetic).
__device__ __forceinline__ void decode_row(uint32_t row, int d, const int* ext, int& r, int* idx) {
  uint32_t rem = row;
  for (int t = d - 2; t >= 0; --t) {
    const uint32_t e = (uint32_t)ext[t];
    const uint32_t q = rem / e;
    idx[t] = (int)(rem - q * e);
    rem = q;
  }
  r = (int)rem;
}

template <typename Real>
__global__ void __launch_bounds__(32 * kScaleWarps)
    k_deconv_crop(const ItemDev* __restrict__ items, const int* __restrict__ offs,
                  const int* __restrict__ block_items, void* out_override, int nrhs_override) {
  using C = typename Cplx<Real>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t first;
  const ItemDev& it = items[block_item(offs, block_items, first)];
  const int nrhs = out_override ? nrhs_override : it.nrhs;
  C* fhat = static_cast<C*>(out_override ? out_override : it.out);
  const C* grid = static_cast<const C*>(it.grid);
  const int d = it.geom.d;
  const int Nl = it.N[d - 1], nl = it.geom.n[d - 1];
  int64_t rows_per_rhs = 1;
  for (int t = 0; t < d - 1; ++t) rows_per_rhs *= it.N[t];
  const int segs = (Nl + kSegment - 1) / kSegment;
  const int64_t total = rows_per_rhs * nrhs * segs;
  const double* cl = it.inv_c[d - 1];
  const int per_block = offs ? kSegsPerBlock : kScaleWarps;
  for (int sb = warp; sb < per_block; sb += kScaleWarps) {
    const int64_t seg = first + sb;
    if (seg >= total) break;
    const uint32_t row = segs == 1 ? (uint32_t)seg : (uint32_t)(seg / segs);
    const int x0 = (int)(seg - (int64_t)row * segs) * kSegment, x1 = min(Nl, x0 + kSegment);
    int r, a[kMaxDim];
    decode_row(row, d, it.N, r, a);
    // grid row of the leading k's (k mod n) and their factor
    int64_t grow = 0;
    double lead = 1.0;
    for (int t = 0; t < d - 1; ++t) {
      const int k = a[t] - it.N[t] / 2;
      grow = grow * it.geom.n[t] + (k < 0 ? k + it.geom.n[t] : k);
      lead *= it.inv_c[t][a[t]];
    }
    const C* src = grid + (int64_t)r * it.geom.grid_cells + grow * nl;
    C* dst = fhat + (int64_t)row * Nl;
    for (int x = x0 + lane; x < x1; x += 32) {
      const int k = x - Nl / 2;
      const C g = src[k < 0 ? k + nl : k];
      const Real f = (Real)(lead * cl[x]);
      C o;
      o.x = g.x * f;
      o.y = g.y * f;
      dst[x] = o;
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(32 * kScaleWarps)
    k_pad_deconv(const ItemDev* __restrict__ items, const int* __restrict__ offs,
                 const int* __restrict__ block_items, const void* in_override, int nrhs_override) {
  using C = typename Cplx<Real>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t first;
  const ItemDev& it = items[block_item(offs, block_items, first)];
  const int nrhs = in_override ? nrhs_override : it.nrhs;
  const C* fhat = static_cast<const C*>(in_override ? in_override : it.in);
  C* grid = static_cast<C*>(it.grid);
  const int d = it.geom.d;
  const int Nl = it.N[d - 1], nl = it.geom.n[d - 1];
  int64_t rows_per_rhs = 1;
  for (int t = 0; t < d - 1; ++t) rows_per_rhs *= it.geom.n[t];
  const int segs = (nl + kSegment - 1) / kSegment;
  const int64_t total = rows_per_rhs * nrhs * segs;
  const double* cl = it.inv_c[d - 1];
  const int half = Nl / 2;
  const C zero = cmake<C>(0.0, 0.0);
  const int per_block = offs ? kSegsPerBlock : kScaleWarps;
  for (int sb = warp; sb < per_block; sb += kScaleWarps) {
    const int64_t seg = first + sb;
    if (seg >= total) break;
    const uint32_t row = segs == 1 ? (uint32_t)seg : (uint32_t)(seg / segs);
    const int x0 = (int)(seg - (int64_t)row * segs) * kSegment, x1 = min(nl, x0 + kSegment);
    int r, l[kMaxDim];
    decode_row(row, d, it.geom.n, r, l);
    // the row's leading k's: inside I_N or not, their fhat row and factor
    bool inside = true;
    int64_t hrow = 0;
    double lead = 1.0;
    for (int t = 0; t < d - 1; ++t) {
      const int ht = it.N[t] / 2;
      int k;
      if (l[t] < ht) k = l[t];
      else if (l[t] >= it.geom.n[t] - ht) k = l[t] - it.geom.n[t];
      else {
        inside = false;
        break;
      }
      const int a = k + ht;
      hrow = hrow * it.N[t] + a;
      lead *= it.inv_c[t][a];
    }
    C* dst = grid + (int64_t)row * nl;
    if (!inside) {
      for (int x = x0 + lane; x < x1; x += 32) dst[x] = zero;
      continue;
    }
    const C* src = fhat + ((int64_t)r * (it.NN / Nl) + hrow) * Nl;
    for (int x = x0 + lane; x < x1; x += 32) {
      int a = -1;
      if (x < half) a = x + half;
      else if (x >= nl - half) a = x - nl + half;
      C o = zero;
      if (a >= 0) {
        const C h = src[a];
        const Real f = (Real)(lead * cl[a]);
        o.x = h.x * f;
        o.y = h.y * f;
      }
      dst[x] = o;
    }
  }
}

}  // namespace

int64_t scale_blocks(int64_t rows, int64_t row_length, bool batched) {
  const int64_t segs = rows * ((row_length + kSegment - 1) / kSegment);
  const int per_block = batched ? kSegsPerBlock : kScaleWarps;
  return (segs + per_block - 1) / per_block;
}

template <typename Real>
cudaError_t launch_deconv_crop(const ItemDev* items, const int* block_offsets, const int* block_items, int64_t blocks,
                               void* out, int nrhs, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  k_deconv_crop<Real><<<(unsigned)blocks, 32 * kScaleWarps, 0, st>>>(items, block_offsets, block_items, out, nrhs);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_pad_deconv(const ItemDev* items, const int* block_offsets, const int* block_items, int64_t blocks,
                              const void* in, int nrhs, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  k_pad_deconv<Real><<<(unsigned)blocks, 32 * kScaleWarps, 0, st>>>(items, block_offsets, block_items, in, nrhs);
  return cudaGetLastError();
}

template cudaError_t launch_deconv_crop<float>(const ItemDev*, const int*, const int*, int64_t, void*, int,
                                               cudaStream_t);
template cudaError_t launch_deconv_crop<double>(const ItemDev*, const int*, const int*, int64_t, void*, int,
                                                cudaStream_t);
template cudaError_t launch_pad_deconv<float>(const ItemDev*, const int*, const int*, int64_t, const void*, int,
                                              cudaStream_t);
template cudaError_t launch_pad_deconv<double>(const ItemDev*, const int*, const int*, int64_t, const void*, int,
                                               cudaStream_t);

}  // namespace gbnfft
