// The learned parameter picker's network: a small MLP
//   x (n_in) -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3 (n_out)
// trained and evaluated by the kernels below: FP16 weights (what forward and
// backward read), FP32 master weights (what Adam updates), FP32 accumulation.
// Loss: masked mean squared error, L = sum mask (y - t)^2 / (2 sum mask).
//
// Kernels: one thread per sample; the block stages the FP16 weights in shared
// memory; per-sample weight gradients are added into a shared FP32 copy of
// the gradient (shared-memory atomics) and each block adds it to the global
// gradient once.  Adam runs one thread per parameter and refreshes the FP16
// copy.  The picker (nfft_pick_params) evaluates the network once per query
// and chooses the cheapest candidate whose predicted error is below eps/2.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gbnfft.h"

namespace {

constexpr int kMaxHidden = 128;
constexpr int kMaxIn = 16;
constexpr int kMaxOut = 256;
constexpr int kThreads = 128;

struct Dims {
  int n_in, n_hidden, n_out;
  int off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, n_params;
};

Dims make_dims(int n_in, int n_hidden, int n_out) {
  Dims d{};
  d.n_in = n_in;
  d.n_hidden = n_hidden;
  d.n_out = n_out;
  d.off_W1 = 0;
  d.off_b1 = d.off_W1 + n_hidden * n_in;
  d.off_W2 = d.off_b1 + n_hidden;
  d.off_b2 = d.off_W2 + n_hidden * n_hidden;
  d.off_W3 = d.off_b2 + n_hidden;
  d.off_b3 = d.off_W3 + n_out * n_hidden;
  d.n_params = d.off_b3 + n_out;
  return d;
}

// y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for one sample, keeping z1, z2.
__device__ void mlp_forward_one(const Dims& d, const __half* w, const float* x, float* z1, float* z2, float* y) {
  for (int j = 0; j < d.n_hidden; ++j) {
    float acc = __half2float(w[d.off_b1 + j]);
    const __half* row = w + d.off_W1 + j * d.n_in;
    for (int i = 0; i < d.n_in; ++i) acc = fmaf(__half2float(row[i]), x[i], acc);
    z1[j] = acc;
  }
  for (int j = 0; j < d.n_hidden; ++j) {
    float acc = __half2float(w[d.off_b2 + j]);
    const __half* row = w + d.off_W2 + j * d.n_hidden;
    for (int i = 0; i < d.n_hidden; ++i) acc = fmaf(__half2float(row[i]), fmaxf(z1[i], 0.f), acc);
    z2[j] = acc;
  }
  for (int k = 0; k < d.n_out; ++k) {
    float acc = __half2float(w[d.off_b3 + k]);
    const __half* row = w + d.off_W3 + k * d.n_hidden;
    for (int i = 0; i < d.n_hidden; ++i) acc = fmaf(__half2float(row[i]), fmaxf(z2[i], 0.f), acc);
    y[k] = acc;
  }
}

__global__ void __launch_bounds__(kThreads) k_forward(Dims d, const __half* __restrict__ w16,
                                                      const float* __restrict__ x, float* __restrict__ y, int B) {
  extern __shared__ __half sw[];
  for (int i = threadIdx.x; i < d.n_params; i += blockDim.x) sw[i] = w16[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float xi[kMaxIn], z1[kMaxHidden], z2[kMaxHidden];
  for (int i = 0; i < d.n_in; ++i) xi[i] = x[(int64_t)b * d.n_in + i];
  float out[kMaxOut];
  mlp_forward_one(d, sw, xi, z1, z2, out);
  for (int k = 0; k < d.n_out; ++k) y[(int64_t)b * d.n_out + k] = out[k];
}

__global__ void k_mask_sum(const float* __restrict__ mask, int64_t n, float* __restrict__ out) {
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += mask[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Gradient of the masked loss, accumulated into grad (FP32, zeroed by the
// caller) and loss (FP32 scalar, zeroed by the caller); denom = sum(mask).
__global__ void __launch_bounds__(kThreads) k_backward(Dims d, const __half* __restrict__ w16,
                                                       const float* __restrict__ x, const float* __restrict__ t,
                                                       const float* __restrict__ mask, int B,
                                                       const float* __restrict__ denom, float* __restrict__ grad,
                                                       float* __restrict__ loss) {
  extern __shared__ unsigned char raw[];
  __half* sw = reinterpret_cast<__half*>(raw);
  float* sg = reinterpret_cast<float*>(raw + ((d.n_params * sizeof(__half) + 15) / 16) * 16);
  for (int i = threadIdx.x; i < d.n_params; i += blockDim.x) {
    sw[i] = w16[i];
    sg[i] = 0.f;
  }
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const float inv = 1.0f / fmaxf(*denom, 1.0f);
  float my_loss = 0.f;
  if (b < B) {
    float xi[kMaxIn], z1[kMaxHidden], z2[kMaxHidden], g2[kMaxHidden], y[kMaxOut];
    for (int i = 0; i < d.n_in; ++i) xi[i] = x[(int64_t)b * d.n_in + i];
    mlp_forward_one(d, sw, xi, z1, z2, y);
    // output layer: gy = mask (y - t) / denom
    for (int i = 0; i < d.n_hidden; ++i) g2[i] = 0.f;
    for (int k = 0; k < d.n_out; ++k) {
      const float mk = mask[(int64_t)b * d.n_out + k];
      const float r = (y[k] - t[(int64_t)b * d.n_out + k]) * mk;
      my_loss += r * r;
      const float gy = r * inv;
      if (gy == 0.f) continue;
      atomicAdd(&sg[d.off_b3 + k], gy);
      const __half* row = sw + d.off_W3 + k * d.n_hidden;
      for (int i = 0; i < d.n_hidden; ++i) {
        atomicAdd(&sg[d.off_W3 + k * d.n_hidden + i], gy * fmaxf(z2[i], 0.f));
        g2[i] = fmaf(gy, __half2float(row[i]), g2[i]);
      }
    }
    // second hidden layer: gz2 = g2 * [z2 > 0]; g1 = W2^T gz2
    float g1[kMaxHidden];
    for (int i = 0; i < d.n_hidden; ++i) g1[i] = 0.f;
    for (int j = 0; j < d.n_hidden; ++j) {
      const float gz = z2[j] > 0.f ? g2[j] : 0.f;
      if (gz == 0.f) continue;
      atomicAdd(&sg[d.off_b2 + j], gz);
      const __half* row = sw + d.off_W2 + j * d.n_hidden;
      for (int i = 0; i < d.n_hidden; ++i) {
        atomicAdd(&sg[d.off_W2 + j * d.n_hidden + i], gz * fmaxf(z1[i], 0.f));
        g1[i] = fmaf(gz, __half2float(row[i]), g1[i]);
      }
    }
    // first hidden layer
    for (int j = 0; j < d.n_hidden; ++j) {
      const float gz = z1[j] > 0.f ? g1[j] : 0.f;
      if (gz == 0.f) continue;
      atomicAdd(&sg[d.off_b1 + j], gz);
      for (int i = 0; i < d.n_in; ++i) atomicAdd(&sg[d.off_W1 + j * d.n_in + i], gz * xi[i]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.n_params; i += blockDim.x)
    if (sg[i] != 0.f) atomicAdd(&grad[i], sg[i]);
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_down_sync(0xffffffffu, my_loss, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, 0.5f * my_loss * inv);
}

__global__ void k_adam(int n, float* __restrict__ master, float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, __half* __restrict__ w16, float lr, float beta1, float beta2,
                       float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * g;
  const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float p = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  master[i] = p;
  w16[i] = __float2half_rn(p);
  grad[i] = 0.f;
}

__global__ void k_to_half(int n, const float* __restrict__ src, __half* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2half_rn(src[i]);
}

__global__ void k_from_half(int n, const __half* __restrict__ src, float* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __half2float(src[i]);
}

// splitmix64 and Box-Muller for the initial weights (host side)
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

double normal01(uint64_t& s) {
  const double u1 = uniform01(s), u2 = uniform01(s);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

#define CK(call)                                                             \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      cudaGetLastError();                                                    \
      return e_ == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA; \
    }                                                                        \
  } while (0)

}  // namespace

struct nfft_mlp {
  Dims d;
  cudaStream_t stream = nullptr;
  float* master = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  __half* w16 = nullptr;
  float* scalars = nullptr;   // [mask sum, loss]
  int64_t step = 0;
  // picker metadata
  bool configured = false;
  std::vector<double> cand_sigma;
  std::vector<int> cand_m, cand_window;
  std::vector<double> feat_mean, feat_std, out_mean, out_std;
  double err_margin = 0.5;    // qualify when predicted error <= eps * err_margin
  double fp32_floor = 0.0;    // FP32 rounding floor per unit of scaling amplification
  float* xq = nullptr;        // one query on the device
  float* yq = nullptr;
};

namespace {

size_t backward_smem(const Dims& d) { return ((d.n_params * sizeof(__half) + 15) / 16) * 16 + d.n_params * sizeof(float); }
constexpr size_t kMaxSmem = 227 * 1024;

int gradients_impl(nfft_mlp* p, const float* x, const float* t, const float* mask, int B) {
  const Dims& d = p->d;
  CK(cudaMemsetAsync(p->scalars, 0, 2 * sizeof(float), p->stream));
  const int64_t nm = (int64_t)B * d.n_out;
  k_mask_sum<<<64, 256, 0, p->stream>>>(mask, nm, p->scalars);
  const size_t smem = backward_smem(d);
  CK(cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_backward<<<(B + kThreads - 1) / kThreads, kThreads, smem, p->stream>>>(d, p->w16, x, t, mask, B, p->scalars,
                                                                         p->grad, p->scalars + 1);
  CK(cudaGetLastError());
  return NFFT_OK;
}

}  // namespace

extern "C" {

int nfft_mlp_create(nfft_mlp** out, int n_in, int n_hidden, int n_out, uint64_t seed, void* cuda_stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_in < 1 || n_in > kMaxIn || n_hidden < 1 || n_hidden > kMaxHidden || n_out < 1 || n_out > kMaxOut)
    return NFFT_ERR_INVALID_ARG;
  if (backward_smem(make_dims(n_in, n_hidden, n_out)) > kMaxSmem) return NFFT_ERR_UNSUPPORTED;
  nfft_mlp* p = new (std::nothrow) nfft_mlp();
  if (!p) return NFFT_ERR_OOM;
  p->d = make_dims(n_in, n_hidden, n_out);
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t np = (size_t)p->d.n_params;
  auto fail = [&](int s) {
    cudaFree(p->master);
    cudaFree(p->grad);
    cudaFree(p->adam_m);
    cudaFree(p->adam_v);
    cudaFree(p->w16);
    cudaFree(p->scalars);
    cudaFree(p->xq);
    cudaFree(p->yq);
    delete p;
    return s;
  };
  if (cudaMalloc(&p->master, np * 4) != cudaSuccess || cudaMalloc(&p->grad, np * 4) != cudaSuccess ||
      cudaMalloc(&p->adam_m, np * 4) != cudaSuccess || cudaMalloc(&p->adam_v, np * 4) != cudaSuccess ||
      cudaMalloc(&p->w16, np * 2) != cudaSuccess || cudaMalloc(&p->scalars, 2 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->xq, kMaxIn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&p->yq, kMaxOut * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(NFFT_ERR_OOM);
  }
  // He initialisation of the weights, zero biases
  std::vector<float> h(np, 0.f);
  uint64_t s = seed;
  const Dims& d = p->d;
  for (int i = 0; i < d.n_hidden * d.n_in; ++i) h[d.off_W1 + i] = (float)(normal01(s) * std::sqrt(2.0 / d.n_in));
  for (int i = 0; i < d.n_hidden * d.n_hidden; ++i)
    h[d.off_W2 + i] = (float)(normal01(s) * std::sqrt(2.0 / d.n_hidden));
  for (int i = 0; i < d.n_out * d.n_hidden; ++i) h[d.off_W3 + i] = (float)(normal01(s) * std::sqrt(1.0 / d.n_hidden));
  const int st = nfft_mlp_set_params(p, h.data());
  if (st != NFFT_OK) return fail(st);
  if (cudaMemset(p->grad, 0, np * 4) != cudaSuccess) return fail(NFFT_ERR_CUDA);
  *out = p;
  return NFFT_OK;
}

int nfft_mlp_destroy(nfft_mlp* p) {
  if (!p) return NFFT_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  cudaFree(p->master);
  cudaFree(p->grad);
  cudaFree(p->adam_m);
  cudaFree(p->adam_v);
  cudaFree(p->w16);
  cudaFree(p->scalars);
  cudaFree(p->xq);
  cudaFree(p->yq);
  delete p;
  return NFFT_OK;
}

int nfft_mlp_num_params(const nfft_mlp* p, int64_t* n) {
  if (!p || !n) return NFFT_ERR_INVALID_ARG;
  *n = p->d.n_params;
  return NFFT_OK;
}

int nfft_mlp_set_params(nfft_mlp* p, const float* host) {
  if (!p || !host) return NFFT_ERR_INVALID_ARG;
  const size_t np = (size_t)p->d.n_params;
  // kernels of earlier calls on the network's stream may still read or
  // update these buffers: wait for them before overwriting
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaMemcpyAsync(p->master, host, np * 4, cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemsetAsync(p->adam_m, 0, np * 4, p->stream));
  CK(cudaMemsetAsync(p->adam_v, 0, np * 4, p->stream));
  k_to_half<<<(unsigned)((np + 255) / 256), 256, 0, p->stream>>>((int)np, p->master, p->w16);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  p->step = 0;
  return NFFT_OK;
}

int nfft_mlp_get_params(nfft_mlp* p, float* host, int fp16_copy) {
  if (!p || !host) return NFFT_ERR_INVALID_ARG;
  const size_t np = (size_t)p->d.n_params;
  CK(cudaStreamSynchronize(p->stream));
  if (!fp16_copy) {
    CK(cudaMemcpy(host, p->master, np * 4, cudaMemcpyDeviceToHost));
    return NFFT_OK;
  }
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, np * 4));
  k_from_half<<<(unsigned)((np + 255) / 256), 256, 0, p->stream>>>((int)np, p->w16, tmp);
  cudaError_t e = cudaMemcpyAsync(host, tmp, np * 4, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  cudaFree(tmp);
  CK(e);
  return NFFT_OK;
}

int nfft_mlp_forward(nfft_mlp* p, const float* x_dev, float* y_dev, int B) {
  if (!p || B < 0 || (B > 0 && (!x_dev || !y_dev))) return NFFT_ERR_INVALID_ARG;
  if (B == 0) return NFFT_OK;
  const size_t smem = (size_t)p->d.n_params * sizeof(__half);
  CK(cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_forward<<<(B + kThreads - 1) / kThreads, kThreads, smem, p->stream>>>(p->d, p->w16, x_dev, y_dev, B);
  CK(cudaGetLastError());
  return NFFT_OK;
}

int nfft_mlp_gradients(nfft_mlp* p, const float* x_dev, const float* t_dev, const float* mask_dev, int B,
                       float* grad_dev, float* loss_host) {
  if (!p || B < 1 || !x_dev || !t_dev || !mask_dev || !grad_dev) return NFFT_ERR_INVALID_ARG;
  const size_t np = (size_t)p->d.n_params;
  CK(cudaMemsetAsync(p->grad, 0, np * 4, p->stream));
  const int s = gradients_impl(p, x_dev, t_dev, mask_dev, B);
  if (s != NFFT_OK) return s;
  CK(cudaMemcpyAsync(grad_dev, p->grad, np * 4, cudaMemcpyDeviceToDevice, p->stream));
  CK(cudaMemsetAsync(p->grad, 0, np * 4, p->stream));
  if (loss_host) {
    CK(cudaMemcpyAsync(loss_host, p->scalars + 1, sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  return NFFT_OK;
}

int nfft_mlp_train_step(nfft_mlp* p, const float* x_dev, const float* t_dev, const float* mask_dev, int B, float lr,
                        float* loss_dev) {
  if (!p || B < 1 || !x_dev || !t_dev || !mask_dev || !(lr > 0.f)) return NFFT_ERR_INVALID_ARG;
  const int s = gradients_impl(p, x_dev, t_dev, mask_dev, B);
  if (s != NFFT_OK) return s;
  p->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - std::pow(b1, (float)p->step), bc2 = 1.f - std::pow(b2, (float)p->step);
  const int np = p->d.n_params;
  k_adam<<<(np + 255) / 256, 256, 0, p->stream>>>(np, p->master, p->grad, p->adam_m, p->adam_v, p->w16, lr, b1, b2,
                                                  1e-8f, bc1, bc2);
  CK(cudaGetLastError());
  if (loss_dev) CK(cudaMemcpyAsync(loss_dev, p->scalars + 1, sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
  return NFFT_OK;
}

int nfft_picker_configure(nfft_mlp* p, int n_candidates, const double* cand_sigma, const int* cand_m,
                          const int* cand_window, const double* feat_mean, const double* feat_std,
                          const double* out_mean, const double* out_std, double err_margin, double fp32_floor) {
  if (!p || n_candidates < 1 || 2 * n_candidates != p->d.n_out || p->d.n_in != NFFT_PICKER_FEATURES)
    return NFFT_ERR_INVALID_ARG;
  if (!(err_margin > 0.0) || err_margin > 1.0 || !(fp32_floor >= 0.0)) return NFFT_ERR_INVALID_ARG;
  if (!cand_sigma || !cand_m || !cand_window || !feat_mean || !feat_std || !out_mean || !out_std)
    return NFFT_ERR_INVALID_ARG;
  p->cand_sigma.assign(cand_sigma, cand_sigma + n_candidates);
  p->cand_m.assign(cand_m, cand_m + n_candidates);
  p->cand_window.assign(cand_window, cand_window + n_candidates);
  p->feat_mean.assign(feat_mean, feat_mean + p->d.n_in);
  p->feat_std.assign(feat_std, feat_std + p->d.n_in);
  p->out_mean.assign(out_mean, out_mean + p->d.n_out);
  p->out_std.assign(out_std, out_std + p->d.n_out);
  p->err_margin = err_margin;
  p->fp32_floor = fp32_floor;
  p->configured = true;
  return NFFT_OK;
}

int nfft_picker_features(int d, const int64_t* N, int64_t M, double cluster_std, double eps, double* f) {
  if (d < 1 || d > 3 || !N || M < 0 || !(eps > 0.0) || !f) return NFFT_ERR_INVALID_ARG;
  double logN[3] = {0.0, 0.0, 0.0};
  double NN = 1.0;
  for (int t = 0; t < d; ++t) {
    if (N[t] < 2) return NFFT_ERR_INVALID_ARG;
    logN[t] = std::log2((double)N[t]);
    NN *= (double)N[t];
  }
  const double Mm = M > 0 ? (double)M : 1.0;
  f[0] = d;
  f[1] = logN[0];
  f[2] = logN[1];
  f[3] = logN[2];
  f[4] = std::log10(Mm);
  f[5] = cluster_std;
  f[6] = std::log10(eps);
  f[7] = std::log10(Mm / NN);
  return NFFT_OK;
}

int nfft_rule_of_thumb(double eps, double* sigma, int* m, int* window) {
  if (!(eps > 0.0) || !sigma || !m || !window) return NFFT_ERR_INVALID_ARG;
  const double s = 2.0;
  int mm = (int)std::ceil(std::log(1.0 / eps) / (2.0 * M_PI * std::sqrt(1.0 - 1.0 / s)));
  if (mm < 2) mm = 2;
  if (mm > 12) mm = 12;
  *sigma = s;
  *m = mm;
  *window = NFFT_KAISER_BESSEL;
  return NFFT_OK;
}

int nfft_pick_params(nfft_mlp* p, int d, const int64_t* N, int64_t M, double cluster_std, double eps, int precision,
                     double* sigma, int* m, int* window, int* used_fallback) {
  if (!sigma || !m || !window) return NFFT_ERR_INVALID_ARG;
  if (precision != NFFT_FP64 && precision != NFFT_FP32_MIXED) return NFFT_ERR_INVALID_ARG;
  double f[NFFT_PICKER_FEATURES];
  const int s = nfft_picker_features(d, N, M, cluster_std, eps, f);
  if (s != NFFT_OK) return s;
  if (used_fallback) *used_fallback = 1;
  if (p && p->configured) {
    float xf[NFFT_PICKER_FEATURES];
    for (int i = 0; i < NFFT_PICKER_FEATURES; ++i)
      xf[i] = (float)((f[i] - p->feat_mean[i]) / (p->feat_std[i] > 0 ? p->feat_std[i] : 1.0));
    CK(cudaMemcpyAsync(p->xq, xf, sizeof(xf), cudaMemcpyHostToDevice, p->stream));
    const int fs = nfft_mlp_forward(p, p->xq, p->yq, 1);
    if (fs != NFFT_OK) return fs;
    std::vector<float> y((size_t)p->d.n_out);
    CK(cudaMemcpyAsync(y.data(), p->yq, sizeof(float) * y.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    const int K = (int)p->cand_sigma.size();
    int best = -1;
    double best_cost = 0.0;
    for (int c = 0; c < K; ++c) {
      // the candidate must be valid for these bandwidths: n_t >= 2m + 2
      bool ok = true;
      for (int t = 0; t < d; ++t)
        if (std::ceil(p->cand_sigma[c] * (double)N[t]) < 2.0 * p->cand_m[c] + 2.0) ok = false;
      if (!ok) continue;
      if (precision == NFFT_FP32_MIXED) {
        // the FP32 grid's rounding, amplified by the scaling step
        double amp = 0.0;
        if (nfft_deconv_amplification(d, N, p->cand_sigma[c], p->cand_m[c], p->cand_window[c], &amp, nullptr) !=
                NFFT_OK ||
            p->fp32_floor * amp > eps * p->err_margin)
          continue;
      }
      const double err = y[c] * p->out_std[c] + p->out_mean[c];              // predicted log10(error / eps)
      const double cost = y[K + c] * p->out_std[K + c] + p->out_mean[K + c];  // predicted log10(cost)
      if (err <= std::log10(p->err_margin) && (best < 0 || cost < best_cost)) {
        best = c;
        best_cost = cost;
      }
    }
    if (best >= 0) {
      *sigma = p->cand_sigma[best];
      *m = p->cand_m[best];
      *window = p->cand_window[best];
      if (used_fallback) *used_fallback = 0;
      return NFFT_OK;
    }
  }
  // no network, or no candidate predicted to reach eps * err_margin: the plain rule
  return nfft_rule_of_thumb(eps, sigma, m, window);
}

}  // extern "C"
