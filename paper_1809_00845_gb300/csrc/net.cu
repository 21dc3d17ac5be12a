// Learned GMRES initial guess: a 1D convolutional network over the
// arclength-ordered boundary cells of a curve (circular padding), trained on
// solutions the FFT method produces; its prediction is passed to bem_solve as
// x0.  The paper has no learned component; this is the training/serving
// pattern layered on top of the operator.
//
// Network: L layers of circular 1D convolution, kernel width K, dilation d_l,
// C_in -> H -> ... -> H -> 1 channels, ReLU between layers.  Storage of the
// weights and activations is BF16 (round to nearest even), arithmetic and
// accumulation FP32; master weights and Adam moments are FP32.  Rounding
// points: every layer input (features and hidden activations) and every
// weight are rounded to BF16 before use; biases, sums and the output stay
// FP32.
//
// Sequences: a batch holds nseq sequences back to back (offsets[s] .. offsets[s+1]),
// each one closed curve, so the circular padding wraps inside each sequence.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "bem_internal.h"

struct bem_net_s {
  int cin = 0, hidden = 0, layers = 0, ksize = 0;
  std::vector<int> dil;
  std::vector<int64_t> woff, boff;  // offsets of layer weights / biases in the parameter vector
  int64_t nparams = 0;
  float* d_w = nullptr;     // FP32 master parameters
  float* d_g = nullptr;     // gradients
  float* d_m = nullptr;     // Adam first moment
  float* d_v = nullptr;     // Adam second moment
  int64_t step = 0;
  // activations: per layer input (BF16) and pre-activation (FP32) for backward
  int64_t cap = 0;          // capacity in positions
  std::vector<__nv_bfloat16*> d_act;  // layers + 1 (input of each layer, BF16)
  std::vector<float*> d_pre;          // layers (pre-activation outputs)
  float* d_grad_a = nullptr;          // scratch: gradient wrt current layer output (positions x H)
  float* d_grad_b = nullptr;          // scratch: gradient wrt current layer input
  __nv_bfloat16* d_wb = nullptr;      // BF16 copy of the weights
  __nv_bfloat16* d_wbt = nullptr;     // the same per layer as [k][cin][cout] (coalesced forward reads)
  // the BF16 copies match d_w: refreshed by the first forward after the
  // parameters change (creation, set_params, a training step), on its stream
  bool wb_fresh = false;
  double* d_loss = nullptr;
  int* d_seq = nullptr;               // sequence index per position
};

namespace bemfft {

__device__ __forceinline__ int seq_wrap(int t, int shift, int s0, int s1) {
  const int len = s1 - s0;
  int u = t - s0 + shift;
  u %= len;
  if (u < 0) u += len;
  return s0 + u;
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// wt[(k * ci + c) * co + o] = bf16(w[(o * ci + c) * K + k]): one layer's weights
// in the order the forward kernel reads them (consecutive threads, consecutive o)
__global__ void k_to_bf16_t(const float* __restrict__ w, __nv_bfloat16* __restrict__ wt, int co, int ci, int K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)co * ci * K) return;
  const int k = (int)(i % K);
  const int c = (int)((i / K) % ci);
  const int o = (int)(i / ((int64_t)K * ci));
  wt[((int64_t)k * ci + c) * co + o] = __float2bfloat16_rn(w[i]);
}

__global__ void k_seq_index(const int32_t* __restrict__ off, int nseq, int* __restrict__ seq) {
  const int s = blockIdx.x;
  if (s >= nseq) return;
  for (int t = off[s] + threadIdx.x; t < off[s + 1]; t += blockDim.x) seq[t] = s;
}

// y[t][o] = b[o] + sum_c sum_k W[o][c][k] x[wrap(t + (k - K/2) d)][c]
// x BF16 [T][cin], W BF16 [cout][cin][K]; output pre-activation FP32 and, for
// hidden layers, the next input relu(y) rounded to BF16.
__global__ void k_conv_fwd(const __nv_bfloat16* __restrict__ x, int cin, int cout, int K, int d,
                           const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
                           const int32_t* __restrict__ off, const int* __restrict__ seq, int64_t T,
                           float* __restrict__ pre, __nv_bfloat16* __restrict__ next) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * cout) return;
  const int64_t t = idx / cout;
  const int o = (int)(idx - t * cout);
  const int s = seq[t];
  const int s0 = off[s], s1 = off[s + 1];
  float acc = bias[o];
  for (int k = 0; k < K; ++k) {
    const int tt = seq_wrap((int)t, (k - K / 2) * d, s0, s1);
    const __nv_bfloat16* xr = x + (int64_t)tt * cin;
    const __nv_bfloat16* wr = Wt + (int64_t)k * cin * cout + o;  // [k][c][o]
    for (int c = 0; c < cin; ++c) acc += __bfloat162float(wr[(int64_t)c * cout]) * __bfloat162float(xr[c]);
  }
  pre[idx] = acc;
  if (next) next[idx] = __float2bfloat16_rn(acc > 0.f ? acc : 0.f);
}

// gx[t][c] = sum_o sum_k W[o][c][k] gy[wrap(t - (k - K/2) d)][o]
__global__ void k_conv_bwd_x(const float* __restrict__ gy, int cin, int cout, int K, int d,
                             const __nv_bfloat16* __restrict__ W, const int32_t* __restrict__ off,
                             const int* __restrict__ seq, int64_t T, float* __restrict__ gx) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * cin) return;
  const int64_t t = idx / cin;
  const int c = (int)(idx - t * cin);
  const int s = seq[t];
  const int s0 = off[s], s1 = off[s + 1];
  float acc = 0.f;
  for (int k = 0; k < K; ++k) {
    const int tt = seq_wrap((int)t, -(k - K / 2) * d, s0, s1);
    const float* g = gy + (int64_t)tt * cout;
    for (int o = 0; o < cout; ++o) acc += __bfloat162float(W[((int64_t)o * cin + c) * K + k]) * g[o];
  }
  gx[idx] = acc;
}

// gW[o][c][k] = sum_t gy[t][o] x[wrap(t + (k - K/2) d)][c]; gb[o] = sum_t gy[t][o].
// One block per (o, c, k) triple (and per o for the bias): deterministic
// block reduction in a fixed order.
__global__ void k_conv_bwd_w(const float* __restrict__ gy, const __nv_bfloat16* __restrict__ x, int cin, int cout,
                             int K, int d, const int32_t* __restrict__ off, const int* __restrict__ seq, int64_t T,
                             float* __restrict__ gW, float* __restrict__ gb) {
  __shared__ float red[256];
  const int64_t nw = (int64_t)cout * cin * K;
  const int64_t job = blockIdx.x;
  float acc = 0.f;
  if (job < nw) {
    const int o = (int)(job / ((int64_t)cin * K));
    const int c = (int)((job / K) % cin);
    const int k = (int)(job % K);
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
      const int s = seq[t];
      const int tt = seq_wrap((int)t, (k - K / 2) * d, off[s], off[s + 1]);
      acc += gy[t * cout + o] * __bfloat162float(x[(int64_t)tt * cin + c]);
    }
  } else {
    const int o = (int)(job - nw);
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) acc += gy[t * cout + o];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
    if ((int)threadIdx.x < sft) red[threadIdx.x] += red[threadIdx.x + sft];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (job < nw) gW[job] = red[0];
    else gb[job - nw] = red[0];
  }
}

// g *= (pre > 0)
__global__ void k_relu_bwd(float* __restrict__ g, const float* __restrict__ pre, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(pre[i] > 0.f)) g[i] = 0.f;
}

// loss = mean (y - target)^2, g = 2 (y - target) / T
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ target, int64_t T, float* __restrict__ g,
                      double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
    const float e = y[i] - target[i];
    g[i] = 2.f * e / (float)T;
    acc += (double)e * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)T);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static inline unsigned nblk(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

static bem_status net_reserve(bem_net_s* net, int64_t T) {
  if (T <= net->cap) return BEM_OK;
  for (auto p : net->d_act) cudaFree(p);
  for (auto p : net->d_pre) cudaFree(p);
  cudaFree(net->d_grad_a);
  cudaFree(net->d_grad_b);
  cudaFree(net->d_seq);
  net->d_act.assign(net->layers + 1, nullptr);
  net->d_pre.assign(net->layers, nullptr);
  const int64_t cap = T + T / 4 + 1024;
  const int wmax = std::max(net->cin, net->hidden);
  for (int l = 0; l <= net->layers; ++l) {
    const int ch = l == 0 ? net->cin : net->hidden;
    BEM_CUDA_TRY(cudaMalloc(&net->d_act[l], (size_t)cap * ch * sizeof(__nv_bfloat16)));
  }
  for (int l = 0; l < net->layers; ++l) {
    const int ch = l == net->layers - 1 ? 1 : net->hidden;
    BEM_CUDA_TRY(cudaMalloc(&net->d_pre[l], (size_t)cap * ch * sizeof(float)));
  }
  BEM_CUDA_TRY(cudaMalloc(&net->d_grad_a, (size_t)cap * wmax * sizeof(float)));
  BEM_CUDA_TRY(cudaMalloc(&net->d_grad_b, (size_t)cap * wmax * sizeof(float)));
  BEM_CUDA_TRY(cudaMalloc(&net->d_seq, (size_t)cap * sizeof(int)));
  net->cap = cap;
  return BEM_OK;
}

static bem_status net_forward(bem_net_s* net, const float* feats, const int32_t* off, int nseq, int64_t T,
                              float* out, cudaStream_t st) {
  bem_status rc = net_reserve(net, T);
  if (rc != BEM_OK) return rc;
  k_seq_index<<<nseq, 256, 0, st>>>(off, nseq, net->d_seq);
  k_to_bf16<<<nblk(T * net->cin, 256), 256, 0, st>>>(feats, net->d_act[0], T * net->cin);
  if (!net->wb_fresh) {
    k_to_bf16<<<nblk(net->nparams, 256), 256, 0, st>>>(net->d_w, net->d_wb, net->nparams);
    for (int l = 0; l < net->layers; ++l) {
      const int cin = l == 0 ? net->cin : net->hidden;
      const int cout = l == net->layers - 1 ? 1 : net->hidden;
      k_to_bf16_t<<<nblk((int64_t)cout * cin * net->ksize, 256), 256, 0, st>>>(
          net->d_w + net->woff[l], net->d_wbt + net->woff[l], cout, cin, net->ksize);
    }
    net->wb_fresh = true;
  }
  for (int l = 0; l < net->layers; ++l) {
    const int cin = l == 0 ? net->cin : net->hidden;
    const bool last = l == net->layers - 1;
    const int cout = last ? 1 : net->hidden;
    k_conv_fwd<<<nblk(T * cout, 256), 256, 0, st>>>(net->d_act[l], cin, cout, net->ksize, net->dil[l],
                                                   net->d_wbt + net->woff[l], net->d_w + net->boff[l], off,
                                                   net->d_seq, T, net->d_pre[l], last ? nullptr : net->d_act[l + 1]);
  }
  if (out)
    BEM_CUDA_TRY(cudaMemcpyAsync(out, net->d_pre[net->layers - 1], T * sizeof(float), cudaMemcpyDeviceToDevice, st));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// loss + gradients (into d_g) for the batch
static bem_status net_backward(bem_net_s* net, const float* target, const int32_t* off, int64_t T, double* loss,
                               cudaStream_t st) {
  BEM_CUDA_TRY(cudaMemsetAsync(net->d_loss, 0, sizeof(double), st));
  const int L = net->layers;
  k_mse<<<std::min<unsigned>(nblk(T, 256), 1024), 256, 0, st>>>(net->d_pre[L - 1], target, T, net->d_grad_a,
                                                                 net->d_loss);
  for (int l = L - 1; l >= 0; --l) {
    const int cin = l == 0 ? net->cin : net->hidden;
    const int cout = l == L - 1 ? 1 : net->hidden;
    if (l < L - 1) k_relu_bwd<<<nblk(T * cout, 256), 256, 0, st>>>(net->d_grad_a, net->d_pre[l], T * cout);
    const int64_t nw = (int64_t)cout * cin * net->ksize;
    k_conv_bwd_w<<<(unsigned)(nw + cout), 256, 0, st>>>(net->d_grad_a, net->d_act[l], cin, cout, net->ksize,
                                                      net->dil[l], off, net->d_seq, T, net->d_g + net->woff[l],
                                                      net->d_g + net->boff[l]);
    if (l > 0) {
      k_conv_bwd_x<<<nblk(T * cin, 256), 256, 0, st>>>(net->d_grad_a, cin, cout, net->ksize, net->dil[l],
                                                      net->d_wb + net->woff[l], off, net->d_seq, T, net->d_grad_b);
      std::swap(net->d_grad_a, net->d_grad_b);
    }
  }
  BEM_CUDA_TRY(cudaMemcpyAsync(loss, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  return BEM_OK;
}

}  // namespace bemfft

using namespace bemfft;

extern "C" {

bem_status bem_net_create(bem_net_t* out, int cin, int hidden, int layers, int ksize, const int* dilations,
                          uint64_t seed) {
  if (!out || !dilations || cin < 1 || hidden < 1 || layers < 1 || layers > 16 || ksize < 1 || (ksize % 2) == 0 ||
      cin > 256 || hidden > 256) {
    set_error("bem_net_create: need 1 <= cin, hidden <= 256, 1 <= layers <= 16, odd ksize");
    return BEM_ERR_ARG;
  }
  for (int l = 0; l < layers; ++l)
    if (dilations[l] < 1) {
      set_error("bem_net_create: dilations must be >= 1");
      return BEM_ERR_ARG;
    }
  auto* net = new bem_net_s();
  net->cin = cin;
  net->hidden = hidden;
  net->layers = layers;
  net->ksize = ksize;
  net->dil.assign(dilations, dilations + layers);
  int64_t off = 0;
  for (int l = 0; l < layers; ++l) {
    const int ci = l == 0 ? cin : hidden, co = l == layers - 1 ? 1 : hidden;
    net->woff.push_back(off);
    off += (int64_t)co * ci * ksize;
    net->boff.push_back(off);
    off += co;
  }
  net->nparams = off;
  // He-style initialisation from a seeded generator
  std::vector<float> w(off, 0.f);
  std::mt19937_64 gen(seed);
  for (int l = 0; l < layers; ++l) {
    const int ci = l == 0 ? cin : hidden, co = l == layers - 1 ? 1 : hidden;
    std::normal_distribution<float> nd(0.f, std::sqrt(2.0f / (float)(ci * ksize)));
    for (int64_t i = 0; i < (int64_t)co * ci * ksize; ++i) w[net->woff[l] + i] = nd(gen);
  }
  auto fail = [&](bem_status rc) {
    bem_net_destroy(net);
    return rc;
  };
  if (cudaMalloc(&net->d_w, off * sizeof(float)) != cudaSuccess || cudaMalloc(&net->d_g, off * sizeof(float)) ||
      cudaMalloc(&net->d_m, off * sizeof(float)) || cudaMalloc(&net->d_v, off * sizeof(float)) ||
      cudaMalloc(&net->d_wb, off * sizeof(__nv_bfloat16)) || cudaMalloc(&net->d_wbt, off * sizeof(__nv_bfloat16)) ||
      cudaMalloc(&net->d_loss, sizeof(double))) {
    set_error("bem_net_create: out of device memory");
    return fail(BEM_ERR_OOM);
  }
  if (cudaMemcpy(net->d_w, w.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->d_m, 0, off * sizeof(float)) != cudaSuccess ||
      cudaMemset(net->d_v, 0, off * sizeof(float)) != cudaSuccess) {
    set_error("bem_net_create: initialising the parameters on the device failed");
    return fail(BEM_ERR_CUDA);
  }
  *out = net;
  return BEM_OK;
}

bem_status bem_net_destroy(bem_net_t net) {
  if (!net) return BEM_OK;
  cudaFree(net->d_w);
  cudaFree(net->d_g);
  cudaFree(net->d_m);
  cudaFree(net->d_v);
  cudaFree(net->d_wb);
  cudaFree(net->d_wbt);
  cudaFree(net->d_loss);
  for (auto p : net->d_act) cudaFree(p);
  for (auto p : net->d_pre) cudaFree(p);
  cudaFree(net->d_grad_a);
  cudaFree(net->d_grad_b);
  cudaFree(net->d_seq);
  delete net;
  return BEM_OK;
}

int64_t bem_net_num_params(bem_net_t net) { return net ? net->nparams : -1; }

bem_status bem_net_get_params(bem_net_t net, float* host) {
  if (!net || !host) {
    set_error("bem_net_get_params: null argument");
    return BEM_ERR_ARG;
  }
  BEM_CUDA_TRY(cudaMemcpy(host, net->d_w, net->nparams * sizeof(float), cudaMemcpyDeviceToHost));
  return BEM_OK;
}

bem_status bem_net_set_params(bem_net_t net, const float* host) {
  if (!net || !host) {
    set_error("bem_net_set_params: null argument");
    return BEM_ERR_ARG;
  }
  BEM_CUDA_TRY(cudaMemcpy(net->d_w, host, net->nparams * sizeof(float), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemset(net->d_m, 0, net->nparams * sizeof(float)));
  BEM_CUDA_TRY(cudaMemset(net->d_v, 0, net->nparams * sizeof(float)));
  net->step = 0;
  net->wb_fresh = false;
  return BEM_OK;
}

static bem_status check_batch(bem_net_t net, const void* feats, const int32_t* off, int nseq, int64_t T) {
  if (!net || !feats || !off || nseq < 1 || T < 1) {
    set_error("bem_net: null argument or empty batch");
    return BEM_ERR_ARG;
  }
  return BEM_OK;
}

bem_status bem_net_forward(bem_net_t net, const float* feats, const int32_t* off, int nseq, int64_t T, float* out,
                           void* stream) {
  bem_status rc = check_batch(net, feats, off, nseq, T);
  if (rc != BEM_OK) return rc;
  if (!out) {
    set_error("bem_net_forward: null output");
    return BEM_ERR_ARG;
  }
  return net_forward(net, feats, off, nseq, T, out, static_cast<cudaStream_t>(stream));
}

bem_status bem_net_gradient(bem_net_t net, const float* feats, const int32_t* off, int nseq, int64_t T,
                            const float* target, float* grad_host, double* loss, void* stream) {
  bem_status rc = check_batch(net, feats, off, nseq, T);
  if (rc != BEM_OK) return rc;
  if (!target || !loss) {
    set_error("bem_net_gradient: null argument");
    return BEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((rc = net_forward(net, feats, off, nseq, T, nullptr, st)) != BEM_OK) return rc;
  if ((rc = net_backward(net, target, off, T, loss, st)) != BEM_OK) return rc;
  if (grad_host) BEM_CUDA_TRY(cudaMemcpy(grad_host, net->d_g, net->nparams * sizeof(float), cudaMemcpyDeviceToHost));
  return BEM_OK;
}

bem_status bem_net_train_step(bem_net_t net, const float* feats, const int32_t* off, int nseq, int64_t T,
                              const float* target, float lr, double* loss, void* stream) {
  bem_status rc = bem_net_gradient(net, feats, off, nseq, T, target, nullptr, loss, stream);
  if (rc != BEM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
  k_adam<<<nblk(net->nparams, 256), 256, 0, st>>>(net->d_w, net->d_g, net->d_m, net->d_v, net->nparams, lr, b1, b2,
                                                 1e-8f, c1, c2);
  net->wb_fresh = false;
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

}  // extern "C"
