// Input features of the learned initial guesses (the paper has no learned
// component): the arclength Dirichlet-to-Neumann estimate of closed curves
// (2D), the network's input columns and the assembled guess (2D), and random
// Fourier features of surface points (3D point network).
//
// Dirichlet-to-Neumann estimate.
// For the interior Laplace problem on a circle the Dirichlet-to-Neumann map is
// diagonal in the Fourier modes of the boundary data, e^{i k theta} -> |k| / R;
// on a smooth closed curve parametrised by arclength it equals the same
// multiplier, 2 pi |k| / Lambda (Lambda the curve length), up to an operator
// that only adds smooth (low-frequency) content.  Per curve, with boundary
// elements j at arclength positions s_j (element midpoints), lengths l_j and
// values u_j:
//   uhat_k = (1 / Lambda) sum_j l_j u_j e^{-2 pi i k s_j / Lambda},  k = 1 .. kmax
//   q_j    = sum_k (2 pi k / Lambda) 2 Re(uhat_k e^{2 pi i k s_j / Lambda}).
// Phases k s_j / Lambda reduced to [0, 1) and their sines and cosines in FP32
// (a feature: a phase error of about k 2^-24 turns), sums in FP64, outputs
// FP32.
#include <cuda_runtime.h>

#include <string>

#include "bem_internal.h"

namespace bemfft {
namespace {

constexpr int kDtnThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kDtnThreads / 32; ++w) s += red[w];  // fixed order
  return s;
}

// block (k - 1, seq): uhat_k of sequence seq; block k = 1 also stores Lambda.
// The phase k s_j / Lambda is reduced to [0, 1) in FP32 (exact below 2^24)
// and its sine and cosine taken in FP32; sums in FP64.
__global__ void __launch_bounds__(kDtnThreads) k_dtn_modes(const float* __restrict__ s, const float* __restrict__ len,
                                                           const float* __restrict__ u,
                                                           const int32_t* __restrict__ off, int kmax,
                                                           double2* __restrict__ uhat, double* __restrict__ lam) {
  __shared__ double red[kDtnThreads / 32];
  const int k = blockIdx.x + 1, q = blockIdx.y;
  const int j0 = off[q], j1 = off[q + 1];
  double L = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads) L += (double)len[j];
  L = block_sum(L, red);
  double re = 0.0, im = 0.0;
  if (L > 0.0) {
    const float il = (float)(1.0 / L);
    for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads) {
      float ph = (float)k * (s[j] * il);
      ph -= floorf(ph);
      float sn, cs;
      sincospif(2.0f * ph, &sn, &cs);
      const double a = (double)len[j] * (double)u[j];
      re += a * cs;
      im -= a * sn;
    }
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  if (threadIdx.x == 0) {
    uhat[(size_t)q * kmax + (k - 1)] = L > 0.0 ? make_double2(re / L, im / L) : make_double2(0.0, 0.0);
    if (k == 1) lam[q] = L;
  }
}

// one warp per element: the lanes take every 32nd mode, then a shuffle sum in
// a fixed order
__global__ void k_dtn_eval(const float* __restrict__ s, const int32_t* __restrict__ off, int nseq, int64_t T,
                           int kmax, const double2* __restrict__ uhat, const double* __restrict__ lam,
                           float* __restrict__ out) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= T) return;
  int lo = 0, hi = nseq;  // the sequence q with off[q] <= j < off[q + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= j) lo = mid;
    else hi = mid;
  }
  const double L = lam[lo];
  double acc = 0.0;
  if (L > 0.0) {
    const float x = s[j] * (float)(1.0 / L);
    for (int k = 1 + lane; k <= kmax; k += 32) {
      float ph = (float)k * x;
      ph -= floorf(ph);
      float sn, cs;
      sincospif(2.0f * ph, &sn, &cs);
      const double2 c = uhat[(size_t)lo * kmax + (k - 1)];
      acc += (double)k * (c.x * (double)cs - c.y * (double)sn);
    }
    acc *= 4.0 * 3.14159265358979323846 / L;  // the multiplier 2 pi k / Lambda, times 2 for Re
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[j] = (float)acc;
}

// out[t][2f] = sin(2 pi B_f . p_t), out[t][2f + 1] = cos(2 pi B_f . p_t); FP64
// dot product reduced to [0, 1) before the sine and cosine (FP32 results)
__global__ void k_fourier_features(const float* __restrict__ pts, int64_t T, const float* __restrict__ B, int F,
                                   float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * F) return;
  const int64_t t = i / F;
  const int f = (int)(i - t * F);
  double ph = (double)B[3 * f] * pts[3 * t] + (double)B[3 * f + 1] * pts[3 * t + 1] + (double)B[3 * f + 2] * pts[3 * t + 2];
  ph -= floor(ph);
  double sn, cs;
  sincospi(2.0 * ph, &sn, &cs);
  out[t * 2 * F + 2 * f] = (float)sn;
  out[t * 2 * F + 2 * f + 1] = (float)cs;
}

// root mean square of u over the sequence's elements, 1 when it is zero (the
// scale of the guess's inputs and outputs)
__device__ __forceinline__ double seq_rms(const float* __restrict__ u, int j0, int j1, double* red) {
  double s = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads) s += (double)u[j] * (double)u[j];
  s = block_sum(s, red);
  const double r = j1 > j0 ? sqrt(s / (double)(j1 - j0)) : 0.0;
  return r > 0.0 ? r : 1.0;
}

// block q: feats[j] = (geo[j][0..G), u_j / sc, radius qd_j / sc), sc the rms of u
__global__ void __launch_bounds__(kDtnThreads) k_guess_features(const float* __restrict__ geo, int G,
                                                                const float* __restrict__ u,
                                                                const float* __restrict__ qd,
                                                                const int32_t* __restrict__ off, float radius,
                                                                float* __restrict__ feats) {
  __shared__ double red[kDtnThreads / 32];
  const int q = blockIdx.x, j0 = off[q], j1 = off[q + 1];
  const double sc = seq_rms(u, j0, j1, red);
  const int C = G + 2;
  for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads) {
    for (int c = 0; c < G; ++c) feats[(size_t)j * C + c] = geo[(size_t)j * G + c];
    feats[(size_t)j * C + G] = (float)((double)u[j] / sc);
    feats[(size_t)j * C + G + 1] = (float)((double)radius * (double)qd[j] / sc);
  }
}

// block q: x_j = qd_j + cscale sc corr_j, out_j = x_j - sum(len x) / sum(len)
__global__ void __launch_bounds__(kDtnThreads) k_guess_finish(const float* __restrict__ qd,
                                                              const float* __restrict__ corr,
                                                              const float* __restrict__ u,
                                                              const float* __restrict__ len,
                                                              const int32_t* __restrict__ off, float cscale,
                                                              float* __restrict__ out) {
  __shared__ double red[kDtnThreads / 32];
  const int q = blockIdx.x, j0 = off[q], j1 = off[q + 1];
  const double f = (double)cscale * seq_rms(u, j0, j1, red);
  double sl = 0.0, sx = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads) {
    const double x = (double)qd[j] + f * (double)corr[j];
    sl += (double)len[j];
    sx += (double)len[j] * x;
  }
  sl = block_sum(sl, red);
  sx = block_sum(sx, red);
  const double mean = sl > 0.0 ? sx / sl : 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += kDtnThreads)
    out[j] = (float)((double)qd[j] + f * (double)corr[j] - mean);
}

}  // namespace
}  // namespace bemfft

using namespace bemfft;

extern "C" bem_status bem_guess_features(const float* geo, int G, const float* u, const float* qd,
                                         const int32_t* offsets, int nseq, int64_t T, float radius, float* feats,
                                         void* stream) {
  if (!geo || !u || !qd || !offsets || !feats || G < 0 || G > 64 || nseq < 1 || T < 1) {
    set_error("bem_guess_features: null pointer, or G, nseq, T out of range");
    return BEM_ERR_ARG;
  }
  k_guess_features<<<nseq, kDtnThreads, 0, static_cast<cudaStream_t>(stream)>>>(geo, G, u, qd, offsets, radius,
                                                                               feats);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

extern "C" bem_status bem_guess_finish(const float* qd, const float* corr, const float* u, const float* len,
                                       const int32_t* offsets, int nseq, int64_t T, float cscale, float* out,
                                       void* stream) {
  if (!qd || !corr || !u || !len || !offsets || !out || nseq < 1 || T < 1) {
    set_error("bem_guess_finish: null pointer, or nseq, T out of range");
    return BEM_ERR_ARG;
  }
  k_guess_finish<<<nseq, kDtnThreads, 0, static_cast<cudaStream_t>(stream)>>>(qd, corr, u, len, offsets, cscale,
                                                                             out);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

extern "C" bem_status bem_fourier_features(const float* points, int64_t T, const float* B, int F, float* out,
                                           void* stream) {
  if (!points || !B || !out || T < 1 || F < 1 || F > 4096) {
    set_error("bem_fourier_features: null pointer, T < 1 or F outside [1, 4096]");
    return BEM_ERR_ARG;
  }
  const int64_t total = T * (int64_t)F;
  k_fourier_features<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(points, T, B, F,
                                                                                                     out);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

extern "C" bem_status bem_dtn_estimate(const float* s, const float* len, const float* u, const int32_t* offsets,
                                       int nseq, int64_t T, int kmax, float* out, void* stream) {
  if (!s || !len || !u || !offsets || !out || nseq < 1 || T < 1 || kmax < 1 || kmax > 65535) {
    set_error("bem_dtn_estimate: null pointer, or nseq, T, kmax out of range");
    return BEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* buf = nullptr;
  const size_t bytes = (size_t)nseq * kmax * sizeof(double2) + (size_t)nseq * sizeof(double);
  BEM_CUDA_TRY(cudaMallocAsync(&buf, bytes, st));
  double2* uhat = static_cast<double2*>(buf);
  double* lam = reinterpret_cast<double*>(uhat + (size_t)nseq * kmax);
  k_dtn_modes<<<dim3(kmax, nseq), kDtnThreads, 0, st>>>(s, len, u, offsets, kmax, uhat, lam);
  k_dtn_eval<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(s, offsets, nseq, T, kmax, uhat, lam, out);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) {
    set_error(std::string("bem_dtn_estimate: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  return BEM_OK;
}
