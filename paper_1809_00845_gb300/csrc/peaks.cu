// bem_measure_peak: the arithmetic peaks this library's rooflines are quoted
// against, measured on the current device with a timed loop of independent
// fused multiply-adds (no clock or device setting is touched).  Not part of
// the paper's method; a measurement helper for the FP32 and FP64 ALU rooflines
// of the column kernels.
#include <cuda_runtime.h>

#include <string>

#include "bem_internal.h"

namespace bemfft {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// x <- x * a + b on kChains independent chains; `sink` is written only when
// the (never true) test on the results holds, so nothing is optimised away
template <typename T>
__global__ void __launch_bounds__(512) k_fma_loop(T a, T b, int iters, int* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) atomicAdd(sink, 1);
}

// the same with packed FP32 pairs (two FMAs per instruction)
__global__ void __launch_bounds__(512) k_fma2_loop(float a, float b, int iters, int* sink) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)threadIdx.x + c, (float)c);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == -12345.0f) atomicAdd(sink, 1);
}

}  // namespace
}  // namespace bemfft

using namespace bemfft;

extern "C" bem_status bem_measure_peak(int kind, double* tflops, void* stream) {
  if (!tflops || kind < 0 || kind > 2) {
    set_error("bem_measure_peak: kind 0 (FP32), 1 (FP64) or 2 (packed FP32 pairs), and an output pointer");
    return BEM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  struct Res {
    int* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Res() {
      if (sink) cudaFree(sink);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } r;
  BEM_CUDA_TRY(cudaMalloc(&r.sink, sizeof(int)));
  BEM_CUDA_TRY(cudaEventCreate(&r.e0));
  BEM_CUDA_TRY(cudaEventCreate(&r.e1));
  const int threads = 512, blocks = nsm * 4;  // 64 warps per SM
  // about 0.1 s per launch at the expected rates (FP64 runs at a small
  // fraction of the FP32 rate on some parts)
  const int iters = kind == 1 ? 64 : 1024;
  auto run = [&]() {
    if (kind == 0) k_fma_loop<float><<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, iters, r.sink);
    else if (kind == 1) k_fma_loop<double><<<blocks, threads, 0, st>>>(0.999999999, 1e-12, iters, r.sink);
    else k_fma2_loop<<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, iters, r.sink);
  };
  run();  // warm-up
  BEM_CUDA_TRY(cudaGetLastError());
  const int reps = 5;
  BEM_CUDA_TRY(cudaEventRecord(r.e0, st));
  for (int i = 0; i < reps; ++i) run();
  BEM_CUDA_TRY(cudaEventRecord(r.e1, st));
  BEM_CUDA_TRY(cudaEventSynchronize(r.e1));
  float ms = 0.f;
  BEM_CUDA_TRY(cudaEventElapsedTime(&ms, r.e0, r.e1));
  const double fmas = (double)reps * blocks * threads * iters * kChains * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return BEM_OK;
}
