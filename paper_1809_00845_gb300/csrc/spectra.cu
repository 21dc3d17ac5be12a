// Kernel tables on the padded grid and their FP64 spectra (Section 4, Fig. 5,
// Eq. 16), computed once per plan on the device.
//
// Table entry at offset delta (delta_a in [-n, n-1], wrapped onto [0, N)):
//   * delta = 0: the kernel's average over the h-cell ("constant elements"):
//       2D U: -(ln h + L2)/(2 pi), L2 = pi/4 - 3/2 - ln(2)/2;  odd kernels: 0;
//   * delta_a = -n on an axis in which the kernel is odd: 0 (that offset never
//     links two cells of the unpadded n-grid, and zero keeps the table exactly
//     odd so its spectrum is exactly imaginary);
//   * otherwise the point value at d = delta h.
// Because every target-source offset of the n-grid lies in [-(n-1), n-1],
// circular convolution on N = 2n equals the linear sum of the direct
// operator at every boundary cell.
//
// The tables are transformed with this library's own FP64 Stockham FFT (one
// line per CTA, all axes in turn), then compressed by parity: for kernels
// even in every axis the spectrum is real and even, for kernels odd in one
// axis it is imaginary and odd in that axis.  Only k_a in [0, n] is kept, as
// S = Re or Im of K^ divided by N^dim (the inverse transform's normalisation
// folded in), rounded once to the plan precision.
#include <cmath>
#include <vector>

#include "bem_internal.h"
#include "fft_reg.cuh"

namespace bemfft {

enum TableKind2D { T2_U = 0, T2_QX = 1, T2_QY = 2 };

__global__ void k_fill2d(cplx<double>* __restrict__ buf, int n, int N, double h, int kind, double u0) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int ix = (int)(idx % N), iy = (int)(idx / N);
  const int dx = ix < n ? ix : ix - N, dy = iy < n ? iy : iy - N;
  const double PI = 3.14159265358979323846;
  double v;
  if (dx == 0 && dy == 0) {
    v = (kind == T2_U) ? u0 : 0.0;
  } else if ((kind == T2_QX && dx == -n) || (kind == T2_QY && dy == -n)) {
    v = 0.0;
  } else {
    const double r2 = (double)dx * dx + (double)dy * dy;  // in units of h^2
    if (kind == T2_U)
      v = -(0.5 * log(r2) + log(h)) / (2.0 * PI);
    else {
      const double da = (kind == T2_QX) ? (double)dx : (double)dy;
      v = -da / (2.0 * PI * h * r2);
    }
  }
  buf[idx] = {v, 0.0};
}

// One line per CTA: load (strided), forward FFT, store.
template <int E>
__global__ void __launch_bounds__(512) k_fft_lines(cplx<double>* data, int log2N, int64_t elem_stride,
                                                   int64_t line_stride0, int64_t lines0, int64_t line_stride1,
                                                   const cplx<double>* qtab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << log2N, t = threadIdx.x, TT = blockDim.x;
  cplx<double>* sbuf = reinterpret_cast<cplx<double>*>(smem_raw);
  cplx<double>* sq = sbuf + (N + (N >> 4));
  for (int i = t; i < (N >> 2); i += TT) sq[i] = qtab[i];
  __syncthreads();
  const Twiddles<double> tw{sq, log2N - 2};
  const int64_t line = blockIdx.x;
  cplx<double>* L = data + (line % lines0) * line_stride0 + (line / lines0) * line_stride1;
  cplx<double> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = L[(int64_t)(t + m * TT) * elem_stride];
  fft_line<E, -1>(v, t, TT, log2N, tw, sbuf);
#pragma unroll
  for (int m = 0; m < E; ++m) L[(int64_t)(t + m * TT) * elem_stride] = v[m];
}

template <typename T>
__global__ void k_compress2d(const cplx<double>* __restrict__ buf, int n, int N, int imag, double scale,
                             T* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t m = (int64_t)(n + 1);
  if (idx >= m * m) return;
  const int kx = (int)(idx / m), ky = (int)(idx % m);
  const cplx<double> z = buf[(int64_t)ky * N + kx];
  out[idx] = (T)((imag ? z.y : z.x) * scale);
}

static bem_status fft_all_lines_2d(cplx<double>* buf, int log2N, const cplx<double>* qtab, cudaStream_t st) {
  const int N = 1 << log2N;
  const int E = log2N >= 8 ? 16 : 8;
  const int threads = N / E;
  const size_t smem = (size_t)(N + N / 16 + N / 4) * sizeof(cplx<double>);
  auto run = [&](auto kern) -> bem_status {
    BEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // rows (x lines): element stride 1, line stride N
    kern<<<N, threads, smem, st>>>(buf, log2N, 1, N, N, 0, qtab);
    // columns (y lines): element stride N, line stride 1
    kern<<<N, threads, smem, st>>>(buf, log2N, N, 1, N, 0, qtab);
    BEM_CUDA_TRY(cudaGetLastError());
    return BEM_OK;
  };
  return E == 16 ? run(k_fft_lines<16>) : run(k_fft_lines<8>);
}

bem_status compute_spectra_2d(bem_plan_s* p, cudaStream_t st) {
  const int n = (int)p->n, N = (int)p->N;
  const double PI = 3.14159265358979323846;
  const double L2 = PI / 4.0 - 1.5 - 0.5 * std::log(2.0);
  const double u0 = -(std::log(p->h) + L2) / (2.0 * PI);

  // FP64 quarter-wave twiddles for the plan-time transforms
  std::vector<cplx<double>> q64(N / 4);
  for (int r = 0; r < N / 4; ++r) q64[r] = {std::cos(2.0 * PI * r / N), std::sin(2.0 * PI * r / N)};
  cplx<double>* d_q64 = nullptr;
  cplx<double>* buf = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&d_q64, q64.size() * sizeof(cplx<double>)));
  BEM_CUDA_TRY(cudaMemcpyAsync(d_q64, q64.data(), q64.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMalloc(&buf, (size_t)N * N * sizeof(cplx<double>)));

  const size_t tb = prec_bytes(p);
  const int64_t m = (int64_t)(n + 1) * (n + 1);
  const double scale = 1.0 / ((double)N * (double)N);
  struct K {
    int kind, imag, oddx, oddy;
  } kinds[3] = {{T2_U, 0, 0, 0}, {T2_QX, 1, 1, 0}, {T2_QY, 1, 0, 1}};
  p->spectra.clear();
  bem_status rc = BEM_OK;
  for (const K& k : kinds) {
    const int64_t total = (int64_t)N * N;
    k_fill2d<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(buf, n, N, p->h, k.kind, u0);
    rc = fft_all_lines_2d(buf, p->log2N, d_q64, st);
    if (rc != BEM_OK) break;
    Spectrum s;
    s.imag = k.imag;
    s.odd[0] = k.oddx;
    s.odd[1] = k.oddy;
    if (cudaMalloc(&s.data, (size_t)m * tb) != cudaSuccess) {
      set_error("out of device memory for spectra");
      rc = BEM_ERR_OOM;
      break;
    }
    if (p->prec == BEM_F64)
      k_compress2d<double><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(buf, n, N, k.imag, scale,
                                                                       static_cast<double*>(s.data));
    else
      k_compress2d<float><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(buf, n, N, k.imag, scale,
                                                                      static_cast<float*>(s.data));
    p->spectra.push_back(s);
    p->spectra_bytes += (size_t)m * tb;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(d_q64);
  if (rc != BEM_OK) return rc;
  if (e != cudaSuccess) {
    set_error(std::string("spectra: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  return BEM_OK;
}

}  // namespace bemfft
