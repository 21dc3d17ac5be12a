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
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
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
    else if (p->prec == BEM_F32X2)
      k_compress2d<f32x2><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(buf, n, N, k.imag, scale,
                                                                      static_cast<f32x2*>(s.data));
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

namespace bemfft {

// ------------------------------------------------------------------ 3D tables
//
// family 0: 3D Laplace U = 1/(4 pi r)          (cell average C3/(4 pi h) at 0)
// family 1: Q_a = -d_a/(4 pi r^3)               (gradient of U, odd in a)
// family 2: Kelvin U_ab of Eq. 7                (cell average at 0, see below)
// family 3: G_abc, the traction kernel of Eq. 8 written linear in the normal:
//           T_ab(d; n) = sum_c G_abc(d) n_c with
//           G_abc = [(1-2nu)(delta_ab d_c + delta_ac d_b - delta_bc d_a)/r^3
//                    + 3 d_a d_b d_c / r^5] / (8 pi (1-nu)),   0 at d = 0.
// d = delta h is the collocation minus integration point offset.
struct Kind3 {
  int family, a, b, c;
  double nu, mu, h, u0;
};

__device__ __forceinline__ int odd_mask3(const Kind3& k) {
  if (k.family == 0) return 0;
  if (k.family == 1) return 1 << k.a;
  if (k.family == 2) return k.a == k.b ? 0 : ((1 << k.a) | (1 << k.b));
  return (1 << k.a) ^ (1 << k.b) ^ (1 << k.c);
}

__global__ void k_fill3d(cplx<double>* __restrict__ buf, int n, int N, Kind3 k) {
  const int64_t total = (int64_t)N * N * N;
  const double PI = 3.14159265358979323846;
  const int om = odd_mask3(k);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % N), iy = (int)((idx / N) % N), iz = (int)(idx / ((int64_t)N * N));
    const int dl[3] = {ix < n ? ix : ix - N, iy < n ? iy : iy - N, iz < n ? iz : iz - N};
    double v = 0.0;
    bool zero = false;
    for (int a = 0; a < 3; ++a)
      if (((om >> a) & 1) && dl[a] == -n) zero = true;
    if (dl[0] == 0 && dl[1] == 0 && dl[2] == 0) {
      v = k.u0;  // cell average (0 for the odd families)
    } else if (!zero) {
      const double d[3] = {dl[0] * k.h, dl[1] * k.h, dl[2] * k.h};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const double r = sqrt(r2), r3 = r2 * r;
      if (k.family == 0) {
        v = 1.0 / (4.0 * PI * r);
      } else if (k.family == 1) {
        v = -d[k.a] / (4.0 * PI * r3);
      } else if (k.family == 2) {
        v = (((k.a == k.b) ? (3.0 - 4.0 * k.nu) / r : 0.0) + d[k.a] * d[k.b] / r3) /
            (16.0 * PI * k.mu * (1.0 - k.nu));
      } else {
        const double c1 = 1.0 - 2.0 * k.nu;
        const double lin = (k.a == k.b ? d[k.c] : 0.0) + (k.a == k.c ? d[k.b] : 0.0) - (k.b == k.c ? d[k.a] : 0.0);
        v = (c1 * lin / r3 + 3.0 * d[k.a] * d[k.b] * d[k.c] / (r3 * r2)) / (8.0 * PI * (1.0 - k.nu));
      }
    }
    buf[idx] = {v, 0.0};
  }
}

// S[kx][ky][kz] = Re(K^[kz][ky][kx] * i^-q) / N^3 for k_a in [0, n]
template <typename T>
__global__ void k_compress3d(const cplx<double>* __restrict__ buf, int n, int N, int q, double scale,
                             T* __restrict__ out) {
  const int64_t m = n + 1;
  const int64_t total = m * m * m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int kz = (int)(idx % m), ky = (int)((idx / m) % m), kx = (int)(idx / (m * m));
    const cplx<double> z = buf[((int64_t)kz * N + ky) * N + kx];
    double s;
    switch (q & 3) {
      case 0: s = z.x; break;
      case 1: s = z.y; break;
      case 2: s = -z.x; break;
      default: s = -z.y; break;
    }
    out[idx] = (T)(s * scale);
  }
}

int kelvin_u_index(int a, int b) {
  if (a > b) std::swap(a, b);
  // (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

bem_status compute_spectra_3d(bem_plan_s* p, cudaStream_t st) {
  const int n = (int)p->n, N = (int)p->N;
  const double PI = 3.14159265358979323846;
  const double C3 = 3.0 * std::log(2.0 + std::sqrt(3.0)) - PI / 2.0;
  std::vector<Kind3> kinds;
  if (p->kernel == BEM_LAPLACE_3D) {
    kinds.push_back({0, 0, 0, 0, p->nu, p->mu, p->h, C3 / (4.0 * PI * p->h)});
    for (int a = 0; a < 3; ++a) kinds.push_back({1, a, 0, 0, p->nu, p->mu, p->h, 0.0});
  } else {
    const double nu = p->nu, mu = p->mu;
    const double ud = (3.0 - 4.0 * nu + 1.0 / 3.0) * C3 / (16.0 * PI * mu * (1.0 - nu) * p->h);
    const int pairs[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (auto& ab : pairs) kinds.push_back({2, ab[0], ab[1], 0, nu, mu, p->h, ab[0] == ab[1] ? ud : 0.0});
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) kinds.push_back({3, a, b, c, nu, mu, p->h, 0.0});
  }
  std::vector<cplx<double>> q64(N / 4);
  for (int r = 0; r < N / 4; ++r) q64[r] = {std::cos(2.0 * PI * r / N), std::sin(2.0 * PI * r / N)};
  cplx<double>* d_q64 = nullptr;
  cplx<double>* buf = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&d_q64, q64.size() * sizeof(cplx<double>)));
  BEM_CUDA_TRY(cudaMemcpy(d_q64, q64.data(), q64.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice));
  const int64_t NN = (int64_t)N * N;
  if (cudaMalloc(&buf, (size_t)NN * N * sizeof(cplx<double>)) != cudaSuccess) {
    cudaFree(d_q64);
    set_error("out of device memory for the 3D kernel tables");
    return BEM_ERR_OOM;
  }
  const int E = p->log2N >= 8 ? 16 : 8;
  const int threads = N / E;
  const size_t smem = (size_t)(N + N / 16 + N / 4) * sizeof(cplx<double>);
  auto kern = E == 16 ? k_fft_lines<16> : k_fft_lines<8>;
  BEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const size_t tb = prec_bytes(p);
  const int64_t m3 = (int64_t)(n + 1) * (n + 1) * (n + 1);
  const double scale = 1.0 / ((double)N * N * N);
  bem_status rc = BEM_OK;
  p->h_specs3.clear();
  for (const Kind3& k : kinds) {
    k_fill3d<<<152 * 16, 256, 0, st>>>(buf, n, N, k);
    // x lines (stride 1), y lines (stride N), z lines (stride N^2)
    kern<<<(unsigned)NN, threads, smem, st>>>(buf, p->log2N, 1, N, NN, 0, d_q64);
    kern<<<(unsigned)NN, threads, smem, st>>>(buf, p->log2N, N, 1, N, NN, d_q64);
    kern<<<(unsigned)NN, threads, smem, st>>>(buf, p->log2N, NN, 1, NN, 0, d_q64);
    int om = 0;
    if (k.family == 1) om = 1 << k.a;
    else if (k.family == 2) om = k.a == k.b ? 0 : ((1 << k.a) | (1 << k.b));
    else if (k.family == 3) om = (1 << k.a) ^ (1 << k.b) ^ (1 << k.c);
    const int q = ((om & 1) ? 1 : 0) + ((om & 2) ? 1 : 0) + ((om & 4) ? 1 : 0);
    Spec3D sp{};
    void* d = nullptr;
    if (cudaMalloc(&d, (size_t)m3 * tb) != cudaSuccess) {
      set_error("out of device memory for the 3D spectra");
      rc = BEM_ERR_OOM;
      break;
    }
    if (p->prec == BEM_F64)
      k_compress3d<double><<<152 * 16, 256, 0, st>>>(buf, n, N, q, scale, static_cast<double*>(d));
    else if (p->prec == BEM_F32X2)
      k_compress3d<f32x2><<<152 * 16, 256, 0, st>>>(buf, n, N, q, scale, static_cast<f32x2*>(d));
    else
      k_compress3d<float><<<152 * 16, 256, 0, st>>>(buf, n, N, q, scale, static_cast<float*>(d));
    sp.data = d;
    sp.q = q;
    sp.oddy = (om >> 1) & 1;
    sp.oddz = (om >> 2) & 1;
    p->h_specs3.push_back(sp);
    p->spectra_bytes += (size_t)m3 * tb;
    if (cudaGetLastError() != cudaSuccess) {
      set_error("3D spectrum kernels failed to launch");
      rc = BEM_ERR_CUDA;
      break;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(d_q64);
  if (rc != BEM_OK) return rc;
  if (e != cudaSuccess) {
    set_error(std::string("3D spectra: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  BEM_CUDA_TRY(cudaMalloc(&p->d_specs3, p->h_specs3.size() * sizeof(Spec3D)));
  BEM_CUDA_TRY(cudaMemcpy(p->d_specs3, p->h_specs3.data(), p->h_specs3.size() * sizeof(Spec3D),
                          cudaMemcpyHostToDevice));
  return BEM_OK;
}

}  // namespace bemfft
