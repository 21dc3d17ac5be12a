// 3D operator apply (3D Laplace, Kelvin): the boundary surface lies in an
// n^3 grid padded to N^3, N = 2n (Section 3: "convolution over the entire
// volume enclosing this surface"; Eq. 7-8, Eq. 15-16).
//
// Pipeline per apply (every field f = one scattered density, every output o
// = one component of the result; the operator couples them through kernel
// spectra K_of):
//   k3_prep   val_f[j]      = coef_f[j] * in[perm[j]*ncomp + comp_f]
//   k3_yfwd   B_f[kx][ky][z] = FFT_y of the grid lines (y, z < n), each line
//             the input-pruned x-DFT sum over its cells of
//             val_f e^{-2 pi i kx x / N}, formed in registers (fft3d.cuh)
//   k3_zpass  per (kx, ky): FFT_z of every B_f, multiply-accumulate
//             Y_o = sum_f K_of * B_f, inverse FFT_z, B_o <- Y_o (z < n)
//   k3_yinv   X_o[kx][z][y] = IFFT_y(B_o[kx][:][z])       (y < n kept)
//   k3_gather out[j, o] = sum_kx c_kx Re(X_o[kx][z_j][y_j] e^{2 pi i kx x_j/N})
//             (+ diagonal term)  - output-pruned inverse x-DFT = the gather.
// The N^3 grid never exists: the largest buffers hold (n+1) x N x n complex
// values per field.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "bem_internal.h"
#include "fft3d.h"
#include "fft_reg.cuh"

namespace bemfft {

// e^{DIR 2 pi i m / N}, m = 64 hi + lo
template <typename T>
struct Tw2 {
  const cplx<T>* hi;
  const cplx<T>* lo;
  template <int DIR>
  __device__ __forceinline__ cplx<T> get(int m) const {
    cplx<T> z = cmul(hi[m >> 6], lo[m & 63]);
    if constexpr (DIR < 0) z.y = -z.y;
    return z;
  }
};

// ------------------------------------------------------------------ kernels

// T: arithmetic type of the passes; TIO: type of the caller's vectors (FP64
// for double-float plans, else T)
template <typename T, typename TIO>
__global__ void k3_prep(int nb, int ncomp, const int32_t* __restrict__ perm, const TIO* __restrict__ in,
                        const Field3D* __restrict__ fields, T* __restrict__ val) {
  const int f = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const Field3D fd = fields[f];
  val[(size_t)f * nb + j] = static_cast<const T*>(fd.coef)[j] * T(in[(size_t)perm[j] * ncomp + fd.comp]);
}

// out[perm[j]*ncomp + o] = sum_kx c_kx Re(X_o[kx][z][y] e^{+2 pi i kx x/N}) + diag * in
template <typename T, typename TIO>
__global__ void k3_gather(int n, int log2N, int nb, int ncomp, const int32_t* __restrict__ perm,
                          const uint16_t* __restrict__ xs, const uint32_t* __restrict__ yz,
                          const cplx<T>* __restrict__ X, const cplx<T>* __restrict__ tw2,
                          const TIO* __restrict__ diag, const TIO* __restrict__ in, TIO* __restrict__ out) {
  __shared__ cplx<T> stw[2048 / 64 + 64 + 64];
  const int N = 1 << log2N;
  const int nhi = N >= 64 ? N >> 6 : 1;
  for (int i = threadIdx.x; i < nhi + 64; i += blockDim.x) stw[i] = tw2[i];
  __syncthreads();
  const Tw2<T> tw{stw, stw + nhi};
  const int o = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int x = xs[j];
  const uint32_t p = yz[j];
  const int y = (int)(p & 0xffffu), z = (int)(p >> 16);
  const int64_t plane = (int64_t)n * n;
  const cplx<T>* src = X + (size_t)o * (n + 1) * plane + (size_t)z * n + y;
  // compensated FP32 sum (FP64 and double-float plans: plain sum)
  T s = T(0), comp = T(0);
  for (int kx = 0; kx <= n; ++kx) {
    const cplx<T> Y = src[(size_t)kx * plane];
    const cplx<T> w = tw.template get<+1>((kx * x) & (N - 1));
    const T ck = (kx == 0 || kx == n) ? T(1) : T(2);
    if constexpr (std::is_same<T, float>::value) {
      const T term = ck * cdot_re(Y, w) - comp;
      const T ns = s + term;
      comp = (ns - s) - term;
      s = ns;
    } else {
      s = s + ck * cdot_re(Y, w);
    }
  }
  const int u = perm[j];
  const size_t oi = (size_t)u * ncomp + o;
  double r = (double)s;
  if (diag) r += (double)diag[oi] * (double)in[oi];
  out[oi] = (TIO)r;
}

// ------------------------------------------------------------------ host

size_t buffers3d_bytes(const bem_plan_s* p, int nf) {
  const size_t tb = 2 * prec_bytes(p);
  const int64_t n = p->n, N = p->N;
  return (size_t)nf * (n + 1) * n * n * tb + (size_t)nf * (n + 1) * N * n * tb;
}

// the line-FFT passes instantiated for this plan's grid size
template <typename T>
struct Passes3D {
  const bem_plan_s* p;
  template <int L>
  using K = Fft3DKernels<T, L>;
  template <class F>
  auto on(F&& f) const {
    switch (p->log2N) {
      case 5: return f(K<5>());
      case 6: return f(K<6>());
      case 7: return f(K<7>());
      case 8: return f(K<8>());
      case 9: return f(K<9>());
      default: return f(K<10>());
    }
  }
};

template <typename T, typename TIO = T>
static bem_status launch3d_t(bem_plan_s* p, const Operator3D& op, const void* in, void* out, void* val, void* X,
                             void* B, bool timed, cudaStream_t st) {
  const int n = (int)p->n, nb = (int)p->nb;
  const int tb = 256;
  k3_prep<T, TIO><<<dim3((nb + tb - 1) / tb, op.nf), tb, 0, st>>>(nb, p->ncomp, p->d_perm,
                                                                   static_cast<const TIO*>(in), op.d_fields,
                                                                   static_cast<T*>(val));
  cudaEvent_t e1 = nullptr;
  if (timed) {
    if (p->ev_used + 2 > (int)p->ev_pool.size())
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        BEM_CUDA_TRY(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
      }
    cudaEvent_t e0 = p->ev_pool[p->ev_used++];
    e1 = p->ev_pool[p->ev_used++];
    BEM_CUDA_TRY(cudaEventRecord(e0, st));
  }
  Passes3D<T>{p}.on([&](auto k) {
    using KK = decltype(k);
    KK::yfwd(op.nf, nb, p->d_lptr, p->d_x3, val, p->d_tw2, B, p->d_ptab3, st);
    KK::zpass(op.nf, op.no, zpass_lpc(p, op.nf), op.d_coup, p->d_specs3, B, p->d_ptab3, st);
    KK::yinv(op.no, B, X, p->d_ptab3, st);
    return 0;
  });
  if (timed) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k3_gather<T, TIO><<<dim3((nb + tb - 1) / tb, op.no), tb, 0, st>>>(
      n, p->log2N, nb, p->ncomp, p->d_perm, p->d_x3, p->d_yz3, static_cast<const cplx<T>*>(X),
      static_cast<const cplx<T>*>(p->d_tw2), static_cast<const TIO*>(op.diag), static_cast<const TIO*>(in),
      static_cast<TIO*>(out));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

template <typename T>
static bem_status configure3d_t(bem_plan_s* p) {
  int dev = 0, optin = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t sm_y = Passes3D<T>{p}.on([](auto k) { return decltype(k)::smem_y(); });
  if (sm_y > (size_t)optin) {
    set_error("3D grid too large for the shared-memory line buffers");
    return BEM_ERR_UNSUPPORTED;
  }
  BEM_CUDA_TRY(Passes3D<T>{p}.on([](auto k) { return decltype(k)::configure(); }));
  return BEM_OK;
}

// lines per CTA of the z pass: four (or the plan's tuned count,
// bem_tune_shapes), fewer where their buffers would pass ~200 KB of shared
// memory or the CTA 512 threads
int zpass_lpc(const bem_plan_s* p, int nf) {
  const size_t cb = 2 * prec_bytes(p);
  const int64_t N = p->N;
  const size_t per = ((size_t)(N + N / 16) + (size_t)nf * N) * cb;
  const size_t budget = 200 * 1024 - (size_t)(N / 4) * cb;
  // four lines per CTA (128 threads at N = 512): the z pass holds 106
  // registers a thread, so small CTAs let several reside per SM and one CTA's
  // loads overlap another's transforms (measured: 16 lines 0.629 ms, 8 lines
  // 0.601 ms, 4 lines 0.588 ms per 256^3 ellipsoid single-layer apply)
  int lpc = p->zpass_lines > 0 ? p->zpass_lines : 4;
  while (lpc > 1 && (size_t)lpc * per > budget) lpc >>= 1;
  while (lpc > 1 && (lpc * (N / 16)) > 512) lpc >>= 1;
  return lpc;
}

// complex table (FP64 values) in the plan's arithmetic type, rounded once
template <typename T>
static bem_status upload_table3_t(const std::vector<double>& re, const std::vector<double>& im, void** dst) {
  std::vector<cplx<T>> t(re.size());
  for (size_t i = 0; i < re.size(); ++i) t[i] = {T(re[i]), T(im[i])};
  BEM_CUDA_TRY(cudaMalloc(dst, t.size() * sizeof(t[0])));
  BEM_CUDA_TRY(cudaMemcpy(*dst, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice));
  return BEM_OK;
}

static bem_status upload_table3(const bem_plan_s* p, const std::vector<double>& re, const std::vector<double>& im,
                                void** dst) {
  if (p->prec == BEM_F64) return upload_table3_t<double>(re, im, dst);
  if (p->prec == BEM_F32X2) return upload_table3_t<f32x2>(re, im, dst);
  return upload_table3_t<float>(re, im, dst);
}

bem_status setup_apply_3d(bem_plan_s* p, int maxnf) {
  if (p->log2N < 5 || p->log2N > 10) {
    set_error("3D grids need 16 <= n <= 512, n a power of two");
    return BEM_ERR_UNSUPPORTED;
  }
  bem_status rc = p->prec == BEM_F64     ? configure3d_t<double>(p)
                  : p->prec == BEM_F32X2 ? configure3d_t<f32x2>(p)
                                         : configure3d_t<float>(p);
  if (rc != BEM_OK) return rc;
  // 2-level twiddles e^{2 pi i m / N}
  const int64_t N = p->N;
  const double PI = 3.14159265358979323846;
  std::vector<double> re, im;
  for (int64_t i = 0; i < std::max<int64_t>(1, N / 64); ++i) {
    re.push_back(std::cos(2 * PI * 64.0 * i / N));
    im.push_back(std::sin(2 * PI * 64.0 * i / N));
  }
  for (int i = 0; i < 64; ++i) {
    re.push_back(std::cos(2 * PI * i / (double)N));
    im.push_back(std::sin(2 * PI * i / (double)N));
  }
  // Stockham pass twiddles of the line FFTs: pass q >= 1 (Ns = 16^q, radix R)
  // holds e^{2 pi i k r / (Ns R)} at off(q) + r Ns + k
  {
    std::vector<double> pre, pim;
    const int npass = (p->log2N + 3) / 4;
    for (int q = 1; q < npass; ++q) {
      const int left = p->log2N - 4 * q;
      const int64_t R = left > 4 ? 16 : (1 << left), Ns = (int64_t)1 << (4 * q);
      for (int64_t r = 0; r < R; ++r)
        for (int64_t k = 0; k < Ns; ++k) {
          pre.push_back(std::cos(2 * PI * (double)(k * r) / (double)(Ns * R)));
          pim.push_back(std::sin(2 * PI * (double)(k * r) / (double)(Ns * R)));
        }
    }
    pre.resize(std::max<size_t>(pre.size(), 1), 0.0);
    pim.resize(pre.size(), 0.0);
    if ((rc = upload_table3(p, pre, pim, &p->d_ptab3)) != BEM_OK) return rc;
  }
  if ((rc = upload_table3(p, re, im, &p->d_tw2)) != BEM_OK) return rc;
  // buffers sized for the widest operator
  const size_t tb = prec_bytes(p);
  BEM_CUDA_TRY(cudaMalloc(&p->d_val3, (size_t)maxnf * p->nb * tb));
  const size_t xb = (size_t)maxnf * (p->n + 1) * p->n * p->n * 2 * tb;
  const size_t bb = (size_t)maxnf * (p->n + 1) * p->N * p->n * 2 * tb;
  BEM_CUDA_TRY(cudaMalloc(&p->d_X3, xb));
  BEM_CUDA_TRY(cudaMalloc(&p->d_B3, bb));
  p->scratch_bytes += (size_t)maxnf * p->nb * tb + xb + bb;
  p->maxnf3 = maxnf;
  p->threads = (int)(p->N / 16);
  p->grid = (int)(p->n + 1);
  return BEM_OK;
}

bem_status launch_apply_3d(bem_plan_s* p, const Operator3D& op, const void* in, void* out, void* val, void* X, void* B,
                           cudaStream_t st) {
  if (op.nf < 1 || op.nf > p->maxnf3) {
    set_error("3D operator wider than the plan's buffers");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->prec == BEM_F64) return launch3d_t<double>(p, op, in, out, val, X, B, p->timing, st);
  if (p->prec == BEM_F32X2) return launch3d_t<f32x2, double>(p, op, in, out, val, X, B, p->timing, st);
  return launch3d_t<float>(p, op, in, out, val, X, B, p->timing, st);
}

}  // namespace bemfft
