// 2D operator apply: sparse row transform fused with the scatter, per-column
// FFT + spectral multiply + inverse FFT in one CTA, and the gather fused into
// the inverse row transform (Section 3-4, Eq. 15-16).
//
// Layout of the padded N x N grid (N = 2n): rows are y, columns are x.  The
// scattered density rho (zero off the boundary cells, Fig. 4) has at most a
// few non-zeros per row, so its forward transform along x is evaluated
// directly from the cell list (an input-pruned DFT: O(cells) per frequency)
// instead of an FFT over a mostly-zero row; only the n+1 non-redundant
// x-frequencies of the real field are formed.  For each x-frequency kx one
// CTA then owns the full column (length N along y) in registers/shared
// memory: forward FFT along y, multiply by the compressed kernel spectrum
// column, inverse FFT along y, and the inverse transform along x evaluated
// only at the boundary cells (an output-pruned inverse DFT that also is the
// gather).  The padded grid never exists in global memory; the only large
// stream from HBM is the spectrum ((n+1)^2 reals per kernel table).
//
// Each CTA accumulates the contributions of its columns to every boundary
// cell (one owner thread per grid row, so no atomics), and a small reduction
// kernel sums the per-CTA partials in FP64 and writes the result in the
// caller's cell order.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "bem_internal.h"
#include "fft_reg.cuh"

namespace bemfft {

template <typename T>
struct Col2DParams {
  int n, log2N, nb;
  const int32_t* rowptr;  // n + 1
  const int32_t* col;     // nb
  const T* rho;           // NF * nb
  const T* spec[kMaxFields];
  int imag[kMaxFields];
  int oddy[kMaxFields];
  const cplx<T>* qtab;  // N/4
  T* partial;           // gridDim.x * nb
  int acc_in_smem;
};

template <typename T, int E>
__device__ __forceinline__ void gather_rows(const cplx<T> (&y)[E], const Col2DParams<T>& p, const int t, const int TT,
                                            const int kx, const Twiddles<T>& tw, T* acc) {
  constexpr int H = E / 2;
  const int N = 1 << p.log2N;
  const T ckx = (kx == 0 || kx == p.n) ? T(1) : T(2);
#pragma unroll
  for (int m = 0; m < H; ++m) {
    const int row = t + m * TT;
    const int j0 = __ldg(p.rowptr + row), j1 = __ldg(p.rowptr + row + 1);
    for (int j = j0; j < j1; ++j) {
      const cplx<T> w = tw.template get<+1>((kx * __ldg(p.col + j)) & (N - 1));
      acc[j] += ckx * (y[m].x * w.x - y[m].y * w.y);
    }
  }
}

template <typename T, int E, int NF, bool ACCREG>
__global__ void __launch_bounds__(512) k_col2d(const Col2DParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x, TT = blockDim.x;
  const int log2N = p.log2N, N = 1 << log2N, n = p.n, nb = p.nb;
  cplx<T>* sbuf = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* sq = sbuf + (N + (N >> 4));
  T* acc = p.acc_in_smem ? reinterpret_cast<T*>(sq + (N >> 2)) : p.partial + (size_t)blockIdx.x * nb;
  for (int i = t; i < (N >> 2); i += TT) sq[i] = p.qtab[i];
  for (int j = t; j < nb; j += TT) acc[j] = T(0);
  __syncthreads();
  const Twiddles<T> tw{sq, log2N - 2};
  constexpr int H = E / 2;

  for (int kx = blockIdx.x; kx <= n; kx += gridDim.x) {
    cplx<T> y[ACCREG ? E : 1];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      cplx<T> v[E];
      const T* rho = p.rho + (size_t)f * nb;
      // scatter fused with the input-pruned forward DFT along x
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int row = t + m * TT;
        const int j0 = __ldg(p.rowptr + row), j1 = __ldg(p.rowptr + row + 1);
        cplx<T> s = {T(0), T(0)};
        for (int j = j0; j < j1; ++j) {
          const T r = __ldg(rho + j);
          const cplx<T> w = tw.template get<-1>((kx * __ldg(p.col + j)) & (N - 1));
          s.x += r * w.x;
          s.y += r * w.y;
        }
        v[m] = s;
      }
#pragma unroll
      for (int m = H; m < E; ++m) v[m] = {T(0), T(0)};
      fft_line<E, -1>(v, t, TT, log2N, tw, sbuf);
      // spectral multiply (Eq. 16), spectrum column kx, folded in ky
      const T* S = p.spec[f] + (size_t)kx * (n + 1);
      const bool im = p.imag[f] != 0, oy = p.oddy[f] != 0;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + m * TT;
        const bool hi = ky > n;
        T sv = __ldg(S + (hi ? N - ky : ky));
        if (hi && oy) sv = -sv;
        const cplx<T> prod = im ? cplx<T>{-v[m].y * sv, v[m].x * sv} : cplx<T>{v[m].x * sv, v[m].y * sv};
        if constexpr (ACCREG) {
          if (f == 0) y[m] = prod;
          else y[m] = y[m] + prod;
        } else {
          v[m] = prod;
        }
      }
      if constexpr (!ACCREG) {
        fft_line<E, +1>(v, t, TT, log2N, tw, sbuf);
        gather_rows<T, E>(v, p, t, TT, kx, tw, acc);
      }
    }
    if constexpr (ACCREG) {
      fft_line<E, +1>(y, t, TT, log2N, tw, sbuf);
      gather_rows<T, E>(y, p, t, TT, kx, tw, acc);
    }
  }
  if (p.acc_in_smem) {
    __syncthreads();
    for (int j = t; j < nb; j += TT) p.partial[(size_t)blockIdx.x * nb + j] = acc[j];
  }
}

// rho_f[j] = coef_f[j] * in[perm[j]*ncomp + comp_f]
template <typename T>
struct PrepParams {
  int nb, ncomp, nf;
  const int32_t* perm;
  const T* in;
  const T* coef[kMaxFields];
  int comp[kMaxFields];
  T* rho;
};

template <typename T>
__global__ void k_prep(const PrepParams<T> p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.nb) return;
  const int u = p.perm[j];
  for (int f = 0; f < p.nf; ++f) p.rho[(size_t)f * p.nb + j] = p.coef[f][j] * p.in[(size_t)u * p.ncomp + p.comp[f]];
}

// out[perm[j]*ncomp + c] = sum_b partial[(b*ncomp + c)*nb + j] + diag * in
template <typename T>
__global__ void k_reduce(const T* __restrict__ partial, int grid, int nb, int ncomp, const int32_t* __restrict__ perm,
                         const T* __restrict__ diag, const T* __restrict__ in, T* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int u = perm[j];
  for (int c = 0; c < ncomp; ++c) {
    double s = 0.0;
    for (int b = 0; b < grid; ++b) s += (double)partial[((size_t)b * ncomp + c) * nb + j];
    const size_t o = (size_t)u * ncomp + c;
    if (diag) s += (double)diag[o] * (double)in[o];
    out[o] = (T)s;
  }
}

// ------------------------------------------------------------------ host side

static int elems_per_thread(int log2N) { return log2N >= 8 ? 16 : 8; }

template <typename T>
static size_t smem_2d(int64_t N, int64_t nb, bool acc) {
  size_t s = (size_t)(N + N / 16) * sizeof(cplx<T>) + (size_t)(N / 4) * sizeof(cplx<T>);
  if (acc) s += (size_t)nb * sizeof(T);
  return s;
}

template <typename T, int E, int NF, bool ACCREG>
static cudaError_t configure_one(size_t smem, int threads, int* blocks_per_sm) {
  auto kern = k_col2d<T, E, NF, ACCREG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, threads, smem);
}

template <typename T, int E>
static cudaError_t configure_all(size_t smem, int threads, int* bps) {
  constexpr bool R = std::is_same<T, float>::value;  // accumulate in registers only for FP32
  int b1 = 0, b2 = 0, b3 = 0;
  cudaError_t e;
  if ((e = configure_one<T, E, 1, false>(smem, threads, &b1)) != cudaSuccess) return e;
  if ((e = configure_one<T, E, 2, R>(smem, threads, &b2)) != cudaSuccess) return e;
  if ((e = configure_one<T, E, 3, R>(smem, threads, &b3)) != cudaSuccess) return e;
  *bps = std::min(b1, std::min(b2, b3));
  return cudaSuccess;
}

template <typename T>
static bem_status setup_t(bem_plan_s* p) {
  const int64_t N = p->N, nb = p->nb;
  const int E = elems_per_thread(p->log2N);
  p->threads = (int)(N / E);
  int dev = 0, nsm = 0, smem_optin = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  p->acc_in_smem = smem_2d<T>(N, nb, true) <= (size_t)smem_optin;
  p->smem_bytes = smem_2d<T>(N, nb, p->acc_in_smem);
  if (p->smem_bytes > (size_t)smem_optin) {
    set_error("grid too large for the shared-memory column buffer");
    return BEM_ERR_UNSUPPORTED;
  }
  int bps = 0;
  if (E == 16)
    BEM_CUDA_TRY((configure_all<T, 16>(p->smem_bytes, p->threads, &bps)));
  else
    BEM_CUDA_TRY((configure_all<T, 8>(p->smem_bytes, p->threads, &bps)));
  if (bps < 1) {
    set_error("column kernel cannot be resident (registers/shared memory)");
    return BEM_ERR_UNSUPPORTED;
  }
  p->grid = (int)std::min<int64_t>((int64_t)bps * nsm, p->n + 1);
  const size_t tb = sizeof(T);
  BEM_CUDA_TRY(cudaMalloc(&p->d_partial, (size_t)p->grid * nb * p->ncomp * tb));
  BEM_CUDA_TRY(cudaMalloc(&p->d_rho, (size_t)kMaxFields * nb * tb));
  p->scratch_bytes = (size_t)p->grid * nb * p->ncomp * tb + (size_t)kMaxFields * nb * tb;
  return BEM_OK;
}

bem_status setup_apply_2d(bem_plan_s* p) {
  if (p->log2N < 3 || p->log2N > 13) {
    set_error("2D grids need 4 <= n <= 4096, n a power of two");
    return BEM_ERR_UNSUPPORTED;
  }
  return p->prec == BEM_F64 ? setup_t<double>(p) : setup_t<float>(p);
}

template <typename T, int E, int NF, bool ACCREG>
static void launch_col(const bem_plan_s* p, const Col2DParams<T>& cp, cudaStream_t st) {
  k_col2d<T, E, NF, ACCREG><<<p->grid, p->threads, p->smem_bytes, st>>>(cp);
}

template <typename T, int E>
static void launch_col_nf(const bem_plan_s* p, int nf, const Col2DParams<T>& cp, cudaStream_t st) {
  constexpr bool R = std::is_same<T, float>::value;
  if (nf == 1) launch_col<T, E, 1, false>(p, cp, st);
  else if (nf == 2) launch_col<T, E, 2, R>(p, cp, st);
  else launch_col<T, E, 3, R>(p, cp, st);
}

template <typename T>
static bem_status launch_t(bem_plan_s* p, const Operator& op, const void* in, void* out, cudaStream_t st) {
  const int nb = (int)p->nb;
  PrepParams<T> pp{};
  pp.nb = nb;
  pp.ncomp = p->ncomp;
  pp.nf = op.nf;
  pp.perm = p->d_perm;
  pp.in = static_cast<const T*>(in);
  pp.rho = static_cast<T*>(p->d_rho);
  for (int f = 0; f < op.nf; ++f) {
    pp.coef[f] = static_cast<const T*>(op.f[f].coef);
    pp.comp[f] = op.f[f].comp;
  }
  const int tb = 256;
  k_prep<T><<<(nb + tb - 1) / tb, tb, 0, st>>>(pp);

  Col2DParams<T> cp{};
  cp.n = (int)p->n;
  cp.log2N = p->log2N;
  cp.nb = nb;
  cp.rowptr = p->d_rowptr;
  cp.col = p->d_col;
  cp.rho = static_cast<const T*>(p->d_rho);
  for (int f = 0; f < op.nf; ++f) {
    const Spectrum& s = p->spectra[op.f[f].spec];
    cp.spec[f] = static_cast<const T*>(s.data);
    cp.imag[f] = s.imag;
    cp.oddy[f] = s.odd[1];
  }
  cp.qtab = static_cast<const cplx<T>*>(p->d_qtab);
  cp.partial = static_cast<T*>(p->d_partial);
  cp.acc_in_smem = p->acc_in_smem ? 1 : 0;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (p->timing) {
    if (p->ev_used + 2 > (int)p->ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        BEM_CUDA_TRY(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
      }
    }
    e0 = p->ev_pool[p->ev_used++];
    e1 = p->ev_pool[p->ev_used++];
    BEM_CUDA_TRY(cudaEventRecord(e0, st));
  }
  if (elems_per_thread(p->log2N) == 16)
    launch_col_nf<T, 16>(p, op.nf, cp, st);
  else
    launch_col_nf<T, 8>(p, op.nf, cp, st);
  if (p->timing) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k_reduce<T><<<(nb + tb - 1) / tb, tb, 0, st>>>(static_cast<const T*>(p->d_partial), p->grid, nb, p->ncomp,
                                                 p->d_perm, static_cast<const T*>(op.diag), static_cast<const T*>(in),
                                                 static_cast<T*>(out));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status launch_apply_2d(bem_plan_s* p, const Operator& op, const void* in, void* out, cudaStream_t st) {
  if (op.nf < 1 || op.nf > 3) {
    set_error("2D operator with unsupported field count");
    return BEM_ERR_UNSUPPORTED;
  }
  return p->prec == BEM_F64 ? launch_t<double>(p, op, in, out, st) : launch_t<float>(p, op, in, out, st);
}

}  // namespace bemfft
