// Line-FFT passes of the 3D apply (Section 3: the convolution over the volume
// enclosing the surface; Eq. 15-16), instantiated per grid size so that the
// Stockham passes, their twiddle indices and all line strides are
// compile-time constants.  N = 2^LOG2N, 16 elements per thread, TT = N/16
// threads per line.
//
//   k3_yfwd  per (kx, block of z planes, field): the input-pruned x-DFT of the
//            grid lines (y, z) evaluated from the cell list straight into the
//            registers of the y transform (no x-transformed buffer in HBM),
//            forward y FFT (inputs y >= n are zero: pruned first pass), result
//            B_f[kx][ky][z] through a padded shared-memory transpose.
//   k3_zpass per (kx, group of ky): forward z FFT of every field (z >= n zero),
//            spectral multiply-accumulate Y_o = sum_f K_of B_f (spectrum reads
//            issued before the transform), inverse z FFT, B_o <- Y_o (z < n).
//            With one output the field spectra are accumulated in registers.
//   k3_yinv  per (kx, block of z planes, output): inverse y FFT, rows y < n to
//            X_o[kx][z][y] for the gather.
//
// Included only by the translation units that instantiate Fft3DKernels.
#pragma once

#include <type_traits>

#include "bem_internal.h"
#include "fft3d.h"
#include "fft4step.cuh"
#include "fft_reg.cuh"

namespace bemfft {

// e^{DIR 2 pi i m / N}, m = 64 hi + lo (tables hi: max(1, N/64), lo: 64)
template <typename T>
struct Tw64 {
  const cplx<T>* hi;
  const cplx<T>* lo;
  template <int DIR>
  __device__ __forceinline__ cplx<T> get(int m) const {
    cplx<T> z = cmul(hi[m >> 6], lo[m & 63]);
    if constexpr (DIR < 0) z.y = -z.y;
    return z;
  }
};

// read-only load of one value of the working type (the read-only cache path
// for float and double; a double-float pair is read as a plain struct)
template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) return __ldg(p);
  else return *p;
}

template <int LOG2N>
struct Line3D {
  static constexpr int N = 1 << LOG2N;
  static constexpr int n = N / 2;
  static constexpr int TT = N / 16;                     // threads per line
  static constexpr bool WARP = TT <= 32;                // lines never straddle warps
  static constexpr int LPB = TT >= 64 ? 512 / TT : 16;  // lines per block of the z pass
  static constexpr int SBUF = N + N / 16;               // padded exchange buffer per line
};

// One Stockham pass of radix R, compile-time position in the transform.
// LOWIN: the first pass's inputs 8..15 are zero.
// z planes per block of the y passes (16: wider blocks give longer contiguous
// z runs of B but were measured slower, 32 planes lowering the resident warps)
template <typename T, int LOG2N>
__host__ __device__ constexpr int yblock() {
  constexpr int TT = Line3D<LOG2N>::TT, n = Line3D<LOG2N>::n;
  constexpr int want = 16;
  constexpr int lim = TT * want > 512 ? 512 / TT : want;
  return lim < n ? lim : n;
}

template <int LOG2N, int R, int LOG2NS, int DIR, bool LAST, bool LOWIN, typename T>
__device__ __forceinline__ void stockham_ct(cplx<T> (&v)[16], const int t, const cplx<T>* pt, cplx<T>* sbuf) {
  using L = Line3D<LOG2N>;
  constexpr int S = 16 / R;
  constexpr int Ns = 1 << LOG2NS;
  constexpr int OFF = PassTab<LOG2N>::off(LOG2NS / 4);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int b = t + s * L::TT;
    const int k = b & (Ns - 1);
    cplx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = v[s + r * S];
    if constexpr (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = pt[OFF + r * Ns + k];
        if constexpr (DIR < 0) w.y = -w.y;
        u[r] = cmul(u[r], w);
      }
    }
    if constexpr (LOWIN && R == 16) dft16_lowhalf<DIR>(u);
    else dft<R, DIR>(u);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[s + r * S] = u[r];
    } else {
      const int base = (b - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sbuf[pad16(base + r * Ns)] = u[r];
    }
  }
  if constexpr (!LAST) {
    line_sync<L::WARP>();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = sbuf[pad16(t + m * L::TT)];
    line_sync<L::WARP>();
  }
}

// Radix-16 passes, then one pass of the remaining radix (2, 4 or 8) when
// LOG2N is not a multiple of 4.  Natural order in and out (positions
// t + m*TT).  Outputs the caller never reads are dead code after inlining.
template <int LOG2N, int DIR, bool LOWIN, typename T, int PASS = 0>
__device__ __forceinline__ void fft_ct(cplx<T> (&v)[16], const int t, const cplx<T>* tw, cplx<T>* sbuf) {
  constexpr int done = 4 * PASS;
  constexpr int left = LOG2N - done;
  static_assert(left >= 1, "line too short");
  if constexpr (left > 4) {
    stockham_ct<LOG2N, 16, done, DIR, false, LOWIN && PASS == 0>(v, t, tw, sbuf);
    fft_ct<LOG2N, DIR, LOWIN, T, PASS + 1>(v, t, tw, sbuf);
  } else {
    constexpr int R = 1 << left;
    stockham_ct<LOG2N, R, done, DIR, true, LOWIN && PASS == 0 && R == 16>(v, t, tw, sbuf);
  }
}

// ---------------------------------------------------------------- kernels

template <typename T, int LOG2N>
__global__ void __launch_bounds__(512) k3_yfwd(int nb, const int32_t* __restrict__ lptr,
                                               const uint16_t* __restrict__ xs, const T* __restrict__ val,
                                               const cplx<T>* __restrict__ tw2, cplx<T>* __restrict__ B,
                                               const cplx<T>* __restrict__ qtab) {
  using L = Line3D<LOG2N>;
  constexpr int N = L::N, n = L::n, TT = L::TT, ZB = yblock<T, LOG2N>();
  constexpr int NHI = N >= 64 ? N / 64 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const int kx = blockIdx.y, z0 = blockIdx.x * ZB, f = blockIdx.z;
  cplx<T>* sq = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* stw = sq + PassTab<LOG2N>::size();
  cplx<T>* sbuf = stw + NHI + 64;  // ZB line buffers, later the tile
  for (int i = threadIdx.x; i < PassTab<LOG2N>::size(); i += blockDim.x) sq[i] = qtab[i];
  for (int i = threadIdx.x; i < NHI + 64; i += blockDim.x) stw[i] = tw2[i];
  __syncthreads();
  const cplx<T>* tw = sq;
  const Tw64<T> t64{stw, stw + NHI};
  // x-DFT of the lines (y = t + m*TT, z = z0 + g) from the cells of each line;
  // the bounds of all eight lines are read first.  (Issuing the first cells of
  // every line together was measured slower: the twiddles of the many empty
  // slots cost more than the latency they hide.)
  const T* vf = val + (size_t)f * nb;
  cplx<T> v[16];
  int j0[8], j1[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int line = (z0 + g) * n + t + m * TT;
    j0[m] = __ldg(lptr + line);
    j1[m] = __ldg(lptr + line + 1);
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    cplx<T> sum = {T(0), T(0)};
    for (int j = j0[m]; j < j1[m]; ++j) {
      const cplx<T> w = t64.template get<-1>((kx * (int)__ldg(xs + j)) & (N - 1));
      const T r = ld_ro(vf + j);
      sum = cmacr(sum, r, w);
    }
    v[m] = sum;
  }
#pragma unroll
  for (int m = 8; m < 16; ++m) v[m] = {T(0), T(0)};
  fft_ct<LOG2N, -1, true>(v, t, tw, sbuf + (size_t)g * L::SBUF);
  __syncthreads();
  cplx<T>* tile = sbuf;  // [N][ZB + 1]
#pragma unroll
  for (int m = 0; m < 16; ++m) tile[(size_t)(t + m * TT) * (ZB + 1) + g] = v[m];
  __syncthreads();
  cplx<T>* dst = B + ((size_t)f * (n + 1) + kx) * (size_t)N * n + z0;
  for (int i = threadIdx.x; i < N * ZB; i += blockDim.x) {
    const int ky = i / ZB, zz = i - ky * ZB;
    dst[(size_t)ky * n + zz] = tile[(size_t)ky * (ZB + 1) + zz];
  }
}

// i^q * sv * x
template <typename T>
__device__ __forceinline__ cplx<T> iq_times(int q, T sv, cplx<T> x) {
  switch (q & 3) {
    case 0: return {x.x * sv, x.y * sv};
    case 1: return {-x.y * sv, x.x * sv};
    case 2: return {-x.x * sv, -x.y * sv};
    default: return {x.y * sv, -x.x * sv};
  }
}

template <typename T, int LOG2N>
__global__ void __launch_bounds__(512) k3_zpass(int nf, int no, int LPC, const int16_t* __restrict__ coup,
                                                const Spec3D* __restrict__ specs, cplx<T>* __restrict__ B,
                                                const cplx<T>* __restrict__ qtab) {
  using L = Line3D<LOG2N>;
  constexpr int N = L::N, n = L::n, TT = L::TT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const int kx = blockIdx.y, ky = blockIdx.x * LPC + g;
  cplx<T>* sq = reinterpret_cast<cplx<T>*>(smem_raw);
  for (int i = threadIdx.x; i < PassTab<LOG2N>::size(); i += blockDim.x) sq[i] = qtab[i];
  __syncthreads();
  const cplx<T>* tw = sq;
  const size_t per_line = (size_t)L::SBUF + (no > 1 ? (size_t)nf * N : 0);
  cplx<T>* sbuf = sq + PassTab<LOG2N>::size() + (size_t)g * per_line;
  cplx<T>* xh = sbuf + L::SBUF;  // nf spectra of this column (several outputs only)
  const size_t fstride = (size_t)(n + 1) * N * n;
  const size_t col = ((size_t)kx * N + ky) * n;
  const bool hiy = ky > n;
  const int fy = hiy ? N - ky : ky;
  // spectrum values of kernel table s at this column, positions kz = t + m*TT
  auto spectrum = [&](int s, T (&sv)[16]) {
    const Spec3D sp = specs[s];
    const T* S = static_cast<const T*>(sp.data) + ((size_t)kx * (n + 1) + fy) * (n + 1);
    const bool negy = hiy && sp.oddy;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int kz = t + m * TT;
      const bool hiz = kz > n;
      const T a = ld_ro(S + (hiz ? N - kz : kz));
      sv[m] = (negy != (hiz && sp.oddz)) ? -a : a;
    }
  };
  auto load_col = [&](int f, cplx<T> (&v)[16]) {
    const cplx<T>* src = B + f * fstride + col;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = src[t + m * TT];
#pragma unroll
    for (int m = 8; m < 16; ++m) v[m] = {T(0), T(0)};
  };
  if (no == 1) {
    cplx<T> y[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) y[m] = {T(0), T(0)};
    for (int f = 0; f < nf; ++f) {
      const int s = coup[f];
      if (s < 0) continue;
      cplx<T> v[16];
      T sv[16];
      load_col(f, v);
      spectrum(s, sv);  // reads in flight during the transform
      fft_ct<LOG2N, -1, true>(v, t, tw, sbuf);
      const int q = specs[s].q;
#pragma unroll
      for (int m = 0; m < 16; ++m) y[m] = y[m] + iq_times(q, sv[m], v[m]);
    }
    fft_ct<LOG2N, +1, false>(y, t, tw, sbuf);
    cplx<T>* dst = B + col;
#pragma unroll
    for (int m = 0; m < 8; ++m) dst[t + m * TT] = y[m];
    return;
  }
  for (int f = 0; f < nf; ++f) {
    cplx<T> v[16];
    load_col(f, v);
    fft_ct<LOG2N, -1, true>(v, t, tw, sbuf);
#pragma unroll
    for (int m = 0; m < 16; ++m) xh[(size_t)f * N + t + m * TT] = v[m];
  }
  for (int o = 0; o < no; ++o) {
    cplx<T> y[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) y[m] = {T(0), T(0)};
    for (int f = 0; f < nf; ++f) {
      const int s = coup[o * nf + f];
      if (s < 0) continue;
      T sv[16];
      spectrum(s, sv);
      const int q = specs[s].q;
#pragma unroll
      for (int m = 0; m < 16; ++m) y[m] = y[m] + iq_times(q, sv[m], xh[(size_t)f * N + t + m * TT]);
    }
    fft_ct<LOG2N, +1, false>(y, t, tw, sbuf);
    cplx<T>* dst = B + o * fstride + col;
#pragma unroll
    for (int m = 0; m < 8; ++m) dst[t + m * TT] = y[m];
  }
}

template <typename T, int LOG2N>
__global__ void __launch_bounds__(512) k3_yinv(const cplx<T>* __restrict__ B, cplx<T>* __restrict__ X,
                                               const cplx<T>* __restrict__ qtab) {
  using L = Line3D<LOG2N>;
  constexpr int N = L::N, n = L::n, TT = L::TT, ZB = yblock<T, LOG2N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const int kx = blockIdx.y, z0 = blockIdx.x * ZB, o = blockIdx.z;
  cplx<T>* sq = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* sbuf = sq + PassTab<LOG2N>::size();
  for (int i = threadIdx.x; i < PassTab<LOG2N>::size(); i += blockDim.x) sq[i] = qtab[i];
  const cplx<T>* src = B + ((size_t)o * (n + 1) + kx) * (size_t)N * n + z0;
  cplx<T>* tile = sbuf;
  // the block is ZB * TT threads: a compile-time trip count puts every load of
  // the tile in flight at once (one load at a time left the pass latency-bound)
  constexpr int THREADS = ZB * TT, PER = N * ZB / THREADS;
  static_assert(N * ZB % THREADS == 0, "tile / threads");
  cplx<T> ld[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = threadIdx.x + j * THREADS;
    const int ky = i / ZB, zz = i - ky * ZB;
    ld[j] = src[(size_t)ky * n + zz];
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = threadIdx.x + j * THREADS;
    const int ky = i / ZB, zz = i - ky * ZB;
    tile[(size_t)ky * (ZB + 1) + zz] = ld[j];
  }
  __syncthreads();
  const cplx<T>* tw = sq;
  cplx<T> v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = tile[(size_t)(t + m * TT) * (ZB + 1) + g];
  __syncthreads();
  fft_ct<LOG2N, +1, false>(v, t, tw, sbuf + (size_t)g * L::SBUF);
  cplx<T>* dst = X + ((size_t)o * (n + 1) + kx) * (size_t)n * n + (size_t)(z0 + g) * n;
#pragma unroll
  for (int m = 0; m < 8; ++m) dst[t + m * TT] = v[m];
}

// ------------------------------------------------------------ launches

template <typename T, int LOG2N>
size_t Fft3DKernels<T, LOG2N>::smem_y() {
  using L = Line3D<LOG2N>;
  constexpr int ZB = yblock<T, LOG2N>();
  constexpr size_t lines = (size_t)ZB * L::SBUF, tile = (size_t)L::N * (ZB + 1);
  return (size_t)(PassTab<LOG2N>::size() + (L::N >= 64 ? L::N / 64 : 1) + 64) * sizeof(cplx<T>) +
         (lines > tile ? lines : tile) * sizeof(cplx<T>);
}

template <typename T, int LOG2N>
int Fft3DKernels<T, LOG2N>::zblock() {
  using L = Line3D<LOG2N>;
  return yblock<T, LOG2N>();
}

template <typename T, int LOG2N>
cudaError_t Fft3DKernels<T, LOG2N>::configure() {
  cudaError_t e;
  if ((e = allow_optin_smem(k3_yfwd<T, LOG2N>)) != cudaSuccess) return e;
  if ((e = allow_optin_smem(k3_zpass<T, LOG2N>)) != cudaSuccess) return e;
  return allow_optin_smem(k3_yinv<T, LOG2N>);
}

template <typename T, int LOG2N>
void Fft3DKernels<T, LOG2N>::yfwd(int nf, int nb, const int32_t* lptr, const uint16_t* xs, const void* val,
                                  const void* tw2, void* B, const void* qtab, cudaStream_t st) {
  using L = Line3D<LOG2N>;
  const int ZB = zblock();
  k3_yfwd<T, LOG2N><<<dim3(L::n / ZB, L::n + 1, nf), ZB * L::TT, smem_y(), st>>>(
      nb, lptr, xs, static_cast<const T*>(val), static_cast<const cplx<T>*>(tw2), static_cast<cplx<T>*>(B),
      static_cast<const cplx<T>*>(qtab));
}

template <typename T, int LOG2N>
void Fft3DKernels<T, LOG2N>::zpass(int nf, int no, int lpc, const int16_t* coup, const Spec3D* specs, void* B,
                                   const void* qtab, cudaStream_t st) {
  using L = Line3D<LOG2N>;
  const size_t per_line = (size_t)L::SBUF + (no > 1 ? (size_t)nf * L::N : 0);
  const size_t smem = ((size_t)PassTab<LOG2N>::size() + (size_t)lpc * per_line) * sizeof(cplx<T>);
  k3_zpass<T, LOG2N><<<dim3(L::N / lpc, L::n + 1), lpc * L::TT, smem, st>>>(
      nf, no, lpc, coup, specs, static_cast<cplx<T>*>(B), static_cast<const cplx<T>*>(qtab));
}

template <typename T, int LOG2N>
void Fft3DKernels<T, LOG2N>::yinv(int no, const void* B, void* X, const void* qtab, cudaStream_t st) {
  using L = Line3D<LOG2N>;
  const int ZB = zblock();
  k3_yinv<T, LOG2N><<<dim3(L::n / ZB, L::n + 1, no), ZB * L::TT, smem_y(), st>>>(
      static_cast<const cplx<T>*>(B), static_cast<cplx<T>*>(X), static_cast<const cplx<T>*>(qtab));
}

}  // namespace bemfft
