// Launch interface of the 3D line-FFT passes (kernels in fft3d.cuh, one
// instantiation per precision and grid size N = 2^LOG2N, LOG2N = 5..10).
#pragma once

#include "bem_internal.h"

namespace bemfft {

// Twiddles of the Stockham passes of a line of N = 2^LOG2N (16 elements per
// thread): pass p >= 1 has Ns = 16^p and radix R = 16 (or the 2/4/8 left
// over), and its factors e^{2 pi i k r / (Ns R)} (k < Ns, r < R) sit at
// off(p) + r Ns + k, so that consecutive butterflies read consecutive entries.
template <int LOG2N>
struct PassTab {
  static constexpr int npass = (LOG2N + 3) / 4;
  static constexpr int radix(int p) { return LOG2N - 4 * p > 4 ? 16 : (1 << (LOG2N - 4 * p)); }
  static constexpr int ns(int p) { return 1 << (4 * p); }
  static constexpr int off(int p) {
    int o = 0;
    for (int q = 1; q < p; ++q) o += ns(q) * radix(q);
    return o;
  }
  static constexpr int size() { return off(npass); }
};

template <typename T, int LOG2N>
struct Fft3DKernels {
  static size_t smem_y();  // dynamic shared memory of the y passes
  static int zblock();     // z planes per CTA of the y passes
  static cudaError_t configure();
  static int ptab_size() { return PassTab<LOG2N>::size(); }
  // forward: x-DFT from the cells + y FFT of nf fields -> B
  static void yfwd(int nf, int nb, const int32_t* lptr, const uint16_t* xs, const void* val, const void* tw2,
                   void* B, const void* qtab, cudaStream_t st);
  // z FFT, coupled spectral multiply, inverse z FFT (in place in B)
  static void zpass(int nf, int no, int lpc, const int16_t* coup, const Spec3D* specs, void* B, const void* qtab,
                    cudaStream_t st);
  // inverse y FFT of no outputs -> X
  static void yinv(int no, const void* B, void* X, const void* qtab, cudaStream_t st);
};

}  // namespace bemfft
