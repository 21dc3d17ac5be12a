// Launch interface of the 3D line-FFT passes (kernels in fft3d.cuh, one
// instantiation per precision and grid size N = 2^LOG2N, LOG2N = 5..10).
#pragma once

#include "bem_internal.h"

namespace bemfft {

template <typename T, int LOG2N>
struct Fft3DKernels {
  static size_t smem_y();  // dynamic shared memory of the y passes
  static int zblock();     // z planes per CTA of the y passes
  static cudaError_t configure();
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
