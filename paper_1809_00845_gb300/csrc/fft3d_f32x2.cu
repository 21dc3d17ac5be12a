// 3D line-FFT passes in double-float arithmetic (pairs of FP32, ff.cuh), for
// N = 32 ... 1024: the residual operator of mixed-precision refinement of 3D
// FP32 plans.
#include "fft3d.h"
#include "fft3d.cuh"

namespace bemfft {
template struct Fft3DKernels<f32x2, 5>;
template struct Fft3DKernels<f32x2, 6>;
template struct Fft3DKernels<f32x2, 7>;
template struct Fft3DKernels<f32x2, 8>;
template struct Fft3DKernels<f32x2, 9>;
template struct Fft3DKernels<f32x2, 10>;
}  // namespace bemfft
