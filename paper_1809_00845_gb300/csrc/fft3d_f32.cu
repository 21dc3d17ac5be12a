// 3D line-FFT passes, FP32, for N = 32 ... 1024.
#include "fft3d.h"
#include "fft3d.cuh"

namespace bemfft {
template struct Fft3DKernels<float, 5>;
template struct Fft3DKernels<float, 6>;
template struct Fft3DKernels<float, 7>;
template struct Fft3DKernels<float, 8>;
template struct Fft3DKernels<float, 9>;
template struct Fft3DKernels<float, 10>;
}  // namespace bemfft
