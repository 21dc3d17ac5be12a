// 3D line-FFT passes, FP64, for N = 32 ... 1024.
#include "fft3d.h"
#include "fft3d.cuh"

namespace bemfft {
template struct Fft3DKernels<double, 5>;
template struct Fft3DKernels<double, 6>;
template struct Fft3DKernels<double, 7>;
template struct Fft3DKernels<double, 8>;
template struct Fft3DKernels<double, 9>;
template struct Fft3DKernels<double, 10>;
}  // namespace bemfft
