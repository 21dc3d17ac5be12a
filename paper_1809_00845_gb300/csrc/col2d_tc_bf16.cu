// Column kernels, FP32 with BF16 hi + lo tensor-core DFT stages, N = 8192,
// 4096 and 2048 (TT = 512, 256, 128 threads).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DTcKernels<512, kTcBf16>;
template struct Col2DTcKernels<256, kTcBf16>;
template struct Col2DTcKernels<128, kTcBf16>;
}  // namespace bemfft
