// Column kernels, FP32 with FP16 hi + lo tensor-core DFT stages (lines
// scaled by powers of two), N = 8192, 4096 and 2048 (TT = 512, 256, 128).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DTcKernels<512, kTcF16>;
template struct Col2DTcKernels<256, kTcF16>;
template struct Col2DTcKernels<128, kTcF16>;
}  // namespace bemfft
