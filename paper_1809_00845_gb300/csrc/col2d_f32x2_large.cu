// Column kernels, double-float arithmetic, N = 8192 and 4096 (TT = 512, 256
// threads, compile-time: every index folds into immediates, no register spills).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<f32x2, 512>;
template struct Col2DKernels<f32x2, 256>;
template struct Col2DEdgeKernels<f32x2, 512>;
template struct Col2DEdgeKernels<f32x2, 256>;
}  // namespace bemfft
