// Column kernels, double-float arithmetic, N = 2048 and 1024 (TT = 128, 64
// threads, compile-time).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<f32x2, 128>;
template struct Col2DKernels<f32x2, 64>;
template struct Col2DEdgeKernels<f32x2, 128>;
template struct Col2DEdgeKernels<f32x2, 64>;
}  // namespace bemfft
