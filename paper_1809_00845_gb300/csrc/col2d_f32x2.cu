// Column kernels, double-float arithmetic (pairs of FP32), any N >= 512 (the
// thread count read from the launch; N = 512 uses it, larger grids have
// compile-time instantiations in col2d_f32x2_large.cu / col2d_f32x2_small.cu).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<f32x2, 0>;
template struct Col2DEdgeKernels<f32x2, 0>;
}  // namespace bemfft
