// Column kernels, double-float arithmetic (pairs of FP32), any N >= 512.
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<f32x2, 0>;
}  // namespace bemfft
