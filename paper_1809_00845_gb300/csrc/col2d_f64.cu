// Column kernels, FP64, any N >= 512 (thread count taken from the launch).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<double, 0>;
template struct Col2DEdgeKernels<double, 0>;
}  // namespace bemfft
