// Column kernels, FP32, N = 8192 and 4096 (TT = 512, 256 threads).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<float, 512>;
template struct Col2DKernels<float, 256>;
template struct Col2DGroupKernels<512>;
template struct Col2DGroupKernels<256>;
template struct Col2DEdgeKernels<float, 512>;
template struct Col2DEdgeKernels<float, 256>;
template struct Col2DPassKernels<512>;
template struct Col2DPassKernels<256>;
}  // namespace bemfft
