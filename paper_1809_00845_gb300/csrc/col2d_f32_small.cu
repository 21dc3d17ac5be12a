// Column kernels, FP32, N = 2048, 1024, 512 (TT = 128, 64, 32 threads).
#include "col2d_v2.cuh"

namespace bemfft {
template struct Col2DKernels<float, 128>;
template struct Col2DKernels<float, 64>;
template struct Col2DKernels<float, 32>;
template struct Col2DGroupKernels<128>;
template struct Col2DGroupKernels<64>;
template struct Col2DGroupKernels<32>;
template struct Col2DEdgeKernels<float, 128>;
template struct Col2DEdgeKernels<float, 64>;
template struct Col2DEdgeKernels<float, 32>;
template struct Col2DPassKernels<128>;
template struct Col2DPassKernels<64>;
template struct Col2DPassKernels<32>;
}  // namespace bemfft
