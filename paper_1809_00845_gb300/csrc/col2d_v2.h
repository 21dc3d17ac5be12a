// Four-step column kernel of the 2D apply (N >= 512): kernel parameters and
// the launch interface.  The kernel itself lives in col2d_v2.cuh and is
// instantiated in separate translation units, one per precision and thread
// count (the thread count TT = N / 16 is a compile-time constant there, so
// every index of the transform, of the interleaved cell arrays and of the
// spectrum column folds into immediate offsets).
#pragma once

#include <cstdint>

#include "bem_internal.h"
#include "fft_reg.cuh"

namespace bemfft {

// Cell word (plan time): x | rowslot(row) << 12 | FLUSH << 29 | CARRY << 30 | type << 31.
constexpr uint32_t kMetaFlush = 1u << 29;
constexpr uint32_t kMetaCarry = 1u << 30;

template <typename T>
struct Col2Dv2Params {
  int n, log2N, nb;
  const int32_t* chunk;   // TT + 1
  const int32_t* tinfo;   // TT: row mask (8 bits) | continuing threads << 8
  const uint32_t* meta;   // Q*TT cell words, interleaved
  const cplx<T>* val;     // Q*TT density pairs, interleaved
  const T* val2;          // edge-flow kernels: Q*TT third densities (y-edge flows), interleaved
  const T* spec[3];
  int imag[3];
  int oddy[3];
  const cplx<T>* fstab;  // four-step tables (lane, warp, t5) then sparse tables (hi, lo)
  T* partial;            // gridDim.x * npos, interleaved positions
  cplx<T>* twc;          // gridDim.x * npos: each cell's sparse twiddle of the current column, or null
  int npos;              // Q*TT
  int acc_rows;          // interleaved cell rows i < acc_rows accumulate in shared memory, the rest in partial
  int has_carry;         // some row is split between threads
  const uint4* tcmat;    // tensor-core stages: the two B matrices (hi, lo), 8 KB
  int* status;           // tensor-core stages: bit 0 set when a device wait gave up
  int tc_no_commit;      // test hook: issue no MMA and no commit, so every wait runs out
  // three-pass form (k_p3_cols): the row transforms of the fields, X[f][kx][y]
  // (f < nf, kx <= n, y < n), come from HBM and the inverse-transformed
  // columns go back to it, Y[kx][y]
  const cplx<T>* X;
  cplx<T>* Y;
};

// cells per batch of the cell walks of the column kernel: the loads of a
// batch are issued together, one batch ahead of its use, so each batch's
// memory round trip overlaps the arithmetic of the one before (two batches of
// loads live at once).  Measured on the 4096^2 star (system apply, us): 1
// cell 612, 2 cells 588, 3 cells 593, 4 cells 599, 5 cells 653, 6 cells 691
// (spills); 2 cells also give the fastest accuracy-mode, double-float and
// FP64 applies.  The interleaved cell arrays hold a multiple of CB cells per
// thread, so a batch is always read whole.
#ifndef COL2D_CELL_BATCH
#define COL2D_CELL_BATCH 2
#endif
constexpr int CB = COL2D_CELL_BATCH;
// the interleaved cell arrays hold a multiple of kCellPad cells per thread: a
// whole number of batches for CB and for the other batch size of the fused
// walks (2 or 4 cells, chosen per plan by bem_tune_shapes)
constexpr int kCellPad = 4;

// per-column sparse twiddles of the fused cell walk: e^{-2 pi i kx x / N} =
// A[x >> 6] * B[x & 63] (x < 4096), B in entries 0..63 and A in 64..127
constexpr int kColTwEntries = 128;

// number of table entries of the four-step kernel for TT threads, N = 16 TT:
// lane, warp and T5 tables, then the sparse twiddles (hi: 128, lo: N / 128)
__host__ __device__ inline int fstab_entries(int TT) { return 512 + (TT / 32) * 16 + 512 + 128 + TT / 8; }
// Shared-memory slot of grid row r.  Rows are read in two patterns: 16
// consecutive rows per half-warp (transform input and output) and rows about
// 8 apart across lanes (neighbouring threads' cells along the curve, in the
// row sums and the gather).  XOR-ing the low 3 bits with bits 4..6 keeps both
// free of bank conflicts (8-byte entries) and stays inside each block of 16.
__host__ __device__ inline int rowslot(int r) { return r ^ ((r >> 4) & 7); }
// spectrum column in shared memory, padded by one entry every 16
__host__ __device__ inline int sspec_entries(int n) { return ((n + 1 + (n + 1) / 16) + 3) & ~3; }

// Column kernels of one precision T for TTC threads per CTA (TTC = 0: any
// thread count, read from the launch).  configure() lifts the shared-memory
// limit of the NF = 1, 2, 3 kernels and returns the smallest number of
// resident CTAs per SM among them; launch() runs the kernel for nf fields.
template <typename T, int TTC>
struct Col2DKernels {
  static cudaError_t configure(size_t smem, int threads, int* blocks_per_sm);
  static void launch(int nf, int grid, int threads, size_t smem, cudaStream_t st, const Col2Dv2Params<T>& cp,
                     int nb);
};

// One persistent launch over the columns of several FP32 plans of the same
// grid (device arrays: plans[nplans] parameters, c0[nplans] first CTA per plan)
template <int TTC>
struct Col2DGroupKernels {
  static cudaError_t configure(size_t smem, int threads, int* blocks_per_sm);
  static void launch(int nf, int grid, int threads, size_t smem, cudaStream_t st, const Col2Dv2Params<float>* plans,
                     const int* c0, int nplans);
};

// Edge-flow form of a node convolution: per node the density triple
// (charge, x-edge flow, y-edge flow); the x flows join the charges after the
// sparse x-DFT with the column factor e^{-2 pi i kx / N} - 1, the y flows are
// transformed as a second field and scaled per frequency by
// e^{-2 pi i ky / N} - 1, and both go through field 0's spectrum (FP32: one
// inverse transform and one gather; FP64 and double-float: one each per
// field).  configure() as for Col2DKernels.
template <typename T, int TTC>
struct Col2DEdgeKernels {
  static cudaError_t configure(size_t smem, int threads, int* blocks_per_sm);
  static void launch(int grid, int threads, size_t smem, cudaStream_t st, const Col2Dv2Params<T>& cp, int nb);
};

// Three-pass form, FP32, TTC = 32 ... 512: the column pass alone (forward
// transforms of the fields' x-DFT rows read from X, spectral multiply, one
// inverse transform written to Y); the row passes live in apply2d.cu.
template <int TTC>
struct Col2DPassKernels {
  static cudaError_t configure(size_t smem, int threads, int* blocks_per_sm);
  static void launch(int nf, int grid, int threads, size_t smem, cudaStream_t st, const Col2Dv2Params<float>& cp);
};

// The same kernels in FP32 with the radix-16 stages of the transforms on the
// tensor cores, TCK = 1 (BF16 hi + lo) or 2 (FP16 hi + lo), TTC = 128, 256 or
// 512.  configure() also bounds the resident CTAs by the tensor memory.
template <int TTC, int TCK>
struct Col2DTcKernels {
  static cudaError_t configure(size_t smem, int threads, int* blocks_per_sm);
  static void launch(int nf, int grid, int threads, size_t smem, cudaStream_t st, const Col2Dv2Params<float>& cp,
                     int nb);
};

}  // namespace bemfft
