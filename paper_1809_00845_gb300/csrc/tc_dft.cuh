// Split-precision tensor-core DFT stages of the four-step column transform
// (tcgen05, sm_103a).
//
// The four-step engine (fft4step.cuh) holds one 16-point line per thread in
// registers at each of its three radix-16 stages.  Here such a stage is a
// matrix product on the tensor cores: with the TT lines of the CTA as the
// rows of A (TT x 32 reals: the 16 complex inputs, real and imaginary parts)
// and the DFT matrix in real form as B (32 x 32), D = A B^T holds every
// line's 16 complex outputs.  Each FP32 operand x is split into a 16-bit hi
// part and a 16-bit lo part for the residual x - hi, and three products
// A_hi B_hi + A_lo B_hi + A_hi B_lo accumulate in FP32 in tensor memory (the
// lo*lo term is below FP32 rounding of the result).  Two element types:
//   KIND 1 (BF16): FP32's exponent range, 8+8 significand bits per value;
//   KIND 2 (FP16): 11+11 bits; each line is scaled by a power of two so that
//                  its largest value sits in [2^14, 2^15) (exact, undone on
//                  the way back), which keeps the hi and lo parts in range.
// The inverse DFT uses the forward matrix on conjugated data:
// IDFT(x) = conj(DFT(conj(x))).
//
// Operand layouts (K-major, no swizzle; "core matrices" of 8 rows x 16
// bytes stored as 128 contiguous bytes):
//   byte(r, k) = (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// i.e. leading-dimension (K) core-matrix offset 128 B and stride-dimension
// (row group) offset 512 B.  Input column k of complex element i, part
// c (0 = real, 1 = imaginary): k = (i / 8) * 16 + c * 8 + i % 8, so that a
// line whose upper 8 inputs are zero (the zero padding of the first stage)
// needs only the first K = 16 half: one MMA per product instead of two.
// Output column n of element f: n = c * 16 + f.
// A: TT rows, hi half then lo half (TT * 64 bytes each), aliasing the
// engine's transpose buffer, which is free at every stage.  B: per matrix
// hi (2 KB) then lo (2 KB), built on the host in FP64.
// Tensor memory: 32 FP32 columns per 128-row tile, lanes = rows; warp w reads
// lanes 32 (w % 4) .. + 31 of tile w / 4, which are exactly its own threads'
// lines (thread t = 32 w + lane = 128 (w / 4) + 32 (w % 4) + lane).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace bemfft {

constexpr int kTcBf16 = 1;
constexpr int kTcF16 = 2;
// shared-memory header of a tensor-core column kernel: mbarrier (8 B), tensor
// memory address (4 B), padding, then two B matrices (4 KB each)
constexpr int kTcMatBytes = 4096;
constexpr int kTcHeader = 16 + 2 * kTcMatBytes;
// a bounded device wait gives up after this many nanoseconds
constexpr unsigned long long kTcWaitNs = 1000000000ull;

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr) {
  // start >> 4 | LBO (128 B) >> 4 << 16 | SBO (512 B) >> 4 << 32 | descriptor version 1 << 46;
  // base offset 0, relative LBO, no swizzle
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, A and B of the
// same 16-bit type (1 = BF16, 0 = FP16), both K-major, N = 32, M = 128
template <int KIND>
__device__ __forceinline__ constexpr uint32_t tc_idesc() {
  constexpr uint32_t fmt = KIND == kTcBf16 ? 1u : 0u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// wait for the mbarrier phase of the given parity, at most kTcWaitNs;
// false when the wait gave up
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0;; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255u) == 0) {
      const unsigned long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kTcWaitNs) return false;
    }
  }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

// hi and lo parts of two FP32 values packed as two 16-bit numbers (first
// value in the low half)
template <int KIND>
__device__ __forceinline__ void tc_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  if constexpr (KIND == kTcBf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const __half2 l = __floats2half2_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

template <int KIND>
struct TcDft {
  uint32_t a_base;  // shared address of the A operand (TT rows, hi then lo)
  uint32_t b_base;  // shared address of the B matrices
  uint32_t mbar;    // shared address of the mbarrier
  uint32_t tmem;    // tensor-memory address of the accumulators
  uint32_t phase;   // parity of the next mbarrier phase
  int t, TT;
  bool failed;      // a wait of this thread gave up (the kernel reports it)

  // One radix-16 stage: v[f] <- sum_i v[i] e^{DIR 2 pi i f i / 16} for the
  // matrix `mat` (0 = the 16-point DFT; 1 = the engine's J-point blocks).
  // LOWHALF: v[8..15] are zero.  PRESYNC: another warp may still read the
  // transpose buffer that A aliases.
  template <int DIR, bool LOWHALF, bool PRESYNC>
  __device__ __forceinline__ void run(cplx<float> (&v)[16], int mat) {
    if (PRESYNC) __syncthreads();
    constexpr int NI = LOWHALF ? 8 : 16;
    float sc = 1.0f, isc = 1.0f;
    if constexpr (KIND == kTcF16) {
      float m = 0.0f;
#pragma unroll
      for (int i = 0; i < NI; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
      const int e = (__float_as_int(m) >> 23) & 0xff;
      const int es = min(268 - e, 253);  // m * 2^(es-127) in [2^14, 2^15)
      sc = __int_as_float(es << 23);
      isc = __int_as_float((254 - es) << 23);
    }
    const float sy = DIR > 0 ? -sc : sc;  // conjugate the input of an inverse stage
    const uint32_t row = a_base + (uint32_t)((t >> 3) * 512 + (t & 7) * 16);
    const uint32_t lo_off = (uint32_t)TT * 64u;
#pragma unroll
    for (int c = 0; c < (LOWHALF ? 2 : 4); ++c) {
      const int i0 = (c >> 1) * 8;
      uint32_t h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const cplx<float> p = v[i0 + 2 * j], q = v[i0 + 2 * j + 1];
        if (c & 1) tc_split2<KIND>(p.y * sy, q.y * sy, h[j], l[j]);
        else tc_split2<KIND>(p.x * sc, q.x * sc, h[j], l[j]);
      }
      st_shared_v4(row + c * 128, h[0], h[1], h[2], h[3]);
      st_shared_v4(row + lo_off + c * 128, l[0], l[1], l[2], l[3]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      constexpr uint32_t id = tc_idesc<KIND>();
      const uint32_t bh = b_base + (uint32_t)mat * 4096u, bl = bh + 2048u;
      for (int m = 0; m < (TT >> 7); ++m) {
        const uint32_t d = tmem + (uint32_t)m * 32u;
        const uint32_t ah = a_base + (uint32_t)m * 8192u, al = ah + lo_off;
#pragma unroll
        for (int s = 0; s < (LOWHALF ? 1 : 2); ++s) {
          const uint32_t ks = (uint32_t)s * 256u;
          tc_mma(d, tc_sdesc(ah + ks), tc_sdesc(bh + ks), id, s > 0 ? 1u : 0u);
          tc_mma(d, tc_sdesc(al + ks), tc_sdesc(bh + ks), id, 1u);
          tc_mma(d, tc_sdesc(ah + ks), tc_sdesc(bl + ks), id, 1u);
        }
      }
      tc_commit(mbar);
    }
    if (!tc_wait(mbar, phase)) failed = true;
    phase ^= 1u;
    tc_fence_after();
    uint32_t r[32];
    const int w = t >> 5;
    const uint32_t taddr = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(w >> 2) * 32u;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const float oy = DIR > 0 ? -isc : isc;
#pragma unroll
    for (int f = 0; f < 16; ++f) {
      v[f].x = __uint_as_float(r[f]) * isc;
      v[f].y = __uint_as_float(r[16 + f]) * oy;
    }
    // the next stage's MMAs overwrite these columns after a barrier
    tc_fence_before();
  }
};

// Kernel prologue (all threads): mbarrier, tensor memory (warp 0 allocates
// `ncols` columns) and the B matrices (nbytes from global) in shared memory.
// Returns the tensor-memory base address.
__device__ __forceinline__ uint32_t tc_setup(unsigned char* hdr, const uint4* mats, int nbytes, int ncols) {
  const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(hdr);
  const uint32_t slot = mbar + 8u;
  uint4* dst = reinterpret_cast<uint4*>(hdr + 16);
  for (int i = threadIdx.x; i < nbytes / 16; i += blockDim.x) dst[i] = mats[i];
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *reinterpret_cast<volatile uint32_t*>(hdr + 8);
}

// Kernel epilogue (all threads): every tensor-memory read has completed
// (tcgen05.wait::ld in each stage); warp 0 frees the columns.
__device__ __forceinline__ void tc_teardown(uint32_t tmem, int ncols) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace bemfft
