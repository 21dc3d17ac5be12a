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
// Operands.  A (each line's 32 input reals as 16-bit hi and lo parts) is
// written by the threads straight from registers into tensor memory
// (tcgen05.st) and read from there by the MMA, so neither the operand stores
// nor the MMA's operand reads touch shared memory, which the transposes of
// the engine keep busy.  Tensor-memory layout of A for M = 128: lane = line,
// 32-bit column j = the 16-bit elements k = 2j (low half) and 2j + 1.  Input
// element k of complex element i, part c (0 = real, 1 = imaginary):
// k = (i / 8) * 16 + c * 8 + i % 8, so that a line whose upper 8 inputs are
// zero (the zero padding of the first stage) needs only the first K = 16 half:
// one MMA per product instead of two.  Output column n of element f:
// n = c * 16 + f.  B (the DFT matrix, 32 x 32) sits in shared memory, K-major
// without swizzle: core matrices of 8 rows x 16 bytes stored as 128
// contiguous bytes, byte(n, k) = (n / 8) * 512 + (k / 8) * 128 + (n % 8) * 16
// + (k % 8) * 2 (K-direction core-matrix offset 128 B, row-group offset
// 512 B); per matrix hi (2 KB) then lo (2 KB), built on the host in FP64.
// Every warpgroup (128 threads, 128 lines) runs its stage on its own, with
// its own 64 tensor-memory columns (D: 32 FP32 columns, then A hi and A lo:
// 16 each), mbarrier, issuing thread (its first) and 128-thread named
// barrier (id 1 + g).  Warp w accesses lanes 32 (w % 4) .. + 31, which are
// exactly its own threads' lines (thread t = 128 g + 32 (w % 4) + lane).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace bemfft {

constexpr int kTcBf16 = 1;
constexpr int kTcF16 = 2;
// shared-memory header of a tensor-core column kernel: one mbarrier per
// warpgroup (4 x 8 B), the tensor-memory address (4 B), padding, then two B
// matrices (4 KB each)
constexpr int kTcMatBytes = 4096;
constexpr int kTcMatOffset = 64;
constexpr int kTcHeader = kTcMatOffset + 2 * kTcMatBytes;
// tensor-memory columns per warpgroup: D (32 FP32) + A hi (16) + A lo (16)
constexpr int kTcGroupCols = 64;
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

// D (tensor memory) (+)= A (tensor memory) x B (shared-memory descriptor)
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

// this warp's 32 lanes, 8 or 16 consecutive 32-bit columns from taddr
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
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
// false when the wait gave up.  try_wait suspends the thread (up to a
// hardware time limit per call) instead of spinning on issue slots.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    const unsigned long long now = global_ns();
    if (t0 == 0) t0 = now;
    else if (now - t0 > kTcWaitNs) return false;
  }
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

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory");
}

template <int KIND>
struct TcDft {
  uint32_t b_base;  // shared address of the B matrices
  uint32_t mbar;    // shared address of this warpgroup's mbarrier
  uint32_t tmem;    // tensor-memory address of this warpgroup's columns (lane 0)
  uint32_t phase;   // parity of the next mbarrier phase
  int t;            // thread index
  bool failed;      // a wait of this thread gave up (the kernel reports it)
  bool no_commit;   // test hook: issue nothing, so the wait runs out

  // One radix-16 stage: v[f] <- sum_i v[i] e^{DIR 2 pi i f i / 16} for the
  // matrix `mat` (0 = the 16-point DFT; 1 = the engine's J-point blocks).
  // LOWHALF: v[8..15] are zero.
  template <int DIR, bool LOWHALF>
  __device__ __forceinline__ void run(cplx<float> (&v)[16], int mat) {
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
    uint32_t h[16], l[16];
#pragma unroll
    for (int c = 0; c < (LOWHALF ? 2 : 4); ++c) {
      const int i0 = (c >> 1) * 8;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const cplx<float> p = v[i0 + 2 * j], q = v[i0 + 2 * j + 1];
        if (c & 1) tc_split2<KIND>(p.y * sy, q.y * sy, h[c * 4 + j], l[c * 4 + j]);
        else tc_split2<KIND>(p.x * sc, q.x * sc, h[c * 4 + j], l[c * 4 + j]);
      }
    }
    const uint32_t lane_base = (uint32_t)(32 * ((t >> 5) & 3)) << 16;
    const uint32_t a_hi = tmem + 32u, a_lo = tmem + 48u;
    if constexpr (LOWHALF) {
      tmem_st8(a_hi + lane_base, h);
      tmem_st8(a_lo + lane_base, l);
    } else {
      tmem_st16(a_hi + lane_base, h);
      tmem_st16(a_lo + lane_base, l);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    tc_fence_before();
    group_sync(t >> 7);
    if ((t & 127) == 0 && !no_commit) {
      tc_fence_after();
      constexpr uint32_t id = tc_idesc<KIND>();
      const uint32_t bh = b_base + (uint32_t)mat * 4096u, bl = bh + 2048u;
#pragma unroll
      for (int s = 0; s < (LOWHALF ? 1 : 2); ++s) {
        const uint32_t ka = (uint32_t)s * 8u, kb = (uint32_t)s * 256u;
        tc_mma(tmem, a_hi + ka, tc_sdesc(bh + kb), id, s > 0 ? 1u : 0u);
        tc_mma(tmem, a_lo + ka, tc_sdesc(bh + kb), id, 1u);
        tc_mma(tmem, a_hi + ka, tc_sdesc(bl + kb), id, 1u);
      }
      tc_commit(mbar);
    }
    // after a wait that gave up, the rest of the column skips its waits (the
    // CTA stops at the next column)
    if (!failed && !tc_wait(mbar, phase)) failed = true;
    phase ^= 1u;
    tc_fence_after();
    uint32_t q[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
          "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]),
          "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]),
          "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
        : "r"(tmem + lane_base));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const float oy = DIR > 0 ? -isc : isc;
#pragma unroll
    for (int f = 0; f < 16; ++f) {
      v[f].x = __uint_as_float(q[f]) * isc;
      v[f].y = __uint_as_float(q[16 + f]) * oy;
    }
    // the warpgroup's next stage overwrites these columns after its barrier
    tc_fence_before();
  }

  // bind this thread to its warpgroup's resources (after tc_setup)
  __device__ __forceinline__ void bind(int t_, uint32_t hdr, uint32_t tmem_base, bool no_commit_) {
    t = t_;
    no_commit = no_commit_;
    const int g = t >> 7;
    mbar = hdr + 8u * (uint32_t)g;
    b_base = hdr + kTcMatOffset;
    tmem = tmem_base + (uint32_t)(kTcGroupCols * g);
    phase = 0u;
    failed = false;
  }
};

// Kernel prologue (all threads): one mbarrier per warpgroup, tensor memory
// (warp 0 allocates `ncols` columns) and the B matrices (nbytes from global)
// in shared memory.  Returns the tensor-memory base address.
__device__ __forceinline__ uint32_t tc_setup(unsigned char* hdr, const uint4* mats, int nbytes, int ncols) {
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(hdr);
  const uint32_t slot = base + 32u;
  uint4* dst = reinterpret_cast<uint4*>(hdr + kTcMatOffset);
  for (int i = threadIdx.x; i < nbytes / 16; i += blockDim.x) dst[i] = mats[i];
  if (threadIdx.x == 0) {
    for (int g = 0; g < (int)(blockDim.x >> 7); ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(base + 8u * (uint32_t)g) : "memory");
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
  return *reinterpret_cast<volatile uint32_t*>(hdr + 32);
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
