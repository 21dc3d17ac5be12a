// Four-step CTA transform of one line of length N = 16 * TT (TT = 32 * J,
// J in {1, 2, 4, 8, 16}: N = 512 ... 8192), sm_103a.
//
// Thread t holds positions t + m*TT (m < 16) in registers, the same map as the
// Stockham engine in fft_reg.cuh, so the scatter fills and the gather reads
// registers directly.  With n = TT*m + t and k = k1 + 16*k2:
//   S1  16-point DFT over m in registers                       -> Y[t][k1]
//   T2  twiddle w_N^{t k1}
//   A   CTA transpose through shared memory: warp w receives the L = 16/W
//       lines k1 = w*L .. w*L+L-1, lane l holding elements t = l + 32 j
//   S4  J-point DFT over j in registers
//   T5  twiddle w_TT^{l kj}
//   B   warp transpose: the 16 remaining 32-point DFTs (index d = a*J + kj)
//       become lane pairs, lane l = 2d + h holding the points l' = 2i + h
//   S7  16-point DFT over i in registers (even / odd half of the 32 points)
//   S8  radix-2 combine across the lane pair with one shuffle exchange.
// The forward output sits in a fixed scrambled order (freq() below).  The
// inverse transform runs the adjoint of every step in reverse order
// (S8^H, S7^H, B^T, T5^H, S4^H, A^T, T2^H, S1^H), which is the inverse DFT
// (unnormalised) and returns natural order in the same register map.
// Per transform: one CTA-wide exchange (two barriers) instead of one per
// Stockham pass; the second exchange stays inside a warp.
#pragma once

#include "fft_reg.cuh"

namespace bemfft {

// a0..a3 with the upper half (a2, a3) known to be zero
template <int DIR, typename T>
__device__ __forceinline__ void dft4_lowhalf(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  const cplx<T> b1 = mul_i<DIR>(a1);
  const cplx<T> x0 = a0 + a1, x2 = a0 - a1, x1 = a0 + b1, x3 = a0 - b1;
  a0 = x0;
  a1 = x1;
  a2 = x2;
  a3 = x3;
}

// 16-point DFT in registers whose inputs 8..15 are zero.
template <int DIR, typename T>
__device__ __forceinline__ void dft16_lowhalf(cplx<T> (&a)[16]) {
  // R1 = 4 over stride-4 subsequences: elements r2 + 4 r1, r1 = 2, 3 are zero
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4_lowhalf<DIR>(a[r2], a[r2 + 4], a[r2 + 8], a[r2 + 12]);
#pragma unroll
  for (int r2 = 1; r2 < 4; ++r2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[r2 + 4 * k1] = twc<16, DIR>(a[r2 + 4 * k1], r2 * k1);
  cplx<T> o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> t0 = a[4 * k1], t1 = a[4 * k1 + 1], t2 = a[4 * k1 + 2], t3 = a[4 * k1 + 3];
    dft4<DIR>(t0, t1, t2, t3);
    o[k1] = t0;
    o[k1 + 4] = t1;
    o[k1 + 8] = t2;
    o[k1 + 12] = t3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = o[i];
}

template <typename T>
struct FourStep {
  int t, TT, log2N, log2TT;
  int w, l;      // warp, lane
  int W, L, J;   // warps, lines per warp, elements per line per lane
  cplx<T>* sA;   // max(N, W*16*34) elements, shared
  Twiddles<T> tw;

  __device__ __forceinline__ void init(int t_, int TT_, int log2N_, cplx<T>* s, const Twiddles<T>& tw_) {
    t = t_;
    TT = TT_;
    log2N = log2N_;
    log2TT = log2N_ - 4;
    w = t >> 5;
    l = t & 31;
    W = TT >> 5;
    L = 16 / W;
    J = TT >> 5;
    sA = s;
    tw = tw_;
  }
  __device__ __forceinline__ void cta_sync() const {
    if (W > 1) __syncthreads();
    else __syncwarp();
  }
  // e^{DIR 2 pi i m / N}
  template <int DIR>
  __device__ __forceinline__ cplx<T> twN(int m) const {
    return tw.template get<DIR>(m & ((1 << log2N) - 1));
  }
  // v[k] *= w^(k) for k = 1..15, w^k = e^{DIR 2 pi i base k / N}: four table
  // lookups (k = 1, 2, 4, 8) and products of at most three of them.
  template <int DIR>
  __device__ __forceinline__ void twiddle16(cplx<T> (&v)[16], int base) const {
    const cplx<T> w1 = twN<DIR>(base), w2 = twN<DIR>(2 * base), w4 = twN<DIR>(4 * base), w8 = twN<DIR>(8 * base);
    const cplx<T> w3 = cmul(w1, w2), w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
    const cplx<T> w9 = cmul(w8, w1), w10 = cmul(w8, w2), w11 = cmul(w8, w3), w12 = cmul(w8, w4);
    const cplx<T> w13 = cmul(w8, w5), w14 = cmul(w8, w6), w15 = cmul(w8, w7);
    v[1] = cmul(v[1], w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    v[4] = cmul(v[4], w4);
    v[5] = cmul(v[5], w5);
    v[6] = cmul(v[6], w6);
    v[7] = cmul(v[7], w7);
    v[8] = cmul(v[8], w8);
    v[9] = cmul(v[9], w9);
    v[10] = cmul(v[10], w10);
    v[11] = cmul(v[11], w11);
    v[12] = cmul(v[12], w12);
    v[13] = cmul(v[13], w13);
    v[14] = cmul(v[14], w14);
    v[15] = cmul(v[15], w15);
  }

  // line-local J-point DFTs on u[a*J + j] (J = 16/L), direction DIR
  template <int DIR>
  __device__ __forceinline__ void dftJ(cplx<T> (&u)[16]) const {
    if (J == 16) {
      dft<16, DIR>(u);
    } else if (J == 8) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        cplx<T> q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = u[a * 8 + j];
        dft<8, DIR>(q);
#pragma unroll
        for (int j = 0; j < 8; ++j) u[a * 8 + j] = q[j];
      }
    } else if (J == 4) {
#pragma unroll
      for (int a = 0; a < 4; ++a) dft4<DIR>(u[a * 4], u[a * 4 + 1], u[a * 4 + 2], u[a * 4 + 3]);
    } else if (J == 2) {
#pragma unroll
      for (int a = 0; a < 8; ++a) dft2<DIR>(u[a * 2], u[a * 2 + 1]);
    }
  }
  // u[a*J + kj] *= e^{DIR 2 pi i l kj / TT}
  template <int DIR>
  __device__ __forceinline__ void twiddleT5(cplx<T> (&u)[16]) const {
    if (J == 1) return;
    const int s = 1 << (log2N - log2TT);  // table stride for N/TT
    if (J == 16) {
      twiddle16<DIR>(u, l * s);
      return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int kj = i & (J - 1);
      if (kj) u[i] = cmul(u[i], twN<DIR>(l * kj * s));
    }
  }

  // ---- forward: registers in natural position order -> scrambled spectrum
  // sync_first: the previous call on this buffer was forward() (its warp
  // transposes may still be reading), so wait before rewriting the buffer.
  template <bool LOWHALF>
  __device__ __forceinline__ void forward(cplx<T> (&v)[16], bool sync_first = false) const {
    if (sync_first) cta_sync();
    if constexpr (LOWHALF) dft16_lowhalf<-1>(v);
    else dft<16, -1>(v);
    twiddle16<-1>(v, t);
    // A: smem[k1][t]
#pragma unroll
    for (int k = 0; k < 16; ++k) sA[k * TT + t] = v[k];
    cta_sync();
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      const int line = w * L + a / J, j = a % J;
      v[a] = sA[line * TT + l + 32 * j];
    }
    cta_sync();
    dftJ<-1>(v);
    twiddleT5<-1>(v);
    // B: warp region, row d = a*J + kj = register index, 34-element rows
    cplx<T>* sB = sA + w * (16 * 34);
#pragma unroll
    for (int d = 0; d < 16; ++d) sB[d * 34 + l] = v[d];
    __syncwarp();
    const int d = l >> 1, h = l & 1;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = sB[d * 34 + 2 * i + h];
    __syncwarp();
    dft<16, -1>(v);
    // S8: X[k] = E0[k] + w32^k E1[k], X[k+16] = E0[k] - w32^k E1[k]
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      cplx<T> mine = h ? twc<32, -1>(v[k], k) : v[k];
      cplx<T> other;
      other.x = __shfl_xor_sync(0xffffffffu, mine.x, 1);
      other.y = __shfl_xor_sync(0xffffffffu, mine.y, 1);
      v[k] = h ? other - mine : mine + other;
    }
  }
  // frequency held by register k after forward()
  __device__ __forceinline__ int freq(int k) const {
    const int d = l >> 1, h = l & 1;
    const int a = d / J, kj = d % J;
    const int k1 = w * L + a;
    const int kl = k + 16 * h;
    return k1 + 16 * (kj + J * kl);
  }
  // ---- inverse: scrambled spectrum -> registers in natural position order
  __device__ __forceinline__ void inverse(cplx<T> (&v)[16]) const {
    const int d = l >> 1, h = l & 1;
    // S8^H: lane 0 holds A, lane 1 holds B: E0 = A + B, E1 = conj(w)(A - B)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      cplx<T> other;
      other.x = __shfl_xor_sync(0xffffffffu, v[k].x, 1);
      other.y = __shfl_xor_sync(0xffffffffu, v[k].y, 1);
      v[k] = h ? twc<32, +1>(other - v[k], k) : v[k] + other;
    }
    dft<16, +1>(v);
    cplx<T>* sB = sA + w * (16 * 34);
#pragma unroll
    for (int i = 0; i < 16; ++i) sB[d * 34 + 2 * i + h] = v[i];
    __syncwarp();
#pragma unroll
    for (int dd = 0; dd < 16; ++dd) v[dd] = sB[dd * 34 + l];
    twiddleT5<+1>(v);
    dftJ<+1>(v);
    cta_sync();  // every warp is done with its B region before A is rewritten
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      const int line = w * L + a / J, j = a % J;
      sA[line * TT + l + 32 * j] = v[a];
    }
    cta_sync();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = sA[k * TT + t];
    cta_sync();
    twiddle16<+1>(v, t);
    dft<16, +1>(v);
  }
};

}  // namespace bemfft
