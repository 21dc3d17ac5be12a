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
// With TCK > 0 (FP32 only, TT a multiple of 128) the three 16-point stages
// S1, S4 and S7 (and their adjoints) run as split-precision tensor-core
// products (tc_dft.cuh); twiddles, transposes and S8 stay on the FP32 pipes.
// Their operands live in tensor memory, so a stage touches no shared memory
// but the DFT matrices and synchronises only its own warpgroup.
#pragma once

#include <type_traits>

#include "fft_reg.cuh"
#include "tc_dft.cuh"

namespace bemfft {

// which radix-16 stages run on the tensor cores when TCK > 0: bit 0 S1,
// 1 S4, 2 S7 (forward), 3 S7^H, 4 S4^H, 5 S1^H (inverse)
#ifndef COL2D_TC_STAGES
#define COL2D_TC_STAGES 0x3F
#endif
constexpr int kTcStages = COL2D_TC_STAGES;

// a0..a3 with the upper half (a2, a3) known to be zero
template <int DIR, typename T, bool PK = true>
__device__ __forceinline__ void dft4_lowhalf(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  const cplx<T> b1 = mul_i<DIR>(a1);
  const cplx<T> x0 = badd<PK>(a0, a1), x2 = bsub<PK>(a0, a1), x1 = a0 + b1, x3 = a0 - b1;
  a0 = x0;
  a1 = x1;
  a2 = x2;
  a3 = x3;
}

// 16-point DFT in registers whose inputs 8..15 are zero.
template <int DIR, typename T, bool PK = true>
__device__ __forceinline__ void dft16_lowhalf(cplx<T> (&a)[16]) {
  // R1 = 4 over stride-4 subsequences: elements r2 + 4 r1, r1 = 2, 3 are zero
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4_lowhalf<DIR, T, PK>(a[r2], a[r2 + 4], a[r2 + 8], a[r2 + 12]);
#pragma unroll
  for (int r2 = 1; r2 < 4; ++r2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[r2 + 4 * k1] = twc<16, DIR>(a[r2 + 4 * k1], r2 * k1);
  cplx<T> o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> t0 = a[4 * k1], t1 = a[4 * k1 + 1], t2 = a[4 * k1 + 2], t3 = a[4 * k1 + 3];
    dft4<DIR, T, PK>(t0, t1, t2, t3);
    o[k1] = t0;
    o[k1 + 4] = t1;
    o[k1 + 8] = t2;
    o[k1 + 12] = t3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = o[i];
}

// Radix-2 combine across a lane pair: mine + other on the even lane (h = 0),
// other - mine on the odd one.  For FP32 one packed fused multiply-add with
// the lane's sign (exact: a product by +-1 rounds nothing) replaces both sums
// and the select.
template <bool PK, typename T>
__device__ __forceinline__ cplx<T> s8_combine(cplx<T> mine, cplx<T> other, int h) {
  if constexpr (PK && std::is_same_v<T, float>) {
    const float sg = h ? -1.0f : 1.0f;
    const float2 r = __ffma2_rn(make_float2(mine.x, mine.y), make_float2(sg, sg), make_float2(other.x, other.y));
    return {r.x, r.y};
  } else {
    return h ? other - mine : mine + other;
  }
}

// Twiddle tables of the four-step engine (forward direction e^{+2 pi i ...},
// conjugated on use), built on the host in FP64 and rounded once:
//   lane[k*32 + l] = e^{2 pi i l k / N}          (T2, lane factor)
//   warp[a*16 + k] = e^{2 pi i 32 a k / N}       (T2, warp factor, a < W)
//   t5[k*32 + l]   = e^{2 pi i l k / TT}         (T5)
// Every read is either lane-contiguous or warp-uniform, so none conflicts.
template <typename T>
struct FourStepTables {
  const cplx<T>* lane;
  const cplx<T>* warp;
  const cplx<T>* t5;
};

// PK: the butterflies' packed FP32-pair adds (fft_reg.cuh badd / bsub)
template <typename T, int TCK = 0, bool PK = true>
struct FourStep {
  int t, TT;
  int w, l;             // warp, lane
  int W, L, J;          // warps, lines per warp, elements per line per lane
  int lgJ;              // log2(J)
  cplx<T>* sA;          // max(16*TT, W*16*34) elements, shared
  FourStepTables<T> tb; // shared-memory copies
  TcDft<TCK> tc;        // tensor-core stages (TCK > 0)

  __device__ __forceinline__ void init(int t_, int TT_, cplx<T>* s, const FourStepTables<T>& tb_) {
    t = t_;
    TT = TT_;
    w = t >> 5;
    l = t & 31;
    W = TT >> 5;
    L = 16 / W;
    J = TT >> 5;
    lgJ = 31 - __clz(J);
    sA = s;
    tb = tb_;
  }
  __device__ __forceinline__ void cta_sync() const {
    if (W > 1) __syncthreads();
    else __syncwarp();
  }
  template <int DIR>
  static __device__ __forceinline__ cplx<T> dirw(cplx<T> z) {
    if constexpr (DIR < 0) z.y = -z.y;
    return z;
  }
  // T2: v[k] *= e^{DIR 2 pi i t k / N}, t = 32 w + l.  The factors for k = 1,
  // 4, 8, 12 come from the tables, the others from at most three further
  // products with the k = 1 factor (a few ulp), which saves 22 of the 30
  // shared-memory reads of a table per k.
  template <int DIR>
  __device__ __forceinline__ void twiddleT2(cplx<T> (&v)[16]) const {
    const cplx<T> z1 = dirw<DIR>(cmul(tb.warp[w * 16 + 1], tb.lane[32 + l]));
    cplx<T> z = z1;
#pragma unroll
    for (int k = 1; k < 16; ++k) {
      if (k == 4 || k == 8 || k == 12) z = dirw<DIR>(cmul(tb.warp[w * 16 + k], tb.lane[k * 32 + l]));
      else if (k > 1) z = cmul(z, z1);
      v[k] = cmul(v[k], z);
    }
  }
  // T5: u[a*J + kj] *= e^{DIR 2 pi i l kj / TT}
  template <int DIR>
  __device__ __forceinline__ void twiddleT5(cplx<T> (&u)[16]) const {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int kj = i & (J - 1);
      if (kj) u[i] = cmul(u[i], dirw<DIR>(tb.t5[kj * 32 + l]));
    }
  }
  // line-local J-point DFTs on u[a*J + j], direction DIR
  template <int DIR>
  __device__ __forceinline__ void dftJ(cplx<T> (&u)[16]) const {
    if (J == 16) {
      dft<16, DIR, T, PK>(u);
    } else if (J == 8) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        cplx<T> q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = u[a * 8 + j];
        dft<8, DIR, T, PK>(q);
#pragma unroll
        for (int j = 0; j < 8; ++j) u[a * 8 + j] = q[j];
      }
    } else if (J == 4) {
#pragma unroll
      for (int a = 0; a < 4; ++a) dft4<DIR, T, PK>(u[a * 4], u[a * 4 + 1], u[a * 4 + 2], u[a * 4 + 3]);
    } else if (J == 2) {
#pragma unroll
      for (int a = 0; a < 8; ++a) dft2<DIR, T, PK>(u[a * 2], u[a * 2 + 1]);
    }
  }
  // shared-memory index of register a in the transposed (line) layout
  __device__ __forceinline__ int lineidx(int a) const {
    return (w * L + (a >> lgJ)) * TT + l + 32 * (a & (J - 1));
  }

  // ---- forward: registers in natural position order -> scrambled spectrum.
  // The caller guarantees that nobody still reads sA (previous use).
  template <bool LOWHALF>
  __device__ __forceinline__ void forward(cplx<T> (&v)[16]) {
    if constexpr (TCK > 0 && (kTcStages & 1)) tc.template run<-1, LOWHALF>(v, 0);
    else if constexpr (LOWHALF) dft16_lowhalf<-1, T, PK>(v);
    else dft<16, -1, T, PK>(v);
    twiddleT2<-1>(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) sA[k * TT + t] = v[k];
    cta_sync();
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = sA[lineidx(a)];
    cta_sync();
    if constexpr (TCK > 0 && (kTcStages & 2)) tc.template run<-1, false>(v, 1);
    else dftJ<-1>(v);
    twiddleT5<-1>(v);
    cplx<T>* sB = sA + w * (16 * 34);
#pragma unroll
    for (int d = 0; d < 16; ++d) sB[d * 34 + l] = v[d];
    __syncwarp();
    const int d = l >> 1, h = l & 1;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = sB[d * 34 + 2 * i + h];
    __syncwarp();
    if constexpr (TCK > 0 && (kTcStages & 4)) tc.template run<-1, false>(v, 0);
    else dft<16, -1, T, PK>(v);
    // S8: X[k] = E0[k] + w32^k E1[k], X[k+16] = E0[k] - w32^k E1[k]
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      cplx<T> mine = h ? twc<32, -1>(v[k], k) : v[k];
      cplx<T> other;
      other.x = shfl_xor(mine.x, 1);
      other.y = shfl_xor(mine.y, 1);
      v[k] = s8_combine<PK>(mine, other, h);
    }
  }
  // frequency held by register k after forward(): freq0() + 16 * J * k
  __device__ __forceinline__ int freq0() const {
    const int d = l >> 1, h = l & 1;
    const int a = d >> lgJ, kj = d & (J - 1);
    return (w * L + a) + 16 * (kj + J * 16 * h);
  }
  __device__ __forceinline__ int freq(int k) const { return freq0() + 16 * J * k; }
  // ---- inverse: scrambled spectrum -> registers in natural position order.
  // Ends with a barrier after its last shared-memory read.
  __device__ __forceinline__ void inverse(cplx<T> (&v)[16]) {
    const int d = l >> 1, h = l & 1;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      cplx<T> other;
      other.x = shfl_xor(v[k].x, 1);
      other.y = shfl_xor(v[k].y, 1);
      const cplx<T> s = s8_combine<PK>(v[k], other, h);
      v[k] = h ? twc<32, +1>(s, k) : s;
    }
    if constexpr (TCK > 0 && (kTcStages & 8)) tc.template run<+1, false>(v, 0);
    else dft<16, +1, T, PK>(v);
    cplx<T>* sB = sA + w * (16 * 34);
#pragma unroll
    for (int i = 0; i < 16; ++i) sB[d * 34 + 2 * i + h] = v[i];
    __syncwarp();
#pragma unroll
    for (int dd = 0; dd < 16; ++dd) v[dd] = sB[dd * 34 + l];
    twiddleT5<+1>(v);
    if constexpr (TCK > 0 && (kTcStages & 16)) tc.template run<+1, false>(v, 1);
    else dftJ<+1>(v);
    cta_sync();  // every warp is done with its B region before A is rewritten
#pragma unroll
    for (int a = 0; a < 16; ++a) sA[lineidx(a)] = v[a];
    cta_sync();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = sA[k * TT + t];
    cta_sync();
    twiddleT2<+1>(v);
    if constexpr (TCK > 0 && (kTcStages & 32)) tc.template run<+1, false>(v, 0);
    else dft<16, +1, T, PK>(v);
  }
};

// e^{DIR 2 pi i m / N} for 0 <= m < N, with m = 2^L hi + lo and
// L = log2(N) - 7: hi[i] = e^{2 pi i i / 128} (128 entries) and the low part
// either from a second table lo[i] = e^{2 pi i i / N} (2^L entries; FP64) or,
// for FP32, from short Taylor series: the angle 2 pi lo / N is below
// 2 pi / 128 = 0.049, so cos to theta^4 and sin to theta^5 are exact to
// 2e-11, well below FP32 rounding, and the table read becomes a few FMAs.
template <typename T>
struct Twiddles2L {
  const cplx<T>* hi;
  const cplx<T>* lo;
  int L;
  T dtheta;  // 2 pi / N
  template <int DIR>
  __device__ __forceinline__ cplx<T> get(int m) const {
    const cplx<T> a = hi[m >> L];
    cplx<T> b;
    if constexpr (sizeof(T) == 4) {
      const T th = (T)(m & ((1 << L) - 1)) * dtheta, t2 = th * th;
      b.x = fmaf(t2, fmaf(t2, 1.0f / 24.0f, -0.5f), 1.0f);
      b.y = th * fmaf(t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    } else {
      b = lo[m & ((1 << L) - 1)];
    }
    cplx<T> z = cmul(a, b);
    if constexpr (DIR < 0) z.y = -z.y;
    return z;
  }
};

}  // namespace bemfft
