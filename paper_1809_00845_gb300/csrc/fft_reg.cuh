// Register-resident mixed-radix Stockham FFT for one line per CTA (sm_103a).
//
// A length-N line (N a power of two) is spread over TT = N/E threads, thread t
// holding the E elements at positions t + m*TT (m = 0..E-1) in registers.  A
// pass of radix R (R | E) performs E/R butterflies per thread: butterfly
// b = t + s*TT reads positions b + r*N/R, i.e. registers s + r*E/R, so the
// register <-> position map is the same in every pass.  Between passes the
// data goes through shared memory (Stockham autosort order, padded by one
// element every 16 to keep both the strided writes of the first pass and
// the unit-stride reads conflict-free).  The last pass writes its outputs
// back in place: afterwards register m holds frequency t + m*TT in natural
// order, which is exactly the register map the first pass of the inverse
// transform reads.  That lets the spectral multiply (Eq. 16) run on registers
// between the forward and inverse transforms with no shared-memory round trip.
//
// Twiddles come from a quarter-wave table of e^{2 pi i r/N}, r in [0, N/4),
// computed in FP64 on the host and rounded once to the working precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ff.cuh"

namespace bemfft {

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T x, y;
};

// lane exchange of one real of the working type (float, double, or a
// double-float pair, moved as its two floats)
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <typename P>
__device__ __forceinline__ P shfl_xor(P v, int m) {
  return P(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return {a.x * s, a.y * s}; }

// Complex add and subtract.  For FP32 both parts go through one packed
// FP32-pair instruction (sm_100 and later), the same IEEE round-to-nearest
// sums as two scalar adds in half the issue slots; the butterflies below use
// them wherever both parts take the same operation.
__device__ __forceinline__ cplx<float> padd(cplx<float> a, cplx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return {r.x, r.y};
}
__device__ __forceinline__ cplx<float> psub(cplx<float> a, cplx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  return {r.x, r.y};
}
// Complex double-float add and subtract with the real and imaginary parts'
// FP32 steps paired into packed instructions: each part sees the scalar
// double-float add's operations in the same order (bitwise the same result)
// in half the issue slots.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ cplx<f32x2> ffc_add(float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 s = f2add(ah, bh), bb = f2sub(s, ah);
  float2 e = f2add(f2sub(ah, f2sub(s, bb)), f2sub(bh, bb));
  e = f2add(e, f2add(al, bl));
  const float2 rh = f2add(s, e), rl = f2sub(e, f2sub(rh, s));
  return {f32x2(rh.x, rl.x), f32x2(rh.y, rl.y)};
}
__device__ __forceinline__ cplx<f32x2> padd(cplx<f32x2> a, cplx<f32x2> b) {
  return ffc_add(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo), make_float2(b.x.hi, b.y.hi),
                 make_float2(b.x.lo, b.y.lo));
}
__device__ __forceinline__ cplx<f32x2> psub(cplx<f32x2> a, cplx<f32x2> b) {
  return ffc_add(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo), make_float2(-b.x.hi, -b.y.hi),
                 make_float2(-b.x.lo, -b.y.lo));
}
// Packed double-float product, lane by lane a * b (Dekker's product: the
// scalar double-float multiply's steps in the same order), and the complex
// double-float products built on it.  (For FP32 the packed complex product
// was measured slower than four scalar operations: its operands need
// broadcast and swapped register pairs.)
__device__ __forceinline__ void ffp_mul(float2 ah, float2 al, float2 bh, float2 bl, float2& rh, float2& rl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  rh = f2add(p, e);
  rl = f2sub(e, f2sub(rh, p));
}
__device__ __forceinline__ cplx<f32x2> cmul(cplx<f32x2> a, cplx<f32x2> b) {
  float2 ph, pl, qh, ql;
  ffp_mul(make_float2(a.x.hi, a.x.hi), make_float2(a.x.lo, a.x.lo), make_float2(b.x.hi, b.y.hi),
          make_float2(b.x.lo, b.y.lo), ph, pl);
  ffp_mul(make_float2(a.y.hi, a.y.hi), make_float2(a.y.lo, a.y.lo), make_float2(-b.y.hi, b.x.hi),
          make_float2(-b.y.lo, b.x.lo), qh, ql);
  return ffc_add(ph, pl, qh, ql);
}
__device__ __forceinline__ cplx<f32x2> cscale(cplx<f32x2> a, f32x2 s) {
  float2 rh, rl;
  ffp_mul(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo), make_float2(s.hi, s.hi), make_float2(s.lo, s.lo),
          rh, rl);
  return {f32x2(rh.x, rl.x), f32x2(rh.y, rl.y)};
}
// s + a * w (real a first: the x-DFT row sums)
__device__ __forceinline__ cplx<f32x2> cmacr(cplx<f32x2> s, f32x2 a, cplx<f32x2> w) {
  float2 rh, rl;
  ffp_mul(make_float2(a.hi, a.hi), make_float2(a.lo, a.lo), make_float2(w.x.hi, w.y.hi), make_float2(w.x.lo, w.y.lo),
          rh, rl);
  return ffc_add(make_float2(s.x.hi, s.y.hi), make_float2(s.x.lo, s.y.lo), rh, rl);
}
// y + v * s (complex v first: the spectral multiply)
__device__ __forceinline__ cplx<f32x2> cmacc(cplx<f32x2> y, cplx<f32x2> v, f32x2 s) {
  float2 rh, rl;
  ffp_mul(make_float2(v.x.hi, v.y.hi), make_float2(v.x.lo, v.y.lo), make_float2(s.hi, s.hi), make_float2(s.lo, s.lo),
          rh, rl);
  return ffc_add(make_float2(y.x.hi, y.y.hi), make_float2(y.x.lo, y.y.lo), rh, rl);
}
// Re(a b) and Re(a conj(b)) (the gathers' output-pruned inverse DFT terms),
// with the two products paired
__device__ __forceinline__ f32x2 cdot_re(cplx<f32x2> a, cplx<f32x2> b) {
  float2 rh, rl;
  ffp_mul(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo), make_float2(b.x.hi, b.y.hi),
          make_float2(b.x.lo, b.y.lo), rh, rl);
  return f32x2(rh.x, rl.x) - f32x2(rh.y, rl.y);
}
__device__ __forceinline__ f32x2 cdot_rc(cplx<f32x2> a, cplx<f32x2> b) {
  float2 rh, rl;
  ffp_mul(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo), make_float2(b.x.hi, b.y.hi),
          make_float2(b.x.lo, b.y.lo), rh, rl);
  return f32x2(rh.x, rl.x) + f32x2(rh.y, rl.y);
}
template <typename T>
__device__ __forceinline__ cplx<T> padd(cplx<T> a, cplx<T> b) { return a + b; }
template <typename T>
__device__ __forceinline__ cplx<T> psub(cplx<T> a, cplx<T> b) { return a - b; }

// Butterfly add / subtract: packed (PK) or the plain complex operators.  The
// kernels pick the form per instantiation (the packed adds cost the
// accuracy mode's edge-flow column kernel 2% while they speed up the others).
template <bool PK, typename T>
__device__ __forceinline__ cplx<T> badd(cplx<T> a, cplx<T> b) {
  if constexpr (PK) return padd(a, b);
  else return a + b;
}
template <bool PK, typename T>
__device__ __forceinline__ cplx<T> bsub(cplx<T> a, cplx<T> b) {
  if constexpr (PK) return psub(a, b);
  else return a - b;
}

// s + a * w and y + v * s for complex s, w, y, v and real a, s (the packed
// double-float forms above keep these operand orders)
template <typename T>
__device__ __forceinline__ cplx<T> cmacr(cplx<T> s, T a, cplx<T> w) {
  return {s.x + a * w.x, s.y + a * w.y};
}
template <typename T>
__device__ __forceinline__ cplx<T> cmacc(cplx<T> y, cplx<T> v, T s) {
  return {y.x + v.x * s, y.y + v.y * s};
}
template <typename T>
__device__ __forceinline__ T cdot_re(cplx<T> a, cplx<T> b) {
  return a.x * b.x - a.y * b.y;
}
template <typename T>
__device__ __forceinline__ T cdot_rc(cplx<T> a, cplx<T> b) {
  return a.x * b.x + a.y * b.y;
}

// multiply by e^{DIR i pi/2} = DIR * i
template <int DIR, typename T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> a) {
  if constexpr (DIR > 0) return {-a.y, a.x};
  else return {a.y, -a.x};
}

// cos and sin of 2 pi j / 32 (j = 0..8); other octants by symmetry.
__device__ __forceinline__ double cos32(int j) {
  switch (j) {
    case 0: return 1.0;
    case 1: return 0.98078528040323044913;
    case 2: return 0.92387953251128675613;
    case 3: return 0.83146961230254523708;
    case 4: return 0.70710678118654752440;
    case 5: return 0.55557023301960222474;
    case 6: return 0.38268343236508977173;
    case 7: return 0.19509032201612826785;
    default: return 0.0;
  }
}

// a * e^{DIR 2 pi i m / R} for a compile-time-foldable m (after unrolling).
template <int R, int DIR, typename T>
__device__ __forceinline__ cplx<T> twc(cplx<T> a, int m) {
  m = m % R;
  if (m == 0) return a;
  if (4 * m == R) return mul_i<DIR>(a);
  if (2 * m == R) return {-a.x, -a.y};
  if (4 * m == 3 * R) return mul_i<-DIR>(a);
  const int j = (32 / R) * m;  // angle 2 pi j / 32
  const int q = j >> 3, r = j & 7;
  // e^{i 2 pi j/32} = i^q e^{i 2 pi r/32}
  T c = (T)cos32(r), s = (T)cos32(8 - r);
  cplx<T> w;
  if (q == 0) w = {c, s};
  else if (q == 1) w = {-s, c};
  else if (q == 2) w = {-c, -s};
  else w = {s, -c};
  if (DIR < 0) w.y = -w.y;
  if (r == 4) {
    // (+-h +- i h): two multiplies
    const T hh = (T)0.70710678118654752440;
    T sx = w.x > 0 ? (T)1 : (T)-1, sy = w.y > 0 ? (T)1 : (T)-1;
    // (a.x + i a.y)(sx h + i sy h) = h[(sx a.x - sy a.y) + i(sy a.x + sx a.y)]
    T re = sx * a.x - sy * a.y, im = sy * a.x + sx * a.y;
    return {re * hh, im * hh};
  }
  return cmul(a, w);
}

template <int DIR, typename T, bool PK = true>
__device__ __forceinline__ void dft2(cplx<T>& a, cplx<T>& b) {
  cplx<T> t = a;
  a = badd<PK>(t, b);
  b = bsub<PK>(t, b);
}

template <int DIR, typename T, bool PK = true>
__device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  const cplx<T> s0 = badd<PK>(a0, a2), d0 = bsub<PK>(a0, a2), s1 = badd<PK>(a1, a3), e1 = bsub<PK>(a1, a3);
  a0 = badd<PK>(s0, s1);
  a2 = bsub<PK>(s0, s1);
  // a1 = d0 + DIR i e1, a3 = d0 - DIR i e1: the rotation swaps e1's parts, so
  // these four sums stay scalar
  if constexpr (DIR > 0) {
    a1 = {d0.x - e1.y, d0.y + e1.x};
    a3 = {d0.x + e1.y, d0.y - e1.x};
  } else {
    a1 = {d0.x + e1.y, d0.y - e1.x};
    a3 = {d0.x - e1.y, d0.y + e1.x};
  }
}

// In-place DFT of R registers: a[k] <- sum_r a[r] e^{DIR 2 pi i r k / R}.
// R = R1 * R2 split: R1-point DFTs on stride-R2 subsequences, twiddles,
// R2-point DFTs, transposed read-out (register renaming after unrolling).
template <int R, int DIR, typename T, bool PK = true>
__device__ __forceinline__ void dft(cplx<T> (&a)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<DIR, T, PK>(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4<DIR, T, PK>(a[0], a[1], a[2], a[3]);
  } else {
    constexpr int R1 = 4;
    constexpr int R2 = R / R1;
#pragma unroll
    for (int r2 = 0; r2 < R2; ++r2) {
      cplx<T> t[R1];
#pragma unroll
      for (int r1 = 0; r1 < R1; ++r1) t[r1] = a[r2 + R2 * r1];
      dft<R1, DIR, T, PK>(t);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[r2 + R2 * k1] = t[k1];
    }
#pragma unroll
    for (int r2 = 1; r2 < R2; ++r2)
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[r2 + R2 * k1] = twc<R, DIR>(a[r2 + R2 * k1], r2 * k1);
    cplx<T> o[R];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cplx<T> t[R2];
#pragma unroll
      for (int r2 = 0; r2 < R2; ++r2) t[r2] = a[r2 + R2 * k1];
      dft<R2, DIR, T, PK>(t);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) o[k1 + R1 * k2] = t[k2];
    }
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = o[i];
  }
}

// Quarter-wave twiddle table of e^{2 pi i r / N}, r < N/4.
template <typename T>
struct Twiddles {
  const cplx<T>* q;  // N/4 entries (shared or global)
  int log2q;         // log2(N/4)
  // e^{DIR 2 pi i m / N} for m in [0, N)
  template <int DIR>
  __device__ __forceinline__ cplx<T> get(int m) const {
    const int quad = m >> log2q;
    const cplx<T> t = q[m & ((1 << log2q) - 1)];
    cplx<T> w;
    // rotate by i^quad
    w.x = (quad & 1) ? -t.y : t.x;
    w.y = (quad & 1) ? t.x : t.y;
    if (quad & 2) {
      w.x = -w.x;
      w.y = -w.y;
    }
    if constexpr (DIR < 0) w.y = -w.y;
    return w;
  }
};

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// One Stockham pass of radix R on the register set v (E per thread).
// Ns: product of the radices of the previous passes.  If LAST, outputs stay
// in registers (natural order); otherwise they go to smem and are read back.
// Barrier between Stockham passes: the whole CTA (one line per CTA) or, with
// WARP, the warp (lines of at most 32 threads, several lines per CTA).
template <bool WARP>
__device__ __forceinline__ void line_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

template <int E, int R, int DIR, bool LAST, typename T, bool WARP = false>
__device__ __forceinline__ void stockham_pass(cplx<T> (&v)[E], const int t, const int TT, const int log2Ns,
                                              const int log2N, const Twiddles<T>& tw, cplx<T>* sbuf) {
  constexpr int S = E / R;
  constexpr int LR = (R == 32) ? 5 : (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : (R == 2) ? 1 : 0;
  const int Ns = 1 << log2Ns;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int b = t + s * TT;
    const int k = b & (Ns - 1);
    cplx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = v[s + r * S];
    if (Ns > 1) {
      // twiddle e^{DIR 2 pi i k r / (Ns R)} = table index k r N/(Ns R) < N
      const int m1 = k << (log2N - log2Ns - LR);
#pragma unroll
      for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw.template get<DIR>(m1 * r));
    }
    dft<R, DIR>(u);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[s + r * S] = u[r];
    } else {
      const int base = (b - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sbuf[pad16(base + r * Ns)] = u[r];
    }
  }
  if constexpr (!LAST) {
    line_sync<WARP>();
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = sbuf[pad16(t + m * TT)];
    line_sync<WARP>();
  }
}

// Full transform of one line held in registers (positions t + m*TT) with
// radix-E passes followed by one smaller last pass when log2(N) is not a
// multiple of log2(E).  Result in natural order in the same register map.
template <int E, int DIR, typename T, bool WARP = false>
__device__ __forceinline__ void fft_line(cplx<T> (&v)[E], const int t, const int TT, const int log2N,
                                         const Twiddles<T>& tw, cplx<T>* sbuf) {
  constexpr int LE = (E == 16) ? 4 : (E == 8) ? 3 : (E == 4) ? 2 : 1;
  const int full = log2N / LE;       // number of radix-E passes possible
  const int rem = log2N - full * LE;  // leftover bits
  // passes: (full - (rem == 0)) radix-E passes not last, then the last pass of radix E or 2^rem
  const int nfirst = rem == 0 ? full - 1 : full;
  int lNs = 0;
  for (int p = 0; p < nfirst; ++p) {
    stockham_pass<E, E, DIR, false, T, WARP>(v, t, TT, lNs, log2N, tw, sbuf);
    lNs += LE;
  }
  if (rem == 0) {
    stockham_pass<E, E, DIR, true, T, WARP>(v, t, TT, lNs, log2N, tw, sbuf);
  } else if (rem == 1) {
    stockham_pass<E, 2, DIR, true, T, WARP>(v, t, TT, lNs, log2N, tw, sbuf);
  } else if (rem == 2) {
    if constexpr (E >= 4) stockham_pass<E, 4, DIR, true, T, WARP>(v, t, TT, lNs, log2N, tw, sbuf);
  } else if (rem == 3) {
    if constexpr (E >= 8) stockham_pass<E, 8, DIR, true, T, WARP>(v, t, TT, lNs, log2N, tw, sbuf);
  }
}

}  // namespace bemfft
