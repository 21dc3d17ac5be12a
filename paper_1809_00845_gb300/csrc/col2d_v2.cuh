// Four-step column kernel of the 2D apply (Section 3-4, Eq. 15-16).
//
// For N >= 512.  Thread t owns the contiguous range of sorted cells
// [chunk[t], chunk[t+1]) (equal cell counts, fixed at plan time; a grid row
// may be split between neighbouring threads).  Per-cell arrays (cell words,
// density pairs, accumulators) are stored interleaved: the i-th cell of
// thread t sits at position i*TT + t, so every warp-wide access of the cell
// loops is one contiguous segment.  Per column kx:
//   1. the thread walks its cells (loads and twiddles batched CB at a time) and
//      forms the input-pruned x-DFT of every field row by row.  A row sum is
//      stored when the row's last cell in the chunk is reached (flag in the
//      cell word): into shared memory at the row's slot (rowslot), field 0
//      into the transform buffer,
//      fields 1.. into staging rows), or, for the first row of a chunk that
//      began in an earlier chunk, into the thread's carry slot.  Empty rows
//      are never written: the transform input masks them (a per-thread bit
//      mask of its eight rows).  After a barrier, the thread holding the
//      first cell of a split row adds the carries of the following threads
//      in thread order (deterministic);
//   2. each field is loaded into the four-step engine's register map
//      (rows t + m*TT), transformed, multiplied by the spectrum column (copied
//      to shared memory asynchronously during the transform) and accumulated;
//   3. the inverse transform leaves rows t + m*TT in registers, they are
//      written to shared memory and every thread gathers its own cells
//      (output-pruned inverse x-DFT) into its accumulators.
// In the kernels that keep every field's row sums in shared memory (FP32 with
// two or three fields) steps 3 and 1 of consecutive columns share one walk
// over the cells (walk_cells): the gather of the CTA's previous column and the
// row sums of the current one, with the sparse twiddles of the current column
// from two 64-entry tables built per column; the CTA's last column is
// gathered after its loop.
//
// Included only by the translation units that instantiate Col2DKernels.
#pragma once

#include "col2d_v2.h"
#include "fft4step.cuh"

namespace bemfft {

__device__ __forceinline__ int meta_x(uint32_t m) { return (int)(m & 0xfffu); }
__device__ __forceinline__ int meta_slot(uint32_t m) { return (int)((m >> 12) & 0xfffu); }  // rowslot(row)
__device__ __forceinline__ int swz16(int i) { return i + (i >> 4); }

constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v / 2); }

// Sizes of one launch: compile-time when TTC > 0, else from the launch and
// the parameters.
template <int TTC>
struct ColDims {
  int TT, log2N, N, n;
  template <typename T>
  __device__ __forceinline__ explicit ColDims(const Col2Dv2Params<T>& p) {
    if constexpr (TTC > 0) {
      TT = TTC;
      log2N = 4 + clog2(TTC);
      N = 16 * TTC;
      n = 8 * TTC;
    } else {
      TT = (int)blockDim.x;
      log2N = p.log2N;
      N = 1 << p.log2N;
      n = p.n;
    }
  }
};

// Walk the thread's cnt cells and store the x-DFT row sums of the selected
// fields: FSEL < 0 = all NF fields (field 0 -> out0[row], field f > 0 ->
// outF[(f-1)*n + row]); FSEL >= 0 = that field only -> out0.  Carried sums go
// to carry[f*TT + t] (f = 0 for FSEL >= 0).
// EDGE (NF = 2): every cell carries the triple (charge a, x-edge flow b,
// y-edge flow c; c from val2); a and b are summed separately and a row is
// stored as sum(a) + fx * sum(b) (fx = e^{-2 pi i kx / N} - 1, the x-difference
// in this column), c as field 1.
template <typename T, int NF, int FSEL, int TTC, bool EDGE = false>
__device__ __forceinline__ void sparse_rows(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int kx, int cnt,
                                            cplx<T>* out0, cplx<T>* outF, cplx<T>* carry,
                                            const Twiddles2L<T>& tw, cplx<T>* twc, cplx<T> fx = {T(0), T(0)}) {
  const int Nm = g.N - 1;
  const int t = threadIdx.x, TT = g.TT;
  cplx<T> s0 = {T(0), T(0)}, s1 = {T(0), T(0)}, s2 = {T(0), T(0)};
  uint32_t mn[CB];
  cplx<T> vn[CB];
  T cn[CB];
  if (cnt > 0) {
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int pos = (i < cnt ? i : cnt - 1) * TT + t;
      mn[i] = __ldg(p.meta + pos);
      vn[i] = p.val[pos];
      if constexpr (EDGE) cn[i] = p.val2[pos];
    }
  }
  for (int i0 = 0; i0 < cnt; i0 += CB) {
    uint32_t mt[CB];
    cplx<T> vv[CB], w[CB];
    T cc3[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      mt[i] = mn[i];
      vv[i] = vn[i];
      if constexpr (EDGE) cc3[i] = cn[i];
    }
    if (i0 + CB < cnt) {
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int pos = (i0 + CB + i < cnt ? i0 + CB + i : cnt - 1) * TT + t;
        mn[i] = __ldg(p.meta + pos);
        vn[i] = p.val[pos];
        if constexpr (EDGE) cn[i] = p.val2[pos];
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) w[i] = tw.template get<-1>((kx * meta_x(mt[i])) & Nm);
    if (twc) {
      // kept for the gather of the same column (the conjugate twiddle)
#pragma unroll
      for (int i = 0; i < CB; ++i)
        if (i0 + i < cnt) twc[(i0 + i) * TT + t] = w[i];
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      if (EDGE && i0 + i < cnt) {
        if (FSEL <= 0) {
          s0.x += vv[i].x * w[i].x;
          s0.y += vv[i].x * w[i].y;
          s1.x += vv[i].y * w[i].x;
          s1.y += vv[i].y * w[i].y;
        }
        if (FSEL < 0 || FSEL == 1) {
          s2.x += cc3[i] * w[i].x;
          s2.y += cc3[i] * w[i].y;
        }
        if (mt[i] & kMetaFlush) {
          const int row = meta_slot(mt[i]);
          const bool car = (mt[i] & kMetaCarry) != 0;
          if (FSEL < 0) {
            (car ? carry + t : out0 + row)[0] = s0 + cmul(fx, s1);
            (car ? carry + TT + t : outF + row)[0] = s2;
          } else {
            (car ? carry + t : out0 + row)[0] = FSEL == 0 ? s0 + cmul(fx, s1) : s2;
          }
          s0 = s1 = s2 = {T(0), T(0)};
        }
      } else if (!EDGE && i0 + i < cnt) {
        const bool ty = (mt[i] >> 31) != 0;
        const T a = vv[i].x, b = vv[i].y;
        const T ca = ty ? T(0) : a, cb = ty ? a : b, cc = ty ? b : T(0);
        if (FSEL < 0 || FSEL == 0) {
          s0.x += ca * w[i].x;
          s0.y += ca * w[i].y;
        }
        if ((FSEL < 0 && NF > 1) || FSEL == 1) {
          s1.x += cb * w[i].x;
          s1.y += cb * w[i].y;
        }
        if ((FSEL < 0 && NF > 2) || FSEL == 2) {
          s2.x += cc * w[i].x;
          s2.y += cc * w[i].y;
        }
        if (mt[i] & kMetaFlush) {
          const int row = meta_slot(mt[i]);
          const bool car = (mt[i] & kMetaCarry) != 0;
          if (FSEL < 0) {
            (car ? carry + t : out0 + row)[0] = s0;
            if (NF > 1) (car ? carry + TT + t : outF + row)[0] = s1;
            if (NF > 2) (car ? carry + 2 * TT + t : outF + g.n + row)[0] = s2;
          } else {
            (car ? carry + t : out0 + row)[0] = FSEL == 0 ? s0 : (FSEL == 1 ? s1 : s2);
          }
          s0 = s1 = s2 = {T(0), T(0)};
        }
      }
    }
  }
}

// After a barrier: the thread holding the first cell of a split row (its
// last row) adds the carries of the `ncont` following threads, in order.
template <typename T, int NF, int FSEL, int TTC>
__device__ __forceinline__ void add_carries(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int cnt, int ncont,
                                            cplx<T>* out0, cplx<T>* outF, const cplx<T>* carry) {
  if (ncont == 0) return;
  const int t = threadIdx.x, TT = g.TT;
  const int row = meta_slot(__ldg(p.meta + (cnt - 1) * TT + t));
  constexpr int nfs = FSEL < 0 ? NF : 1;
#pragma unroll
  for (int f = 0; f < nfs; ++f) {
    cplx<T>* dst = f == 0 ? out0 + row : outF + (size_t)(f - 1) * g.n + row;
    cplx<T> s = *dst;
    for (int i = 1; i <= ncont; ++i) s = s + carry[f * TT + t + i];
    *dst = s;
  }
}

// accumulators: rows i < qs of the thread's cells in shared memory (sacc), the
// rest in the CTA's slice of the partial sums (gacc); the row index is the
// same for every lane of a warp, so the choice never diverges
template <typename T>
__device__ __forceinline__ T* acc_at(T* sacc, T* gacc, int qs, int i, int TT, int t) {
  return (i < qs ? sacc : gacc) + (size_t)i * TT + t;
}

template <typename T, int TTC>
__device__ __forceinline__ void gather_cells(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int kx, int cnt,
                                             const cplx<T>* rows, const Twiddles2L<T>& tw, T* sacc, T* gacc,
                                             int qs, const cplx<T>* twc) {
  const int Nm = g.N - 1;
  const int t = threadIdx.x, TT = g.TT;
  const T ckx = (kx == 0 || kx == g.n) ? T(1) : T(2);
  uint32_t mn[CB];
  cplx<T> wn[CB];
  if (cnt > 0) {
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const int pos = (i < cnt ? i : cnt - 1) * TT + t;
      mn[i] = __ldg(p.meta + pos);
      if (twc) wn[i] = twc[pos];
    }
  }
  for (int i0 = 0; i0 < cnt; i0 += CB) {
    uint32_t mt[CB];
    cplx<T> Y[CB], w[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      mt[i] = mn[i];
      if (twc) w[i] = wn[i];  // the sparse pass's e^{-i...}: conjugated below
    }
    if (i0 + CB < cnt) {
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const int pos = (i0 + CB + i < cnt ? i0 + CB + i : cnt - 1) * TT + t;
        mn[i] = __ldg(p.meta + pos);
        if (twc) wn[i] = twc[pos];
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      Y[i] = rows[meta_slot(mt[i])];
      if (twc) w[i].y = -w[i].y;
      else w[i] = tw.template get<+1>((kx * meta_x(mt[i])) & Nm);
    }
#pragma unroll
    for (int i = 0; i < CB; ++i)
      if (i0 + i < cnt) *acc_at(sacc, gacc, qs, i0 + i, TT, t) += ckx * cdot_re(Y[i], w[i]);
  }
}

// Per-column sparse twiddles of the fused walk (kColTwEntries entries):
// stw[j] = e^{-2 pi i kx j / N} and stw[64 + j] = e^{-2 pi i kx 64 j / N}
// (j < 64), so a cell at x < 4096 takes stw[64 + (x >> 6)] * stw[x & 63]:
// two table reads and one product instead of the table-and-series twiddle.
template <typename T, int TTC>
__device__ __forceinline__ void column_twiddles(const ColDims<TTC>& g, int kx, const Twiddles2L<T>& tw,
                                                cplx<T>* stw) {
  const int Nm = g.N - 1;
  for (int i = threadIdx.x; i < kColTwEntries; i += g.TT) {
    const int j = i & 63;
    stw[i] = tw.template get<-1>((kx * (i < 64 ? j : 64 * j)) & Nm);
  }
}

// One batch of NB cells of a walk: cell words, densities (EDGE: and the third
// density) and the cached twiddles of the previous column.
template <typename T, int NB>
struct CellBatch {
  uint32_t m[NB];
  cplx<T> v[NB], w[NB];
  T c[NB], a[NB];
};

// One walk over the thread's cells that serves two columns (kernels with the
// field sums in shared memory): GATHER adds the output-pruned inverse x-DFT
// of the previous column kxp (its rows already scaled by the column weight, 1
// or 2) into the accumulators, SPARSE forms the x-DFT row sums of every field
// for column kx (as sparse_rows with FSEL < 0; field 0 to out0 at the row
// slot), with the twiddles of the column's tables stw.  The cell words are
// loaded once for both; the gather's twiddle is column kxp's cached one
// (conjugated), which the sparse pass then replaces by column kx's.  Sums and
// accumulators see the same terms in the same order as the separate passes.
// Batches of NB cells (2 or 4, a launch shape the tuner picks); the next
// batch's loads are issued before the current batch is used (two alternating
// register sets spill in the 512-thread kernels); the cell arrays hold a
// multiple of 4 cells per thread, so every batch load stays inside them.
template <typename T, int NF, int TTC, bool EDGE, bool SPARSE, bool GATHER, int NB>
__device__ __forceinline__ void walk_cells(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int kxp, int cnt,
                                           cplx<T>* out0, cplx<T>* outF, cplx<T>* carry, const cplx<T>* rows,
                                           T* sacc, T* gacc, int qs, const Twiddles2L<T>& tw, const cplx<T>* stw,
                                           cplx<T>* twc, cplx<T> fx) {
  const int Nm = g.N - 1;
  const int t = threadIdx.x, TT = g.TT;
  cplx<T> s0 = {T(0), T(0)}, s1 = {T(0), T(0)}, s2 = {T(0), T(0)};
  auto fetch = [&](CellBatch<T, NB>& B, int base) {
    const int pos = base * TT + t;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      B.m[i] = __ldg(p.meta + pos + i * TT);
      if constexpr (SPARSE) {
        B.v[i] = p.val[pos + i * TT];
        if constexpr (EDGE) B.c[i] = p.val2[pos + i * TT];
      }
      if constexpr (GATHER) {
        if (twc) B.w[i] = twc[pos + i * TT];
      }
    }
    // accumulator rows kept in the partial sums (not in shared memory) are
    // read with the batch, so their L2 round trip overlaps the batch before.
    // Only in the edge-flow kernels (the accuracy mode's node plans, whose
    // ~100 nodes a thread overflow shared memory): it costs the paper-form
    // star kernel, whose rows all fit, 5 us in register allocation.
    if constexpr (GATHER && EDGE) {
      if (base + NB > qs) {
#pragma unroll
        for (int i = 0; i < NB; ++i) B.a[i] = base + i >= qs ? gacc[(size_t)(base + i) * TT + t] : T(0);
      }
    }
  };
  auto process = [&](CellBatch<T, NB>& B, int i0) {
    if constexpr (GATHER) {
      cplx<T> Y[NB], wp[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        Y[i] = rows[meta_slot(B.m[i])];
        if (twc) wp[i] = {B.w[i].x, -B.w[i].y};
        else wp[i] = tw.template get<+1>((kxp * meta_x(B.m[i])) & Nm);
      }
      if (i0 + NB <= qs) {
        T* acc = sacc + (size_t)i0 * TT + t;
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (i0 + i < cnt) acc[i * TT] += Y[i].x * wp[i].x - Y[i].y * wp[i].y;
      } else if constexpr (EDGE) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i0 + i >= cnt) continue;
          const T term = Y[i].x * wp[i].x - Y[i].y * wp[i].y;
          if (i0 + i < qs) sacc[(size_t)(i0 + i) * TT + t] += term;
          else gacc[(size_t)(i0 + i) * TT + t] = B.a[i] + term;
        }
      } else {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (i0 + i < cnt) *acc_at(sacc, gacc, qs, i0 + i, TT, t) += Y[i].x * wp[i].x - Y[i].y * wp[i].y;
      }
    }
    if constexpr (SPARSE) {
      cplx<T> w[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) w[i] = cmul(stw[64 + ((B.m[i] >> 6) & 63)], stw[B.m[i] & 63]);
      if (twc) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (i0 + i < cnt) twc[(i0 + i) * TT + t] = w[i];
      }
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i0 + i >= cnt) continue;
        const uint32_t mt = B.m[i];
        if constexpr (EDGE) {
          s0.x += B.v[i].x * w[i].x;
          s0.y += B.v[i].x * w[i].y;
          s1.x += B.v[i].y * w[i].x;
          s1.y += B.v[i].y * w[i].y;
          s2.x += B.c[i] * w[i].x;
          s2.y += B.c[i] * w[i].y;
          if (mt & kMetaFlush) {
            const int row = meta_slot(mt);
            const bool car = (mt & kMetaCarry) != 0;
            (car ? carry + t : out0 + row)[0] = s0 + cmul(fx, s1);
            (car ? carry + TT + t : outF + row)[0] = s2;
            s0 = s1 = s2 = {T(0), T(0)};
          }
        } else {
          const bool ty = (mt >> 31) != 0;
          const T a = B.v[i].x, b = B.v[i].y;
          const T ca = ty ? T(0) : a, cb = ty ? a : b, cc = ty ? b : T(0);
          s0.x += ca * w[i].x;
          s0.y += ca * w[i].y;
          if (NF > 1) {
            s1.x += cb * w[i].x;
            s1.y += cb * w[i].y;
          }
          if (NF > 2) {
            s2.x += cc * w[i].x;
            s2.y += cc * w[i].y;
          }
          if (mt & kMetaFlush) {
            const int row = meta_slot(mt);
            const bool car = (mt & kMetaCarry) != 0;
            (car ? carry + t : out0 + row)[0] = s0;
            if (NF > 1) (car ? carry + TT + t : outF + row)[0] = s1;
            if (NF > 2) (car ? carry + 2 * TT + t : outF + g.n + row)[0] = s2;
            s0 = s1 = s2 = {T(0), T(0)};
          }
        }
      }
    }
  };
  CellBatch<T, NB> A, B;
  if (cnt > 0) fetch(B, 0);
  for (int i0 = 0; i0 < cnt; i0 += NB) {
    A = B;
    if (i0 + NB < cnt) fetch(B, i0 + NB);
    process(A, i0);
  }
}

// One walk over the thread's cells for the kernels that take the fields one at
// a time (FP64, double-float, one field): SPARSE forms the x-DFT row sums of
// field FSEL of column kx (as sparse_rows; to out0 at the row slot), GATHER
// adds the output-pruned inverse x-DFT of the field transformed before it in
// the same column from its rows (scaled by the column weight) into the
// accumulators.  Both use the column's sparse twiddle: the first walk of a
// column (FIRST) evaluates it and keeps it in the cache, the later walks read
// it there (or evaluate it again when there is no cache).
template <typename T, int NF, int FSEL, int TTC, bool EDGE, bool SPARSE, bool GATHER, bool FIRST>
__device__ __forceinline__ void walk_field(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int kx, int cnt,
                                           cplx<T>* out0, cplx<T>* carry, const cplx<T>* rows, T* sacc, T* gacc,
                                           int qs, const Twiddles2L<T>& tw, cplx<T>* twc, cplx<T> fx) {
  static_assert(!(FIRST && GATHER), "the first walk of a column gathers nothing");
  const int Nm = g.N - 1;
  const int t = threadIdx.x, TT = g.TT;
  const bool cached = !FIRST && twc != nullptr;
  cplx<T> s0 = {T(0), T(0)}, s1 = {T(0), T(0)}, s2 = {T(0), T(0)};
  uint32_t mn[CB];
  cplx<T> vn[CB], wn[CB];
  T cn[CB];
  auto fetch = [&](int base) {
    const int pos = base * TT + t;
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      mn[i] = __ldg(p.meta + pos + i * TT);
      if constexpr (SPARSE) {
        vn[i] = p.val[pos + i * TT];
        if constexpr (EDGE) cn[i] = p.val2[pos + i * TT];
      }
      if (cached) wn[i] = twc[pos + i * TT];
    }
  };
  if (cnt > 0) fetch(0);
  for (int i0 = 0; i0 < cnt; i0 += CB) {
    uint32_t mt[CB];
    cplx<T> vv[CB], w[CB];
    T cc3[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      mt[i] = mn[i];
      if constexpr (SPARSE) {
        vv[i] = vn[i];
        if constexpr (EDGE) cc3[i] = cn[i];
      }
      if (cached) w[i] = wn[i];
    }
    if (i0 + CB < cnt) fetch(i0 + CB);
    if (!cached) {
#pragma unroll
      for (int i = 0; i < CB; ++i) w[i] = tw.template get<-1>((kx * meta_x(mt[i])) & Nm);
      if (FIRST && twc) {
#pragma unroll
        for (int i = 0; i < CB; ++i)
          if (i0 + i < cnt) twc[(i0 + i) * TT + t] = w[i];
      }
    }
    if constexpr (GATHER) {
      cplx<T> Y[CB];
#pragma unroll
      for (int i = 0; i < CB; ++i) Y[i] = rows[meta_slot(mt[i])];
#pragma unroll
      for (int i = 0; i < CB; ++i)
        if (i0 + i < cnt) *acc_at(sacc, gacc, qs, i0 + i, TT, t) += cdot_rc(Y[i], w[i]);
    }
    if constexpr (SPARSE) {
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        if (i0 + i >= cnt) continue;
        if constexpr (EDGE) {
          if (FSEL <= 0) {
            s0.x += vv[i].x * w[i].x;
            s0.y += vv[i].x * w[i].y;
            s1.x += vv[i].y * w[i].x;
            s1.y += vv[i].y * w[i].y;
          } else {
            s2.x += cc3[i] * w[i].x;
            s2.y += cc3[i] * w[i].y;
          }
          if (mt[i] & kMetaFlush) {
            const int row = meta_slot(mt[i]);
            const bool car = (mt[i] & kMetaCarry) != 0;
            (car ? carry + t : out0 + row)[0] = FSEL <= 0 ? s0 + cmul(fx, s1) : s2;
            s0 = s1 = s2 = {T(0), T(0)};
          }
        } else {
          const bool ty = (mt[i] >> 31) != 0;
          const T a = vv[i].x, b = vv[i].y;
          const T c = FSEL <= 0 ? (ty ? T(0) : a) : (FSEL == 1 ? (ty ? a : b) : (ty ? b : T(0)));
          s0 = cmacr(s0, c, w[i]);
          if (mt[i] & kMetaFlush) {
            const int row = meta_slot(mt[i]);
            const bool car = (mt[i] & kMetaCarry) != 0;
            (car ? carry + t : out0 + row)[0] = s0;
            s0 = {T(0), T(0)};
          }
        }
      }
    }
  }
}

// field-indexed parameters without dynamic indexing of the parameter arrays
template <typename T>
__device__ __forceinline__ const T* spec_of(const Col2Dv2Params<T>& p, int f) {
  return f == 0 ? p.spec[0] : (f == 1 ? p.spec[1] : p.spec[2]);
}
template <typename T>
__device__ __forceinline__ int imag_of(const Col2Dv2Params<T>& p, int f) {
  return f == 0 ? p.imag[0] : (f == 1 ? p.imag[1] : p.imag[2]);
}
template <typename T>
__device__ __forceinline__ int oddy_of(const Col2Dv2Params<T>& p, int f) {
  return f == 0 ? p.oddy[0] : (f == 1 ? p.oddy[1] : p.oddy[2]);
}

template <typename T, int TTC>
__device__ __forceinline__ void load_spectrum(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int f, int kx,
                                              T* sS) {
  // asynchronous global -> shared copies (no register staging): issued before
  // the forward transform, waited for (spectrum_ready) just before the
  // multiply, so the HBM latency hides behind the transform
  const T* S = spec_of(p, f) + (size_t)kx * (g.n + 1);
  for (int i = threadIdx.x; i <= g.n; i += g.TT) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sS + swz16(i));
    if constexpr (sizeof(T) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(S + i) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(S + i) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void spectrum_ready() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
}

// e^{-2 pi i K / N} - 1 for 0 <= K < N, written as -2 i s e^{-i pi K / N} with
// s = sin(pi K / N) and evaluated from the half-angle twiddle (half =
// e^{-i pi / N}), so that it keeps full relative accuracy at small K, where it
// is of size 2 pi K / N (forming cos - 1 directly would lose it).
template <typename T>
__device__ __forceinline__ cplx<T> diff_factor(const Twiddles2L<T>& tw, int K, cplx<T> half) {
  cplx<T> e = tw.template get<-1>(K >> 1);
  if (K & 1) e = cmul(e, half);
  const T c = e.x, sn = -e.y;
  return {T(-2) * sn * sn, T(-2) * sn * c};
}

// Where a thread reads the spectrum column.  After the forward transform
// register k holds frequency K_k = K0 + S k (S = 16 J).  Lanes with h = 0 have
// every K_k < n and read index K_k; lanes with h = 1 have every K_k >= n and
// read the mirrored index N - K_k.  With S a multiple of 16 the padded
// (swizzled) index is base + k * step for both, so the 16 reads are one base
// register plus constant offsets.  The mirror flips the sign of kernels odd
// in y, except on the line K = n itself (K_0 of one thread), which is its
// own mirror.
struct SpecAddr {
  int base, step;
  bool mirror, nyq;
};

template <typename FS, int TTC>
__device__ __forceinline__ SpecAddr spec_addr(const FS& fs, const ColDims<TTC>& g) {
  const int K0 = fs.freq0();
  const int S = 16 * fs.J;
  SpecAddr a;
  a.mirror = K0 >= g.n;
  a.nyq = K0 == g.n;
  a.base = a.mirror ? swz16(g.N - K0) : swz16(K0);
  a.step = a.mirror ? -(S + S / 16) : (S + S / 16);
  return a;
}

// y[k] (+)= i^im * sign * S(K_k) * v[k]
template <typename T, bool ACC>
__device__ __forceinline__ void spectral_multiply(const T* sS, const SpecAddr& a, bool im, bool oy,
                                                  const cplx<T> (&v)[16], cplx<T> (&y)[16]) {
  const T sg = (a.mirror && oy) ? T(-1) : T(1);
  const T sg0 = a.nyq ? T(1) : sg;
  const T* s = sS + a.base;
  if (im) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const T sv = s[k * a.step] * (k == 0 ? sg0 : sg);
      const cplx<T> term = {-v[k].y * sv, v[k].x * sv};
      y[k] = ACC ? y[k] + term : term;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const T sv = s[k * a.step] * (k == 0 ? sg0 : sg);
      y[k] = ACC ? cmacc(y[k], v[k], sv) : cscale(v[k], sv);
    }
  }
}

// rows t + m*TT (m < 8) of a field into the engine's register map (rows the
// thread holds no cell in are zero)
template <typename T, int TTC>
__device__ __forceinline__ void load_rows(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, const cplx<T>* src,
                                          cplx<T> (&v)[16]) {
  const int t = threadIdx.x;
  const unsigned rmask = (unsigned)__ldg(p.tinfo + t) & 0xffu;
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = (rmask >> m) & 1u ? src[rowslot(t + m * g.TT)] : cplx<T>{T(0), T(0)};
#pragma unroll
  for (int m = 8; m < 16; ++m) v[m] = {T(0), T(0)};
}

// Shared-memory regions of a column CTA
template <typename T>
struct ColSmem {
  cplx<T>* sA;     // transform buffer / row sums of field 0
  cplx<T>* sF;     // row sums of fields 1, 2 (ACCREG kernels)
  T* sS;           // spectrum column
  cplx<T>* carry;  // carries of split rows (aliases sS)
  cplx<T>* stw;    // per-column sparse twiddles (fused walks)
};

// One x-frequency column kx of plan p: sparse x-DFT of the fields, column
// transforms, spectral multiply, inverse, gather into the accumulators.  The
// caller has synchronised since the previous column's gather.
// EDGE (ACCREG, NF = 2): the edge-flow form; field 1 (y-edge flows) is
// scaled by e^{-2 pi i K / N} - 1 after its forward transform and both fields
// use field 0's spectrum (the host passes it for both).
// FUSED (ACCREG only): the cell walk of column kx also gathers the previous
// column kxp (kxp < 0: none), field 0's row sums go to the upper half of the
// transform buffer (sA + n; rows y < n of the previous column's output stay
// in sA[0, n) until that gather), and the column ends with its scaled output
// rows in sA: the caller gathers the CTA's last column after its loop.
template <typename T, int NF, bool ACCREG, int TTC, int TCK, bool EDGE = false, bool FUSED = false, int NB = CB>
__device__ __forceinline__ void col2d_column(const Col2Dv2Params<T>& p, const ColDims<TTC>& g, int kx,
                                             FourStep<T, TCK, !EDGE>& fs, const Twiddles2L<T>& tw, const ColSmem<T>& sm,
                                             T* sacc, T* gacc, int qs, cplx<T>* twc,
                                             cplx<T> half = {T(1), T(0)}, int kxp = -1) {
  static_assert(!EDGE || NF == 2, "edge-flow form: two fields");
  static_assert(!FUSED || ACCREG, "fused cell walk: field sums in shared memory");
  const int t = threadIdx.x, TT = g.TT, n = g.n;
  const int cnt = __ldg(p.chunk + t + 1) - __ldg(p.chunk + t);
  cplx<T>* sA = sm.sA;
  cplx<T>* sF = sm.sF;
  if constexpr (ACCREG) {
    cplx<T>* r0 = FUSED ? sA + n : sA;  // field 0's row sums
    if constexpr (FUSED) {
      cplx<T> fx = {T(0), T(0)};
      if constexpr (EDGE) fx = diff_factor(tw, kx, half);
      if (kxp >= 0)
        walk_cells<T, NF, TTC, EDGE, true, true, NB>(p, g, kxp, cnt, r0, sF, sm.carry, sA, sacc, gacc, qs, tw, sm.stw,
                                                 twc, fx);
      else
        walk_cells<T, NF, TTC, EDGE, true, false, NB>(p, g, kxp, cnt, r0, sF, sm.carry, sA, sacc, gacc, qs, tw, sm.stw,
                                                  twc, fx);
    } else if constexpr (EDGE) {
      sparse_rows<T, 2, -1, TTC, true>(p, g, kx, cnt, sA, sF, sm.carry, tw, twc, diff_factor(tw, kx, half));
    } else {
      sparse_rows<T, NF, -1>(p, g, kx, cnt, sA, sF, sm.carry, tw, twc);
    }
    __syncthreads();
    if (p.has_carry) {
      add_carries<T, NF, -1>(p, g, cnt, __ldg(p.tinfo + t) >> 8, r0, sF, sm.carry);
      __syncthreads();
    }
    cplx<T> y[16];
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
      cplx<T> v[16];
      load_rows(p, g, f == 0 ? r0 : sF + (size_t)(f - 1) * n, v);
      __syncthreads();  // rows read before the transform reuses sA; previous spectrum no longer read
      load_spectrum(p, g, f, kx, sm.sS);
      fs.template forward<true>(v);
      if constexpr (EDGE) {
        if (f == 1) {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = cmul(v[k], diff_factor(tw, fs.freq(k), half));
        }
      }
      spectrum_ready();
      const SpecAddr sa = spec_addr(fs, g);
      if (f == 0) spectral_multiply<T, false>(sm.sS, sa, imag_of(p, f) != 0, oddy_of(p, f) != 0, v, y);
      else spectral_multiply<T, true>(sm.sS, sa, imag_of(p, f) != 0, oddy_of(p, f) != 0, v, y);
    }
    fs.inverse(y);
    if constexpr (FUSED) {
      // the gather's column weight (2 for the columns whose mirror image is
      // not computed) applied to the rows: exact, so the sums are unchanged
      const T sc = (kx == 0 || kx == n) ? T(1) : T(2);
#pragma unroll
      for (int m = 0; m < 8; ++m) sA[rowslot(t + m * TT)] = cscale(y[m], sc);
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) sA[rowslot(t + m * TT)] = y[m];
      __syncthreads();
      gather_cells(p, g, kx, cnt, sA, tw, sacc, gacc, qs, twc);
    }
  } else {
    // one field at a time; the walk that forms field f's rows also gathers
    // field f - 1 (whose output rows wait in sA[0, n) while the new sums go to
    // sA + n), and the column's last field is gathered by a walk of its own
    cplx<T> fx = {T(0), T(0)};
    if constexpr (EDGE) fx = diff_factor(tw, kx, half);
    cplx<T>* r0 = sA + n;
    const bool dbl = kx != 0 && kx != n;  // the gather's column weight 2
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
      if (f == 0) walk_field<T, NF, 0, TTC, EDGE, true, false, true>(p, g, kx, cnt, r0, sm.carry, sA, sacc, gacc, qs,
                                                                     tw, twc, fx);
      else if (f == 1) walk_field<T, NF, 1, TTC, EDGE, true, true, false>(p, g, kx, cnt, r0, sm.carry, sA, sacc, gacc,
                                                                          qs, tw, twc, fx);
      else walk_field<T, NF, 2, TTC, EDGE, true, true, false>(p, g, kx, cnt, r0, sm.carry, sA, sacc, gacc, qs, tw,
                                                              twc, fx);
      __syncthreads();
      if (p.has_carry) {
        add_carries<T, NF, 0>(p, g, cnt, __ldg(p.tinfo + t) >> 8, r0, sF, sm.carry);
        __syncthreads();
      }
      cplx<T> v[16];
      load_rows(p, g, r0, v);
      __syncthreads();
      load_spectrum(p, g, f, kx, sm.sS);
      fs.template forward<true>(v);
      if constexpr (EDGE) {
        if (f == 1) {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] = cmul(v[k], diff_factor(tw, fs.freq(k), half));
        }
      }
      spectrum_ready();
      spectral_multiply<T, false>(sm.sS, spec_addr(fs, g), imag_of(p, f) != 0, oddy_of(p, f) != 0, v, v);
      fs.inverse(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) sA[rowslot(t + m * TT)] = dbl ? v[m] + v[m] : v[m];
      __syncthreads();
    }
    walk_field<T, NF, 0, TTC, EDGE, false, true, false>(p, g, kx, cnt, nullptr, nullptr, sA, sacc, gacc, qs, tw, twc,
                                                        fx);
  }
}

template <int TTC>
struct ColBounds {
  static constexpr int threads = TTC > 0 ? TTC : 512;
  static constexpr int blocks = TTC >= 64 ? 512 / TTC : (TTC > 0 ? 16 : 1);
};

// TCK > 0: the radix-16 stages on the tensor cores (tc_dft.cuh; T = float,
// TTC a multiple of 128); shared memory then starts with their header.
template <typename T, int NF, bool ACCREG, int TTC, int TCK = 0, bool EDGE = false, int NB = CB>
__global__ void __launch_bounds__(ColBounds<TTC>::threads, ColBounds<TTC>::blocks)
    k_col2d_v2(const Col2Dv2Params<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(TCK == 0 || (std::is_same<T, float>::value && TTC % 128 == 0), "tensor-core stages: FP32, TT % 128");
  const ColDims<TTC> g(p);
  const int t = threadIdx.x, TT = g.TT, W = TT >> 5;
  const int N = g.N, n = g.n;
  const int nbuf = (16 * TT > W * 544) ? 16 * TT : W * 544;
  const int ntab = fstab_entries(TT);
  cplx<T>* sA = reinterpret_cast<cplx<T>*>(smem_raw + (TCK > 0 ? kTcHeader : 0));
  cplx<T>* stab = sA + nbuf;
  T* sS = reinterpret_cast<T*>(stab + ntab);
  // carries of split rows (3 * TT entries) share the spectrum buffer: both
  // are dead between the last multiply of a column and the first spectrum
  // copy of the next one
  cplx<T>* carry = reinterpret_cast<cplx<T>*>(sS);
  cplx<T>* sF = reinterpret_cast<cplx<T>*>(sS + sspec_entries(n));
  T* sacc = reinterpret_cast<T*>(sF + (ACCREG ? (NF - 1) * n : 0));
  T* gacc = p.partial + (size_t)blockIdx.x * p.npos;
  const int qs = p.acc_rows;
  cplx<T>* twc = p.twc ? p.twc + (size_t)blockIdx.x * p.npos : nullptr;
  for (int i = t; i < ntab; i += TT) stab[i] = p.fstab[i];
  const int cnt = __ldg(p.chunk + t + 1) - __ldg(p.chunk + t);
  for (int i = 0; i < cnt; ++i) *acc_at(sacc, gacc, qs, i, TT, t) = T(0);
  __syncthreads();
  const FourStepTables<T> ftab{stab, stab + 512, stab + 512 + W * 16};
  const Twiddles2L<T> tw{stab + 1024 + W * 16, stab + 1024 + W * 16 + 128, g.log2N - 7,
                         (T)(6.283185307179586476925 / (double)N)};
  FourStep<T, TCK, !EDGE> fs;  // the edge-flow kernels keep the plain butterfly adds
  fs.init(t, TT, sA, ftab);
  if constexpr (TCK > 0) {
    const uint32_t tm = tc_setup(smem_raw, p.tcmat, 2 * kTcMatBytes, TTC / 128 * kTcGroupCols);
    fs.tc.bind(t, (uint32_t)__cvta_generic_to_shared(smem_raw), tm, p.tc_no_commit != 0);
  }
  // per-column twiddles of the fused walks, after the accumulator rows
  cplx<T>* stw = reinterpret_cast<cplx<T>*>(sacc + (size_t)qs * TT);
  const ColSmem<T> sm{sA, sF, sS, carry, stw};
  if constexpr (ACCREG) column_twiddles(g, (int)blockIdx.x, tw, stw);
  cplx<T> half = {T(1), T(0)};  // e^{-i pi / N} (edge-flow form)
  if constexpr (EDGE) half = {(T)cospi(1.0 / (double)N), (T)-sinpi(1.0 / (double)N)};
  int kxp = -1;  // the column whose gather is pending (fused walks)
  for (int kx = blockIdx.x; kx <= n; kx += gridDim.x) {
    // the previous column's output rows are in place (fused walks) or its
    // gather has finished reading sA; with tensor-core stages the CTA also
    // stops after a device wait that gave up
    if constexpr (TCK > 0) {
      if (__syncthreads_or(fs.tc.failed ? 1 : 0)) break;
    } else {
      __syncthreads();
    }
    col2d_column<T, NF, ACCREG, TTC, TCK, EDGE, ACCREG, NB>(p, g, kx, fs, tw, sm, sacc, gacc, qs, twc, half, kxp);
    // the next column's tables: this column's walk read the current ones
    // several barriers ago, the next walk follows the loop's barrier
    if constexpr (ACCREG) column_twiddles(g, kx + (int)gridDim.x, tw, stw);
    kxp = kx;
  }
  if constexpr (ACCREG) {
    if (kxp >= 0) {
      __syncthreads();
      walk_cells<T, NF, TTC, EDGE, false, true, NB>(p, g, kxp, cnt, nullptr, nullptr, nullptr, sA, sacc, gacc, qs, tw,
                                                sm.stw, twc, cplx<T>{T(0), T(0)});
    }
  }
  if constexpr (TCK > 0) {
    if (fs.tc.failed) {
      atomicOr(p.status, 1);
      tc_wait(fs.tc.mbar, fs.tc.phase ^ 1u);  // bounded: the last commit, if it still arrives
    }
    tc_teardown(fs.tc.tmem - (uint32_t)(kTcGroupCols * (t >> 7)), TTC / 128 * kTcGroupCols);
  }
  for (int i = 0; i < cnt && i < qs; ++i) gacc[(size_t)i * TT + t] = sacc[(size_t)i * TT + t];
}

// Grouped launch: the plans of a batch that share the grid (same N and thread
// count) in one persistent launch, with the fused cell walks of k_col2d_v2
// (each CTA gathers the last column of a plan's range before it flushes).
// The P (n + 1) columns of the group are split into gridDim.x contiguous
// ranges, one per CTA; a CTA walks the plans
// its range touches, for each one zeroing its accumulators, running its
// columns and flushing them into the plan's partial sums at row
// blockIdx.x - c0[plan] (c0: the first CTA whose range reaches the plan, so
// the plan's reduction sums the rows of the CTAs that touched it).  Every plan
// passed here has the same n, TT and field count as the launch.
template <typename T, int NF, bool ACCREG, int TTC>
__global__ void __launch_bounds__(ColBounds<TTC>::threads, ColBounds<TTC>::blocks)
    k_col2d_group(const Col2Dv2Params<T>* __restrict__ plans, const int* __restrict__ c0, int nplans) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Col2Dv2Params<T>& p0 = plans[0];
  const ColDims<TTC> g(p0);
  const int t = threadIdx.x, TT = g.TT, W = TT >> 5;
  const int N = g.N, n = g.n;
  const int nbuf = (16 * TT > W * 544) ? 16 * TT : W * 544;
  const int ntab = fstab_entries(TT);
  cplx<T>* sA = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* stab = sA + nbuf;
  T* sS = reinterpret_cast<T*>(stab + ntab);
  cplx<T>* carry = reinterpret_cast<cplx<T>*>(sS);
  cplx<T>* sF = reinterpret_cast<cplx<T>*>(sS + sspec_entries(n));
  T* sacc = reinterpret_cast<T*>(sF + (ACCREG ? (NF - 1) * n : 0));
  for (int i = t; i < ntab; i += TT) stab[i] = p0.fstab[i];  // tables depend on N and TT only
  __syncthreads();
  const FourStepTables<T> ftab{stab, stab + 512, stab + 512 + W * 16};
  const Twiddles2L<T> tw{stab + 1024 + W * 16, stab + 1024 + W * 16 + 128, g.log2N - 7,
                         (T)(6.283185307179586476925 / (double)N)};
  FourStep<T, 0> fs;
  fs.init(t, TT, sA, ftab);
  const int64_t C = (int64_t)nplans * (n + 1);
  const int64_t lo = (int64_t)blockIdx.x * C / gridDim.x, hi = ((int64_t)blockIdx.x + 1) * C / gridDim.x;
  for (int64_t c = lo; c < hi;) {
    const int pi = (int)(c / (n + 1));
    const Col2Dv2Params<T>& p = plans[pi];
    const int k0 = (int)(c - (int64_t)pi * (n + 1));
    const int k1 = (int)std::min<int64_t>(hi - (int64_t)pi * (n + 1), n + 1);
    const int slot = blockIdx.x - c0[pi];
    T* gacc = p.partial + (size_t)slot * p.npos;
    cplx<T>* twc = p.twc ? p.twc + (size_t)slot * p.npos : nullptr;
    const int qs = p.acc_rows;
    const int cnt = __ldg(p.chunk + t + 1) - __ldg(p.chunk + t);
    // per-column twiddles of the fused walks, after this plan's accumulator rows
    cplx<T>* stw = reinterpret_cast<cplx<T>*>(sacc + (size_t)qs * TT);
    const ColSmem<T> sm{sA, sF, sS, carry, stw};
    __syncthreads();  // the previous plan's accumulators have been flushed and its tables read
    for (int i = 0; i < cnt; ++i) *acc_at(sacc, gacc, qs, i, TT, t) = T(0);
    if constexpr (ACCREG) column_twiddles(g, k0, tw, stw);
    int kxp = -1;  // the column whose gather is pending (fused walks)
    for (int kx = k0; kx < k1; ++kx) {
      __syncthreads();
      col2d_column<T, NF, ACCREG, TTC, 0, false, ACCREG>(p, g, kx, fs, tw, sm, sacc, gacc, qs, twc,
                                                         cplx<T>{T(1), T(0)}, kxp);
      if constexpr (ACCREG) column_twiddles(g, kx + 1, tw, stw);
      kxp = kx;
    }
    if constexpr (ACCREG) {
      if (kxp >= 0) {
        __syncthreads();
        walk_cells<T, NF, TTC, false, false, true, CB>(p, g, kxp, cnt, nullptr, nullptr, nullptr, sA, sacc, gacc, qs,
                                                      tw, stw, twc, cplx<T>{T(0), T(0)});
      }
    }
    __syncthreads();
    for (int i = 0; i < cnt && i < qs; ++i) gacc[(size_t)i * TT + t] = sacc[(size_t)i * TT + t];
    c = (int64_t)(pi + 1) * (n + 1);
  }
}

// Three-pass column kernel (FP32): one persistent CTA per SM walks columns
// kx = blockIdx.x, + gridDim.x, ...; per column the NF fields' rows (X, n
// complex each, staged in shared memory by cp.async one column ahead: the
// copies of the next column's field f are issued as soon as this column has
// read field f into registers, each thread copying exactly the slots it reads)
// are transformed forward, multiplied by their spectrum columns and summed in
// registers, transformed back, and rows y < n are written to Y.
template <int NF, int TTC>
__global__ void __launch_bounds__(TTC, ColBounds<TTC>::blocks) k_p3_cols(const Col2Dv2Params<float> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(TTC >= 32, "three-pass column kernel: TT >= 32");
  const ColDims<TTC> g(p);
  constexpr int TT = TTC, W = TT >> 5;
  const int t = threadIdx.x, n = g.n;
  constexpr int nbuf = (16 * TT > W * 544) ? 16 * TT : W * 544;
  const int ntab = fstab_entries(TT);
  cplx<float>* sA = reinterpret_cast<cplx<float>*>(smem_raw);
  cplx<float>* stab = sA + nbuf;
  float* sS = reinterpret_cast<float*>(stab + ntab);
  cplx<float>* stage = reinterpret_cast<cplx<float>*>(sS + sspec_entries(n));  // NF * n
  for (int i = t; i < ntab; i += TT) stab[i] = p.fstab[i];
  const FourStepTables<float> ftab{stab, stab + 512, stab + 512 + W * 16};
  FourStep<float, 0> fs;
  fs.init(t, TT, sA, ftab);
  auto stage_field = [&](int kx, int f) {
    const cplx<float>* src = p.X + ((size_t)f * (n + 1) + kx) * n;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(stage + f * n + t + m * TT);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src + t + m * TT) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (blockIdx.x <= n)
    for (int f = 0; f < NF; ++f) stage_field(blockIdx.x, f);
  for (int kx = blockIdx.x; kx <= n; kx += gridDim.x) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // this column's rows have landed; the previous column no longer reads sA
    const int next = kx + gridDim.x;
    cplx<float> y[16];
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
      cplx<float> v[16];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = stage[f * n + t + m * TT];
#pragma unroll
      for (int m = 8; m < 16; ++m) v[m] = {0.f, 0.f};
      if (next <= n) stage_field(next, f);
      if (f > 0) __syncthreads();  // the previous field's spectrum and transform buffer are no longer read
      load_spectrum(p, g, f, kx, sS);
      fs.template forward<true>(v);
      spectrum_ready();
      const SpecAddr sa = spec_addr(fs, g);
      if (f == 0) spectral_multiply<float, false>(sS, sa, imag_of(p, f) != 0, oddy_of(p, f) != 0, v, y);
      else spectral_multiply<float, true>(sS, sa, imag_of(p, f) != 0, oddy_of(p, f) != 0, v, y);
    }
    fs.inverse(y);
    cplx<float>* dst = p.Y + (size_t)kx * n;
#pragma unroll
    for (int m = 0; m < 8; ++m) dst[t + m * TT] = y[m];
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int TTC>
cudaError_t Col2DPassKernels<TTC>::configure(size_t smem, int threads, int* blocks_per_sm) {
  int b[3] = {0, 0, 0};
  cudaError_t e;
  if ((e = allow_optin_smem(k_p3_cols<1, TTC>)) != cudaSuccess) return e;
  if ((e = allow_optin_smem(k_p3_cols<2, TTC>)) != cudaSuccess) return e;
  if ((e = allow_optin_smem(k_p3_cols<3, TTC>)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[0], k_p3_cols<1, TTC>, threads, smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[1], k_p3_cols<2, TTC>, threads, smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[2], k_p3_cols<3, TTC>, threads, smem)) != cudaSuccess)
    return e;
  *blocks_per_sm = std::min(b[0], std::min(b[1], b[2]));
  return cudaSuccess;
}

template <int TTC>
void Col2DPassKernels<TTC>::launch(int nf, int grid, int threads, size_t smem, cudaStream_t st,
                                   const Col2Dv2Params<float>& cp) {
  if (nf == 1) k_p3_cols<1, TTC><<<grid, threads, smem, st>>>(cp);
  else if (nf == 2) k_p3_cols<2, TTC><<<grid, threads, smem, st>>>(cp);
  else k_p3_cols<3, TTC><<<grid, threads, smem, st>>>(cp);
}

// resident CTAs of one kernel, folded into the running minimum
template <typename K>
static cudaError_t min_residency(K kern, int threads, size_t smem, int* bmin) {
  cudaError_t e = allow_optin_smem(kern);
  if (e != cudaSuccess) return e;
  int b = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem)) != cudaSuccess) return e;
  *bmin = std::min(*bmin, b);
  return cudaSuccess;
}

template <typename T, int TTC>
cudaError_t Col2DKernels<T, TTC>::configure(size_t smem, int threads, int* blocks_per_sm) {
  constexpr bool R = std::is_same<T, float>::value;
  int b = 1 << 30;
  cudaError_t e;
  if ((e = min_residency(k_col2d_v2<T, 1, false, TTC>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<T, 2, R, TTC>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<T, 3, R, TTC>, threads, smem, &b)) != cudaSuccess) return e;
  if constexpr (R) {
    if ((e = min_residency(k_col2d_v2<T, 2, true, TTC, 0, false, 4>, threads, smem, &b)) != cudaSuccess) return e;
    if ((e = min_residency(k_col2d_v2<T, 3, true, TTC, 0, false, 4>, threads, smem, &b)) != cudaSuccess) return e;
  }
  *blocks_per_sm = b;
  return cudaSuccess;
}

template <int TTC>
void Col2DGroupKernels<TTC>::launch(int nf, int grid, int threads, size_t smem, cudaStream_t st,
                                    const Col2Dv2Params<float>* plans, const int* c0, int nplans) {
  if (nf == 1) k_col2d_group<float, 1, false, TTC><<<grid, threads, smem, st>>>(plans, c0, nplans);
  else if (nf == 2) k_col2d_group<float, 2, true, TTC><<<grid, threads, smem, st>>>(plans, c0, nplans);
  else k_col2d_group<float, 3, true, TTC><<<grid, threads, smem, st>>>(plans, c0, nplans);
}

template <int TTC>
cudaError_t Col2DGroupKernels<TTC>::configure(size_t smem, int threads, int* blocks_per_sm) {
  int b[3] = {0, 0, 0};
  cudaError_t e;
  if ((e = allow_optin_smem(k_col2d_group<float, 1, false, TTC>)) != cudaSuccess) return e;
  if ((e = allow_optin_smem(k_col2d_group<float, 2, true, TTC>)) != cudaSuccess) return e;
  if ((e = allow_optin_smem(k_col2d_group<float, 3, true, TTC>)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[0], k_col2d_group<float, 1, false, TTC>, threads,
                                                         smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[1], k_col2d_group<float, 2, true, TTC>, threads,
                                                         smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[2], k_col2d_group<float, 3, true, TTC>, threads,
                                                         smem)) != cudaSuccess)
    return e;
  *blocks_per_sm = std::min(b[0], std::min(b[1], b[2]));
  return cudaSuccess;
}

template <typename T, int TTC>
void Col2DKernels<T, TTC>::launch(int nf, int grid, int threads, size_t smem, cudaStream_t st,
                                  const Col2Dv2Params<T>& cp, int nb) {
  constexpr bool R = std::is_same<T, float>::value;
  if (nf == 1) {
    k_col2d_v2<T, 1, false, TTC><<<grid, threads, smem, st>>>(cp);
  } else if constexpr (R) {
    // the fused walks take the tuned cell batch
    if (nf == 2 && nb == 4) k_col2d_v2<T, 2, true, TTC, 0, false, 4><<<grid, threads, smem, st>>>(cp);
    else if (nf == 2) k_col2d_v2<T, 2, true, TTC><<<grid, threads, smem, st>>>(cp);
    else if (nb == 4) k_col2d_v2<T, 3, true, TTC, 0, false, 4><<<grid, threads, smem, st>>>(cp);
    else k_col2d_v2<T, 3, true, TTC><<<grid, threads, smem, st>>>(cp);
  } else {
    if (nf == 2) k_col2d_v2<T, 2, false, TTC><<<grid, threads, smem, st>>>(cp);
    else k_col2d_v2<T, 3, false, TTC><<<grid, threads, smem, st>>>(cp);
  }
}

template <typename T, int TTC>
cudaError_t Col2DEdgeKernels<T, TTC>::configure(size_t smem, int threads, int* blocks_per_sm) {
  constexpr bool R = std::is_same<T, float>::value;
  int b = 1 << 30;
  cudaError_t e;
  if ((e = min_residency(k_col2d_v2<T, 2, R, TTC, 0, true>, threads, smem, &b)) != cudaSuccess) return e;
  if constexpr (R) {
    if ((e = min_residency(k_col2d_v2<T, 2, true, TTC, 0, true, 4>, threads, smem, &b)) != cudaSuccess) return e;
  }
  *blocks_per_sm = b;
  return cudaSuccess;
}

template <typename T, int TTC>
void Col2DEdgeKernels<T, TTC>::launch(int grid, int threads, size_t smem, cudaStream_t st,
                                      const Col2Dv2Params<T>& cp, int nb) {
  constexpr bool R = std::is_same<T, float>::value;
  if constexpr (R) {
    if (nb == 4) {
      k_col2d_v2<T, 2, true, TTC, 0, true, 4><<<grid, threads, smem, st>>>(cp);
      return;
    }
  }
  k_col2d_v2<T, 2, R, TTC, 0, true><<<grid, threads, smem, st>>>(cp);
}

template <int TTC, int TCK>
cudaError_t Col2DTcKernels<TTC, TCK>::configure(size_t smem, int threads, int* blocks_per_sm) {
  int b = 1 << 30;
  cudaError_t e;
  if ((e = min_residency(k_col2d_v2<float, 1, false, TTC, TCK>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<float, 2, true, TTC, TCK>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<float, 3, true, TTC, TCK>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<float, 2, true, TTC, TCK, false, 4>, threads, smem, &b)) != cudaSuccess) return e;
  if ((e = min_residency(k_col2d_v2<float, 3, true, TTC, TCK, false, 4>, threads, smem, &b)) != cudaSuccess) return e;
  // each resident CTA holds TTC / 128 * kTcGroupCols tensor-memory columns (512 per SM)
  *blocks_per_sm = std::min(b, 512 / (TTC / 128 * kTcGroupCols));
  return cudaSuccess;
}

template <int TTC, int TCK>
void Col2DTcKernels<TTC, TCK>::launch(int nf, int grid, int threads, size_t smem, cudaStream_t st,
                                      const Col2Dv2Params<float>& cp, int nb) {
  if (nf == 1) k_col2d_v2<float, 1, false, TTC, TCK><<<grid, threads, smem, st>>>(cp);
  else if (nf == 2 && nb == 4) k_col2d_v2<float, 2, true, TTC, TCK, false, 4><<<grid, threads, smem, st>>>(cp);
  else if (nf == 2) k_col2d_v2<float, 2, true, TTC, TCK><<<grid, threads, smem, st>>>(cp);
  else if (nb == 4) k_col2d_v2<float, 3, true, TTC, TCK, false, 4><<<grid, threads, smem, st>>>(cp);
  else k_col2d_v2<float, 3, true, TTC, TCK><<<grid, threads, smem, st>>>(cp);
}

}  // namespace bemfft
