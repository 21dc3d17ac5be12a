// 2D operator apply: sparse row transform fused with the scatter, per-column
// FFT + spectral multiply + inverse FFT in one CTA, and the gather fused into
// the inverse row transform (Section 3-4, Eq. 15-16).
//
// Layout of the padded N x N grid (N = 2n): rows are y, columns are x.  The
// scattered density rho (zero off the boundary cells, Fig. 4) has at most a
// few non-zeros per row, so its forward transform along x is evaluated
// directly from the cell list (an input-pruned DFT: O(cells) per frequency)
// instead of an FFT over a mostly-zero row; only the n+1 non-redundant
// x-frequencies of the real field are formed.  For each x-frequency kx one
// CTA then owns the full column (length N along y) in registers/shared
// memory: forward FFT along y, multiply by the compressed kernel spectrum
// column, inverse FFT along y, and the inverse transform along x evaluated
// only at the boundary cells (an output-pruned inverse DFT that also is the
// gather).  The padded grid never exists in global memory; the only large
// stream from HBM is the spectrum ((n+1)^2 reals per kernel table).
//
// Thread t of a CTA owns grid rows t + m*TT (m < E/2): these are exactly the
// positions its registers hold in the first pass of the forward transform
// and after the last pass of the inverse one, so the scatter writes and the
// gather reads registers directly.  Cells are read through a warp-coalesced
// slot layout (see SlotSet) so each load of the sparse loops is contiguous
// across a warp and every loop has a warp-uniform trip count.  Each CTA
// accumulates the contributions of its columns per cell slot (shared memory
// when it fits, else its own slice of the partial buffer), and a reduction
// kernel sums the per-CTA partials in a fixed order (compensated FP32 for FP32
// plans, FP64 otherwise) in the caller's cell order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bem_internal.h"
#include "col2d_v2.h"
#include "fft4step.cuh"
#include "fft_reg.cuh"

namespace bemfft {

template <typename T>
struct Col2DParams {
  int n, log2N, G, H;
  const T* spec[kMaxFields];
  int imag[kMaxFields];
  int oddy[kMaxFields];
  const int32_t* cnt[kMaxFields];
  const int32_t* off[kMaxFields];
  const uint16_t* xs[kMaxFields];
  const T* rho[kMaxFields];
  const int32_t* gcnt;
  const int32_t* goff;
  const uint16_t* gx;
  int64_t gnelem;
  const cplx<T>* qtab;  // N/4
  T* partial;           // gridDim.x * gnelem
  int acc_in_smem;
};

template <typename T, int E>
__device__ __forceinline__ void gather_rows(const cplx<T> (&y)[E], const Col2DParams<T>& p, const int grp,
                                            const int lane, const int kx, const Twiddles<T>& tw, T* acc) {
  constexpr int H = E / 2;
  const int N = 1 << p.log2N;
  const T ckx = (kx == 0 || kx == p.n) ? T(1) : T(2);
#pragma unroll
  for (int m = 0; m < H; ++m) {
    const int c = __ldg(p.gcnt + grp * H + m);
    const int64_t base = (int64_t)__ldg(p.goff + grp * H + m) * p.G + lane;
    const T yr = ckx * y[m].x, yi = ckx * y[m].y;
#pragma unroll 4
    for (int i = 0; i < c; ++i) {
      const int64_t e = base + (int64_t)i * p.G;
      const cplx<T> w = tw.template get<+1>((kx * (int)__ldg(p.gx + e)) & (N - 1));
      acc[e] += yr * w.x - yi * w.y;
    }
  }
}

template <typename T, int E, int NF, bool ACCREG>
__global__ void __launch_bounds__(512) k_col2d(const Col2DParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = threadIdx.x, TT = blockDim.x;
  const int log2N = p.log2N, N = 1 << log2N, n = p.n;
  const int grp = t / p.G, lane = t - grp * p.G;
  cplx<T>* sbuf = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* sq = sbuf + (N + (N >> 4));
  T* acc = p.acc_in_smem ? reinterpret_cast<T*>(sq + (N >> 2)) : p.partial + (size_t)blockIdx.x * p.gnelem;
  for (int i = t; i < (N >> 2); i += TT) sq[i] = p.qtab[i];
  for (int64_t e = t; e < p.gnelem; e += TT) acc[e] = T(0);
  __syncthreads();
  const Twiddles<T> tw{sq, log2N - 2};
  constexpr int H = E / 2;

  for (int kx = blockIdx.x; kx <= n; kx += gridDim.x) {
    cplx<T> y[ACCREG ? E : 1];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      cplx<T> v[E];
      // scatter fused with the input-pruned forward DFT along x
      const T* rho = p.rho[f];
      const uint16_t* xs = p.xs[f];
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int c = __ldg(p.cnt[f] + grp * H + m);
        const int64_t base = (int64_t)__ldg(p.off[f] + grp * H + m) * p.G + lane;
        cplx<T> s = {T(0), T(0)};
#pragma unroll 4
        for (int i = 0; i < c; ++i) {
          const int64_t e = base + (int64_t)i * p.G;
          const T r = __ldg(rho + e);
          const cplx<T> w = tw.template get<-1>((kx * (int)__ldg(xs + e)) & (N - 1));
          s.x += r * w.x;
          s.y += r * w.y;
        }
        v[m] = s;
      }
#pragma unroll
      for (int m = H; m < E; ++m) v[m] = {T(0), T(0)};
      fft_line<E, -1>(v, t, TT, log2N, tw, sbuf);
      // spectral multiply (Eq. 16), spectrum column kx, folded in ky
      const T* S = p.spec[f] + (size_t)kx * (n + 1);
      const bool im = p.imag[f] != 0, oy = p.oddy[f] != 0;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int ky = t + m * TT;
        const bool hi = ky > n;
        T sv = __ldg(S + (hi ? N - ky : ky));
        if (hi && oy) sv = -sv;
        const cplx<T> prod = im ? cplx<T>{-v[m].y * sv, v[m].x * sv} : cplx<T>{v[m].x * sv, v[m].y * sv};
        if constexpr (ACCREG) {
          if (f == 0) y[m] = prod;
          else y[m] = y[m] + prod;
        } else {
          v[m] = prod;
        }
      }
      if constexpr (!ACCREG) {
        fft_line<E, +1>(v, t, TT, log2N, tw, sbuf);
        gather_rows<T, E>(v, p, grp, lane, kx, tw, acc);
      }
    }
    if constexpr (ACCREG) {
      fft_line<E, +1>(y, t, TT, log2N, tw, sbuf);
      gather_rows<T, E>(y, p, grp, lane, kx, tw, acc);
    }
  }
  if (p.acc_in_smem) {
    __syncthreads();
    for (int64_t e = t; e < p.gnelem; e += TT) p.partial[(size_t)blockIdx.x * p.gnelem + e] = acc[e];
  }
}

// rho_f[e] = coef_f[cidx[e]] * in[perm[cidx[e]]*ncomp + comp_f]  (0 on padding)
template <typename T>
struct PrepParams {
  int ncomp, nf;
  const int32_t* perm;
  const T* in;
  const T* coef[kMaxFields];
  const int32_t* cidx[kMaxFields];
  int64_t nelem[kMaxFields];
  int comp[kMaxFields];
  T* rho[kMaxFields];
};

template <typename T>
__global__ void k_prep(const PrepParams<T> p) {
  const int f = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.nelem[f]) return;
  const int c = p.cidx[f][e];
  p.rho[f][e] = c >= 0 ? p.coef[f][c] * p.in[(int64_t)p.perm[c] * p.ncomp + p.comp[f]] : T(0);
}

// out[perm[cidx[e]]] = sum_b partial[b][e] + diag * in  over valid slots e,
// in FP64 and a fixed order: 32 slots per block, 16 warps each summing every
// 16th CTA's partial (four interleaved chains keep four loads in flight),
// then the 16 warp sums in order
template <typename T>
__global__ void __launch_bounds__(512) k_reduce(const T* __restrict__ partial, int grid, int64_t nelem,
                                                const int32_t* __restrict__ cidx, const int32_t* __restrict__ perm,
                                                const T* __restrict__ diag, const T* __restrict__ in,
                                                T* __restrict__ out) {
  constexpr int W = 16;
  __shared__ double red[W][33];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  const int c = e < nelem ? cidx[e] : -1;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (c >= 0) {
    int b = wp;
    for (; b + 3 * W < grid; b += 4 * W) {
      s0 += (double)partial[(size_t)b * nelem + e];
      s1 += (double)partial[(size_t)(b + W) * nelem + e];
      s2 += (double)partial[(size_t)(b + 2 * W) * nelem + e];
      s3 += (double)partial[(size_t)(b + 3 * W) * nelem + e];
    }
    for (; b < grid; b += W) s0 += (double)partial[(size_t)b * nelem + e];
  }
  red[wp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (wp == 0 && c >= 0) {
    double t = 0.0;
    for (int k = 0; k < W; ++k) t += red[k][lane];
    const int u = perm[c];
    if (diag) t += (double)diag[u] * (double)in[u];
    out[u] = (T)t;
  }
}


// val[pos] = (coefA[pos], coefB[pos]) * in[perm[pos]] (interleaved positions;
// padding positions have perm < 0 and get zero)
template <typename T, typename TIO>
__global__ void k_prep_v2(int npos, const int32_t* __restrict__ perm, const TIO* __restrict__ in,
                          const T* __restrict__ coefA, const T* __restrict__ coefB, cplx<T>* __restrict__ val) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npos) return;
  const int u = perm[j];
  const T x = u >= 0 ? T(in[u]) : T(0);
  val[j] = {coefA[j] * x, coefB[j] * x};
}

// Error-free sum (Knuth's TwoSum): returns s = fl(a + b) and sets e so that
// a + b = s + e exactly (round-to-nearest, no contraction).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}

// Running compensated FP32 sum (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), algorithm Sum2): p carries the
// rounded sum, c the exactly captured rounding errors; the result p + c is as
// accurate as the sum taken in twice the working precision and rounded once.
struct CompSum {
  float p, c;
  __device__ __forceinline__ void add(float x) {
    float e;
    p = two_sum(p, x, e);
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void add(const CompSum& o) {
    add(o.p);
    c = __fadd_rn(c, o.c);
  }
};

// out[perm[j]] = sum_b partial[b*npos + j] (+ diag * in) over interleaved
// positions j (padding skipped), in a fixed order: 32 cells per block, 16
// warps each summing every 16th partial (four interleaved chains, so that four
// loads are in flight), then the 16 warp sums in order.  FP32 plans sum with
// the compensated FP32 sum above (GB300's FP64 rate would make the FP64 adds
// and conversions the reduction's cost); FP64 and double-float plans in FP64.
template <typename T, typename TIO>
__global__ void __launch_bounds__(512) k_reduce_v2(const T* __restrict__ partial, int grid, int npos,
                                                   const int32_t* __restrict__ perm, const TIO* __restrict__ diag,
                                                   const TIO* __restrict__ in, TIO* __restrict__ out) {
  constexpr int W = 16;  // warps, each summing every W-th CTA's partial
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  if constexpr (std::is_same<T, float>::value && std::is_same<TIO, float>::value) {
    __shared__ CompSum red[W][33];
    CompSum s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f}, s3{0.f, 0.f};
    if (j < npos) {
      int b = wp;
      for (; b + 3 * W < grid; b += 4 * W) {
        s0.add(partial[(size_t)b * npos + j]);
        s1.add(partial[(size_t)(b + W) * npos + j]);
        s2.add(partial[(size_t)(b + 2 * W) * npos + j]);
        s3.add(partial[(size_t)(b + 3 * W) * npos + j]);
      }
      for (; b < grid; b += W) s0.add(partial[(size_t)b * npos + j]);
    }
    s0.add(s1);
    s0.add(s2);
    s0.add(s3);
    red[wp][lane] = s0;
    __syncthreads();
    if (wp == 0 && j < npos && perm[j] >= 0) {
      CompSum t{0.f, 0.f};
      for (int k = 0; k < W; ++k) t.add(red[k][lane]);
      const int u = perm[j];
      if (diag) {
        // exact product as pr + epr (FMA error term)
        const float pr = __fmul_rn(diag[u], in[u]);
        const float epr = fmaf(diag[u], in[u], -pr);
        t.add(pr);
        t.c = __fadd_rn(t.c, epr);
      }
      out[u] = __fadd_rn(t.p, t.c);
    }
  } else {
    __shared__ double red[W][33];
    // four independent chains keep four loads in flight; fixed order throughout
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (j < npos) {
      int b = wp;
      for (; b + 3 * W < grid; b += 4 * W) {
        s0 += (double)partial[(size_t)b * npos + j];
        s1 += (double)partial[(size_t)(b + W) * npos + j];
        s2 += (double)partial[(size_t)(b + 2 * W) * npos + j];
        s3 += (double)partial[(size_t)(b + 3 * W) * npos + j];
      }
      for (; b < grid; b += W) s0 += (double)partial[(size_t)b * npos + j];
    }
    red[wp][lane] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (wp == 0 && j < npos && perm[j] >= 0) {
      double t = 0.0;
      for (int k = 0; k < W; ++k) t += red[k][lane];
      const int u = perm[j];
      if (diag) t += (double)diag[u] * (double)in[u];
      out[u] = (TIO)t;
    }
  }
}

// ------------------------------------------------------------------ host side

// elements per thread of the small-grid column kernel (N <= 256): four, so a
// column of N = 256 runs on 64 threads (two warps: its FP64 arithmetic issues
// from two SM sub-partitions and every thread's dependent chains are short),
// eight below N = 64
static int elems_per_thread(int log2N) { return log2N >= 6 ? 4 : 8; }

// Records the start event of a timed column-kernel launch on st and returns
// the end event to record after it (nullptr on failure).
static cudaEvent_t timing_begin(bem_plan_s* p, cudaStream_t st) {
  if (p->ev_used + 2 > (int)p->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        set_error("cudaEventCreate failed");
        return nullptr;
      }
      p->ev_pool.push_back(e);
    }
  }
  cudaEvent_t e0 = p->ev_pool[p->ev_used++];
  cudaEvent_t e1 = p->ev_pool[p->ev_used++];
  if (cudaEventRecord(e0, st) != cudaSuccess) {
    set_error("cudaEventRecord failed");
    return nullptr;
  }
  return e1;
}

void free_slot_set(SlotSet* s) {
  cudaFree(s->d_cnt);
  cudaFree(s->d_off);
  cudaFree(s->d_x);
  cudaFree(s->d_cidx);
  *s = SlotSet();
}

bem_status build_slot_set(bem_plan_s* p, const std::vector<uint8_t>& member, SlotSet* s) {
  const int E = elems_per_thread(p->log2N);
  const int TT = (int)(p->N / E), H = E / 2;
  const int G = TT < 32 ? TT : 32;
  const int ngroups = TT / G;
  // cells per row (rows sorted, x ascending within a row)
  const int64_t n = p->n;
  std::vector<int32_t> rowbeg(n + 1, 0);
  for (int64_t j = 0; j < p->nb; ++j)
    if (member[j]) rowbeg[p->h_row[j] + 1]++;
  for (int64_t r = 0; r < n; ++r) rowbeg[r + 1] += rowbeg[r];
  std::vector<int32_t> rowcells(rowbeg[n]);
  {
    std::vector<int32_t> fill(rowbeg.begin(), rowbeg.end() - 1);
    for (int64_t j = 0; j < p->nb; ++j)
      if (member[j]) rowcells[fill[p->h_row[j]]++] = (int32_t)j;
  }
  std::vector<int32_t> cnt((size_t)ngroups * H), off((size_t)ngroups * H);
  int64_t total = 0;
  for (int g = 0; g < ngroups; ++g)
    for (int m = 0; m < H; ++m) {
      int mx = 0;
      for (int l = 0; l < G; ++l) {
        const int64_t row = (int64_t)(g * G + l) + (int64_t)m * TT;
        mx = std::max(mx, rowbeg[row + 1] - rowbeg[row]);
      }
      cnt[(size_t)g * H + m] = mx;
      off[(size_t)g * H + m] = (int32_t)total;
      total += mx;
    }
  if (total * G >= ((int64_t)1 << 31)) {
    set_error("slot layout too large");
    return BEM_ERR_UNSUPPORTED;
  }
  const int64_t nelem = std::max<int64_t>(1, total * G);
  std::vector<uint16_t> xs(nelem, 0);
  std::vector<int32_t> cidx(nelem, -1);
  for (int g = 0; g < ngroups; ++g)
    for (int m = 0; m < H; ++m)
      for (int l = 0; l < G; ++l) {
        const int64_t row = (int64_t)(g * G + l) + (int64_t)m * TT;
        const int64_t base = (int64_t)off[(size_t)g * H + m] * G + l;
        for (int i = 0; i < rowbeg[row + 1] - rowbeg[row]; ++i) {
          const int32_t j = rowcells[rowbeg[row] + i];
          xs[base + (int64_t)i * G] = (uint16_t)p->h_col[j];
          cidx[base + (int64_t)i * G] = j;
        }
      }
  free_slot_set(s);
  s->ngroups = ngroups;
  s->G = G;
  s->H = H;
  s->nelem = nelem;
  BEM_CUDA_TRY(cudaMalloc(&s->d_cnt, cnt.size() * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMalloc(&s->d_off, off.size() * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMalloc(&s->d_x, nelem * sizeof(uint16_t)));
  BEM_CUDA_TRY(cudaMalloc(&s->d_cidx, nelem * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMemcpy(s->d_cnt, cnt.data(), cnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemcpy(s->d_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemcpy(s->d_x, xs.data(), nelem * sizeof(uint16_t), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemcpy(s->d_cidx, cidx.data(), nelem * sizeof(int32_t), cudaMemcpyHostToDevice));
  s->h_cidx = std::move(cidx);
  return BEM_OK;
}

bem_status alloc_field_rho(bem_plan_s* p, Operator& op) {
  for (int f = 0; f < op.nf; ++f) {
    void* d = nullptr;
    const size_t bytes = (size_t)op.f[f].set->nelem * prec_bytes(p);
    BEM_CUDA_TRY(cudaMalloc(&d, bytes));
    BEM_CUDA_TRY(cudaMemset(d, 0, bytes));
    op.owned.push_back(d);
    op.f[f].rho = d;
    p->scratch_bytes += bytes;
  }
  return BEM_OK;
}

template <typename T>
static size_t smem_2d(int64_t N, int64_t nelem, bool acc) {
  size_t s = (size_t)(N + N / 16) * sizeof(cplx<T>) + (size_t)(N / 4) * sizeof(cplx<T>);
  if (acc) s += (size_t)nelem * sizeof(T);
  return s;
}

template <typename T, int E, int NF, bool ACCREG>
static cudaError_t configure_one(size_t smem, int threads, int* blocks_per_sm) {
  auto kern = k_col2d<T, E, NF, ACCREG>;
  cudaError_t e = allow_optin_smem(kern);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, threads, smem);
}

template <typename T, int E>
static cudaError_t configure_all(size_t smem, int threads, int* bps) {
  constexpr bool R = std::is_same<T, float>::value;  // accumulate in registers only for FP32
  int b1 = 0, b2 = 0, b3 = 0;
  cudaError_t e;
  if ((e = configure_one<T, E, 1, false>(smem, threads, &b1)) != cudaSuccess) return e;
  if ((e = configure_one<T, E, 2, R>(smem, threads, &b2)) != cudaSuccess) return e;
  if ((e = configure_one<T, E, 3, R>(smem, threads, &b3)) != cudaSuccess) return e;
  *bps = std::min(b1, std::min(b2, b3));
  return cudaSuccess;
}

template <typename T>
static bem_status setup_t(bem_plan_s* p) {
  const int64_t N = p->N;
  const int E = elems_per_thread(p->log2N);
  p->threads = (int)(N / E);
  std::vector<uint8_t> all(p->nb, 1);
  bem_status rc = build_slot_set(p, all, &p->all_set);
  if (rc != BEM_OK) return rc;
  const int64_t nelem = p->all_set.nelem;
  int dev = 0, nsm = 0, smem_optin = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  p->acc_in_smem = smem_2d<T>(N, nelem, true) <= (size_t)smem_optin;
  p->smem_bytes = smem_2d<T>(N, nelem, p->acc_in_smem);
  if (p->smem_bytes > (size_t)smem_optin) {
    set_error("grid too large for the shared-memory column buffer");
    return BEM_ERR_UNSUPPORTED;
  }
  int bps = 0;
  if (E == 4)
    BEM_CUDA_TRY((configure_all<T, 4>(p->smem_bytes, p->threads, &bps)));
  else
    BEM_CUDA_TRY((configure_all<T, 8>(p->smem_bytes, p->threads, &bps)));
  if (bps < 1) {
    set_error("column kernel cannot be resident (registers/shared memory)");
    return BEM_ERR_UNSUPPORTED;
  }
  p->grid = (int)std::min<int64_t>((int64_t)bps * nsm, p->n + 1);
  const size_t tb = sizeof(T);
  BEM_CUDA_TRY(cudaMalloc(&p->d_partial, (size_t)p->grid * nelem * p->ncomp * tb));
  p->scratch_bytes += (size_t)p->grid * nelem * p->ncomp * tb;
  return BEM_OK;
}

// 16-bit encodings (round to nearest even) for the tensor-core B matrices
static uint16_t bf16_bits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static double bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// |x| < 2 (DFT entries and their residuals)
static uint16_t f16_bits(double x) {
  const uint16_t sgn = x < 0 ? 0x8000u : 0u;
  const double a = std::fabs(x);
  if (a == 0.0) return sgn;
  int E;
  std::frexp(a, &E);  // a in [2^(E-1), 2^E)
  const int e = E - 1;
  if (e < -14) return (uint16_t)(sgn | (uint16_t)std::nearbyint(std::ldexp(a, 24)));  // subnormal (or min normal)
  int q = (int)std::nearbyint((std::ldexp(a, -e) - 1.0) * 1024.0);
  int eb = e + 15;
  if (q == 1024) {
    q = 0;
    ++eb;
  }
  return (uint16_t)(sgn | (uint16_t)(eb << 10) | (uint16_t)q);
}
static double f16_value(uint16_t b) {
  const int eb = (b >> 10) & 31, q = b & 1023;
  const double v = eb == 0 ? std::ldexp((double)q, -24) : std::ldexp(1.0 + q / 1024.0, eb - 15);
  return (b & 0x8000u) ? -v : v;
}

// B operands of the tensor-core stages (tc_dft.cuh): matrix 0 the forward
// 16-point DFT, matrix 1 the J-point DFT blocks of the middle stage (J =
// TT / 32), in the real form acting on (re, im) columns, each as hi then lo
// 16-bit parts in the K-major core-matrix layout.  FP64 angles from the exact
// index product mod J.
static std::vector<uint16_t> tc_matrices(int kind, int J) {
  const double PI = 3.14159265358979323846;
  std::vector<uint16_t> out(2 * 2048, 0);  // 2 matrices x (hi, lo) x 32 x 32
  for (int mat = 0; mat < 2; ++mat) {
    const int B = mat == 0 ? 16 : J;
    for (int n = 0; n < 32; ++n)
      for (int k = 0; k < 32; ++k) {
        const int f = n & 15, co = n >> 4;                 // output element, part
        const int i = (k >> 4) * 8 + (k & 7), ci = (k >> 3) & 1;  // input element, part
        double v = 0.0;
        if (f / B == i / B) {
          const int m = ((f % B) * (i % B)) % B;
          double c = std::cos(2.0 * PI * m / B), sn = std::sin(2.0 * PI * m / B);
          if (std::fabs(c) < 1e-15) c = 0.0;
          if (std::fabs(sn) < 1e-15) sn = 0.0;
          // forward: Re X = re c + im s, Im X = im c - re s
          v = co == 0 ? (ci == 0 ? c : sn) : (ci == 0 ? -sn : c);
        }
        uint16_t hb, lb;
        if (kind == kTcBf16) {
          hb = bf16_bits(v);
          lb = bf16_bits(v - bf16_value(hb));
        } else {
          hb = f16_bits(v);
          lb = f16_bits(v - f16_value(hb));
        }
        const int idx = ((n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
        out[mat * 2048 + idx] = hb;
        out[mat * 2048 + 1024 + idx] = lb;
      }
  }
  return out;
}

static bem_status setup_p3(bem_plan_s* p);

// largest per-CTA twiddle cache (bytes over all CTAs) the column kernel keeps
constexpr size_t kTwiddleCacheMax = (size_t)40 << 20;

// shared memory of the four-step kernel
template <typename T>
static size_t smem_v2(int64_t n, int TT, int64_t nb, bool accreg, bool acc, bool tc) {
  const int W = TT / 32;
  const size_t nbuf = (size_t)std::max(16 * TT, W * 544);
  size_t s = (nbuf + (size_t)fstab_entries(TT) + kColTwEntries) * sizeof(cplx<T>) +
             (size_t)sspec_entries((int)n) * sizeof(T);
  if (tc) s += kTcHeader;
  if (accreg) s += (size_t)2 * n * sizeof(cplx<T>);
  if (acc) s += (size_t)nb * sizeof(T);
  return s;
}

// the column kernels for TT threads: compile-time thread counts for FP32,
// the generic kernel for FP64; tc selects the tensor-core stages (FP32,
// TT = 128, 256, 512; checked at plan time)
template <int TCK>
static cudaError_t configure_tc(int TT, size_t smem, int* bps) {
  switch (TT) {
    case 512: return Col2DTcKernels<512, TCK>::configure(smem, TT, bps);
    case 256: return Col2DTcKernels<256, TCK>::configure(smem, TT, bps);
    default: return Col2DTcKernels<128, TCK>::configure(smem, TT, bps);
  }
}

template <int TCK>
static void launch_tc(const bem_plan_s* p, int nf, const Col2Dv2Params<float>& cp, cudaStream_t st) {
  const int TT = p->threads;
  switch (TT) {
    case 512: Col2DTcKernels<512, TCK>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
    case 256: Col2DTcKernels<256, TCK>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
    default: Col2DTcKernels<128, TCK>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
  }
}

template <typename T>
static cudaError_t configure_col2d(int TT, int tc, size_t smem, int* bps) {
  if constexpr (std::is_same<T, f32x2>::value) {
    switch (TT) {
      case 512: return Col2DKernels<f32x2, 512>::configure(smem, TT, bps);
      case 256: return Col2DKernels<f32x2, 256>::configure(smem, TT, bps);
      case 128: return Col2DKernels<f32x2, 128>::configure(smem, TT, bps);
      case 64: return Col2DKernels<f32x2, 64>::configure(smem, TT, bps);
      default: return Col2DKernels<f32x2, 0>::configure(smem, TT, bps);
    }
  } else if constexpr (std::is_same<T, float>::value) {
    if (tc == kTcBf16) return configure_tc<kTcBf16>(TT, smem, bps);
    if (tc == kTcF16) return configure_tc<kTcF16>(TT, smem, bps);
    switch (TT) {
      case 512: return Col2DKernels<float, 512>::configure(smem, TT, bps);
      case 256: return Col2DKernels<float, 256>::configure(smem, TT, bps);
      case 128: return Col2DKernels<float, 128>::configure(smem, TT, bps);
      case 64: return Col2DKernels<float, 64>::configure(smem, TT, bps);
      default: return Col2DKernels<float, 32>::configure(smem, TT, bps);
    }
  } else {
    return Col2DKernels<T, 0>::configure(smem, TT, bps);
  }
}

template <typename T>
static void launch_col2d(const bem_plan_s* p, int nf, const Col2Dv2Params<T>& cp, cudaStream_t st) {
  const int TT = p->threads;
  if constexpr (std::is_same<T, f32x2>::value) {
    switch (TT) {
      case 512: Col2DKernels<f32x2, 512>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 256: Col2DKernels<f32x2, 256>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 128: Col2DKernels<f32x2, 128>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 64: Col2DKernels<f32x2, 64>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      default: Col2DKernels<f32x2, 0>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
    }
  } else if constexpr (std::is_same<T, float>::value) {
    if (p->tc == kTcBf16) return launch_tc<kTcBf16>(p, nf, cp, st);
    if (p->tc == kTcF16) return launch_tc<kTcF16>(p, nf, cp, st);
    switch (TT) {
      case 512: Col2DKernels<float, 512>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 256: Col2DKernels<float, 256>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 128: Col2DKernels<float, 128>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      case 64: Col2DKernels<float, 64>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
      default: Col2DKernels<float, 32>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch); break;
    }
  } else {
    Col2DKernels<T, 0>::launch(nf, p->grid, TT, p->smem_bytes, st, cp, p->cell_batch);
  }
}

template <typename T>
static bem_status setup_v2_t(bem_plan_s* p) {
  constexpr bool R = std::is_same<T, float>::value;
  const int64_t n = p->n, nb = p->nb;
  const int TT = (int)(p->N / 16);
  p->threads = TT;
  // equal contiguous cell ranges; a row may be split between neighbouring
  // threads (its first holder stores the row, the others carry)
  std::vector<int32_t> chunk(TT + 1), tinfo(TT, 0);
  {
    // q or q + 1 cells per thread; with fewer cells than threads the empty
    // ranges all come last
    const int64_t q = nb / TT, r = nb % TT;
    for (int t = 0; t <= TT; ++t) chunk[t] = (int32_t)(t * q + std::min<int64_t>(t, r));
  }
  p->h_cellflag.assign(nb, 0u);
  p->v2_carry = false;
  for (int t = 0; t < TT; ++t) {
    const int64_t c0 = chunk[t], c1 = chunk[t + 1];
    if (c0 == c1) continue;
    const bool cont = c0 > 0 && p->h_row[c0 - 1] == p->h_row[c0];
    for (int64_t j = c0; j < c1; ++j) {
      if (j + 1 == c1 || p->h_row[j + 1] != p->h_row[j]) p->h_cellflag[j] |= 1u;  // last of its row here
      if (cont && p->h_row[j] == p->h_row[c0]) p->h_cellflag[j] |= 2u;            // carried
    }
    // threads after t whose first row continues t's last row (t holds its first cell)
    const int32_t last = p->h_row[c1 - 1];
    const bool owner = !(cont && last == p->h_row[c0]);
    if (owner) {
      int k = 0;
      for (int u = t + 1; u < TT && chunk[u] < chunk[u + 1] && p->h_row[chunk[u]] == last; ++u) ++k;
      tinfo[t] |= k << 8;
      if (k) p->v2_carry = true;
    }
  }
  for (int64_t j = 0; j < nb; ++j) {
    const int32_t r = p->h_row[j];
    tinfo[r % TT] |= 1 << (r / TT);  // row r = t + m*TT, m < 8
  }
  // interleaved positions: i-th cell of thread t at i*TT + t
  const int64_t Q = (nb + TT * kCellPad - 1) / (TT * kCellPad) * kCellPad;  // whole batches of either size
  p->v2_npos = Q * TT;
  p->h_pos.assign(nb, 0);
  std::vector<int32_t> perm_il(p->v2_npos, -1);
  for (int t = 0; t < TT; ++t)
    for (int64_t j = chunk[t]; j < chunk[t + 1]; ++j) {
      const int64_t pos = (j - chunk[t]) * TT + t;
      p->h_pos[j] = pos;
      perm_il[pos] = p->h_perm[j];
    }
  BEM_CUDA_TRY(cudaMalloc(&p->d_perm_il, p->v2_npos * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMemcpy(p->d_perm_il, perm_il.data(), p->v2_npos * sizeof(int32_t), cudaMemcpyHostToDevice));
  {
    // four-step and sparse twiddle tables, FP64 on the host, rounded once
    const int W = TT / 32;
    const int64_t N = p->N;
    const double PI = 3.14159265358979323846;
    std::vector<cplx<T>> tab;
    auto push = [&](double num, double den) {
      const double a = 2.0 * PI * num / den;
      tab.push_back({(T)std::cos(a), (T)std::sin(a)});
    };
    for (int k = 0; k < 16; ++k)
      for (int l = 0; l < 32; ++l) push((double)(l * k), (double)N);                  // lane
    for (int a = 0; a < W; ++a)
      for (int k = 0; k < 16; ++k) push((double)(32 * a * k % N), (double)N);         // warp
    for (int k = 0; k < 16; ++k)
      for (int l = 0; l < 32; ++l) push((double)((l * k) % TT), (double)TT);           // t5
    for (int i = 0; i < 128; ++i) push((double)i, 128.0);                             // hi
    for (int64_t i = 0; i < N / 128; ++i) push((double)i, (double)N);                 // lo
    if ((int)tab.size() != fstab_entries(TT)) {
      set_error("internal: twiddle table size");
      return BEM_ERR_CUDA;
    }
    BEM_CUDA_TRY(cudaMalloc(&p->d_fstab, tab.size() * sizeof(cplx<T>)));
    BEM_CUDA_TRY(cudaMemcpy(p->d_fstab, tab.data(), tab.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice));
  }
  if (p->tc) {
    if (!std::is_same<T, float>::value || (TT != 128 && TT != 256 && TT != 512)) {
      set_error("tensor-core DFT stages need FP32 and n = 1024, 2048 or 4096");
      return BEM_ERR_UNSUPPORTED;
    }
    const std::vector<uint16_t> mats = tc_matrices(p->tc, TT / 32);
    BEM_CUDA_TRY(cudaMalloc(&p->d_tcmat, mats.size() * sizeof(uint16_t)));
    BEM_CUDA_TRY(cudaMemcpy(p->d_tcmat, mats.data(), mats.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    BEM_CUDA_TRY(cudaMalloc(&p->d_status, sizeof(int)));
    BEM_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)));
  }
  BEM_CUDA_TRY(cudaMalloc(&p->d_tinfo, TT * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMalloc(&p->d_chunk, (TT + 1) * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMemcpy(p->d_tinfo, tinfo.data(), TT * sizeof(int32_t), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemcpy(p->d_chunk, chunk.data(), (TT + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  int dev = 0, nsm = 0, smem_optin = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // staging rows for fields 1, 2 only when the multi-field kernels can run
  const bool staging = R && !p->single_only;
  const int64_t Qc = (nb + TT - 1) / TT;  // most cells of one thread
  p->acc_in_smem = smem_v2<T>(n, TT, Qc * TT, staging, true, p->tc != 0) <= (size_t)smem_optin;
  p->acc_rows = p->acc_in_smem ? (int)Qc : 0;
  if (!p->acc_in_smem && TT == 512) {
    // one CTA per SM either way: fill the rest of shared memory with as many
    // accumulator rows as fit, the others stay in the partial sums
    const size_t base = smem_v2<T>(n, TT, 0, staging, false, p->tc != 0);
    if (base < (size_t)smem_optin)
      p->acc_rows = (int)std::min<int64_t>(Qc, (int64_t)(((size_t)smem_optin - base) / ((size_t)TT * sizeof(T))));
  }
  p->smem_bytes = smem_v2<T>(n, TT, 0, staging, false, p->tc != 0) + (size_t)p->acc_rows * TT * sizeof(T);
  if (p->smem_bytes > (size_t)smem_optin) {
    set_error("grid too large for the shared-memory column buffers");
    return BEM_ERR_UNSUPPORTED;
  }
  int bps = 0;
  BEM_CUDA_TRY(configure_col2d<T>(TT, p->tc, p->smem_bytes, &bps));
  if (bps < 1) {
    set_error("column kernel cannot be resident (registers/shared memory)");
    return BEM_ERR_UNSUPPORTED;
  }
  p->grid = (int)std::min<int64_t>((int64_t)bps * nsm, n + 1);
  const size_t tb = sizeof(T);
  const int64_t npos = p->v2_npos;
  BEM_CUDA_TRY(cudaMalloc(&p->d_partial, (size_t)p->grid * npos * tb));
  BEM_CUDA_TRY(cudaMalloc(&p->d_val, (size_t)npos * 2 * tb));
  // per-CTA cache of each cell's sparse twiddle for the gather: kept only while
  // it stays L2-resident beside the streamed spectra and the partial sums
  // (larger cell sets recompute the twiddle in the gather)
  const size_t twc_bytes = (size_t)p->grid * npos * 2 * tb;
  if (twc_bytes <= kTwiddleCacheMax) BEM_CUDA_TRY(cudaMalloc(&p->d_twc, twc_bytes));
  p->scratch_bytes += (size_t)p->grid * npos * tb + (size_t)npos * 2 * tb + (p->d_twc ? twc_bytes : 0);
  if constexpr (std::is_same<T, float>::value) {
    if (p->p3) return setup_p3(p);
  }
  return BEM_OK;
}

bem_status setup_apply_2d(bem_plan_s* p) {
  if (p->log2N < 3 || p->log2N > 13) {
    set_error("2D grids need 4 <= n <= 4096, n a power of two");
    return BEM_ERR_UNSUPPORTED;
  }
  p->v2 = p->log2N >= 9;
  if (p->v2) {
    if (p->prec == BEM_F32X2) return setup_v2_t<f32x2>(p);
    return p->prec == BEM_F64 ? setup_v2_t<double>(p) : setup_v2_t<float>(p);
  }
  if (p->prec == BEM_F32X2) {
    set_error("BEM_F32X2 needs the four-step column kernel (n >= 256)");
    return BEM_ERR_UNSUPPORTED;
  }
  return p->prec == BEM_F64 ? setup_t<double>(p) : setup_t<float>(p);
}

bem_status build_op_v2(bem_plan_s* p, Operator& op, const std::vector<double>& coefA, const std::vector<double>& coefB,
                       const std::vector<uint8_t>& type) {
  // cell words and coefficients in the interleaved position order (padding:
  // zero word, zero coefficients)
  const int64_t nb = p->nb, npos = p->v2_npos;
  std::vector<uint32_t> meta(npos, 0u);
  for (int64_t j = 0; j < nb; ++j)
    meta[p->h_pos[j]] = (uint32_t)p->h_col[j] | ((uint32_t)rowslot(p->h_row[j]) << 12) |
                        ((uint32_t)p->h_cellflag[j] << 29) | ((uint32_t)(type[j] ? 1u : 0u) << 31);
  void* dm = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&dm, npos * sizeof(uint32_t)));
  BEM_CUDA_TRY(cudaMemcpy(dm, meta.data(), npos * sizeof(uint32_t), cudaMemcpyHostToDevice));
  op.owned.push_back(dm);
  op.meta = static_cast<const uint32_t*>(dm);
  for (int k = 0; k < 2; ++k) {
    const std::vector<double>& csort = k == 0 ? coefA : coefB;
    std::vector<double> c(npos, 0.0);
    for (int64_t j = 0; j < nb; ++j) c[p->h_pos[j]] = csort[j];
    void* d = nullptr;
    bem_status rc = upload_real(p, c.data(), c.size(), false, &d);
    if (rc != BEM_OK) return rc;
    op.owned.push_back(d);
    (k == 0 ? op.coefA : op.coefB) = d;
  }
  return BEM_OK;
}

template <typename T, int E, int NF, bool ACCREG>
static void launch_col(const bem_plan_s* p, const Col2DParams<T>& cp, cudaStream_t st) {
  k_col2d<T, E, NF, ACCREG><<<p->grid, p->threads, p->smem_bytes, st>>>(cp);
}

template <typename T, int E>
static void launch_col_nf(const bem_plan_s* p, int nf, const Col2DParams<T>& cp, cudaStream_t st) {
  constexpr bool R = std::is_same<T, float>::value;
  if (nf == 1) launch_col<T, E, 1, false>(p, cp, st);
  else if (nf == 2) launch_col<T, E, 2, R>(p, cp, st);
  else launch_col<T, E, 3, R>(p, cp, st);
}

template <typename T>
static bem_status launch_v1(bem_plan_s* p, const Operator& op, const void* in, void* out, const ScratchPtrs& sp,
                            bool timed, cudaStream_t st) {
  PrepParams<T> pp{};
  pp.ncomp = p->ncomp;
  pp.nf = op.nf;
  pp.perm = p->d_perm;
  pp.in = static_cast<const T*>(in);
  int64_t maxe = 1;
  for (int f = 0; f < op.nf; ++f) {
    pp.coef[f] = static_cast<const T*>(op.f[f].coef);
    pp.cidx[f] = op.f[f].set->d_cidx;
    pp.nelem[f] = op.f[f].set->nelem;
    pp.comp[f] = op.f[f].comp;
    pp.rho[f] = static_cast<T*>(sp.rho[f]);
    maxe = std::max(maxe, op.f[f].set->nelem);
  }
  const int tb = 256;
  k_prep<T><<<dim3((unsigned)((maxe + tb - 1) / tb), op.nf), tb, 0, st>>>(pp);
  const SlotSet& ga = p->all_set;
  Col2DParams<T> cp{};
  cp.n = (int)p->n;
  cp.log2N = p->log2N;
  cp.G = ga.G;
  cp.H = ga.H;
  for (int f = 0; f < op.nf; ++f) {
    const Spectrum& s = p->spectra[op.f[f].spec];
    cp.spec[f] = static_cast<const T*>(s.data);
    cp.imag[f] = s.imag;
    cp.oddy[f] = s.odd[1];
    cp.cnt[f] = op.f[f].set->d_cnt;
    cp.off[f] = op.f[f].set->d_off;
    cp.xs[f] = op.f[f].set->d_x;
    cp.rho[f] = static_cast<const T*>(sp.rho[f]);
  }
  cp.gcnt = ga.d_cnt;
  cp.goff = ga.d_off;
  cp.gx = ga.d_x;
  cp.gnelem = ga.nelem;
  cp.qtab = static_cast<const cplx<T>*>(p->d_qtab);
  cp.partial = static_cast<T*>(sp.partial);
  cp.acc_in_smem = p->acc_in_smem ? 1 : 0;
  cudaEvent_t e1 = nullptr;
  if (timed && (e1 = timing_begin(p, st)) == nullptr) return BEM_ERR_CUDA;
  if (elems_per_thread(p->log2N) == 4)
    launch_col_nf<T, 4>(p, op.nf, cp, st);
  else
    launch_col_nf<T, 8>(p, op.nf, cp, st);
  if (timed) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k_reduce<T><<<(unsigned)((ga.nelem + 31) / 32), 512, 0, st>>>(
      static_cast<const T*>(sp.partial), p->grid, ga.nelem, ga.d_cidx, p->d_perm, static_cast<const T*>(op.diag),
      static_cast<const T*>(in), static_cast<T*>(out));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// kernel parameters of one plan's four-step apply
template <typename T>
static Col2Dv2Params<T> col2d_params(const bem_plan_s* p, const Operator& op, const ScratchPtrs& sp) {
  const int nb = (int)p->nb;
  const int npos = (int)p->v2_npos;
  Col2Dv2Params<T> cp{};
  cp.n = (int)p->n;
  cp.log2N = p->log2N;
  cp.nb = nb;
  cp.chunk = p->d_chunk;
  cp.tinfo = p->d_tinfo;
  cp.meta = op.meta;
  cp.val = static_cast<const cplx<T>*>(sp.val);
  for (int f = 0; f < op.nf; ++f) {
    const Spectrum& s = p->spectra[op.f[f].spec];
    cp.spec[f] = static_cast<const T*>(s.data);
    cp.imag[f] = s.imag;
    cp.oddy[f] = s.odd[1];
  }
  cp.fstab = static_cast<const cplx<T>*>(p->d_fstab);
  cp.partial = static_cast<T*>(sp.partial);
  cp.twc = static_cast<cplx<T>*>(sp.twc);
  cp.npos = npos;
  cp.acc_rows = p->acc_rows;
  cp.has_carry = p->v2_carry ? 1 : 0;
  cp.tcmat = static_cast<const uint4*>(p->d_tcmat);
  cp.status = p->d_status;
  cp.tc_no_commit = (p->test_flags & BEM_TEST_WAIT_RUNS_OUT) != 0 ? 1 : 0;
  return cp;
}

// T: arithmetic type of the column kernel; TIO: type of the caller's vectors
template <typename T, typename TIO>
static bem_status launch_v2(bem_plan_s* p, const Operator& op, const void* in, void* out, const ScratchPtrs& sp,
                            bool timed, cudaStream_t st) {
  const int tb = 256;
  const int npos = (int)p->v2_npos;
  k_prep_v2<T, TIO><<<(npos + tb - 1) / tb, tb, 0, st>>>(npos, p->d_perm_il, static_cast<const TIO*>(in),
                                                  static_cast<const T*>(op.coefA), static_cast<const T*>(op.coefB),
                                                  static_cast<cplx<T>*>(sp.val));
  const Col2Dv2Params<T> cp = col2d_params<T>(p, op, sp);
  cudaEvent_t e1 = nullptr;
  if (timed && (e1 = timing_begin(p, st)) == nullptr) return BEM_ERR_CUDA;
  launch_col2d<T>(p, op.nf, cp, st);
  if (timed) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k_reduce_v2<T, TIO><<<(npos + 31) / 32, 512, 0, st>>>(
      static_cast<const T*>(sp.partial), p->grid, npos, p->d_perm_il, static_cast<const TIO*>(op.diag),
      static_cast<const TIO*>(in), static_cast<TIO*>(out));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// ------------------------------------------------------------ three-pass form
// The same operator in three passes through HBM (FP32 four-step plans): the
// input-pruned x-DFT of every field row by row (k_p3_rows, X[f][kx][y]), the
// column transforms with the spectral multiply (k_p3_cols, Y[kx][y]), and the
// output-pruned inverse x-DFT at the cells (k_p3_gather: partial sums per chunk
// of columns, then k_p3_reduce in a fixed order).  Each row pass gives a warp
// 32 consecutive grid rows, one per lane, and a chunk of columns, so every
// load and store of X and Y is one contiguous segment per warp; the per-cell
// work no longer repeats in every CTA of the column pass.

// per sorted cell: x (as int bits) and the three field values of the apply
__global__ void k_p3_prep(int nb, const int32_t* __restrict__ perm, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ pos, const uint32_t* __restrict__ meta,
                          const float* __restrict__ coefA, const float* __restrict__ coefB,
                          const float* __restrict__ in, float4* __restrict__ cell4) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb) return;
  const int ps = pos[c];
  const float x = in[perm[c]];
  const float a = coefA[ps] * x, b = coefB[ps] * x;
  const bool ty = (meta[ps] >> 31) != 0;
  cell4[c] = make_float4(__int_as_float(col[c]), ty ? 0.f : a, ty ? a : b, ty ? b : 0.f);
}

constexpr int kP3Rows = 256;  // threads per block of the row passes (8 warps of 32 rows)

template <int NF>
__global__ void __launch_bounds__(kP3Rows) k_p3_rows(int n, int log2N, const int32_t* __restrict__ rowptr,
                                                      const float4* __restrict__ cell4,
                                                      const cplx<float>* __restrict__ hi, int kc,
                                                      cplx<float>* __restrict__ X) {
  __shared__ cplx<float> shi[128];
  for (int i = threadIdx.x; i < 128; i += kP3Rows) shi[i] = hi[i];
  __syncthreads();
  const int Nm = (1 << log2N) - 1;
  const Twiddles2L<float> tw{shi, nullptr, log2N - 7, (float)(6.283185307179586476925 / (double)(1 << log2N))};
  const int r = blockIdx.x * kP3Rows + threadIdx.x;
  if (r >= n) return;
  const int c0 = rowptr[r], c1 = rowptr[r + 1];
  const int k0 = blockIdx.y * kc, k1 = min(k0 + kc, n + 1);
  // four columns per pass over the row's cells: each cell load serves four
  // independent twiddles and sums
  constexpr int KU = 4;
  for (int kb = k0; kb < k1; kb += KU) {
    cplx<float> s[KU][3];
#pragma unroll
    for (int i = 0; i < KU; ++i) s[i][0] = s[i][1] = s[i][2] = {0.f, 0.f};
    for (int c = c0; c < c1; ++c) {
      const float4 q = cell4[c];
      const int x = __float_as_int(q.x);
#pragma unroll
      for (int i = 0; i < KU; ++i) {
        const cplx<float> w = tw.template get<-1>(((kb + i) * x) & Nm);
        s[i][0].x += q.y * w.x;
        s[i][0].y += q.y * w.y;
        if (NF > 1) {
          s[i][1].x += q.z * w.x;
          s[i][1].y += q.z * w.y;
        }
        if (NF > 2) {
          s[i][2].x += q.w * w.x;
          s[i][2].y += q.w * w.y;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < KU; ++i) {
      const int kx = kb + i;
      if (kx < k1) {
        X[(size_t)kx * n + r] = s[i][0];
        if (NF > 1) X[((size_t)(n + 1) + kx) * n + r] = s[i][1];
        if (NF > 2) X[((size_t)2 * (n + 1) + kx) * n + r] = s[i][2];
      }
    }
  }
}

// columns per chunk of the row passes
constexpr int kP3Chunk = 32;

// One lane per grid row: the row's values of the chunk's columns are loaded
// into registers first (all loads in flight at once), then every cell of the
// row sums its chunk of the inverse x-DFT.
__global__ void __launch_bounds__(kP3Rows) k_p3_gather(int n, int log2N, int nb, const int32_t* __restrict__ rowptr,
                                                        const float4* __restrict__ cell4,
                                                        const cplx<float>* __restrict__ hi,
                                                        const cplx<float>* __restrict__ Y, float* __restrict__ part) {
  __shared__ cplx<float> shi[128];
  for (int i = threadIdx.x; i < 128; i += kP3Rows) shi[i] = hi[i];
  __syncthreads();
  const int Nm = (1 << log2N) - 1;
  const Twiddles2L<float> tw{shi, nullptr, log2N - 7, (float)(6.283185307179586476925 / (double)(1 << log2N))};
  const int r = blockIdx.x * kP3Rows + threadIdx.x;
  if (r >= n) return;
  const int c0 = rowptr[r], c1 = rowptr[r + 1];
  if (c0 == c1) return;
  const int k0 = blockIdx.y * kP3Chunk;
  cplx<float> yv[kP3Chunk];
#pragma unroll
  for (int j = 0; j < kP3Chunk; ++j) {
    const int kx = k0 + j;
    yv[j] = kx <= n ? Y[(size_t)kx * n + r] : cplx<float>{0.f, 0.f};
  }
  for (int c = c0; c < c1; ++c) {
    const int x = __float_as_int(cell4[c].x);
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kP3Chunk; ++j) {
      const int kx = k0 + j;
      const cplx<float> w = tw.template get<+1>((kx * x) & Nm);
      const float ck = (kx == 0 || kx == n) ? 1.f : 2.f;
      acc += ck * (yv[j].x * w.x - yv[j].y * w.y);  // beyond n: yv is zero
    }
    part[(size_t)blockIdx.y * nb + c] = acc;
  }
}

// out[perm[c]] = sum over chunks of part[chunk][c] (compensated, fixed order)
// + diag * in; eight loads in flight per thread
__global__ void __launch_bounds__(64) k_p3_reduce(int nb, int nchunk, const float* __restrict__ part,
                                                  const int32_t* __restrict__ perm, const float* __restrict__ diag,
                                                  const float* __restrict__ in, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb) return;
  CompSum t{0.f, 0.f};
  int k = 0;
  for (; k + 8 <= nchunk; k += 8) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = part[(size_t)(k + i) * nb + c];
#pragma unroll
    for (int i = 0; i < 8; ++i) t.add(v[i]);
  }
  for (; k < nchunk; ++k) t.add(part[(size_t)k * nb + c]);
  const int u = perm[c];
  if (diag) {
    const float pr = __fmul_rn(diag[u], in[u]);
    const float epr = fmaf(diag[u], in[u], -pr);
    t.add(pr);
    t.c = __fadd_rn(t.c, epr);
  }
  out[u] = __fadd_rn(t.p, t.c);
}

static cudaError_t p3_configure(int TT, size_t smem, int* bps) {
  switch (TT) {
    case 512: return Col2DPassKernels<512>::configure(smem, TT, bps);
    case 256: return Col2DPassKernels<256>::configure(smem, TT, bps);
    case 128: return Col2DPassKernels<128>::configure(smem, TT, bps);
    case 64: return Col2DPassKernels<64>::configure(smem, TT, bps);
    default: return Col2DPassKernels<32>::configure(smem, TT, bps);
  }
}

static bem_status setup_p3(bem_plan_s* p) {
  const int TT = p->threads, W = TT / 32;
  const int64_t n = p->n, nb = p->nb;
  const int nf = p->single_only ? 1 : 3;
  int dev = 0, nsm = 0, smem_optin = 0, bps = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t nbuf = (size_t)std::max(16 * TT, W * 544);
  p->p3_smem = (nbuf + (size_t)fstab_entries(TT)) * sizeof(cplx<float>) + (size_t)sspec_entries((int)n) * sizeof(float) +
               (size_t)nf * n * sizeof(cplx<float>);
  if (p->p3_smem > (size_t)smem_optin) {
    set_error("three-pass form: column buffers exceed shared memory");
    return BEM_ERR_UNSUPPORTED;
  }
  BEM_CUDA_TRY(p3_configure(TT, p->p3_smem, &bps));
  if (bps < 1) {
    set_error("three-pass column kernel cannot be resident");
    return BEM_ERR_UNSUPPORTED;
  }
  p->p3_grid = (int)std::min<int64_t>((int64_t)bps * nsm, n + 1);
  p->p3_nchunk = (int)((n + 1 + kP3Chunk - 1) / kP3Chunk);
  std::vector<int32_t> pos(nb);
  for (int64_t c = 0; c < nb; ++c) pos[c] = (int32_t)p->h_pos[c];
  const size_t xb = (size_t)nf * (n + 1) * n * sizeof(cplx<float>), yb = (size_t)(n + 1) * n * sizeof(cplx<float>);
  BEM_CUDA_TRY(cudaMalloc(&p->d_p3X, xb));
  BEM_CUDA_TRY(cudaMalloc(&p->d_p3Y, yb));
  BEM_CUDA_TRY(cudaMalloc(&p->d_p3part, (size_t)p->p3_nchunk * nb * sizeof(float)));
  BEM_CUDA_TRY(cudaMalloc(&p->d_p3cell, (size_t)nb * sizeof(float4)));
  BEM_CUDA_TRY(cudaMalloc(&p->d_p3pos, (size_t)nb * sizeof(int32_t)));
  BEM_CUDA_TRY(cudaMemcpy(p->d_p3pos, pos.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice));
  p->scratch_bytes += xb + yb + (size_t)p->p3_nchunk * nb * sizeof(float) + (size_t)nb * (sizeof(float4) + 4);
  return BEM_OK;
}

static bem_status launch_p3(bem_plan_s* p, const Operator& op, const float* in, float* out, bool timed,
                            cudaStream_t st) {
  const int n = (int)p->n, nb = (int)p->nb, TT = p->threads, W = TT / 32;
  const cplx<float>* hi = static_cast<const cplx<float>*>(p->d_fstab) + 1024 + W * 16;
  cplx<float>* X = static_cast<cplx<float>*>(p->d_p3X);
  cplx<float>* Y = static_cast<cplx<float>*>(p->d_p3Y);
  float4* cell4 = static_cast<float4*>(p->d_p3cell);
  k_p3_prep<<<(nb + 255) / 256, 256, 0, st>>>(nb, p->d_perm, p->d_col, p->d_p3pos, op.meta,
                                               static_cast<const float*>(op.coefA), static_cast<const float*>(op.coefB),
                                               in, cell4);
  const dim3 rg((unsigned)((n + kP3Rows - 1) / kP3Rows), (unsigned)p->p3_nchunk);
  if (op.nf == 1) k_p3_rows<1><<<rg, kP3Rows, 0, st>>>(n, p->log2N, p->d_rowptr, cell4, hi, kP3Chunk, X);
  else if (op.nf == 2) k_p3_rows<2><<<rg, kP3Rows, 0, st>>>(n, p->log2N, p->d_rowptr, cell4, hi, kP3Chunk, X);
  else k_p3_rows<3><<<rg, kP3Rows, 0, st>>>(n, p->log2N, p->d_rowptr, cell4, hi, kP3Chunk, X);
  ScratchPtrs sp{};
  Col2Dv2Params<float> cp = col2d_params<float>(p, op, sp);
  cp.X = X;
  cp.Y = Y;
  cudaEvent_t e1 = nullptr;
  if (timed && (e1 = timing_begin(p, st)) == nullptr) return BEM_ERR_CUDA;
  switch (TT) {
    case 512: Col2DPassKernels<512>::launch(op.nf, p->p3_grid, TT, p->p3_smem, st, cp); break;
    case 256: Col2DPassKernels<256>::launch(op.nf, p->p3_grid, TT, p->p3_smem, st, cp); break;
    case 128: Col2DPassKernels<128>::launch(op.nf, p->p3_grid, TT, p->p3_smem, st, cp); break;
    case 64: Col2DPassKernels<64>::launch(op.nf, p->p3_grid, TT, p->p3_smem, st, cp); break;
    default: Col2DPassKernels<32>::launch(op.nf, p->p3_grid, TT, p->p3_smem, st, cp); break;
  }
  if (timed) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k_p3_gather<<<rg, kP3Rows, 0, st>>>(n, p->log2N, nb, p->d_rowptr, cell4, hi, Y, static_cast<float*>(p->d_p3part));
  k_p3_reduce<<<(nb + 63) / 64, 64, 0, st>>>(nb, p->p3_nchunk, static_cast<const float*>(p->d_p3part), p->d_perm,
                                             static_cast<const float*>(op.diag), in, out);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

// ------------------------------------------------ edge-flow node convolution

template <typename T>
static cudaError_t edge_configure(int TT, size_t smem, int* bps) {
  if constexpr (std::is_same<T, float>::value) {
    switch (TT) {
      case 512: return Col2DEdgeKernels<float, 512>::configure(smem, TT, bps);
      case 256: return Col2DEdgeKernels<float, 256>::configure(smem, TT, bps);
      case 128: return Col2DEdgeKernels<float, 128>::configure(smem, TT, bps);
      case 64: return Col2DEdgeKernels<float, 64>::configure(smem, TT, bps);
      default: return Col2DEdgeKernels<float, 32>::configure(smem, TT, bps);
    }
  } else if constexpr (std::is_same<T, f32x2>::value) {
    switch (TT) {
      case 512: return Col2DEdgeKernels<f32x2, 512>::configure(smem, TT, bps);
      case 256: return Col2DEdgeKernels<f32x2, 256>::configure(smem, TT, bps);
      case 128: return Col2DEdgeKernels<f32x2, 128>::configure(smem, TT, bps);
      case 64: return Col2DEdgeKernels<f32x2, 64>::configure(smem, TT, bps);
      default: return Col2DEdgeKernels<f32x2, 0>::configure(smem, TT, bps);
    }
  } else {
    return Col2DEdgeKernels<T, 0>::configure(smem, TT, bps);
  }
}

template <typename T>
static void edge_launch(const bem_plan_s* p, const Col2Dv2Params<T>& cp, cudaStream_t st) {
  const int TT = p->threads, G = p->edge_grid;
  const size_t sm = p->edge_smem;
  if constexpr (std::is_same<T, float>::value) {
    switch (TT) {
      case 512: Col2DEdgeKernels<float, 512>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 256: Col2DEdgeKernels<float, 256>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 128: Col2DEdgeKernels<float, 128>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 64: Col2DEdgeKernels<float, 64>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      default: Col2DEdgeKernels<float, 32>::launch(G, TT, sm, st, cp, p->cell_batch); break;
    }
  } else if constexpr (std::is_same<T, f32x2>::value) {
    switch (TT) {
      case 512: Col2DEdgeKernels<f32x2, 512>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 256: Col2DEdgeKernels<f32x2, 256>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 128: Col2DEdgeKernels<f32x2, 128>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      case 64: Col2DEdgeKernels<f32x2, 64>::launch(G, TT, sm, st, cp, p->cell_batch); break;
      default: Col2DEdgeKernels<f32x2, 0>::launch(G, TT, sm, st, cp, p->cell_batch); break;
    }
  } else {
    Col2DEdgeKernels<T, 0>::launch(G, TT, sm, st, cp, p->cell_batch);
  }
}

template <typename T>
static bem_status setup_edge_t(bem_plan_s* p) {
  constexpr bool R = std::is_same<T, float>::value;
  const int TT = p->threads;
  const int64_t n = p->n, Q = (p->nb + TT - 1) / TT;  // most cells of one thread
  int dev = 0, nsm = 0, smem_optin = 0, bps = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // FP32: staging rows for the second field (its row sums are kept while the
  // first is transformed); accumulator rows as in setup_v2_t
  const size_t base = smem_v2<T>(n, TT, 0, R, false, false);
  if (base > (size_t)smem_optin) {
    set_error("grid too large for the edge-flow column buffers");
    return BEM_ERR_UNSUPPORTED;
  }
  int rows = (int)Q;
  if (smem_v2<T>(n, TT, Q * TT, R, true, false) > (size_t)smem_optin)
    rows = TT == 512 ? (int)std::min<int64_t>(Q, (int64_t)(((size_t)smem_optin - base) / ((size_t)TT * sizeof(T))))
                     : 0;
  p->edge_acc_rows = rows;
  p->edge_smem = base + (size_t)rows * TT * sizeof(T);
  BEM_CUDA_TRY(edge_configure<T>(TT, p->edge_smem, &bps));
  if (bps < 1) {
    set_error("edge-flow column kernel cannot be resident (registers/shared memory)");
    return BEM_ERR_UNSUPPORTED;
  }
  // never more CTAs than the plan's partial sums have rows for
  p->edge_grid = (int)std::min<int64_t>(std::min<int64_t>((int64_t)bps * nsm, n + 1), p->grid);
  if (!p->d_val2) {
    BEM_CUDA_TRY(cudaMalloc(&p->d_val2, (size_t)p->v2_npos * sizeof(T)));
    BEM_CUDA_TRY(cudaMemset(p->d_val2, 0, (size_t)p->v2_npos * sizeof(T)));
    p->scratch_bytes += (size_t)p->v2_npos * sizeof(T);
  }
  return BEM_OK;
}

bem_status setup_edge_2d(bem_plan_s* p) {
  if (!p->v2 || p->tc != 0 || p->threads < 32 || p->threads > 512) {
    set_error("internal: the edge-flow form needs a four-step plan without tensor-core stages");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->prec == BEM_F32X2) return setup_edge_t<f32x2>(p);
  return p->prec == BEM_F64 ? setup_edge_t<double>(p) : setup_edge_t<float>(p);
}

template <typename T, typename TIO>
static bem_status launch_edge_t(bem_plan_s* p, TIO* out, cudaStream_t st) {
  const int npos = (int)p->v2_npos;
  ScratchPtrs sp{};
  sp.val = p->d_val;
  sp.partial = p->d_partial;
  sp.twc = p->d_twc;
  Col2Dv2Params<T> cp = col2d_params<T>(p, p->op_single, sp);
  // both fields go through the single-layer spectrum (field 0)
  cp.spec[1] = cp.spec[0];
  cp.imag[1] = cp.imag[0];
  cp.oddy[1] = cp.oddy[0];
  cp.val2 = static_cast<const T*>(p->d_val2);
  cp.acc_rows = p->edge_acc_rows;
  cudaEvent_t e1 = nullptr;
  if (p->timing && (e1 = timing_begin(p, st)) == nullptr) return BEM_ERR_CUDA;
  edge_launch<T>(p, cp, st);
  if (p->timing) BEM_CUDA_TRY(cudaEventRecord(e1, st));
  k_reduce_v2<T, TIO><<<(npos + 31) / 32, 512, 0, st>>>(static_cast<const T*>(sp.partial), p->edge_grid, npos,
                                                       p->d_perm_il, nullptr, nullptr, out);
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

bem_status launch_edge_2d(bem_plan_s* p, void* out, cudaStream_t st) {
  if (p->prec == BEM_F32X2) return launch_edge_t<f32x2, double>(p, static_cast<double*>(out), st);
  if (p->prec == BEM_F64) return launch_edge_t<double, double>(p, static_cast<double*>(out), st);
  return launch_edge_t<float, float>(p, static_cast<float*>(out), st);
}

// ------------------------------------------------------ grouped batch applies

bool group_eligible(const bem_plan_s* p) {
  return p->dim == 2 && p->v2 && p->prec == BEM_F32 && p->tc == 0 && !p->pf && p->threads >= 32;
}

static const Operator* op_of(const bem_plan_s* p, bem_layer layer) {
  if (layer == BEM_SINGLE) return &p->op_single;
  if (layer == BEM_DOUBLE) return &p->op_double;
  return p->have_bc ? &p->op_system : nullptr;
}

void group_free(BatchGroup& g) {
  cudaFree(g.d_params);
  cudaFree(g.d_c0);
  g.d_params = nullptr;
  g.d_c0 = nullptr;
}

// resident CTAs per SM of the grouped kernels (their registers may differ
// from the per-plan kernels')
static cudaError_t group_configure(int TT, size_t smem, int* bps) {
  switch (TT) {
    case 512: return Col2DGroupKernels<512>::configure(smem, TT, bps);
    case 256: return Col2DGroupKernels<256>::configure(smem, TT, bps);
    case 128: return Col2DGroupKernels<128>::configure(smem, TT, bps);
    case 64: return Col2DGroupKernels<64>::configure(smem, TT, bps);
    default: return Col2DGroupKernels<32>::configure(smem, TT, bps);
  }
}

bem_status group_build(BatchGroup& g, const std::vector<bem_plan_s*>& plans, bem_layer layer) {
  group_free(g);
  const int P = (int)g.members.size();
  const bem_plan_s* p0 = plans[g.members[0]];
  g.threads = p0->threads;
  g.smem = 0;
  std::vector<Col2Dv2Params<float>> hp(P);
  for (int m = 0; m < P; ++m) {
    const bem_plan_s* p = plans[g.members[m]];
    const Operator* op = op_of(p, layer);
    if (!op) {
      set_error("bem_batch: BEM_SYSTEM needs bem_set_bc on every plan");
      return BEM_ERR_ARG;
    }
    ScratchPtrs sp{};
    sp.val = p->d_val;
    sp.partial = p->d_partial;
    sp.twc = p->d_twc;
    hp[m] = col2d_params<float>(p, *op, sp);
    g.nf = op->nf;
    g.smem = std::max(g.smem, p->smem_bytes);
  }
  int dev = 0, nsm = 0, bps = 0;
  BEM_CUDA_TRY(cudaGetDevice(&dev));
  BEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BEM_CUDA_TRY(group_configure(g.threads, g.smem, &bps));
  // never more CTAs than any member's partial sums have rows for
  int rows_max = p0->grid;
  for (int m = 0; m < P; ++m) rows_max = std::min(rows_max, plans[g.members[m]]->grid);
  const int64_t cols = (int64_t)P * (p0->n + 1);
  g.grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>((int64_t)std::max(bps, 1) * nsm, cols), (int64_t)P * (rows_max - 1)));
  // contiguous column ranges [b C / G, (b + 1) C / G); a member's rows are the
  // CTAs whose range meets its columns
  std::vector<int> c0(P, -1);
  g.rows.assign(P, 0);
  for (int b = 0; b < g.grid; ++b) {
    const int64_t lo = (int64_t)b * cols / g.grid, hi = ((int64_t)b + 1) * cols / g.grid;
    if (lo >= hi) continue;
    const int m0 = (int)(lo / (p0->n + 1)), m1 = (int)((hi - 1) / (p0->n + 1));
    for (int m = m0; m <= m1; ++m) {
      if (c0[m] < 0) c0[m] = b;
      g.rows[m] = b - c0[m] + 1;
    }
  }
  for (int m = 0; m < P; ++m)
    if (g.rows[m] > rows_max) {
      set_error("internal: grouped launch needs more partial rows than a plan holds");
      return BEM_ERR_UNSUPPORTED;
    }
  BEM_CUDA_TRY(cudaMalloc(&g.d_params, P * sizeof(Col2Dv2Params<float>)));
  BEM_CUDA_TRY(cudaMalloc(&g.d_c0, P * sizeof(int)));
  BEM_CUDA_TRY(cudaMemcpy(g.d_params, hp.data(), P * sizeof(Col2Dv2Params<float>), cudaMemcpyHostToDevice));
  BEM_CUDA_TRY(cudaMemcpy(g.d_c0, c0.data(), P * sizeof(int), cudaMemcpyHostToDevice));
  return BEM_OK;
}

bem_status group_issue(const BatchGroup& g, const std::vector<bem_plan_s*>& plans, bem_layer layer, const void* in,
                       void* out, const std::vector<size_t>& offset, cudaStream_t st) {
  const int tb = 256;
  const int P = (int)g.members.size();
  const float* fin = static_cast<const float*>(in);
  float* fout = static_cast<float*>(out);
  for (int m = 0; m < P; ++m) {
    const bem_plan_s* p = plans[g.members[m]];
    const Operator* op = op_of(p, layer);
    const int npos = (int)p->v2_npos;
    k_prep_v2<float, float><<<(npos + tb - 1) / tb, tb, 0, st>>>(
        npos, p->d_perm_il, fin + offset[g.members[m]], static_cast<const float*>(op->coefA),
        static_cast<const float*>(op->coefB), static_cast<cplx<float>*>(p->d_val));
  }
  const auto* dp = static_cast<const Col2Dv2Params<float>*>(g.d_params);
  switch (g.threads) {
    case 512: Col2DGroupKernels<512>::launch(g.nf, g.grid, 512, g.smem, st, dp, g.d_c0, P); break;
    case 256: Col2DGroupKernels<256>::launch(g.nf, g.grid, 256, g.smem, st, dp, g.d_c0, P); break;
    case 128: Col2DGroupKernels<128>::launch(g.nf, g.grid, 128, g.smem, st, dp, g.d_c0, P); break;
    case 64: Col2DGroupKernels<64>::launch(g.nf, g.grid, 64, g.smem, st, dp, g.d_c0, P); break;
    default: Col2DGroupKernels<32>::launch(g.nf, g.grid, 32, g.smem, st, dp, g.d_c0, P); break;
  }
  for (int m = 0; m < P; ++m) {
    const bem_plan_s* p = plans[g.members[m]];
    const Operator* op = op_of(p, layer);
    const int npos = (int)p->v2_npos;
    const size_t o = offset[g.members[m]];
    k_reduce_v2<float, float><<<(npos + 31) / 32, 512, 0, st>>>(
        static_cast<const float*>(p->d_partial), g.rows[m], npos, p->d_perm_il, static_cast<const float*>(op->diag),
        fin + o, fout + o);
  }
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

static inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t apply_scratch_bytes(const bem_plan_s* p, const Operator& op) {
  const size_t tb = prec_bytes(p);
  size_t need = 0;
  if (p->v2) {
    need += align256((size_t)p->v2_npos * 2 * tb);
    need += align256((size_t)p->grid * p->v2_npos * tb);
  } else {
    for (int f = 0; f < op.nf; ++f) need += align256((size_t)op.f[f].set->nelem * tb);
    need += align256((size_t)p->grid * p->all_set.nelem * p->ncomp * tb);
  }
  return need;
}

void carve_scratch(const bem_plan_s* p, const Operator& op, void* base, ScratchPtrs* sp) {
  const size_t tb = prec_bytes(p);
  unsigned char* b = static_cast<unsigned char*>(base);
  size_t off = 0;
  if (p->v2) {
    sp->val = b + off;
    off += align256((size_t)p->v2_npos * 2 * tb);
    sp->partial = b + off;
  } else {
    for (int f = 0; f < op.nf; ++f) {
      sp->rho[f] = b + off;
      off += align256((size_t)op.f[f].set->nelem * tb);
    }
    sp->partial = b + off;
  }
}

bem_status launch_apply_2d_with(bem_plan_s* p, const Operator& op, const void* in, void* out, const ScratchPtrs& sp,
                                bool timed, cudaStream_t st) {
  if (op.nf < 1 || op.nf > 3) {
    set_error("2D operator with unsupported field count");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->v2) {
    if (p->p3 && sp.partial == p->d_partial)
      return launch_p3(p, op, static_cast<const float*>(in), static_cast<float*>(out), timed, st);
    if (p->prec == BEM_F32X2) return launch_v2<f32x2, double>(p, op, in, out, sp, timed, st);
    return p->prec == BEM_F64 ? launch_v2<double, double>(p, op, in, out, sp, timed, st)
                              : launch_v2<float, float>(p, op, in, out, sp, timed, st);
  }
  return p->prec == BEM_F64 ? launch_v1<double>(p, op, in, out, sp, timed, st)
                            : launch_v1<float>(p, op, in, out, sp, timed, st);
}

bem_status launch_apply_2d(bem_plan_s* p, const Operator& op, const void* in, void* out, cudaStream_t st) {
  ScratchPtrs sp{};
  if (p->v2) {
    sp.val = p->d_val;
  } else {
    for (int f = 0; f < op.nf; ++f) sp.rho[f] = op.f[f].rho;
  }
  sp.partial = p->d_partial;
  sp.twc = p->d_twc;
  return launch_apply_2d_with(p, op, in, out, sp, p->timing, st);
}

}  // namespace bemfft
