// Restarted GMRES around the FFT operator apply (Section 4 solves for the
// unknown flux with a Krylov iteration whose matrix-vector product is the FFT
// apply; the paper uses conjugate gradients, this library uses GMRES(m) so
// that mixed boundary conditions, which make the system non-symmetric, are
// covered).
//
// Vectors live on the device in FP64.  Each iteration issues one operator
// apply in the plan precision, classical Gram-Schmidt with one
// re-orthogonalisation (two fused dot-product sweeps and two fused update
// sweeps over the basis), the norm and the normalisation, and copies the
// 2(j+1)+1 new Hessenberg entries to the host in one transfer.  Givens
// rotations, the least-squares update and the stop test run on the host in
// FP64 (a few hundred flops per iteration).
#include <chrono>
#include <cmath>
#include <vector>

#include "bem_internal.h"

namespace bemfft {

static constexpr int kDotThreads = 256;
static constexpr int kDotChunk = kDotThreads * 8;

// partial[v * nchunk + c] = sum over chunk c of V[v] . w
__global__ void k_dots_partial(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w, int64_t M,
                               int nchunk, double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  const int v = blockIdx.y, c = blockIdx.x;
  const double* a = V + (int64_t)v * ldv;
  double s = 0.0;
  const int64_t beg = (int64_t)c * kDotChunk;
  const int64_t end = beg + kDotChunk < M ? beg + kDotChunk : M;
  for (int64_t i = beg + threadIdx.x; i < end; i += kDotThreads) s += a[i] * w[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[(int64_t)v * nchunk + c] = s;
  }
}

// out[v] (+)= sum_c partial[v * nchunk + c]   (fixed order: deterministic)
__global__ void k_dots_final(const double* __restrict__ partial, int nvec, int nchunk, double* __restrict__ out,
                             int accumulate) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partial[(int64_t)v * nchunk + c];
  out[v] = accumulate ? out[v] + s : s;
}

// w[i] -= sum_k V[k][i] h[k]
__global__ void k_sub_basis(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                            double* __restrict__ w, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double s = w[i];
  for (int k = 0; k < nvec; ++k) s -= V[(int64_t)k * ldv + i] * h[k];
  w[i] = s;
}

// x[i] += sum_k V[k][i] y[k]
__global__ void k_add_basis(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ y,
                            double* __restrict__ x, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double s = x[i];
  for (int k = 0; k < nvec; ++k) s += V[(int64_t)k * ldv + i] * y[k];
  x[i] = s;
}

// dst = src / sqrt(*nrm2) (nrm2 is a squared norm on the device)
__global__ void k_normalize(const double* __restrict__ src, const double* __restrict__ nrm2, double* __restrict__ dst,
                            int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double s = sqrt(*nrm2);
  dst[i] = s > 0.0 ? src[i] / s : 0.0;
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ src, B* __restrict__ dst, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) dst[i] = (B)src[i];
}

// y = a * x + b * y
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) y[i] = a * x[i] + b * y[i];
}

// out[b*bs + i] = sum_j inv_b[i][j] in[b*bs + j]   (block-Jacobi M^-1): CTA
// (b, r) computes rows r*8 .. r*8+7 of block b, one warp per row (the lanes
// read the row contiguously and add their products in a fixed tree)
constexpr int kBlockApplyRows = 8;
__global__ void __launch_bounds__(32 * kBlockApplyRows) k_block_apply(const double* __restrict__ inv, int bs,
                                                                     int64_t M, const double* __restrict__ in,
                                                                     double* __restrict__ out) {
  extern __shared__ double xin[];
  const int b = blockIdx.x, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)b * bs;
  const int sz = (int)(M - i0 < bs ? M - i0 : bs);
  for (int j = threadIdx.x; j < sz; j += blockDim.x) xin[j] = in[i0 + j];
  __syncthreads();
  const int i = blockIdx.y * kBlockApplyRows + wp;
  if (i >= sz) return;
  const double* row = inv + ((size_t)b * bs + i) * bs;
  double s = 0.0;
  for (int j = lane; j < sz; j += 32) s += row[j] * xin[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[i0 + i] = s;
}

static inline dim3 block_apply_grid(int nblocks, int bs) {
  return dim3((unsigned)nblocks, (unsigned)((bs + kBlockApplyRows - 1) / kBlockApplyRows));
}

// z = M^-1 v on one plan's segment (m unknowns per block)
static void block_apply(const bem_plan_s* p, int m, int64_t M, const double* v, double* z, cudaStream_t st) {
  k_block_apply<<<block_apply_grid(p->pc.nblocks, m), 32 * kBlockApplyRows, m * sizeof(double), st>>>(p->pc.d_inv, m,
                                                                                                   M, v, z);
}

// masked copies: um = data * (1 - bc), qm = data * bc
__global__ void k_split_known(const double* __restrict__ data, const uint8_t* __restrict__ bc, double* __restrict__ um,
                              double* __restrict__ qm, int64_t M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double d = data[i];
  const bool neu = bc[i] != 0;
  um[i] = neu ? 0.0 : d;
  qm[i] = neu ? d : 0.0;
}

static inline unsigned blocks_for(int64_t M, int tb) { return (unsigned)((M + tb - 1) / tb); }

// Relative tolerance of the inner low-precision solve of one refinement step,
// for outer residual `rel` (relative to b) and target `tol`: deep enough that
// one step can reach tol (0.3 tol / rel), never below what the FP32 operator's
// own recomputed residuals resolve (plain FP32 GMRES stalls near 2e-6 on the
// 4096^2 star; the floor keeps a margin of five), and at most 0.1.  One deep
// inner solve keeps its Krylov space, where several shallow ones would restart
// it; a good initial guess (small rel) then saves whole refinement steps.
// ||r|| / ||b|| with 0 for b = 0 and NaN when either norm is not finite (so
// that non-finite data end the solve with BEM_ERR_NONFINITE)
static inline double rel_norm(double r, double b) {
  if (!std::isfinite(r) || !std::isfinite(b)) return NAN;
  return b > 0 ? r / b : 0.0;
}

// whether residuals formed with plan r are accurate to FP64 level (FP64 or
// double-float arithmetic)
static inline bool fp64_residual(const bem_plan_s* r) { return r->prec == BEM_F64 || r->prec == BEM_F32X2; }

static inline double inner_tolerance(double tol, double rel) {
  return std::min(std::max(1e-5, 0.3 * tol / std::max(rel, 1e-300)), 0.1);
}

struct Gm {
  bem_plan_s* p;
  cudaStream_t st;
  int64_t M;
  double* partial = nullptr;
  int nchunk = 0;
  bool fp64;

  // w (FP64) = A x (FP64) with the plan-precision apply
  bem_status apply(bem_layer layer, const double* x, double* w) {
    if (fp64) return apply_operator(p, layer, x, w, st);
    k_convert<double, float><<<blocks_for(M, 256), 256, 0, st>>>(x, static_cast<float*>(p->d_tin), M);
    bem_status rc = apply_operator(p, layer, p->d_tin, p->d_tout, st);
    if (rc != BEM_OK) return rc;
    k_convert<float, double><<<blocks_for(M, 256), 256, 0, st>>>(static_cast<const float*>(p->d_tout), w, M);
    return BEM_OK;
  }
  // w (FP64) = A' x with the complementary mask's operator (apply_complement)
  bem_status apply_comp(const double* x, double* w) {
    if (fp64) return apply_complement(p, x, w, st);
    k_convert<double, float><<<blocks_for(M, 256), 256, 0, st>>>(x, static_cast<float*>(p->d_tin), M);
    bem_status rc = apply_complement(p, p->d_tin, p->d_tout, st);
    if (rc != BEM_OK) return rc;
    k_convert<float, double><<<blocks_for(M, 256), 256, 0, st>>>(static_cast<const float*>(p->d_tout), w, M);
    return BEM_OK;
  }
  // z = M^-1 v (or a copy when unpreconditioned)
  void precond(const double* v, double* z) {
    if (p->pc.kind == 0) {
      cudaMemcpyAsync(z, v, M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
      const int m = p->pc.bs * p->ncomp;
      block_apply(p, m, M, v, z, st);
    }
  }
  // out[0..nvec) = V[0..nvec) . w   (device)
  void dots(const double* V, int64_t ldv, int nvec, const double* w, double* out, bool accumulate) {
    dim3 g(nchunk, nvec);
    k_dots_partial<<<g, kDotThreads, 0, st>>>(V, ldv, w, M, nchunk, partial);
    k_dots_final<<<blocks_for(nvec, 64), 64, 0, st>>>(partial, nvec, nchunk, out, accumulate ? 1 : 0);
  }
};

struct GmresWs {
  double* V;
  double* w;
  double* z;
  double* h;
  double* h2;
  double* y;
  int m;
};

struct GmresOut {
  int iters = 0, restarts = 0, applies = 0;
  double rel = 1.0, rel_est = 1.0;
  bem_status status = BEM_ERR_NOT_CONVERGED;
};

// Restarted right-preconditioned GMRES on A x = b with the plan-precision
// apply of g.p; stops when ||b - A x|| <= tol * bnorm (recomputed at every
// restart with the same apply), after max_iter iterations, or when the
// recomputed residual stagnates for three restarts.  x is updated in place.
// x_zero: x is zero on entry, so the first residual is b (no apply).
// trust_estimate: a correction solve inside refinement, whose caller forms
// the residual of the updated x with its own operator next; the solve ends
// when the Arnoldi estimate meets tol (or at max_iter) without recomputing
// the residual with the low-precision apply.
static bem_status gmres_core(Gm& g, const GmresWs& ws, const double* d_b, double bnorm, double* d_x, double tol,
                             int max_iter, GmresOut* out, bool x_zero = false, bool trust_estimate = false) {
  const int64_t M = g.M;
  const int m = ws.m;
  cudaStream_t st = g.st;
  bem_status rc;
  double* V = ws.V;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hbuf(2 * (m + 1) + 1), y(m);
  double best_rel = INFINITY;
  int stagnant = 0;
  out->status = BEM_ERR_NOT_CONVERGED;
  bool first = true;
  while (true) {
    // r = b - A x  -> V[0]
    BEM_CUDA_TRY(cudaMemcpyAsync(V, d_b, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!(first && x_zero)) {
      if ((rc = g.apply(BEM_SYSTEM, d_x, ws.w)) != BEM_OK) return rc;
      ++out->applies;
      k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, ws.w, 1.0, V, M);
    }
    first = false;
    double beta2 = 0.0;
    g.dots(V, M, 1, V, ws.h, false);
    BEM_CUDA_TRY(cudaMemcpyAsync(&beta2, ws.h, sizeof(double), cudaMemcpyDeviceToHost, st));
    BEM_CUDA_TRY(cudaStreamSynchronize(st));
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) {
      set_error("bem_solve: residual is not finite");
      out->status = BEM_ERR_NONFINITE;
      return BEM_OK;
    }
    out->rel = bnorm > 0 ? beta / bnorm : 0.0;
    if (out->rel <= tol) {
      out->status = BEM_OK;
      return BEM_OK;
    }
    if (out->rel < best_rel * 0.999) {
      best_rel = out->rel;
      stagnant = 0;
    } else if (++stagnant >= 3) {
      set_error("bem_solve: residual stagnates (precision floor of the apply reached)");
      return BEM_OK;
    }
    if (out->iters >= max_iter) {
      set_error("bem_solve: max_iter reached");
      return BEM_OK;
    }
    k_normalize<<<blocks_for(M, 256), 256, 0, st>>>(V, ws.h, V, M);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    bool est_done = false;
    for (; j < m && out->iters < max_iter; ++j) {
      double* vj = V + (int64_t)j * M;
      double* vn = V + (int64_t)(j + 1) * M;
      g.precond(vj, ws.z);
      if ((rc = g.apply(BEM_SYSTEM, ws.z, ws.w)) != BEM_OK) return rc;
      ++out->applies;
      ++out->iters;
      // classical Gram-Schmidt with one re-orthogonalisation (FP64)
      g.dots(V, M, j + 1, ws.w, ws.h, false);
      k_sub_basis<<<blocks_for(M, 256), 256, 0, st>>>(V, M, j + 1, ws.h, ws.w, M);
      g.dots(V, M, j + 1, ws.w, ws.h2, false);
      k_sub_basis<<<blocks_for(M, 256), 256, 0, st>>>(V, M, j + 1, ws.h2, ws.w, M);
      g.dots(ws.w, M, 1, ws.w, ws.h + (j + 1), false);
      k_normalize<<<blocks_for(M, 256), 256, 0, st>>>(ws.w, ws.h + (j + 1), vn, M);
      BEM_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), ws.h, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
      BEM_CUDA_TRY(cudaMemcpyAsync(hbuf.data() + (m + 1), ws.h2, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      BEM_CUDA_TRY(cudaStreamSynchronize(st));
      double* col = &H[(size_t)j * (m + 1)];
      for (int i = 0; i <= j; ++i) col[i] = hbuf[i] + hbuf[m + 1 + i];
      col[j + 1] = std::sqrt(hbuf[j + 1]);
      if (!std::isfinite(col[j + 1])) {
        set_error("bem_solve: Arnoldi vector is not finite");
        out->status = BEM_ERR_NONFINITE;
        return BEM_OK;
      }
      for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
      }
      const double a = col[j], b = col[j + 1];
      const double r = std::hypot(a, b);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b / r : 0.0;
      col[j] = r;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      out->rel_est = bnorm > 0 ? std::fabs(gv[j + 1]) / bnorm : 0.0;
      if (out->rel_est <= tol || std::sqrt(hbuf[j + 1]) <= 1e-14 * bnorm) {
        ++j;
        est_done = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular j x j), x += M^-1 (V y)
    for (int i = j - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k = i + 1; k < j; ++k) s -= H[(size_t)k * (m + 1) + i] * y[k];
      y[i] = s / H[(size_t)i * (m + 1) + i];
    }
    if (j > 0) {
      BEM_CUDA_TRY(cudaMemcpyAsync(ws.y, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, st));
      BEM_CUDA_TRY(cudaMemsetAsync(ws.w, 0, M * sizeof(double), st));
      k_add_basis<<<blocks_for(M, 256), 256, 0, st>>>(V, M, j, ws.y, ws.w, M);
      g.precond(ws.w, ws.z);
      k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(1.0, ws.z, 1.0, d_x, M);
    }
    ++out->restarts;
    if (trust_estimate && (est_done || out->iters >= max_iter)) {
      out->rel = out->rel_est;
      if (est_done) out->status = BEM_OK;
      return BEM_OK;
    }
  }
}

bem_status solve_gmres(bem_plan_s* p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                       int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                       cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t M = p->nb * p->ncomp;
  if (restart < 1 || restart > 512 || max_iter < 0 || !(tol > 0.0)) {
    set_error("bem_solve: need 1 <= restart <= 512, max_iter >= 0, tol > 0");
    return BEM_ERR_ARG;
  }
  bem_status rc = bem_set_bc(p, bc, c);
  if (rc != BEM_OK) return rc;
  bem_plan_s* R = p->companion ? p->companion : p;  // residual (outer) operator
  if (R != p && (rc = bem_set_bc(R, bc, c)) != BEM_OK) return rc;
  const int m = restart;
  // workspace
  if (p->gm_m < m) {
    cudaFree(p->d_V);
    p->d_V = nullptr;
    BEM_CUDA_TRY(cudaMalloc(&p->d_V, (size_t)(m + 1) * M * sizeof(double)));
    p->gm_m = m;
  }
  if ((rc = build_preconditioner(p)) != BEM_OK) return rc;
  if (!p->d_vec) BEM_CUDA_TRY(cudaMalloc(&p->d_vec, (size_t)9 * M * sizeof(double) + (size_t)M));
  const int nchunk = (int)((M + kDotChunk - 1) / kDotChunk);
  const size_t small = (size_t)3 * 520 + (size_t)520 * nchunk + 8;
  if (p->small_len < small) {
    cudaFree(p->d_small);
    p->d_small = nullptr;
    BEM_CUDA_TRY(cudaMalloc(&p->d_small, small * sizeof(double)));
    p->small_len = small;
  }
  for (bem_plan_s* q : {p, R})
    if (!q->d_tin) {
      BEM_CUDA_TRY(cudaMalloc(&q->d_tin, (size_t)M * prec_bytes(q)));
      BEM_CUDA_TRY(cudaMalloc(&q->d_tout, (size_t)M * prec_bytes(q)));
    }
  double* d_b = p->d_vec;
  double* d_x = d_b + M;
  double* d_w = d_x + M;
  double* d_um = d_w + M;
  double* d_qm = d_um + M;
  double* d_data = d_qm + M;
  double* d_z = d_data + M;
  double* d_r = d_z + M;
  double* d_d = d_r + M;
  uint8_t* d_bc = reinterpret_cast<uint8_t*>(d_d + M);
  double* d_h = p->d_small;   // 520: first CGS sweep, then norm^2 at [j+1]
  double* d_h2 = d_h + 520;   // 520: second sweep
  double* d_y = d_h2 + 520;   // 520
  double* d_partial = d_y + 520;
  Gm g{p, st, M, d_partial, nchunk, p->prec != BEM_F32};
  Gm gr{R, st, M, d_partial, nchunk, R->prec != BEM_F32};
  GmresWs ws{p->d_V, d_w, d_z, d_h, d_h2, d_y, m};
  int applies = 0;

  BEM_CUDA_TRY(cudaMemcpyAsync(d_data, data, M * sizeof(double), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(d_bc, bc, M, cudaMemcpyHostToDevice, st));
  k_split_known<<<blocks_for(M, 256), 256, 0, st>>>(d_data, d_bc, d_um, d_qm, M);
  // b = c um - sigma K2 um - K1 qm,  sigma K2 = +D (Laplace) or -T (Kelvin)
  const double sigma = p->kernel == BEM_KELVIN_3D ? -1.0 : 1.0;
  // an apply of an all-zero density (no Dirichlet or no Neumann entries) is
  // skipped; with both kinds an FP64-accurate residual operator gives b in
  // one apply where it has the complementary mask's operator (b = -(A'
  // data)).  An FP32 operator keeps the two layer applies and adds c um in
  // FP64: with b from one FP32 apply, plain FP32 GMRES on the 4096^2 star
  // stalled at 6.2e-6 instead of 2.3e-6.
  int64_t nneu = 0;
  for (int64_t i = 0; i < M; ++i) nneu += bc[i] != 0;
  if (fp64_residual(R) && has_complement(R)) {
    if ((rc = gr.apply_comp(d_data, d_w)) != BEM_OK) return rc;
    ++applies;
    BEM_CUDA_TRY(cudaMemsetAsync(d_b, 0, M * sizeof(double), st));
    k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, d_w, 0.0, d_b, M);
  } else {
    if (nneu < M) {
      if ((rc = gr.apply(BEM_DOUBLE, d_um, d_b)) != BEM_OK) return rc;
      ++applies;
    } else {
      BEM_CUDA_TRY(cudaMemsetAsync(d_b, 0, M * sizeof(double), st));
    }
    if (nneu > 0) {
      if ((rc = gr.apply(BEM_SINGLE, d_qm, d_w)) != BEM_OK) return rc;
      ++applies;
    } else {
      BEM_CUDA_TRY(cudaMemsetAsync(d_w, 0, M * sizeof(double), st));
    }
    k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, d_w, -sigma, d_b, M);  // b = -sigma K2 um - K1 qm
    k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(c, d_um, 1.0, d_b, M);       // b += c um
  }
  if (x0)
    BEM_CUDA_TRY(cudaMemcpyAsync(d_x, x0, M * sizeof(double), cudaMemcpyHostToDevice, st));
  else
    BEM_CUDA_TRY(cudaMemsetAsync(d_x, 0, M * sizeof(double), st));

  double bnorm2 = 0.0;
  g.dots(d_b, M, 1, d_b, d_h, false);
  BEM_CUDA_TRY(cudaMemcpyAsync(&bnorm2, d_h, sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bnorm2);
  if (!std::isfinite(bnorm)) {
    set_error("bem_solve: right-hand side is not finite");
    return BEM_ERR_NONFINITE;
  }

  GmresOut tot;
  int refine_steps = 0;
  bem_status result = BEM_ERR_NOT_CONVERGED;
  double rel = 1.0, rel_est = 1.0;
  if (R == p) {
    if ((rc = gmres_core(g, ws, d_b, bnorm, d_x, tol, max_iter, &tot, x0 == nullptr)) != BEM_OK) return rc;
    result = tot.status;
    rel = tot.rel;
    rel_est = tot.rel_est;
  } else {
    // Mixed-precision iterative refinement: residuals with the FP64 operator,
    // corrections from the preconditioned low-precision GMRES.
    double best = INFINITY;
    int stagnant = 0;
    bool x_zero = x0 == nullptr;  // the first residual of a zero start is b itself
    if (x0) {
      // first step from the initial guess: low-precision GMRES from x0 on A x = b
      GmresOut in;
      if ((rc = gmres_core(g, ws, d_b, bnorm, d_x, inner_tolerance(tol, 1.0), max_iter, &in, false, true)) !=
          BEM_OK)
        return rc;
      tot.iters += in.iters;
      tot.restarts += in.restarts;
      tot.applies += in.applies;
      ++refine_steps;
    }
    for (;;) {
      BEM_CUDA_TRY(cudaMemcpyAsync(d_r, d_b, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
      if (!x_zero) {
        if ((rc = gr.apply(BEM_SYSTEM, d_x, d_w)) != BEM_OK) return rc;
        ++applies;
        k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, d_w, 1.0, d_r, M);
      }
      x_zero = false;
      double r2 = 0.0;
      g.dots(d_r, M, 1, d_r, d_h, false);
      BEM_CUDA_TRY(cudaMemcpyAsync(&r2, d_h, sizeof(double), cudaMemcpyDeviceToHost, st));
      BEM_CUDA_TRY(cudaStreamSynchronize(st));
      const double rn = std::sqrt(r2);
      if (!std::isfinite(rn)) {
        set_error("bem_solve: residual is not finite");
        result = BEM_ERR_NONFINITE;
        break;
      }
      rel = bnorm > 0 ? rn / bnorm : 0.0;
      if (rel <= tol) {
        result = BEM_OK;
        break;
      }
      if (rel < best * 0.5) {
        best = rel;
        stagnant = 0;
      } else if (++stagnant >= 2) {
        set_error("bem_solve: refinement stagnates");
        break;
      }
      if (tot.iters >= max_iter) {
        set_error("bem_solve: max_iter reached");
        break;
      }
      // inner solve A d = r to a modest relative accuracy
      BEM_CUDA_TRY(cudaMemsetAsync(d_d, 0, M * sizeof(double), st));
      GmresOut in;
      if ((rc = gmres_core(g, ws, d_r, rn, d_d, inner_tolerance(tol, rel), max_iter - tot.iters, &in, true, true)) !=
          BEM_OK)
        return rc;
      tot.iters += in.iters;
      tot.restarts += in.restarts;
      tot.applies += in.applies;
      rel_est = in.rel_est * rn / std::max(bnorm, 1e-300);
      k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(1.0, d_d, 1.0, d_x, M);
      ++refine_steps;
    }
  }
  applies += tot.applies;

  // outputs
  std::vector<double> x(M);
  BEM_CUDA_TRY(cudaMemcpyAsync(x.data(), d_x, M * sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < M; ++i) {
    const bool neu = bc[i] != 0;
    if (u_out) u_out[i] = neu ? x[i] : data[i];
    if (q_out) q_out[i] = neu ? data[i] : x[i];
  }
  if (info) {
    info->iters = tot.iters;
    info->restarts = tot.restarts;
    info->rel_residual = rel;
    info->rel_residual_fp64 = fp64_residual(R) ? rel : NAN;
    info->rel_residual_est = rel_est;
    info->applies = applies;
    info->refine_steps = refine_steps;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

}  // namespace bemfft

// ======================================================================
// Batched solve: the boundary-condition systems of every plan of a batch,
// solved together by one GMRES running in lockstep (a common Arnoldi index j
// for all systems).  Each Arnoldi step - preconditioner, the batched apply of
// all operators, two classical Gram-Schmidt sweeps, the norms, the next basis
// vectors and the Givens rotations of every system - is one CUDA graph, with
// j kept on the device, so the host replays the same graph every step and
// reads back one integer (the number of systems still iterating).  Vectors are
// packed like the batch buffers (system s at offset[s]); every reduction runs
// per system in a fixed order.

struct BatchSolveWs {
  int K = 0, m = 0;
  int64_t Mt = 0;
  double *V = nullptr, *vin = nullptr, *zz = nullptr, *w = nullptr, *x = nullptr, *b = nullptr, *r = nullptr,
         *d = nullptr, *e = nullptr, *rhs = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *nrm = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
         *y = nullptr, *bnorm = nullptr, *tolv = nullptr, *relest = nullptr;
  int *jdev = nullptr, *jstop = nullptr, *active = nullptr;
  int64_t* off = nullptr;
  int32_t* sys = nullptr;
  int* h_active = nullptr;  // pinned
  int C = 1;                 // chunks per system segment of the dot products
  double* dpart = nullptr;   // K * (m + 1) * C partial dot products (C > 1)
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> segoff;        // host copy of the system offsets (K + 1)
  std::vector<uint64_t> versions;     // plan operator versions the graph was captured with
  std::vector<uint64_t> pc_versions;  // and their preconditioner versions
  std::vector<void*> allocs;
};

namespace bemfft {

void batch_solve_free(bem_batch_s* bt) {
  BatchSolveWs* W = bt->ws;
  if (!W) return;
  if (W->exec) cudaGraphExecDestroy(W->exec);
  if (W->graph) cudaGraphDestroy(W->graph);
  for (void* a : W->allocs) cudaFree(a);
  if (W->h_active) cudaFreeHost(W->h_active);
  if (W->st) cudaStreamDestroy(W->st);
  delete W;
  bt->ws = nullptr;
}

// dst = V[*j]
__global__ void k_b_copy_vj(const double* __restrict__ V, int64_t Mt, const int* __restrict__ jdev,
                            double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Mt) dst[i] = V[(int64_t)(*jdev) * Mt + i];
}

// <V_k, w> over chunk c of the segment of system s, for k < nvec (nvec =
// *jdev + 1, or nfix when jdev is null); one block per (k, s, c), the segment
// cut into gridDim.z equal chunks.  With one chunk the result goes to
// out[s*ldo + k], else to part[(s*ldo + k)*C + c] for k_b_dots_final.
__global__ void k_b_dots(const double* __restrict__ V, int64_t ldv, const int* __restrict__ jdev, int nfix,
                         const double* __restrict__ w, const int64_t* __restrict__ off, double* __restrict__ out,
                         int ldo, double* __restrict__ part) {
  __shared__ double red[kDotThreads / 32];
  const int k = blockIdx.x, s = blockIdx.y, c = blockIdx.z, C = gridDim.z;
  const int nvec = jdev ? *jdev + 1 : nfix;
  if (k >= nvec) return;
  const double* a = V + (int64_t)k * ldv;
  const int64_t a0 = off[s], len = off[s + 1] - a0;
  const int64_t i0 = a0 + len * c / C, i1 = a0 + len * (c + 1) / C;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kDotThreads) acc += a[i] * w[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) {
      if (C == 1) out[(int64_t)s * ldo + k] = acc;
      else part[((int64_t)s * ldo + k) * C + c] = acc;
    }
  }
}

// out[s*ldo + k] = sum over the C chunks in order, for k < nvec
__global__ void k_b_dots_final(const int* __restrict__ jdev, int nfix, int K, int C,
                               const double* __restrict__ part, double* __restrict__ out, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // s * ldo + k
  if (i >= K * ldo) return;
  const int k = i % ldo;
  const int nvec = jdev ? *jdev + 1 : nfix;
  if (k >= nvec) return;
  double acc = 0.0;
  for (int c = 0; c < C; ++c) acc += part[(int64_t)i * C + c];
  out[i] = acc;
}

// w[i] -= sum_{k <= *j} V[k][i] h[sys(i)][k]
__global__ void k_b_sub(const double* __restrict__ V, int64_t ldv, const int* __restrict__ jdev,
                        const int32_t* __restrict__ sys, const double* __restrict__ h, int ldh,
                        double* __restrict__ w, int64_t Mt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mt) return;
  const int nvec = *jdev + 1;
  const double* hs = h + (int64_t)sys[i] * ldh;
  double acc = w[i];
  for (int k = 0; k < nvec; ++k) acc -= V[(int64_t)k * ldv + i] * hs[k];
  w[i] = acc;
}

// V[*j + 1] = w / |w|_sys (zero when the norm is zero or not finite)
__global__ void k_b_next(const double* __restrict__ w, const double* __restrict__ nrm2,
                         const int32_t* __restrict__ sys, double* __restrict__ V, int64_t ldv,
                         const int* __restrict__ jdev, int m, int64_t Mt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mt) return;
  const int j = *jdev;
  if (j >= m) return;
  const double s = sqrt(nrm2[sys[i]]);
  V[(int64_t)(j + 1) * ldv + i] = (s > 0.0 && isfinite(s)) ? w[i] / s : 0.0;
}

// Per system (one warp each, WPB systems side by side, more in turn): the new
// Hessenberg column from the two Gram-Schmidt sweeps and the norm, the earlier
// rotations, a new rotation, the residual estimate and the stop test; then j
// advances.  The warp stages the column and the rotations in shared memory
// (all loads in flight), lane 0 runs the rotations there, the warp writes the
// rotated column back.  One block; dynamic shared memory WPB * (3m + 1) doubles.
__global__ void k_b_givens(int K, int m, int* __restrict__ jdev, const double* __restrict__ h1,
                           const double* __restrict__ h2, int ldh, const double* __restrict__ nrm2,
                           double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                           double* __restrict__ g, const double* __restrict__ bnorm, const double* __restrict__ tolv,
                           int* __restrict__ jstop, double* __restrict__ relest, int* __restrict__ active) {
  extern __shared__ double gsm[];
  __shared__ int n_live;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, WPB = blockDim.x >> 5;
  const int j = *jdev;
  if (threadIdx.x == 0) n_live = 0;
  __syncthreads();
  double* hb = gsm + (size_t)wp * (3 * m + 1);  // j + 1 column entries, then the rotated ones
  double* cc = hb + (m + 1);
  double* ss = cc + m;
  int live = 0;
  for (int s = wp; s < K; s += WPB) {
    if (!(j < m && jstop[s] < 0)) continue;  // warp-uniform
    double* col = H + ((int64_t)s * m + j) * (m + 1);
    double* c = cs + (int64_t)s * m;
    double* sv = sn + (int64_t)s * m;
    const double* h1s = h1 + (int64_t)s * ldh;
    const double* h2s = h2 + (int64_t)s * ldh;
    for (int i = lane; i <= j; i += 32) hb[i] = h1s[i] + h2s[i];
    for (int i = lane; i < j; i += 32) {
      cc[i] = c[i];
      ss[i] = sv[i];
    }
    __syncwarp();
    if (lane == 0) {
      // the earlier rotations down the new column: entry i + 1 enters rotation
      // i unrotated, entry i leaves it final
      double* gv = g + (int64_t)s * (m + 1);
      const double hn = sqrt(nrm2[s]);
      double run = hb[0];
      for (int i = 0; i < j; ++i) {
        const double bb = hb[i + 1];
        hb[i] = cc[i] * run + ss[i] * bb;
        run = -ss[i] * run + cc[i] * bb;
      }
      const double a = run, bb = hn;
      const double r = hypot(a, bb);
      c[j] = r > 0 ? a / r : 1.0;
      sv[j] = r > 0 ? bb / r : 0.0;
      col[j] = r;
      col[j + 1] = 0.0;
      gv[j + 1] = -sv[j] * gv[j];
      gv[j] = c[j] * gv[j];
      const double rel = bnorm[s] > 0 ? fabs(gv[j + 1]) / bnorm[s] : 0.0;
      relest[s] = rel;
      if (!(rel > tolv[s]) || !(hn > 1e-14 * bnorm[s]) || j + 1 == m) jstop[s] = j + 1;
      else ++live;
    }
    __syncwarp();
    for (int i = lane; i < j; i += 32) col[i] = hb[i];
    __syncwarp();  // the warp's staging buffers are free for its next system
  }
  if (live) atomicAdd(&n_live, live);
  __syncthreads();
  if (threadIdx.x == 0) {
    *active = n_live;
    if (j < m) *jdev = j + 1;
  }
}

// launch shape of k_b_givens: systems side by side (warps) and the dynamic
// shared memory they stage in
static void givens_shape(int K, int m, int* warps, size_t* smem) {
  const size_t per = (size_t)(3 * m + 1) * sizeof(double);
  int wpb = std::min(K, 32);
  while (wpb > 1 && (size_t)wpb * per > (size_t)200 * 1024) wpb >>= 1;
  *warps = std::max(1, wpb);
  *smem = (size_t)*warps * per;
}

// y_s = H_s^{-1} g_s over the system's own number of columns
__global__ void k_b_backsolve(int K, int m, const int* __restrict__ jdev, const int* __restrict__ jstop,
                              const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= K) return;
  const int nj = jstop[s] >= 0 ? jstop[s] : *jdev;
  const double* Hs = H + (int64_t)s * m * (m + 1);
  double* ys = y + (int64_t)s * m;
  for (int i = nj - 1; i >= 0; --i) {
    double acc = g[(int64_t)s * (m + 1) + i];
    for (int k = i + 1; k < nj; ++k) acc -= Hs[(int64_t)k * (m + 1) + i] * ys[k];
    const double dia = Hs[(int64_t)i * (m + 1) + i];
    ys[i] = dia != 0.0 ? acc / dia : 0.0;
  }
}

// out[i] = sum_{k < ncols(sys)} V[k][i] y[sys][k]
__global__ void k_b_combine(const double* __restrict__ V, int64_t ldv, const int* __restrict__ jdev,
                            const int* __restrict__ jstop, const int32_t* __restrict__ sys,
                            const double* __restrict__ y, int m, double* __restrict__ out, int64_t Mt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mt) return;
  const int s = sys[i];
  const int nj = jstop[s] >= 0 ? jstop[s] : *jdev;
  double acc = 0.0;
  for (int k = 0; k < nj; ++k) acc += V[(int64_t)k * ldv + i] * y[(int64_t)s * m + k];
  out[i] = acc;
}

// V0 = (rhs - w) / beta_sys, zero for systems that need no iteration
__global__ void k_b_start(const double* __restrict__ rhs, const double* __restrict__ w,
                          const double* __restrict__ beta2, const int* __restrict__ jstop,
                          const int32_t* __restrict__ sys, double* __restrict__ V0, int64_t Mt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mt) return;
  const int s = sys[i];
  const double bt = sqrt(beta2[s]);
  V0[i] = (jstop[s] < 0 && bt > 0.0) ? (rhs[i] - w[i]) / bt : 0.0;
}

namespace {

template <typename T>
bem_status dalloc(BatchSolveWs& W, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    set_error("bem_batch_solve: out of device memory");
    return BEM_ERR_OOM;
  }
  W.allocs.push_back(q);
  *p = static_cast<T*>(q);
  return BEM_OK;
}

// z = M^-1 v on every system's segment (the plans' own preconditioners)
void batch_precond(bem_batch_s* bt, const double* v, double* z, cudaStream_t st) {
  for (size_t i = 0; i < bt->plans.size(); ++i) {
    bem_plan_s* p = bt->plans[i];
    const int64_t o = (int64_t)bt->offset[i], M = (int64_t)(bt->offset[i + 1] - bt->offset[i]);
    if (p->pc.kind == 0) {
      cudaMemcpyAsync(z + o, v + o, M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
      const int mb = p->pc.bs * p->ncomp;
      block_apply(p, mb, M, v + o, z + o, st);
    }
  }
}

// w = A v for all systems with the batch's operators (FP64 vectors)
bem_status batch_apply_f64(bem_batch_s* bt, const double* v, double* w, cudaStream_t st, bool replay) {
  const int64_t Mt = (int64_t)bt->total;
  if (bt->prec == BEM_F32)
    k_convert<double, float><<<blocks_for(Mt, 256), 256, 0, st>>>(v, static_cast<float*>(bt->d_in), Mt);
  else
    BEM_CUDA_TRY(cudaMemcpyAsync(bt->d_in, v, Mt * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (replay) {
    BEM_CUDA_TRY(cudaGraphLaunch(bt->exec, st));
  } else {
    bem_status rc = batch_issue_applies(bt, bt->d_in, bt->d_out, st);
    if (rc != BEM_OK) return rc;
  }
  if (bt->prec == BEM_F32)
    k_convert<float, double><<<blocks_for(Mt, 256), 256, 0, st>>>(static_cast<const float*>(bt->d_out), w, Mt);
  else
    BEM_CUDA_TRY(cudaMemcpyAsync(w, bt->d_out, Mt * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return BEM_OK;
}

// out[s*ldo + k] = <V_k, w>_s for k < nvec (gx >= nvec blocks per system),
// each segment in W.C chunks summed in a fixed order
void b_dots(const BatchSolveWs& W, const double* V, int64_t ldv, const int* jdev, int nfix, const double* w,
            double* out, int ldo, int gx, cudaStream_t st) {
  k_b_dots<<<dim3(gx, W.K, W.C), kDotThreads, 0, st>>>(V, ldv, jdev, nfix, w, W.off, out, ldo, W.dpart);
  if (W.C > 1)
    k_b_dots_final<<<blocks_for((int64_t)W.K * ldo, 128), 128, 0, st>>>(jdev, nfix, W.K, W.C, W.dpart, out, ldo);
}

// per-system squared norms of v into W.nrm (device) and `out` (host)
bem_status seg_norms(BatchSolveWs& W, const double* v, std::vector<double>& out) {
  cudaStream_t st = W.st;
  b_dots(W, v, W.Mt, nullptr, 1, v, W.nrm, 1, 1, st);
  out.resize(W.K);
  BEM_CUDA_TRY(cudaMemcpyAsync(out.data(), W.nrm, W.K * sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  return BEM_OK;
}

// The Arnoldi step graph: vin = V[j]; zz = M^-1 vin; w = A zz; CGS2; norms;
// V[j+1]; Givens; active count to the host.
bem_status capture_arnoldi(bem_batch_s* bt, BatchSolveWs& W) {
  if (W.exec) cudaGraphExecDestroy(W.exec);
  if (W.graph) cudaGraphDestroy(W.graph);
  W.exec = nullptr;
  W.graph = nullptr;
  const int64_t Mt = W.Mt;
  const int K = W.K, m = W.m, ldh = m + 1;
  cudaStream_t cs = W.st;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error("bem_batch_solve: stream capture failed to begin");
    return BEM_ERR_CUDA;
  }
  k_b_copy_vj<<<blocks_for(Mt, 256), 256, 0, cs>>>(W.V, Mt, W.jdev, W.vin);
  batch_precond(bt, W.vin, W.zz, cs);
  bem_status rc = batch_apply_f64(bt, W.zz, W.w, cs, false);
  if (rc == BEM_OK) {
    b_dots(W, W.V, Mt, W.jdev, 0, W.w, W.h1, ldh, m + 1, cs);
    k_b_sub<<<blocks_for(Mt, 256), 256, 0, cs>>>(W.V, Mt, W.jdev, W.sys, W.h1, ldh, W.w, Mt);
    b_dots(W, W.V, Mt, W.jdev, 0, W.w, W.h2, ldh, m + 1, cs);
    k_b_sub<<<blocks_for(Mt, 256), 256, 0, cs>>>(W.V, Mt, W.jdev, W.sys, W.h2, ldh, W.w, Mt);
    b_dots(W, W.w, Mt, nullptr, 1, W.w, W.nrm, 1, 1, cs);
    k_b_next<<<blocks_for(Mt, 256), 256, 0, cs>>>(W.w, W.nrm, W.sys, W.V, Mt, W.jdev, m, Mt);
    int gw = 1;
    size_t gsmem = 0;
    givens_shape(K, m, &gw, &gsmem);
    if (gsmem > 48 * 1024) cudaFuncSetAttribute(k_b_givens, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
    k_b_givens<<<1, 32 * gw, gsmem, cs>>>(K, m, W.jdev, W.h1, W.h2, ldh, W.nrm, W.H, W.cs, W.sn, W.g,
                                                   W.bnorm, W.tolv, W.jstop, W.relest, W.active);
    cudaMemcpyAsync(W.h_active, W.active, sizeof(int), cudaMemcpyDeviceToHost, cs);
  }
  cudaGraph_t gph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &gph);
  if (rc != BEM_OK) {
    if (gph) cudaGraphDestroy(gph);
    return rc;
  }
  if (e != cudaSuccess || !gph) {
    set_error(std::string("bem_batch_solve: capture failed: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  W.graph = gph;
  if (cudaGraphInstantiate(&W.exec, gph, 0) != cudaSuccess) {
    set_error("bem_batch_solve: graph instantiation failed");
    return BEM_ERR_CUDA;
  }
  W.versions.clear();
  W.pc_versions.clear();
  for (auto* p : bt->plans) {
    W.versions.push_back(p->op_version);
    W.pc_versions.push_back(p->pc_version);
  }
  return BEM_OK;
}

struct BatchCounters {
  int iters = 0, restarts = 0, applies = 0;
};

// Lockstep GMRES(m) on A x = rhs (per system: stop when |rhs - A x| <=
// tol_s * rn_s, recomputed with A at every restart).  x is updated in place;
// rel[s] holds the last recomputed relative residual.  x_zero and
// trust_estimate as in gmres_core: a zero start takes rhs as its first
// residual, and a correction solve inside refinement ends on the Arnoldi
// estimates (every system stopped, or max_iter) without a closing apply.
bem_status batch_gmres(bem_batch_s* bt, BatchSolveWs& W, const double* rhs, const std::vector<double>& rn,
                       double* x, const std::vector<double>& tols, int max_iter, BatchCounters* cnt,
                       std::vector<double>& rel, bool x_zero = false, bool trust_estimate = false) {
  const int K = W.K, m = W.m;
  const int64_t Mt = W.Mt;
  cudaStream_t st = W.st;
  BEM_CUDA_TRY(cudaMemcpyAsync(W.bnorm, rn.data(), K * sizeof(double), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(W.tolv, tols.data(), K * sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<double> beta2;
  std::vector<int> jstop(K);
  std::vector<double> g0((size_t)K * (m + 1), 0.0);
  std::vector<double> best(K, INFINITY);
  std::vector<int> stagnant(K, 0);
  rel.assign(K, 1.0);
  const int iters0 = cnt->iters;
  bool first = true;
  for (;;) {
    bem_status rc;
    // r = rhs - A x, per-system norms
    BEM_CUDA_TRY(cudaMemcpyAsync(W.r, rhs, Mt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (!(first && x_zero)) {
      if ((rc = batch_apply_f64(bt, x, W.w, st, true)) != BEM_OK) return rc;
      ++cnt->applies;
      k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(-1.0, W.w, 1.0, W.r, Mt);
    }
    if ((rc = seg_norms(W, W.r, beta2)) != BEM_OK) return rc;
    if (cnt->iters == iters0 && !(first && x_zero)) {
      // a starting point worse than zero (an initial guess) is replaced by zero
      bool any = false;
      for (int s = 0; s < K; ++s)
        if (!(std::sqrt(beta2[s]) <= rn[s])) {
          const int64_t o = W.segoff[s], len = W.segoff[s + 1] - o;
          BEM_CUDA_TRY(cudaMemsetAsync(x + o, 0, len * sizeof(double), st));
          BEM_CUDA_TRY(cudaMemcpyAsync(W.r + o, rhs + o, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
          any = true;
        }
      // the norms again, on the device too (the Arnoldi start reads them there)
      if (any && (rc = seg_norms(W, W.r, beta2)) != BEM_OK) return rc;
    }
    int live = 0;
    for (int s = 0; s < K; ++s) {
      const double b = std::sqrt(beta2[s]);
      rel[s] = rel_norm(b, rn[s]);
      bool go = std::isfinite(rel[s]) && rel[s] > tols[s];
      if (go) {
        if (rel[s] < best[s] * 0.999) {
          best[s] = rel[s];
          stagnant[s] = 0;
        } else if (++stagnant[s] >= 3) {
          go = false;  // precision floor of the apply
        }
      }
      jstop[s] = go ? -1 : 0;
      g0[(size_t)s * (m + 1)] = b;
      live += go;
    }
    if (live == 0 || cnt->iters >= max_iter) return BEM_OK;
    BEM_CUDA_TRY(cudaMemcpyAsync(W.jstop, jstop.data(), K * sizeof(int), cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaMemcpyAsync(W.g, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    BEM_CUDA_TRY(cudaMemsetAsync(W.jdev, 0, sizeof(int), st));
    // V0 = r / beta (W.r already holds rhs - A x; pass a zero w)
    BEM_CUDA_TRY(cudaMemsetAsync(W.w, 0, Mt * sizeof(double), st));
    k_b_start<<<blocks_for(Mt, 256), 256, 0, st>>>(W.r, W.w, W.nrm, W.jstop, W.sys, W.V, Mt);
    first = false;
    bool stopped = false;
    for (int j = 0; j < m && cnt->iters < max_iter; ++j) {
      BEM_CUDA_TRY(cudaGraphLaunch(W.exec, st));
      BEM_CUDA_TRY(cudaStreamSynchronize(st));
      ++cnt->iters;
      ++cnt->applies;
      if (*W.h_active == 0) {
        stopped = true;
        break;
      }
    }
    k_b_backsolve<<<blocks_for(K, 64), 64, 0, st>>>(K, m, W.jdev, W.jstop, W.H, W.g, W.y);
    k_b_combine<<<blocks_for(Mt, 256), 256, 0, st>>>(W.V, Mt, W.jdev, W.jstop, W.sys, W.y, m, W.d, Mt);
    batch_precond(bt, W.d, W.zz, st);
    k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(1.0, W.zz, 1.0, x, Mt);
    ++cnt->restarts;
    if (trust_estimate && (stopped || cnt->iters >= max_iter)) return BEM_OK;
  }
}

}  // namespace

}  // namespace bemfft

using namespace bemfft;

extern "C" bem_status bem_batch_solve(bem_batch_t bt, const uint8_t* bc, const double* data, double c, double tol,
                                      int max_iter, int restart, const double* x0, double* u_out, double* q_out,
                                      bem_solve_info* info, void* stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!bt || !bc || !data) {
    set_error("bem_batch_solve: null pointer argument");
    return BEM_ERR_ARG;
  }
  if (bt->layer != BEM_SYSTEM) {
    set_error("bem_batch_solve: the batch must apply BEM_SYSTEM");
    return BEM_ERR_ARG;
  }
  if (bem_status dc = check_device(bt->plans[0], "bem_batch_solve"); dc != BEM_OK) return dc;
  if (restart < 1 || restart > 512 || max_iter < 0 || !(tol > 0.0)) {
    set_error("bem_batch_solve: need 1 <= restart <= 512, max_iter >= 0, tol > 0");
    return BEM_ERR_ARG;
  }
  const int K = (int)bt->plans.size();
  if (K > 1024) {
    set_error("bem_batch_solve: at most 1024 systems");
    return BEM_ERR_UNSUPPORTED;
  }
  const bool refine = bt->plans[0]->companion != nullptr;
  for (auto* p : bt->plans)
    if ((p->companion != nullptr) != refine) {
      set_error("bem_batch_solve: either every plan or none has refinement enabled");
      return BEM_ERR_ARG;
    }
  const int64_t Mt = (int64_t)bt->total;
  cudaStream_t ust = static_cast<cudaStream_t>(stream);
  bem_status rc;
  // boundary conditions, preconditioners, graphs
  for (int s = 0; s < K; ++s) {
    bem_plan_s* p = bt->plans[s];
    if ((rc = bem_set_bc(p, bc + bt->offset[s], c)) != BEM_OK) return rc;
    if (refine && (rc = bem_set_bc(p->companion, bc + bt->offset[s], c)) != BEM_OK) return rc;
    if ((rc = build_preconditioner(p)) != BEM_OK) return rc;
  }
  if ((rc = batch_refresh(bt)) != BEM_OK) return rc;
  if (refine) {
    bool fresh = bt->companions == nullptr;
    if (!fresh)
      for (int s = 0; s < K; ++s) fresh = fresh || bt->companions->plans[s] != bt->plans[s]->companion;
    if (fresh) {
      if (bt->companions) bem_batch_destroy(bt->companions);
      bt->companions = nullptr;
      std::vector<bem_plan_t> cp;
      for (auto* p : bt->plans) cp.push_back(p->companion);
      if ((rc = bem_batch_create(&bt->companions, cp.data(), K, BEM_SYSTEM, bt->nstreams, nullptr)) != BEM_OK)
        return rc;
    } else if ((rc = batch_refresh(bt->companions)) != BEM_OK) {
      return rc;
    }
  }
  // workspace
  const int m = restart;
  BatchSolveWs* W = bt->ws;
  if (!W || W->m != m) {
    batch_solve_free(bt);
    W = bt->ws = new BatchSolveWs();
    W->K = K;
    W->m = m;
    W->Mt = Mt;
    if (cudaStreamCreateWithFlags(&W->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&W->h_active, sizeof(int)) != cudaSuccess) {
      set_error("bem_batch_solve: stream or pinned memory creation failed");
      batch_solve_free(bt);
      return BEM_ERR_CUDA;
    }
    bool ok = dalloc(*W, &W->V, (size_t)(m + 1) * Mt) == BEM_OK;
    for (double** v : {&W->vin, &W->zz, &W->w, &W->x, &W->b, &W->r, &W->d, &W->e, &W->rhs})
      ok = ok && dalloc(*W, v, Mt) == BEM_OK;
    ok = ok && dalloc(*W, &W->h1, (size_t)K * (m + 1)) == BEM_OK && dalloc(*W, &W->h2, (size_t)K * (m + 1)) == BEM_OK;
    ok = ok && dalloc(*W, &W->nrm, K) == BEM_OK && dalloc(*W, &W->H, (size_t)K * m * (m + 1)) == BEM_OK;
    ok = ok && dalloc(*W, &W->cs, (size_t)K * m) == BEM_OK && dalloc(*W, &W->sn, (size_t)K * m) == BEM_OK;
    ok = ok && dalloc(*W, &W->g, (size_t)K * (m + 1)) == BEM_OK && dalloc(*W, &W->y, (size_t)K * m) == BEM_OK;
    ok = ok && dalloc(*W, &W->bnorm, K) == BEM_OK && dalloc(*W, &W->tolv, K) == BEM_OK &&
         dalloc(*W, &W->relest, K) == BEM_OK;
    ok = ok && dalloc(*W, &W->jdev, 1) == BEM_OK && dalloc(*W, &W->jstop, K) == BEM_OK &&
         dalloc(*W, &W->active, 1) == BEM_OK;
    ok = ok && dalloc(*W, &W->off, K + 1) == BEM_OK && dalloc(*W, &W->sys, Mt) == BEM_OK;
    // dot-product chunks: about 2048 elements each (32 blocks at most per vector and system)
    int64_t maxseg = 0;
    for (int s = 0; s < K; ++s) maxseg = std::max<int64_t>(maxseg, (int64_t)(bt->offset[s + 1] - bt->offset[s]));
    W->C = (int)std::min<int64_t>(32, std::max<int64_t>(1, maxseg / 2048));
    if (W->C > 1) ok = ok && dalloc(*W, &W->dpart, (size_t)K * (m + 1) * W->C) == BEM_OK;
    if (!ok) {
      batch_solve_free(bt);
      return BEM_ERR_OOM;
    }
    std::vector<int64_t> off(bt->offset.begin(), bt->offset.end());
    W->segoff = off;
    std::vector<int32_t> sys(Mt);
    for (int s = 0; s < K; ++s)
      for (size_t i = bt->offset[s]; i < bt->offset[s + 1]; ++i) sys[i] = s;
    BEM_CUDA_TRY(cudaMemcpy(W->off, off.data(), (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    BEM_CUDA_TRY(cudaMemcpy(W->sys, sys.data(), Mt * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  bool recap = W->exec == nullptr;
  for (int s = 0; s < K && !recap; ++s)
    recap = W->versions[s] != bt->plans[s]->op_version || W->pc_versions[s] != bt->plans[s]->pc_version;
  if (recap && (rc = capture_arnoldi(bt, *W)) != BEM_OK) return rc;
  cudaStream_t st = W->st;
  // the solve runs on its own stream, ordered after the caller's stream
  cudaEvent_t ev;
  BEM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  BEM_CUDA_TRY(cudaEventRecord(ev, ust));
  BEM_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
  cudaEventDestroy(ev);

  // right-hand sides b = c um - sigma K2 um - K1 qm with the residual operators
  std::vector<double> um(Mt), qm(Mt);
  for (int64_t i = 0; i < Mt; ++i) {
    um[i] = bc[i] ? 0.0 : data[i];
    qm[i] = bc[i] ? data[i] : 0.0;
  }
  BEM_CUDA_TRY(cudaMemcpyAsync(W->vin, um.data(), Mt * sizeof(double), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(W->zz, qm.data(), Mt * sizeof(double), cudaMemcpyHostToDevice, st));
  BEM_CUDA_TRY(cudaMemcpyAsync(W->rhs, data, Mt * sizeof(double), cudaMemcpyHostToDevice, st));
  // per plan on the batch's side streams (fork from st, join back); an apply
  // of an all-zero density is skipped, and a plan with both condition types
  // that has the complementary mask's operator forms its part in one apply
  // (w = A' data, with its um zeroed so that the sum below gives -(A' data);
  // FP64-accurate residual operators only, as in bem_solve)
  BEM_CUDA_TRY(cudaMemsetAsync(W->b, 0, Mt * sizeof(double), st));
  BEM_CUDA_TRY(cudaMemsetAsync(W->w, 0, Mt * sizeof(double), st));
  const int S = bt->nstreams;
  BEM_CUDA_TRY(cudaEventRecord(bt->events[0], st));
  for (int k = 1; k < S; ++k) BEM_CUDA_TRY(cudaStreamWaitEvent(bt->side[k], bt->events[0], 0));
  int rhs_applies = 0;
  for (int s = 0; s < K; ++s) {
    bem_plan_s* R = refine ? bt->plans[s]->companion : bt->plans[s];
    const int64_t o = (int64_t)bt->offset[s], M = (int64_t)(bt->offset[s + 1] - bt->offset[s]);
    cudaStream_t ss = s % S == 0 ? st : bt->side[s % S];
    Gm gr{R, ss, M, nullptr, 0, R->prec != BEM_F32};
    if (!R->d_tin) {
      BEM_CUDA_TRY(cudaMalloc(&R->d_tin, (size_t)M * prec_bytes(R)));
      BEM_CUDA_TRY(cudaMalloc(&R->d_tout, (size_t)M * prec_bytes(R)));
    }
    if (fp64_residual(R) && has_complement(R)) {
      if ((rc = gr.apply_comp(W->rhs + o, W->w + o)) != BEM_OK) return rc;
      BEM_CUDA_TRY(cudaMemsetAsync(W->vin + o, 0, M * sizeof(double), ss));
      ++rhs_applies;
      continue;
    }
    int64_t nneu = 0;
    for (int64_t i = 0; i < M; ++i) nneu += bc[o + i] != 0;
    if (nneu < M) {
      if ((rc = gr.apply(BEM_DOUBLE, W->vin + o, W->b + o)) != BEM_OK) return rc;
      ++rhs_applies;
    }
    if (nneu > 0) {
      if ((rc = gr.apply(BEM_SINGLE, W->zz + o, W->w + o)) != BEM_OK) return rc;
      ++rhs_applies;
    }
  }
  for (int k = 1; k < S; ++k) {
    BEM_CUDA_TRY(cudaEventRecord(bt->events[S + k], bt->side[k]));
    BEM_CUDA_TRY(cudaStreamWaitEvent(st, bt->events[S + k], 0));
  }
  const double sigma = bt->plans[0]->kernel == BEM_KELVIN_3D ? -1.0 : 1.0;
  k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(-1.0, W->w, -sigma, W->b, Mt);
  k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(c, W->vin, 1.0, W->b, Mt);
  if (x0)
    BEM_CUDA_TRY(cudaMemcpyAsync(W->x, x0, Mt * sizeof(double), cudaMemcpyHostToDevice, st));
  else
    BEM_CUDA_TRY(cudaMemsetAsync(W->x, 0, Mt * sizeof(double), st));
  std::vector<double> bn2;
  if ((rc = seg_norms(*W, W->b, bn2)) != BEM_OK) return rc;
  std::vector<double> bnorm(K);
  for (int s = 0; s < K; ++s) bnorm[s] = std::sqrt(bn2[s]);

  BatchCounters cnt;
  cnt.applies = rhs_applies;
  std::vector<double> rel(K, 1.0);
  int refine_steps = 0;
  if (!refine) {
    if ((rc = batch_gmres(bt, *W, W->b, bnorm, W->x, std::vector<double>(K, tol), max_iter, &cnt, rel,
                          x0 == nullptr)) != BEM_OK)
      return rc;
  } else {
    // residuals with the companions' operator, corrections from the lockstep
    // low-precision GMRES (per system inner tolerance as in bem_solve)
    bem_batch_s* cb = bt->companions;
    std::vector<double> best(K, INFINITY);
    int stagnant = 0;
    bool x_zero = x0 == nullptr;  // the first residual of a zero start is b itself
    if (x0) {
      // first step from the initial guess: the low-precision GMRES starts at
      // x0 on A x = b itself (its first residual is the low-precision one,
      // accurate far beyond this step's tolerance), so the guess costs no
      // residual with the companion operator
      std::vector<double> first_tol(K, inner_tolerance(tol, 1.0));
      std::vector<double> rin;
      if ((rc = batch_gmres(bt, *W, W->b, bnorm, W->x, first_tol, max_iter, &cnt, rin, false, true)) != BEM_OK)
        return rc;
      ++refine_steps;
    }
    for (;;) {
      BEM_CUDA_TRY(cudaMemcpyAsync(W->r, W->b, Mt * sizeof(double), cudaMemcpyDeviceToDevice, st));
      if (!x_zero) {
        if ((rc = batch_apply_f64(cb, W->x, W->w, st, true)) != BEM_OK) return rc;
        ++cnt.applies;
        k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(-1.0, W->w, 1.0, W->r, Mt);
      }
      x_zero = false;
      std::vector<double> r2;
      if ((rc = seg_norms(*W, W->r, r2)) != BEM_OK) return rc;
      std::vector<double> rn(K), inner_tol(K);
      bool all = true, progress = false;
      for (int s = 0; s < K; ++s) {
        rn[s] = std::sqrt(r2[s]);
        rel[s] = rel_norm(rn[s], bnorm[s]);
        const bool done = !(rel[s] > tol);
        all = all && done;
        if (rel[s] < best[s] * 0.5) progress = true;
        best[s] = std::min(best[s], rel[s]);
        // a converged system gets tolerance 1: its inner GMRES does nothing
        inner_tol[s] = done ? 1.0 : inner_tolerance(tol, rel[s]);
      }
      if (all) break;
      stagnant = progress ? 0 : stagnant + 1;
      if (stagnant >= 2 || cnt.iters >= max_iter) break;
      // inner solve A e = r from zero (its own right-hand side buffer)
      BEM_CUDA_TRY(cudaMemcpyAsync(W->rhs, W->r, Mt * sizeof(double), cudaMemcpyDeviceToDevice, st));
      BEM_CUDA_TRY(cudaMemsetAsync(W->e, 0, Mt * sizeof(double), st));
      std::vector<double> rin;
      if ((rc = batch_gmres(bt, *W, W->rhs, rn, W->e, inner_tol, max_iter, &cnt, rin, true, true)) != BEM_OK)
        return rc;
      k_axpby<<<blocks_for(Mt, 256), 256, 0, st>>>(1.0, W->e, 1.0, W->x, Mt);
      ++refine_steps;
    }
  }
  // outputs
  std::vector<double> x(Mt);
  BEM_CUDA_TRY(cudaMemcpyAsync(x.data(), W->x, Mt * sizeof(double), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < Mt; ++i) {
    const bool neu = bc[i] != 0;
    if (u_out) u_out[i] = neu ? x[i] : data[i];
    if (q_out) q_out[i] = neu ? data[i] : x[i];
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bem_status result = BEM_OK;
  for (int s = 0; s < K; ++s) {
    const bool ok = std::isfinite(rel[s]) && rel[s] <= tol;
    if (!std::isfinite(rel[s])) result = BEM_ERR_NONFINITE;
    else if (!ok && result == BEM_OK) result = BEM_ERR_NOT_CONVERGED;
    if (info) {
      info[s].iters = cnt.iters;
      info[s].restarts = cnt.restarts;
      info[s].rel_residual = rel[s];
      info[s].rel_residual_fp64 = fp64_residual(refine ? bt->plans[s]->companion : bt->plans[s]) ? rel[s] : NAN;
      info[s].rel_residual_est = rel[s];
      info[s].seconds = secs;
      info[s].applies = cnt.applies;
      info[s].refine_steps = refine_steps;
    }
  }
  if (result == BEM_ERR_NOT_CONVERGED) set_error("bem_batch_solve: some systems did not reach tol");
  if (result == BEM_ERR_NONFINITE) set_error("bem_solve: non-finite data or residual");
  return result;
}

namespace bemfft {

bem_status solve_graph(bem_plan_s* p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                       int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                       cudaStream_t st) {
  if (restart < 1 || restart > 512 || max_iter < 0 || !(tol > 0.0)) {
    set_error("bem_solve: need 1 <= restart <= 512, max_iter >= 0, tol > 0");
    return BEM_ERR_ARG;
  }
  bem_status rc = bem_set_bc(p, bc, c);
  if (rc != BEM_OK) return rc;
  // the batch switches its plans' kernel timing off (no event records inside
  // captured graphs); the caller's setting comes back after the solve
  const bool timing = p->timing;
  if (!p->self_batch) {
    bem_plan_t one = p;
    rc = bem_batch_create(&p->self_batch, &one, 1, BEM_SYSTEM, 1, st);
    if (rc != BEM_OK) {
      p->self_batch = nullptr;
      p->timing = timing;
      return rc;
    }
  }
  p->timing = false;
  rc = bem_batch_solve(p->self_batch, bc, data, c, tol, max_iter, restart, x0, u_out, q_out, info, st);
  p->timing = timing;
  return rc;
}

}  // namespace bemfft
