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

// out[b*bs + i] = sum_j inv_b[i][j] in[b*bs + j]   (block-Jacobi M^-1)
__global__ void k_block_apply(const double* __restrict__ inv, int bs, int64_t M, const double* __restrict__ in,
                              double* __restrict__ out) {
  extern __shared__ double xin[];
  const int b = blockIdx.x, i = threadIdx.x;
  const int64_t i0 = (int64_t)b * bs;
  const int sz = (int)(M - i0 < bs ? M - i0 : bs);
  if (i < sz) xin[i] = in[i0 + i];
  __syncthreads();
  if (i >= sz) return;
  const double* row = inv + ((size_t)b * bs + i) * bs;
  double s = 0.0;
  for (int j = 0; j < sz; ++j) s += row[j] * xin[j];
  out[i0 + i] = s;
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
  // z = M^-1 v (or a copy when unpreconditioned)
  void precond(const double* v, double* z) {
    if (p->pc.kind == 0) {
      cudaMemcpyAsync(z, v, M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
      const int m = p->pc.bs * p->ncomp;
      k_block_apply<<<p->pc.nblocks, m, m * sizeof(double), st>>>(p->pc.d_inv, m, M, v, z);
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
static bem_status gmres_core(Gm& g, const GmresWs& ws, const double* d_b, double bnorm, double* d_x, double tol,
                             int max_iter, GmresOut* out) {
  const int64_t M = g.M;
  const int m = ws.m;
  cudaStream_t st = g.st;
  bem_status rc;
  double* V = ws.V;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hbuf(2 * (m + 1) + 1), y(m);
  double best_rel = INFINITY;
  int stagnant = 0;
  out->status = BEM_ERR_NOT_CONVERGED;
  while (true) {
    // r = b - A x  -> V[0]
    if ((rc = g.apply(BEM_SYSTEM, d_x, ws.w)) != BEM_OK) return rc;
    ++out->applies;
    BEM_CUDA_TRY(cudaMemcpyAsync(V, d_b, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, ws.w, 1.0, V, M);
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
  if ((rc = gr.apply(BEM_DOUBLE, d_um, d_b)) != BEM_OK) return rc;
  if ((rc = gr.apply(BEM_SINGLE, d_qm, d_w)) != BEM_OK) return rc;
  applies += 2;
  k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, d_w, -sigma, d_b, M);  // b = -sigma K2 um - K1 qm
  k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(c, d_um, 1.0, d_b, M);       // b += c um
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
    if ((rc = gmres_core(g, ws, d_b, bnorm, d_x, tol, max_iter, &tot)) != BEM_OK) return rc;
    result = tot.status;
    rel = tot.rel;
    rel_est = tot.rel_est;
  } else {
    // Mixed-precision iterative refinement: residuals with the FP64 operator,
    // corrections from the preconditioned low-precision GMRES.
    double best = INFINITY;
    int stagnant = 0;
    for (;;) {
      if ((rc = gr.apply(BEM_SYSTEM, d_x, d_w)) != BEM_OK) return rc;
      ++applies;
      BEM_CUDA_TRY(cudaMemcpyAsync(d_r, d_b, M * sizeof(double), cudaMemcpyDeviceToDevice, st));
      k_axpby<<<blocks_for(M, 256), 256, 0, st>>>(-1.0, d_w, 1.0, d_r, M);
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
      const double eta = std::max(1e-4, 0.1 * tol / std::max(rel, 1e-300));
      if ((rc = gmres_core(g, ws, d_r, rn, d_d, std::min(eta, 1e-2), max_iter - tot.iters, &in)) != BEM_OK)
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
    info->rel_residual_est = rel_est;
    info->applies = applies;
    info->refine_steps = refine_steps;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

}  // namespace bemfft
