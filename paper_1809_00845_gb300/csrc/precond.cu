// Block-Jacobi near-field preconditioner for bem_solve.
//
// The single layer of Eq. 15 is a first-kind operator: its eigenvalues decay
// like 1/k for oscillation k along the boundary, so restarted GMRES on the
// BC-split system stalls as n grows.  The oscillatory part of the operator is
// local (it comes from the near-singular kernel values between neighbouring
// cells), so inverting the operator restricted to blocks of neighbouring
// cells and using those inverses as a right preconditioner removes most of
// that ill-conditioning.  Blocks are runs of consecutive cells in the
// caller's order.  Entries are the same kernel point values (and singular-cell
// average) as the FFT tables.  2D blocks of up to 512 unknowns are assembled
// and inverted on the device, one CTA per block (Gauss-Jordan with partial
// pivoting in FP32: the preconditioner only has to be a fixed nonsingular
// approximation of the block inverse); other blocks are assembled and
// inverted in FP64 on the host.
#include <cmath>
#include <vector>

#include "bem_internal.h"

namespace bemfft {

// 2D kernel value at grid offset (dx, dy): kind 0 = U, 1 = Q_x, 2 = Q_y,
// same definition as the FFT tables (Eq. 3, Eq. 15; singular cell = cell
// average for U, 0 for the odd kernels).
__host__ __device__ double kernel2d_point(int kind, int dx, int dy, double h) {
  const double PI = 3.14159265358979323846;
  if (dx == 0 && dy == 0) {
    if (kind != 0) return 0.0;
    const double L2 = PI / 4.0 - 1.5 - 0.5 * ::log(2.0);
    return -(::log(h) + L2) / (2.0 * PI);
  }
  const double r2 = (double)dx * dx + (double)dy * dy;
  if (kind == 0) return -(0.5 * ::log(r2) + ::log(h)) / (2.0 * PI);
  const double da = kind == 1 ? (double)dx : (double)dy;
  return -da / (2.0 * PI * h * r2);
}

// 3D kernels at grid offset delta (d = delta h), same definitions as the FFT
// tables: U3 = 1/(4 pi r), Q3_a = -d_a/(4 pi r^3), Kelvin U_ab (Eq. 7) and the
// traction block T_ab(d; n) = sum_c G_abc(d) n_c (Eq. 8); singular cell as in
// the tables.
static void kernel3d_block(int kernel, const int* dl, const double* nrm, double h, double nu, double mu,
                           bool single, double* out) {
  const double PI = 3.14159265358979323846;
  const double C3 = 3.0 * std::log(2.0 + std::sqrt(3.0)) - PI / 2.0;
  const bool zero = dl[0] == 0 && dl[1] == 0 && dl[2] == 0;
  const double d[3] = {dl[0] * h, dl[1] * h, dl[2] * h};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double r = std::sqrt(r2), r3 = r2 * r;
  if (kernel == BEM_LAPLACE_3D) {
    if (single) {
      out[0] = zero ? C3 / (4.0 * PI * h) : 1.0 / (4.0 * PI * r);
    } else {
      out[0] = 0.0;
      if (!zero)
        for (int a = 0; a < 3; ++a) out[0] += -d[a] / (4.0 * PI * r3) * nrm[a];
    }
    return;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      if (single) {
        if (zero)
          v = a == b ? (3.0 - 4.0 * nu + 1.0 / 3.0) * C3 / (16.0 * PI * mu * (1.0 - nu) * h) : 0.0;
        else
          v = (((a == b) ? (3.0 - 4.0 * nu) / r : 0.0) + d[a] * d[b] / r3) / (16.0 * PI * mu * (1.0 - nu));
      } else if (!zero) {
        for (int c = 0; c < 3; ++c) {
          const double lin = (a == b ? d[c] : 0.0) + (a == c ? d[b] : 0.0) - (b == c ? d[a] : 0.0);
          const double g = ((1.0 - 2.0 * nu) * lin / r3 + 3.0 * d[a] * d[b] * d[c] / (r3 * r2)) / (8.0 * PI * (1.0 - nu));
          v += g * nrm[c];
        }
      }
      out[a * 3 + b] = v;
    }
}

// Gauss-Jordan inversion with partial pivoting (row-major m x m, in place).
static bool invert(std::vector<double>& A, int m) {
  std::vector<double> I((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + c]) > std::fabs(A[(size_t)piv * m + c])) piv = r;
    const double pv = A[(size_t)piv * m + c];
    if (!(std::fabs(pv) > 0.0) || !std::isfinite(pv)) return false;
    if (piv != c)
      for (int k = 0; k < m; ++k) {
        std::swap(A[(size_t)piv * m + k], A[(size_t)c * m + k]);
        std::swap(I[(size_t)piv * m + k], I[(size_t)c * m + k]);
      }
    const double inv = 1.0 / A[(size_t)c * m + c];
    for (int k = 0; k < m; ++k) {
      A[(size_t)c * m + k] *= inv;
      I[(size_t)c * m + k] *= inv;
    }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * m + c];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) {
        A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
        I[(size_t)r * m + k] -= f * I[(size_t)c * m + k];
      }
    }
  }
  A.swap(I);
  return true;
}

constexpr int kPcSmemMax = 128;  // largest block inverted in shared memory
constexpr int kPcGpuMax = 512;   // largest block inverted on the device (in global scratch beyond 128)
constexpr int kPcThreads = 256;

// One CTA per block of bs consecutive caller-order cells (2D Laplace): the
// block of the BC-split operator (U for Dirichlet columns, Q.n for Neumann
// columns minus c on their diagonal), Gauss-Jordan with partial pivoting in
// shared memory (blocks up to 128 cells) or in an L2-resident global scratch
// (up to 512), inverse written as FP64 (padded to m x m).  A block whose pivot
// vanishes gets the identity.
template <bool GLOBAL, int NT = GLOBAL ? 1024 : kPcThreads>
__global__ void __launch_bounds__(NT) k_pc_build2d(int64_t nb, int bs, double h, double c,
                                                          const int32_t* __restrict__ cell,
                                                          const double* __restrict__ w,
                                                          const double* __restrict__ nrm,
                                                          const uint8_t* __restrict__ bc, double* __restrict__ inv,
                                                          float* __restrict__ scratch) {
  extern __shared__ float pcs[];
  __shared__ int s_piv;
  __shared__ int s_bad;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int64_t i0 = (int64_t)b * bs;
  const int sz = (int)(nb - i0 < bs ? nb - i0 : bs);
  // working matrices: shared memory, or this block's slice of a global
  // scratch (L2-resident) for blocks too large for shared memory
  float* A = GLOBAL ? scratch + (size_t)b * (2 * (size_t)bs * bs + bs) : pcs;
  float* I = A + sz * sz;
  float* fac = I + sz * sz;
  for (int e = tid; e < sz * sz; e += NT) {
    const int ia = e / sz, jb = e - ia * sz;
    const int64_t i = i0 + ia, j = i0 + jb;
    const int dx = cell[2 * i] - cell[2 * j], dy = cell[2 * i + 1] - cell[2 * j + 1];
    double v;
    if (!bc[j]) {
      v = kernel2d_point(0, dx, dy, h) * w[j];
    } else {
      v = (kernel2d_point(1, dx, dy, h) * nrm[2 * j] + kernel2d_point(2, dx, dy, h) * nrm[2 * j + 1]) * w[j];
      if (i == j) v -= c;
    }
    A[e] = (float)v;
    I[e] = ia == jb ? 1.0f : 0.0f;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int col = 0; col < sz; ++col) {
    if (tid < 32) {
      float best = -1.0f;
      int bi = col;
      for (int r = col + tid; r < sz; r += 32) {
        const float a = fabsf(A[r * sz + col]);
        if (a > best) {
          best = a;
          bi = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        if (!(best > 0.0f) || !isfinite(best)) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int piv = s_piv;
    if (piv != col)
      for (int k = tid; k < sz; k += NT) {
        float t = A[piv * sz + k];
        A[piv * sz + k] = A[col * sz + k];
        A[col * sz + k] = t;
        t = I[piv * sz + k];
        I[piv * sz + k] = I[col * sz + k];
        I[col * sz + k] = t;
      }
    __syncthreads();
    const float pinv = 1.0f / A[col * sz + col];
    for (int r = tid; r < sz; r += NT) fac[r] = r == col ? 0.0f : A[r * sz + col];
    __syncthreads();
    for (int k = tid; k < sz; k += NT) {
      A[col * sz + k] *= pinv;
      I[col * sz + k] *= pinv;
    }
    __syncthreads();
    for (int e = tid; e < sz * sz; e += NT) {
      const int r = e / sz, k = e - r * sz;
      const float f = fac[r];
      if (f != 0.0f) {
        A[e] -= f * A[col * sz + k];
        I[e] -= f * I[col * sz + k];
      }
    }
    __syncthreads();
  }
  const int m = bs;
  double* dst = inv + (size_t)b * m * m;
  for (int e = tid; e < m * m; e += NT) {
    const int a = e / m, k = e - a * m;
    double v = 0.0;
    if (a < sz && k < sz) v = s_bad ? (a == k ? 1.0 : 0.0) : (double)I[a * sz + k];
    dst[e] = v;
  }
}

static bem_status build_preconditioner_gpu2d(bem_plan_s* p) {
  const int64_t nb = p->nb;
  const int bs = p->pc.bs;
  const int nblocks = (int)((nb + bs - 1) / bs);
  int32_t* d_cell = nullptr;
  double *d_w = nullptr, *d_n = nullptr;
  uint8_t* d_bc = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_cell);
    cudaFree(d_w);
    cudaFree(d_n);
    cudaFree(d_bc);
  };
  if (cudaMalloc(&d_cell, nb * 2 * sizeof(int32_t)) != cudaSuccess || cudaMalloc(&d_w, nb * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_n, nb * 2 * sizeof(double)) != cudaSuccess || cudaMalloc(&d_bc, nb) != cudaSuccess) {
    cleanup();
    set_error("preconditioner: out of device memory");
    return BEM_ERR_OOM;
  }
  cudaFree(p->pc.d_inv);
  p->pc.d_inv = nullptr;
  const size_t per = ((size_t)2 * bs * bs + bs) * sizeof(float);
  const bool global = bs > kPcSmemMax;
  float* d_scr = nullptr;
  cudaError_t e = cudaMalloc(&p->pc.d_inv, (size_t)nblocks * bs * bs * sizeof(double));
  if (e == cudaSuccess && global) e = cudaMalloc(&d_scr, (size_t)nblocks * per);
  if (e == cudaSuccess) e = cudaMemcpy(d_cell, p->h_cell_user.data(), nb * 2 * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_w, p->h_w_user.data(), nb * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_n, p->h_normal_user.data(), nb * 2 * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_bc, p->h_bc.data(), nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !global) e = allow_optin_smem(k_pc_build2d<false>);
  if (e == cudaSuccess) {
    if (global)
      k_pc_build2d<true><<<nblocks, 1024, 0>>>(nb, bs, p->h, p->c, d_cell, d_w, d_n, d_bc, p->pc.d_inv, d_scr);
    else
      k_pc_build2d<false><<<nblocks, kPcThreads, per>>>(nb, bs, p->h, p->c, d_cell, d_w, d_n, d_bc, p->pc.d_inv,
                                                        nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_scr);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("preconditioner: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  p->pc.nblocks = nblocks;
  p->pc.valid = true;
  return BEM_OK;
}

bem_status build_preconditioner(bem_plan_s* p) {
  if (p->pc.kind == 0 || p->pc.valid) return BEM_OK;
  if (!p->have_bc) {
    set_error("preconditioner needs boundary conditions");
    return BEM_ERR_ARG;
  }
  ++p->pc_version;  // new inverse blocks (a new allocation): captured solve graphs are stale
  if (p->dim == 2 && !p->pf && p->pc.bs * p->ncomp <= kPcGpuMax) return build_preconditioner_gpu2d(p);
  const int64_t nb = p->nb;
  const int bs = p->pc.bs;
  const int nc = p->ncomp;
  const int nblocks = (int)((nb + bs - 1) / bs);
  const int m = bs * nc;
  std::vector<double> all((size_t)nblocks * m * m, 0.0);
  const double c = p->c;
  const int dim = p->dim;
  const double sigma = p->kernel == BEM_KELVIN_3D ? -1.0 : 1.0;  // K2 = +D or -T
  for (int b = 0; b < nblocks; ++b) {
    const int64_t i0 = (int64_t)b * bs;
    const int sz = (int)std::min<int64_t>(bs, nb - i0) * nc;
    std::vector<double> A((size_t)sz * sz);
    if (p->pf) panel_block(p, i0, sz, A.data());  // accuracy mode: exact panel integrals
    for (int ia = 0; ia < sz && !p->pf; ++ia) {
      const int64_t i = i0 + ia / nc;
      const int ca = ia % nc;
      for (int jb = 0; jb < sz; ++jb) {
        const int64_t j = i0 + jb / nc;
        const int cb = jb % nc;
        const double wj = p->h_w_user[j];
        const bool neu = p->h_bc[j * nc + cb] != 0;
        double v;
        if (dim == 2) {
          const int dx = p->h_cell_user[i * dim] - p->h_cell_user[j * dim];
          const int dy = p->h_cell_user[i * dim + 1] - p->h_cell_user[j * dim + 1];
          if (!neu)
            v = kernel2d_point(0, dx, dy, p->h) * wj;
          else
            v = (kernel2d_point(1, dx, dy, p->h) * p->h_normal_user[j * dim] +
                 kernel2d_point(2, dx, dy, p->h) * p->h_normal_user[j * dim + 1]) *
                wj;
        } else {
          const int dl[3] = {p->h_cell_user[i * 3] - p->h_cell_user[j * 3],
                             p->h_cell_user[i * 3 + 1] - p->h_cell_user[j * 3 + 1],
                             p->h_cell_user[i * 3 + 2] - p->h_cell_user[j * 3 + 2]};
          double blk[9];
          kernel3d_block(p->kernel, dl, &p->h_normal_user[j * 3], p->h, p->nu, p->mu, !neu, blk);
          v = (nc == 1 ? blk[0] : blk[ca * 3 + cb]) * wj * (neu ? sigma : 1.0);
        }
        if (neu && i == j && ca == cb) v -= c;
        A[(size_t)ia * sz + jb] = v;
      }
    }
    if (!invert(A, sz)) {
      A.assign((size_t)sz * sz, 0.0);
      for (int a = 0; a < sz; ++a) A[(size_t)a * sz + a] = 1.0;
    }
    // store padded to m x m
    double* dst = &all[(size_t)b * m * m];
    for (int a = 0; a < sz; ++a)
      for (int e = 0; e < sz; ++e) dst[(size_t)a * m + e] = A[(size_t)a * sz + e];

  }
  cudaFree(p->pc.d_inv);
  p->pc.d_inv = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&p->pc.d_inv, all.size() * sizeof(double)));
  BEM_CUDA_TRY(cudaMemcpy(p->pc.d_inv, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice));
  p->pc.nblocks = nblocks;
  p->pc.valid = true;
  return BEM_OK;
}

}  // namespace bemfft
