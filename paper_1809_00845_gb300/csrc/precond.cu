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
// average) as the FFT tables, assembled and inverted in FP64 on the host.
#include <cmath>
#include <vector>

#include "bem_internal.h"

namespace bemfft {

// 2D kernel value at grid offset (dx, dy): kind 0 = U, 1 = Q_x, 2 = Q_y,
// same definition as the FFT tables (Eq. 3, Eq. 15; singular cell = cell
// average for U, 0 for the odd kernels).
double kernel2d_point(int kind, int dx, int dy, double h) {
  const double PI = 3.14159265358979323846;
  if (dx == 0 && dy == 0) {
    if (kind != 0) return 0.0;
    const double L2 = PI / 4.0 - 1.5 - 0.5 * std::log(2.0);
    return -(std::log(h) + L2) / (2.0 * PI);
  }
  const double r2 = (double)dx * dx + (double)dy * dy;
  if (kind == 0) return -(0.5 * std::log(r2) + std::log(h)) / (2.0 * PI);
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

bem_status build_preconditioner(bem_plan_s* p) {
  if (p->pc.kind == 0 || p->pc.valid) return BEM_OK;
  if (!p->have_bc) {
    set_error("preconditioner needs boundary conditions");
    return BEM_ERR_ARG;
  }
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
    for (int ia = 0; ia < sz; ++ia) {
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
