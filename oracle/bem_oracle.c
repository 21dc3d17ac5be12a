/*
 * CPU FP64 direct-summation oracle for the FFT-accelerated boundary element
 * method (Benad, "Acceleration of the Boundary Element Method for arbitrary
 * shapes with the Fast Fourier Transformation").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes is the plain definition of the discrete operator that the
 * FFT path reaches exactly (up to rounding order): for boundary cells i, j on a
 * uniform grid of spacing h, with node positions x_g = (g + 1/2) h and the
 * offset d_ij = x_gi - x_gj (collocation point minus integration point, the
 * argument order of Eq. 15),
 *
 *   (S f)_i = sum_j U(d_ij) w_j f_j                       first integral of Eq. 15
 *   (D u)_i = sum_j sum_a Q_a(d_ij) w_j n_{a,j} u_j        second and third integrals
 *
 * with U = -ln r / (2 pi) (Eq. 3, 11) and Q_a = -d_a / (2 pi r^2) in 2D
 * (Eq. 15), U = 1/(4 pi r) and Q_a = -d_a/(4 pi r^3) in 3D, and for Navier's
 * equation the Kelvin tensor of Eq. 7 plus the traction kernel derived from it
 * with Hooke's law (the paper only says t* follows "with the material law";
 * the textbook Kelvin traction is used).
 *
 * w_j is the boundary measure carried by cell j (the "divide by the
 * discretisation length" of Section 4 folded into the source weight).
 *
 * Singular cell (d = 0): the kernel tables of Section 4 are "constant elements
 * on the entire parameter space", so the d = 0 entry is the average of the
 * kernel over the h-cell (square in 2D, cube in 3D):
 *   2D: mean of -ln r/(2 pi) over a square of side h = -(ln h + L2)/(2 pi),
 *       L2 = mean of ln r over [-1/2,1/2]^2 = pi/4 - 3/2 - ln(2)/2.
 *   3D: mean of 1/(4 pi r) over a cube of side h = C3/(4 pi h),
 *       C3 = integral of 1/r over [-1/2,1/2]^3 = 3 ln(2 + sqrt 3) - pi/2.
 *   Kelvin: mean of d_a d_b / r^3 over the cube = delta_ab C3/(3h).
 *   All odd kernels (Q_a, traction) average to zero over the symmetric cell.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define BO_PI 3.14159265358979323846

enum { BO_LAPLACE_2D = 0, BO_LAPLACE_3D = 1, BO_KELVIN_3D = 2 };
enum { BO_SINGLE = 0, BO_DOUBLE = 1 };

/* Mean of ln r over the unit square centred at the origin (closed form). */
double bo_L2(void) { return BO_PI / 4.0 - 1.5 - 0.5 * log(2.0); }

/* Integral of 1/r over the unit cube centred at the origin (closed form). */
double bo_C3(void) { return 3.0 * log(2.0 + sqrt(3.0)) - BO_PI / 2.0; }

int bo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void bo_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ---------------------------------------------------------------- kernels -- */

/* 2D Laplace fundamental solution, Eq. 3 / Eq. 11, d = target - source. */
double bo_lap2d_U(double dx, double dy, double h) {
  double r2 = dx * dx + dy * dy;
  if (r2 == 0.0) return -(log(h) + bo_L2()) / (2.0 * BO_PI);
  return -0.5 * log(r2) / (2.0 * BO_PI);
}

/* 2D kernel of the second/third integral of Eq. 15: -d_a / (2 pi r^2). */
double bo_lap2d_Q(int a, double dx, double dy) {
  double r2 = dx * dx + dy * dy;
  if (r2 == 0.0) return 0.0;
  double da = (a == 0) ? dx : dy;
  return -da / (2.0 * BO_PI * r2);
}

/* 3D Laplace fundamental solution 1/(4 pi r). */
double bo_lap3d_U(double dx, double dy, double dz, double h) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (r2 == 0.0) return bo_C3() / (4.0 * BO_PI * h);
  return 1.0 / (4.0 * BO_PI * sqrt(r2));
}

/* Gradient of the 3D fundamental solution with respect to d: -d_a/(4 pi r^3). */
double bo_lap3d_Q(int a, double dx, double dy, double dz) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (r2 == 0.0) return 0.0;
  double d[3] = {dx, dy, dz};
  double r = sqrt(r2);
  return -d[a] / (4.0 * BO_PI * r2 * r);
}

/* Kelvin displacement tensor, Eq. 7: U_ab = [(3-4nu) delta_ab / r +
 * d_a d_b / r^3] / (16 pi mu (1 - nu)).  Written row-major into U[9]. */
void bo_kelvin_U(const double d[3], double nu, double mu, double h, double U[9]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double pref = 1.0 / (16.0 * BO_PI * mu * (1.0 - nu));
  if (r2 == 0.0) {
    /* cube averages: <1/r> = C3/h, <d_a d_b / r^3> = delta_ab C3/(3h) */
    double diag = pref * (3.0 - 4.0 * nu + 1.0 / 3.0) * bo_C3() / h;
    for (int k = 0; k < 9; ++k) U[k] = 0.0;
    U[0] = U[4] = U[8] = diag;
    return;
  }
  double r = sqrt(r2);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      U[3 * a + b] = pref * (((a == b) ? (3.0 - 4.0 * nu) / r : 0.0) + d[a] * d[b] / (r2 * r));
}

/* Kelvin traction tensor T_ab(d; n): traction component b on a surface with
 * unit normal n at the integration point, due to a unit point force in
 * direction a at the collocation point (textbook form, e.g. Brebbia and
 * Dominguez), expressed with d = collocation - integration point.  With
 * r_,a = (x_a - x0_a)/r = -d_a/r:
 *   T_ab = -[ dr/dn ((1-2nu) delta_ab + 3 r_,a r_,b)
 *             - (1-2nu)(r_,a n_b - r_,b n_a) ] / (8 pi (1-nu) r^2).
 * Zero at d = 0 (odd kernel on the symmetric cell). */
void bo_kelvin_T(const double d[3], const double n[3], double nu, double T[9]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (r2 == 0.0) {
    for (int k = 0; k < 9; ++k) T[k] = 0.0;
    return;
  }
  double r = sqrt(r2);
  double rd[3] = {-d[0] / r, -d[1] / r, -d[2] / r}; /* r_,a */
  double drdn = rd[0] * n[0] + rd[1] * n[1] + rd[2] * n[2];
  double c = 1.0 - 2.0 * nu;
  double pref = -1.0 / (8.0 * BO_PI * (1.0 - nu) * r2);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double t = drdn * (((a == b) ? c : 0.0) + 3.0 * rd[a] * rd[b]) - c * (rd[a] * n[b] - rd[b] * n[a]);
      T[3 * a + b] = pref * t;
    }
}

/* ---------------------------------------------------------- direct sums -- */

static int bo_ncomp(int kernel) { return kernel == BO_KELVIN_3D ? 3 : 1; }
static int bo_dim(int kernel) { return kernel == BO_LAPLACE_2D ? 2 : 3; }

/* Coefficient block A_ij (ncomp x ncomp, row-major) of the discrete operator:
 * the weight w_j is included, so that out_i = sum_j A_ij in_j. */
static void bo_block(int kernel, int layer, const int32_t* ci, const int32_t* cj, double h, double wj,
                     const double* nj, double nu, double mu, double* blk) {
  int dim = bo_dim(kernel);
  double d[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < dim; ++a) d[a] = (double)(ci[a] - cj[a]) * h;
  if (kernel == BO_LAPLACE_2D) {
    if (layer == BO_SINGLE)
      blk[0] = bo_lap2d_U(d[0], d[1], h) * wj;
    else
      blk[0] = (bo_lap2d_Q(0, d[0], d[1]) * nj[0] + bo_lap2d_Q(1, d[0], d[1]) * nj[1]) * wj;
  } else if (kernel == BO_LAPLACE_3D) {
    if (layer == BO_SINGLE)
      blk[0] = bo_lap3d_U(d[0], d[1], d[2], h) * wj;
    else
      blk[0] = (bo_lap3d_Q(0, d[0], d[1], d[2]) * nj[0] + bo_lap3d_Q(1, d[0], d[1], d[2]) * nj[1] +
                bo_lap3d_Q(2, d[0], d[1], d[2]) * nj[2]) *
               wj;
  } else {
    double K[9];
    if (layer == BO_SINGLE)
      bo_kelvin_U(d, nu, mu, h, K);
    else
      bo_kelvin_T(d, nj, nu, K);
    for (int k = 0; k < 9; ++k) blk[k] = K[k] * wj;
  }
}

/* out[r - row0] = (K in)_r for target rows r in [row0, row0 + nrows).
 * kernel: 0 = 2D Laplace, 1 = 3D Laplace, 2 = 3D Kelvin; layer: 0 = single
 * (S or U), 1 = double (D or T).  cell: nb x dim grid indices; w: nb weights;
 * normal: nb x dim unit normals; in: nb x ncomp; out: nrows x ncomp. */
int bo_apply(int kernel, int layer, int64_t nb, const int32_t* cell, double h, const double* w,
             const double* normal, double nu, double mu, const double* in, double* out, int64_t row0,
             int64_t nrows) {
  if (kernel < 0 || kernel > 2 || layer < 0 || layer > 1) return 1;
  if (row0 < 0 || nrows < 0 || row0 + nrows > nb) return 1;
  const int dim = bo_dim(kernel), nc = bo_ncomp(kernel);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = row0; r < row0 + nrows; ++r) {
    double acc[3] = {0.0, 0.0, 0.0};
    double blk[9];
    for (int64_t j = 0; j < nb; ++j) {
      bo_block(kernel, layer, cell + r * dim, cell + j * dim, h, w[j], normal + j * dim, nu, mu, blk);
      for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) acc[a] += blk[a * nc + b] * in[j * nc + b];
    }
    for (int a = 0; a < nc; ++a) out[(r - row0) * nc + a] = acc[a];
  }
  return 0;
}

/* Dense operator matrix (nb*ncomp)^2, row-major, for the dense LU solve. */
int bo_matrix(int kernel, int layer, int64_t nb, const int32_t* cell, double h, const double* w,
              const double* normal, double nu, double mu, double* A) {
  if (kernel < 0 || kernel > 2 || layer < 0 || layer > 1) return 1;
  const int dim = bo_dim(kernel), nc = bo_ncomp(kernel);
  const int64_t ld = nb * nc;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nb; ++i) {
    double blk[9];
    for (int64_t j = 0; j < nb; ++j) {
      bo_block(kernel, layer, cell + i * dim, cell + j * dim, h, w[j], normal + j * dim, nu, mu, blk);
      for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) A[(i * nc + a) * ld + j * nc + b] = blk[a * nc + b];
    }
  }
  return 0;
}

/* Point evaluation of a kernel at an arbitrary offset d (continuum check of
 * signs and magnitudes through Green's/Somigliana's identity).  Returns the
 * ncomp x ncomp block with unit weight; for the double layer, n is the normal
 * at the integration point.  d must be non-zero. */
int bo_kernel_point(int kernel, int layer, const double* d, const double* n, double nu, double mu,
                    double* blk) {
  if (kernel == BO_LAPLACE_2D) {
    if (layer == BO_SINGLE)
      blk[0] = bo_lap2d_U(d[0], d[1], 1.0);
    else
      blk[0] = bo_lap2d_Q(0, d[0], d[1]) * n[0] + bo_lap2d_Q(1, d[0], d[1]) * n[1];
    return 0;
  }
  if (kernel == BO_LAPLACE_3D) {
    if (layer == BO_SINGLE)
      blk[0] = bo_lap3d_U(d[0], d[1], d[2], 1.0);
    else
      blk[0] = bo_lap3d_Q(0, d[0], d[1], d[2]) * n[0] + bo_lap3d_Q(1, d[0], d[1], d[2]) * n[1] +
               bo_lap3d_Q(2, d[0], d[1], d[2]) * n[2];
    return 0;
  }
  if (kernel == BO_KELVIN_3D) {
    if (layer == BO_SINGLE)
      bo_kelvin_U(d, nu, mu, 1.0, blk);
    else
      bo_kelvin_T(d, n, nu, blk);
    return 0;
  }
  return 1;
}
