// Accuracy mode: the paper's grid convolution (Section 4, Eq. 16) with the
// unknowns on the boundary itself, by the precorrected-FFT construction
// (Phillips and White, IEEE TCAD 16(10), 1997).
//
// The boundary is a set of flat panels (A_j -> B_j, length L_j, outward
// normal n_j = tangent turned clockwise, collocation at the midpoint m_j),
// with piecewise-constant densities.  Operators with the paper's signs
// (Eq. 15, c u = S q + D u, c = 1/2 at a midpoint):
//   (S q)_i = sum_j q_j int_{panel j} U(|m_i - y|) ds_y,   U(r) = -ln r / (2 pi)
//   (D u)_i = sum_j u_j int_{panel j} -(m_i - y).n_j / (2 pi |m_i - y|^2) ds_y
// Grid: node k at ((kx + 1/2) h, (ky + 1/2) h).  A point's stencil of order p
// has (p + 1)^2 nodes, per axis a - 1 .. a + p - 1 around the anchor
// a = floor(u + 1/2) (p = 2) or floor(u) (p = 3), u = m / h - 1/2, with
// tensor-product Lagrange weights.  The apply is
//   out = I (G (P x)) + C x + diag x
//   P: each panel's moments on the stencil of its midpoint,
//      single layer int_panel L_l ds, dipole -int_panel n . grad L_l ds
//      (Gauss-Legendre, p + 1 points: exact for these polynomials);
//   G: the paper's node-to-node operator (the inner plan over the active
//      nodes, single layer, unit weights: same tables, spectra and kernels);
//   I: interpolation of the node potentials at the midpoints;
//   C: near pairs (anchors within R along both axes): exact panel integral
//      minus the grid-mediated value of the same pair;
//   diag: double layer only, 1/2 - (row sum of the rest): Gauss's law makes
//      the exact rows sum to 1/2 on a closed curve; restoring it leaves the
//      far-field error acting on u_j - u_i.
// Host code builds every table in FP64; the two kernels accumulate in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "bem_internal.h"
#include "fft_reg.cuh"

namespace bemfft {

namespace {

constexpr double kPi = 3.14159265358979323846;

// 1D Lagrange weights and their derivatives (per node spacing) at local
// coordinate xi on the offsets -1 .. order - 1
void lagrange(int order, double xi, double* w, double* dw) {
  const int q = order + 1;
  for (int a = 0; a < q; ++a) {
    const double oa = a - 1;
    double den = 1.0, num = 1.0, der = 0.0;
    for (int b = 0; b < q; ++b) {
      if (b == a) continue;
      den *= oa - (b - 1);
      num *= xi - (b - 1);
    }
    for (int c = 0; c < q; ++c) {
      if (c == a) continue;
      double t = 1.0;
      for (int b = 0; b < q; ++b)
        if (b != a && b != c) t *= xi - (b - 1);
      der += t;
    }
    w[a] = num / den;
    dw[a] = der / den;
  }
}

int anchor(int order, double u) { return (int)std::floor(order == 2 ? u + 0.5 : u); }

// Gauss-Legendre points and weights on [-1, 1] (order + 1 points)
void gauss(int order, double* x, double* w) {
  if (order == 2) {
    const double a = std::sqrt(0.6);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
  } else {
    const double r = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
    const double a = std::sqrt(3.0 / 7.0 - r), b = std::sqrt(3.0 / 7.0 + r);
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
  }
}

struct Panel {
  double ax, ay, tx, ty, nx, ny, L, mx, my;
};

Panel make_panel(const double* P) {
  Panel q;
  q.ax = P[0];
  q.ay = P[1];
  const double dx = P[2] - P[0], dy = P[3] - P[1];
  q.L = std::hypot(dx, dy);
  q.tx = dx / q.L;
  q.ty = dy / q.L;
  q.nx = q.ty;
  q.ny = -q.tx;
  q.mx = 0.5 * (P[0] + P[2]);
  q.my = 0.5 * (P[1] + P[3]);
  return q;
}

// exact integrals over panel q at target (x, y): single layer and double
// layer (paper sign); on the panel's own line the double layer vanishes
// (principal value)
void exact_pair(const Panel& q, double x, double y, double* s, double* d) {
  const double rx = x - q.ax, ry = y - q.ay;
  const double s0 = rx * q.tx + ry * q.ty;
  double eta = rx * q.nx + ry * q.ny;
  if (std::fabs(eta) < 1e-11 * q.L) eta = 0.0;
  // int ln sqrt(u^2 + eta^2) du = u ln sqrt(u^2 + eta^2) - u + eta atan(u / eta)
  auto F = [&](double u) {
    const double r2 = u * u + eta * eta;
    double v = -u;
    if (r2 > 0.0) v += 0.5 * u * std::log(r2);
    if (eta != 0.0) v += eta * std::atan(u / eta);
    return v;
  };
  *s = -(F(q.L - s0) - F(-s0)) / (2.0 * kPi);
  *d = eta == 0.0 ? 0.0 : -(std::atan((q.L - s0) / eta) - std::atan(-s0 / eta)) / (2.0 * kPi);
}

template <typename T, typename TI>
__global__ void k_pf_project(int64_t nnodes, const int64_t* __restrict__ ptr, const int32_t* __restrict__ pj,
                             const double* __restrict__ ws, const double* __restrict__ wd,
                             const uint8_t* __restrict__ bc, int layer, const T* __restrict__ x,
                             TI* __restrict__ rho) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nnodes) return;
  double acc = 0.0;
  for (int64_t e = ptr[l]; e < ptr[l + 1]; ++e) {
    const int32_t j = pj[e];
    const bool dip = layer == BEM_DOUBLE || (layer == BEM_SYSTEM && bc[j] != 0);
    acc += (dip ? wd[e] : ws[e]) * (double)x[j];
  }
  rho[l] = (TI)acc;
}

// Edge-flow form (FP32 inner plans): each projected dipole's node charges sum
// to zero, so they are the divergence of flows along the grid edges inside
// its stencil (c_m = p_{m - e} - p_m summed over x and y edges); the inner
// plan convolves the flows with the difference of the grid kernel instead of
// the charges with the kernel.  Same operator; but the flows enter the FP32
// transforms where the rounding of large, cancelling charges would have
// reached every target through the logarithm's long range.  Densities are
// written straight to the inner plan's interleaved positions: (charge,
// x-edge flow) pairs and the y-edge flows; padding positions get zeros.
template <typename T, typename TA>
__global__ void k_pf_project_edge(int npos, const int32_t* __restrict__ perm, const int64_t* __restrict__ ptr,
                                  const int32_t* __restrict__ pj, const double* __restrict__ ws,
                                  const double* __restrict__ wx, const double* __restrict__ wy,
                                  const uint8_t* __restrict__ bc, int layer, const T* __restrict__ x,
                                  cplx<TA>* __restrict__ val, TA* __restrict__ val2) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= npos) return;
  const int l = perm[pos];
  double a = 0.0, b = 0.0, c = 0.0;
  if (l >= 0) {
    for (int64_t e = ptr[l]; e < ptr[l + 1]; ++e) {
      const int32_t j = pj[e];
      const double xj = (double)x[j];
      if (layer == BEM_DOUBLE || (layer == BEM_SYSTEM && bc[j] != 0)) {
        b += wx[e] * xj;
        c += wy[e] * xj;
      } else {
        a += ws[e] * xj;
      }
    }
  }
  val[pos] = {TA(a), TA(b)};
  val2[pos] = TA(c);
}

template <typename T, typename TI>
__global__ void k_pf_interp(int64_t nb, int S, const int32_t* __restrict__ node, const T* __restrict__ W,
                            const TI* __restrict__ phi, const int64_t* __restrict__ nptr,
                            const int32_t* __restrict__ nj, const T* __restrict__ cS, const T* __restrict__ cD,
                            const T* __restrict__ delta, const uint8_t* __restrict__ bc, double c, int layer,
                            const T* __restrict__ x, T* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double acc = 0.0;
  for (int s = 0; s < S; ++s) acc += (double)W[i * S + s] * (double)phi[node[i * S + s]];
  for (int64_t e = nptr[i]; e < nptr[i + 1]; ++e) {
    const int32_t j = nj[e];
    const bool dip = layer == BEM_DOUBLE || (layer == BEM_SYSTEM && bc[j] != 0);
    acc += (double)(dip ? cD[e] : cS[e]) * (double)x[j];
  }
  double dg = 0.0;
  if (layer == BEM_DOUBLE) dg = (double)delta[i];
  else if (layer == BEM_SYSTEM && bc[i] != 0) dg = (double)delta[i] - c;
  out[i] = (T)(acc + dg * (double)x[i]);
}

template <typename T>
bem_status upload(const std::vector<double>& v, void** d) {
  std::vector<T> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) t[i] = (T)v[i];
  BEM_CUDA_TRY(cudaMalloc(d, std::max<size_t>(1, t.size()) * sizeof(T)));
  if (!t.empty()) BEM_CUDA_TRY(cudaMemcpy(*d, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
  return BEM_OK;
}

template <typename X>
bem_status upload_raw(const std::vector<X>& v, X** d) {
  BEM_CUDA_TRY(cudaMalloc(d, std::max<size_t>(1, v.size()) * sizeof(X)));
  if (!v.empty()) BEM_CUDA_TRY(cudaMemcpy(*d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
  return BEM_OK;
}

// T: the plan's I/O type; TI: the inner node plan's (FP64 inner plans serve
// FP32 accuracy-mode plans on grids below the four-step kernel's)
template <typename T, typename TI>
bem_status launch_t(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st) {
  PanelOp& f = *p->pf;
  const int tb = 256;
  bem_status rc;
  if (f.edge && layer != BEM_SINGLE) {
    const int npos = (int)f.inner->v2_npos;
    const unsigned nblk = (unsigned)((npos + tb - 1) / tb);
    const T* x = static_cast<const T*>(in);
    bem_plan_s* q = f.inner;
    if (q->prec == BEM_F32)
      k_pf_project_edge<T, float><<<nblk, tb, 0, st>>>(npos, q->d_perm_il, f.d_pptr, f.d_pj, f.d_pws, f.d_pwx,
                                                       f.d_pwy, f.d_bc, (int)layer, x,
                                                       static_cast<cplx<float>*>(q->d_val),
                                                       static_cast<float*>(q->d_val2));
    else if (q->prec == BEM_F64)
      k_pf_project_edge<T, double><<<nblk, tb, 0, st>>>(npos, q->d_perm_il, f.d_pptr, f.d_pj, f.d_pws, f.d_pwx,
                                                        f.d_pwy, f.d_bc, (int)layer, x,
                                                        static_cast<cplx<double>*>(q->d_val),
                                                        static_cast<double*>(q->d_val2));
    else
      k_pf_project_edge<T, f32x2><<<nblk, tb, 0, st>>>(npos, q->d_perm_il, f.d_pptr, f.d_pj, f.d_pws, f.d_pwx,
                                                       f.d_pwy, f.d_bc, (int)layer, x,
                                                       static_cast<cplx<f32x2>*>(q->d_val),
                                                       static_cast<f32x2*>(q->d_val2));
    BEM_CUDA_TRY(cudaGetLastError());
    if ((rc = launch_edge_2d(q, f.d_phi, st)) != BEM_OK) return rc;
  } else {
    k_pf_project<T, TI><<<(unsigned)((f.nnodes + tb - 1) / tb), tb, 0, st>>>(
        f.nnodes, f.d_pptr, f.d_pj, f.d_pws, f.d_pwd, f.d_bc, (int)layer, static_cast<const T*>(in),
        static_cast<TI*>(f.d_rho));
    BEM_CUDA_TRY(cudaGetLastError());
    if ((rc = apply_operator(f.inner, BEM_SINGLE, f.d_rho, f.d_phi, st)) != BEM_OK) return rc;
  }
  k_pf_interp<T, TI><<<(unsigned)((p->nb + tb - 1) / tb), tb, 0, st>>>(
      p->nb, f.S, f.d_node, static_cast<const T*>(f.d_W), static_cast<const TI*>(f.d_phi), f.d_nptr, f.d_nj,
      static_cast<const T*>(f.d_cS), static_cast<const T*>(f.d_cD), static_cast<const T*>(f.d_delta), f.d_bc, p->c,
      (int)layer, static_cast<const T*>(in), static_cast<T*>(out));
  BEM_CUDA_TRY(cudaGetLastError());
  return BEM_OK;
}

}  // namespace

bem_status launch_apply_panels(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st) {
  if (layer != BEM_SINGLE && layer != BEM_DOUBLE && layer != BEM_SYSTEM) {
    set_error("bem_apply: unknown layer");
    return BEM_ERR_ARG;
  }
  if (layer == BEM_SYSTEM && !p->have_bc) {
    set_error("bem_apply: BEM_SYSTEM needs bem_set_bc first");
    return BEM_ERR_ARG;
  }
  if (p->prec != BEM_F32) return launch_t<double, double>(p, layer, in, out, st);
  return p->pf->inner->prec == BEM_F32 ? launch_t<float, float>(p, layer, in, out, st)
                                       : launch_t<float, double>(p, layer, in, out, st);
}

bem_status panel_set_bc(bem_plan_s* p, const uint8_t* bc, double c) {
  if (p->have_bc && c == p->c && std::equal(p->h_bc.begin(), p->h_bc.end(), bc)) return BEM_OK;
  ++p->op_version;
  p->h_bc.assign(bc, bc + p->nb);
  p->c = c;
  BEM_CUDA_TRY(cudaMemcpy(p->pf->d_bc, bc, p->nb, cudaMemcpyHostToDevice));
  p->have_bc = true;
  p->pc.valid = false;
  return BEM_OK;
}

void panel_block(const bem_plan_s* p, int64_t i0, int sz, double* A) {
  const PanelOp& f = *p->pf;
  for (int a = 0; a < sz; ++a) {
    const int64_t i = i0 + a;
    const Panel qi = make_panel(&f.h_panels[4 * i]);
    for (int b = 0; b < sz; ++b) {
      const int64_t j = i0 + b;
      double s, d;
      exact_pair(make_panel(&f.h_panels[4 * j]), qi.mx, qi.my, &s, &d);
      const bool neu = p->h_bc[j] != 0;
      double v = neu ? d : s;
      if (neu && i == j) v += f.h_delta[i] - p->c;
      A[(size_t)a * sz + b] = v;
    }
  }
}

void panel_destroy(bem_plan_s* p) {
  PanelOp* f = p->pf;
  if (!f) return;
  if (f->inner) bem_destroy(f->inner);
  for (void* q : {(void*)f->d_node, f->d_W, (void*)f->d_pptr, (void*)f->d_pj, (void*)f->d_pws, (void*)f->d_pwd,
                  (void*)f->d_pwx, (void*)f->d_pwy, (void*)f->d_nptr, (void*)f->d_nj, f->d_cS, f->d_cD, f->d_delta,
                  (void*)f->d_bc, f->d_rho, f->d_phi})
    cudaFree(q);
  delete f;
  p->pf = nullptr;
}

// The Gauss row-sum term of an FP32 plan, delta_i = 1/2 - (D 1)_i without
// it, in FP64: the node potentials of the projected dipoles of u = 1 from a
// temporary FP64 node plan (the grid convolution on the device), the
// interpolation and the near-pair sums on the host.  The double layer of
// random data is two orders of magnitude smaller than its terms, so delta
// has to be exact to far below FP32 rounding of the row sums (about 1/2).
template <typename T>
static bem_status fp64_row_sums(bem_plan_s* p, const std::vector<int32_t>& node, const std::vector<double>& W,
                                const std::vector<int64_t>& pptr, const std::vector<double>& pwd,
                                const std::vector<int32_t>& cells) {
  PanelOp& f = *p->pf;
  const int64_t nn = f.nnodes, nb = p->nb;
  const int S = f.S;
  std::vector<double> rho1(nn, 0.0), phi1(nn);
  for (int64_t l = 0; l < nn; ++l)
    for (int64_t e = pptr[l]; e < pptr[l + 1]; ++e) rho1[l] += pwd[e];
  bem_plan_t tmp = nullptr;
  const int64_t n2[2] = {p->n, p->n};
  std::vector<double> w1(nn, 1.0), nrm(2 * nn, 0.0);
  for (int64_t k = 0; k < nn; ++k) nrm[2 * k] = 1.0;
  bem_status rc = bem_plan(&tmp, 2, n2, p->h, nn, cells.data(), w1.data(), nrm.data(), BEM_LAPLACE_2D, 0.3, 1.0,
                           BEM_F64, BEM_PLAN_SINGLE_LAYER_ONLY, nullptr);
  if (rc != BEM_OK) return rc;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 2 * nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(buf, rho1.data(), nn * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) rc = apply_operator(tmp, BEM_SINGLE, buf, buf + nn, nullptr);
  if (e == cudaSuccess && rc == BEM_OK) e = cudaMemcpy(phi1.data(), buf + nn, nn * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  bem_destroy(tmp);
  if (e != cudaSuccess) {
    set_error(std::string("bem_plan_panels: row-sum term: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (rc != BEM_OK) return rc;
  f.h_delta.resize(nb);
  std::vector<T> dt(nb);
  for (int64_t i = 0; i < nb; ++i) {
    double acc = 0.0;
    for (int s2 = 0; s2 < S; ++s2) acc += W[(size_t)i * S + s2] * phi1[node[(size_t)i * S + s2]];
    for (int64_t k = f.h_nptr[i]; k < f.h_nptr[i + 1]; ++k) acc += f.h_cD[k];
    f.h_delta[i] = 0.5 - acc;
    dt[i] = (T)f.h_delta[i];
  }
  BEM_CUDA_TRY(cudaMemcpy(f.d_delta, dt.data(), nb * sizeof(T), cudaMemcpyHostToDevice));
  return BEM_OK;
}

template <typename T, typename TI>
static bem_status upload_all(bem_plan_s* p, const std::vector<int32_t>& node, const std::vector<double>& W,
                             const std::vector<int64_t>& pptr, const std::vector<int32_t>& pj,
                             const std::vector<double>& pws, const std::vector<double>& pwd,
                             const std::vector<double>& pwx, const std::vector<double>& pwy,
                             const std::vector<int32_t>& cells) {
  PanelOp& f = *p->pf;
  bem_status rc;
  if ((rc = upload_raw(node, &f.d_node)) != BEM_OK) return rc;
  if ((rc = upload<T>(W, &f.d_W)) != BEM_OK) return rc;
  if ((rc = upload_raw(pptr, &f.d_pptr)) != BEM_OK) return rc;
  if ((rc = upload_raw(pj, &f.d_pj)) != BEM_OK) return rc;
  if ((rc = upload_raw(pws, &f.d_pws)) != BEM_OK) return rc;
  if ((rc = upload_raw(pwd, &f.d_pwd)) != BEM_OK) return rc;
  if (f.edge) {
    if ((rc = upload_raw(pwx, &f.d_pwx)) != BEM_OK) return rc;
    if ((rc = upload_raw(pwy, &f.d_pwy)) != BEM_OK) return rc;
  }
  if ((rc = upload_raw(f.h_nptr, &f.d_nptr)) != BEM_OK) return rc;
  if ((rc = upload_raw(f.h_nj, &f.d_nj)) != BEM_OK) return rc;
  if ((rc = upload<T>(f.h_cS, &f.d_cS)) != BEM_OK) return rc;
  if ((rc = upload<T>(f.h_cD, &f.d_cD)) != BEM_OK) return rc;
  std::vector<double> zero(p->nb, 0.0);
  if ((rc = upload<T>(zero, &f.d_delta)) != BEM_OK) return rc;
  BEM_CUDA_TRY(cudaMalloc(&f.d_bc, p->nb));
  BEM_CUDA_TRY(cudaMemset(f.d_bc, 0, p->nb));
  BEM_CUDA_TRY(cudaMalloc(&f.d_rho, f.nnodes * sizeof(TI)));
  BEM_CUDA_TRY(cudaMalloc(&f.d_phi, f.nnodes * sizeof(TI)));
  f.bytes = node.size() * 4 + (W.size() + f.h_cS.size() + f.h_cD.size() + p->nb) * sizeof(T) +
            2 * f.nnodes * sizeof(TI) + (pws.size() + pwd.size() + (f.edge ? pwx.size() + pwy.size() : 0)) * 8 +
            (pptr.size() + f.h_nptr.size()) * 8 + (pj.size() + f.h_nj.size()) * 4 + p->nb;
  if constexpr (std::is_same<T, float>::value) return fp64_row_sums<T>(p, node, W, pptr, pwd, cells);
  // Gauss row-sum term: delta = 1/2 - (D 1) of the operator without it
  // (ones and the result share one scratch allocation, freed on every path)
  T* buf = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&buf, 2 * p->nb * sizeof(T)));
  T* ones = buf;
  T* dl = buf + p->nb;
  std::vector<T> h1(p->nb, (T)1);
  cudaError_t e = cudaMemcpy(ones, h1.data(), p->nb * sizeof(T), cudaMemcpyHostToDevice);
  rc = e == cudaSuccess ? launch_t<T, TI>(p, BEM_DOUBLE, ones, dl, nullptr) : BEM_ERR_CUDA;
  if (rc == BEM_OK) e = cudaMemcpy(h1.data(), dl, p->nb * sizeof(T), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) {
    set_error(std::string("bem_plan_panels: row-sum term: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (rc != BEM_OK) return rc;
  f.h_delta.resize(p->nb);
  std::vector<T> dt(p->nb);
  for (int64_t i = 0; i < p->nb; ++i) {
    f.h_delta[i] = 0.5 - (double)h1[i];
    dt[i] = (T)f.h_delta[i];
  }
  BEM_CUDA_TRY(cudaMemcpy(f.d_delta, dt.data(), p->nb * sizeof(T), cudaMemcpyHostToDevice));
  return BEM_OK;
}

bem_status panel_plan_impl(bem_plan_s** out, int64_t n, double h, int64_t nb, const double* panels, int order,
                           int R, bem_precision prec, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  *out = nullptr;
  if (order != 2 && order != 3) {
    set_error("bem_plan_panels: stencil order must be 2 or 3");
    return BEM_ERR_ARG;
  }
  if (R < order || R > 64) {
    set_error("bem_plan_panels: need order <= near radius <= 64");
    return BEM_ERR_ARG;
  }
  if (nb < 1 || nb > (int64_t)1 << 28 || !(h > 0.0) || !std::isfinite(h) || n < 4) {
    set_error("bem_plan_panels: need nb >= 1, h > 0, n >= 4");
    return BEM_ERR_ARG;
  }
  const int q = order + 1, S = q * q;
  std::vector<Panel> pan(nb);
  for (int64_t j = 0; j < nb; ++j) {
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(panels[4 * j + k])) {
        set_error("bem_plan_panels: non-finite panel coordinate");
        return BEM_ERR_ARG;
      }
    pan[j] = make_panel(&panels[4 * j]);
    if (!(pan[j].L > 0.0)) {
      set_error("bem_plan_panels: zero-length panel");
      return BEM_ERR_ARG;
    }
  }
  // stencils of the midpoints: anchors, interpolation weights, node keys
  std::vector<int32_t> anc(2 * nb);
  std::vector<double> W((size_t)nb * S), PS((size_t)nb * S, 0.0), PD((size_t)nb * S, 0.0);
  std::vector<int64_t> key((size_t)nb * S);
  double gx[4], gw[4];
  gauss(order, gx, gw);
  for (int64_t j = 0; j < nb; ++j) {
    const Panel& P = pan[j];
    const double ux = P.mx / h - 0.5, uy = P.my / h - 0.5;
    const int axj = anchor(order, ux), ayj = anchor(order, uy);
    anc[2 * j] = axj;
    anc[2 * j + 1] = ayj;
    if (axj - 1 < 0 || ayj - 1 < 0 || axj + order - 1 >= n || ayj + order - 1 >= n) {
      set_error("bem_plan_panels: a panel's stencil leaves the grid (keep the boundary 2 cells inside)");
      return BEM_ERR_ARG;
    }
    double wx[4], dwx[4], wy[4], dwy[4];
    lagrange(order, ux - axj, wx, dwx);
    lagrange(order, uy - ayj, wy, dwy);
    for (int by = 0; by < q; ++by)
      for (int bx = 0; bx < q; ++bx) {
        const int s = by * q + bx;
        W[(size_t)j * S + s] = wx[bx] * wy[by];
        key[(size_t)j * S + s] = (int64_t)(ayj - 1 + by) * n + (axj - 1 + bx);
      }
    // moments of the panel on the same nodes (Gauss-Legendre along the panel)
    for (int g = 0; g <= order; ++g) {
      const double sg = 0.5 * (gx[g] + 1.0) * P.L, ww = 0.5 * gw[g] * P.L;
      const double yx = P.ax + sg * P.tx, yy = P.ay + sg * P.ty;
      lagrange(order, yx / h - 0.5 - axj, wx, dwx);
      lagrange(order, yy / h - 0.5 - ayj, wy, dwy);
      for (int by = 0; by < q; ++by)
        for (int bx = 0; bx < q; ++bx) {
          const int s = by * q + bx;
          PS[(size_t)j * S + s] += ww * wx[bx] * wy[by];
          PD[(size_t)j * S + s] -= ww * (dwx[bx] * wy[by] * P.nx + wx[bx] * dwy[by] * P.ny) / h;
        }
    }
  }
  // active nodes (sorted keys) and the inner node plan
  std::vector<int64_t> nodes(key);
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
  const int64_t nn = (int64_t)nodes.size();
  std::vector<int32_t> node((size_t)nb * S);
  for (size_t e = 0; e < key.size(); ++e)
    node[e] = (int32_t)(std::lower_bound(nodes.begin(), nodes.end(), key[e]) - nodes.begin());
  auto* p = new bem_plan_s();
  p->pf = new PanelOp();
  PanelOp& f = *p->pf;
  f.order = order;
  f.R = R;
  f.S = S;
  f.nnodes = nn;
  f.public_prec = prec;
  f.h_panels.assign(panels, panels + 4 * nb);
  p->dim = 2;
  p->ncomp = 1;
  p->kernel = BEM_LAPLACE_2D;
  p->nb = nb;
  p->n = n;
  p->N = 2 * n;
  p->h = h;
  p->pc.bs = 64;
  cudaGetDevice(&p->device);
  auto fail = [&](bem_status rc) {
    bem_destroy(p);
    return rc;
  };
  std::vector<int32_t> cells(2 * nn);  // the active nodes as the inner plan's cells
  for (int64_t k = 0; k < nn; ++k) {
    cells[2 * k] = (int32_t)(nodes[k] % n);
    cells[2 * k + 1] = (int32_t)(nodes[k] / n);
  }
  {
    const std::vector<int32_t>& cell = cells;
    std::vector<double> w1(nn, 1.0), nrm(2 * nn, 0.0);
    for (int64_t k = 0; k < nn; ++k) nrm[2 * k] = 1.0;
    const int64_t nn2[2] = {n, n};
    // FP32 on grids below the four-step kernel (n < 256): the node convolution
    // in FP64, which costs little there
    const bem_precision iprec = (prec == BEM_F32 && n < 256) ? BEM_F64 : prec;
    bem_status rc = bem_plan(&f.inner, 2, nn2, h, nn, cell.data(), w1.data(), nrm.data(), BEM_LAPLACE_2D, 0.3, 1.0,
                             iprec, BEM_PLAN_SINGLE_LAYER_ONLY, st);
    if (rc != BEM_OK) return fail(rc);
  }
  p->prec = prec == BEM_F32 ? BEM_F32 : f.inner->prec;
  p->tc = f.inner->tc;
  // FP32 four-step inner plans take the double layer in the edge-flow form
  // (FP64 and double-float convolve the charges to 1e-13 already; the edge
  // form would cost them a second inverse transform and gather per apply)
  f.edge = f.inner->prec == BEM_F32 && f.inner->v2 && f.inner->tc == 0;
  if (f.edge) {
    bem_status rc = setup_edge_2d(f.inner);
    if (rc != BEM_OK) return fail(rc);
  }
  // projection CSR by node
  std::vector<int64_t> pptr(nn + 1, 0);
  for (size_t e = 0; e < node.size(); ++e) ++pptr[node[e] + 1];
  for (int64_t k = 0; k < nn; ++k) pptr[k + 1] += pptr[k];
  // edge flows of each panel's dipole charges c on its stencil (row by of q
  // nodes): x flows carry every row's charges towards its first node,
  // px[by][bx] = sum_{b > bx} c[by][b]; the row totals r[by] then go down the
  // first column, py[by][0] = sum_{b > by} r[b].  c = div p holds exactly
  // because each panel's charges sum to zero.
  std::vector<double> PX((size_t)nb * S, 0.0), PY((size_t)nb * S, 0.0);
  for (int64_t j = 0; j < nb; ++j) {
    const double* c = &PD[(size_t)j * S];
    double rt[4] = {0.0, 0.0, 0.0, 0.0};
    for (int by = 0; by < q; ++by) {
      double acc = 0.0;
      for (int bx = q - 1; bx >= 1; --bx) {
        acc += c[by * q + bx];
        PX[(size_t)j * S + by * q + bx - 1] = acc;
      }
      rt[by] = acc + c[by * q];
    }
    double acc = 0.0;
    for (int by = q - 1; by >= 1; --by) {
      acc += rt[by];
      PY[(size_t)j * S + (by - 1) * q] = acc;
    }
  }
  std::vector<int32_t> pj(node.size());
  std::vector<double> pws(node.size()), pwd(node.size()), pwx(node.size()), pwy(node.size());
  {
    std::vector<int64_t> fill(pptr.begin(), pptr.end() - 1);
    for (int64_t j = 0; j < nb; ++j)
      for (int s = 0; s < S; ++s) {
        const size_t e = (size_t)j * S + s;
        const int64_t at = fill[node[e]]++;
        pj[at] = (int32_t)j;
        pws[at] = PS[e];
        pwd[at] = PD[e];
        pwx[at] = PX[e];
        pwy[at] = PY[e];
      }
  }
  // near pairs and their precorrections.  Grid kernel between stencil nodes
  // from the library's table values (the inner plan's own entries)
  const int E = R + order + 1;
  const int TW = 2 * E + 1;
  std::vector<double> Ut((size_t)TW * TW);
  for (int dy = -E; dy <= E; ++dy)
    for (int dx = -E; dx <= E; ++dx) Ut[(size_t)(dy + E) * TW + (dx + E)] = kernel2d_point(0, dx, dy, h);
  std::unordered_map<int64_t, std::vector<int32_t>> bucket;
  auto akey = [](int32_t ax, int32_t ay) { return ((int64_t)(ay + 8) << 32) | (uint32_t)(ax + 8); };
  for (int64_t j = 0; j < nb; ++j) bucket[akey(anc[2 * j], anc[2 * j + 1])].push_back((int32_t)j);
  f.h_nptr.assign(nb + 1, 0);
  std::vector<double> gi(S);
  for (int64_t i = 0; i < nb; ++i) {
    const Panel& Pi = pan[i];
    const int32_t ax = anc[2 * i], ay = anc[2 * i + 1];
    std::vector<int32_t> cand;
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        auto it = bucket.find(akey(ax + dx, ay + dy));
        if (it != bucket.end()) cand.insert(cand.end(), it->second.begin(), it->second.end());
      }
    std::sort(cand.begin(), cand.end());
    for (int32_t j : cand) {
      double es, ed;
      exact_pair(pan[j], Pi.mx, Pi.my, &es, &ed);
      // grid-mediated value: sum_s W_is sum_t U(node_s - node_t) (PS | PD)_jt
      const int ox = ax - anc[2 * j], oy = ay - anc[2 * j + 1];
      double gs = 0.0, gd = 0.0;
      for (int t = 0; t < S; ++t) {
        const int tx = t % q, ty = t / q;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) {
          const int sx = s % q, sy = s / q;
          acc += W[(size_t)i * S + s] * Ut[(size_t)(oy + sy - ty + E) * TW + (ox + sx - tx + E)];
        }
        gs += acc * PS[(size_t)j * S + t];
        gd += acc * PD[(size_t)j * S + t];
      }
      f.h_nj.push_back(j);
      f.h_eS.push_back(es);
      f.h_eD.push_back(ed);
      f.h_cS.push_back(es - gs);
      f.h_cD.push_back(ed - gd);
    }
    f.h_nptr[i + 1] = (int64_t)f.h_nj.size();
  }
  bem_status rc =
      p->prec != BEM_F32 ? upload_all<double, double>(p, node, W, pptr, pj, pws, pwd, pwx, pwy, cells)
      : f.inner->prec == BEM_F32 ? upload_all<float, float>(p, node, W, pptr, pj, pws, pwd, pwx, pwy, cells)
                                 : upload_all<float, double>(p, node, W, pptr, pj, pws, pwd, pwx, pwy, cells);
  if (rc != BEM_OK) return fail(rc);
  BEM_CUDA_TRY(cudaDeviceSynchronize());
  p->threads = f.inner->threads;
  p->grid = f.inner->grid;
  p->scratch_bytes = f.inner->scratch_bytes + f.bytes;
  p->spectra_bytes = f.inner->spectra_bytes;
  p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return BEM_OK;
}

}  // namespace bemfft
