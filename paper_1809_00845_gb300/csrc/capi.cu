// C ABI entry points (include/bem.h): argument checking, plan construction
// (cell sorting, boundary metadata, operator field lists, spectra) and
// dispatch of applies and solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "bem_internal.h"
#include "fft_reg.cuh"

namespace bemfft {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// bytes of one I/O value (float for BEM_F32, double otherwise); also the
// storage size of one value of the plan's arithmetic type
size_t prec_bytes(const bem_plan_s* p) { return p->prec == BEM_F32 ? sizeof(float) : sizeof(double); }

// v converted to the plan's arithmetic type (io = false) or to its I/O type
// (io = true: the diagonal term, added in FP64 to FP64/FP32 I/O values)
bem_status upload_real(const bem_plan_s* p, const double* v, size_t count, bool io, void** dst) {
  void* d = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&d, count * prec_bytes(p)));
  cudaError_t e;
  if (p->prec == BEM_F32) {
    std::vector<float> f(v, v + count);
    e = cudaMemcpy(d, f.data(), count * sizeof(float), cudaMemcpyHostToDevice);
  } else if (p->prec == BEM_F32X2 && !io) {
    std::vector<f32x2> f(count);
    for (size_t i = 0; i < count; ++i) f[i] = f32x2(v[i]);
    e = cudaMemcpy(d, f.data(), count * sizeof(f32x2), cudaMemcpyHostToDevice);
  } else {
    e = cudaMemcpy(d, v, count * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFree(d);
    set_error(std::string("upload: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  *dst = d;
  return BEM_OK;
}

// The calling thread's current device must be the one the plan was built
// on: every array the plan holds lives there, and its kernels launch there.
bem_status check_device(const bem_plan_s* p, const char* who) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string(who) + ": cudaGetDevice: " + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (dev != p->device) {
    set_error(std::string(who) + ": the plan belongs to device " + std::to_string(p->device) + " but device " +
              std::to_string(dev) + " is current");
    return BEM_ERR_ARG;
  }
  return BEM_OK;
}

// A caller buffer handed to the plan's kernels: device (or managed) memory of
// another device is refused; host memory is left to the caller's contract.
bem_status check_buffer_device(const bem_plan_s* p, const void* ptr, const char* who) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not a CUDA allocation: clear the sticky-free error state
    return BEM_OK;
  }
  if ((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device != p->device) {
    set_error(std::string(who) + ": a buffer lives on device " + std::to_string(a.device) +
              ", the plan on device " + std::to_string(p->device));
    return BEM_ERR_ARG;
  }
  return BEM_OK;
}

// [a, a + bytes) and [b, b + bytes) share at least one byte
bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

static bem_status upload_coef(bem_plan_s* p, Operator& op, const std::vector<double>& v, const void** dst,
                              bool io = false) {
  void* d = nullptr;
  bem_status rc = upload_real(p, v.data(), v.size(), io, &d);
  if (rc != BEM_OK) return rc;
  op.owned.push_back(d);
  *dst = d;
  return BEM_OK;
}

static void free_operator(Operator& op) {
  for (void* d : op.owned) cudaFree(d);
  op.owned.clear();
  for (auto& st : op.sets) free_slot_set(&st);
  op.nf = 0;
  op.diag = nullptr;
}

// Laplace 2D operators.  Spectra: 0 = U, 1 = Q_x, 2 = Q_y.
static bem_status build_ops_2d(bem_plan_s* p) {
  const int64_t nb = p->nb;
  std::vector<double> w(p->h_w), wx(nb), wy(nb);
  for (int64_t j = 0; j < nb; ++j) {
    wx[j] = p->h_w[j] * p->h_normal[2 * j];
    wy[j] = p->h_w[j] * p->h_normal[2 * j + 1];
  }
  bem_status rc;
  if (p->v2) {
    std::vector<double> zero(nb, 0.0);
    std::vector<uint8_t> t0(nb, 0);
    Operator& s = p->op_single;
    s.nf = 1;
    s.f[0] = {nullptr, 0, 0, 0, nullptr, nullptr};
    if ((rc = build_op_v2(p, s, w, zero, t0)) != BEM_OK) return rc;
    Operator& d = p->op_double;
    d.nf = 2;
    d.f[0] = {nullptr, 0, 1, 0, nullptr, nullptr};
    d.f[1] = {nullptr, 0, 2, 0, nullptr, nullptr};
    return build_op_v2(p, d, wx, wy, t0);
  }
  Operator& s = p->op_single;
  s.nf = 1;
  s.f[0] = {nullptr, 0, 0, 0, &p->all_set, nullptr};
  if ((rc = upload_coef(p, s, w, &s.f[0].coef)) != BEM_OK) return rc;
  if ((rc = alloc_field_rho(p, s)) != BEM_OK) return rc;
  Operator& d = p->op_double;
  d.nf = 2;
  d.f[0] = {nullptr, 0, 1, 0, &p->all_set, nullptr};
  d.f[1] = {nullptr, 0, 2, 0, &p->all_set, nullptr};
  if ((rc = upload_coef(p, d, wx, &d.f[0].coef)) != BEM_OK) return rc;
  if ((rc = upload_coef(p, d, wy, &d.f[1].coef)) != BEM_OK) return rc;
  if ((rc = alloc_field_rho(p, d)) != BEM_OK) return rc;
  return BEM_OK;
}

static void free_operator3(Operator3D& op) {
  for (void* d : op.owned) cudaFree(d);
  op.owned.clear();
  op.nf = op.no = 0;
  op.d_fields = nullptr;
  op.d_coup = nullptr;
  op.diag = nullptr;
}

// coefs[f] (sorted order, FP64 on the host), comps[f], coupling no x nf
static bem_status build_op3(bem_plan_s* p, Operator3D& op, const std::vector<std::vector<double>>& coefs,
                            const std::vector<int>& comps, int no, const std::vector<int16_t>& coup) {
  free_operator3(op);
  const int nf = (int)coefs.size();
  std::vector<Field3D> fields(nf);
  for (int f = 0; f < nf; ++f) {
    void* d = nullptr;
    bem_status rc = upload_real(p, coefs[f].data(), coefs[f].size(), false, &d);
    if (rc != BEM_OK) return rc;
    op.owned.push_back(d);
    fields[f] = {d, comps[f]};
  }
  void* df = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&df, nf * sizeof(Field3D)));
  BEM_CUDA_TRY(cudaMemcpy(df, fields.data(), nf * sizeof(Field3D), cudaMemcpyHostToDevice));
  op.owned.push_back(df);
  void* dc = nullptr;
  BEM_CUDA_TRY(cudaMalloc(&dc, coup.size() * sizeof(int16_t)));
  BEM_CUDA_TRY(cudaMemcpy(dc, coup.data(), coup.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  op.owned.push_back(dc);
  op.d_fields = static_cast<Field3D*>(df);
  op.d_coup = static_cast<int16_t*>(dc);
  op.nf = nf;
  op.no = no;
  op.lpc = zpass_lpc(p, nf);
  return BEM_OK;
}

// Leaves out the fields whose coefficients are all zero (for the boundary
// conditions set, no cell feeds them: the sums they would add are zeros);
// coup holds no rows of one entry per field.  At least one field stays.
static void drop_zero_fields(std::vector<std::vector<double>>& cf, std::vector<int>& comps, int no,
                             std::vector<int16_t>& coup) {
  const int nf = (int)cf.size();
  std::vector<int> keep;
  for (int f = 0; f < nf; ++f)
    if (std::any_of(cf[f].begin(), cf[f].end(), [](double v) { return v != 0.0; })) keep.push_back(f);
  if (keep.empty()) keep.push_back(0);
  if ((int)keep.size() == nf) return;
  std::vector<std::vector<double>> cf2;
  std::vector<int> comps2;
  std::vector<int16_t> coup2;
  for (int f : keep) {
    cf2.push_back(std::move(cf[f]));
    comps2.push_back(comps[f]);
  }
  for (int o = 0; o < no; ++o)
    for (int f : keep) coup2.push_back(coup[(size_t)o * nf + f]);
  cf.swap(cf2);
  comps.swap(comps2);
  coup.swap(coup2);
}

// Single and double layer of the 3D kernels.  Laplace: U / (Q_x, Q_y, Q_z)
// (spectra 0, 1..3).  Kelvin: U_ab (fields b, outputs a) and T_ab = sum_c
// G_abc n_c (fields (b, c) with coefficient w n_c, outputs a).
static bem_status build_ops_3d(bem_plan_s* p) {
  const int64_t nb = p->nb;
  const std::vector<double>& w = p->h_w;
  bem_status rc;
  if (p->kernel == BEM_LAPLACE_3D) {
    if ((rc = build_op3(p, p->op3_single, {w}, {0}, 1, {0})) != BEM_OK) return rc;
    std::vector<std::vector<double>> c(3, std::vector<double>(nb));
    for (int a = 0; a < 3; ++a)
      for (int64_t j = 0; j < nb; ++j) c[a][j] = w[j] * p->h_normal[3 * j + a];
    return build_op3(p, p->op3_double, c, {0, 0, 0}, 1, {1, 2, 3});
  }
  {
    std::vector<int16_t> coup(9);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) coup[a * 3 + b] = (int16_t)kelvin_u_index(a, b);
    if ((rc = build_op3(p, p->op3_single, {w, w, w}, {0, 1, 2}, 3, coup)) != BEM_OK) return rc;
  }
  std::vector<std::vector<double>> c;
  std::vector<int> comps;
  for (int b = 0; b < 3; ++b)
    for (int cc = 0; cc < 3; ++cc) {
      std::vector<double> v(nb);
      for (int64_t j = 0; j < nb; ++j) v[j] = w[j] * p->h_normal[3 * j + cc];
      c.push_back(v);
      comps.push_back(b);
    }
  std::vector<int16_t> coup(27);
  for (int a = 0; a < 3; ++a)
    for (int f = 0; f < 9; ++f) coup[a * 9 + f] = (int16_t)(6 + 9 * a + f);  // f = 3b + c
  return build_op3(p, p->op3_double, c, comps, 3, coup);
}

}  // namespace bemfft

using namespace bemfft;

static bem_status plan_impl(bem_plan_t* out, int dim, const int64_t* n, double h, int64_t nb, const int32_t* cell,
                            const double* w, const double* normal, bem_kernel kernel, double nu, double mu,
                            bem_precision prec, uint32_t flags, void* stream) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out || !n || !cell || !w || !normal) {
    set_error("bem_plan: null pointer argument");
    return BEM_ERR_ARG;
  }
  *out = nullptr;
  if (kernel != BEM_LAPLACE_2D && kernel != BEM_LAPLACE_3D && kernel != BEM_KELVIN_3D) {
    set_error("bem_plan: unknown kernel");
    return BEM_ERR_ARG;
  }
  if ((kernel == BEM_LAPLACE_2D) != (dim == 2) || (dim != 2 && dim != 3)) {
    set_error("bem_plan: dimension does not match the kernel");
    return BEM_ERR_ARG;
  }
  if (prec != BEM_F64 && prec != BEM_F32 && prec != BEM_F32X2 && prec != BEM_TC_BF16X3 && prec != BEM_TC_F16X3) {
    set_error("bem_plan: unknown precision");
    return BEM_ERR_ARG;
  }
  if (prec == BEM_F32X2 && dim == 2 && n[0] < 256) {
    set_error("bem_plan: BEM_F32X2 needs n >= 256 in 2D");
    return BEM_ERR_UNSUPPORTED;
  }
  // tensor-core DFT stages: an FP32 plan whose column kernel runs its
  // radix-16 stages as split 16-bit products
  int tc = 0;
  if (prec == BEM_TC_BF16X3 || prec == BEM_TC_F16X3) {
    if (dim != 2 || (n[0] != 1024 && n[0] != 2048 && n[0] != 4096)) {
      set_error("bem_plan: tensor-core precisions need a 2D grid with n = 1024, 2048 or 4096");
      return BEM_ERR_UNSUPPORTED;
    }
    tc = prec == BEM_TC_BF16X3 ? 1 : 2;
    prec = BEM_F32;
  }
  if ((flags & ~(BEM_PLAN_SINGLE_LAYER_ONLY | BEM_PLAN_THREE_PASS)) != 0) {
    set_error("bem_plan: unknown flags");
    return BEM_ERR_ARG;
  }
  if (!(h > 0.0) || !std::isfinite(h) || nb < 1 || nb > (int64_t)1 << 30) {
    set_error("bem_plan: need h > 0 and 1 <= nb <= 2^30");
    return BEM_ERR_ARG;
  }
  for (int a = 0; a < dim; ++a)
    if (n[a] < 1) {
      set_error("bem_plan: grid size must be positive");
      return BEM_ERR_ARG;
    }
  for (int a = 1; a < dim; ++a)
    if (n[a] != n[0]) {
      set_error("bem_plan: unequal grid sizes per axis are not supported");
      return BEM_ERR_UNSUPPORTED;
    }
  const int64_t nn = n[0];
  if ((nn & (nn - 1)) != 0 || nn < 4) {
    set_error("bem_plan: n must be a power of two >= 4");
    return BEM_ERR_UNSUPPORTED;
  }
  if (kernel == BEM_KELVIN_3D && (!(mu > 0.0) || !(nu < 0.5) || !(nu > -1.0))) {
    set_error("bem_plan: need mu > 0 and -1 < nu < 1/2");
    return BEM_ERR_ARG;
  }
  // validate cells, weights, normals
  for (int64_t j = 0; j < nb; ++j) {
    for (int a = 0; a < dim; ++a) {
      const int32_t g = cell[j * dim + a];
      if (g < 0 || g >= nn) {
        set_error("bem_plan: cell index outside the grid");
        return BEM_ERR_ARG;
      }
      if (!std::isfinite(normal[j * dim + a])) {
        set_error("bem_plan: non-finite normal");
        return BEM_ERR_ARG;
      }
    }
    if (!std::isfinite(w[j])) {
      set_error("bem_plan: non-finite weight");
      return BEM_ERR_ARG;
    }
  }
  auto* p = new bem_plan_s();
  p->dim = dim;
  p->ncomp = kernel == BEM_KELVIN_3D ? 3 : 1;
  p->kernel = kernel;
  p->prec = prec;
  p->tc = tc;
  p->single_only = (flags & BEM_PLAN_SINGLE_LAYER_ONLY) != 0;
  // three passes through HBM: FP32 four-step plans without tensor-core stages
  p->p3 = (flags & BEM_PLAN_THREE_PASS) != 0 && prec == BEM_F32 && tc == 0 && dim == 2 && n[0] >= 256;
  p->pc.bs = dim == 2 ? 128 : 64;  // default block-Jacobi block (cells)
  p->n = nn;
  p->N = 2 * nn;
  p->log2N = 0;
  while ((int64_t(1) << p->log2N) < p->N) ++p->log2N;
  p->nb = nb;
  p->h = h;
  p->nu = nu;
  p->mu = mu;
  cudaGetDevice(&p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // sort cells by row (y), then x; reject duplicates
  std::vector<int32_t> perm(nb);
  std::iota(perm.begin(), perm.end(), 0);
  auto key = [&](int32_t j) {
    const int64_t z = dim == 3 ? cell[(int64_t)j * dim + 2] : 0;
    return (z * nn + cell[(int64_t)j * dim + 1]) * nn + cell[(int64_t)j * dim];
  };
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key(a) < key(b); });
  for (int64_t j = 1; j < nb; ++j)
    if (key(perm[j]) == key(perm[j - 1])) {
      set_error("bem_plan: duplicate boundary cell");
      delete p;
      return BEM_ERR_ARG;
    }
  std::vector<int32_t> rowptr(nn + 1, 0), col(nb);
  p->h_w.resize(nb);
  p->h_normal.resize(nb * dim);
  p->h_row.resize(nb);
  p->h_col.resize(nb);
  p->h_cell_user.assign(cell, cell + nb * dim);
  p->h_w_user.assign(w, w + nb);
  p->h_normal_user.assign(normal, normal + nb * dim);
  for (int64_t j = 0; j < nb; ++j) {
    const int32_t u = perm[j];
    rowptr[cell[(int64_t)u * dim + 1] + 1]++;
    col[j] = cell[(int64_t)u * dim];
    p->h_row[j] = cell[(int64_t)u * dim + 1];
    p->h_col[j] = col[j];
    if (dim == 3) p->h_z.push_back(cell[(int64_t)u * dim + 2]);
    p->h_w[j] = w[u];
    for (int a = 0; a < dim; ++a) p->h_normal[j * dim + a] = normal[(int64_t)u * dim + a];
  }
  for (int64_t r = 0; r < nn; ++r) rowptr[r + 1] += rowptr[r];
  p->h_perm = perm;
  p->nlines = nn;

  auto fail = [&](bem_status rc) {
    bem_destroy(p);
    return rc;
  };
#define PLAN_CUDA(expr)                                                          \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));            \
      return fail(_e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA); \
    }                                                                            \
  } while (0)
  PLAN_CUDA(cudaMalloc(&p->d_perm, nb * sizeof(int32_t)));
  PLAN_CUDA(cudaMalloc(&p->d_rowptr, (nn + 1) * sizeof(int32_t)));
  PLAN_CUDA(cudaMalloc(&p->d_col, nb * sizeof(int32_t)));
  PLAN_CUDA(cudaMemcpy(p->d_perm, perm.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice));
  PLAN_CUDA(cudaMemcpy(p->d_rowptr, rowptr.data(), (nn + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  PLAN_CUDA(cudaMemcpy(p->d_col, col.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice));

  // quarter-wave twiddles e^{2 pi i r / N}, FP64 on the host, rounded once
  {
    const int64_t N = p->N;
    const double PI = 3.14159265358979323846;
    if (prec != BEM_F32) {
      std::vector<cplx<double>> q(N / 4);
      for (int64_t r = 0; r < N / 4; ++r) q[r] = {std::cos(2.0 * PI * r / N), std::sin(2.0 * PI * r / N)};
      PLAN_CUDA(cudaMalloc(&p->d_qtab, q.size() * sizeof(q[0])));
      PLAN_CUDA(cudaMemcpy(p->d_qtab, q.data(), q.size() * sizeof(q[0]), cudaMemcpyHostToDevice));
    } else {
      std::vector<cplx<float>> q(N / 4);
      for (int64_t r = 0; r < N / 4; ++r)
        q[r] = {(float)std::cos(2.0 * PI * r / N), (float)std::sin(2.0 * PI * r / N)};
      PLAN_CUDA(cudaMalloc(&p->d_qtab, q.size() * sizeof(q[0])));
      PLAN_CUDA(cudaMemcpy(p->d_qtab, q.data(), q.size() * sizeof(q[0]), cudaMemcpyHostToDevice));
    }
  }
  bem_status rc;
  if (dim == 2) {
    if ((rc = compute_spectra_2d(p, st)) != BEM_OK) return fail(rc);
    if ((rc = setup_apply_2d(p)) != BEM_OK) return fail(rc);
    if ((rc = build_ops_2d(p)) != BEM_OK) return fail(rc);
  } else {
    // line pointers over the sorted cells (line = z*n + y) and packed coordinates
    std::vector<int32_t> lptr(nn * nn + 1, 0);
    std::vector<uint16_t> x3(nb);
    std::vector<uint32_t> yz3(nb);
    for (int64_t j = 0; j < nb; ++j) {
      lptr[(int64_t)p->h_z[j] * nn + p->h_row[j] + 1]++;
      x3[j] = (uint16_t)p->h_col[j];
      yz3[j] = (uint32_t)p->h_row[j] | ((uint32_t)p->h_z[j] << 16);
    }
    for (int64_t l = 0; l < nn * nn; ++l) lptr[l + 1] += lptr[l];
    PLAN_CUDA(cudaMalloc(&p->d_lptr, lptr.size() * sizeof(int32_t)));
    PLAN_CUDA(cudaMalloc(&p->d_x3, nb * sizeof(uint16_t)));
    PLAN_CUDA(cudaMalloc(&p->d_yz3, nb * sizeof(uint32_t)));
    PLAN_CUDA(cudaMemcpy(p->d_lptr, lptr.data(), lptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    PLAN_CUDA(cudaMemcpy(p->d_x3, x3.data(), nb * sizeof(uint16_t), cudaMemcpyHostToDevice));
    PLAN_CUDA(cudaMemcpy(p->d_yz3, yz3.data(), nb * sizeof(uint32_t), cudaMemcpyHostToDevice));
    if ((rc = compute_spectra_3d(p, st)) != BEM_OK) return fail(rc);
    if ((rc = setup_apply_3d(p, kernel == BEM_KELVIN_3D ? 12 : 4)) != BEM_OK) return fail(rc);
    if ((rc = build_ops_3d(p)) != BEM_OK) return fail(rc);
  }
  PLAN_CUDA(cudaStreamSynchronize(st));
#undef PLAN_CUDA
  p->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return BEM_OK;
}

extern "C" {

bem_status bem_plan(bem_plan_t* out, int dim, const int64_t* n, double h, int64_t nb, const int32_t* cell,
                    const double* w, const double* normal, bem_kernel kernel, double nu, double mu,
                    bem_precision prec, uint32_t flags, void* stream) {
  return plan_impl(out, dim, n, h, nb, cell, w, normal, kernel, nu, mu, prec, flags, stream);
}

bem_status bem_plan_panels(bem_plan_t* out, int64_t n, double h, int64_t nb, const double* panels, int order,
                           int near_radius, bem_precision prec, uint32_t flags, void* stream) {
  if (!out || !panels) {
    set_error("bem_plan_panels: null pointer argument");
    return BEM_ERR_ARG;
  }
  *out = nullptr;
  if (flags != 0) {
    set_error("bem_plan_panels: flags must be 0");
    return BEM_ERR_ARG;
  }
  if (prec != BEM_F64 && prec != BEM_F32 && prec != BEM_F32X2 && prec != BEM_TC_BF16X3 && prec != BEM_TC_F16X3) {
    set_error("bem_plan_panels: unknown precision");
    return BEM_ERR_ARG;
  }
  if ((n & (n - 1)) != 0 || n < 4 || n > 4096) {
    set_error("bem_plan_panels: n must be a power of two in [4, 4096]");
    return BEM_ERR_UNSUPPORTED;
  }
  return panel_plan_impl(out, n, h, nb, panels, order, near_radius, prec, static_cast<cudaStream_t>(stream));
}

// BC-split system operator of a 2D four-step plan, A x = S(x m_D) + D(x m_N)
// - c x m_N (Eq. 15 with the BC split), for the mask bc or (complement) its
// complement: per sorted cell a type and two coefficients, type 0
// (Dirichlet): (w, 0) -> fields (U, -); type 1 (Neumann): (w n_x, w n_y) ->
// (Q_x, Q_y); all-Neumann: type 0 with (w n_x, w n_y) -> fields (Q_x, Q_y).
// Fields that no cell feeds are left out (exact: they would add zeros).
static bem_status build_system_v2(bem_plan_s* p, const uint8_t* bc, double c, bool complement, Operator& s) {
  const int64_t nb = p->nb;
  auto neu_of = [&](int64_t i) { return (bc[i] != 0) != complement; };
  int64_t nneu = 0;
  for (int64_t i = 0; i < nb; ++i) nneu += neu_of(i) ? 1 : 0;
  const bool all_d = nneu == 0, all_n = nneu == nb;
  std::vector<double> ca(nb), cb(nb), dg(nb);
  std::vector<uint8_t> ty(nb);
  for (int64_t j = 0; j < nb; ++j) {
    const bool neu = neu_of(p->h_perm[j]);
    ty[j] = neu && !all_n ? 1 : 0;
    ca[j] = neu ? p->h_w[j] * p->h_normal[2 * j] : p->h_w[j];
    cb[j] = neu ? p->h_w[j] * p->h_normal[2 * j + 1] : 0.0;
  }
  for (int64_t i = 0; i < nb; ++i) dg[i] = neu_of(i) ? -c : 0.0;  // user order
  s.nf = all_d ? 1 : (all_n ? 2 : 3);
  s.f[0] = {nullptr, 0, all_n ? 1 : 0, 0, nullptr, nullptr};
  s.f[1] = {nullptr, 0, all_n ? 2 : 1, 0, nullptr, nullptr};
  s.f[2] = {nullptr, 0, 2, 0, nullptr, nullptr};
  bem_status rc;
  if ((rc = build_op_v2(p, s, ca, cb, ty)) != BEM_OK) return rc;
  return upload_coef(p, s, dg, &s.diag, true);
}

bem_status bem_set_bc(bem_plan_t p, const uint8_t* bc, double c) {
  if (!p || !bc) {
    set_error("bem_set_bc: null pointer argument");
    return BEM_ERR_ARG;
  }
  if (!std::isfinite(c)) {
    set_error("bem_set_bc: c must be finite");
    return BEM_ERR_ARG;
  }
  const int64_t nb = p->nb;
  for (int64_t i = 0; i < nb * p->ncomp; ++i)
    if (bc[i] > 1) {
      set_error("bem_set_bc: bc entries must be 0 or 1");
      return BEM_ERR_ARG;
    }
  if (p->pf) return panel_set_bc(p, bc, c);
  if (p->single_only) {
    set_error("bem_set_bc: the plan serves the single layer only (BEM_PLAN_SINGLE_LAYER_ONLY)");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->have_bc && c == p->c && std::equal(p->h_bc.begin(), p->h_bc.end(), bc)) return BEM_OK;
  free_operator(p->op_system);
  free_operator(p->op_comp);
  p->have_comp = false;
  ++p->op_version;
  p->h_bc.assign(bc, bc + nb * p->ncomp);
  p->c = c;
  Operator& s = p->op_system;
  bem_status rc;
  if (p->kernel == BEM_LAPLACE_2D) {
    // A x = S(x m_D) + D(x m_N) - c x m_N   (Eq. 15 with the BC split)
    std::vector<double> aq(nb), ax(nb), ay(nb), dg(nb);
    for (int64_t j = 0; j < nb; ++j) {
      const int32_t u = p->h_perm[j];
      const double mN = bc[u] ? 1.0 : 0.0, mD = 1.0 - mN;
      aq[j] = p->h_w[j] * mD;
      ax[j] = p->h_w[j] * p->h_normal[2 * j] * mN;
      ay[j] = p->h_w[j] * p->h_normal[2 * j + 1] * mN;
    }
    for (int64_t i = 0; i < nb; ++i) dg[i] = bc[i] ? -c : 0.0;  // user order
    // fields that no cell feeds are left out (exact: they would add zeros):
    // all-Dirichlet data needs U alone, all-Neumann data Q_x and Q_y alone
    int64_t nneu = 0;
    for (int64_t i = 0; i < nb; ++i) nneu += bc[i] ? 1 : 0;
    const bool all_d = nneu == 0, all_n = nneu == nb;
    if (p->v2) {
      if ((rc = build_system_v2(p, bc, c, false, s)) != BEM_OK) return rc;
      p->have_bc = true;
      p->pc.valid = false;
      return BEM_OK;
    }
    std::vector<uint8_t> memD(nb), memN(nb);
    for (int64_t j = 0; j < nb; ++j) {
      memN[j] = bc[p->h_perm[j]] ? 1 : 0;
      memD[j] = 1 - memN[j];
    }
    if ((rc = build_slot_set(p, memD, &s.sets[0])) != BEM_OK) return rc;
    if ((rc = build_slot_set(p, memN, &s.sets[1])) != BEM_OK) return rc;
    s.nf = 0;
    if (!all_n) {
      s.f[s.nf] = {nullptr, 0, 0, 0, &s.sets[0], nullptr};
      if ((rc = upload_coef(p, s, aq, &s.f[s.nf++].coef)) != BEM_OK) return rc;
    }
    if (!all_d) {
      s.f[s.nf] = {nullptr, 0, 1, 0, &s.sets[1], nullptr};
      if ((rc = upload_coef(p, s, ax, &s.f[s.nf++].coef)) != BEM_OK) return rc;
      s.f[s.nf] = {nullptr, 0, 2, 0, &s.sets[1], nullptr};
      if ((rc = upload_coef(p, s, ay, &s.f[s.nf++].coef)) != BEM_OK) return rc;
    }
    if ((rc = upload_coef(p, s, dg, &s.diag, true)) != BEM_OK) return rc;
    if ((rc = alloc_field_rho(p, s)) != BEM_OK) return rc;
  } else if (p->kernel == BEM_LAPLACE_3D) {
    // A x = S(x m_D) + D(x m_N) - c x m_N: fields U (w m_D), Q_a (w n_a m_N)
    std::vector<std::vector<double>> cf(4, std::vector<double>(nb));
    std::vector<double> dg(nb);
    for (int64_t j = 0; j < nb; ++j) {
      const double mN = bc[p->h_perm[j]] ? 1.0 : 0.0;
      cf[0][j] = p->h_w[j] * (1.0 - mN);
      for (int a = 0; a < 3; ++a) cf[1 + a][j] = p->h_w[j] * p->h_normal[3 * j + a] * mN;
    }
    for (int64_t i = 0; i < nb; ++i) dg[i] = bc[i] ? -c : 0.0;
    std::vector<int> comps = {0, 0, 0, 0};
    std::vector<int16_t> coup = {0, 1, 2, 3};
    drop_zero_fields(cf, comps, 1, coup);
    if ((rc = build_op3(p, p->op3_system, cf, comps, 1, coup)) != BEM_OK) return rc;
    if ((rc = upload_coef(p, s, dg, &s.diag, true)) != BEM_OK) return rc;
    p->op3_system.diag = s.diag;
  } else {
    // Navier (Eq. 8): A x = U(x m_D) - T(x m_N) - c x m_N per component:
    // fields b (w m_D,b) -> U_ab and fields (b, c) (-w n_c m_N,b) -> G_abc
    std::vector<std::vector<double>> cf;
    std::vector<int> comps;
    for (int b = 0; b < 3; ++b) {
      std::vector<double> v(nb);
      for (int64_t j = 0; j < nb; ++j) v[j] = bc[(int64_t)p->h_perm[j] * 3 + b] ? 0.0 : p->h_w[j];
      cf.push_back(v);
      comps.push_back(b);
    }
    for (int b = 0; b < 3; ++b)
      for (int cc = 0; cc < 3; ++cc) {
        std::vector<double> v(nb);
        for (int64_t j = 0; j < nb; ++j)
          v[j] = bc[(int64_t)p->h_perm[j] * 3 + b] ? -p->h_w[j] * p->h_normal[3 * j + cc] : 0.0;
        cf.push_back(v);
        comps.push_back(b);
      }
    std::vector<int16_t> coup(3 * 12);
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) coup[a * 12 + b] = (int16_t)kelvin_u_index(a, b);
      for (int f = 0; f < 9; ++f) coup[a * 12 + 3 + f] = (int16_t)(6 + 9 * a + f);
    }
    std::vector<double> dg(nb * 3);
    for (int64_t i = 0; i < nb * 3; ++i) dg[i] = bc[i] ? -c : 0.0;
    drop_zero_fields(cf, comps, 3, coup);
    if ((rc = build_op3(p, p->op3_system, cf, comps, 3, coup)) != BEM_OK) return rc;
    if ((rc = upload_coef(p, s, dg, &s.diag, true)) != BEM_OK) return rc;
    p->op3_system.diag = s.diag;
  }
  p->have_bc = true;
  p->pc.valid = false;
  return BEM_OK;
}

bem_status bem_set_preconditioner(bem_plan_t p, int kind, int block_size) {
  if (!p) {
    set_error("bem_set_preconditioner: null plan");
    return BEM_ERR_ARG;
  }
  if (kind < 0 || kind > 1 || (kind == 1 && (block_size < 1 || block_size * p->ncomp > 1024))) {
    set_error("bem_set_preconditioner: kind 0 or 1, 1 <= block_size*ncomp <= 1024");
    return BEM_ERR_ARG;
  }
  p->pc.kind = kind;
  if (kind == 1) p->pc.bs = block_size;
  p->pc.valid = false;
  ++p->pc_version;
  return BEM_OK;
}

bem_status bem_apply(bem_plan_t p, bem_layer layer, const void* in_dev, void* out_dev, int nbatch, void* stream) {
  if (!p || !in_dev || !out_dev) {
    set_error("bem_apply: null pointer argument");
    return BEM_ERR_ARG;
  }
  if (nbatch < 1) {
    set_error("bem_apply: nbatch must be >= 1");
    return BEM_ERR_ARG;
  }
  const size_t vec = (size_t)p->nb * p->ncomp * prec_bytes(p);
  if (ranges_overlap(in_dev, out_dev, vec * (size_t)nbatch)) {
    set_error("bem_apply: input and output must not overlap");
    return BEM_ERR_ARG;
  }
  bem_status rc;
  if ((rc = check_device(p, "bem_apply")) != BEM_OK) return rc;
  if ((rc = check_buffer_device(p, in_dev, "bem_apply")) != BEM_OK) return rc;
  if ((rc = check_buffer_device(p, out_dev, "bem_apply")) != BEM_OK) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned char* in = static_cast<const unsigned char*>(in_dev);
  unsigned char* out = static_cast<unsigned char*>(out_dev);
  // the vectors one after another on the stream: every apply reuses the plan's
  // scratch, so they must not run concurrently
  for (int r = 0; r < nbatch; ++r)
    if ((rc = apply_operator(p, layer, in + (size_t)r * vec, out + (size_t)r * vec, st)) != BEM_OK) return rc;
  return BEM_OK;
}

bem_status bem_apply_host(bem_plan_t p, bem_layer layer, const void* in_host, void* out_host, void* stream) {
  if (!p || !in_host || !out_host) {
    set_error("bem_apply_host: null pointer argument");
    return BEM_ERR_ARG;
  }
  bem_status rc = check_device(p, "bem_apply_host");
  if (rc != BEM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)p->nb * p->ncomp * prec_bytes(p);
  if (!p->d_tin) {
    BEM_CUDA_TRY(cudaMalloc(&p->d_tin, bytes));
    BEM_CUDA_TRY(cudaMalloc(&p->d_tout, bytes));
  }
  BEM_CUDA_TRY(cudaMemcpyAsync(p->d_tin, in_host, bytes, cudaMemcpyHostToDevice, st));
  rc = apply_operator(p, layer, p->d_tin, p->d_tout, st);
  if (rc != BEM_OK) return rc;
  BEM_CUDA_TRY(cudaMemcpyAsync(out_host, p->d_tout, bytes, cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  return BEM_OK;
}

bem_status bem_solve(bem_plan_t p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                     int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                     void* stream) {
  if (!p || !bc || !data) {
    set_error("bem_solve: null pointer argument");
    return BEM_ERR_ARG;
  }
  const bem_status dc = check_device(p, "bem_solve");
  if (dc != BEM_OK) return dc;
  const bem_status rc =
      (p->test_flags & BEM_TEST_HOST_ARNOLDI)
          ? solve_gmres(p, bc, data, c, tol, max_iter, restart, x0, u_out, q_out, info, static_cast<cudaStream_t>(stream))
          : solve_graph(p, bc, data, c, tol, max_iter, restart, x0, u_out, q_out, info, static_cast<cudaStream_t>(stream));
  const bem_status ds = bem_device_status(p, stream);
  return ds != BEM_OK ? ds : rc;
}

bem_status bem_enable_refinement(bem_plan_t p, int enable) {
  if (!p) {
    set_error("bem_enable_refinement: null plan");
    return BEM_ERR_ARG;
  }
  if (!enable || p->prec != BEM_F32) {
    if (p->companion) {
      // the solve graphs of the plan's one-plan batch hold the companion
      if (p->self_batch) bem_batch_destroy(p->self_batch);
      p->self_batch = nullptr;
      bem_destroy(p->companion);
    }
    p->companion = nullptr;
    return BEM_OK;
  }
  if (p->companion) return BEM_OK;
  if (p->self_batch) bem_batch_destroy(p->self_batch);
  p->self_batch = nullptr;
  const int64_t n[3] = {p->n, p->n, p->n};
  bem_plan_t c = nullptr;
  if (p->pf) {
    const PanelOp& f = *p->pf;
    bem_status rc = panel_plan_impl(&c, p->n, p->h, p->nb, f.h_panels.data(), f.order, f.R,
                                    p->n >= 256 ? BEM_F32X2 : BEM_F64, nullptr);
    if (rc != BEM_OK) return rc;
    c->pc.kind = 0;
    p->companion = c;
    return BEM_OK;
  }
  bem_status rc = plan_impl(&c, p->dim, n, p->h, p->nb, p->h_cell_user.data(), p->h_w_user.data(),
                            p->h_normal_user.data(), (bem_kernel)p->kernel, p->nu, p->mu,
                            p->dim == 3 || p->n >= 256 ? BEM_F32X2 : BEM_F64, 0, nullptr);
  if (rc != BEM_OK) return rc;
  c->pc.kind = 0;
  p->companion = c;
  return BEM_OK;
}

bem_status bem_get_info(bem_plan_t p, bem_plan_info* info) {
  if (!p || !info) {
    set_error("bem_get_info: null pointer argument");
    return BEM_ERR_ARG;
  }
  info->dim = p->dim;
  info->ncomp = p->ncomp;
  info->n = p->n;
  info->N = p->N;
  info->nb = p->nb;
  info->precision = p->pf ? p->pf->public_prec : (p->tc == 1 ? BEM_TC_BF16X3 : (p->tc == 2 ? BEM_TC_F16X3 : p->prec));
  info->grid_ctas = p->grid;
  info->threads_per_cta = p->threads;
  info->scratch_bytes = p->scratch_bytes;
  info->spectra_bytes = p->spectra_bytes;
  info->plan_seconds = p->plan_seconds;
  info->grid_nodes = p->pf ? p->pf->nnodes : p->nb;
  return BEM_OK;
}

bem_status bem_set_kernel_timing(bem_plan_t p, int enable) {
  if (!p) {
    set_error("bem_set_kernel_timing: null plan");
    return BEM_ERR_ARG;
  }
  p->timing = enable != 0;
  p->ev_used = 0;
  p->timed_ms = 0;
  p->timed_launches = 0;
  if (p->pf) return bem_set_kernel_timing(p->pf->inner, enable);
  return BEM_OK;
}

bem_status bem_kernel_time(bem_plan_t p, double* total_ms, int64_t* launches) {
  if (!p || !total_ms || !launches) {
    set_error("bem_kernel_time: null pointer argument");
    return BEM_ERR_ARG;
  }
  if (p->pf) return bem_kernel_time(p->pf->inner, total_ms, launches);
  for (int i = 0; i + 1 < p->ev_used; i += 2) {
    BEM_CUDA_TRY(cudaEventSynchronize(p->ev_pool[i + 1]));
    float ms = 0.f;
    BEM_CUDA_TRY(cudaEventElapsedTime(&ms, p->ev_pool[i], p->ev_pool[i + 1]));
    p->timed_ms += ms;
    p->timed_launches += 1;
  }
  p->ev_used = 0;
  *total_ms = p->timed_ms;
  *launches = p->timed_launches;
  return BEM_OK;
}

bem_status bem_device_status(bem_plan_t p, void* stream) {
  if (!p) {
    set_error("bem_device_status: null plan");
    return BEM_ERR_ARG;
  }
  if (p->pf) return bem_device_status(p->pf->inner, stream);
  if (!p->d_status) return BEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  BEM_CUDA_TRY(cudaMemcpyAsync(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  if (h == 0) return BEM_OK;
  BEM_CUDA_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int), st));
  BEM_CUDA_TRY(cudaStreamSynchronize(st));
  set_error("a tensor-core column kernel gave up waiting for its products; outputs since the last check are invalid");
  return BEM_ERR_TIMEOUT;
}

bem_status bem_set_test_flags(bem_plan_t p, uint32_t flags) {
  if (!p || (flags & ~(BEM_TEST_WAIT_RUNS_OUT | BEM_TEST_HOST_ARNOLDI)) != 0) {
    set_error("bem_set_test_flags: null plan or unknown flags");
    return BEM_ERR_ARG;
  }
  p->test_flags = flags;
  if (p->pf) p->pf->inner->test_flags = flags;
  return BEM_OK;
}

int bem_launches_per_apply(bem_plan_t p, bem_layer layer) {
  if (!p) return -1;
  // project, node plan (prep, column kernel, reduction), interpolate; the
  // edge-flow form writes the node plan's densities in the projection
  if (p->pf) return (p->pf->edge && layer != BEM_SINGLE) ? 4 : 2 + bem_launches_per_apply(p->pf->inner, BEM_SINGLE);
  if (p->dim == 3) return 6;  // prep, x-DFT, y pass, z pass, inverse y pass, gather
  return 3;                   // prep (weighted densities), fused column kernel, reduction
}

bem_status bem_destroy(bem_plan_t p) {
  if (!p) return BEM_OK;
  if (p->self_batch) bem_batch_destroy(p->self_batch);
  if (p->companion) bem_destroy(p->companion);
  panel_destroy(p);
  cudaFree(p->d_perm);
  cudaFree(p->d_rowptr);
  cudaFree(p->d_col);
  cudaFree(p->d_line);
  cudaFree(p->d_qtab);
  for (auto& s : p->spectra) cudaFree(s.data);
  free_operator(p->op_single);
  free_operator(p->op_double);
  free_operator(p->op_system);
  free_operator(p->op_comp);
  free_slot_set(&p->all_set);
  cudaFree(p->d_tinfo);
  cudaFree(p->d_perm_il);
  cudaFree(p->d_chunk);
  cudaFree(p->d_val);
  cudaFree(p->d_val2);
  cudaFree(p->d_p3X);
  cudaFree(p->d_p3Y);
  cudaFree(p->d_p3part);
  cudaFree(p->d_p3cell);
  cudaFree(p->d_p3pos);
  cudaFree(p->d_twc);
  cudaFree(p->d_fstab);
  cudaFree(p->d_tcmat);
  cudaFree(p->d_status);
  free_operator3(p->op3_single);
  free_operator3(p->op3_double);
  free_operator3(p->op3_system);
  cudaFree(p->d_lptr);
  cudaFree(p->d_x3);
  cudaFree(p->d_yz3);
  cudaFree(p->d_tw2);
  cudaFree(p->d_ptab3);
  cudaFree(p->d_val3);
  cudaFree(p->d_X3);
  cudaFree(p->d_B3);
  for (auto& sp : p->h_specs3) cudaFree(const_cast<void*>(sp.data));
  cudaFree(p->d_specs3);
  cudaFree(p->pc.d_inv);
  cudaFree(p->d_rho);
  cudaFree(p->d_partial);
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  cudaFree(p->d_V);
  cudaFree(p->d_vec);
  cudaFree(p->d_small);
  cudaFree(p->d_tin);
  cudaFree(p->d_tout);
  delete p;
  return BEM_OK;
}

const char* bem_status_string(bem_status s) {
  switch (s) {
    case BEM_OK: return "ok";
    case BEM_ERR_ARG: return "invalid argument";
    case BEM_ERR_CUDA: return "CUDA error";
    case BEM_ERR_OOM: return "out of device memory";
    case BEM_ERR_NOT_CONVERGED: return "not converged";
    case BEM_ERR_BREAKDOWN: return "GMRES breakdown";
    case BEM_ERR_NONFINITE: return "non-finite value";
    case BEM_ERR_TIMEOUT: return "device wait timed out";
    case BEM_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* bem_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace bemfft {

bool has_complement(const bem_plan_s* p) {
  if (!p->have_bc || p->pf || p->dim != 2 || !p->v2 || p->kernel != BEM_LAPLACE_2D) return false;
  bool d = false, n = false;
  for (uint8_t b : p->h_bc) (b ? n : d) = true;
  return d && n;
}

bem_status apply_complement(bem_plan_s* p, const void* in, void* out, cudaStream_t st) {
  if (!has_complement(p)) {
    set_error("apply_complement: needs a 2D four-step plan with both condition types set");
    return BEM_ERR_UNSUPPORTED;
  }
  if (!p->have_comp) {
    bem_status rc = build_system_v2(p, p->h_bc.data(), p->c, true, p->op_comp);
    if (rc != BEM_OK) {
      free_operator(p->op_comp);
      return rc;
    }
    p->have_comp = true;
  }
  return launch_apply_2d(p, p->op_comp, in, out, st);
}

bem_status apply_operator(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st) {
  if (p->pf) return launch_apply_panels(p, layer, in, out, st);
  if (p->single_only && layer != BEM_SINGLE) {
    set_error("bem_apply: the plan serves the single layer only (BEM_PLAN_SINGLE_LAYER_ONLY)");
    return BEM_ERR_UNSUPPORTED;
  }
  if (p->dim == 3) {
    const Operator3D* op3 = nullptr;
    if (layer == BEM_SINGLE) op3 = &p->op3_single;
    else if (layer == BEM_DOUBLE) op3 = &p->op3_double;
    else if (layer == BEM_SYSTEM) {
      if (!p->have_bc) {
        set_error("bem_apply: BEM_SYSTEM needs bem_set_bc first");
        return BEM_ERR_ARG;
      }
      op3 = &p->op3_system;
    } else {
      set_error("bem_apply: unknown layer");
      return BEM_ERR_ARG;
    }
    return launch_apply_3d(p, *op3, in, out, p->d_val3, p->d_X3, p->d_B3, st);
  }
  const Operator* op = nullptr;
  if (layer == BEM_SINGLE) op = &p->op_single;
  else if (layer == BEM_DOUBLE) op = &p->op_double;
  else if (layer == BEM_SYSTEM) {
    if (!p->have_bc) {
      set_error("bem_apply: BEM_SYSTEM needs bem_set_bc first");
      return BEM_ERR_ARG;
    }
    op = &p->op_system;
  } else {
    set_error("bem_apply: unknown layer");
    return BEM_ERR_ARG;
  }
  return launch_apply_2d(p, *op, in, out, st);
}

}  // namespace bemfft
