// Internal declarations shared by the translation units of libbem_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bem.h"

namespace bemfft {

constexpr int kMaxFields = 12;

// Thread-local error message + status helper.
void set_error(const std::string& msg);
#define BEM_CUDA_TRY(expr)                                                                        \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess) {                                                                      \
      ::bemfft::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
      return _e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA;                        \
    }                                                                                             \
  } while (0)

// One scattered field of an operator: rho_f[j] = coef_f[j] * in[perm[j]*ncomp + comp_f],
// transformed, multiplied by the compressed spectrum spec_f (parity flags) and
// accumulated into output component out_f.
struct FieldDesc {
  const void* coef;   // nb, sorted order, plan precision
  int comp;           // input component
  int spec;           // index into plan spectra
  int out;            // output component
};

// Compressed spectrum of one kernel table: K^(k) = i^imag * S(k) with S real,
// stored for k_a in [0, n] (kx-major: S[(kx*(n+1) + ky)(n+1) + kz] in 3D).
struct Spectrum {
  void* data = nullptr;  // plan precision
  int imag = 0;          // 1: spectrum purely imaginary (kernel odd in one axis)
  int odd[3] = {0, 0, 0};  // kernel parity per axis (1 = odd)
};

struct Operator {
  int nf = 0;
  FieldDesc f[kMaxFields];
  const void* diag = nullptr;  // nb*ncomp diagonal term (plan precision) or null
  std::vector<void*> owned;    // coefficient arrays owned by this operator
};

}  // namespace bemfft

struct bem_plan_s {
  int dim = 2, ncomp = 1, kernel = 0, prec = 0, device = 0;
  int64_t n = 0, N = 0, nb = 0;
  int log2N = 0;
  double h = 0, nu = 0.3, mu = 1.0, c = 0.5;
  // sorted cell metadata (sorted by (row) = (gy) in 2D, (gz, gy) lines in 3D)
  int32_t* d_perm = nullptr;    // sorted j -> user index
  int32_t* d_rowptr = nullptr;  // lines+1
  int32_t* d_col = nullptr;     // x grid index per sorted cell
  int32_t* d_line = nullptr;    // line index per sorted cell (3D)
  int64_t nlines = 0;
  void* d_qtab = nullptr;       // quarter twiddle table, plan precision
  std::vector<bemfft::Spectrum> spectra;
  std::vector<double> h_w, h_normal;  // host copies in sorted order
  std::vector<int32_t> h_perm;
  bemfft::Operator op_single, op_double, op_system;
  bool have_bc = false;
  std::vector<uint8_t> h_bc;
  // scratch
  void* d_rho = nullptr;       // kMaxFields * nb
  void* d_partial = nullptr;   // grid * nb * ncomp
  int grid = 0, threads = 0;
  size_t smem_bytes = 0;
  bool acc_in_smem = false;
  size_t scratch_bytes = 0, spectra_bytes = 0;
  double plan_seconds = 0;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  int ev_used = 0;
  double timed_ms = 0;
  int64_t timed_launches = 0;
  // GMRES workspace (FP64)
  int gm_m = 0;
  double* d_V = nullptr;
  double* d_vec = nullptr;  // several nb*ncomp FP64 vectors
  double* d_small = nullptr;
  void* d_tin = nullptr;    // plan-precision in/out buffers for the apply
  void* d_tout = nullptr;
};

namespace bemfft {

// spectra.cu
bem_status compute_spectra_2d(bem_plan_s* p, cudaStream_t st);
// apply2d.cu
bem_status setup_apply_2d(bem_plan_s* p);
bem_status launch_apply_2d(bem_plan_s* p, const Operator& op, const void* in, void* out, cudaStream_t st);
// gmres.cu
bem_status solve_gmres(bem_plan_s* p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                       int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                       cudaStream_t st);
bem_status apply_operator(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st);
size_t prec_bytes(const bem_plan_s* p);

}  // namespace bemfft
