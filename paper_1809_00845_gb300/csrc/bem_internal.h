// Internal declarations shared by the translation units of libbem_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bem.h"
#include "ff.cuh"

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

// Warp-coalesced "slot" layout of a set of boundary cells for the fused
// column kernel.  Thread t of the CTA owns grid rows t + m*TT (m < H).  Lanes
// are grouped by G (32, or TT when TT < 32); for group g and row slot m all
// lanes loop over cnt[g*H + m] cells (the maximum over the group, padding
// entries have x = 0, cidx = -1 and a zero density), so every load of the
// loop is one contiguous G-element access.  Element (g, m, i, lane) sits at
// (off[g*H + m] + i) * G + lane.
struct SlotSet {
  int ngroups = 0, G = 0, H = 0;
  int64_t nelem = 0;            // total elements (slot rows * G)
  int32_t* d_cnt = nullptr;     // ngroups * H
  int32_t* d_off = nullptr;     // ngroups * H
  uint16_t* d_x = nullptr;      // nelem: x grid index (0 on padding)
  int32_t* d_cidx = nullptr;    // nelem: sorted cell index, -1 on padding
  std::vector<int32_t> h_cidx;  // host copy of d_cidx
};

// One scattered field of an operator: rho_f[e] = coef_f[cidx[e]] * in[perm[cidx[e]]*ncomp + comp_f]
// over the slot layout of its cell set, transformed, multiplied by the
// compressed spectrum spec_f (parity flags) and accumulated into output out_f.
struct FieldDesc {
  const void* coef;   // nb, sorted order, plan precision
  int comp;           // input component
  int spec;           // index into plan spectra
  int out;            // output component
  const SlotSet* set = nullptr;
  void* rho = nullptr;  // set->nelem values, plan precision (operator-owned scratch)
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
  std::vector<void*> owned;    // device arrays owned by this operator
  SlotSet sets[2];             // operator-specific cell sets (BC-split operator)
  // four-step column kernel (N >= 512): per sorted cell a packed word
  // x | row << 16 | type << 31 and two coefficients; the density pair of cell
  // j is (coefA[j], coefB[j]) * in[perm[j]], routed to fields (0, 1) for
  // type 0 and (1, 2) for type 1.
  const uint32_t* meta = nullptr;
  const void* coefA = nullptr;
  const void* coefB = nullptr;
};

// 3D operators: field f scatters coef_f[j] * in[perm[j]*ncomp + comp]; output
// o sums K_{coup[o][f]} * field f over the fields (coup < 0: no coupling).
struct Field3D {
  const void* coef;  // nb, sorted order, plan precision
  int comp;
};
struct Spec3D {
  const void* data;  // (n+1)^3 reals, [kx][ky][kz]; K^ = i^q * S
  int q;             // number of axes in which the kernel is odd
  int oddy, oddz;    // fold signs for ky, kz > n
};
struct Operator3D {
  int nf = 0, no = 0, lpc = 1;
  Field3D* d_fields = nullptr;  // nf (device)
  int16_t* d_coup = nullptr;    // no * nf (device)
  const void* diag = nullptr;   // nb*ncomp (caller order) or null
  std::vector<void*> owned;
};

// Block-Jacobi near-field preconditioner: dense inverses of the operator's
// diagonal blocks of consecutive cells (caller order).
struct BlockPrecond {
  int kind = 1;     // 0 none, 1 block Jacobi
  int bs = 64;      // block size (cells)
  int nblocks = 0;
  double* d_inv = nullptr;  // nblocks * (bs*ncomp)^2, row-major per block
  bool valid = false;
};

// Accuracy mode (panels.cu): the unknowns live on flat boundary panels; a
// panel's source and dipole are projected onto a stencil of grid nodes, the
// grid convolution of an inner node plan carries the far field, the
// potential is interpolated back to the panel midpoints, and near pairs get
// their exact panel integrals (precorrection).
struct PanelOp {
  int order = 3, R = 3, S = 16;       // stencil order, near radius (anchor cells), nodes per stencil
  int64_t nnodes = 0;
  bem_plan_s* inner = nullptr;        // paper-form plan over the active nodes (w = 1)
  int public_prec = 0;                // precision requested by the caller
  std::vector<double> h_panels;       // nb * 4 (A.x, A.y, B.x, B.y)
  std::vector<double> h_delta;        // nb: Gauss row-sum term of the double layer
  // near pairs, CSR by target: exact panel integrals (preconditioner) and
  // precorrections exact - grid-mediated
  std::vector<int64_t> h_nptr;
  std::vector<int32_t> h_nj;
  std::vector<double> h_eS, h_eD, h_cS, h_cD;
  // device (T = the plan's I/O type)
  int32_t* d_node = nullptr;          // nb * S inner node indices of each midpoint's stencil
  void* d_W = nullptr;                // nb * S interpolation weights
  int64_t* d_pptr = nullptr;          // nnodes + 1: projection CSR by node
  int32_t* d_pj = nullptr;
  double* d_pws = nullptr;            // single-layer moments (FP64)
  double* d_pwd = nullptr;            // dipole moments (FP64)
  double* d_pwx = nullptr;            // edge-flow form: the dipole moments as x-edge flows (FP64)
  double* d_pwy = nullptr;            // ... and as y-edge flows
  bool edge = false;                  // double layer through the inner plan's edge-flow form
  int64_t* d_nptr = nullptr;          // nb + 1: near CSR by target
  int32_t* d_nj = nullptr;
  void* d_cS = nullptr;
  void* d_cD = nullptr;
  void* d_delta = nullptr;            // nb
  uint8_t* d_bc = nullptr;            // nb
  void* d_rho = nullptr;              // nnodes node charges (inner plan precision)
  void* d_phi = nullptr;              // nnodes node potentials (inner plan precision)
  size_t bytes = 0;
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
  bemfft::SlotSet all_set;      // every cell (gather layout, single/double layer fields)
  std::vector<bemfft::Spectrum> spectra;
  std::vector<double> h_w, h_normal;  // host copies in sorted order
  std::vector<int32_t> h_perm;
  std::vector<int32_t> h_row, h_col;  // sorted order: grid row (y) and column (x)
  std::vector<int32_t> h_cell_user;   // caller order copies of the geometry
  std::vector<double> h_w_user, h_normal_user;
  bemfft::Operator op_single, op_double, op_system;
  bool have_bc = false;
  // the BC-split operator of the complementary mask (built on first use by
  // apply_complement; dropped when the conditions change)
  bemfft::Operator op_comp;
  bool have_comp = false;
  std::vector<uint8_t> h_bc;
  bemfft::BlockPrecond pc;
  // four-step column kernel: per-thread equal cell ranges
  bool v2 = false;
  bool v2_carry = false;              // some grid row is split between threads
  std::vector<uint32_t> h_cellflag;   // sorted order: 1 = last cell of its row in the chunk, 2 = carried
  int32_t* d_tinfo = nullptr;   // threads: row mask | continuing threads << 8
  int64_t v2_npos = 0;          // interleaved cell positions (cells rounded up to a multiple of threads)
  std::vector<int64_t> h_pos;   // sorted cell -> interleaved position
  int32_t* d_perm_il = nullptr; // interleaved position -> caller index (-1: padding)
  int32_t* d_chunk = nullptr;   // threads + 1
  void* d_val = nullptr;        // nb density pairs (scratch)
  void* d_twc = nullptr;        // grid * npos cached sparse twiddles (scratch)
  int cell_batch = 2;           // cells per load batch of the fused 2D cell walks (2 or 4; bem_tune_shapes)
  int zpass_lines = 0;          // 3D z-pass lines per CTA (0: the default rule; bem_tune_shapes)
  void* d_fstab = nullptr;      // twiddle tables of the four-step kernel
  int tc = 0;                   // tensor-core DFT stages: 0 none, 1 BF16 hi + lo, 2 FP16 hi + lo
  void* d_tcmat = nullptr;      // their B matrices (hi, lo; 8 KB)
  int* d_status = nullptr;      // device status word (bit 0: a bounded wait gave up)
  uint32_t test_flags = 0;      // bem_set_test_flags (bounded-wait tests)
  // edge-flow form of the node convolution (accuracy mode): third density per
  // position (plan arithmetic type), launch shape of the edge-flow column kernel
  // three-pass form (FP32 four-step plans with BEM_PLAN_THREE_PASS)
  bool p3 = false;
  void* d_p3X = nullptr;        // fields' x-DFT rows, nf * (n+1) * n complex
  void* d_p3Y = nullptr;        // inverse-transformed columns, (n+1) * n complex
  void* d_p3part = nullptr;     // gather partials per chunk of columns
  void* d_p3cell = nullptr;     // per sorted cell: x and three field values
  int32_t* d_p3pos = nullptr;   // sorted cell -> interleaved position
  size_t p3_smem = 0;
  int p3_grid = 0, p3_nchunk = 0;
  void* d_val2 = nullptr;
  size_t edge_smem = 0;
  int edge_acc_rows = 0, edge_grid = 0;
  // 3D path
  int32_t* d_lptr = nullptr;    // n*n + 1 line pointers over sorted cells (line = z*n + y)
  uint16_t* d_x3 = nullptr;     // x per sorted cell
  uint32_t* d_yz3 = nullptr;    // y | z << 16 per sorted cell
  void* d_tw2 = nullptr;        // 2-level twiddles (N/64 + 64)
  void* d_ptab3 = nullptr;      // Stockham pass twiddles of the 3D line FFTs
  void* d_val3 = nullptr;       // maxnf * nb
  void* d_X3 = nullptr;         // maxnf * (n+1) * n * n complex
  void* d_B3 = nullptr;         // maxnf * (n+1) * N * n complex
  int maxnf3 = 0;
  bemfft::Spec3D* d_specs3 = nullptr;
  std::vector<bemfft::Spec3D> h_specs3;
  std::vector<int32_t> h_z;     // sorted order z
  bemfft::Operator3D op3_single, op3_double, op3_system;
  // scratch
  void* d_rho = nullptr;       // unused (densities live with the operators)
  void* d_partial = nullptr;   // grid * all_set.nelem * ncomp
  int grid = 0, threads = 0;
  size_t smem_bytes = 0;
  bool acc_in_smem = false;
  int acc_rows = 0;             // four-step kernel: interleaved cell rows accumulated in shared memory
  bool single_only = false;     // BEM_PLAN_SINGLE_LAYER_ONLY: only BEM_SINGLE applies (smaller footprint)
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
  size_t small_len = 0;
  bem_plan_s* companion = nullptr;  // FP64 plan of the same geometry for refinement residuals
  void* d_tin = nullptr;    // plan-precision in/out buffers for the apply
  void* d_tout = nullptr;
  uint64_t op_version = 0;  // bumped whenever bem_set_bc rebuilds the system operator
  uint64_t pc_version = 0;  // bumped whenever the preconditioner changes (captured solve graphs hold it)
  bem_batch_s* self_batch = nullptr;  // one-plan batch that runs bem_solve's Arnoldi steps as graphs
  bemfft::PanelOp* pf = nullptr;  // accuracy mode (bem_plan_panels), else null
};

namespace bemfft {
// Plans of a batch applied by one persistent column-kernel launch (FP32
// four-step plans with the same grid and thread count; apply2d.cu)
struct BatchGroup {
  std::vector<int> members;  // indices into the batch's plans
  std::vector<int> rows;     // per member: CTAs whose column range reaches it (rows of its partial sums)
  void* d_params = nullptr;  // Col2Dv2Params<float>[members]
  int* d_c0 = nullptr;       // per member: the first such CTA
  int grid = 0, threads = 0, nf = 0;
  size_t smem = 0;
};
}  // namespace bemfft

// Batch of plans applied through one CUDA graph (batch.cu); the batched
// GMRES (gmres.cu) keeps its workspace here too.
struct BatchSolveWs;
struct bem_batch_s {
  std::vector<bem_plan_s*> plans;
  std::vector<uint64_t> versions;  // plans' operator versions at capture
  std::vector<size_t> offset;      // count + 1 element offsets into the packed buffers
  size_t total = 0;
  int prec = 0;
  bem_layer layer = BEM_SINGLE;
  int nstreams = 1;
  void* d_in = nullptr;
  void* d_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> side;  // side[0] is the capture stream
  std::vector<cudaEvent_t> events;
  int launches = 0;
  BatchSolveWs* ws = nullptr;
  bem_batch_s* companions = nullptr;  // batch over the plans' refinement companions (solve only)
  std::vector<bemfft::BatchGroup> groups;  // plans applied by one grouped launch per grid size
  std::vector<int> solo;                   // the others, applied one by one
  bool grouped = true;                     // form grouped launches (bem_batch_set_grouping)
};

namespace bemfft {

// spectra.cu
bem_status compute_spectra_2d(bem_plan_s* p, cudaStream_t st);
bem_status compute_spectra_3d(bem_plan_s* p, cudaStream_t st);
// apply3d.cu
bem_status setup_apply_3d(bem_plan_s* p, int maxnf);
int zpass_lpc(const bem_plan_s* p, int nf);
bem_status launch_apply_3d(bem_plan_s* p, const Operator3D& op, const void* in, void* out, void* val, void* X, void* B,
                           cudaStream_t st);
size_t buffers3d_bytes(const bem_plan_s* p, int nf);
// index of a 3D spectrum: Laplace U=0, Q_a=1+a; Kelvin U_ab (a<=b) 0..5, G_abc 6 + 9a + 3b + c
int kelvin_u_index(int a, int b);
// apply2d.cu
bem_status setup_apply_2d(bem_plan_s* p);
bem_status build_slot_set(bem_plan_s* p, const std::vector<uint8_t>& member, SlotSet* s);
void free_slot_set(SlotSet* s);
bem_status alloc_field_rho(bem_plan_s* p, Operator& op);
bem_status build_op_v2(bem_plan_s* p, Operator& op, const std::vector<double>& coefA, const std::vector<double>& coefB,
                       const std::vector<uint8_t>& type);
size_t apply_scratch_bytes(const bem_plan_s* p, const Operator& op);
// grouped batch applies (apply2d.cu)
bool group_eligible(const bem_plan_s* p);
bem_status group_build(BatchGroup& g, const std::vector<bem_plan_s*>& plans, bem_layer layer);
bem_status group_issue(const BatchGroup& g, const std::vector<bem_plan_s*>& plans, bem_layer layer,
                       const void* in, void* out, const std::vector<size_t>& offset, cudaStream_t st);
void group_free(BatchGroup& g);
bem_status launch_apply_2d(bem_plan_s* p, const Operator& op, const void* in, void* out, cudaStream_t st);
// edge-flow form of a node plan (four-step kernel): set-up of its launch
// shape and third density buffer, and one convolution of the densities the
// caller wrote to p->d_val (charge, x-edge flow pairs) and p->d_val2 (y-edge
// flows) at the interleaved positions, in the plan's arithmetic type; result
// in caller order, I/O type (apply2d.cu)
bem_status setup_edge_2d(bem_plan_s* p);
bem_status launch_edge_2d(bem_plan_s* p, void* out, cudaStream_t st);
// Device scratch of one apply: per-field densities (slot layout kernel) or
// density pairs (four-step kernel), and the per-CTA partial sums.
struct ScratchPtrs {
  void* rho[kMaxFields];
  void* val;
  void* partial;
  void* twc = nullptr;  // per-CTA cached sparse twiddles (four-step kernel; optional)
};
void carve_scratch(const bem_plan_s* p, const Operator& op, void* base, ScratchPtrs* sp);
bem_status launch_apply_2d_with(bem_plan_s* p, const Operator& op, const void* in, void* out, const ScratchPtrs& sp,
                                bool timed, cudaStream_t st);
// batch.cu: issue the applies of every plan of the batch from `in` to `out`
// (packed) on the batch's side streams, forked from and joined back into
// `cap`, which is being captured; (re)capture of the batch's own graph
bem_status batch_issue_applies(bem_batch_s* b, const void* in, void* out, cudaStream_t cap);
bem_status batch_capture(bem_batch_s* b);
bem_status batch_refresh(bem_batch_s* b);  // re-capture when a plan's operator changed
void batch_solve_free(bem_batch_s* b);     // gmres.cu
// gmres.cu
bem_status solve_gmres(bem_plan_s* p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                       int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                       cudaStream_t st);
// bem_solve's default path: the same GMRES with every Arnoldi step one CUDA
// graph replay and the Givens rotations on the device (a one-plan batch)
bem_status solve_graph(bem_plan_s* p, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                       int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                       cudaStream_t st);
bem_status apply_operator(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st);
// Right-hand side of the mixed problem in one apply: with data d (u on the
// Dirichlet cells, q on the Neumann cells) the right-hand side c u_D - D u_D -
// S q_N equals -(A' d), A' the BC-split system operator of the complementary
// mask.  has_complement: the plan can do this (2D four-step plans with both
// condition types set); apply_complement writes A' d (plan-precision I/O).
bool has_complement(const bem_plan_s* p);
bem_status apply_complement(bem_plan_s* p, const void* in, void* out, cudaStream_t st);
// argument checks of the entry points (capi.cu)
bem_status check_device(const bem_plan_s* p, const char* who);
bem_status check_buffer_device(const bem_plan_s* p, const void* ptr, const char* who);
bool ranges_overlap(const void* a, const void* b, size_t bytes);
size_t prec_bytes(const bem_plan_s* p);
bem_status upload_real(const bem_plan_s* p, const double* v, size_t count, bool io, void** dst);
// Lets `kern` launch with up to the device's opt-in shared-memory maximum.  The
// limit is a property of the function, shared by every plan, so it is never set
// to one plan's (smaller) need: a plan made later would otherwise lower it below
// what an earlier plan launches with.
template <typename K>
inline cudaError_t allow_optin_smem(K kern) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);  // the limit excludes static shared memory
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}
bem_status build_preconditioner(bem_plan_s* p);
// accuracy mode (panels.cu)
bem_status panel_plan_impl(bem_plan_s** out, int64_t n, double h, int64_t nb, const double* panels, int order,
                           int R, bem_precision prec, cudaStream_t st);
bem_status launch_apply_panels(bem_plan_s* p, bem_layer layer, const void* in, void* out, cudaStream_t st);
bem_status panel_set_bc(bem_plan_s* p, const uint8_t* bc, double c);
void panel_destroy(bem_plan_s* p);
// the system operator's exact entries (block of consecutive panels i0 .. i0+sz)
void panel_block(const bem_plan_s* p, int64_t i0, int sz, double* A);
__host__ __device__ double kernel2d_point(int kind, int dx, int dy, double h);

}  // namespace bemfft
