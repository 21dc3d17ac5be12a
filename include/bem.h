/*
 * bem.h — C ABI of the GB300 (sm_103a) FFT-accelerated boundary element
 * operator after Benad, "Acceleration of the Boundary Element Method for
 * arbitrary shapes with the Fast Fourier Transformation" (arXiv:1809.00845).
 *
 * The method (Section 3, Section 4, Eq. 15-16): a boundary integral over a
 * curve (surface) S is a convolution over the grid that encloses S, one
 * dimension higher, once the densities are extended with zeros off S.  Each
 * operator apply therefore
 *   1. scatters the weighted boundary densities onto a zero-padded uniform grid
 *      (u extended with zeros, Fig. 4; q, and u n_a for the double layer),
 *   2. transforms forward (FFT),
 *   3. multiplies by the precomputed spectra of the kernel tables (Eq. 16),
 *   4. transforms back, and
 *   5. reads the result at the boundary cells (Section 4, last paragraph).
 * bem_solve wraps the apply in a Krylov iteration (Section 4 uses conjugate
 * gradients; this library uses restarted GMRES).
 *
 * Discretisation conventions (all calls):
 *   * grid of n cells per axis, spacing h; node of cell g at (g + 1/2) h;
 *   * boundary cell j: grid index g_j (dim int32, axis 0 = x), boundary
 *     measure w_j (length in 2D, area in 3D; the "divide by the discretisation
 *     length" of Section 4 folded into the source weight) and unit outward
 *     normal n_j;
 *   * d_ij = x_gi - x_gj (collocation minus integration point, Eq. 15);
 *   * single layer (S f)_i = sum_j U(d_ij) w_j f_j; double layer
 *     (D u)_i = sum_j sum_a Q_a(d_ij) w_j n_{a,j} u_j with
 *     2D Laplace U = -ln r/(2 pi) (Eq. 3), Q_a = -d_a/(2 pi r^2) (Eq. 15);
 *     3D Laplace U = 1/(4 pi r), Q_a = -d_a/(4 pi r^3);
 *     Kelvin (Eq. 7) U_ab and the traction kernel T_ab (Eq. 8);
 *   * the singular cell (d = 0) carries the kernel's average over the h-cell
 *     ("constant elements", Section 4), odd kernels carry 0;
 *   * BIE row (Eq. 4, Eq. 8): c u = S q + D u (Laplace), c u = U t - T u
 *     (Navier), c = 1/2 unless set otherwise.
 *
 * Errors: every call returns a bem_status; nothing throws or aborts across
 * the ABI.  bem_last_error() returns a thread-local message for the last
 * failing call on the calling thread.  On a CUDA error the plan stays valid
 * only if the CUDA context survived.
 *
 * Threading: a plan may be used by one thread at a time (it owns one set of
 * scratch buffers); use one plan per concurrent stream.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_plan_s* bem_plan_t;

typedef enum {
  BEM_OK = 0,
  BEM_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, duplicate/out-of-grid cell) */
  BEM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  BEM_ERR_OOM = 3,            /* device allocation failed */
  BEM_ERR_NOT_CONVERGED = 4,  /* bem_solve hit max_iter; best iterate written, info filled */
  BEM_ERR_BREAKDOWN = 5,      /* GMRES breakdown before reaching tol */
  BEM_ERR_NONFINITE = 6,      /* NaN/Inf in data or residual */
  BEM_ERR_TIMEOUT = 7,        /* a bounded device-side wait expired */
  BEM_ERR_UNSUPPORTED = 8     /* valid but unsupported configuration (e.g. grid size) */
} bem_status;

typedef enum { BEM_LAPLACE_2D = 0, BEM_LAPLACE_3D = 1, BEM_KELVIN_3D = 2 } bem_kernel;
/* BEM_F64: FP64 arithmetic, double I/O.  BEM_F32: FP32 arithmetic, float I/O.
 * BEM_F32X2: double-float arithmetic (each value a pair of FP32 numbers, a
 * 48-bit significand) on the FP32 pipes, double I/O; about 1e-13 relative
 * accuracy at several times the speed of FP64 on GPUs with reduced FP64
 * throughput.  BEM_F32X2 is available for 2D plans with n >= 256 (the
 * four-step column kernel) and for 3D plans, and returns BEM_ERR_UNSUPPORTED
 * for 2D plans with n < 256.
 * BEM_TC_BF16X3, BEM_TC_F16X3: FP32 I/O and arithmetic except the radix-16
 * DFT stages of the column transforms (Eq. 16), which run on the tensor cores
 * as DFT-matrix products with every FP32 operand split into a 16-bit hi and
 * lo part (BF16, or FP16 with each line scaled by a power of two) and three
 * products accumulated in FP32.  2D plans with n = 1024, 2048 or 4096 only
 * (BEM_ERR_UNSUPPORTED otherwise).  The paper transforms in full precision;
 * these are an added speed/accuracy trade-off, with the error bound stated
 * where they are tested. */
typedef enum {
  BEM_F64 = 0,
  BEM_F32 = 1,
  BEM_F32X2 = 2,
  BEM_TC_BF16X3 = 3,
  BEM_TC_F16X3 = 4
} bem_precision;

/* BEM_SINGLE: S (Laplace) or U (Kelvin).  BEM_DOUBLE: D (Laplace) or T
 * (Kelvin).  BEM_SYSTEM: the boundary-condition-split operator A of the last
 * bem_set_bc call: A x = K1(x m_D) + K2(x m_N) - c x m_N with K1 = S|U,
 * K2 = +D (Laplace, Eq. 15) or -T (Navier, Eq. 8), m_D/m_N the Dirichlet and
 * Neumann masks (per component). */
typedef enum { BEM_SINGLE = 0, BEM_DOUBLE = 1, BEM_SYSTEM = 2 } bem_layer;

typedef struct {
  int iters;                 /* total GMRES iterations (operator applies inside the Krylov loop) */
  int restarts;              /* number of restarts performed */
  double rel_residual;       /* ||b - A x|| / ||b|| recomputed with the plan's own apply (FP64 norms) */
  double rel_residual_est;   /* GMRES (Givens) estimate at exit */
  double seconds;            /* wall time of the solve (host clock) */
  int applies;               /* all operator applies, right-hand side and final check included */
  int refine_steps;          /* outer steps of mixed-precision refinement (0 without it) */
  double rel_residual_fp64;  /* rel_residual when its operator is accurate to FP64 level (an FP64 plan, or the
                                double-float / FP64 companion of a refined solve), else NaN: a plain FP32 or
                                tensor-core solve has no FP64-accurate residual to report */
} bem_solve_info;

typedef struct {
  int dim, ncomp;            /* 2 or 3; 1 (Laplace) or 3 (Kelvin) */
  int64_t n, N, nb;          /* cells per axis, padded transform length (2n), boundary cells */
  int precision;             /* bem_precision */
  int grid_ctas;             /* persistent CTAs of the fused column kernel */
  int threads_per_cta;
  size_t scratch_bytes;      /* device scratch owned by the plan (partials, weighted densities) */
  size_t spectra_bytes;      /* device bytes of the compressed kernel spectra */
  double plan_seconds;       /* wall time of bem_plan */
  int64_t grid_nodes;        /* accuracy mode: active grid nodes of the inner convolution; else nb */
} bem_plan_info;

/* Build a plan (Section 3-4: kernel tables on the padded grid and their
 * spectra; Fig. 5, Eq. 16).
 *   dim     2 (BEM_LAPLACE_2D) or 3 (BEM_LAPLACE_3D, BEM_KELVIN_3D)
 *   n       host array of dim cell counts; all equal (else BEM_ERR_UNSUPPORTED)
 *   h       grid spacing (> 0)
 *   nb      number of boundary cells (>= 1)
 *   cell    host, nb*dim int32 grid indices in [0, n), row-major (cell j axis a
 *           at cell[j*dim + a]); duplicates are rejected (BEM_ERR_ARG)
 *   w       host, nb boundary measures
 *   normal  host, nb*dim unit outward normals
 *   nu, mu  Poisson ratio and shear modulus (Kelvin only; ignored otherwise)
 *   prec    arithmetic of the apply; spectra are always computed in FP64 on
 *           the device and rounded to prec
 *   flags   0, or BEM_PLAN_SINGLE_LAYER_ONLY and/or BEM_PLAN_THREE_PASS
 *           (below); BEM_PLAN_SINGLE_LAYER_ONLY: the plan serves BEM_SINGLE
 *           applies only (bem_set_bc and the other layers return
 *           BEM_ERR_UNSUPPORTED); the column kernel then needs no staging
 *           rows for the double layer's fields and keeps more of its
 *           accumulators in shared memory
 *   stream  cudaStream_t (may be NULL) used for the set-up kernels; the call
 *           synchronises it before returning
 * The plan copies every input.  Device memory: spectra (ncomp-dependent,
 * (n+1)^dim reals each), scratch, boundary metadata. */
#define BEM_PLAN_SINGLE_LAYER_ONLY 1u
/* BEM_PLAN_THREE_PASS (BEM_F32, 2D, n >= 256, no tensor-core stages; ignored
 * otherwise): apply in three passes through device memory instead of the
 * fused column kernel: the input-pruned x-DFT of the fields row by row into
 * a (n+1) x n buffer per field, the column transforms with the spectral
 * multiply into one (n+1) x n buffer, and the output-pruned inverse x-DFT at
 * the cells.  Same operator, same FP32 arithmetic (sums in another order);
 * about 4 (n+1) n complex values of extra device memory. */
#define BEM_PLAN_THREE_PASS 2u
bem_status bem_plan(bem_plan_t* out, int dim, const int64_t* n, double h, int64_t nb, const int32_t* cell,
                    const double* w, const double* normal, bem_kernel kernel, double nu, double mu,
                    bem_precision prec, uint32_t flags, void* stream);

/* Accuracy mode: a plan whose unknowns live on flat boundary panels instead
 * of grid nodes (one value per panel), applied with the paper's grid
 * convolution (Section 4, Eq. 16) by the precorrected-FFT construction.  The
 * paper-form operator of bem_plan (sources and targets on grid nodes) does
 * not converge on curved boundaries; this one converges to the flat-panel
 * collocation BEM up to an error set by the stencil order and near radius.
 *   n, h        grid (n a power of two in [4, 4096]; node k at (k + 1/2) h)
 *   nb          number of panels (>= 1)
 *   panels      host, nb*4 doubles: A.x, A.y, B.x, B.y of panel j; the
 *               outward normal is the tangent (B - A) turned clockwise
 *               (counter-clockwise closed curves); collocation at (A + B)/2;
 *               every midpoint's stencil must lie inside the grid (about
 *               two cells of margin), else BEM_ERR_ARG
 *   order       2 or 3: (order + 1)^2-node Lagrange stencils
 *   near_radius R >= order (at most 64): panel pairs whose stencil anchors
 *               differ by at most R cells along both axes get exact panel
 *               integrals (closed forms), the rest goes through the grid
 *   prec        as bem_plan (the grid convolution's arithmetic and the I/O
 *               type); the projection, interpolation and corrections sum in
 *               FP64 and are stored in the I/O type
 * Operators (bem_apply, BEM_SINGLE / BEM_DOUBLE / BEM_SYSTEM, and bem_solve):
 * S and D with the paper's signs (Eq. 15), c = 1/2; the double layer carries a
 * diagonal term that makes its rows sum to 1/2 (Gauss's law, exact for closed
 * curves; the mode assumes closed curves and the interior problem).
 * bem_set_bc, bem_solve, bem_enable_refinement (companion: the same panels in
 * BEM_F32X2 for n >= 256, else BEM_F64), bem_set_preconditioner (blocks of
 * consecutive panels from the exact panel integrals), batches, bem_get_info
 * and kernel timing (the grid convolution) apply; bem_apply_static_scratch
 * returns BEM_ERR_UNSUPPORTED.  Not in the paper: an added discretisation
 * (Phillips and White, IEEE TCAD 16(10), 1997) around the paper's kernels. */
bem_status bem_plan_panels(bem_plan_t* out, int64_t n, double h, int64_t nb, const double* panels, int order,
                           int near_radius, bem_precision prec, uint32_t flags, void* stream);

/* Set the boundary-condition types used by BEM_SYSTEM and bem_solve.
 *   bc  host, nb*ncomp bytes: 0 = Dirichlet (u known, q/t unknown),
 *       1 = Neumann (q/t known, u unknown)
 *   c   free-term coefficient (Section 2: 1/2 on a smooth boundary) */
bem_status bem_set_bc(bem_plan_t plan, const uint8_t* bc, double c);

/* Operator applies on the device (Section 4, Eq. 15-16): nbatch densities
 * through the same operator.  The kernel spectra are fixed per plan (Eq. 16),
 * so every right-hand side reuses them.
 *   in_dev, out_dev  device pointers, nbatch*nb*ncomp values of the plan
 *                    precision (double for BEM_F64 and BEM_F32X2, float for
 *                    BEM_F32 and the tensor-core forms); vector r at element
 *                    offset r*nb*ncomp, component fastest; caller-owned; the
 *                    two ranges must not overlap (BEM_ERR_ARG), and device
 *                    memory of another GPU than the plan's is refused
 *                    (BEM_ERR_ARG)
 *   nbatch           number of vectors (>= 1)
 *   stream           cudaStream_t (may be NULL); the call is asynchronous and
 *                    the vectors are applied in order on this stream
 * The plan's device must be the current device (BEM_ERR_ARG otherwise).
 * BEM_SYSTEM needs a prior bem_set_bc. */
bem_status bem_apply(bem_plan_t plan, bem_layer layer, const void* in_dev, void* out_dev, int nbatch, void* stream);

/* One apply with HOST buffers (nb*ncomp values, plan precision): copies in,
 * applies, copies out and synchronises the stream before returning.  The
 * plan's device must be current. */
bem_status bem_apply_host(bem_plan_t plan, bem_layer layer, const void* in_host, void* out_host, void* stream);

/* bem_apply without touching the CUDA allocator, for callers that cannot
 * allocate device memory at the point where they apply the operator (device
 * memory fully reserved by another framework's pool, latency-critical loops
 * that must not enter the allocator, hosts that forbid device allocation after
 * start-up).  The paper has no counterpart: this is a deployment variant of
 * the apply above, same arguments, same results.
 * The densities and per-CTA partial sums go to one static 16 MiB device
 * buffer linked into the library (held on every GPU that uses this call until
 * the process exits) instead of the plan's scratch.  The first call on a
 * device looks up the buffer's address (make it before any stream capture).
 * Plans whose scratch does not fit return BEM_ERR_UNSUPPORTED with the needed
 * size in bem_last_error().  All calls share the buffer: calls that overlap on
 * the GPU (unordered streams, concurrent threads) race.  No cudaMalloc, no
 * cudaFree, no allocating library call. */
bem_status bem_apply_static_scratch(bem_plan_t plan, bem_layer layer, const void* in_dev, void* out_dev,
                                    void* stream);

/* Solve the boundary-condition split system for the unknowns (Section 4:
 * Krylov iteration on the FFT apply; restarted GMRES here).  Each Arnoldi step
 * (preconditioner, apply, two Gram-Schmidt sweeps, norm, next basis vector,
 * Givens rotation) is one CUDA graph replay with the step index and the
 * rotations kept on the device; the host reads one integer per step.  The
 * solve runs on an internal stream ordered after `stream` and returns when
 * the outputs are on the host.
 *   bc        host nb*ncomp (as bem_set_bc; also sets the plan's BC state)
 *   data      host nb*ncomp FP64 known values: u where bc = 0, q/t where bc = 1
 *   c         free-term coefficient
 *   tol       stop when the relative residual ||b - A x||/||b|| <= tol
 *   max_iter  total iteration cap;  restart  Krylov dimension m (<= 512)
 *   x0        host nb*ncomp FP64 initial guess of the unknowns, or NULL (zero);
 *             a guess whose residual exceeds that of zero is replaced by zero
 *   u_out, q_out  host nb*ncomp FP64 full boundary fields (known entries
 *             copied from data, unknown ones from the solution); either may be NULL
 *   info      may be NULL
 * Returns BEM_ERR_NOT_CONVERGED with the best iterate written if max_iter is
 * reached.  Arnoldi, Givens rotations and residual norms are FP64.  The
 * plan's device must be current (BEM_ERR_ARG otherwise). */
bem_status bem_solve(bem_plan_t plan, const uint8_t* bc, const double* data, double c, double tol, int max_iter,
                     int restart, const double* x0, double* u_out, double* q_out, bem_solve_info* info,
                     void* stream);

/* Preconditioner of bem_solve (right preconditioning, GMRES on A M^-1).
 *   kind 0: none.  kind 1 (default; block_size 128 cells in 2D, 64 in 3D):
 *   block Jacobi on the near field: M = the diagonal blocks of A over
 *   consecutive cells in the caller's order (pass cells in boundary order,
 *   e.g. arclength along a curve, so that a block is a connected piece of S);
 *   the blocks are assembled from the same kernel point values as the
 *   operator when a solve first needs them after bem_set_bc, and inverted on
 *   the device in FP32 (2D, block_size <= 512) or in FP64 on the host.
 * The paper solves without a preconditioner (Section 4); the single layer is
 * a first-kind operator whose condition number grows with n, so unpreconditioned
 * restarted GMRES stalls on mixed problems. */
bem_status bem_set_preconditioner(bem_plan_t plan, int kind, int block_size);

/* Mixed-precision iterative refinement for BEM_F32 plans: with enable != 0
 * the plan builds a companion plan of the same geometry in BEM_F32X2 (3D, and
 * 2D with n >= 256) or BEM_F64 (2D, n < 256); bem_solve then forms the right-hand side
 * and every residual with the companion operator and solves
 * for the corrections with the preconditioned FP32 GMRES, so that tolerances
 * below the FP32 operator's own accuracy (plain FP32 GMRES stalls at a
 * relative residual of 1.7e-6 on the 4096^2 star) are reached.  rel_residual then is the companion's
 * residual.  No effect on BEM_F64 and BEM_F32X2 plans. */
bem_status bem_enable_refinement(bem_plan_t plan, int enable);

/* Query sizes and launch shape of a plan. */
bem_status bem_get_info(bem_plan_t plan, bem_plan_info* info);

/* Kernel timing: when enabled, every apply records CUDA events around the
 * fused column kernel on the apply's stream; bem_kernel_time returns the sum
 * of their elapsed times (ms) and the count since the last reset.  Reading
 * the times synchronises the recorded events. */
bem_status bem_set_kernel_timing(bem_plan_t plan, int enable);
bem_status bem_kernel_time(bem_plan_t plan, double* total_ms, int64_t* launches);

/* Number of kernel launches one apply of the given layer issues. */
int bem_launches_per_apply(bem_plan_t plan, bem_layer layer);

/* Device-side status of the plan's kernels since the last call (tensor-core
 * precisions: every wait of a kernel on its tensor-core products is bounded
 * to about one second; a wait that gave up makes the kernel stop early and
 * record it).  Synchronises `stream` (cudaStream_t, may be NULL), reads and
 * clears the record.  Returns BEM_ERR_TIMEOUT when a wait gave up (the
 * outputs of the applies since the last call are then invalid), else BEM_OK.
 * No counterpart in the paper: a safeguard of the device implementation.
 * bem_solve checks it before returning. */
bem_status bem_device_status(bem_plan_t plan, void* stream);

/* Test hook for the bounded device waits (no counterpart in the paper).
 * BEM_TEST_WAIT_RUNS_OUT: the tensor-core column kernels of this plan issue no
 * tensor-core product and no completion signal, so every wait of theirs runs
 * out after its bound (about one second); the CTAs then stop, free their tensor
 * memory and record the event for bem_device_status.  Nothing faults, traps
 * or hangs; outputs of such applies are invalid.  Pass 0 to clear.  Plans
 * without tensor-core stages ignore the flag.  Returns BEM_ERR_ARG for a null
 * plan or unknown bits. */
#define BEM_TEST_WAIT_RUNS_OUT 1u
/* BEM_TEST_HOST_ARNOLDI: bem_solve runs the host-driven Arnoldi loop (Givens
 * rotations on the host, one stream synchronisation per step) instead of its
 * default path (each Arnoldi step one CUDA graph replay, Givens rotations on
 * the device); for comparing the two. */
#define BEM_TEST_HOST_ARNOLDI 2u
bem_status bem_set_test_flags(bem_plan_t plan, uint32_t flags);

/* ---- batched apply (many geometries, one CUDA graph) --------------------
 * The applies of `count` plans (one precision, grids of any sizes) captured
 * once into a CUDA graph, the plans spread round-robin over `streams` forked
 * capture streams so that small geometries run side by side; bem_batch_apply
 * then replays the whole batch with one graph launch.  Inputs and outputs are
 * two packed device buffers owned by the batch (plan i's nb_i*ncomp_i values at
 * element offset bem_batch_offset(i)), so the captured pointers stay valid.
 * The plans must outlive the batch and be distinct (a plan listed twice
 * returns BEM_ERR_ARG); when bem_set_bc changes a plan's system operator, the
 * next bem_batch_apply captures the graph again.  The plans' kernel timing is
 * switched off.  FP32 four-step plans of one grid size are applied by one
 * grouped launch (bem_batch_set_grouping). */
typedef struct bem_batch_s* bem_batch_t;
bem_status bem_batch_create(bem_batch_t* out, const bem_plan_t* plans, int count, bem_layer layer, int streams,
                            void* stream);
bem_status bem_batch_buffers(bem_batch_t batch, void** in_dev, void** out_dev, size_t* total);
bem_status bem_batch_offset(bem_batch_t batch, int i, size_t* offset);
bem_status bem_batch_apply(bem_batch_t batch, void* stream);

/* Grouped launches (default on): the batch's FP32 four-step plans (2D,
 * n >= 256, no tensor-core stages) that share a grid size are applied by ONE
 * persistent column-kernel launch per size, whose CTAs take contiguous ranges
 * of the columns of all those plans (no per-plan tail), between the plans'
 * own density and reduction launches; the other plans are applied one by one.
 * Results are deterministic but, the columns being split over the CTAs
 * differently, not bit-identical to bem_apply of each plan (FP32 rounding).
 * enable = 0 applies every plan on its own (bit-identical to bem_apply).  The
 * batch graph is captured again. */
bem_status bem_batch_set_grouping(bem_batch_t batch, int enable);
int bem_batch_launches(bem_batch_t batch);  /* kernel launches inside one replay */
bem_status bem_batch_destroy(bem_batch_t batch);

/* Solve the boundary-condition systems of every plan of a BEM_SYSTEM batch
 * together (Section 4's Krylov solve, batched): one restarted GMRES(restart)
 * runs in lockstep over all systems, each Arnoldi step being one CUDA graph
 * replay (each plan's preconditioner, the batched apply, classical
 * Gram-Schmidt with re-orthogonalisation per system, Givens rotations on the
 * device); a system stops iterating at its own tolerance.  When every plan has
 * refinement enabled, residuals use the companions (batched too) and the
 * lockstep GMRES solves for corrections, as in bem_solve.
 *   bc, data       host, packed like the batch buffers (plan i's nb_i*ncomp_i
 *                  entries at bem_batch_offset(i)); meaning as in bem_solve;
 *                  the plans' boundary conditions are set to bc
 *   x0             host, packed initial guess of the unknowns, or NULL
 *   u_out, q_out   host, packed (may be NULL)
 *   info           host array of count entries (per plan), or NULL; iters,
 *                  restarts and applies are the common lockstep counts
 *   stream         the solve runs on an internal stream ordered after it and
 *                  returns when the outputs are on the host
 * Returns BEM_ERR_NOT_CONVERGED when some system misses tol (outputs and info
 * are still written), BEM_ERR_UNSUPPORTED for more than 1024 plans. */
bem_status bem_batch_solve(bem_batch_t batch, const uint8_t* bc, const double* data, double c, double tol,
                           int max_iter, int restart, const double* x0, double* u_out, double* q_out,
                           bem_solve_info* info, void* stream);

/* ---- measured launch choices (autotuning) -------------------------------
 * Choices that the problem's shape alone does not fix are timed on the device
 * with the caller's data and kept in a process-wide table keyed by the shape
 * (grid sizes, cell counts, kernel, precision), so later plans or batches of
 * the same shape take the stored choice without timing again.
 * bem_tune_batch: the number of forked capture streams of the batch graph
 *   (candidates 1, 2, 4, 8; `reps` timed replays each); the batch is captured
 *   again with the winner, returned in *streams (may be NULL).
 * bem_tune_preconditioner: the block size of the block-Jacobi preconditioner
 *   (candidates 32, 64, 128, 256 cells, within 256 unknowns per block in 2D
 *   and 192 in 3D), by the wall time of a full bem_solve with these arguments,
 *   including the block inversion; the plan keeps the winner, returned in
 *   *block (may be NULL).  BEM_ERR_NOT_CONVERGED when no candidate converges. */
bem_status bem_tune_batch(bem_batch_t batch, int reps, int* streams);
/* bem_tune_shapes: the launch shape of the plan's apply that is a runtime
 *   choice - the cells per load batch of the 2D fused cell walks (2 or 4;
 *   FP32 and tensor-core plans with n >= 256, and the node plan of an
 *   accuracy-mode plan) or the lines per CTA of the 3D z pass (1, 2, 4, 8,
 *   16, capped by shared memory and 512 threads).  Each candidate is timed
 *   over `reps` applies (after one warm-up) of the system operator when
 *   boundary conditions are set, else the single layer, on zero data with
 *   CUDA events on `stream` (synchronised); the plan keeps the fastest,
 *   returned in *chosen with its milliseconds per apply in *best_ms (both may
 *   be NULL; the time is 0 when the choice came from the table).  Captured
 *   solve and batch graphs of the plan are captured again on their next use.
 *   Plans without such a choice return BEM_OK with *chosen = 0.  The
 *   operator's result does not depend on the choice. */
bem_status bem_tune_shapes(bem_plan_t plan, int reps, void* stream, int* chosen, double* best_ms);
bem_status bem_tune_preconditioner(bem_plan_t plan, const uint8_t* bc, const double* data, double c, double tol,
                                   int max_iter, int restart, int* block);

/* ---- learned initial guess (serving/training pattern on top of the operator;
 * the paper has no learned component) ------------------------------------
 * A 1D convolutional network over the arclength-ordered cells of closed
 * curves: `layers` circular convolutions of odd width `ksize` with per-layer
 * dilation, cin -> hidden -> ... -> hidden -> 1 channels, ReLU between layers.
 * Weights and activations are stored in BF16 (round to nearest even), sums are
 * FP32; the FP32 master weights are trained with Adam (beta 0.9/0.999,
 * eps 1e-8) on the mean squared error.  A batch is nseq sequences stored back
 * to back: feats device [T x cin] FP32 (position-major), offsets device
 * [nseq + 1] int32 (offsets[0] = 0, offsets[nseq] = T), the circular padding
 * wraps inside each sequence.  Parameter layout (host vectors): per layer the
 * weights [cout][cin][ksize] followed by the biases [cout]. */
typedef struct bem_net_s* bem_net_t;
bem_status bem_net_create(bem_net_t* out, int cin, int hidden, int layers, int ksize, const int* dilations,
                          uint64_t seed);
bem_status bem_net_destroy(bem_net_t net);
/* Arclength Dirichlet-to-Neumann estimate (a feature of the learned guess):
 * per closed curve q of the batch (elements offsets[q] .. offsets[q+1] in
 * arclength order, midpoints at arclength s_j from the curve's start, lengths
 * len_j, total length Lambda, values u_j)
 *   uhat_k = (1/Lambda) sum_j len_j u_j e^{-2 pi i k s_j / Lambda}, k = 1..kmax,
 *   out_j  = sum_k (2 pi k / Lambda) 2 Re(uhat_k e^{2 pi i k s_j / Lambda}),
 * the interior flux of the harmonic extension of u on a circle of length
 * Lambda (exact there; on a smooth curve the error is smooth).  s, len, u,
 * out: device FP32 [T]; offsets: device int32 [nseq + 1]; FP32 phases
 * (reduced to [0, 1) turns), FP64 sums.  Asynchronous on `stream`. */
bem_status bem_dtn_estimate(const float* s, const float* len, const float* u, const int32_t* offsets, int nseq,
                            int64_t T, int kmax, float* out, void* stream);
/* Input columns of the 2D guess network per curve q (elements offsets[q] ..
 * offsets[q+1]): with sc_q the root mean square of u over the curve (1 when it
 * is zero),
 *   feats[j] = (geo[j][0 .. G), u_j / sc_q, radius * qd_j / sc_q),
 * geo device FP32 [T][G] (G <= 64), u and qd (the Dirichlet-to-Neumann
 * estimate) device FP32 [T], feats device FP32 [T][G + 2]; offsets device
 * int32 [nseq + 1], non-decreasing from 0 to T (not checked on the device).
 * FP64 scale, FP32 results; asynchronous on `stream`. */
bem_status bem_guess_features(const float* geo, int G, const float* u, const float* qd, const int32_t* offsets,
                              int nseq, int64_t T, float radius, float* feats, void* stream);
/* The guess of the interior Dirichlet problem from the network's output per
 * curve q (sc_q as above):
 *   x_j = qd_j + cscale * sc_q * corr_j,
 *   out_j = x_j - (sum_j len_j x_j) / (sum_j len_j),
 * so that the guessed flux integrates to zero over the curve, as the flux of
 * every field harmonic inside does (divergence theorem).  qd, corr, u, len,
 * out device FP32 [T]; offsets as above; FP64 sums; asynchronous. */
bem_status bem_guess_finish(const float* qd, const float* corr, const float* u, const float* len,
                            const int32_t* offsets, int nseq, int64_t T, float cscale, float* out, void* stream);
/* Random Fourier features of 3D points (the input encoding of the 3D point
 * network, which is bem_net_* with ksize = 1: the same weights applied to
 * every point independently):
 *   out[t][2f] = sin(2 pi B_f . p_t),  out[t][2f+1] = cos(2 pi B_f . p_t)
 * points device FP32 [T][3], B device FP32 [F][3] (frequencies, caller-drawn),
 * out device FP32 [T][2F].  FP64 phases, FP32 results; asynchronous. */
bem_status bem_fourier_features(const float* points, int64_t T, const float* B, int F, float* out, void* stream);
int64_t bem_net_num_params(bem_net_t net);
bem_status bem_net_get_params(bem_net_t net, float* host_params);
bem_status bem_net_set_params(bem_net_t net, const float* host_params);
/* out: device [T] FP32 predictions */
bem_status bem_net_forward(bem_net_t net, const float* feats, const int32_t* offsets, int nseq, int64_t T, float* out,
                           void* stream);
/* loss (host) and the gradient of the loss wrt the parameters (host, may be NULL) for target device [T] */
bem_status bem_net_gradient(bem_net_t net, const float* feats, const int32_t* offsets, int nseq, int64_t T,
                            const float* target, float* grad_host, double* loss, void* stream);
/* one Adam step with learning rate lr; loss (host) of the batch before the step */
bem_status bem_net_train_step(bem_net_t net, const float* feats, const int32_t* offsets, int nseq, int64_t T,
                              const float* target, float lr, double* loss, void* stream);

/* Arithmetic peak of the current device for the rooflines of the column
 * kernels, measured with a timed loop of independent fused multiply-adds
 * (CUDA events on `stream`, which the call synchronises; no clock or device
 * setting is changed).  kind 0: FP32 FMA, 1: FP64 FMA, 2: packed FP32 pairs
 * (two FMAs per instruction).  *tflops receives TFLOP/s (2 flops per FMA).
 * No counterpart in the paper: a measurement helper. */
bem_status bem_measure_peak(int kind, double* tflops, void* stream);

bem_status bem_destroy(bem_plan_t plan);
const char* bem_status_string(bem_status s);
const char* bem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BEM_GB300_H */
