/*
 * eddy_theta.h -- C ABI of the GB300 theta-method library for eddy-current
 * transients, after arXiv 2407.11993 (Chiariello et al., "Modal Decomposition
 * in Numerical Computation of Eddy Current Transients").
 *
 * The library integrates the discrete eddy-current system (Sec. 3.1,
 * Eq. discrete_version_1a/b)
 *
 *     R I + L dI/dt + E^T phi = V_0 + V_D,      E I = i_D,
 *     V_0 = -M di_0/dt,  V_D = -M^D di_D/dt     (Eq. induced_voltages_d/0)
 *
 * with the theta-method of Sec. 3.3, in one of two forms:
 *
 *   EC_FORM_PLAIN  Sec. 3.3.1, Eq. time_integration: Z = L_i + theta dt R_i is
 *                  factored once, Z = C C^T, and every step solves with C and C^T
 *                  (by default as two products with the inverted factor C^{-1},
 *                  EC_SOLVE_INVERSE; by substitution with EC_SOLVE_SUBSTITUTION).
 *   EC_FORM_MODAL  Sec. 3.2 (Eq. generalized_eigenvalues_discrete,
 *                  modal_decomposition_discrete) and Sec. 3.3.2: the pencil
 *                  L_i u = tau R_i u is solved once; every mode then follows a
 *                  scalar theta-recurrence.
 *
 * Electrode constraints are eliminated as in Sec. 3.1 (Eq. current_electrodes,
 * discrete_version_2, circuit_equations_v2): I = K I_i + E^T (E E^T)^{-1} i_D
 * with K an orthonormal basis of ker E (built from Householder reflectors).
 *
 * Conventions for every entry point:
 *   - All floating-point data are IEEE binary64 (double).
 *   - Dense matrices are row-major with the shapes stated below; L and R are
 *     symmetric and only their lower triangle (row >= column) is read.
 *   - `mem` says where the caller's pointers live: EC_MEM_HOST (pageable or
 *     pinned host memory) or EC_MEM_DEVICE (device memory on the context's
 *     GPU).  The library copies inputs into storage it owns; the caller keeps
 *     ownership of its buffers and may free them when the call returns.
 *   - Work is enqueued on the context's CUDA stream.  Calls that return data
 *     to host memory synchronise that stream; calls with device outputs do not
 *     (use ec_sync to wait and collect errors raised inside kernels).
 *   - Every call returns an ec_status; nothing throws across the ABI and
 *     nothing calls exit().  A failed call leaves the context usable for
 *     ec_destroy, and for a new ec_setup.
 */
#ifndef EDDY_THETA_H
#define EDDY_THETA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define EC_API __attribute__((visibility("default")))
#else
#define EC_API
#endif

typedef struct ec_ctx ec_ctx;

typedef enum ec_status {
  EC_OK = 0,
  EC_ERR_ARG = 1,          /* invalid argument (null pointer, theta outside [0,1], dt <= 0, ...) */
  EC_ERR_SHAPE = 2,        /* inconsistent sizes */
  EC_ERR_NOT_SPD = 3,      /* Z (plain) or R_i (modal) is not positive definite; see ec_last_info */
  EC_ERR_RANK = 4,         /* E does not have full row rank */
  EC_ERR_OOM = 5,          /* device allocation failed */
  EC_ERR_CUDA = 6,         /* CUDA runtime error */
  EC_ERR_TIMEOUT = 7,      /* a bounded inter-block wait inside a kernel gave up */
  EC_ERR_STATE = 8,        /* call out of order (e.g. ec_run before ec_setup) */
  EC_ERR_NOT_CONVERGED = 9,/* an iterative eigen step did not converge */
  EC_ERR_UNSUPPORTED = 10  /* valid request outside what the library implements */
} ec_status;

typedef enum ec_form { EC_FORM_PLAIN = 0, EC_FORM_MODAL = 1 } ec_form;
typedef enum ec_mem { EC_MEM_HOST = 0, EC_MEM_DEVICE = 1 } ec_mem;

typedef struct ec_config {
  int form;               /* ec_form */
  double theta;           /* theta of Sec. 3.3, in [0, 1] */
  double dt;              /* time step [s], > 0 */
  void* stream;           /* cudaStream_t to enqueue on; NULL = the legacy default stream */
  int device;             /* CUDA device ordinal */
  long long spin_limit;   /* polls before a kernel-side wait gives up (EC_ERR_TIMEOUT); 0 = default */
  int profile;            /* nonzero: ec_run times its dominant kernels with CUDA events (see ec_timing) */
  int plain_solver;       /* plain form only: EC_SOLVE_INVERSE (default) or EC_SOLVE_SUBSTITUTION */
  int precision;          /* EC_PREC_FP64 (default); modal form: EC_PREC_BF16 / _BF16X3 /
                             _FP32 / _FP32X2; plain form: EC_PREC_FP32 / _FP32X2; see below */
  int integrator;         /* modal form: EC_INTEG_THETA (default) or EC_INTEG_EXACT, see below */
  int rhs_mode;           /* EC_RHS_SUM (default), EC_RHS_INDEPENDENT or EC_RHS_PAIRED, see below */
  int refine_steps;       /* plain form with EC_PREC_FP32: FP64 iterative-refinement sweeps per
                             step (0 .. 8; 0 = plain FP32 solves), see below */
  int tile_variant;       /* plain form, EC_SOLVE_INVERSE: 0 (default) = ec_setup times every launch
                             shape of the per-step products on the actual factor and keeps the
                             fastest; 1 .. 3 = use that shape.  No shape changes a result bit. */
  int setup_gemm;         /* EC_GEMM_TENSOR (default), EC_GEMM_FP64 or EC_GEMM_TENSOR_PAIRSYMV */
  int release_inputs;     /* nonzero: when ec_setup succeeds, free the device copies of L and R
                             (and, for the plain form with EC_SOLVE_INVERSE, of the Cholesky factor
                             of Z) that stepping does not read -- 2-3 N^2 doubles, 69-103 GB at
                             N = 65,536.  The plain form then refuses ec_set_step (EC_ERR_STATE):
                             a new dt needs a new ec_setup.  Everything else is unaffected. */
} ec_config;

/* Arithmetic units of the setup's large dense products (both FP64-accurate): the
 * Cholesky factorisations' trailing updates, the triangular solves of the reduction
 * and back-transformation, the divide-and-conquer merges, the inverse factor and
 * the modal snapshot reconstruction.
 *   EC_GEMM_TENSOR  FP64 operands cut into 8-bit integer slices and multiplied on the
 *                   tensor cores with exact accumulation (see ec_gemm_f64_emulated).
 *   EC_GEMM_FP64    the FP64 CUDA cores (about 1.1 TFLOP/s on GB300).
 *   EC_GEMM_TENSOR_PAIRSYMV  as EC_GEMM_TENSOR, and the tridiagonalisation's symmetric
 *                   products (one pass over the trailing matrix per column, bound by
 *                   the FP64 pipe) in compensated FP32: each FP64 entry split into an
 *                   FP32 hi/lo pair, float-float sums, about 2^-46 relative per product
 *                   instead of 2^-53.  Reflectors, updates and everything else as
 *                   EC_GEMM_TENSOR.  Modal form only (the plain form treats it as
 *                   EC_GEMM_TENSOR).
 * The two differ by rounding only. */
enum { EC_GEMM_TENSOR = 0, EC_GEMM_FP64 = 1, EC_GEMM_TENSOR_PAIRSYMV = 2 };

/* How the s coil columns of M drive the system (batched right-hand sides).
 *   EC_RHS_SUM          all coils act on one trajectory (their voltages add).
 *   EC_RHS_INDEPENDENT  coil k drives its own trajectory k (s trajectories in one run;
 *                       the plain form solves with s right-hand sides per step, the modal
 *                       form runs s sets of mode recurrences).  ec_run writes probes as
 *                       T x s x p (row (k-1) s + j = the p probes of trajectory j) and
 *                       snapshots as nsnap x s x n.  Requires m = 0.
 *   EC_RHS_PAIRED       as INDEPENDENT, but trajectory j is read by probe row j only
 *                       (p = s, e.g. C = M^T: each coil's own pickup); probes are T x s.
 * For the independent modes the state holds s trajectories (ec_state_size = s N_0) and
 * ec_set_current starts every trajectory from the same current. */
enum { EC_RHS_SUM = 0, EC_RHS_INDEPENDENT = 1, EC_RHS_PAIRED = 2 };

/* Per-mode time integrator of the modal form.
 *   EC_INTEG_THETA  the theta-method of Sec. 3.3.2 (same scheme as the plain form).
 *   EC_INTEG_EXACT  exact integration of each decoupled mode, tau x' + x = e(t), for
 *                   sources linear between their samples (the analytical route Sec. 3.3
 *                   points to): x^{k+1} = e^{-h} x^k + (1 - e^{-h}) e0 + (1 - (1 - e^{-h})/h) e1,
 *                   h = dt / tau, e0 and e1 the forcing at the step start and its change
 *                   over the step.  theta is ignored. */
enum { EC_INTEG_THETA = 0, EC_INTEG_EXACT = 1 };

/* Arithmetic of the modal form's dense contractions.  The Cholesky of R_i, the
 * pencil reduction, the eigensolve and the per-mode recurrence are FP64 in every
 * variant (tau and mode orthogonality need it).
 *   EC_PREC_FP64  projections U^T [R_D | L_D | M_0], U^T (C K)^T and the snapshot
 *                 reconstruction U X in FP64.
 *   EC_PREC_BF16  the same three products with BF16 operands on the tensor cores
 *                 (tcgen05), FP32 accumulation; each product carries BF16 rounding
 *                 (2^-9 relative per entry), which cancellation in the modal sums
 *                 can amplify (see ec_gemm_bf16 and the documented error tables).
 *   EC_PREC_BF16X3  split BF16: each operand is stored as hi + lo BF16 parts and each
 *                 product is hi*hi + hi*lo + lo*hi on the tensor cores, summed in
 *                 FP64 (about 2^-16 relative per entry, three times the tensor work).
 *   EC_PREC_FP32  the same three products with U and the right-hand columns rounded to
 *                 FP32 (each under a power-of-two scale), FP32 multiply-adds and FP32
 *                 sums within K segments of at least 512, the segments added in FP64
 *                 (2^-24 relative per entry plus the FP32 sum's rounding).  With a few
 *                 right-hand columns the products stream U once: half the bytes of FP64
 *                 and arithmetic on the FP32 pipe.
 *   EC_PREC_FP32X2  U as FP32 hi/lo pairs (8 bytes, about 48 significant bits) and
 *                 compensated FP32 arithmetic (exact hi*hi products by FMA, the cross
 *                 terms, float-float sums, FP64 sums every 64 products): about 2^-46
 *                 relative per entry.
 *   FP32 / FP32X2 keep the FP64 U (ec_modes) and add a copy of 4 / 8 bytes per entry.
 *   ec_batch_run and ec_grad, which serve the plain form, are unaffected. */
enum { EC_PREC_FP64 = 0, EC_PREC_BF16 = 1, EC_PREC_BF16X3 = 2, EC_PREC_FP32 = 3,
       EC_PREC_FP32X2 = 4 };

/* Arithmetic of the plain form's per-step solve (EC_SOLVE_INVERSE, EC_RHS_SUM, no
 * electrodes).  The Cholesky factor and its inverse are computed in FP64 in every case.
 *   EC_PREC_FP64  both triangular products in FP64 (default).
 *   EC_PREC_FP32  the inverse factor is rounded to FP32 (half the bytes) and the two
 *                 products run in FP32 with FP64 partial sums; each of cfg.refine_steps
 *                 sweeps then forms the residual b - Z x in FP64 (L from its packed FP64
 *                 lower half, R from its sparse form) and adds the FP32 solve of it.
 *                 ec_grad, ec_get_inverse_factor and ec_batch_run need EC_PREC_FP64
 *                 (EC_ERR_UNSUPPORTED); electrodes (m > 0) are EC_ERR_UNSUPPORTED.
 *   EC_PREC_FP32X2  the inverse factor is stored as FP32 hi/lo pairs (hi = fp32(w),
 *                 lo = fp32(w - hi): about 48 significant bits in the same 8 bytes as
 *                 FP64) and the products run in compensated FP32 arithmetic (exact
 *                 hi*hi products by FMA, float-float sums, FP64 partial rows): on GB300
 *                 the products then move from the FP64 pipe's limit to HBM bandwidth.
 *                 Error about 2^-46 relative per product entry; electrodes allowed; the
 *                 same calls as EC_PREC_FP32 need EC_PREC_FP64. */

/* How the plain form applies its Cholesky factor C each step (Sec. 3.3.1).
 *   EC_SOLVE_INVERSE       C^{-1} is formed once at setup (N^3/3 extra flops); each
 *                          step computes y = C^{-1} b and x = C^{-T} y as triangular
 *                          matrix-vector products (all tiles independent).
 *   EC_SOLVE_SUBSTITUTION  forward then backward substitution with C itself, in a
 *                          persistent kernel whose blocks wait on each other's
 *                          published results (bounded waits).
 * Both do N^2 multiply-adds per step. */
enum { EC_SOLVE_INVERSE = 0, EC_SOLVE_SUBSTITUTION = 1 };

/* Wall-clock phases of the last ec_setup / ec_run, in milliseconds, measured
 * with CUDA events on the context's stream.  Phases a form does not run are 0. */
typedef struct ec_timing {
  double elim_ms;         /* constraint elimination (Householder reflectors, Sec. 3.1) */
  double factor_ms;       /* plain: Cholesky of Z (Sec. 3.3.1); modal: Cholesky of R_i */
  double reduce_ms;       /* modal: A = C_R^{-1} L_i C_R^{-T} */
  double tridiag_ms;      /* modal: Householder tridiagonalisation of A */
  double eig_ms;          /* modal: tridiagonal eigensolver (reported on its own) */
  double backtransform_ms;/* modal: U = C_R^{-T} Q S */
  double project_ms;      /* modal: source / probe projections and per-mode coefficients */
  double setup_ms;        /* whole ec_setup */
  double run_ms;          /* whole last ec_run */
  int64_t run_steps;      /* steps of the last ec_run */
  /* With cfg.profile set: summed device time and number of timed launches of the
   * forward / backward solve kernels (plain form; a sample of steps) and of the
   * modal scan kernel (modal form; every launch) during the last ec_run. */
  double fwd_ms, bwd_ms, scan_ms;
  int64_t fwd_launches, bwd_launches, scan_launches;
  /* Plain form, EC_SOLVE_INVERSE: launch shape of the per-step products in use
   * (1 .. 3) and, when ec_setup tuned it, the time of one product pair per shape
   * (entries past the number of shapes are 0). */
  int64_t tile_variant;
  double tile_tune_ms[4];
} ec_timing;

/* Create a context on cfg->device.  *out receives the handle. */
EC_API ec_status ec_create(ec_ctx** out, const ec_config* cfg);

/* One-time setup (Sec. 3.3.1 for the plain form; Sec. 3.2 for the modal form).
 *   n        number of current unknowns N (>= 1)
 *   L, R     n x n, symmetric positive definite inductance / resistance
 *   m, E     reduced electrode incidence, m x n (m = N_e - 1 >= 0, E may be NULL if m = 0);
 *            Eq. definition_E.  Must have full row rank (else EC_ERR_RANK).
 *   s, M     coil mutuals, s x n (row k is the mutual between coil k and the n unknowns);
 *            the coils induce V_0 = -M^T di_0/dt.  M may be NULL if s = 0.
 *   MD       electrode-source mutuals, m x n (row j: M^D column j), or NULL for zero.
 *   p, C     probe rows, p x n; probe outputs are y = C I.  C may be NULL if p = 0.
 * Copies every input; the caller's buffers are not retained.  Resets the state to I = 0.
 * A NaN or infinite entry in L, R, E, M, MD or C is refused with EC_ERR_ARG before any
 * factorisation (ec_last_info: 0 L, 1 R, 2 E, 3 M, 4 MD, 5 C). */
EC_API ec_status ec_setup(ec_ctx* ctx, int64_t n, const double* L, const double* R, int64_t m,
                          const double* E, int64_t s, const double* M, const double* MD,
                          int64_t p, const double* C, int mem);

/* Change theta and dt.  Plain form: re-forms and re-factors Z (O(N^3)).
 * Modal form: recomputes the per-mode coefficients only (O(N)); the modes do not
 * depend on dt (Sec. 5). */
EC_API ec_status ec_set_step(ec_ctx* ctx, double theta, double dt);

/* Modal form only: switch the arithmetic of the products with the mode matrix U
 * (EC_PREC_FP64 / _BF16 / _BF16X3 / _FP32 / _FP32X2, see above) on a set-up context.
 * The modes (Sec. 3.2) are kept: the reduced copy of U is rebuilt from the FP64 U and
 * the projections B = U^T [R_D | L_D | M_0], G^T = U^T (C K)^T are recomputed with the
 * new arithmetic; the current modal state is kept.  Works after release_inputs.
 * EC_ERR_STATE before ec_setup, EC_ERR_UNSUPPORTED for the plain form, EC_ERR_ARG for
 * an unknown value, EC_ERR_OOM when the copy does not fit (the context then keeps
 * FP64 products). */
EC_API ec_status ec_set_precision(ec_ctx* ctx, int precision);

/* Advance T steps of Eq. time_integration (plain) or its modal image (modal).
 *   src     s x (T+1) coil currents i_0 at t_k = k dt, k = 0..T (row-major; NULL if s = 0)
 *   iD      m x (T+1) electrode currents i_D (row-major; NULL if m = 0)
 *   probes  T x p output, row k-1 = C I^k for k = 1..T (NULL if p = 0)
 *   snap_stride, snaps   if snap_stride > 0: (T / snap_stride) x n output, row j = I^{(j+1) stride}
 * Starts from the current state and leaves I^T as the new state. */
EC_API ec_status ec_run(ec_ctx* ctx, int64_t T, const double* src, const double* iD,
                        double* probes, int64_t snap_stride, double* snaps, int mem);

/* Batched instances (no counterpart in the paper, which runs one problem at a time).  Advances `count` independent plain-form problems of different sizes by T
 * steps each, as if ec_run were called on each (same arguments per instance, one common
 * snap_stride), in one pass per step:
 *   - every instance's tile products go into one work list (all instances' units,
 *     largest first) run by one persistent grid; right-hand sides, partial sums and
 *     updates are one launch each over all instances;
 *   - one step of all instances is captured once into a CUDA graph and replayed T times;
 *   - the launch shape of the products is timed on the batch before the run.
 * Each instance computes exactly what its own ec_run computes (bitwise): the instances
 * keep their own factors, work decomposition and reduction order.
 *   ctxs       count distinct contexts, 1 <= count <= EC_BATCH_MAX, all set up, all on
 *              one device, all EC_FORM_PLAIN with EC_SOLVE_INVERSE and EC_RHS_SUM
 *              (else EC_ERR_UNSUPPORTED)
 *   src, iD    arrays of count pointers (entry i as ec_run's src / iD of instance i; the
 *              array may be NULL when no instance needs it)
 *   probes, snaps   arrays of count output pointers (entries may be NULL)
 *   mem        memory space of every data pointer (the pointer arrays are host arrays)
 * Blocking: returns after the outputs are written.  The run uses its own stream, after
 * synchronising every instance's stream.  ec_timings(ctx) of each instance reports the
 * batch's run time. */
#define EC_BATCH_MAX 64
EC_API ec_status ec_batch_run(ec_ctx* const* ctxs, int count, int64_t T, const double* const* src,
                              const double* const* iD, double* const* probes, int64_t snap_stride,
                              double* const* snaps, int mem);

/* Set the state from a physical current I (length n): I_i = K^T I (the particular
 * part is rebuilt from i_D at the next step). */
EC_API ec_status ec_set_current(ec_ctx* ctx, const double* I, int mem);

/* Internal state of length ec_state_size(): I_i (plain) or the modal amplitudes x
 * (modal).  ec_set_state(ec_get_state()) resumes bit-identically. */
EC_API int64_t ec_state_size(const ec_ctx* ctx);
EC_API ec_status ec_get_state(ec_ctx* ctx, double* state, int mem);
EC_API ec_status ec_set_state(ec_ctx* ctx, const double* state, int mem);

/* Modal form only: tau (N_0, decreasing) and U (N_0 x N_0, column j = mode j,
 * column-major, U^T R_i U = 1) in the internal basis of ker E. */
EC_API ec_status ec_get_modes(ec_ctx* ctx, double* tau, double* U, int mem);

/* Plain form only: solve Z x = b, Z = L_i + theta dt R_i (the matrix of Eq. time_integration,
 * Sec. 3.3.1), with the context's Cholesky factor and its configured solver.  b and x have
 * length ec_state_size() and live in the internal basis of ker E; they may alias. */
EC_API ec_status ec_solve_z(ec_ctx* ctx, const double* b, double* x, int mem);

/* Plain form with EC_SOLVE_INVERSE only: copy out C^{-1}, the inverse of the lower
 * Cholesky factor of Z (N_0 x N_0, column-major, zeros above the diagonal), so that
 * Z^{-1} = C^{-T} C^{-1}. */
EC_API ec_status ec_get_inverse_factor(ec_ctx* ctx, double* W, int mem);

/* Allocation-free solve with an inverse Cholesky factor: x = Winv^T (Winv b), i.e.
 * x = Z^{-1} b when Winv = C^{-1} and Z = C C^T (the same two triangular products
 * the plain form runs every step; see ec_get_inverse_factor).  The paper has no
 * counterpart: this entry point exists for callers that must not allocate device
 * memory themselves -- e.g. a host application whose GPU memory is entirely owned
 * by another allocator (a framework's caching pool or a fixed arena), or a
 * real-time loop that cannot take the latency and implicit synchronisation of
 * cudaMalloc -- and therefore cannot create a context.
 *
 *   n        system size, 1 <= n <= EC_NOALLOC_MAX_N (larger n: EC_ERR_SHAPE, nothing runs)
 *   Winv     device pointer, n x n column-major with leading dimension ldw >= n (at
 *            least ldw (n - 1) + n elements); the lower block triangle is read in
 *            64 x 64 tiles, including the whole diagonal tiles, which must hold zeros
 *            above the diagonal (as ec_get_inverse_factor returns them); blocks above
 *            the block diagonal are never read
 *   b, x     device pointers of length n (b is read, x written; they may alias)
 *   stream   cudaStream_t to enqueue on (NULL = legacy default stream)
 * Allocates nothing: no cudaMalloc or cudaFree is called.  Its scratch is a
 * fixed-size device array inside the library (about 1.1 MB, held on every GPU
 * that loads the library until the process exits).  The first call on a device
 * looks up that array's device address with the device current, and the lookup is
 * repeated on the first call after the device's context was replaced (for example
 * by cudaDeviceReset); make that first call before any stream capture.  All calls share the array, so calls that may
 * overlap on the GPU (different streams without ordering) race and corrupt each
 * other's results.  The call is asynchronous: it returns after enqueueing, and
 * reports only argument and launch errors. */
#define EC_NOALLOC_MAX_N 8192
EC_API ec_status ec_solve_inverse_noalloc(int64_t n, const double* Winv, int64_t ldw,
                                          const double* b, double* x, void* stream);

/* Plain form, no electrodes (m = 0), EC_SOLVE_INVERSE: value and gradient of the probe
 * misfit  J = sum_{k=1..T} || C I^k - v^k ||^2  of a T-step run from the current state,
 * by the discrete adjoint of Eq. time_integration (Sec. 3.3.1):
 *   Z lambda^k = (Z - dt R) lambda^{k+1} + 2 C^T (C I^k - v^k),  k = T..1, lambda^{T+1} = 0.
 * The paper has no gradient; this serves inversion (e.g. resistivity from probe signals).
 *   src        s x (T+1) coil currents, as for ec_run
 *   v          T x p target probe signals (row k-1 = v^k)
 *   ckpt_every states are checkpointed every ckpt_every steps and each segment is
 *              recomputed once in the backward sweep (memory n x (T/ckpt_every + ckpt_every + 2))
 *   J          1 value;  dJ_dRdiag: n values, dJ/dR_ee (R's diagonal entries);
 *   dJ_dsrc    s x (T+1), dJ/ds^k_j.  Any output may be NULL.
 * The state after the call is I^T of the forward run (as after ec_run). */
EC_API ec_status ec_grad(ec_ctx* ctx, int64_t T, const double* src, const double* v,
                         int64_t ckpt_every, double* J, double* dJ_dRdiag, double* dJ_dsrc,
                         int mem);

/* Dense product on the tensor cores: C = bf16(A) bf16(B) with FP32 accumulation (tcgen05,
 * the kernel behind EC_PREC_BF16).  Device pointers, column-major FP64: A is M x K, B is
 * K x N, C is M x N; inputs are rounded to BF16 into temporary buffers.  Synchronous. */
EC_API ec_status ec_gemm_bf16(int64_t M, int64_t N, int64_t K, const double* A, const double* B,
                              double* C, void* stream);

/* FP64-accurate dense product on the tensor cores (the kernel behind the setup's large
 * contractions, Sec. 3.2 and Sec. 3.3.1; the paper, which ran ScaLAPACK on CPUs, has no
 * counterpart):  C = alpha op(A) op(B) + beta C, op(X) = X (t = 0) or X^T (t = 1).
 * Device pointers, column-major FP64 with leading dimensions lda, ldb, ldc; op(A) is
 * M x K, op(B) is K x N.  `lower` holds flags: bit 0 (value 1, M = N) updates only the
 * lower triangle of C; bit 1 (value 2, with alpha = 1, beta = 0 and bit 0 clear) runs the
 * path of the modal snapshot products: op(A)'s slices are cut once into their own buffer
 * (64 KB blocks in the kernel's shared-memory image) and the product reads them, one
 * stream-K launch over all row tiles and K chunks per group of up to 32 columns.
 * Each row of op(A) and column of op(B) is scaled by a power of two and cut into eight
 * 8-bit integer slices held exactly in BF16; the slice products (tcgen05, FP32
 * accumulation kept exact per slice diagonal) are recombined in integer arithmetic.
 * Error per entry: below 2^-60 sqrt(K) max_k|op(A)_ik| max_k|op(B)_kj| plus one FP64
 * rounding per 192-long K chunk, comparable to an FP64 GEMM.  Entries must be finite: a
 * NaN or infinity does not propagate as in an FP64 GEMM but leaves its row of C (column,
 * for op(B)) meaningless; the setup paths refuse non-finite inputs before they reach this
 * product.  Allocates a temporary workspace (about 16 (M + N) K bytes, in panels beyond
 * 4 GB).  Synchronous. */
EC_API ec_status ec_gemm_f64_emulated(int ta, int tb, int64_t M, int64_t N, int64_t K,
                                      double alpha, const double* A, int64_t lda, const double* B,
                                      int64_t ldb, double beta, double* C, int64_t ldc, int lower,
                                      void* stream);

/* Modal form only: selective integration (the decoupled modes can be advanced "in a
 * selective manner", Sec. 2.3).  From now on only the n_keep modes of largest tau are
 * integrated and reconstructed; the others are set to zero and stay there.  For a
 * source-free run the result is the R_i-orthogonal projection of the full trajectory
 * on the kept modes.  1 <= n_keep <= ec_state_size(); n_keep = ec_state_size()
 * restores the full modal form. */
EC_API ec_status ec_set_mode_count(ec_ctx* ctx, int64_t n_keep);

/* Phasors of sampled signals at given frequencies (the Fourier post-processing of the
 * time-domain responses, Sec. 4.6):  X_{j,p} = (2/T) sum_{k<T} y[k][p] exp(-i 2 pi f_j (t0 + k dt)).
 *   y      T x p samples (row-major: row k = all p signals at t0 + k dt, as ec_run writes probes)
 *   freqs  nf frequencies [Hz];  out  nf x p x 2 (real, imaginary), row-major.
 * For a record spanning an integer number of periods of tone f, a signal
 * Im(W exp(i 2 pi f t)) gives X = -i W.  Synchronous; uses the current device. */
EC_API ec_status ec_phasors(int64_t T, int64_t p, const double* y, double t0, double dt,
                            int64_t nf, const double* freqs, double* out, int mem);

/* Copy the context's phase timings (see ec_timing) into *out. */
EC_API ec_status ec_timings(ec_ctx* ctx, ec_timing* out);
/* Wait for the context's stream and report any error raised inside kernels. */
EC_API ec_status ec_sync(ec_ctx* ctx);
/* Extra information about the last error (global pivot index for EC_ERR_NOT_SPD). */
EC_API int64_t ec_last_info(const ec_ctx* ctx);
/* Static English text for a status code (never NULL). */
EC_API const char* ec_error_string(ec_status status);
/* Wait for the context's stream, free everything the context owns, and the context
 * itself.  NULL is a no-op. */
EC_API void ec_destroy(ec_ctx* ctx);

/* Number of CUDA kernels the library has launched in this process, over all
 * contexts (a monotonically increasing counter; take differences). */
EC_API int64_t ec_launch_count(void);

/* Self-test of the bounded kernel-side wait: launches one wait on a flag that
 * nothing sets, with at most spin_limit polls, and stores the status the kernel
 * reported (EC_ERR_TIMEOUT when the bound works) in *code_out. */
EC_API ec_status ec_selftest_wait_timeout(long long spin_limit, int* code_out);

/* Test hook for the out-of-memory paths (failures are made on the host; nothing is
 * injected on the GPU).  With after >= 0, the library's next `after` device
 * allocations succeed and every later one reports failure, as cudaMalloc does when
 * device memory is exhausted: the call that needed it returns EC_ERR_OOM and leaves
 * the context usable for ec_destroy or a new ec_setup.  after < 0 disarms the hook
 * (the default).  Process-wide; not for use while other threads call the library. */
EC_API ec_status ec_selftest_fail_alloc(int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* EDDY_THETA_H */
