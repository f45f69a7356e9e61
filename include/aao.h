/*
 * aao.h -- C ABI of the GB300 (sm_103a) solver for the all-at-once BDF2
 * system of the Riesz fractional diffusion equation
 * (Gu, Zhao, Zhao, Carpentieri, Huang, arXiv:2003.07020).
 *
 * Problem (Sec. 2.1, Eqs. 11-12): find U = [u^1; ...; u^Nt] with
 *     calA U = F,   calA = C (x) I_s - tau I_t (x) K,
 * C the BDF2 time matrix of Eq. 1.7 (BDF1 in its first row), K the
 * fractional-centred-difference Jacobian A = -(kappa/h^alpha) T(g)
 * (Sec. 2.1; Eq. 4.2 in 2D), tau = T/Nt, h = 1/(M+1) on (0,1).
 *
 * Notation: alpha is the fractional order (the paper's gamma); eps is the
 * circulant parameter of the preconditioner (the paper's alpha, Eq. 1.11).
 *
 * Conventions for every call below:
 *   - Vectors are caller-owned DEVICE buffers unless a name ends in _host.
 *     Space-time vectors are double[Nt][M], row-major: row k is time level
 *     k+1, space contiguous (the stacking of Eq. 12).  No alignment beyond
 *     the natural 8 bytes is required.
 *   - The plan owns all workspace (Krylov bases, spectra, tables); it is
 *     allocated in aao_plan_create and released in aao_plan_destroy.
 *   - Work is enqueued on the plan's stream.  aao_matvec and
 *     aao_bc_precond_apply return without synchronising; aao_gmres_solve and
 *     aao_gmres_solve_host synchronise the stream before returning.
 *   - Errors are reported by return code only; aao_last_error gives a
 *     message for the last failing call on a plan.  A plan is not
 *     thread-safe: calls on one plan must not overlap.
 */
#ifndef AAO_H
#define AAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AAO_OK = 0,
  AAO_EINVAL = 1,       /* bad argument (size, pointer, parameter range) */
  AAO_ENOMEM = 2,       /* device or host allocation failed */
  AAO_ECUDA = 3,        /* a CUDA runtime call failed */
  AAO_ENOCONV = 4,      /* solver hit its iteration cap above tolerance */
  AAO_EBREAKDOWN = 5,   /* Krylov breakdown (zero pivot) */
  AAO_ENONFINITE = 6    /* NaN or Inf detected */
} aao_status;

typedef enum {
  AAO_PREC_FP64 = 0,    /* every step in FP64 ("plain") */
  AAO_PREC_MIXED = 1    /* preconditioner steps (a)-(c) in FP32, rest FP64 */
} aao_precision;

typedef enum {
  AAO_INNER_STRANG = 0, /* Strang circulant S of T.  Mixed 1D plans with M <= 8192 apply
                           (lambda_n I + c S)^{-1} as a precomputed L-point circulant spectrum per
                           shifted system (2 FFTs of L); the FP64 path and larger M apply it by
                           Bluestein FFTs of the M-point circulant (4 FFTs of L) */
  AAO_INNER_TAU = 1,    /* natural tau-matrix T - H(T), applied by DST-I (Sec. 3.2), as the COCG
                           preconditioner: Step (b) still solves with T to inner_tol */
  AAO_INNER_TAU_DIRECT = 2 /* the paper's own Step (b) (Sec. 3.2, Eq. 3.9; 2D: Example 2, Eq. 4.5):
                           each shifted system solved once, directly, with T replaced by its natural
                           tau matrix, x_n = (lambda_n I + c tau(T))^{-1} zhat_n by one DST-I pair; no
                           inner iterations (inner_tol and inner_maxit are ignored).  The
                           preconditioner is then P_eps with tau(A) in place of A, a fixed linear
                           operator (usable with aao_bicgstab_solve).  Needs M + 1 (and My + 1) to be
                           powers of two */
} aao_inner_precond;

/* How the Toeplitz product c T v of the matvec (Sec. 3.2) is computed (1D). */
typedef enum {
  AAO_MATVEC_FFT64 = 0, /* FP64 FFT convolution (circulant embedding) */
  AAO_MATVEC_NTT = 1    /* exact integer convolution of the rows quantised to 58-bit fixed point
                           (2^-59 relative to the row's largest entry) by NTTs modulo four primes
                           and CRT */
} aao_matvec_kind;

/*
 * Problem description (Sec. 2.1; 2D: Eq. 4.1-4.2 on (0,1)^2).
 * 1D: unknowns per time level M, vectors double[Nt][M].
 * 2D: K = I (x) K_x + K_y (x) I with x fastest, unknowns per time level
 *     M * My, vectors double[Nt][My][M]; M + 1 and My + 1 must be powers of
 *     two.  Inner preconditioners in 2D: AAO_INNER_STRANG, the 2D Strang
 *     (BCCB) circulant I (x) S_x + S_y (x) I (2D FFTs of the embedding, with
 *     per-system spectra of the BCCB inverses built at plan creation: about
 *     (Nt/2+1) (2 M + 2) (2 My + 2 + My) complex of workspace); AAO_INNER_TAU,
 *     the 2D tau matrix by DSTs; AAO_INNER_TAU_DIRECT (no COCG).
 */
typedef struct {
  int dim;              /* 1 or 2 */
  int64_t M;            /* interior points (x direction in 2D); h = 1/(M+1); M+1 a power of two for AAO_INNER_TAU */
  int64_t Nt;           /* time steps, a power of two >= 4; tau = T/Nt.  The time DFTs keep all Nt rows
                           of a column tile in shared memory, which bounds Nt: at most 4096 with
                           AAO_PREC_MIXED and 2048 with AAO_PREC_FP64 on a GPU with 227 KB per block
                           (larger Nt: AAO_EINVAL at plan creation) */
  double T;             /* final time (> 0) */
  double alpha;         /* fractional order (x direction in 2D), 1 < alpha <= 2 */
  double kappa;         /* diffusion coefficient (x direction in 2D), > 0 */
  double eps;           /* circulant parameter in (0,1]; <= 0 selects min(0.5, 0.5 tau) (Sec. 4) for
                           AAO_PREC_FP64 and max(min(0.5, 0.5 tau), 1/16) for AAO_PREC_MIXED */
  int64_t My;           /* 2D: interior points in y, h_y = 1/(My+1); ignored in 1D */
  double alpha_y;       /* 2D: fractional order in y */
  double kappa_y;       /* 2D: diffusion coefficient in y */
} aao_problem;

#define AAO_COCG_TMEM (-1) /* aao_opts.cocg_threads: the Step (b) kernel with its vectors in tensor memory */

/* Solver options.  aao_default_opts fills the defaults given in brackets. */
typedef struct {
  int restart;          /* FGMRES restart length m [20], 1..64 */
  int max_cycles;       /* restart cycles before AAO_ENOCONV [50] */
  double tol;           /* true relative residual ||F - calA U||/||F|| [1e-10] */
  double inner_tol;     /* COCG relative residual per shifted system [1e-6 mixed, 1e-12 fp64] */
  int inner_maxit;      /* COCG iteration cap per system [200] */
  aao_precision prec;   /* [AAO_PREC_MIXED] */
  aao_inner_precond inner; /* [AAO_INNER_STRANG] */
  int use_graphs;       /* [1] run each restart cycle as one CUDA graph (the Arnoldi steps as
                           conditional nodes, Givens rotations on the device, one host synchronisation
                           per cycle instead of one per step; in 2D the COCG iterations of Step (b)
                           are a conditional WHILE node inside each step); ignored while profiling
                           or while recording pairs.  0: host-driven steps (2D Step (b) then still
                           runs as one graph launch with its WHILE loop, except while profiling) */
  aao_matvec_kind matvec; /* [AAO_MATVEC_NTT] matvec arithmetic: exact-integer convolutions of rows quantised
                           to 58 bits (1D rows; 2D the rows and columns of each time level, one scale per
                           level), or FP64 FFTs */
  int cocg_threads;     /* [0] mixed 1D, M <= 8192: CTA size of the register-resident COCG kernel
                           (64, 128, 256 or 512, at least M / 16), or AAO_COCG_TMEM: the kernel that
                           keeps the COCG vectors in tensor memory (Strang preconditioner,
                           4096 < M <= 8191; the learned warm start still runs on the 512-thread
                           register kernel).  0 picks the tensor-memory kernel where it applies and
                           otherwise times the admissible sizes on the plan's own systems and keeps
                           the fastest (cached per problem shape for the process) */
  int poly_m;           /* [0] 0..16: apply the m-step polynomial preconditioner of Sec. 3.1 (the
                           remark after Thm 3.1) instead of P_eps:
                           P(m) v = sum_{k=0}^{m} (P_eps^{-1} S_eps)^k P_eps^{-1} v,
                           S_eps = (C_eps - C) (x) I, by Horner's rule z <- P_eps^{-1}(v + S_eps z):
                           m + 1 applications of Steps (a)-(c) per preconditioner call (plus n
                           doubles of plan workspace) */
} aao_opts;

/* Result of a solve. */
typedef struct {
  int outer_iters;      /* FGMRES iterations (preconditioner applications) */
  int cycles;           /* restart cycles */
  int inner_iters_max;  /* largest COCG iteration count of any shifted system */
  int matvecs;          /* calA v products, including true-residual checks */
  double true_rel_res;  /* final ||F - calA U||_2 / ||F||_2 computed in FP64 */
  int status_detail;    /* AAO_OK, or the inner failure code that was seen */
  int64_t inner_iters_sum; /* COCG iterations summed over all systems and applications */
  int64_t warm_accepted;   /* shifted systems that started from the learned initial guess
                              (aao_plan_set_warm_start), summed over applications */
} aao_info;

typedef struct aao_plan aao_plan;

/* Fills *opts with the defaults listed in aao_opts for precision prec. */
void aao_default_opts(aao_opts* opts, aao_precision prec);

/*
 * g_k of Eq. 2.4, k = 0 .. n-1, on the HOST in FP64:
 *   g_k = (-1)^k Gamma(1+alpha) / (Gamma(1+alpha/2-k) Gamma(1+alpha/2+k)),
 * evaluated by g_0 = Gamma(1+alpha)/Gamma(1+alpha/2)^2 and the ratio
 * g_{k+1} = g_k (k - alpha/2)/(alpha/2 + k + 1) (from Gamma(z+1) = z Gamma(z)).
 * g_host: caller-owned host array of n doubles.  AAO_EINVAL if n < 1,
 * g_host is NULL or alpha is outside (0, 2].
 */
aao_status aao_setup_coeffs(double alpha, int64_t n, double* g_host);

/*
 * Creates a plan for one problem: host FP64 setup of g_k, the circulant
 * embedding spectrum of T, the eigenvalues lambda_n of C_eps (Eq. 1.6a) for
 * n = 0..Nt/2, the inner preconditioner's spectrum, FFT twiddle tables, and
 * all device workspace: about (2m+6) * 8 * M * Nt bytes for restart m, plus
 * 24 * M * Nt bytes of NTT scratch (AAO_MATVEC_NTT) and, for the mixed Strang
 * path, the per-system spectra of the Strang inverse ((Nt/2+1) * L * 8 bytes,
 * L the embedding length, a power of two >= 2M).  Mixed 1D plans with
 * M <= 8192 launch kernels during creation (those spectra, and the CTA-size
 * autotuner when opts.cocg_threads is 0) and synchronise the stream.
 * cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 * On failure *out is NULL.
 */
aao_status aao_plan_create(const aao_problem* prob, const aao_opts* opts, void* cuda_stream,
                           aao_plan** out);
aao_status aao_plan_destroy(aao_plan* plan);

/* Bytes of device workspace the plan holds. */
size_t aao_plan_workspace_bytes(const aao_plan* plan);

/* Launch shapes the plan uses: *cocg_threads = CTA size of the Step (b) kernel
 * (0 where the shared-memory kernel serves: FP64, M > 8192 or 2D). */
aao_status aao_plan_get_tuning(const aao_plan* plan, int* cocg_threads);  /* AAO_COCG_TMEM: tensor-memory kernel */

/*
 * Right-hand side of Eq. 12: F_1 = tau f^1 + u^0, F_2 = tau f^2 - u^0/2,
 * F_k = tau f^k (k >= 3).  u0_dev: double[M]; f_dev: double[Nt][M] holding
 * f^1 .. f^Nt; F_dev: double[Nt][M] output (may alias f_dev).
 */
aao_status aao_build_rhs(aao_plan* plan, const double* u0_dev, const double* f_dev, double* F_dev);

/*
 * w = calA v (Sec. 3.2): row k of w is sum_{j<=2} C[k,k-j] v_{k-j} - tau K v_k,
 * with the Toeplitz product by circulant embedding.  opts.matvec selects the
 * arithmetic: AAO_MATVEC_NTT (the default in 1D) quantises each row of v to
 * 58-bit fixed point and convolves it exactly by NTTs modulo four primes;
 * AAO_MATVEC_FFT64 (and every 2D plan) uses FP64 FFTs.  Either way the
 * result carries FP64 accuracy.  v_dev, w_dev: double[Nt][M], must not alias.
 */
aao_status aao_matvec(aao_plan* plan, const double* v_dev, double* w_dev);

/*
 * z ~= P_eps^{-1} v by Steps (a)-(c) of Sec. 3.1: (a) scale row k by
 * eps^{k/Nt} and DFT along time (half spectrum n = 0..Nt/2, Sec. 3.2);
 * (b) solve (lambda_n I - tau K) x_n = zhat_n for every n by preconditioned
 * COCG to the plan's inner_tol; (c) inverse DFT along time and unscale.
 * Precision of (a)-(c) follows opts.prec.  v_dev, z_dev: double[Nt][M];
 * they may alias.
 */
aao_status aao_bc_precond_apply(aao_plan* plan, const double* v_dev, double* z_dev);

/*
 * Solves calA U = F by restarted right-preconditioned flexible GMRES with
 * the preconditioner of aao_bc_precond_apply, CGS2 orthogonalisation and
 * Givens rotations (AAO_PREC_FP64: basis and CGS2 in FP64; AAO_PREC_MIXED:
 * the basis in float-float pairs of ~48 bits with CGS2 on the FP32 pipe;
 * Hessenberg matrix, rotations and the update of U in FP64 in both).  Stops
 * when the true relative residual, computed in FP64 at the end of a cycle,
 * is <= opts.tol.
 * F_dev: double[Nt][M]; U_dev: double[Nt][M], initial guess on entry (zero it
 * for x0 = 0), solution on exit.  info may be NULL.  Returns AAO_ENOCONV if
 * max_cycles pass without meeting tol (U then holds the last iterate).
 * Synchronises the plan's stream.
 */
aao_status aao_gmres_solve(aao_plan* plan, const double* F_dev, double* U_dev, aao_info* info);

/*
 * As aao_gmres_solve with HOST buffers: copies F_host to the device, solves
 * from x0 = 0, copies U back to U_host.  Both are double[Nt][M] in host
 * memory (pinned memory gives the fastest copies).
 */
aao_status aao_gmres_solve_host(aao_plan* plan, const double* F_host, double* U_host, aao_info* info);

/*
 * Solves calA U = F by preconditioned BiCGSTAB (van der Vorst; the outer
 * solver of Example 2, Sec. 4) with the preconditioner of
 * aao_bc_precond_apply (use AAO_INNER_TAU_DIRECT, or a tight inner_tol, so
 * that P is a fixed operator; opts.poly_m applies as well).  P^{-1} is applied
 * to the two search directions of each step and U is updated with them, so
 * the recurrence carries the residual of calA U = F; the iteration stops when
 * ||r_k||_2 <= opts.tol ||r_0||_2, tested after every half step (the paper's
 * stopping rule, x0 = U_dev on entry; its Tables 4-6 count these half steps).
 * At most opts.max_cycles * opts.restart iterations (AAO_ENOCONV beyond).
 * The plan's Krylov workspace holds the seven BiCGSTAB vectors, so
 * opts.restart must be >= 7.  U_dev: initial guess on entry, solution on
 * exit.  info (may be NULL): outer_iters = half steps (one preconditioner
 * application each; the paper's Iter is outer_iters / 2), true_rel_res =
 * ||F - calA U||_2 / ||F||_2 recomputed in FP64 at exit, inner statistics as
 * for aao_gmres_solve.  A zero denominator (rho, (r0^, v) or (t, t)) returns
 * AAO_EBREAKDOWN with U at its last update.  Synchronises the stream (several
 * times per iteration: the scalars live on the host).
 */
aao_status aao_bicgstab_solve(aao_plan* plan, const double* F_dev, double* U_dev, aao_info* info);

/*
 * The windowed restart of Sec. 2.2 (the remark after Thm 2.1): the interval
 * [0, n_windows T] is covered by n_windows all-at-once systems of the plan's
 * size (Nt steps of tau = T/Nt each); window q solves Eq. 12 with u^0 = the
 * last time level of window q - 1 (u0_dev for q = 0) by aao_gmres_solve from
 * x0 = 0.  f_dev: double[n_windows Nt][M] holding f at every time level
 * t_k = (k+1) tau, k < n_windows Nt; U_dev: double[n_windows Nt][M], the
 * solution at those levels (must not alias f_dev).  info (may be NULL):
 * outer_iters, matvecs, cycles, inner_iters_* summed over the windows,
 * true_rel_res the largest window's.  Stops at the first window that fails.
 * Synchronises the stream.
 */
aao_status aao_solve_windows(aao_plan* plan, int n_windows, const double* u0_dev, const double* f_dev,
                             double* U_dev, aao_info* info);

/*
 * Solves n independent problems (different M, Nt, alpha, kappa, precision)
 * at once on the current device.  F[i], U[i]: device vectors of plans[i]'s
 * shape; U[i] is the initial guess on entry.  infos (may be NULL) receives
 * n results.  Returns AAO_OK if every solve did, else the first failing
 * status (the other solves still complete).  Two schedules:
 *   - max_workers <= 0 and plans that are all 1D AAO_PREC_MIXED with the
 *     register-resident Step (b) (M <= 8192, AAO_INNER_STRANG or
 *     AAO_INNER_TAU of one kind, the same restart length, no warm start,
 *     recording, profiling or poly_m): the restart cycles of all instances
 *     run in lockstep, each instance's Steps (a), (c), matvec and CGS2 on its
 *     own stream and the shifted solves of ALL instances as ONE kernel launch
 *     per Arnoldi step (a work list of (instance, system) pairs, the CTA size
 *     the largest of the plans' cocg_threads; results equal single solves
 *     when every plan has that CTA size); Givens rotations on the device, one
 *     host synchronisation per step;
 *   - otherwise (or max_workers > 0): each plan runs aao_gmres_solve on its
 *     own non-blocking stream from a pool of max_workers host threads (<= 0:
 *     32), largest problems first.
 * Each plan's stream is synchronised first and restored afterwards.
 */
aao_status aao_solve_batched(int n, aao_plan* const* plans, const double* const* F, double* const* U,
                             aao_info* infos, int max_workers);

/*
 * Tracing.  When profiling is on, every kernel the plan launches is
 * bracketed by CUDA events recorded on the plan's stream, and the elapsed
 * times are accumulated per stage.  Stages: 0 matvec (Sec. 3.2), 1 Step (a)
 * time DFT, 2 Step (b) shifted solves, 3 Step (c) inverse time DFT,
 * 4 Gram-Schmidt and other vector kernels, 5 learned warm-start inference.  aao_plan_get_profile
 * synchronises the stream, fills ms[i] (milliseconds) and launches[i] for
 * i < AAO_NUM_STAGES, and resets the counters when reset != 0.
 */
#define AAO_NUM_STAGES 6
aao_status aao_plan_set_profiling(aao_plan* plan, int on);
aao_status aao_plan_get_profile(aao_plan* plan, double* ms, int64_t* launches, int reset);

/*
 * Per-system record of the most recent Step (b) (Sec. 3.1: the Nt/2 + 1
 * shifted solves (lambda_n I - tau K) x_n = y_n of one preconditioner
 * application, n = 0 .. Nt/2).  n_sys must equal Nt/2 + 1.  iters_host[n]
 * receives the inner iterations of system n (0 for the direct tau solve),
 * flags_host[n] its outcome: 0 converged, 1 iteration cap reached,
 * 2 breakdown (|u^T w| at rounding level of ||u|| ||w|| for a COCG divisor),
 * 3 non-finite values, plus 4 when the learned warm start was accepted.
 * Either pointer may be null.  Synchronises the plan's stream; AAO_EINVAL
 * for a bad n_sys.
 */
aao_status aao_plan_get_inner_record(aao_plan* plan, int n_sys, int* iters_host, int* flags_host);

/*
 * The preconditioner apply of aao_bc_precond_apply (mixed precision only)
 * without a plan and without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, e.g. code
 * running inside another library's memory pool or a pipeline that must not
 * synchronise the device through an allocation.  Scratch spectrum and tables
 * live in one fixed 16 MiB device array of the library, held by every GPU
 * that loads it until the process exits; problems whose scratch
 * (nsys * M * 8 bytes plus tables, nsys = Nt/2 + 1) exceeds it are rejected
 * with AAO_EINVAL.  Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress).  Each call writes its tables into the array with small kernels that carry them
 * as launch parameters, so it copies nothing from pageable host memory and
 * does not wait for work already queued on cuda_stream.  Calls share the
 * array, so calls that overlap on the GPU race.  The shifted solves are not
 * reported: a system that reaches opts.inner_maxit without meeting
 * opts.inner_tol leaves its last iterate in z without an error code (use a
 * plan and aao_gmres_solve's info for that).  opts.prec must be
 * AAO_PREC_MIXED; v_dev, z_dev: double[Nt][M] on the device; cuda_stream as
 * in aao_plan_create.  Errors: see aao_last_error(NULL).
 */
aao_status aao_bc_precond_apply_noalloc(const aao_problem* prob, const aao_opts* opts,
                                        const double* v_dev, double* z_dev, void* cuda_stream);

/*
 * Learned warm start for Step (b).  The paper solves every shifted system
 * (lambda_n I - tau K) x = zhat_n from x0 = 0; it has no learned component.
 * An aao_fno is a Fourier neural operator that predicts x0 from
 * (zhat_n, lambda_n, alpha) and is trained on the GPU on (zhat_n, x_n) pairs
 * that the solver itself records (aao_plan_record_pairs).
 *
 * Architecture, per grid point i = 0..M-1 of one system with right-hand
 * side b (channels last):
 *   features [Re bh_i, Im bh_i, Re lambda, Im lambda, alpha, (i+1)/(M+1)],
 *   bh = b / ||b||;  lift 6 -> 32;  4 Fourier layers, each: DFT of every
 *   channel truncated to modes k < 16, a complex 32 x 32 matrix per mode,
 *   inverse (real part, modes k >= 1 counted twice, divided by M), plus a
 *   point-wise 32 x 32 matrix and bias, GELU (erf form) after all but the
 *   last layer;  projection 32 -> 2 giving y;  x0 = ||b|| (y_0 + i y_1).
 * Parameters: one flat float array of aao_fno_num_params() values in the
 * order lift W (32 x 6, row-major), lift bias (32), then per layer the
 * spectral weights (16 x 32 x 32 complex as [mode][out][in][re, im]), the
 * point-wise W (32 x 32, [out][in]), the bias (32), then projection W
 * (2 x 32) and bias (2).  Inference and training read the weights as BF16
 * and accumulate in FP32; training keeps FP32 master weights and Adam
 * moments.  The loss of one sample with target t = x / ||b|| is
 * sum |y - t|^2 / sum |t|^2, averaged over the batch.
 *
 * Buffers: b, x: complex float [B][M] (re, im interleaved) on the device;
 * lambda: complex double [B]; alpha: float [B]; all device pointers.
 * cuda_stream as in aao_plan_create.  Calls on one model must not overlap
 * (its activations are reused).  Errors: see aao_last_error(NULL).
 */
typedef struct aao_fno aao_fno;

int64_t aao_fno_num_params(void);

/* Model for grid size M (32 <= M <= 8191) and batches of up to max_batch
 * systems; weights drawn from a seeded scaled Gaussian (fan-in), biases 0. */
aao_status aao_fno_create(int64_t M, int max_batch, uint64_t seed, aao_fno** out);
aao_status aao_fno_destroy(aao_fno* fno);

/* Host float[aao_fno_num_params()] in the flat order above.  set_params
 * also resets the optimiser.  get_params returns the FP32 master weights,
 * or, if bf16_rounded != 0, the BF16 values the kernels read. */
aao_status aao_fno_set_params(aao_fno* fno, const float* params_host);
aao_status aao_fno_get_params(aao_fno* fno, float* params_host, int bf16_rounded);

/* Save / load the FP32 weights: one line of JSON (format, version, sizes,
 * number of parameters, Adam step count) followed by the parameters as
 * little-endian float32.  load accepts a file written for any M. */
aao_status aao_fno_save(aao_fno* fno, const char* path);
aao_status aao_fno_load(aao_fno* fno, const char* path);

/* x0 = prediction for B systems (1 <= B <= max_batch). */
aao_status aao_fno_predict(aao_fno* fno, int B, const void* b_dev, const void* lambda_dev,
                           const float* alpha_dev, void* x0_dev, void* cuda_stream);

/* Mean loss over the batch and, if grad_host != NULL, its gradient in the
 * flat order (host float[aao_fno_num_params()]); synchronises the stream. */
aao_status aao_fno_loss_grad(aao_fno* fno, int B, const void* b_dev, const void* lambda_dev,
                             const float* alpha_dev, const void* x_dev, double* loss, float* grad_host,
                             void* cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * batch; *loss (may be NULL) receives the batch loss before the step. */
aao_status aao_fno_train_step(aao_fno* fno, int B, const void* b_dev, const void* lambda_dev,
                              const float* alpha_dev, const void* x_dev, float lr, double* loss,
                              void* cuda_stream);

/*
 * Trains fno for `steps` Adam steps (as aao_fno_train_step) on n_pairs
 * stored pairs (b, lambda, alpha, x as in aao_fno_loss_grad, n_pairs rows
 * each; typically recorded by aao_plan_record_pairs), batch systems per
 * step (1 <= batch <= max_batch, batch <= n_pairs), with the cosine
 * learning-rate schedule lr_t = lr0 (1 + cos(pi t / steps)) / 2,
 * t = 0 .. steps-1.  Batches: with seed 0, step t takes the contiguous
 * pairs [o, o + batch), o = (t batch) mod (n_pairs - batch) (the pairs
 * should then be stored in random order; o = 0 when n_pairs = batch);
 * with seed != 0, every epoch of floor(n_pairs / batch) steps visits the
 * pairs in a fresh permutation (Fisher-Yates driven by SplitMix64 from
 * seed), gathered into model-owned buffers (allocated on the first such
 * call).  losses_host (may be NULL): host double[steps] receiving each
 * step's batch loss before its update.  Runs without host synchronisation
 * per step; synchronises the stream at the end when losses_host is given.
 */
aao_status aao_fno_train(aao_fno* fno, int64_t n_pairs, const void* b_dev, const void* lambda_dev,
                         const float* alpha_dev, const void* x_dev, int steps, int batch, float lr0, uint64_t seed,
                         double* losses_host, void* cuda_stream);

/*
 * Attaches fno (not owned; NULL detaches) to a 1D AAO_PREC_MIXED plan with
 * M <= 8191 equal to the model's M and Nt/2 + 1 <= its max_batch.  Every
 * Step (b) then predicts x0 for all shifted systems and COCG starts system n
 * from its prediction only if the FP32 residual ||zhat_n - A_n x0|| is
 * below ||zhat_n||, else from 0; the stopping test stays relative to
 * ||zhat_n||.  The model must stay alive while attached and must not be
 * used by another call meanwhile.
 */
aao_status aao_plan_set_warm_start(aao_plan* plan, aao_fno* fno);

/*
 * Records training pairs from every later Step (b) of a 1D AAO_PREC_MIXED
 * plan: system n's right-hand side zhat_n (b_dev), its COCG solution
 * (x_dev, both complex float [capacity][M]) and lambda_n (lambda_dev,
 * complex double [capacity]) are appended until capacity pairs are stored.
 * capacity 0 (or NULL buffers) stops recording; a new call restarts the
 * count.  aao_plan_recorded_pairs returns the number stored so far.
 */
aao_status aao_plan_record_pairs(aao_plan* plan, int64_t capacity, void* b_dev, void* x_dev, void* lambda_dev);
aao_status aao_plan_recorded_pairs(const aao_plan* plan, int64_t* count);

/* Message for the last failing call on plan (or on plan creation, or on a
 * call without a plan, if NULL). */
const char* aao_last_error(const aao_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* AAO_H */
