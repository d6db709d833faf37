/*
 * cofem.h — C ABI of libcofem, a GB300 (sm_103a) implementation of the hot
 * path of covariance-free expectation-maximisation (CoFEM) for sparse Bayesian
 * learning (Lin, Song, Bilgic, Ba, "Covariance-Free Sparse Bayesian Learning").
 *
 * Problem (Sec. I, Eq. sparse-coding; Sec. II-A, Eq. model):
 *     y = Phi z + eps,  z ~ N(0, diag(alpha)^-1),  y | z ~ N(Phi z, beta^-1 I),
 *     Phi in R^{N x D}.
 * One fit runs Alg. 1 (CovarianceFreeEM): for t = 1..T_em it solves the K+1
 * systems A X = B,  A = beta Phi^T Phi + diag(alpha^(t)),
 *     B = [beta Phi^T y | p_1 .. p_K]  (Sec. III-A, Eq. mat-eq; mu in column 0),
 * by Alg. 2 (ParallelConjGradient) with the diagonal preconditioner
 * M = diag(beta theta + alpha) (Sec. III-C), forms mu = x_0 and the diagonal
 * estimate s_j = (1/K) sum_k p_kj x_kj (Eq. diag-estimate) and, for t < T_em,
 * applies the M-step alpha_j = 1 / (mu_j^2 + s_j) (Eq. mstep with s for Sigma_jj;
 * or the rectified Gaussian prior's M-step, see COFEM_PRIOR_RECTIFIED).
 *
 * Conventions for every function below:
 *  - Return value is a cofem_status; COFEM_OK (0) on success.  No C++
 *    exception crosses this boundary.  On failure, cofem_last_error() returns a
 *    human-readable message for the calling thread.
 *  - "Device or host" pointers are classified with cudaPointerGetAttributes;
 *    host memory may be pageable or pinned.  "Device" pointers must be CUDA
 *    device (or managed) memory of the handle's device; device memory of
 *    another GPU is rejected with COFEM_ERR_INVALID_ARG where the entry point
 *    checks it (the operator output, the allocation-free entry point).
 *  - The caller owns every buffer it passes; the library never frees them.
 *    The library owns the memory it allocates inside a handle.
 *  - Floating-point inputs are IEEE binary32; vectors are dense, unit stride.
 *  - Calls on one handle are serialised on that handle's stream; different
 *    handles may be used from different threads concurrently.
 *  - Errors in arguments are detected before any device work is enqueued.
 */
#ifndef COFEM_H
#define COFEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COFEM_API_VERSION 1

typedef int cofem_status;
#define COFEM_OK               0
#define COFEM_ERR_INVALID_ARG  1  /* bad size, null pointer, unsupported combination */
#define COFEM_ERR_NOMEM        2  /* device allocation failed / over the memory budget */
#define COFEM_ERR_CUDA         3  /* a CUDA runtime call failed (message has details) */
#define COFEM_ERR_NONFINITE    4  /* NaN/Inf in inputs (a CG breakdown during a fit is not an
                                     error: the column is frozen and COFEM_FLAG_BREAKDOWN set) */
#define COFEM_ERR_UNSUPPORTED  5  /* no sm_103a device, or feature not built */
#define COFEM_ERR_NOT_FOUND    6  /* unknown ticket (serving) */

/* Dictionary kinds (Sec. V-A "Dictionary"). */
#define COFEM_OP_DENSE     0  /* explicit N x D matrix, row-major (Phi_ij at phi[i*D + j]) */
#define COFEM_OP_TOEPLITZ  1  /* causal convolution, N = D: (Phi v)_i = sum_{tau<L} h[tau] v[i-tau];
                                 column j of Phi is h delayed by j and truncated at N (Sec. V-A, VI-A) */
#define COFEM_OP_DCT       2  /* Phi = M Omega^-1: N rows of the inverse orthonormal DCT-II of size D
                                 (Sec. V-A "DCT"); created with cofem_create_dct */

/* Storage / multiply precision of a dense Phi (the CG state is always FP32,
 * CG inner products always FP64). */
#define COFEM_F32   0  /* Phi kept in FP32; products in FP32 FMA on the CUDA cores */
#define COFEM_BF16  1  /* Phi quantised once to bfloat16 (round to nearest even); the
                          method then runs exactly on that quantised dictionary (the
                          vector block enters the tensor cores as three bf16 terms) */
#define COFEM_FP8_E4M3 3 /* Phi stored as FP8 E4M3 codes with per-row FP32 scales:
                          s_i = max_j |Phi_ij| / 448, code = E4M3(Phi_ij / s_i) (round to
                          nearest even, saturating); the method runs on
                          Phi~_ij = s_i code_ij.  The codes are widened to BF16 in shared
                          memory (exactly) for the tensor cores; the vector block is split
                          into three bf16 terms as in COFEM_BF16.  Needs 3(K+1) <= 128. */
#define COFEM_F32_TF32X3 2 /* Phi kept in FP32; products on the tensor cores with the
                          error-compensated TF32 split: x = x_hi + x_lo for the
                          dictionary and the vector block, x_hi and x_lo rounded to
                          TF32, all four partial products accumulated in FP32
                          (about 2^-22 relative error per product) */

/* Preconditioner theta (Sec. III-C): M = diag(beta theta + alpha). */
#define COFEM_PRECOND_JACOBI 0  /* theta_j = sum_i Phi_ij^2  (M_jj = A_jj) */
#define COFEM_PRECOND_ONE    1  /* theta_j = 1 (the paper's experiments, Sec. V-C) */
#define COFEM_PRECOND_NONE   2  /* M = I: unpreconditioned CG (the comparison of the paper's
                                   preconditioner study, Sec. V empirical insights, Fig. 3b) */

/* CG stopping rule (Alg. 2). */
#define COFEM_CONV_PER_COLUMN 0  /* column q stops (and is frozen) once ||r_q|| <= tol ||b_q|| */
#define COFEM_CONV_FROBENIUS  1  /* all columns stop once ||R||_F <= tol ||B||_F (as printed in Alg. 2) */

/* Prior of the weights z_j (selects the M-step).  GAUSSIAN: N(0, 1/alpha_j),
 * alpha_j = 1 / (mu_j^2 + s_j) (Alg. 1).  RECTIFIED: the rectified Gaussian
 * prior of the non-negativity subsection of Sec. III; alpha_j = 1 / E[z_j^2]
 * with E[z_j^2] the second moment of N(mu_j, s_j) restricted to z_j >= 0,
 * mu_j^2 + s_j + mu_j sqrt(2 s_j / pi) / erfcx(-mu_j / sqrt(2 s_j)) (the
 * printed formula with its third term's factor 2 restored; no term where
 * s_j <= 0), evaluated in FP64.  Both floor the moment at 1/alpha_max.  mu is
 * the Gaussian posterior mean in both cases. */
#define COFEM_PRIOR_GAUSSIAN  0
#define COFEM_PRIOR_RECTIFIED 1

/* Fit flags (bit set in *flags). */
#define COFEM_FLAG_CG_NOT_CONVERGED 1u /* some EM iteration hit cg_maxit with a column still active */
#define COFEM_FLAG_ALPHA_CLAMPED    2u /* some mu_j^2 + s_j fell below 1/alpha_max and was clamped */
#define COFEM_FLAG_BREAKDOWN        4u /* p^T A p <= 0 or non-finite in some column (column frozen) */
#define COFEM_FLAG_DEVICE_TIMEOUT   8u /* a bounded on-device wait gave up (the call returns COFEM_ERR_CUDA) */

typedef struct cofem_opts {
    int precision;            /* COFEM_F32 | COFEM_BF16 | COFEM_F32_TF32X3 | COFEM_FP8_E4M3 (the
                                 last three dense only) */
    int precond;              /* COFEM_PRECOND_JACOBI | COFEM_PRECOND_ONE */
    int conv;                 /* COFEM_CONV_PER_COLUMN | COFEM_CONV_FROBENIUS */
    int rr_period;            /* precision form (0 = off): every rr_period CG iterations the
                                 active columns take R <- B - A X computed accurately (see
                                 residual_path and cofem_true_residuals),
                                 with X held as an exact FP32 pair; and when the CG loop
                                 ends, every column's true residual is checked against
                                 cg_tol: a column that misses it restarts from that
                                 residual (P <- M^-1 R) and CG goes on within cg_maxit.
                                 Needs products that are exact on the stored dictionary:
                                 COFEM_F32, COFEM_BF16, COFEM_FP8_E4M3 or a convolution
                                 dictionary (UNSUPPORTED with COFEM_F32_TF32X3, whose split
                                 holds Phi to about 2^-22 only) */
    double alpha_max;         /* alpha_j = 1 / max(mu_j^2 + s_j, 1/alpha_max); default 1e12 */
    unsigned long long seed;  /* probe seed: p_{t,k,j} from Philox4x64-10 with key (seed, 0),
                                 counter (j >> 8, k, t, 0), bit j & 255 (1 -> -1, 0 -> +1) */
    void* stream;             /* cudaStream_t to run on; NULL = a stream owned by the handle */
    int use_graph;            /* 1 (default): the whole fit is one CUDA-graph launch whose EM and
                                 CG loops are device-side conditional WHILE nodes;
                                 0: host-driven loop (one host sync per CG iteration) */
    int dense_path;           /* BF16 dense operator: COFEM_PATH_AUTO (default),
                                 COFEM_PATH_TWO_PASS or COFEM_PATH_SINGLE_PASS */
    int max_sms;              /* upper bound on the SMs the handle's persistent operator
                                 kernels occupy (0 = all): lets concurrent fits share the GPU */
    int overlap_launch;       /* 1 (default): the kernels of the CG step after the first use
                                 programmatic dependent launch (a kernel starts, and the dense
                                 GEMMs prefetch dictionary tiles, while its predecessor
                                 finishes; data dependences still wait for completion);
                                 0: plain stream order */
    int prior;                /* COFEM_PRIOR_GAUSSIAN (default) | COFEM_PRIOR_RECTIFIED */
    int check_residual;       /* 1: measure every column's true relative residual
                                 ||B - A X|| / ||B|| (accurately, as for rr_period) when
                                 each E-step's CG loop ends, without acting on it; read it
                                 with cofem_true_residuals.  X is then held as the FP32
                                 pair as well.  0 (default): only when rr_period > 0. */
    int warm_start;           /* 1: warm start with probe reuse (beyond the paper, which
                                 starts every E-step at X = 0 with fresh probes): every
                                 E-step draws the probes of t = 1, and E-step t >= 2 starts
                                 its K+1 columns from the previous E-step's X (R = B - A X,
                                 one extra operator application per E-step).  0 (default):
                                 Alg. 1 and Alg. 2 as printed. */
    int toeplitz_path;        /* convolution dictionary: COFEM_TOEPLITZ_AUTO (default: the
                                 direct form, the faster one on GB300 so far),
                                 COFEM_TOEPLITZ_DIRECT (tiled direct convolution, O(L) per
                                 output) or COFEM_TOEPLITZ_FFT (overlap-save FFTs of 8192
                                 points in shared memory, O(log F) per output, the paper's
                                 method for this dictionary, Sec. VI-A) */
    int residual_path;        /* how the precision form computes its accurate residual
                                 B - A X (rr_period > 0 or check_residual = 1):
                                 COFEM_RESIDUAL_AUTO (default: SLICED where it applies,
                                 else FP32_PAIRS), COFEM_RESIDUAL_FP32_PAIRS or
                                 COFEM_RESIDUAL_SLICED (see below) */
} cofem_opts;

/* Accurate residual forms (the precision form's B - A X; not in the paper).
 * FP32_PAIRS: X as the FP32 pair X + Xlo, A X with compensated FP32-pair
 * products on the CUDA cores (TwoProduct and TwoSum, about 2^-48 relative
 * error), every dictionary kind.  SLICED: BF16 or FP8 E4M3 dense dictionaries
 * with K + 1 <= 48 and N, D <= 40960: both products of A X = beta Phi~^T
 * (Phi~ X) + alpha X from exact integer slices on the tensor cores (each
 * dictionary entry, or FP8 code, as three signed 8-bit digits relative to a
 * power of two per dictionary row, or per column for Phi~^T; each entry of X
 * and of Phi~ X as five relative to a power of two per column; digit products
 * summed exactly in integers; the FP8 row scales applied to Phi~ X in FP64),
 * relative error about 2^-38 of sum_k |Phi~_ik| |x_k| per product.  Requesting SLICED where it does not apply makes the first fit
 * fail with COFEM_ERR_UNSUPPORTED. */
#define COFEM_RESIDUAL_AUTO       0
#define COFEM_RESIDUAL_FP32_PAIRS 1
#define COFEM_RESIDUAL_SLICED     2

#define COFEM_TOEPLITZ_AUTO   0
#define COFEM_TOEPLITZ_DIRECT 1
#define COFEM_TOEPLITZ_FFT    2

/* Dense BF16 operator forms.  TWO_PASS streams the dictionary for Phi V and a
 * transposed copy for Phi^T T (2 N D bytes of HBM per application).
 * SINGLE_PASS reads each dictionary tile from HBM once: a cooperative kernel
 * (one CTA per SM) forms Phi V for a wave of rows, then Phi^T T from the same
 * tiles while they are still in L2; it needs 3(K+1) <= 112, at most two
 * 128-column tiles of D per SM, and occupies the whole GPU while it runs.
 * AUTO takes TWO_PASS (on GB300 the two-pass kernels are faster so far: the
 * single-pass kernel is bound by its shared-memory fill, not by HBM).
 * Requesting SINGLE_PASS where it does not apply makes the first fit or
 * application fail with COFEM_ERR_UNSUPPORTED. */
#define COFEM_PATH_AUTO        0
#define COFEM_PATH_TWO_PASS    1
#define COFEM_PATH_SINGLE_PASS 2

/* Fill *o with the defaults: F32, Jacobi, per-column, rr_period 0,
 * alpha_max 1e12, seed 2, stream NULL, use_graph 1, dense_path AUTO, max_sms 0,
 * overlap_launch 1, prior GAUSSIAN, check_residual 0, warm_start 0, toeplitz_path AUTO,
 * residual_path AUTO. */
void cofem_default_opts(cofem_opts* o);

/* Create a handle for one dictionary (step a0: upload, optional BF16
 * quantisation, theta).
 *   N, D   : Phi is N x D (TOEPLITZ: N must equal D).  1 <= N, D <= 2^31 - 1.
 *   kind   : COFEM_OP_DENSE or COFEM_OP_TOEPLITZ (a DCT dictionary: cofem_create_dct).
 *   phi    : DENSE: N*D floats, row-major; TOEPLITZ: the filter h[0..L).
 *            Host or device; copied (and quantised) into memory the handle owns.
 *   L      : TOEPLITZ filter length, 1 <= L <= 1024 and L <= N; must be 0 for DENSE.
 *   opts   : NULL for defaults.
 * Errors: INVALID_ARG for bad sizes/kind/pointers, NONFINITE if phi holds
 * NaN/Inf, NOMEM, CUDA, UNSUPPORTED (no sm_103a device). */
cofem_status cofem_create(struct cofem_ctx** out, long long N, long long D, int kind,
                          const float* phi, long long L, const cofem_opts* opts);

/* Create a handle for the DCT dictionary of Sec. V-A: Phi = M Omega^-1, Omega
 * the orthonormal DCT-II of size D (Omega_kn = c_k cos(pi k (2n+1) / 2D),
 * c_0 = sqrt(1/D), c_k = sqrt(2/D)), M keeping the N rows rows[0..N) of
 * Omega^-1 v = Omega^T v.  Phi is never formed: Phi v and Phi^T u are a
 * DCT-III and a DCT-II of length D, each a complex FFT of length D/2 in one
 * thread block's shared memory, O(D log D) per column.
 *   D    : a power of two, 16 <= D <= 32768.
 *   rows : N distinct indices in [0, D), 1 <= N <= D (host or device ints).
 *   opts : precision COFEM_F32 only; rr_period and check_residual must be 0
 *          (UNSUPPORTED otherwise).
 * Errors: INVALID_ARG (sizes, repeated or out-of-range rows), UNSUPPORTED,
 * NOMEM, CUDA. */
cofem_status cofem_create_dct(struct cofem_ctx** out, long long N, long long D, const int* rows,
                              const cofem_opts* opts);

/* Run one CoFEM fit (Alg. 1 with Alg. 2): steps a1-a8 of the hot path.
 *   y         : N floats (host or device).
 *   beta      : noise precision, > 0.
 *   alpha0    : D floats (host or device) or NULL for alpha^(1) = 1 (Alg. 1 initialisation).
 *   K         : probes per EM iteration, 1 <= K <= 63 (Q = K + 1 systems).
 *   T_em      : EM iterations, >= 1 (T_em E-steps, T_em - 1 M-steps).
 *   cg_tol    : > 0, relative residual tolerance of Alg. 2.
 *   cg_maxit  : >= 1, the U of Alg. 2.
 *   mu, s     : D floats each (host or device): mu and s of the last E-step.
 *   alpha     : D floats (host or device): alpha^(T_em), the precisions used in the
 *               last E-step (Alg. 1 return value).
 *   cg_iters  : T_em ints (host or device) or NULL: CG iterations in each EM iteration.
 *   flags     : host unsigned or NULL: COFEM_FLAG_* bits.
 * Blocks until the results are written.  Non-convergence is not an error
 * (Alg. 2 returns X after U steps); it is reported in flags.  Errors:
 * INVALID_ARG, NONFINITE (y, alpha0 or beta non-finite), NOMEM, CUDA. */
cofem_status cofem_fit(struct cofem_ctx* h, const float* y, double beta, const float* alpha0,
                       int K, int T_em, double cg_tol, int cg_maxit,
                       float* mu, float* s, float* alpha, int* cg_iters, unsigned* flags);

/* Multi-task CoFEM (the multi-task subsection of Sec. III) with the handle's
 * dictionary shared by the L tasks (multiple measurement vectors): the tasks
 * share alpha (and beta), and their L (K+1) systems, task l's columns being
 * l (K+1) .. l (K+1) + K, are solved together by one batched Alg. 2 with the
 * shared preconditioner M = beta theta + alpha and per-column stopping.  Each
 * task draws its own probes (the counter's last word is l; task 0 draws the
 * probes of cofem_fit).  M-step: alpha_j = L / sum_l (mu_lj^2 + s_lj), floored
 * at 1/alpha_max.
 *   L         : tasks, >= 1, with L (K+1) <= 64 (K >= 1).
 *   Y         : L x N floats, row l = y_l (host or device).
 *   mu, s     : L x D floats each, row l = task l (host or device).
 *   alpha     : D floats: the shared alpha^(T_em).
 *   cg_iters  : T_em ints or NULL: CG iterations of each E-step's batched
 *               loop (the largest over the tasks' columns).
 * Everything else as cofem_fit; L = 1 is cofem_fit.  Errors: as cofem_fit,
 * and UNSUPPORTED for L > 1 with the rectified prior (its multi-task M-step
 * is not defined here). */
cofem_status cofem_fit_multitask(struct cofem_ctx* h, int L, const float* Y, double beta, const float* alpha0,
                                 int K, int T_em, double cg_tol, int cg_maxit, float* mu, float* s,
                                 float* alpha, int* cg_iters, unsigned* flags);

/* Release the handle and all memory it owns.  NULL is accepted. */
cofem_status cofem_destroy(struct cofem_ctx* h);

/* Static string for a status code. */
const char* cofem_status_string(cofem_status s);

/* Message describing the last failure on the calling thread ("" if none). */
const char* cofem_last_error(void);

/* ---- Step-level entry points (one row of the hot path each; used for
 * ---- parity checks of the individual steps).  All run on the handle's
 * ---- stream and block until done. */

/* Step a2: probe block P (K x D floats, row k-1 = p_k at EM iteration t, entries
 * +-1) written to `out` (device).  K >= 1, D >= 1, t >= 0. */
cofem_status cofem_probe_fill(unsigned long long seed, int t, int K, long long D,
                              float* out, void* stream);

/* Step a4 (Alg. 2 "Apply matrix"): Psi = A V = beta Phi^T (Phi V) + diag(alpha) V
 * for a block of Q vectors.  V and Psi are Q x D row-major (row q = vector q),
 * alpha is D floats; all three device pointers.  1 <= Q <= 64.  If pi is not
 * NULL, pi[q] = v_q^T A v_q is written there (host, Q doubles). */
cofem_status cofem_apply_operator(struct cofem_ctx* h, const float* V, int Q,
                                  const float* alpha, double beta, float* Psi, double* pi);

/* Step a0: theta as used by the preconditioner (D floats, host or device). */
cofem_status cofem_get_theta(struct cofem_ctx* h, float* theta);

/* Step a1: b = beta Phi^T y (y: N floats, b: D floats; host or device). */
cofem_status cofem_phit_y(struct cofem_ctx* h, const float* y, double beta, float* b);

/* Step a4 timing: run the operator kernels of a K+1 = Q column fit `reps` times
 * on the handle's current CG direction block, in the launch configuration a fit
 * uses, bracketed by CUDA events on the handle's stream.  *ms_per_apply gets the
 * mean event time of one application (all operator kernels of one CG step).
 * Requires a previous cofem_fit (or cofem_apply_operator) with the same Q. */
cofem_status cofem_time_operator(struct cofem_ctx* h, int Q, int reps, double* ms_per_apply);

/* ---- Serving: continuous batching of independent fits ----
 * A server runs up to max_slots fits at once, each on its own CUDA stream, so
 * their kernels overlap on the GPU.  Requests are admitted in FIFO order as soon
 * as a slot is idle and the request's device-memory estimate
 * (cofem_estimate_bytes) fits in the unused part of hbm_budget_bytes; each fit
 * is the same computation as cofem_create + cofem_fit (one graph launch with
 * device-side EM and CG loops), so a request gives the same result alone and
 * among others.  The server uses the device that is current when it is created. */
typedef struct cofem_request {
    int kind;                 /* COFEM_OP_DENSE | COFEM_OP_TOEPLITZ */
    long long N, D, L;        /* as cofem_create */
    const float* phi;         /* as cofem_create (host or device) */
    const float* y;           /* N floats (host or device) */
    double beta;
    const float* alpha0;      /* D floats or NULL */
    int K, T_em;
    double cg_tol;
    int cg_maxit;
    int precision, precond, conv, rr_period;   /* as cofem_opts */
    double alpha_max;         /* <= 0 means 1e12 */
    unsigned long long seed;
    float* mu;                /* outputs, as cofem_fit (host or device) */
    float* s;
    float* alpha;
    int* cg_iters;            /* T_em ints or NULL */
    int max_sms;              /* as cofem_opts (0 = all SMs) */
    int prior;                /* as cofem_opts (COFEM_PRIOR_*) */
} cofem_request;              /* every pointer must stay valid until the ticket completes */

typedef struct cofem_result {
    cofem_status status;      /* status of the fit (COFEM_OK or the failing call's code) */
    unsigned flags;           /* COFEM_FLAG_* of the fit */
    double queue_ms;          /* submit -> a worker started the request */
    double run_ms;            /* start -> results written */
    char message[160];        /* error text when status != COFEM_OK */
} cofem_result;

typedef struct cofem_server cofem_server;

/* Device bytes a request is admitted with (an upper estimate of what
 * cofem_create + cofem_fit allocate for it). */
long long cofem_estimate_bytes(int kind, long long N, long long D, long long L, int precision, int K);

/* Start a server with max_slots workers (1..256) and an HBM budget in bytes. */
cofem_status cofem_server_create(cofem_server** out, long long hbm_budget_bytes, int max_slots);

/* Start a server in packed mode: the CG steps of all admitted fits run in
 * shared launches (instead of one fit per stream).  prep_threads (1..64)
 * threads create each request's handle and run its prologue (dictionary
 * copies and images, b = beta Phi^T y, the first E-step's initialisation);
 * an engine thread then runs one CUDA graph per set of admitted fits whose
 * WHILE node repeats a step on the device: one launch of a tensor-core GEMM
 * applies Phi (then Phi^T) to the direction blocks of every fit (each fit's
 * work cut into fixed segments, the segments of all fits spread over the
 * SMs), and one launch each of the T reduction, the CG update, the stopping
 * test and direction, the M-step (fits whose CG loop ended) and the next
 * E-step's initialisation serve every fit.  The loop returns to the host
 * when a fit finishes, new fits are ready to join, or after 4096 steps.
 * Every fit keeps alpha, mu and its CG state on the device; a fit's
 * arithmetic does not depend on the others, so a request gives the same bits
 * alone and among any others (within the tolerances of the tests, the same
 * results as cofem_fit, whose GEMM splits its work differently).
 * Requests: dense dictionaries, precision COFEM_BF16 or COFEM_F32_TF32X3,
 * rr_period 0, BF16 with K <= 41 (else cofem_submit returns UNSUPPORTED).
 * At most max_fits (1..1024) fits are prepared or in the step at once; the
 * HBM budget bounds them too.  flags: 0, or COFEM_SERVE_HOST_LOOP to launch
 * every step from the host (no graph; slower, but profilers see each
 * kernel).  Same submit / poll / wait / destroy calls. */
#define COFEM_SERVE_HOST_LOOP 1
cofem_status cofem_server_create_packed(cofem_server** out, long long hbm_budget_bytes, int max_fits,
                                        int prep_threads, int flags);

/* Counters of a packed server (zero for an independent one): graph launches
 * of the step loop, steps run, fit-steps (the sum over steps of the fits in
 * the step: fit_steps / steps is the mean number of fits a step serves), and
 * step graphs built (once per table capacity and dictionary-precision mix). */
typedef struct cofem_server_stats {
    long long launches, steps, fit_steps, graphs_built;
} cofem_server_stats;
cofem_status cofem_server_get_stats(cofem_server* srv, cofem_server_stats* out);

/* Queue a request (never blocks on the GPU).  *ticket identifies it.  Errors:
 * INVALID_ARG (incomplete request), NOMEM (needs more than the whole budget),
 * UNSUPPORTED (a packed server and a request it does not take). */
cofem_status cofem_submit(cofem_server* srv, const cofem_request* req, unsigned long long* ticket);

/* *done = 1 once the request's outputs are written. NOT_FOUND for an unknown ticket. */
cofem_status cofem_poll(cofem_server* srv, unsigned long long ticket, int* done);

/* Block until the request completes, fill *out and forget the ticket. */
cofem_status cofem_wait(cofem_server* srv, unsigned long long ticket, cofem_result* out);

/* Finish every queued request, stop the workers and free the server. */
cofem_status cofem_server_destroy(cofem_server* srv);

/* ---- Allocation-free operator application ----
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code that runs while a stream capture is active
 * (the global capture mode rejects allocation calls), processes whose device
 * memory is already fully owned by another allocator (for example a
 * framework's caching pool), and latency-critical loops that must not take the
 * driver's allocation path.  It computes the same step a4 product as
 * cofem_apply_operator, Psi = beta Phi^T (Phi V) + diag(alpha) V for an FP32
 * dense dictionary, without a handle and without allocating anything:
 *   phi    : N x D floats, row-major with leading dimension ld >= D (device).
 *   V, Psi : Q x D floats, row q = vector q (device); alpha: D floats (device).
 *   1 <= Q <= 64 and N*Q <= COFEM_NOALLOC_MAX_ELEMS, else COFEM_ERR_INVALID_ARG
 *   (nothing is launched).
 *   stream : cudaStream_t (NULL = default stream).  The call only enqueues
 *   kernels and returns; synchronise the stream before reading Psi.
 * The intermediate Phi V lives in one fixed array of COFEM_NOALLOC_MAX_ELEMS
 * floats (4 MiB) in the library's device memory, which every GPU that loads the
 * library keeps until the process exits.  All calls on a device share that
 * array: calls whose kernels can overlap on the GPU (different streams without
 * ordering) race on it and give wrong results; serialise them.  Every call
 * leaves its T = Phi V in the array; nothing in it needs to start at zero.
 * The first call on each device looks up the array's device address with that
 * device current; make that first call before any stream capture begins.
 * Later calls do no set-up unless the device's context has changed (after a
 * cudaDeviceReset the next call looks the address up again, so make it
 * outside a capture too).  phi, V, alpha and Psi must be device memory of the
 * current device (or managed memory).  A CUDA error left pending on the
 * calling thread by earlier work is returned as COFEM_ERR_CUDA before anything
 * is launched.  Errors: INVALID_ARG (sizes, NULL pointers, host memory or
 * another device's memory), NONFINITE (beta), CUDA (pending error, launch
 * failure). */
#define COFEM_NOALLOC_MAX_ELEMS 1048576
cofem_status cofem_apply_dense_noalloc(const float* phi, long long N, long long D, long long ld,
                                       const float* V, int Q, const float* alpha, double beta,
                                       float* Psi, void* stream);

/* Timing of the precision form's accurate residual B - A X (row a6), in the
 * launch configuration a fit uses, on the handle's current X, bracketed by
 * CUDA events on the handle's stream: *ms_residual = mean time of one whole
 * accurate residual (all its kernels), *ms_first = mean time of its first
 * product Phi~ X (with the digits of X in the SLICED form; dense
 * dictionaries; 0 otherwise).  Either
 * pointer may be NULL (not both).  Requires a previous fit with the same Q on
 * a handle with rr_period > 0 or check_residual = 1.  Errors: INVALID_ARG,
 * CUDA. */
cofem_status cofem_time_true_residual(struct cofem_ctx* h, int Q, int reps, double* ms_residual, double* ms_first);

/* The accurate product of the precision form alone (row a6): out = Phi~^T
 * (Phi~ (Xh + Xl)) in FP64 for a block of Q vectors, by the handle's accurate
 * residual form (opts.residual_path; beta and alpha are left out), on the
 * dictionary the handle computes with.  Xh, Xl: Q x D floats row-major (the
 * FP32 pair of each vector); out: Q x D doubles; all three host or device
 * pointers of the handle's device.  1 <= Q <= 64 (SLICED: Q <= 48).  Dense
 * dictionaries on a handle with rr_period > 0 or check_residual = 1.
 * Errors: INVALID_ARG (NULL, Q, kind, options), NONFINITE (Xh or Xl), NOMEM,
 * UNSUPPORTED, CUDA. */
cofem_status cofem_accurate_product(struct cofem_ctx* h, const float* Xh, const float* Xl, int Q, double* out);

/* Failure-detection self-test: runs the library's two bounded on-device wait
 * routines (the grid-counter wait of the single-pass operator, bounded by
 * `seconds` of %globaltimer, 1e-3 <= seconds <= 2, and the mbarrier wait of
 * the tensor-core pipeline, bounded by 4096 rounds) on a counter and an
 * mbarrier that nothing completes, on the current device.  Both waits give
 * up by their limits (no fault, no hang), set COFEM_FLAG_DEVICE_TIMEOUT and
 * the call returns COFEM_ERR_CUDA with that flag in *flags (NULL accepted),
 * as a fit whose wait ran out does; the context stays usable.  Errors:
 * INVALID_ARG (seconds), NOMEM, CUDA. */
cofem_status cofem_selftest_bounded_wait(double seconds, unsigned* flags);

/* Bytes of device memory the handle holds (Phi copy, theta, fit workspace). */
long long cofem_device_bytes(struct cofem_ctx* h);

/* The dense dictionary the handle computes with, as FP32 (N x D row-major, host
 * or device pointer): the FP32 copy, bf16(Phi) for COFEM_BF16, or s_i code_ij
 * (each product rounded to FP32) for COFEM_FP8_E4M3.  Paper counterpart: the
 * Phi of Sec. III in the stored precision.  Errors: INVALID_ARG (NULL, or a
 * convolution handle), NOMEM, CUDA. */
cofem_status cofem_get_dictionary(struct cofem_ctx* h, float* out);

/* How the CG loop of Alg. 2 runs for the current Q (valid after a fit or
 * cofem_apply_operator): *path = COFEM_PATH_TWO_PASS or
 * COFEM_PATH_SINGLE_PASS for a BF16 or 3xTF32 dense dictionary, COFEM_PATH_AUTO
 * (0) for the FP32 FMA and DCT forms, COFEM_TOEPLITZ_DIRECT or COFEM_TOEPLITZ_FFT
 * for a convolution dictionary; *kernels_cg = kernels
 * launched per operator application inside the CG loop; *kernels_rr = per
 * accurate residual (a residual replacement or a true-residual check); *kernels_step = kernels of the CG
 * update, stopping test and direction per CG step (2).  Any output pointer
 * may be NULL.  Errors:
 * INVALID_ARG (NULL handle, or no fit or application yet). */
cofem_status cofem_operator_info(struct cofem_ctx* h, int* path, int* kernels_cg, int* kernels_rr,
                                 int* kernels_step);

/* True relative residuals of the last fit (precision form, Alg. 2 stopping
 * test applied to the returned X): out[t * (K+1) + q] = ||b_q - A x_q|| / ||b_q||
 * for EM iteration t (0-based) and column q (0 = mu), with A = beta Phi~^T Phi~
 * + diag(alpha^(t)) on the dictionary the handle computes with, measured on the
 * GPU when the E-step's CG loop ended (after the last restart): A X from the
 * FP32 pair X + Xlo by the handle's accurate residual form (opts.residual_path)
 * and FP64 partial sums.  0 for a zero
 * right-hand side.  out: host, T_em * (K+1) doubles of the last cofem_fit.
 * Errors: INVALID_ARG (NULL, no fit yet, or a handle with rr_period = 0 and
 * check_residual = 0), CUDA. */
cofem_status cofem_true_residuals(struct cofem_ctx* h, double* out);

/* Counts of the last fit's precision-form steps: *replacements = residual
 * replacements (each one accurate residual, cofem_operator_info's
 * kernels_rr launches), *checks = true-residual checks (each one accurate
 * residual, one check kernel and, in the CUDA graph, one loop-gate kernel).
 * Either pointer may be NULL.  Errors: INVALID_ARG (NULL handle, no fit). */
cofem_status cofem_fit_stats(struct cofem_ctx* h, int* replacements, int* checks);

/* The fit graph of the handle (use_graph = 1): *built = 1 once a fit has
 * recorded it, else 0; *overlapped = 1 if its CG-step kernels are joined by
 * programmatic (overlapping) edges, 0 if by plain ones (overlap_launch = 0,
 * or the driver did not take the programmatic edges and the graph was
 * rebuilt plain).  Either pointer may be NULL.  Errors: INVALID_ARG (NULL
 * handle). */
cofem_status cofem_graph_info(struct cofem_ctx* h, int* built, int* overlapped);

#ifdef __cplusplus
}
#endif
#endif /* COFEM_H */
