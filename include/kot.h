/*
 * kot.h -- C ABI of the GB300 library for the specialized semismooth Newton (SSN) method for
 * kernel-based optimal transport (Lin, Cuturi & Jordan).
 *
 * Notation: n = samples per measure (the paper's n_sample), l = filling points (the paper's n),
 * d = dimension of x and of y.  All matrices are row-major, contiguous, FP64.
 *
 * Pointers: every array argument is a DEVICE pointer (CUDA global memory of the context's
 * device) unless the context was created with kot_options.host_pointers = 1, in which case every
 * array argument is HOST memory and the library copies it in and out on its stream inside the
 * call.  The caller owns all argument arrays; the context owns every internal buffer and frees
 * them in kot_destroy.  Calls are stream-ordered on kot_options.stream and return after that
 * stream has finished the call's work (outputs are ready on return).
 *
 * Errors: every entry point returns a kot_status.  Arguments are validated before any GPU work
 * (KOT_ERR_INVALID leaves the context unchanged).  kot_last_error() gives a one-line reason.
 * No entry point aborts the process, and no kernel waits without an iteration bound.
 *
 * Threads: a context is used by one host thread at a time.
 *
 * Launches: kernels that follow one another on the context's stream are launched with
 * programmatic stream serialisation (each waits for its predecessor's completion inside the
 * kernel, after its own set-up), so set-up overlaps the previous kernel's tail.  Setting the
 * environment variable KOT_PDL=0 before the first call gives plain stream-ordered launches of
 * the same kernels (same arithmetic, same results).
 */
#ifndef KOT_H
#define KOT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kot_ctx kot_ctx;

typedef enum {
  KOT_OK = 0,
  KOT_ERR_INVALID = 1,        /* bad argument; nothing was launched                      */
  KOT_ERR_CUDA = 2,           /* a CUDA runtime call failed                              */
  KOT_ERR_OOM = 3,            /* device allocation failed                                */
  KOT_ERR_NOT_PD = 4,         /* Cholesky of K + eps I failed up to the jitter limit      */
  KOT_ERR_NO_CONVERGENCE = 5, /* iteration cap reached; outputs hold the last iterate    */
  KOT_ERR_NONFINITE = 6,      /* NaN/Inf met in the iteration                            */
  KOT_ERR_TIMEOUT = 7,        /* a bounded device wait gave up                           */
  KOT_ERR_STATE = 8,          /* call order: e.g. solve before features                  */
  KOT_ERR_TOO_LARGE = 9       /* size above the fixed capacity of an allocation-free call */
} kot_status;

typedef enum {
  KOT_FP64 = 0,       /* every step in FP64 (a cold eigen-decomposition up to l = 160
                         starts from an FP32 shared-memory Jacobi basis, refined to FP64) */
  KOT_MIXED = 1       /* every O(l^3) product on the tcgen05 tensor cores: FP64-accuracy
                         products (residual, projection, EG, eigenbasis refinement, Newton
                         right-hand side and check) emulated with six fixed-point BF16
                         slices; the Jacobian products inside CG with three (about FP32
                         accuracy), or exact FP64 kernels with at most 32 carried rows;
                         products below opt.tc_min_flops on the FP64 pipes; FP64 features,
                         Jacobi rotations (a cold start up to l = 160 in FP32, refined to
                         FP64), vectors and stop test                                   */
} kot_precision;

/* Algorithm constants.  Defaults (kot_default_options): the values of Sec. 5 for alpha1,
 * alpha2, beta0, beta1, beta2; CG cap 20 (Sec. 4.4 remark); tau = 0.1, kappa = 1,
 * theta0 = 1, theta_min = 1e-6, theta_max = 1e6, eg_step = 0 (use 1/L), jitter = 1e-10,
 * jitter_max = 1e-6, max_iter = 200. */
typedef struct {
  int device;              /* CUDA device ordinal                                        */
  void* stream;            /* cudaStream_t to order work on; NULL = a stream of its own   */
  int precision;           /* kot_precision                                              */
  int host_pointers;       /* 1: array arguments are host memory (see above)             */
  int max_iter;            /* outer iterations of Algorithm 2                            */
  int cg_max_iter;         /* CG iterations per Newton direction                         */
  double tau, kappa;       /* inexact Newton test, Eq. (4.3)                              */
  double alpha1, alpha2;   /* theta rule thresholds (Sec. 4.3)                           */
  double beta0, beta1, beta2;
  double theta0, theta_min, theta_max;
  double eg_step;          /* <= 0: 1/L, L = max rowsum|Q|/(2 l2) + sqrt(max rowsum (Kt o Kt)) */
  double jitter;           /* eps = jitter * max_i K_ii, x10 on failure ...              */
  double jitter_max;       /* ... up to jitter_max * max_i K_ii                          */
  int use_eg;              /* 1: Algorithm 2 with the EG safeguard; 0: plain SSN steps   */
  int record_history;      /* 1: keep ||R(w_k)|| per iteration (kot_get_history)         */
  int eig_ctas;            /* CTAs of the cooperative Jacobi eigensolver; 0 = one per SM  */
  double mixed_switch;     /* mixed form: reduced-precision (three-slice) CG products for the
                              Newton direction while ||R(w_k)|| > this (the result is always
                              re-checked against Eq. (4.3) with FP64-accuracy products and
                              finished with them if short), FP64-accuracy CG products below
                              it (default 1e-4)                                            */
  int batch_workers;       /* kot_batch_solve: problems solved concurrently (0 = 4)        */
  int eig_refine;          /* eigen-decompositions: at most this many refinement steps from a
                              start basis (the previous one of the same sequence, then the
                              slot's own previous one, or the identity when there is none)
                              before falling back to Jacobi sweeps; 0 = always Jacobi (default 5) */
  int schur_solver;        /* Krylov method for the Schur system of Algorithm 1 (Sec. 4.3 names
                              both): 0 = conjugate gradients (default), 1 = symmetric QMR
                              (Freund-Nachtigal, no preconditioner); both stop on Eq. (4.3)
                              measured with the true residual and cap at cg_max_iter */
  int gram_fp32;           /* kot_build_features: 1 = the Gram matrices Q and K (Sec. 3) from FP32
                              distances and exponentials (entries ~1e-7 relative to FP64; the
                              embeddings, q2, z and the Cholesky stay FP64); 0 = FP64 (default) */
  double tc_min_flops;     /* mixed form: a product of fewer multiply-add flops (2 M N K, halved
                              for a symmetric result) runs exact on the FP64 pipes instead of
                              the tensor cores, where the emulated product's three launches take
                              longer (default 8e6: l x l x l products up to l ~ 158, and the
                              projection's l x l x min(|alpha|, |alpha-bar|) ones); CG directions
                              whose products all fall below it need no FP64 re-check;
                              0 = every product on the tensor cores                        */
} kot_options;

typedef struct {
  int status;              /* kot_status of the solve                                    */
  int iters, ssn_accepted, eg_taken, cg_total;
  double residual;         /* ||R(w)|| = ||r1||_2 + ||r2||_F at the returned iterate      */
  double r1_norm, r2_norm;
  double objective;        /* dual objective of Eq. (3.3) at gamma                       */
  double ot_hat;           /* estimator OT-hat (Sec. 3)                                  */
  double eps;              /* Cholesky jitter used                                       */
  double seconds;          /* wall time of the call                                      */
  int eig_calls;           /* symmetric eigen-decompositions performed by the solve      */
  int eig_sweeps;          /* Jacobi sweeps summed over them                             */
  int eig_refined;         /* decompositions finished by refinement (no FP64 sweep)      */
  int eig_refine_steps;    /* refinement steps summed over them                          */
} kot_result;

/* Fill *opt with the defaults listed above.  Returns KOT_ERR_INVALID if opt is NULL. */
kot_status kot_default_options(kot_options* opt);

/* Create a context on opt->device (opt NULL = defaults).  *out receives the handle. */
kot_status kot_create(kot_ctx** out, const kot_options* opt);

/* Release every buffer of the context.  NULL is accepted. */
kot_status kot_destroy(kot_ctx* ctx);

/* One-line description of the last error of this context (never NULL). */
const char* kot_last_error(const kot_ctx* ctx);

/* Feature assembly (Sec. 3, definitions following Eq. (3.2)):
 *   w_mu(xf_i) = (1/n) sum_j k(x_j, xf_i),  w_nu(yf_i) = (1/n) sum_j k(y_j, yf_i),
 *   q2 = (1/n^2) sum_ij k(x_i, x_j) + (1/n^2) sum_ij k(y_i, y_j),
 *   Q_ij = k(xf_i, xf_j) + k(yf_i, yf_j),  c_i = ||xf_i - yf_i||^2,
 *   z_i = w_mu(xf_i) + w_nu(yf_i) - lambda2 c_i,
 *   K_ij = k((xf_i, yf_i), (xf_j, yf_j)),  R upper triangular with R^T R = K + eps I.
 * k(a, b) = exp(-||a - b||^2 / (2 sigma^2)).
 * X, Y: n x d.  Xf, Yf: l x d (the x and y halves of the filling pairs).
 * Requires d, n, l >= 1 and sigma, lambda1, lambda2 > 0.  KOT_ERR_NOT_PD if K + eps I is not
 * positive definite for eps up to jitter_max * max K_ii. */
kot_status kot_build_features(kot_ctx* ctx, int d, int n, const double* X, const double* Y,
                              int l, const double* Xf, const double* Yf, double sigma,
                              double lambda1, double lambda2);

/* Inject the dual problem data directly (Eq. (3.3)): Q (l x l, symmetric), z (l), q2, R (l x l,
 * upper triangular, the rows below the diagonal are ignored).  w_mu + w_nu is taken as
 * z (so ot_hat uses z); used for closed-form cases. */
kot_status kot_set_features(kot_ctx* ctx, int l, const double* Q, const double* z, double q2,
                            const double* R, double lambda1, double lambda2);

/* Copy out the assembled features; any output pointer may be NULL.  Q, K, R: l x l; z, w_mu,
 * w_nu, c: l; q2, eps: one double each. */
kot_status kot_get_features(kot_ctx* ctx, double* Q, double* K, double* R, double* z,
                            double* w_mu, double* w_nu, double* c, double* q2, double* eps);

/* Natural residual map R(w) of Eq. (4.2) at w = (gamma, X):
 *   r1 = (Q gamma - z)/(2 lambda2) - Phi(X),  Phi(X)_i = (R^T X R)_ii,
 *   r2 = X - Pi_{S+}(X - (Phi*(gamma) + lambda1 I)),  Phi*(gamma) = R diag(gamma) R^T,
 * with Pi_{S+} by spectral decomposition (Eq. (4.4)).  gamma: l; X: l x l symmetric.
 * Outputs (any may be NULL): r1 (l), r2 (l x l), proj = Pi_{S+}(Z) (l x l), sig = eigenvalues
 * of Z in ascending order (l), norms[3] = {||r1||_2, ||r2||_F, ||R(w)||}. */
kot_status kot_residual(kot_ctx* ctx, const double* gamma, const double* X, double* r1,
                        double* r2, double* proj, double* sig, double* norms);

/* Regularised Newton direction of Eq. (4.2)-(4.3) by Algorithm 1 at w = (gamma, X) with
 * regularisation mu > 0: CG on (Q/(2 lambda2) + mu I + Phi T Phi*) dgamma = a1 with the
 * operator T_k of Sec. 4.3.  CG applies Phi T Phi* in the eigenbasis of Z (Cb = P^T R formed once
 * per direction; the alpha rows of Psi o Cb diag(p) Cb^T with the G + G^T weights) and forms a1
 * and dX there too; schur_solver = 1 applies T directly (G + G^T form when |alpha| <= l/2,
 * complement form otherwise).  Both are T_k in exact arithmetic.
 * cg_tol_abs > 0 stops CG at ||residual||_2 <= cg_tol_abs (at most 10 l + 50 iterations);
 * cg_tol_abs <= 0 uses the inexact test of Eq. (4.3) with the context's tau, kappa and
 * cg_max_iter.  Outputs: dgamma (l), dX (l x l), cg_iters (host int, may be NULL). */
kot_status kot_newton_direction(kot_ctx* ctx, const double* gamma, const double* X, double mu,
                                double cg_tol_abs, double* dgamma, double* dX, int* cg_iters);

/* Algorithm 2 from w0 = (gamma0, X0) (NULL = zeros) until ||R(w_k)|| <= tol or max_iter.
 * gamma_out (l) is required; X_out (l x l) may be NULL; res may be NULL.
 * Returns KOT_ERR_NO_CONVERGENCE at the cap with the last iterate in the outputs. */
kot_status kot_ssn_solve(kot_ctx* ctx, double tol, double* gamma_out, double* X_out,
                         const double* gamma0, const double* X0, kot_result* res);

/* The pure extragradient method (the comparison method of App. F, Fig. 6): from v0 = (gamma0, X0)
 * (NULL = zeros), v_{k+1} = EG(v_k) -- the projected extragradient step of Algorithm 2's
 * safeguard, with step opt.eg_step (<= 0: 1/L) -- until ||R(v_k)|| <= tol or opt.max_iter steps.
 * Outputs and history as for kot_ssn_solve (iters = eg_taken = steps; the history holds
 * ||R(v_k)||).  Returns KOT_ERR_NO_CONVERGENCE at the cap with the last iterate in the outputs. */
kot_status kot_eg_solve(kot_ctx* ctx, double tol, double* gamma_out, double* X_out,
                        const double* gamma0, const double* X0, kot_result* res);

/* Residual history of the last solve (record_history = 1): copies min(cap, iters + 1) values
 * of ||R(w_k)|| to the host array hist; *count receives the number copied. */
kot_status kot_get_history(kot_ctx* ctx, double* hist, int cap, int* count);

/* Per-iteration trace of the last solve (record_history = 1): up to cap rows of five doubles
 * {||R(w_{k+1})||, mu_k, CG steps, theta_{k+1}, direction kind (0 FP64 products, 1 tensor-core
 * products that passed the FP64 check of Eq. (4.3) as they were, 2 tensor-core products plus
 * FP64 CG steps)} into the host array out (5 * cap doubles);
 * *count receives the number of rows. */
kot_status kot_get_trace(kot_ctx* ctx, double* out, int cap, int* count);

/* Potentials and transport map from dual weights gamma (l), at m query points (m x d):
 * stationarity of the Lagrangian of Eq. (3.2) gives the empirical Kantorovich potentials
 *   u(x) = (w_mu(x) - sum_i gamma_i k(xf_i, x)) / (2 lambda2),  w_mu(x) = (1/n) sum_j k(x_j, x)
 * (side 0; side 1: v(y) with the y samples and yf), so that averaging u over the x samples plus v
 * over the y samples gives OT-hat (Sec. 3).  Outputs (any may be NULL, not all): u (m), grad (m x d)
 * = grad u, tmap (m x d) = x - grad u(x), the map estimate for the cost ||x - y||^2/2 used for
 * Figs. 1, 4 and 7.  Needs the samples of kot_build_features (KOT_ERR_STATE after
 * kot_set_features).  Pointers follow the context's pointer mode. */
kot_status kot_potentials(kot_ctx* ctx, int side, int m, const double* points, const double* gamma,
                          double* u, double* grad, double* tmap);

/* One problem of a batch.  Arrays follow the context's pointer mode. */
typedef struct {
  int d, n, l;
  const double *X, *Y, *Xf, *Yf;
  double sigma, lambda1, lambda2, tol;
  double* gamma_out;       /* l, required */
} kot_problem;

/* Solve B independent problems (features + Algorithm 2 each).  res receives B results (host
 * array).  Problems are handed out largest-first to batch_workers concurrent worker contexts
 * (each with its own stream and buffers, driven by its own host thread; their eigensolver
 * launches share the SMs) on the context's device.  The call returns the first non-OK status
 * in problem order (KOT_OK if all converged); each res[i].status is per problem. */
kot_status kot_batch_solve(kot_ctx* ctx, int B, const kot_problem* probs, kot_result* res);

/* Bootstrap resamples with shared filling points (the bandwidth and bootstrap settings of Sec. 5
 * keep the filling points fixed while the samples change).  After kot_build_features(ctx, d, ...,
 * l, Xf, Yf, sigma, lambda1, lambda2), solves B problems whose samples are the resamples
 * Xs[b], Ys[b] (b < B; each n x d, stored one after another: Xs is B x n x d) with the context's
 * filling points, sigma, lambda1 and lambda2.  Q, K and the Cholesky factor R (Sec. 3), the
 * jitter and the EG step bound depend on the filling points only, so they are built once (by
 * kot_build_features) and shared; each resample rebuilds the kernel embeddings w_mu, w_nu, q2 and
 * z (Sec. 3) and runs Algorithm 2 from zero to ||R(w)|| <= tol.  gamma_out: B x l, resample b's
 * gamma in row b.  res: B host results.  Arrays follow the context's pointer mode.  After the
 * call the context holds the last resample's problem (kot_potentials uses its samples).
 * Returns KOT_ERR_STATE without kot_build_features before it, else the first non-OK status in
 * resample order (each res[b].status is per resample).  n may differ from kot_build_features's. */
kot_status kot_bootstrap_solve(kot_ctx* ctx, int B, int n, const double* Xs, const double* Ys, double tol,
                               double* gamma_out, kot_result* res);

/* ---- building block: symmetric eigen-decomposition (Sec. 4.1, Eq. (4.4)) ----
 * The projection onto the PSD cone and the weights Omega of the generalized Jacobian are read
 * off Z = P diag(sig) P^T.  Z: l x l, row-major, symmetric (the library uses (Z + Z^T)/2).
 * P: l x l output, row-major, column j = eigenvector j; sig: l eigenvalues, ascending.
 * warm (may be NULL): an orthogonal l x l basis (row-major, orthonormal columns) close to the
 * eigenbasis, e.g. the one of a nearby matrix.  With it the library first refines warm into
 * the eigenbasis (Ogita-Aishima iteration, at most opt.eig_refine steps of FP64 products) and
 * rebuilds by Jacobi sweeps from warm when that does not converge.  Without it the refinement
 * starts from the identity (a nearly diagonal Z then needs no sweeps); failing that, for
 * l <= 160 from an FP32 basis computed by Jacobi in one CTA's shared memory, and the FP64
 * sweeps, if still needed, start from that basis orthonormalised.  info (host, may be NULL)
 * receives {FP64 Jacobi sweeps, refinement steps} of the call.
 * Pointers follow the context's pointer mode.  No features are needed.  KOT_ERR_TIMEOUT if a
 * bounded wait of the cooperative Jacobi kernel gave up, KOT_ERR_NO_CONVERGENCE if the sweeps
 * did not converge. */
kot_status kot_eig_sym(kot_ctx* ctx, int l, const double* Z, const double* warm, double* P,
                       double* sig, int* info);

/* ---- building block of the mixed form: dense product on the tensor cores ----
 * C = alpha * op(A) * op(B)^T + beta * C, C: M x N (ldc), op(A): M x K, op(B): N x K, where
 * op(X)(r, k) = X[r * ldx + k] (transX = 0) or X[k * ldx + r] (transX = 1).  FP64 in and out;
 * the arithmetic runs on tcgen05 tensor cores in BF16 x BF16 -> FP32 with each operand split
 * into `pieces` BF16 terms (1: BF16 accuracy, about 4e-3 relative; 3: about FP32 accuracy).
 * This is how the mixed form computes the Jacobian-matvec products of Algorithm 1 (Sec. 4.3).
 * pieces = 0 runs the same product in FP64 on the CUDA cores (the FP64 form's GEMM).
 * pieces = -s (s = 3..8) runs it FP64-accurate on the tensor cores: every row of op(A) and of
 * op(B) is cut into s fixed-point BF16 slices relative to its largest magnitude, the slice
 * products of total level < s are summed exactly in FP32 and combined in float-float (error
 * about 2^-(8 s - 1) max|op(A) row| max|op(B) row| K per element; s = 6 is what the mixed form
 * uses for its FP64-accuracy products).
 * Pointers follow the context's pointer mode.  KOT_ERR_TIMEOUT if a tensor-core wait gave up. */
kot_status kot_dense_product(kot_ctx* ctx, int M, int N, int K, double alpha, const double* A,
                             int lda, int transA, const double* B, int ldb, int transB,
                             double beta, double* C, int ldc, int pieces);

/* ---- autotuner (not part of the paper's method) ----
 * Times, on inputs it generates itself on the context's device and stream:
 *   - the emulated-FP64 product (three and six slices) at l x l x l for output-tile widths 64
 *     and 128 and split counts 1, 2, 3, 4, 6, 8, 12, 16;
 *   - a cold Jacobi decomposition of a symmetric l x l matrix for SMs/4, SMs/2 and SMs CTAs of
 *     256, 512 and 1024 threads (the eigensolver's block size).
 * It records the fastest of each per size bucket (ceil log2 l) in a process-wide table for the
 * device.  Every later product of that size bucket and slice count, and every later decomposition
 * of that bucket (when kot_options.eig_ctas is 0), on any context of the device, uses the table.
 * choice (host, may be NULL, 6 ints) receives {splits with 3 slices, splits with 6 slices,
 * Jacobi CTAs, tile width with 3 slices, tile width with 6 slices, Jacobi threads per CTA}.
 * Takes a few tens of milliseconds (longer for large l).  Returns KOT_ERR_INVALID for l outside
 * 1..32768. */
kot_status kot_autotune(kot_ctx* ctx, int l, int* choice);

/* ---- tracing: per-kernel-class launch statistics (not part of the paper's method) ----
 * Kernel classes: 0 FP64 GEMM tiles, 1 Jacobi eigensolver (FP64, one launch per
 * decomposition), 2 reserved (unused), 3 kernel mean embeddings and potentials,
 * 4 embedding-norm pair sums, 5 Gram matrices Q and K, 6 Cholesky diagonal block,
 * 7 tensor-core (tcgen05) GEMM tiles, 8 eigenbasis refinement correction, 9 FP64-emulating
 * tensor-core GEMM (k_oz_gemm), 10 its slicing and finalize kernels, 11 one application of the
 * Schur operator H p = Q p/(2 lambda2) + mu p + Phi(T[Phi*(p)]) inside CG (Algorithm 1; all of
 * its launches between one event pair).
 * kot_profile(ctx, mask) turns on timing of the classes whose bit is set in mask (0 = off) and
 * clears the statistics.  While on, every launch of an enabled class is bracketed by CUDA events
 * on the context's stream.  kot_profile_read fills, for class cls, the number of launches, the
 * summed event time in milliseconds, the summed algorithmic flops and bytes of those launches
 * (the counts each launch site states for the method's arithmetic and its compulsory traffic),
 * and the summed flops they executed.  Algorithmic flops are the method's count: 2MNK for an
 * FP64-accurate product however it is computed (class 9 executes 2MNK per BF16 slice pair), and
 * for class 11 F_mv = (4/3) l^3 + 8 a l^2 + 2 l^2 with a = min(|alpha|, |alpha-bar|) (Phi* and Phi
 * on the triangular factor, T_k in the cost-reduced forms of Sec. 4.3, Q p); class 11 executes
 * the eigenbasis form, 4 a l^2 + 2 l^2 in FP64-accurate terms. */
typedef struct {
  long long launches;
  double ms, flops, bytes, exec_flops;
} kot_kernel_stats;

kot_status kot_profile(kot_ctx* ctx, int mask);
/* Time only one launch in `every` (>= 1, default 1) of each enabled class, so that the events
 * perturb a latency-bound run less; the statistics then cover the sampled launches (clears them). */
kot_status kot_profile_every(kot_ctx* ctx, int every);
/* Total number of kernels this library has launched in the process so far (all contexts). */
kot_status kot_launch_count(long long* out);
kot_status kot_profile_read(kot_ctx* ctx, int cls, kot_kernel_stats* out);

/* ---- failure detection self-test (not part of the paper's method) ----
 * Launches a kernel that waits, with the bounded poll every tensor-core pipeline wait uses, on an
 * mbarrier that nothing completes; after `polls` polls (1..1e8, each at least 20 ns) it gives up,
 * sets the error flag, and returns.  The call therefore returns KOT_ERR_TIMEOUT -- the status a
 * starved pipeline stage turns into -- and leaves the context usable.  KOT_ERR_INVALID for polls
 * out of range. */
kot_status kot_wait_probe(kot_ctx* ctx, long long polls);

/* ---- allocation-free entry point (the paper has no counterpart; an interface addition) ----
 * ||w||^2 = (1/n^2) sum_{i,j} exp(-||s_i - s_j||^2 / (2 sigma^2)) over the n x d samples S (one
 * half of q2 in kot_build_features), for callers that must not allocate device memory while
 * they run: code inside a custom device-memory allocator or pool, a process that reserved all
 * of its device memory up front, or a host that forbids driver allocations after start-up.
 * It calls no cudaMalloc/cudaFree and no allocating library routine.  Its per-tile partial sums
 * live in a fixed device array compiled into the library (32 KB, 4096 doubles, held on every
 * GPU that loads the library until process exit), which caps n at 4096 samples: larger n
 * returns KOT_ERR_TOO_LARGE before any GPU work.
 * S and out (one double) are device pointers on the caller's current device; stream is a
 * cudaStream_t of that device (NULL = legacy default stream).  The call returns after the
 * stream has finished (the result is in *out).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps it for the process;
 * make that first call before any stream capture.  The kept address belongs to the device's
 * current primary context: after cudaDeviceReset on that device (or anything else that destroys
 * and re-creates its primary context) the array may move, so a process that resets a device must
 * not call this entry point on it again.  All calls share the one array and it keeps the last
 * call's partial sums; every slot a call reads is written by that same call, so nothing needs
 * clearing, but calls whose GPU work overlaps (other host threads or streams at the same time)
 * race on it and must be serialised by the caller.  Errors: KOT_ERR_TOO_LARGE for n > 4096
 * (nothing is launched); KOT_ERR_INVALID for n, d < 1, NULL pointers, sigma <= 0 or not finite,
 * or a current device ordinal of 64 or more (the per-device address table has 64 entries);
 * KOT_ERR_CUDA for a failed CUDA call. */
kot_status kot_embedding_sqnorm_noalloc(int n, int d, const double* S, double sigma, double* out,
                                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KOT_H */
