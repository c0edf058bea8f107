/*
 * rpca.h -- C ABI of the GB300 (sm_103a) Split-SPCP engine.
 *
 * Method: Driggs, Becker, Aravkin, "Adapting Regularized Low-Rank Models for Parallel
 * Architectures" (arXiv 1702.02241).  The engine minimises the smooth non-convex RPCA
 * objective of Eq. (Thm5) / Eq. (7),
 *
 *     F(U, V) = lam_L/2 (||U||_F^2 + ||V||_F^2) + sum_{(i,j) in Omega} psi_{lam_S}((U V^T - X)_ij),
 *
 * where psi is the Huber function left by marginalising the l1-penalised sparse part S
 * (Sec. 1, "Marginalization in S"), Omega the observed entries (Sec. 6.2), with L-BFGS of
 * memory 10 (Sec. 5.1), and checks optimality with the computable certificate of Sec. 3.4.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major float32 in DEVICE memory unless stated otherwise.  X is
 *     m x n with leading dimension ldx >= m; U is m x k (ld m); V is n x k (ld n).
 *   - X and the mask are BORROWED: they must stay valid and unchanged until rpca_destroy.
 *     U, V, gU, gV and all other matrix arguments are caller-owned device buffers.
 *   - Work is ordered on the CUDA stream given to rpca_create; calls that return host
 *     scalars or structs (f, rpca_result, rpca_cert) synchronise that stream.
 *   - Every entry returns an rpca_status and never aborts; rpca_last_error() gives a
 *     message for the last failure on a context.  A context is not thread-safe: serialise
 *     calls on one context.
 *   - Any CUDA error (including a device wait that gave up, see RPCA_ETIMEOUT) is reported,
 *     never hidden; there is no CPU fallback.
 */
#ifndef RPCA_H
#define RPCA_H

#include <stdint.h>

#if defined(__GNUC__)
#define RPCA_API __attribute__((visibility("default")))
#else
#define RPCA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpca_ctx rpca_ctx; /* opaque, owned by the library */
typedef struct rpca_ws rpca_ws;   /* learned warm-start model, opaque (see the end of this file) */

typedef enum {
  RPCA_OK = 0,
  RPCA_EINVAL = -1,       /* bad argument (sizes, k, lambdas, null pointers, non-finite observed X) */
  RPCA_ENOMEM = -2,       /* device allocation failed */
  RPCA_ECUDA = -3,        /* CUDA runtime/driver error */
  RPCA_ENOTCONV = -4,     /* solver stopped (iteration cap, line-search failure) above cert_tol */
  RPCA_ETIMEOUT = -5,     /* a bounded device wait gave up; results are invalid */
  RPCA_EUNSUPPORTED = -6  /* combination not compiled (e.g. k > 16) */
} rpca_status;

typedef enum { RPCA_F32 = 0, RPCA_BF16 = 1, RPCA_FP8E4M3 = 2 } rpca_dtype;

typedef enum {
  RPCA_INIT_SKETCH = 0, /* randomized SVD of A*(X): U0 = U_k S^1/2, V0 = V_k S^1/2 (Sec. 4.2) */
  RPCA_INIT_RANDOM = 1, /* iid N(0, 1e-2) factors from the seeded device generator */
  RPCA_INIT_LEARNED = 2, /* the sketch start with each component scaled by a trained network's
                            share w_j (rpca_set_warm_start); kept only when F is lower there */
  RPCA_INIT_USER = 3    /* start from the U, V passed to rpca_solve */
} rpca_init_kind;

typedef struct {
  int lbfgs_mem;         /* L-BFGS memory (10, Sec. 5.1); 1..32 */
  int max_iter;          /* iteration cap of rpca_solve */
  double cert_tol;       /* stop when cert_rel <= cert_tol (1e-4) */
  int cert_every;        /* first certificate check after cert_every iterations, later ones when the
                            gradient norm predicts cert_tol is met (at most 2 cert_every apart); 0 = only
                            at the end */
  int init;              /* rpca_init_kind */
  uint64_t seed;         /* seed of the device generator (sketch, random init) */
  rpca_dtype x_dtype;    /* storage of X the objective pass reads: RPCA_F32 (the caller's X),
                            RPCA_BF16 or RPCA_FP8E4M3 (a copy the library makes at create;
                            k <= 8); see rpca_create and rpca_solve */
  int refine_fp32;       /* with narrow storage: 1 (default) = finish rpca_solve on float32 X */
  double timeout_s;      /* wall-clock limit of rpca_solve (0 = none) */
  double gtol;           /* also stop when ||grad F||_F <= gtol * max(1, |F|) (0 = off) */
  int sketch_oversample; /* rSVD oversampling p (10) */
  int sketch_power;      /* rSVD power iterations q (2) */
  double ls_noise;       /* relative noise level of F below which the line search also accepts
                            the approximate Wolfe conditions (Hager & Zhang 2005); 1e-8 */
  int autotune;          /* 1 (default): time the best launch configurations of the planner's
                            model on the device; 0: take the model's choice */
} rpca_options;

typedef struct {
  double cert;     /* ||E||_F, E in the subdifferential of lam_L ||L||_* + phi(L) at L = U V^T */
  double cert_rel; /* cert / lam_L, compared against cert_tol */
  double t1, t2, t3, t4; /* the four terms of ||E||_F^2 (Sec. 3.4) */
  double normL_F;  /* ||U V^T||_F */
  double F;        /* F(U, V) */
  double F_bound;  /* min(F(0), best F seen by this context) */
  double gap_bound;/* cert * (||L||_F + F_bound / lam_L) + F_trunc >= G(L) - G*,
                      G(L) = lam_L ||L||_* + phi(L) (the convex objective, Sec. 3.4) */
  int rank_r;      /* numerical rank of U V^T used by the certificate: singular values
                      > 1e-8 sigma_1, less the directions moved to the complement block
                      (sigma_i <= 1e-3 sigma_1 with |lam_L + u_i^T D v_i| > lam_L / 2, or
                      lam_L sigma_i <= 1e-12 F) */
  int krylov_steps;/* block Lanczos steps used for t4 */
  double sigma1_perp; /* largest singular value of P_U1perp D P_V1perp found */
  double F_trunc;  /* 2 lam_L sum of the singular values moved to the complement block: the
                      certificate is that of L with them truncated, and this bounds what the
                      truncation adds to the optimality gap (not in the paper) */
  double trunc_rel;/* F_trunc / (lam_L ||L||_F + F_bound), in the units of cert_rel:
                      gap_bound = (cert_rel + trunc_rel)(lam_L ||L||_F + F_bound).  A point
                      counts as certified at cert_tol only when cert_rel <= cert_tol and
                      trunc_rel <= cert_tol. */
} rpca_cert;

typedef struct {
  double F;        /* final objective */
  int iters;       /* L-BFGS iterations */
  int evals;       /* objective/gradient evaluations (one pass over X each) */
  int cert_evals;  /* certificate evaluations */
  double seconds;  /* wall time of rpca_solve */
  rpca_cert cert;  /* certificate at the returned point */
  rpca_status status;
  double ms_init;  /* device time of the initialisation (sketch or random), CUDA events */
  double ms_iter;  /* device time of the L-BFGS iterations (graph launches) */
  double ms_cert;  /* device time of the certificate evaluations */
  int init_used;   /* rpca_init_kind of the start actually used (RPCA_INIT_LEARNED falls back
                      to RPCA_INIT_SKETCH when the learned start's objective is not lower) */
} rpca_result;

/* Fills *opt with the defaults named in the comments above. */
RPCA_API void rpca_default_options(rpca_options *opt);

/*
 * Creates a solver context for X (m x n with 1 <= m, n <= 2^27, device, column-major,
 * ldx >= m; ldx * 4 must be a
 * multiple of 16 bytes and X 16-byte aligned, as the tiled TMA copies require), an optional
 * observation mask (device uint8, m x n column-major with ldmask >= m, nonzero = observed,
 * NULL = all observed; Sec. 6.2), factor rank k (1..16), lambda_L > 0 and lambda_S > 0
 * (lambda_S = +inf gives plain least squares, phi = 1/2 ||P_Omega(L - X)||^2).
 * opt may be NULL (defaults).  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Checks that every observed X entry is finite (RPCA_EINVAL otherwise).  Allocates the
 * context's device workspaces (partial-sum buffers, L-BFGS history of 2 * mem (m + n) k
 * floats, certificate buffers) and packs the mask into a bitmap it owns.
 * Precision form (opt.x_dtype = RPCA_BF16 or RPCA_FP8E4M3, k <= 8): the library also keeps
 * its own copy of X in that type (m x n, column-major; unobserved entries 0), rounded to
 * nearest even; FP8 E4M3 stores x / s_j, s_j = max_i |x_ij| / 448 over the observed entries
 * of column j (1 for an all-zero column), saturating at +-448.  X must still outlive the
 * context (the float32 refinement and the certificate read it).
 */
RPCA_API rpca_status rpca_create(rpca_ctx **out, int64_t m, int64_t n, const float *X, int64_t ldx,
                        const uint8_t *mask, int64_t ldmask, int k, double lambda_L, double lambda_S,
                        const rpca_options *opt, void *cuda_stream);

/*
 * One evaluation of F and its gradient at (U, V) (Eq. Thm5; gradient of phi from Sec. 3.2
 * through L = U V^T):  gU = D V + lam_L U,  gV = D^T U + lam_L V,  D = P_Omega(clip(U V^T - X)).
 * One pass over X.  f is a HOST pointer (may be NULL; the call then does not synchronise);
 * gU (m x k) and gV (n x k) are required device buffers.  The objective is summed in float64.
 * With narrow storage (opt.x_dtype) the pass reads the library's copy: F and the gradient
 * are those of the stored values (float32 arithmetic throughout).
 */
RPCA_API rpca_status rpca_fg(rpca_ctx *c, const float *U, const float *V, double *f, float *gU, float *gV);

/*
 * Products with the clipped residual D = P_Omega(clip(U V^T - X, +-lam_S)) at (U, V):
 *   DBv = D Bv  (m x b, device),   DtBu = D^T Bu  (n x b, device),
 * for 1 <= b <= 8, with Bv n x b and Bu m x b (device, column-major).  These are the matrix products the
 * certificate's spectral term needs (Sec. 3.4); one pass over X for both.
 */
RPCA_API rpca_status rpca_apply(rpca_ctx *c, const float *U, const float *V, int b, const float *Bv,
                       const float *Bu, float *DBv, float *DtBu);

/*
 * Randomized-SVD initialisation (Sec. 4.2): U0 = U_k S^1/2, V0 = V_k S^1/2 from a rank
 * k + p sketch of A*(X) (observed entries, rescaled by 1/p_hat when masked) with q power
 * iterations.  Omega is an optional device n x (k + p) Gaussian test matrix; NULL draws
 * one from the context's seeded device generator.  Writes U (m x k) and V (n x k).
 */
RPCA_API rpca_status rpca_init_sketch(rpca_ctx *c, const float *Omega, float *U, float *V);

/*
 * Minimises F with L-BFGS (memory opt.lbfgs_mem, Sec. 5.1) and a strong-Wolfe line search,
 * all on the device (direction, line search and its decisions are kernels inside a CUDA
 * graph; the host only polls a status word between graph launches).  U, V: in = the start
 * point when opt.init == RPCA_INIT_USER, out = the solution.  Stops at cert_rel <= cert_tol,
 * max_iter, gtol, or timeout.  res may be NULL.  The certificate is first evaluated after
 * cert_every iterations; after a check that did not certify, the ratio of cert_rel to the
 * gradient norm at that point predicts cert_rel from the gradient norm (read every 5
 * iterations), and the next check runs once the prediction meets cert_tol (at least 5 and at
 * most 2 cert_every iterations after the last; the narrow-storage phase keeps checks every
 * cert_every iterations).  A certificate that passes its cheap terms adds the spectral term
 * at the same point.
 * Returns RPCA_OK when the certificate tolerance was met, RPCA_ENOTCONV otherwise.
 * With narrow storage the iterations first read the library's copy of X; when the
 * (float32) certificate stops halving between checks, or that phase's iteration stops, the
 * solve continues from the point reached on float32 X with fresh L-BFGS memory (unless
 * opt.refine_fp32 == 0).  The certificate and res->F are always those of float32 X.
 */
RPCA_API rpca_status rpca_solve(rpca_ctx *c, float *U, float *V, rpca_result *res);

/*
 * Batched form: count independent problems (m[i] x n[i] float32 X[i] on the device,
 * column-major, leading dimension ldx[i] (NULL: m[i]), rank k[i], lambda_L[i], lambda_S[i],
 * fully observed), each a context of its own (rpca_create's checks and ownership rules,
 * options opt for all, launch configurations from the planner's model without device
 * timing), each with a CUDA stream the batch owns.  The paper has no counterpart: it
 * solves one problem at a time; this is an interface of this library for many small ones.
 * Errors: rpca_batch_last_error(NULL).
 */
typedef struct rpca_batch rpca_batch;
RPCA_API rpca_status rpca_create_batch(rpca_batch **out, int count, const int64_t *m, const int64_t *n,
                                       const float *const *X, const int64_t *ldx, const int *k,
                                       const double *lambda_L, const double *lambda_S, const rpca_options *opt,
                                       void *cuda_stream);
/*
 * Solves every problem of the batch as rpca_solve does (U[i], V[i]: device m[i] x k[i] and
 * n[i] x k[i] buffers, in and out), concurrently, with one of three drivers:
 *   RPCA_DRIVER_GROUPED (the default where every instance has float32 X, a factor rank
 *     <= 16 and an L-BFGS memory <= 10): the line-search trials of all unfinished instances
 *     run in shared launches, one launch of the fused objective/gradient pass per group of
 *     instances of the same factor rank and block size plus one launch each of the gradient
 *     assembly with the line-search step, the inner products with the two-loop scalars, and
 *     the direction, every kernel finding its instance from a device table; chunks of five
 *     trial rounds, between which the host takes each instance's decisions; an instance
 *     whose certificate is due leaves the table while a host worker thread evaluates it on the
 *     instance's stream, and the others keep iterating.  Each instance's iterates are those of
 *     rpca_solve on its context (the same kernels on the same grids); the iteration at which
 *     it stops can differ (decisions come after whole chunks of its trials).  res[i].ms_iter
 *     counts the instance's own launches only (the shared ones are not divided among them).
 *   RPCA_DRIVER_THREADS (RPCA_BATCH_MODE=threads, or where the grouped driver does not apply):
 *     host worker threads (environment variable RPCA_BATCH_THREADS, default 4 per hardware
 *     thread up to 64) drive the instances' solves on their own streams, so that their
 *     kernels overlap on the GPU.
 *   RPCA_DRIVER_ROUNDS (RPCA_BATCH_MODE=rounds; float32 X, k <= 16): one CUDA graph launch runs
 *     five L-BFGS iterations of every unfinished instance, each instance's kernels on a branch
 *     of their own; the host takes the certificate decisions between launches; the graph is
 *     kept by the batch for later solves.
 * Certificates (all drivers) are evaluated by host worker threads, up to RPCA_BATCH_THREADS at
 * a time.  res (may be NULL) receives count results.  Work on cuda_stream before the call is
 * ordered before the solves, and the stream is ordered after them.  Returns RPCA_OK when every
 * instance met its certificate tolerance, RPCA_ENOTCONV when some did not (see res[i].status),
 * another status on an error.
 */
RPCA_API rpca_status rpca_solve_batch(rpca_batch *b, float *const *U, float *const *V, rpca_result *res);
enum { RPCA_DRIVER_THREADS = 0, RPCA_DRIVER_ROUNDS = 1, RPCA_DRIVER_GROUPED = 2 };
/* The driver of the batch's last rpca_solve_batch (RPCA_DRIVER_*), -1 before the first. */
RPCA_API int rpca_batch_driver(const rpca_batch *b);
RPCA_API rpca_ctx *rpca_batch_context(rpca_batch *b, int i); /* instance i's context (owned by b) */
RPCA_API int rpca_batch_size(const rpca_batch *b);
RPCA_API const char *rpca_batch_last_error(const rpca_batch *b);
RPCA_API void rpca_destroy_batch(rpca_batch *b);

/*
 * The library's narrow copy of X (precision form): *dtype receives the storage type
 * (RPCA_F32 when the context keeps none, and nothing else is written).  host_out (may be
 * NULL) receives the stored elements, m x n column-major with leading dimension ld_out >= m,
 * 2 bytes each (bfloat16 bits) or 1 byte each (E4M3 codes); scales_out (may be NULL) the n
 * per-column FP8 scales.  Synchronous.
 */
RPCA_API rpca_status rpca_x_storage(rpca_ctx *c, int *dtype, void *host_out, int64_t ld_out, float *scales_out);

/*
 * The convergence certificate of Sec. 3.4 at L = U V^T: one pass over X for F and the
 * gradient terms, small float64 factorisations on the device for t1..t3, and block
 * Lanczos (passes over X through rpca_apply's kernel) for the spectral term t4.
 */
RPCA_API rpca_status rpca_certificate(rpca_ctx *c, const float *U, const float *V, rpca_cert *out);

/*
 * Releases the context and every buffer it owns (not X or the mask). NULL is allowed.  It
 * waits for the device first; the context's device and pinned host blocks are then kept by
 * the library (up to 4 GiB each) and handed to the next contexts, whose set-up then takes
 * no cudaMalloc / cudaMallocHost.
 */
RPCA_API void rpca_destroy(rpca_ctx *c);

/*
 * Returns the device and pinned host memory the library keeps from destroyed contexts to the
 * CUDA runtime, after waiting for the device.  Returns the bytes released.  Live contexts
 * keep their own buffers.
 */
RPCA_API size_t rpca_release_memory(void);

/* Message of the last failure on c (or of the last failed rpca_create when c is NULL). */
RPCA_API const char *rpca_last_error(const rpca_ctx *c);

/*
 * Launch configuration the planner picked for the fused kernel of this context
 * (which = 0: objective/gradient -- the narrow-storage plan when the context keeps a narrow
 * copy of X, the one rpca_fg uses; 1, 2: the certificate's and the sketch's D Bv products;
 * those two are planned, and tuned, on first use).
 * out[0..8] = {rows per lane R, consumer warps per CTA, row blocks, column splits,
 * columns per CTA, threads per CTA, dynamic shared memory bytes, CTAs per SM, pipeline
 * stages}.
 * The planner can be overridden with the environment variable RPCA_PLAN="warps,splits[,stages]".
 */
RPCA_API rpca_status rpca_plan_info(rpca_ctx *c, int which, int64_t *out);

/*
 * Which form of the fused objective/gradient pass a plan of c uses (which as for
 * rpca_plan_info).  out[0] = 0: the CUDA-core kernel (every product on the fp32x2 FMA pipe);
 * 1: the tensor-core kernel (R^T = X - V U^T and D^T U as warp-level tf32 MMAs with a
 * three-term hi / lo split of every operand, D V on the FMA pipe; float32 X, fg mode,
 * k <= 8, no mask); 2: factor ranks above 16 (GEMMs around an elementwise pass); 3: the
 * tcgen05 kernel (U V^T as tf32 MMAs of the 5th-generation tensor cores, four-term hi / lo
 * split, accumulated in tensor memory; D V and D^T U on the FMA pipe; float32 X, fg mode,
 * k <= 6, no mask).  out[1] =
 * row passes per CTA of the tensor-core kernel (its CTA covers out[1] x 32 x warps rows;
 * 1 otherwise).  The CUDA-core form is the default (it is faster on the workloads measured);
 * the environment variable RPCA_FG_KERNEL=mma (or =tc), set before rpca_create, plans the
 * warp-level tensor-core form (or the tcgen05 form) where it applies.  RPCA_EINVAL for a NULL argument, which out of range,
 * or a plan that cannot be made.
 */
RPCA_API rpca_status rpca_plan_kernel(rpca_ctx *c, int which, int64_t *out);

/*
 * Instrumentation (tracing).  rpca_profile(c, 1) starts recording: CUDA events bracket every
 * launch of the fused objective/gradient kernel and of its finalize kernel issued outside a
 * CUDA graph, on the context's stream, and every kernel the library issues is counted
 * (kernels inside a solver graph launch are counted from the iterations and line-search
 * trials it ran).  rpca_profile(c, 0) stops.  rpca_profile_read fills out[0..5] with
 * {fused-kernel launches timed, their total milliseconds, finalize launches timed, their
 * total milliseconds, kernels launched, CUDA-graph launches} since recording started; it
 * synchronises the stream.
 */
RPCA_API rpca_status rpca_profile(rpca_ctx *c, int enable);
RPCA_API rpca_status rpca_profile_read(rpca_ctx *c, double *out);

/*
 * Per-iteration log of the last rpca_solve on c (device log ring, copied out here): fills
 * up to max_rows rows of 7 doubles, oldest first: {iteration, F, ||grad F||_F, accepted
 * step, line-search trials, outcome (1 accepted, 2 failed), L-BFGS pairs in use}.
 * *rows receives the number of rows written (the ring keeps the last 256 iterations).
 */
RPCA_API rpca_status rpca_solve_log(rpca_ctx *c, double *out, int max_rows, int *rows);

/*
 * Per-trial log of the line searches of the last rpca_solve on c (device ring of the last
 * 256 trials, copied out here): up to max_rows rows of 7 doubles, oldest first:
 * {iteration, trial step a, F(x + a d) - F(x), phi'(a) / |phi'(0)| (directional derivative
 * along d, relative), ||grad F(x + a d)||_F^2, phase (0 bracketing, 1 zoom), trial number}.
 * The line search is the strong-Wolfe search of Nocedal & Wright Alg. 3.5/3.6 around the
 * L-BFGS iteration of Sec. 5.1.  *rows receives the number of rows written.
 */
RPCA_API rpca_status rpca_solve_trials(rpca_ctx *c, double *out, int max_rows, int *rows);

/*
 * One objective/gradient evaluation, as rpca_fg (same formulas, same kernels), that
 * allocates nothing: for callers that cannot allocate device memory where they evaluate
 * (an application that owns all device memory through its own arena and allows no
 * cudaMalloc or cudaFree on its hot path, a plugin host that hands the library only the
 * buffers it owns).  The paper has no counterpart; this is an interface of this library.  No context: X (m x n, ldx, 16-byte aligned, ldx a multiple
 * of 4, fully observed -- no mask), k in [1, 16], lambda_L, lambda_S as in rpca_create; U,
 * V in; f (HOST pointer, may be NULL), gU, gV out.  The scratch comes from one file-scope
 * device array of 32 MiB that every GPU loading the library holds until exit; shapes whose
 * partial sums need more ((ncs m + nrb n) k floats plus a little) are rejected with
 * RPCA_EINVAL and a message (use rpca_fg).  X is not checked for non-finite values.  The
 * first call on a device looks up the array's device address (make that first call before
 * any stream capture).  The call waits for the stream before it returns.  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Errors: rpca_last_error(NULL).  No launch-configuration
 * timing is done, so it can be slower than rpca_fg.
 */
RPCA_API rpca_status rpca_fg_noalloc(int64_t m, int64_t n, const float *X, int64_t ldx, int k, double lambda_L,
                                     double lambda_S, const float *U, const float *V, double *f, float *gU,
                                     float *gV, void *cuda_stream);

/*
 * Row-partitioned evaluation (the multi-GPU form of the pass; Sec. 5.4 scales the video
 * problem by its rows).  With X and U split by rows over G devices and V shared, F and its
 * gradient separate: G_{U_g} = D_g V + lam_L U_g is complete on its device, and
 *   G_V = sum_g D_g^T U_g + lam_L V,   F = sum_g (sum_{Omega_g} psi + lam_L/2 ||U_g||^2) + lam_L/2 ||V||^2.
 * rpca_fg_rows runs on a context created for one row block X_g (its own m = m_g; X_g is the
 * caller's pointer into X, 16-byte aligned, so the block starts at a row that is a multiple of
 * 4 in a column-major X whose ld is a multiple of 4) and writes the shard's terms: gU (m_g x k,
 * device) = D_g V + lam_L U_g, PV (n x k, device) = D_g^T U_g (no lam_L V), *f_part (host, may be
 * NULL; the call then does not synchronise) = sum over the shard's observed entries of psi +
 * lam_L/2 ||U_g||^2.  The caller sums PV and f_part over the shards (one all-reduce of n k + 1
 * values per evaluation, by its own communicator), then rpca_fg_rows_finish (any shard's
 * context, same n, k, lam_L) writes gV (n x k, device) = PV_sum + lam_L V and *f (host, may be
 * NULL) = f_sum + lam_L/2 ||V||^2.  k <= 16.  The paper has no counterpart for the split itself.
 */
RPCA_API rpca_status rpca_fg_rows(rpca_ctx *c, const float *U, const float *V, double *f_part, float *gU, float *PV);
RPCA_API rpca_status rpca_fg_rows_finish(rpca_ctx *c, const float *V, const float *PV_sum, double f_sum, double *f,
                                         float *gV);

/* Library version string. */
RPCA_API const char *rpca_version(void);

/*
 * Failure injection, for tests of the failure paths (the paper has no counterpart).  Faults
 * are made on the host side or by withholding work, never by a bad access on the GPU:
 *   RPCA_FAULT_FG_STARVE (c required): the next `count` launches of the fused objective/
 *     gradient kernel on c (CUDA-core form, outside CUDA graphs: rpca_fg, rpca_apply, the
 *     certificate) run with their producer warp issuing no copies and a 1 ms limit on the
 *     consumers' waits, which then run out; the call reports RPCA_ETIMEOUT, the status word is
 *     cleared, no copy is left in flight and the context stays usable.
 *   RPCA_FAULT_ALLOC (c ignored): the next `count` device allocations of context set-up
 *     (rpca_create and the workspaces it sizes) fail as out of memory (RPCA_ENOMEM); the
 *     partly built context is released.
 * count = 0 clears the fault.  RPCA_EINVAL for an unknown kind or count < 0.
 */
enum { RPCA_FAULT_FG_STARVE = 1, RPCA_FAULT_ALLOC = 2 };
RPCA_API rpca_status rpca_inject_fault(rpca_ctx *c, int kind, int count);

/*
 * Unit singular vectors (u: device m floats, v: device n floats) of the largest singular value
 * of P_U1perp D P_V1perp at the point of this context's last full certificate (the spectral
 * term of Sec. 3.4), from its block-Lanczos bases; *sigma1 (may be NULL) = that singular value,
 * u^T D v = sigma1.  Needs a certificate with a spectral step (rpca_certificate, or the end of
 * rpca_solve) on this context.  The spectral step locates the Ritz values alone; the first call
 * after it forms the leading Ritz pairs by a one-sided Jacobi SVD of its projected matrix (one
 * launch, tens of microseconds), later calls reuse them.  Synchronous.
 */
RPCA_API rpca_status rpca_perp_direction(rpca_ctx *c, float *u, float *v, double *sigma1);
/* The q <= min(qmax, 16) leading pairs of the same: U (device, m x q, ld ldu >= m), V (device,
 * n x q, ld ldv >= n), sig (host, q values, descending), *q_out = q (at most the Ritz values
 * the last spectral step computed).  Synchronous. */
RPCA_API rpca_status rpca_perp_directions(rpca_ctx *c, int qmax, float *U, int64_t ldu, float *V, int64_t ldv,
                                          double *sig, int *q_out);

/*
 * Dynamic rank increase (Sec. 4.1).  U, V: device m x kmax and n x kmax buffers (column-major,
 * leading dimensions m and n); the first k columns (k of the context) follow rpca_solve's
 * rules.  Solves; a solve at a rank that cannot certify stops once t1..t3 meet the tolerance
 * while t4 > 0.  While the certificate's spectral term shows directions the factors cannot
 * represent (singular values sigma_i of P_U1perp D P_V1perp above lam_L) and the rank is below
 * kmax (<= 16), one column (sqrt(t_i) u_i, -sqrt(t_i) v_i), t_i = sigma_i - lam_L, is added per
 * such direction (the minimiser of the quadratic upper bound of F along it; the paper leaves
 * the column open and allows growing k aggressively), kept when F drops, and the solve
 * continues from the grown point at the new rank (contexts for larger ranks are made on demand
 * and owned by c).  *k_out = the final rank; res (may be NULL) = the last solve's result with the
 * iteration, evaluation and time counts of all of them.
 */
RPCA_API rpca_status rpca_solve_grow(rpca_ctx *c, float *U, float *V, int kmax, rpca_result *res, int *k_out);

/*
 * Frank-Wolfe method with marginalization (Sec. 6.2, Algorithm 1), the paper's alternative
 * solver of the convex program min over ||L||_* <= t of lam_L t + phi(L), on a dense L.
 * L: device m x n float32 (column-major, ld ldl >= m a multiple of 4, 16-byte aligned), the
 * start on entry (the zero matrix: t_0 = 0) and the iterate on return.  Each iteration: the
 * gradient G = P_Omega(clip(L - X)), the top singular pair of G by power_iters power
 * iterations (warm-started), the vertex V = -B u v^T (or 0 when sigma_1 <= lam_L), the exact
 * line search of the printed quadratic with S fixed (its lam_L term read as lam_L ((1 - eta) t
 * + eta Vt)), L <- (1 - eta) L + eta V, t likewise, the radius bound B as printed.  Stops when
 * the Frank-Wolfe gap <G, L - V> + lam_L (t - Vt) <= gap_tol max(1, |F|) or after max_iter
 * iterations.  log (host, may be NULL): 4 doubles per iteration {F(L, t) before the step,
 * gap, sigma_1, eta}.  float32 X only (no narrow storage).  Synchronous.
 */
typedef struct {
  double F;        /* phi(L) + lam_L t at the returned iterate */
  double t;        /* the nuclear-norm bound (>= ||L||_*) */
  double gap;      /* Frank-Wolfe gap of the last iteration */
  double sigma1;   /* top singular value of the last gradient */
  int iters;       /* iterations taken */
  double seconds;  /* wall time */
} rpca_fw_result;
RPCA_API rpca_status rpca_fw_solve(rpca_ctx *c, float *L, int64_t ldl, int max_iter, double gap_tol, int power_iters,
                                   double *log, rpca_fw_result *res);

/*
 * TSQR (Sec. 6.1, after Demmel, Grigori, Hoemmen and Langou 2012): A = Q R for a tall-skinny
 * device matrix A (rows x l, float32, column-major, ld lda >= rows; 1 <= l <= 32, rows >= l),
 * by a reduction tree of float32 Householder QRs (row blocks first, then groups of stacked R's).
 * Q: device rows x l (column-major, ld ldq >= rows) with orthonormal columns; R: device l x l
 * (column-major, may be NULL), upper triangular with a non-negative diagonal (the unique QR of a
 * full-rank A).  A rank-deficient A still gives an orthonormal Q with Q R = A.  Scratch is
 * allocated and freed on c's stream.  Synchronous.  RPCA_EINVAL on bad sizes.
 */
RPCA_API rpca_status rpca_tsqr(rpca_ctx *c, const float *A, int64_t lda, int64_t rows, int l, float *Q, int64_t ldq,
                               float *R);

/*
 * The convex baseline of Sec. 6.1: FISTA (unit step) on the Lagrangian program
 * min_L lam_L ||L||_* + phi(L) (S marginalised), whose singular-value thresholding is taken on a
 * rank-l randomized SVD of the gradient point Z = Y - P_Omega clip(Y - X) with power_iters power
 * iterations and every QR a TSQR (rpca_tsqr's algorithm); the test matrix of each iteration is
 * the right singular basis found by the previous one (Omega0 for the first).  Iteration k:
 * Y = L_k + beta_k (L_k - L_{k-1}) (beta_0 = 0, beta_k = (t_{k-1} - 1) / t_k, t_0 = 1,
 * t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2), L_{k+1} = left diag(max(s - lam_L, 0)) right^T.
 * L: device m x n float32 (column-major, ld ldl >= m a multiple of 4, 16-byte aligned); the
 * solve starts from L = 0 and returns the last iterate L_k in it.  l: the sketch width, 1 <= l
 * <= min(32, m, n); the prox is exact while fewer than l singular values of Z exceed lam_L
 * (res->truncated reports the last one that was not).  Omega0: device n x l float32
 * (column-major, ld n), e.g. standard normal.  Stops at the first k >= 1 with
 * ||L_k - L_{k-1}||_F <= tol max(1, ||L_k||_F), or at k = max_iter.  profile != 0 times the
 * phases with CUDA events.  log (host, may be NULL): 4 doubles per iterate k = 0 .. iters
 * {F(L_k) = lam_L ||L_k||_* + phi(L_k), the relative change, rank L_k, the l-th sketch singular
 * value that formed L_k}.  float32 X only.  Synchronous.
 */
typedef struct {
  double F;           /* lam_L ||L||_* + phi(L) at the returned iterate */
  double phi;         /* phi(L) */
  double nuclear;     /* ||L||_* (the thresholded singular values that formed L) */
  double rel_change;  /* ||L_k - L_{k-1}||_F / max(1, ||L_k||_F) */
  int iters;          /* prox steps taken (the returned iterate is L_iters) */
  int rank;           /* rank of the returned L */
  int truncated;      /* 1 if the last prox kept all l sketch directions (l may be too small) */
  double seconds;     /* wall time */
  double ms_pass, ms_rsvd, ms_tsqr, ms_recon; /* device time of the phases (profile), else 0;
                                                 ms_tsqr is part of ms_rsvd */
} rpca_convex_result;
RPCA_API rpca_status rpca_convex_solve(rpca_ctx *c, float *L, int64_t ldl, int l, int power_iters,
                                       const float *Omega0, int max_iter, double tol, int profile, double *log,
                                       rpca_convex_result *res);

/*
 * Corrected Akaike information criterion of the solution L = U V^T (Sec. 5.2), the paper's
 * model-quality measure: S = shrink(X - L, lam_S) on the observed set, Z = L + S - X,
 * sigma^2 = ||X||^2 / N, b = ||S||_1 / N, b_* = ||L||_* / rank(L) (N = observed entries),
 * ell = -(N/2) log(2 pi sigma^2) - ||Z||^2/(2 sigma^2) - N log(2b) - ||S||_1/(2b)
 *       - rank(L) log(2 b_*) - ||L||_* / (2 b_*),
 * p = r (m + n - r) + nnz(S) + (||Z||^2 / ||X||^2) N, AIC_c = 2 (p - ell) + 2 p (p + 1) / (N - p - 1);
 * rank(L) counts singular values above 1e-6 of the largest.  U, V: device factors (k columns).
 * float32 X only.  Synchronous.
 */
typedef struct {
  double aicc, loglik, dof;
  int rank;         /* rank of L */
  double nuclear;   /* ||L||_* */
  double s_l1;      /* ||S||_1 */
  int64_t nnz_s;    /* nonzeros of S */
  double resid2;    /* ||Z||_F^2 */
  double x2;        /* ||X||_F^2 over the observed entries */
  int64_t count;    /* observed entries */
} rpca_aicc_result;
RPCA_API rpca_status rpca_aicc(rpca_ctx *c, const float *U, const float *V, rpca_aicc_result *out);

/* ---- Learned warm start ---------------------------------------------------------------
 * An extension of this library (the paper compares SVD, randomized-SVD and random starts,
 * Sec. 4.2, and finds that the start matters).  A three-layer network (40 inputs, two hidden
 * layers of 256 with ReLU, 16 sigmoid outputs; weight matrices used in bfloat16, float32
 * arithmetic) maps features of the randomized sketch's spectrum to the share w_j in [0, 1]
 * of each sketch component that the solution keeps; the learned start is the sketch start
 * with column j of U0 and V0 scaled by sqrt(w_j).
 *
 * Features x (40 floats) of a context whose last initialisation ran the sketch, with
 * s_1 >= ... >= s_l its singular values of A*(X) (l = k + sketch_oversample, <= 32):
 *   x_j = log(s_j / s_l) (j < l; 0 for l <= j < 32), x_32 = log(lam_L / s_l),
 *   x_33 = log(lam_S sqrt(m n) / s_l) (0 when lam_S is infinite), x_34 = k / 16,
 *   x_35 = l / 32, x_36 = log(m / n) / 4, x_37 = log(m n) / 20, x_38 = x_39 = 0.
 * Target of component j: w*_j = clip(u_j^T L* v_j / s_j, 0, 1), u_j and v_j the sketch's unit
 * singular vectors, L* = U V^T a solution.  Loss (1 / B) sum_b sum_{j < k_b} (w_j - w*_j)^2,
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on float32 master parameters, the gradient taken
 * at the bfloat16-rounded weights.
 *
 * Parameters (rpca_ws_nparam() floats, packed): W1 (256 x 40, row-major) | b1 (256) |
 * W2T (256 x 256, W2T[i][u] = W2[u][i]) | b2 (256) | W3 (16 x 256, row-major) | b3 (16).
 * Errors of the model calls: rpca_ws_last_error(model) (NULL before a model exists).
 */
RPCA_API int rpca_ws_nparam(void);
/* A model with parameters theta (host, rpca_ws_nparam() floats); calls run on cuda_stream. */
RPCA_API rpca_status rpca_ws_create(rpca_ws **out, const float *theta, void *cuda_stream);
/* Replaces the parameters (host) and resets the optimiser state.  Synchronous. */
RPCA_API rpca_status rpca_ws_set_params(rpca_ws *w, const float *theta);
/* Copies the parameters and (grad may be NULL) the last training step's gradient to host. */
RPCA_API rpca_status rpca_ws_get_params(rpca_ws *w, float *theta, float *grad);
/* W (device, B x 16) = the network's outputs for the features X (device, B x 40, row-major). */
RPCA_API rpca_status rpca_ws_predict(rpca_ws *w, const float *X, int B, float *W);
/* One Adam step on the batch (device X: B x 40, T: B x 16 targets, K: B factor ranks; outputs
 * j >= K[b] are ignored) with step size lr; *loss (host, may be NULL; synchronises) = the
 * batch loss at the parameters before the step. */
RPCA_API rpca_status rpca_ws_train_step(rpca_ws *w, const float *X, const float *T, const int *K, int B, float lr,
                                        float *loss);
RPCA_API const char *rpca_ws_last_error(const rpca_ws *w);
RPCA_API void rpca_ws_destroy(rpca_ws *w);
/* The model opt.init == RPCA_INIT_LEARNED uses on this context (not owned; NULL clears). */
RPCA_API rpca_status rpca_set_warm_start(rpca_ctx *c, const rpca_ws *w);
/* The l singular values (host, <= 32 floats) of the context's last sketch; *l = 0 if none. */
RPCA_API rpca_status rpca_sketch_spectrum(rpca_ctx *c, float *s, int *l);
/* A training sample: x (device, 40) = the features of the context's last sketch; if wstar
 * (device, 16) is not NULL, the targets of the sketch start (Us, Vs: device m x k and n x k,
 * as rpca_init_sketch wrote them) against the solution (U, V); entries j >= k are 0. */
RPCA_API rpca_status rpca_ws_sample(rpca_ctx *c, const float *Us, const float *Vs, const float *U, const float *V,
                                    float *x, float *wstar);

/* ---- Counter-based generator of planted instances (training data) ------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011), key = seed (low word first).
 * rpca_gen_planted writes X (device, m x n column-major, ld ldx >= m) = A B^T + S + N and,
 * if L0 is not NULL (device, m x n, ld m), A B^T:
 *   A[i][c]: counter (i, c, 0, instance); B[j][c]: (j, c, 1, instance); entry (i, j): (i, j, 2,
 *   instance).  uniform24(w) = (w >> 8) 2^-24; normal(wa, wb) = sqrt(-2 ln(((wa >> 8) + 1) 2^-24))
 *   cos(2 pi uniform24(wb)).  A, B = rank^(-1/4) normal(w0, w1) (L entries of unit variance);
 *   outlier where uniform24(w0) < p_outlier, value +-(1 + 4 (w1 & 0xffffff) 2^-24), negative
 *   when the top bit of w1 is set; N = noise_std normal(w2, w3).  m, n < 2^32, rank <= 64.
 * rpca_philox4x32_10 writes count x 4 words (device out) for the counters (ctr[0] + t, ctr[1],
 * ctr[2], ctr[3]) (host ctr), t < count.  Both are asynchronous on cuda_stream; errors:
 * rpca_last_error(NULL).
 */
RPCA_API rpca_status rpca_gen_planted(int64_t m, int64_t n, int rank, double p_outlier, double noise_std, uint64_t seed,
                                      uint32_t instance, float *X, int64_t ldx, float *L0, void *cuda_stream);
RPCA_API rpca_status rpca_philox4x32_10(uint32_t *out, int64_t count, const uint32_t *ctr, uint64_t key,
                                        void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RPCA_H */
