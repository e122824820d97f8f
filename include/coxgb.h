/*
 * coxgb.h -- C ABI of the GB300 l1-regularised Cox proportional-hazards
 * proximal-gradient library (libcoxgb.so).
 *
 * Method: Ko, Zhou, Zhou & Won, "DistStat.jl" (arXiv 2010.16114), Section 5.3
 * (partial likelihood, proximal-gradient iteration, sorted cumulative sums,
 * step size), Section 4.2 (soft threshold), Section 4.4 (power method),
 * Section 6 (Breslow ties, lag-10 stopping rule).
 *
 * Notation: n subjects, p predictors (SNPs), k penalty values solved
 * together (k <= 64 on the tensor cores in the e4m3 form, k <= 16 in the e2m1
 * form; calls with more return COX_ERR_ARG).  y = observed times, delta =
 * event indicators.  The library
 * centres the design, X_c = X - 1 mu^T with mu_j the column mean, when
 * cox_options.center is 1, and works with
 *     f(beta)  = -(1/n) sum_i delta_i [ eta_i - log sum_{j: y_j >= y_i} exp(eta_j) ],
 *     eta      = X_c beta,
 *     g(beta)  = X_c^T (delta - u) / n = -grad f,   u = P delta (Section 5.3),
 *     F(beta)  = f(beta) + lambda ||beta||_1,
 *     one step : beta <- S(beta + sigma g, sigma lambda),  sigma = step.
 * Ties in y are handled by Breslow's rule: every subject with y_j >= t is in
 * the risk set at t, and tied events share that risk set.
 *
 * Conventions for every call:
 *   - Return value: COX_OK (0) or a negative COX_ERR_* code; no call throws
 *     or aborts across this boundary.  cox_strerror() names the code.
 *   - Pointers named *_dev are device pointers on the handle's device;
 *     *_host are host pointers.  The caller owns every buffer it passes; the
 *     library owns the handle and everything it allocates for it.
 *   - Coefficient matrices are p x k column-major: entry (j, c) at c*p + j,
 *     column c belonging to lambdas[c].  Element type: float, except for a
 *     handle created with precision COX_FP64, where it is double.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is ordered on it.  Calls that return host values
 *     synchronise the stream before returning; cox_prox_step does not, and a
 *     device-side error it meets is reported by the next synchronising call
 *     (cox_sync, cox_loss_grad, cox_path_fit, cox_prox_step_host).
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef COXGB_H
#define COXGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cox_handle *cox_h;

enum {
    COX_OK = 0,
    COX_ERR_ARG = -1,           /* bad shape, pointer, option or value        */
    COX_ERR_CODE3 = -2,         /* genotype code 3 (not in {0,1,2})           */
    COX_ERR_OOM = -3,           /* device or host allocation failed           */
    COX_ERR_CUDA = -4,          /* a CUDA runtime call failed                 */
    COX_ERR_TIMEOUT = -5,       /* a device-side wait ran out its limit       */
    COX_ERR_NONFINITE = -6,     /* eta, W or the loss became non-finite       */
    COX_ERR_NOT_CONVERGED = -7, /* warning: a path column hit max_iter        */
    COX_ERR_STATE = -8,         /* state blob does not match the handle       */
    COX_ERR_UNSUPPORTED = -9    /* no sm_103a device, or mode/format mismatch */
};

/* How X is passed to cox_setup. */
enum {
    COX_X_INT8_HOST = 0,    /* uint8 codes {0,1,2}, n x p row-major, host          */
    COX_X_F64_HOST = 1,     /* double, n x p row-major, host (COX_FP64 only)        */
    COX_X_PACKED2_HOST = 2, /* 2-bit codes, row-major, ceil(p/4) bytes per row,     */
    COX_X_PACKED2_DEV = 3   /*   SNP j in bits 2*(j%4)+{0,1} of byte j/4; host/dev  */
};

/* Arithmetic of the two products X_c B and X_c^T V. */
enum {
    COX_SPLIT_E4M3 = 0, /* tcgen05 tensor cores (kind::f8f6f4): genotype codes as
                           e4m3, coefficients split into 4 e4m3 limbs under a
                           power-of-two column scale, FP32 accumulation; FP64
                           risk-set scans (default)                            */
    COX_FP64 = 1,       /* FP64 everywhere, dense X (COX_X_F64_HOST)          */
    COX_FP32_GEMV = 2,  /* baseline: one lambda at a time, FP32 CUDA-core GEMV
                           on the packed genotypes, unfused soft threshold    */
    COX_SPLIT_E2M1 = 3  /* tcgen05 tensor cores (kind::mxf4, unit block scales):
                           genotype codes as e2m1 (two per byte, K = 64 per
                           MMA), coefficients split into 8 e2m1 limbs on the
                           grid of halves under a power-of-two column scale
                           (within 2^-23 of the column's largest magnitude),
                           FP32 accumulation; FP64 risk-set scans; k <= 16  */
};

typedef struct cox_options {
    int precision;        /* COX_SPLIT_E4M3 (default), COX_SPLIT_E2M1, COX_FP64,
                             COX_FP32_GEMV                                         */
    int center;           /* 1: X_c = X - 1 mu^T (default 1; COX_FP64 default 0)    */
    int device;           /* CUDA device ordinal (default: current device)           */
    int tile_m;           /* 128-row tiles per pipeline stage of the tensor-core
                             products (1 or 2); 0 = automatic: the cox_autotune
                             choice for the call's k if there is one, else a
                             built-in default                                       */
    int stages;           /* shared-memory pipeline depth; 0 = automatic             */
    int lag;              /* stopping-rule lag in iterations (default 10, Section 6) */
    double wait_limit_s;  /* device-side wait limit in seconds (default 2.0)         */
    int chunks;           /* 128-wide K chunks per pipeline stage (1 or 2; 3 with
                             two row tiles at 64 limb columns, k = 9..16, where
                             the product's chunk count divides by 3; COX_SPLIT_E2M1:
                             2, or 4 with one row tile);
                             0 = automatic, as tile_m                               */
    int window;           /* K chunks a TMEM accumulator sums in FP32 before decoder
                             warps add it into FP32 sums (>= chunks; 0 = 256)       */
    int issue;            /* MMA issue of the tensor-core products: 1 = one issuer
                             warp per row tile, every stage (4 chunks MMAs per
                             commit); 2 = two issuer warps on alternate stages,
                             each issuing every row tile of its stage (4 chunks
                             tile_m MMAs per commit); 3 = as 1, each issuer
                             committing after every second stage (8 chunks MMAs
                             per pair of commits); 0 = automatic, as tile_m      */
    int active_set;       /* 1: the X B product streams only the SNP columns where
                             some coefficient is nonzero (a gathered copy of those
                             columns, rebuilt when the support leaves it), or the
                             dense copy when the support exceeds a quarter of the
                             columns; each iteration then synchronises its stream
                             once, and cox_path_fit runs plain launches instead
                             of graph replays.  0 (default): always dense        */
} cox_options;

/* Fill *opt with the defaults above. */
void cox_default_options(cox_options *opt);

/*
 * Create a handle for one data set (Section 5.3 problem statement: X, y,
 * delta).  Sorts subjects by y (stable), records Breslow tie groups, computes
 * column means mu (exact integer sums for genotypes), and lays X out in
 * device memory: two 2-bit tiled copies (subject-major and SNP-major) for the
 * genotype modes, dense row- and column-major FP64 copies for COX_FP64.
 *   X       : as x_format says; host buffers are copied, a COX_X_PACKED2_DEV
 *             buffer is read during setup only (the caller may free it after).
 *   n, p    : >= 1.  Genotype modes accept n, p up to 2^31 - 1 each.
 *   time    : n finite doubles (host).  event: n bytes, 0 or 1 (host).
 *   opt     : NULL for defaults.
 * Errors: COX_ERR_ARG (shapes, non-finite time, event not 0/1, format not
 * allowed for the precision), COX_ERR_CODE3, COX_ERR_OOM, COX_ERR_CUDA,
 * COX_ERR_UNSUPPORTED (device is not sm_103).  On error *out is NULL.
 */
int cox_setup(cox_h *out, const void *X, int64_t n, int64_t p, int x_format,
              const double *time, const uint8_t *event, const cox_options *opt);

/* Release the handle and all device memory it owns.  NULL is a no-op. */
void cox_destroy(cox_h h);

/*
 * L = 2 ||X_c||_2^2 / n, the Lipschitz constant the step 1/L is built from
 * (Section 5.3 step-size remark, rescaled to the 1/n loss), with ||X_c||_2
 * from the power method of Section 4.4: stop when the estimate changes by at
 * most tol relative (tol <= 0: the paper's 1e-6) or after maxiter iterations
 * (maxiter <= 0: the paper's 1000).  start_host: p doubles, the start vector
 * (NULL: all ones).  Synchronous.
 */
int cox_lipschitz(cox_h h, const double *start_host, double tol, int maxiter, double *L_out);

/*
 * cox_lipschitz without any device allocation.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory at
 * call time: a process whose GPU memory is already reserved by another
 * allocator (a framework's caching pool, a fixed arena), so that cudaMalloc
 * fails or must not be used, and latency-sensitive loops that cannot afford
 * the device-wide synchronisation cudaFree implies.
 *
 * Same arguments, result and power method as cox_lipschitz.  The work
 * vectors live in a 16 MiB array built into the library (every GPU that loads
 * the library holds it until the process exits).  Limit: the call needs
 *   4 (p + 2 n_pad + p_pad) + 256   bytes (genotype handles),
 *   8 (2 p + n) + 256               bytes (COX_FP64 handles),
 * plus 8 p when start_host is given, each term rounded up to 256; larger
 * problems get COX_ERR_ARG (n_pad, p_pad from cox_get_info).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture.  A device
 * reset (cudaDeviceReset, or an embedder resetting the primary context)
 * invalidates that address as it does every handle: neither a handle nor
 * this call may be used across a reset.  Calls share the array: calls that
 * overlap on the GPU race; each call writes everything it reads.  Calls no
 * cudaMalloc, cudaFree or allocating library routine.  Synchronous (legacy
 * stream).
 */
int cox_lipschitz_noalloc(cox_h h, const double *start_host, double tol, int maxiter, double *L_out);

/* lambda_max = ||g(0)||_inf: the smallest lambda for which beta = 0 solves
 * the problem (g(0) uses u(0), the Nelson-Aalen hazard).  Synchronous. */
int cox_lambda_max(cox_h h, double *lmax_out);

/*
 * Loss and gradient at k coefficient vectors (Section 5.3 Delta, no prox):
 *   beta_dev : p x k coefficients (device, column-major).
 *   loss_host: k doubles, f(beta_c) (no penalty).  May be NULL.
 *   grad_dev : p x k, grad f = -X_c^T (delta - u) / n (device).  May be NULL.
 * Synchronous (returns after the stream has drained).
 */
int cox_loss_grad(cox_h h, const void *beta_dev, int k, double *loss_host, void *grad_dev,
                  void *stream);

/*
 * Linear predictor eta = X_c B for k columns (Section 5.3, first step of the
 * iteration), the quantity a column-sharded run would add up across shards:
 * with X split by SNP columns into X_1 .. X_G, eta = sum_g (X_g)_c B_g.
 *   beta_dev : p x k (device; float, double for COX_FP64 handles).
 *   eta_dev  : k x n doubles (device), subjects in the handle's sorted order
 *              (rank r = entry r of the order from cox_get_mu_order).
 * Synchronous.  Errors: COX_ERR_UNSUPPORTED for COX_FP32_GEMV handles.
 */
int cox_eta(cox_h h, const void *beta_dev, int k, double *eta_dev, void *stream);

/*
 * One proximal-gradient iteration for k penalties at once (Section 5.3):
 * eta = X_c B, risk-set scans, G = X_c^T V, beta <- S(beta + step g, step lambda).
 *   beta_dev : p x k in/out (device).
 *   lambdas  : k penalties (host, >= 0).  step: sigma > 0.
 * Asynchronous on `stream`.  The handle keeps F(beta entering this step)
 * per column; cox_last_objective() reads it.
 */
int cox_prox_step(cox_h h, void *beta_dev, const double *lambdas, int k, double step,
                  void *stream);

/* As cox_prox_step with beta in host memory (copied in and out inside the
 * call); synchronous.  The end-to-end form of one iteration. */
int cox_prox_step_host(cox_h h, void *beta_host, const double *lambdas, int k, double step,
                       void *stream);

/*
 * One iteration of a column shard (Section 5.3 with X split by SNP columns
 * over devices, as the paper's distributed matrices split it): given the
 * linear predictor summed over all shards, eta = sum_g (X_g)_c B_g (each
 * shard's part from cox_eta, added by the caller, e.g. by an all-reduce),
 * run the risk-set scans (every shard computes the same ones) and this
 * handle's X_g^T V with the soft-threshold step on its coefficients.
 *   beta_dev: p_g x k in/out (device; this shard's columns).
 *   eta_dev : k x n doubles (device), sorted order as cox_eta writes it.
 * With covariates set (the same Z on every shard) the handle adds Z gamma and
 * steps gamma, identically on every shard.  F of the entering iterate needs
 * ||beta||_1 over all shards: cox_last_loss_l1 gives this shard's part.
 * Asynchronous.  Errors: COX_ERR_UNSUPPORTED for COX_FP32_GEMV handles.
 */
int cox_prox_step_eta(cox_h h, void *beta_dev, const double *eta_dev, const double *lambdas, int k,
                      double step, void *stream);
/* f (the loss, k doubles) and this handle's ||beta||_1 (k doubles) at the
 * iterate that entered the last step or evaluation; either may be NULL.
 * Synchronous. */
int cox_last_loss_l1(cox_h h, double *f_host, double *l1_host, int k, void *stream);

/* Wait for `stream` and report any device-side error of earlier calls. */
int cox_sync(cox_h h, void *stream);

/* F_lambda at the iterate that entered the last cox_prox_step, per column
 * (k doubles, host).  Synchronous. */
int cox_last_objective(cox_h h, double *obj_host, int k, void *stream);

/*
 * Solve k penalties from beta = 0 (or from beta_dev when warm != 0), each
 * column until |F_t - F_{t-lag}| / |F_t + 1| < tol (Section 6 stopping rule,
 * F = penalised objective) or max_iter.  A converged column is frozen: its
 * result equals a solo run.  Iterations run as CUDA-graph replays of `lag`
 * steps; the host reads k objectives per replay.
 *   beta_dev  : p x k (device) out (in too when warm).
 *   iters_host: k ints, iterations each column ran.  obj_host: k doubles,
 *               final F.  Either may be NULL.
 * Returns COX_OK, or COX_ERR_NOT_CONVERGED if some column hit max_iter.
 */
int cox_path_fit(cox_h h, const double *lambdas, int k, int max_iter, double tol, double step,
                 int warm, void *beta_dev, int *iters_host, double *obj_host, void *stream);

/*
 * The Section 6 lambda path, one penalty after another (the UK Biobank fit
 * ran each lambda of its grid to the stopping rule): lambdas[l] is solved
 * from beta = 0 (warm = 0) or from the solution of lambdas[l-1] (warm = 1),
 * with its unpenalised coefficients gamma likewise (when covariates are set),
 * each to |F_t - F_{t-lag}| / |F_t + 1| < tol or max_iter iterations, as
 * CUDA-graph replays of `lag` steps (the rule of cox_path_fit with k = 1).
 *   B_dev     : p x L coefficients (device) out, column l at lambdas[l].
 *   G_host    : q x L doubles (host) out, column l = gamma at lambdas[l]; may
 *               be NULL (and is not written when no covariates are set).
 *   iters_host: L ints; obj_host: L doubles (final F).  Either may be NULL.
 * Returns COX_OK, or COX_ERR_NOT_CONVERGED if some lambda hit max_iter.
 */
int cox_path_seq(cox_h h, const double *lambdas, int L, int max_iter, double tol, double step, int warm,
                 void *B_dev, double *G_host, int *iters_host, double *obj_host, void *stream);

/*
 * Unpenalised covariates (Section 6: sex and ten principal components enter
 * the UK Biobank model without a penalty).  With Z set, every iteration works
 * with eta = X_c beta + Z gamma: beta takes the soft-threshold step, gamma the
 * plain gradient step gamma <- gamma + step Z^T (delta - u) / n, and the
 * penalty covers beta only (F = f + lambda ||beta||_1).  Z is used as given
 * (the partial likelihood does not see a shift of a column).
 *   Z_host: n x q doubles, row-major, subjects in cox_setup's order; finite.
 *   q     : 0 .. COX_MAX_COVARIATES (0 removes the covariates).
 * gamma (q x k doubles, column c for lambdas[c]) belongs to the handle: it is
 * zero after this call and whenever the number of columns k changes, and
 * cox_path_fit with warm = 0 starts it from zero (warm = 1 keeps it, warm = 2
 * restores the checkpoint's).  cox_lambda_max and cox_loss_grad evaluate at
 * the handle's gamma; cox_eta returns X_c B alone.  Drops the per-k workspace.
 */
enum { COX_MAX_COVARIATES = 16 };
int cox_set_covariates(cox_h h, const double *Z_host, int q);
/* gamma of the handle for k columns (q x k doubles, host): read, or write
 * (gamma_host NULL: zero).  No covariates: no-op.  cox_get_gamma needs the
 * workspace for k (a call with k columns since the last change). */
int cox_get_gamma(cox_h h, double *gamma_host, int k);
int cox_set_gamma(cox_h h, const double *gamma_host, int k);
/* The gradient of f with respect to gamma at the last evaluation for k
 * columns (q x k doubles, host): -Z^T (delta - u) / n. */
int cox_grad_gamma(cox_h h, double *grad_host, int k);

/* Checkpoint: the solver state of the last path fit / step (coefficients,
 * gamma, iteration counters, objective history).  cox_get_state with buf ==
 * NULL sets *size to the bytes needed.  cox_set_state restores it (same n, p,
 * k, precision, covariate count) so a path fit resumes bit-identically. */
int cox_get_state(cox_h h, void *buf, size_t *size);
int cox_set_state(cox_h h, const void *buf, size_t size);

/* Handle facts: n, p, padded sizes, precision, tile choice, device bytes,
 * and the number of kernels the library has launched on this handle. */
typedef struct cox_info {
    int64_t n, p, n_pad, p_pad;
    int precision, center, tile_m, stages, sm_count;
    int64_t device_bytes;
    int64_t n_tie_groups;
    int64_t launches;
    int chunks, ring;     /* K chunks per stage and TMEM slots of the X B product  */
    int issue, issue_xtv; /* issue mode (cox_options.issue) of the X B and X^T V
                             products in use                                       */
    int64_t active_cols;  /* active set: SNP columns in it (-1: off or not built)  */
    int64_t active_rebuilds; /* times the active set was rebuilt                    */
} cox_info;
int cox_get_info(cox_h h, cox_info *info);

/*
 * Autotuner of the tensor-core products (COX_SPLIT_E4M3 and COX_SPLIT_E2M1
 * handles; the choice is kept per operand form and k).  For k coefficient
 * columns it times every plannable pipeline shape of the handle's operand form
 * (row tiles and K chunks per stage; per-tile and alternating issuers) of both products at
 * the planner's shared-memory depth on the handle's resident genotypes: one
 * warm-up and `reps` launches each, CUDA events on the legacy stream, the
 * device synchronised after each shape, partial outputs only (no coefficient
 * changes).  The fastest shape per product is kept for k and used by later
 * calls with k columns unless cox_options forces tile_m, chunks or stages.
 * xb / xtv (either may be NULL) receive the choice and its mean launch time.
 * Drops the per-k workspace.  Synchronous.  Errors: COX_ERR_UNSUPPORTED for
 * other precisions; COX_ERR_ARG for k outside 1..64 (1..16 for COX_SPLIT_E2M1)
 * or reps < 1.
 */
typedef struct cox_tune_choice {
    int tile_m, chunks, stages, candidates;
    double ms;
    int issue;            /* cox_options.issue of the choice (1 or 2)               */
} cox_tune_choice;
int cox_autotune(cox_h h, int k, int reps, cox_tune_choice *xb, cox_tune_choice *xtv);

/*
 * Pipeline plan of the tensor-core products (the genotype products X beta and
 * X^T (delta - u) of each iteration, Section 5.3), computed on the host
 * without a device or handle: for k coefficient columns (1..64) and a shape
 * (tile_m 128-row tiles per CTA, chunks 128-wide K chunks per stage, issue as
 * cox_options.issue; 0 = the built-in default) at a shared-memory depth
 * (stages; 0 = the deepest that fits), the plan cox_setup's handles would
 * launch.  Every plan it returns keeps the pipeline's invariants: ring >=
 * decoder_groups, ring < stages (e2m1: ring < limb_stages), named_barriers <= 15, tmem_cols <= 512,
 * smem_bytes within the device's per-block limit, and for issue 2 two decoder
 * groups with an even ring and an even number of stages.  Errors: COX_ERR_ARG
 * for a NULL out, k outside 1..64, a shape not compiled for k's limb-column
 * class, or a depth outside those invariants.
 */
typedef struct cox_plan {
    int tile_m, chunks, stages;
    int ring;             /* TMEM slots of decoded genotype codes                  */
    int decoder_groups;   /* decoder warp groups (each takes every G-th stage)     */
    int named_barriers;   /* hardware barriers in use: lcm(groups, ring) x tile_m  */
    int limb_cols;        /* e4m3 limb columns: N of every MMA                     */
    int tmem_cols;        /* accumulators + slots, of the 512 an SM has            */
    long long smem_bytes; /* dynamic shared memory per CTA                         */
    int issue;            /* 1 one issuer per row tile, 2 two on alternate stages,
                             3 one per row tile committing every second stage      */
    int issuers;          /* MMA issuer warps                                      */
    int mmas_per_commit;  /* tcgen05.mma instructions per issuer commit            */
    int limb_stages;      /* COX_SPLIT_E2M1: slots of the limb ring, ring + 2 (the
                             codes then have a ring of their own, `stages` deep,
                             freed as soon as they are decoded); 0 otherwise      */
} cox_plan;
int cox_plan_shape(int k, int tile_m, int chunks, int stages, int issue, cox_plan *out);
/* The same plan for either operand form: precision COX_SPLIT_E4M3 (as
 * cox_plan_shape) or COX_SPLIT_E2M1 (k <= 16; issue 0 or 1 only; limb_cols
 * counts e2m1 limb columns, tmem_cols includes the 8 scale-factor columns).
 * COX_ERR_ARG for any other precision or a shape that is not compiled. */
int cox_plan_shape_prec(int precision, int k, int tile_m, int chunks, int stages, int issue, cox_plan *out);

/*
 * SNP ranking of Section 6 on a lambda path's coefficients (host arithmetic,
 * no device or handle): every SNP with a nonzero coefficient at some lambda
 * is ranked by the largest lambda at which it is nonzero, ties broken by the
 * absolute value of its coefficient at that lambda (when it joins the model),
 * then by SNP index.
 *   lambdas   : L penalties (host, finite, any order).
 *   B_host    : p x L coefficients, column-major as cox_path_fit writes them
 *               (column l at lambdas[l]); float, or double when dbl != 0.
 *   order_host: p int64 (out): the ranked SNP indices in entries 0 .. count-1.
 *   entry_host: p int64 (out): per SNP the index l of its entry lambda, or -1.
 *   count_out : the number of ranked SNPs.
 * Errors: COX_ERR_ARG for NULL pointers, p < 1, L < 1 or a non-finite lambda.
 */
int cox_rank_by_entry(int64_t p, int L, const double *lambdas, const void *B_host, int dbl,
                      int64_t *order_host, int64_t *entry_host, int64_t *count_out);

/* Turn the active-set X B product (cox_options.active_set) on or off for the
 * following calls.  Errors: COX_ERR_ARG for on outside {0, 1}. */
int cox_set_active_set(cox_h h, int on);

/* Switch a genotype handle between COX_SPLIT_E4M3 and COX_FP32_GEMV; both
 * read the same resident tiles.  Drops the per-k workspace.  Errors:
 * COX_ERR_UNSUPPORTED for COX_FP64 handles or targets. */
int cox_set_precision(cox_h h, int precision);

/*
 * Per-kernel timing with CUDA events recorded on the launching stream around
 * each kernel class of an iteration: 0 = X_c B product, 1 = X_c^T V product
 * with the fused step, 2 = risk-set scans (all their launches), 3 = other
 * (coefficient limbs, ||beta||_1).  cox_profile(h, 1) clears and starts
 * recording; cox_profile(h, 0) stops.  cox_profile_read synchronises, then
 * fills total_ms[4] and launches[4] for the recorded iterations.  Recording
 * is off inside cox_path_fit graphs.
 */
int cox_profile(cox_h h, int enable);
int cox_profile_read(cox_h h, double *total_ms, int64_t *launches);

/* Column means mu (p doubles, host) and the sorted order (n int64, host;
 * entry r = subject at rank r).  Either may be NULL. */
int cox_get_mu_order(cox_h h, double *mu_host, int64_t *order_host);

const char *cox_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* COXGB_H */
