/*
 * cox_oracle.c -- plain, slow FP64 CPU oracle for the l1-regularised Cox
 * proportional-hazards proximal-gradient iteration of Ko, Zhou, Zhou & Won,
 * "DistStat.jl" (arXiv 2010.16114), Section 5.3 and Appendix B.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA solver, and the solver never calls
 * it.
 *
 * Notation (the paper writes X in R^{m x n}; here n subjects, p predictors):
 *   y_i observed time, delta_i = 1 for an event, 0 for censoring.
 *   eta = X_c beta, X_c = X - 1 mu^T (mu = column means, or 0 when uncentred).
 *   Log partial likelihood (Section 5.3, first display; the minus sign inside
 *   the bracket is lost in the source and restored here):
 *     l(beta) = sum_i delta_i [ eta_i - log sum_{j: y_j >= y_i} exp(eta_j) ].
 *   f(beta) = -l(beta)/n,   F_lambda(beta) = f(beta) + lambda ||beta||_1.
 *   Iteration (Section 5.3, second display):
 *     w_i = exp(eta_i);  W_j = sum_{i: y_i >= y_j} w_i;
 *     pi_ij = I(y_i >= y_j) w_i / W_j;  u = P delta,
 *       i.e. u_i = w_i sum_{j: y_j <= y_i} delta_j / W_j;
 *     g = X_c^T (delta - u) / n   (= -grad f);
 *     beta <- S(beta + sigma g, sigma lambda)   (soft threshold, Section 4.2).
 *   Ties (Section 6): Breslow -- every subject with y_j >= t is at risk at t,
 *   tied events share one W.  exp is evaluated as exp(eta - max eta); the
 *   common factor cancels in w/W and in the loss.
 *
 * Compiled with -ffp-contract=off.  Built a second time with
 * -DORC_LONG_DOUBLE, which carries every intermediate in long double; the
 * two builds are compared to bound the FP64 build's own rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_LONG_DOUBLE
typedef long double real;
#define EXP expl
#define LOG logl
#define SQRT sqrtl
#define FABS fabsl
#else
typedef double real;
#define EXP exp
#define LOG log
#define SQRT sqrt
#define FABS fabs
#endif

/* ---- sorting ---------------------------------------------------------- */

static void merge_pass(int64_t n, const double *y, int64_t *a, int64_t *tmp)
{
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = (y[a[j]] < y[a[i]]) ? a[j++] : a[i++];
            while (i < mid) tmp[k++] = a[i++];
            while (j < hi) tmp[k++] = a[j++];
        }
        memcpy(a, tmp, (size_t)n * sizeof(int64_t));
    }
}

/* Stable ascending argsort of y (merge sort). Returns 0, or -2 on OOM. */
int orc_argsort(int64_t n, const double *y, int64_t *ord)
{
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp) return -2;
    for (int64_t i = 0; i < n; ++i) ord[i] = i;
    merge_pass(n, y, ord, tmp);
    free(tmp);
    return 0;
}

/* ---- risk sets -------------------------------------------------------- */

/*
 * Risk-set sums by sorting (Section 5.3: once subjects are ordered by time,
 * the sum over {j: y_j >= y_i} is a cumulative sum).  Sorted ascending, so
 * W is a reverse cumulative sum read at the first member of each tie group
 * (Breslow), and C_i = sum_{j: y_j <= y_i} delta_j / W_j is a forward
 * cumulative sum read at the last member of the tie group.
 * Outputs in subject order: W, u = P delta, and *loss = f(beta).
 * Returns 0, -1 on bad arguments, -2 on OOM, -4 on a non-finite value.
 */
int orc_risk(int64_t n, const double *y, const uint8_t *delta, const double *eta,
             double *W_out, double *u_out, double *loss)
{
    if (n <= 0) return -1;
    int64_t *ord = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    real *w = (real *)malloc((size_t)n * sizeof(real));
    real *R = (real *)malloc((size_t)n * sizeof(real));
    real *Ws = (real *)malloc((size_t)n * sizeof(real));
    real *F = (real *)malloc((size_t)n * sizeof(real));
    if (!ord || !w || !R || !Ws || !F) {
        free(ord); free(w); free(R); free(Ws); free(F);
        return -2;
    }
    orc_argsort(n, y, ord);

    real c = (real)eta[0];
    for (int64_t i = 1; i < n; ++i)
        if ((real)eta[i] > c) c = (real)eta[i];
    for (int64_t r = 0; r < n; ++r) w[r] = EXP((real)eta[ord[r]] - c);

    /* R[r] = sum_{s >= r} w[s] */
    R[n - 1] = w[n - 1];
    for (int64_t r = n - 2; r >= 0; --r) R[r] = R[r + 1] + w[r];

    /* W at each position = R at the first position of its tie group */
    for (int64_t r = 0; r < n;) {
        int64_t e = r;
        while (e + 1 < n && y[ord[e + 1]] == y[ord[r]]) ++e;
        for (int64_t s = r; s <= e; ++s) Ws[s] = R[r];
        r = e + 1;
    }

    /* F[r] = sum_{s <= r} delta_s / W_s */
    real acc = 0;
    for (int64_t r = 0; r < n; ++r) {
        if (delta[ord[r]]) acc += (real)1 / Ws[r];
        F[r] = acc;
    }

    /* C at each position = F at the last position of its tie group; u = w C */
    real lsum = 0;
    int bad = 0;
    for (int64_t r = 0; r < n;) {
        int64_t e = r;
        while (e + 1 < n && y[ord[e + 1]] == y[ord[r]]) ++e;
        for (int64_t s = r; s <= e; ++s) {
            int64_t i = ord[s];
            real u = w[s] * F[e];
            W_out[i] = (double)Ws[s];
            u_out[i] = (double)u;
            if (delta[i]) lsum += LOG(Ws[s]) - ((real)eta[i] - c);
            if (!isfinite((double)u) || !isfinite((double)Ws[s])) bad = 1;
        }
        r = e + 1;
    }
    if (loss) *loss = (double)(lsum / (real)n);

    free(ord); free(w); free(R); free(Ws); free(F);
    return bad ? -4 : 0;
}

/*
 * The same quantities from the literal definitions, O(n^2), no sorting
 * (Section 5.3 display for W_j and pi_ij; Appendix B computes P delta with
 * the same double loop).  For tiny n only.
 */
int orc_risk_bruteforce(int64_t n, const double *y, const uint8_t *delta, const double *eta,
                        double *W_out, double *u_out, double *loss)
{
    if (n <= 0) return -1;
    real *w = (real *)malloc((size_t)n * sizeof(real));
    real *W = (real *)malloc((size_t)n * sizeof(real));
    if (!w || !W) { free(w); free(W); return -2; }
    real c = (real)eta[0];
    for (int64_t i = 1; i < n; ++i)
        if ((real)eta[i] > c) c = (real)eta[i];
    for (int64_t i = 0; i < n; ++i) w[i] = EXP((real)eta[i] - c);
    for (int64_t j = 0; j < n; ++j) {
        real s = 0;
        for (int64_t i = 0; i < n; ++i)
            if (y[i] >= y[j]) s += w[i];
        W[j] = s;
    }
    real lsum = 0;
    for (int64_t i = 0; i < n; ++i) {
        real s = 0; /* (P delta)_i = sum_j pi_ij delta_j */
        for (int64_t j = 0; j < n; ++j)
            if (y[i] >= y[j] && delta[j]) s += w[i] / W[j];
        u_out[i] = (double)s;
        W_out[i] = (double)W[i];
        if (delta[i]) lsum += LOG(W[i]) - ((real)eta[i] - c);
    }
    if (loss) *loss = (double)(lsum / (real)n);
    free(w); free(W);
    return 0;
}

/* ---- products with the centred design -------------------------------- */

/* eta_i = sum_t (x_{i,t} - mu_t) beta_t over the m given columns, t in order.
 * Xcols is column-major n x m; mu may be NULL (uncentred). */
void orc_eta(int64_t n, int64_t m, const double *Xcols, const double *mu, const double *beta,
             double *eta)
{
    for (int64_t i = 0; i < n; ++i) {
        real s = 0;
        for (int64_t t = 0; t < m; ++t) {
            real xc = (real)Xcols[t * n + i] - (mu ? (real)mu[t] : (real)0);
            s += xc * (real)beta[t];
        }
        eta[i] = (double)s;
    }
}

/* g_t = (1/n) sum_i (x_{i,t} - mu_t)(delta_i - u_i): the t-th entry of
 * X_c^T (I - P) delta / n (Section 5.3, Delta), i.e. minus the gradient of f. */
void orc_grad(int64_t n, int64_t m, const double *Xcols, const double *mu, const uint8_t *delta,
              const double *u, double *g)
{
    for (int64_t t = 0; t < m; ++t) {
        real s = 0;
        for (int64_t i = 0; i < n; ++i) {
            real xc = (real)Xcols[t * n + i] - (mu ? (real)mu[t] : (real)0);
            s += xc * ((real)delta[i] - (real)u[i]);
        }
        g[t] = (double)(s / (real)n);
    }
}

/* The same two products with the columns given as bytes (genotype codes):
 * each x is converted to real exactly and the loops are those of orc_eta and
 * orc_grad, term for term, so the results are bitwise theirs.  They let a
 * caller hold a large genotype design at one byte per code. */
void orc_eta_u8(int64_t n, int64_t m, const uint8_t *Xcols, const double *mu, const double *beta,
                double *eta)
{
    for (int64_t i = 0; i < n; ++i) {
        real s = 0;
        for (int64_t t = 0; t < m; ++t) {
            real xc = (real)Xcols[t * n + i] - (mu ? (real)mu[t] : (real)0);
            s += xc * (real)beta[t];
        }
        eta[i] = (double)s;
    }
}

void orc_grad_u8(int64_t n, int64_t m, const uint8_t *Xcols, const double *mu, const uint8_t *delta,
                 const double *u, double *g)
{
    for (int64_t t = 0; t < m; ++t) {
        real s = 0;
        for (int64_t i = 0; i < n; ++i) {
            real xc = (real)Xcols[t * n + i] - (mu ? (real)mu[t] : (real)0);
            s += xc * ((real)delta[i] - (real)u[i]);
        }
        g[t] = (double)(s / (real)n);
    }
}

/* Soft threshold (Section 4.2): x - t if x > t, x + t if x < -t, else 0. */
double orc_soft_threshold(double x, double t)
{
    if (x > t) return x - t;
    if (x < -t) return x + t;
    return 0.0;
}

/* beta_out = S(beta + sigma g, sigma lambda) elementwise (Section 5.3). */
void orc_prox(int64_t m, const double *beta, const double *g, double sigma, double lam,
              double *beta_out)
{
    for (int64_t t = 0; t < m; ++t)
        beta_out[t] = orc_soft_threshold((double)((real)beta[t] + (real)sigma * (real)g[t]),
                                         (double)((real)sigma * (real)lam));
}

/* F_lambda(beta) = f(beta) + lambda ||beta||_1 on a dense column-major X. */
int orc_objective(int64_t n, int64_t p, const double *X, const double *mu, const double *y,
                  const uint8_t *delta, const double *beta, double lam, double *F)
{
    double *eta = (double *)malloc((size_t)n * sizeof(double));
    double *W = (double *)malloc((size_t)n * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    if (!eta || !W || !u) { free(eta); free(W); free(u); return -2; }
    orc_eta(n, p, X, mu, beta, eta);
    double f;
    int rc = orc_risk(n, y, delta, eta, W, u, &f);
    real l1 = 0;
    for (int64_t j = 0; j < p; ++j) l1 += FABS((real)beta[j]);
    *F = (double)((real)f + (real)lam * l1);
    free(eta); free(W); free(u);
    return rc;
}

/*
 * Proximal gradient (ISTA) from the given beta for `iters` iterations on a
 * dense column-major X (Section 5.3).  F_trace[t] = F_lambda(beta_t) for the
 * iterate entering iteration t; g_last (may be NULL) = g at the last entering
 * iterate.  beta is updated in place.
 */
int orc_ista(int64_t n, int64_t p, const double *X, const double *mu, const double *y,
             const uint8_t *delta, double sigma, double lam, int64_t iters, double *beta,
             double *F_trace, double *g_last)
{
    double *eta = (double *)malloc((size_t)n * sizeof(double));
    double *W = (double *)malloc((size_t)n * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    double *g = (double *)malloc((size_t)p * sizeof(double));
    if (!eta || !W || !u || !g) { free(eta); free(W); free(u); free(g); return -2; }
    int rc = 0;
    for (int64_t t = 0; t < iters; ++t) {
        orc_eta(n, p, X, mu, beta, eta);
        double f;
        rc = orc_risk(n, y, delta, eta, W, u, &f);
        if (rc) break;
        if (F_trace) {
            real l1 = 0;
            for (int64_t j = 0; j < p; ++j) l1 += FABS((real)beta[j]);
            F_trace[t] = (double)((real)f + (real)lam * l1);
        }
        orc_grad(n, p, X, mu, delta, u, g);
        if (g_last) memcpy(g_last, g, (size_t)p * sizeof(double));
        orc_prox(p, beta, g, sigma, lam, beta);
    }
    free(eta); free(W); free(u); free(g);
    return rc;
}

/*
 * ||X_c||_2 by power iteration on X_c^T X_c (Section 4.4, operator norms:
 * power method with a tolerance and an iteration cap).  v0 is the start
 * vector (drawn by the caller).  Stops when the Rayleigh estimate changes by
 * at most tol relative.  Returns the norm; *iters_out = iterations used.
 */
double orc_opnorm2(int64_t n, int64_t p, const double *X, const double *mu, const double *v0,
                   double tol, int64_t maxiter, int64_t *iters_out)
{
    real *v = (real *)malloc((size_t)p * sizeof(real));
    real *a = (real *)malloc((size_t)n * sizeof(real));
    real *b = (real *)malloc((size_t)p * sizeof(real));
    if (!v || !a || !b) { free(v); free(a); free(b); return -1.0; }
    real nv = 0;
    for (int64_t j = 0; j < p; ++j) { v[j] = (real)v0[j]; nv += v[j] * v[j]; }
    nv = SQRT(nv);
    for (int64_t j = 0; j < p; ++j) v[j] /= nv;
    real s_prev = 0, s = 0;
    int64_t it = 0;
    for (it = 1; it <= maxiter; ++it) {
        for (int64_t i = 0; i < n; ++i) {
            real acc = 0;
            for (int64_t j = 0; j < p; ++j)
                acc += ((real)X[j * n + i] - (mu ? (real)mu[j] : (real)0)) * v[j];
            a[i] = acc;
        }
        real nb = 0;
        for (int64_t j = 0; j < p; ++j) {
            real acc = 0;
            for (int64_t i = 0; i < n; ++i)
                acc += ((real)X[j * n + i] - (mu ? (real)mu[j] : (real)0)) * a[i];
            b[j] = acc;
            nb += acc * acc;
        }
        nb = SQRT(nb);          /* ||X_c^T X_c v|| -> sigma_max^2 */
        s = nb;
        for (int64_t j = 0; j < p; ++j) v[j] = b[j] / nb;
        if (it > 1 && FABS(s - s_prev) <= (real)tol * s) break;
        s_prev = s;
    }
    if (iters_out) *iters_out = it > maxiter ? maxiter : it;
    free(v); free(a); free(b);
    return (double)SQRT(s);
}

/* ---- Section 6: unpenalised covariates, the lambda path, SNP ranking -- */

/*
 * ISTA with an unpenalised block (Section 6: sex and the top ten principal
 * components enter the UK Biobank model without a penalty):
 *   eta   = X_c beta + Z gamma,
 *   g_X   = X_c^T (delta - u) / n,   g_Z = Z^T (delta - u) / n,
 *   beta  <- S(beta + sigma g_X, sigma lambda),   gamma <- gamma + sigma g_Z,
 *   F     = f(beta, gamma) + lambda ||beta||_1.
 * Z is column-major n x q and used as given (the partial likelihood does not
 * change when a column of Z is shifted).  q = 0 is plain ISTA.  beta and gamma
 * are updated in place; F_trace[t] (may be NULL) is F at the iterate entering
 * iteration t.
 */
int orc_ista_unpen(int64_t n, int64_t p, const double *X, const double *mu, int64_t q,
                   const double *Z, const double *y, const uint8_t *delta, double sigma,
                   double lam, int64_t iters, double *beta, double *gamma, double *F_trace)
{
    double *eta = (double *)malloc((size_t)n * sizeof(double));
    double *etz = (double *)malloc((size_t)n * sizeof(double));
    double *W = (double *)malloc((size_t)n * sizeof(double));
    double *u = (double *)malloc((size_t)n * sizeof(double));
    double *gx = (double *)malloc((size_t)(p > 0 ? p : 1) * sizeof(double));
    double *gz = (double *)malloc((size_t)(q > 0 ? q : 1) * sizeof(double));
    if (!eta || !etz || !W || !u || !gx || !gz) {
        free(eta); free(etz); free(W); free(u); free(gx); free(gz);
        return -2;
    }
    int rc = 0;
    for (int64_t t = 0; t < iters; ++t) {
        orc_eta(n, p, X, mu, beta, eta);
        if (q > 0) {
            orc_eta(n, q, Z, NULL, gamma, etz);
            for (int64_t i = 0; i < n; ++i) eta[i] = (double)((real)eta[i] + (real)etz[i]);
        }
        double f;
        rc = orc_risk(n, y, delta, eta, W, u, &f);
        if (rc) break;
        if (F_trace) {
            real l1 = 0;
            for (int64_t j = 0; j < p; ++j) l1 += FABS((real)beta[j]);
            F_trace[t] = (double)((real)f + (real)lam * l1);
        }
        orc_grad(n, p, X, mu, delta, u, gx);
        if (q > 0) orc_grad(n, q, Z, NULL, delta, u, gz);
        orc_prox(p, beta, gx, sigma, lam, beta);
        for (int64_t c = 0; c < q; ++c) gamma[c] = (double)((real)gamma[c] + (real)sigma * (real)gz[c]);
    }
    free(eta); free(etz); free(W); free(u); free(gx); free(gz);
    return rc;
}

/*
 * The lambda path of Section 6: for each lambda_l (in the order given), ISTA
 * with the unpenalised block from beta = gamma = 0, or, when warm != 0, from
 * the previous lambda's solution, run in blocks of `lag` iterations until
 * the stopping rule |F_t - F_{t-lag}| / |F_t + 1| < tol holds (F_t = F at the
 * iterate entering iteration t; tested after each block once more than lag
 * values exist; F penalised) or max_iter iterations have run.
 *   B: p x L (column l = beta at lambda_l), G: q x L, iters: L (may be NULL).
 * Returns 0, -1 for bad arguments, -2 for allocation failure, -3 if a
 * lambda's risk set degenerates (as orc_risk).
 */
int orc_path(int64_t n, int64_t p, const double *X, const double *mu, int64_t q, const double *Z,
             const double *y, const uint8_t *delta, double sigma, int64_t L, const double *lams,
             double tol, int64_t lag, int64_t max_iter, int warm, double *B, double *G,
             int64_t *iters)
{
    if (lag < 1 || max_iter < 0 || L < 0) return -1;
    double *beta = (double *)calloc((size_t)(p > 0 ? p : 1), sizeof(double));
    double *gamma = (double *)calloc((size_t)(q > 0 ? q : 1), sizeof(double));
    double *hist = (double *)malloc((size_t)(max_iter > 0 ? max_iter : 1) * sizeof(double));
    if (!beta || !gamma || !hist) { free(beta); free(gamma); free(hist); return -2; }
    int rc = 0;
    for (int64_t l = 0; l < L && rc == 0; ++l) {
        if (!warm) {
            memset(beta, 0, (size_t)(p > 0 ? p : 1) * sizeof(double));
            memset(gamma, 0, (size_t)(q > 0 ? q : 1) * sizeof(double));
        }
        int64_t t = 0;
        while (t < max_iter) {
            const int64_t steps = (max_iter - t < lag) ? (max_iter - t) : lag;
            rc = orc_ista_unpen(n, p, X, mu, q, Z, y, delta, sigma, lams[l], steps, beta, gamma, hist + t);
            if (rc) break;
            t += steps;
            if (t > lag && FABS((real)hist[t - 1] - (real)hist[t - 1 - lag]) / FABS((real)hist[t - 1] + 1) < (real)tol)
                break;
        }
        memcpy(B + l * p, beta, (size_t)p * sizeof(double));
        if (q > 0) memcpy(G + l * q, gamma, (size_t)q * sizeof(double));
        if (iters) iters[l] = t;
    }
    free(beta); free(gamma); free(hist);
    return rc;
}

/* ranking keys of one SNP: the index of its entry lambda and |beta| there */
typedef struct { int64_t j; int64_t entry; double mag; } orc_entry;

static const double *orc_rank_lams;

static int cmp_entry(const void *pa, const void *pb)
{
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    const double la = orc_rank_lams[a->entry], lb = orc_rank_lams[b->entry];
    if (la != lb) return la > lb ? -1 : 1;        /* larger entry lambda first */
    if (a->mag != b->mag) return a->mag > b->mag ? -1 : 1;  /* then larger |beta| */
    return (a->j > b->j) - (a->j < b->j);         /* then the SNP index */
}

/*
 * SNP ranking of Section 6: each SNP with a nonzero coefficient somewhere on
 * the path is ranked by the largest lambda at which its coefficient is
 * nonzero, ties broken by the absolute value of the coefficient at that
 * lambda (when it joins the model), then by SNP index.  B is p x L
 * column-major, lams the L penalties (any order).  Writes the ranked SNP
 * indices to order[0 .. count) and, per SNP, the index of its entry lambda
 * to entry[j] (-1 if never selected); returns count, or -2 on allocation
 * failure.
 */
int64_t orc_rank_by_entry(int64_t p, int64_t L, const double *lams, const double *B, int64_t *order,
                          int64_t *entry)
{
    orc_entry *e = (orc_entry *)malloc((size_t)(p > 0 ? p : 1) * sizeof(orc_entry));
    if (!e) return -2;
    int64_t count = 0;
    for (int64_t j = 0; j < p; ++j) {
        int64_t best = -1;
        for (int64_t l = 0; l < L; ++l)
            if (B[l * p + j] != 0.0 && (best < 0 || lams[l] > lams[best])) best = l;
        entry[j] = best;
        if (best >= 0) {
            e[count].j = j;
            e[count].entry = best;
            e[count].mag = fabs(B[best * p + j]);
            ++count;
        }
    }
    orc_rank_lams = lams;
    qsort(e, (size_t)count, sizeof(orc_entry), cmp_entry);
    for (int64_t c = 0; c < count; ++c) order[c] = e[c].j;
    free(e);
    return count;
}


/* ---- Section 5.1: nonnegative matrix factorization ------------------------
 * X (m x n, row-major) ~ V W with V (m x r, row-major: V[i r + c] is entry
 * (i, c), the paper's Vt transposed) and W (r x n, row-major), both
 * nonnegative; f(V, W) = ||X - V W||_F^2.  One iteration updates V from the
 * current W, then W from the new V (Section 5.1 displays and listings):
 *   multiplicative (Lee-Seung):
 *     V <- V .* (X W^T) ./ (V (W W^T) + eps)
 *     W <- W .* (V^T X) ./ ((V^T V) W + eps)
 *   alternating projected gradient:
 *     sigma = 1 / (2 ||W W^T||_F^2 + eps),  V <- max(0, V - sigma (V (W W^T) - X W^T))
 *     tau   = 1 / (2 ||V^T V||_F^2 + eps),  W <- max(0, W - tau ((V^T V) W - V^T X))
 */

/* f = ||X - V W||_F^2 by the entries of the residual. */
double orc_nmf_objective(int64_t m, int64_t n, int64_t r, const double *X, const double *V, const double *W)
{
    real f = 0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            real vw = 0;
            for (int64_t c = 0; c < r; ++c) vw += (real)V[i * r + c] * (real)W[c * n + j];
            real d = (real)X[i * n + j] - vw;
            f += d * d;
        }
    return (double)f;
}

/* iters NMF iterations in place; algo 0 multiplicative, 1 APG.  Returns 0, -1
 * on bad arguments, -2 on allocation failure. */
int orc_nmf(int64_t m, int64_t n, int64_t r, const double *X, double *V, double *W, int64_t iters, int algo,
            double eps)
{
    if (m < 1 || n < 1 || r < 1 || iters < 0 || (algo != 0 && algo != 1)) return -1;
    real *XWt = (real *)malloc((size_t)(m * r) * sizeof(real));  /* X W^T, m x r     */
    real *WWt = (real *)malloc((size_t)(r * r) * sizeof(real));  /* W W^T, r x r     */
    real *VtX = (real *)malloc((size_t)(r * n) * sizeof(real));  /* V^T X, r x n     */
    real *VtV = (real *)malloc((size_t)(r * r) * sizeof(real));  /* V^T V, r x r     */
    real *Vold = (real *)malloc((size_t)r * sizeof(real));
    real *Wold = (real *)malloc((size_t)r * sizeof(real));
    if (!XWt || !WWt || !VtX || !VtV || !Vold || !Wold) {
        free(XWt); free(WWt); free(VtX); free(VtV); free(Vold); free(Wold);
        return -2;
    }
    for (int64_t t = 0; t < iters; ++t) {
        /* V from W */
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < r; ++c) {
                real s = 0;
                for (int64_t j = 0; j < n; ++j) s += (real)X[i * n + j] * (real)W[c * n + j];
                XWt[i * r + c] = s;
            }
        real g2 = 0;
        for (int64_t c = 0; c < r; ++c)
            for (int64_t d = 0; d < r; ++d) {
                real s = 0;
                for (int64_t j = 0; j < n; ++j) s += (real)W[c * n + j] * (real)W[d * n + j];
                WWt[c * r + d] = s;
                g2 += s * s;
            }
        const real sigma = (real)1 / ((real)2 * g2 + (real)eps);
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t c = 0; c < r; ++c) Vold[c] = (real)V[i * r + c];
            for (int64_t c = 0; c < r; ++c) {
                real den = 0; /* (V W W^T)_{ic} */
                for (int64_t d = 0; d < r; ++d) den += Vold[d] * WWt[d * r + c];
                real v;
                if (algo == 0) {
                    v = Vold[c] * XWt[i * r + c] / (den + (real)eps);
                } else {
                    v = Vold[c] - sigma * (den - XWt[i * r + c]);
                    if (v < 0) v = 0;
                }
                V[i * r + c] = (double)v;
            }
        }
        /* W from the new V.  (V^T X)_cj = sum_i V_ic X_ij, added in increasing i
         * for every (c, j); the loop over j is innermost so that X is read
         * along its rows. */
        for (int64_t c = 0; c < r; ++c) {
            for (int64_t j = 0; j < n; ++j) VtX[c * n + j] = 0;
            for (int64_t i = 0; i < m; ++i) {
                const real v = (real)V[i * r + c];
                for (int64_t j = 0; j < n; ++j) VtX[c * n + j] += v * (real)X[i * n + j];
            }
        }
        real h2 = 0;
        for (int64_t c = 0; c < r; ++c)
            for (int64_t d = 0; d < r; ++d) {
                real s = 0;
                for (int64_t i = 0; i < m; ++i) s += (real)V[i * r + c] * (real)V[i * r + d];
                VtV[c * r + d] = s;
                h2 += s * s;
            }
        const real tau = (real)1 / ((real)2 * h2 + (real)eps);
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t c = 0; c < r; ++c) Wold[c] = (real)W[c * n + j];
            for (int64_t c = 0; c < r; ++c) {
                real den = 0; /* (V^T V W)_{cj} */
                for (int64_t d = 0; d < r; ++d) den += VtV[c * r + d] * Wold[d];
                real w;
                if (algo == 0) {
                    w = Wold[c] * VtX[c * n + j] / (den + (real)eps);
                } else {
                    w = Wold[c] - tau * (den - VtX[c * n + j]);
                    if (w < 0) w = 0;
                }
                W[c * n + j] = (double)w;
            }
        }
    }
    free(XWt); free(WWt); free(VtX); free(VtV); free(Vold); free(Wold);
    return 0;
}
