/*
 * synth.c -- seeded synthetic inputs for the l1-regularised Cox workloads.
 *
 * This module generates inputs only.  It holds none of the Cox method's
 * arithmetic (no risk sets, no scans, no gradients): the solver library and
 * the FP64 oracle both consume what it writes, and neither is linked to it.
 *
 * Every random number is a pure function of (seed, stream, a, b), built from
 * the SplitMix64 output function (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  Any entry x_ij of a
 * genotype matrix can therefore be regenerated on its own, which is what
 * lets the oracle check sampled outputs of workloads too large to hold on
 * the host.  synth_dev.cu implements the same genotype draw on the GPU; the
 * two agree bit for bit because the draw is integer-only.
 *
 * Workload shapes follow the paper's simulated Cox data (Section 5.3:
 * Gaussian covariates, exponential survival times) and its UK Biobank
 * analysis (Section 6: genotypes in {0,1,2}, integer ages with ties,
 * a few percent of subjects with events).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_GAMMA 0x9E3779B97F4A7C15ULL

enum {
    SYN_STREAM_MAF = 1,
    SYN_STREAM_X = 2,
    SYN_STREAM_CAUSAL_IDX = 3,
    SYN_STREAM_CAUSAL_EFF = 4,
    SYN_STREAM_EVENT = 5,
    SYN_STREAM_CENSOR = 6,
    SYN_STREAM_NMF_X = 7,
    SYN_STREAM_NMF_V = 8,
    SYN_STREAM_NMF_W = 9
};

uint64_t syn_mix64(uint64_t z)
{
    z += SYN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One 64-bit draw keyed by (seed, stream) at counter (a, b). */
uint64_t syn_draw(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    uint64_t key = syn_mix64(seed ^ (stream * 0xD1B54A32D192ED03ULL));
    return syn_mix64(syn_mix64(key + a) ^ b);
}

/* Uniform in [0, 1) with 53 random bits. */
static double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }
/* Uniform in (0, 1): never 0, so log() is finite. */
static double u01_open(uint64_t h) { return ((double)(h >> 11) + 0.5) * 0x1.0p-53; }

static double std_normal(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    double u1 = u01_open(syn_draw(seed, stream, a, 2 * b));
    double u2 = u01(syn_draw(seed, stream, a, 2 * b + 1));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Minor-allele frequencies MAF_j ~ U(lo, hi) and the uint32 thresholds the
 * genotype draw compares against: thr_j = floor(MAF_j * 2^32). */
void syn_maf(uint64_t seed, int64_t p, double lo, double hi, double *maf, uint32_t *thr)
{
    for (int64_t j = 0; j < p; ++j) {
        double m = lo + (hi - lo) * u01(syn_draw(seed, SYN_STREAM_MAF, (uint64_t)j, 0));
        if (maf) maf[j] = m;
        thr[j] = (uint32_t)floor(m * 4294967296.0);
    }
}

/* x_ij ~ Binomial(2, MAF_j): two Bernoulli draws from the two 32-bit halves. */
static inline uint8_t geno(uint64_t seed, uint32_t t, int64_t i, int64_t j)
{
    uint64_t h = syn_draw(seed, SYN_STREAM_X, (uint64_t)i, (uint64_t)j);
    return (uint8_t)(((uint32_t)h < t) + ((uint32_t)(h >> 32) < t));
}

/* Row-major block X[i0:i0+ni, j0:j0+nj] as uint8 codes {0,1,2}. */
void syn_genotypes(uint64_t seed, const uint32_t *thr, int64_t i0, int64_t ni,
                   int64_t j0, int64_t nj, uint8_t *out)
{
    for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < nj; ++j)
            out[i * nj + j] = geno(seed, thr[j0 + j], i0 + i, j0 + j);
}

/* Selected genotype columns as doubles, column-major n x m. */
void syn_genotype_cols(uint64_t seed, const uint32_t *thr, int64_t n,
                       const int64_t *cols, int64_t m, double *out)
{
    for (int64_t c = 0; c < m; ++c) {
        int64_t j = cols[c];
        for (int64_t i = 0; i < n; ++i)
            out[c * n + i] = (double)geno(seed, thr[j], i, j);
    }
}

/* Row-major packed genotypes: ceil(p/4) bytes per row, SNP j in bits
 * 2*(j%4)..2*(j%4)+1 of byte j/4, unused tail bits zero. Rows i0..i0+ni. */
/* Columns cols[0..m) of X as bytes, column-major: out[c * n + i] = x_{i, cols[c]}. */
void syn_genotype_cols_u8(uint64_t seed, const uint32_t *thr, int64_t n,
                          const int64_t *cols, int64_t m, uint8_t *out)
{
    for (int64_t c = 0; c < m; ++c) {
        int64_t j = cols[c];
        for (int64_t i = 0; i < n; ++i)
            out[c * n + i] = geno(seed, thr[j], i, j);
    }
}

void syn_genotypes_packed(uint64_t seed, const uint32_t *thr, int64_t p,
                          int64_t i0, int64_t ni, uint8_t *out)
{
    int64_t rb = (p + 3) / 4;
    for (int64_t i = 0; i < ni; ++i) {
        uint8_t *row = out + i * rb;
        memset(row, 0, (size_t)rb);
        for (int64_t j = 0; j < p; ++j)
            row[j >> 2] |= (uint8_t)(geno(seed, thr[j], i0 + i, j) << (2 * (j & 3)));
    }
}

/* iid N(0,1) covariates, row-major block X[i0:i0+ni, j0:j0+nj]. */
void syn_normals(uint64_t seed, int64_t i0, int64_t ni, int64_t j0, int64_t nj, double *out)
{
    for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < nj; ++j)
            out[i * nj + j] = std_normal(seed, SYN_STREAM_X, (uint64_t)(i0 + i), (uint64_t)(j0 + j));
}

/* A seeded standard-normal vector on an arbitrary stream (start vectors,
 * perturbations, coordinate picks). */
void syn_normal_vec(uint64_t seed, uint64_t stream, int64_t m, double *out)
{
    for (int64_t t = 0; t < m; ++t)
        out[t] = std_normal(seed, stream, (uint64_t)t, 0);
}

/* A seeded uniform [0,1) vector on an arbitrary stream. */
void syn_uniform_vec(uint64_t seed, uint64_t stream, int64_t m, double *out)
{
    for (int64_t t = 0; t < m; ++t)
        out[t] = u01(syn_draw(seed, stream, (uint64_t)t, 0));
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* nc distinct causal indices (partial Fisher-Yates, then sorted ascending)
 * and their effects ~ N(0, sd^2). */
int syn_causal(uint64_t seed, int64_t p, int64_t nc, double sd, int64_t *idx, double *eff)
{
    if (nc > p || nc < 0) return -1;
    int64_t *perm = (int64_t *)malloc((size_t)p * sizeof(int64_t));
    if (!perm) return -2;
    for (int64_t j = 0; j < p; ++j) perm[j] = j;
    for (int64_t t = 0; t < nc; ++t) {
        uint64_t h = syn_draw(seed, SYN_STREAM_CAUSAL_IDX, (uint64_t)t, 0);
        int64_t r = t + (int64_t)(h % (uint64_t)(p - t));
        int64_t tmp = perm[t]; perm[t] = perm[r]; perm[r] = tmp;
    }
    memcpy(idx, perm, (size_t)nc * sizeof(int64_t));
    free(perm);
    qsort(idx, (size_t)nc, sizeof(int64_t), cmp_i64);
    for (int64_t t = 0; t < nc; ++t)
        eff[t] = sd * std_normal(seed, SYN_STREAM_CAUSAL_EFF, (uint64_t)t, 0);
    return 0;
}

static int cmp_f64(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* The value q such that exactly round(frac*n) of the q_i lie below it
 * (midpoint between neighbouring order statistics). */
static double split_quantile(double *q, int64_t n, double frac)
{
    qsort(q, (size_t)n, sizeof(double), cmp_f64);
    int64_t m = (int64_t)llround(frac * (double)n);
    if (m <= 0) return q[0] * 0.5;
    if (m >= n) return q[n - 1] * 2.0;
    return 0.5 * (q[m - 1] + q[m]);
}

/* Continuous times (paper's simulated data): T_i ~ Exp(rate exp(eta_i)),
 * C_i ~ Exp(rate r) with r set so a fraction cens_frac is censored;
 * y = min(T, C), delta = [T <= C]. */
int syn_times_exp(uint64_t seed, int64_t n, const double *eta, double cens_frac,
                  double *y, uint8_t *delta, double *rate_out)
{
    double *T = (double *)malloc((size_t)n * sizeof(double));
    double *E2 = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    if (!T || !E2 || !q) { free(T); free(E2); free(q); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        double e1 = -log(u01_open(syn_draw(seed, SYN_STREAM_EVENT, (uint64_t)i, 0)));
        E2[i] = -log(u01_open(syn_draw(seed, SYN_STREAM_CENSOR, (uint64_t)i, 0)));
        T[i] = e1 * exp(-eta[i]);
        q[i] = E2[i] / T[i]; /* censored iff r > q_i */
    }
    double r = split_quantile(q, n, cens_frac);
    for (int64_t i = 0; i < n; ++i) {
        double C = E2[i] / r;
        delta[i] = (uint8_t)(T[i] <= C);
        y[i] = T[i] <= C ? T[i] : C;
    }
    if (rate_out) *rate_out = r;
    free(T); free(E2); free(q);
    return 0;
}

/* Integer-day times (UK Biobank-like): T_i = E_i / (h0 exp(eta_i)), E ~ Exp(1);
 * C_i ~ U(1, dmax); h0 set so a fraction event_frac has T <= C;
 * y = clamp(ceil(min(T, C)), 1, dmax) -> ties; delta = [T <= C]. */
int syn_times_days(uint64_t seed, int64_t n, const double *eta, double event_frac,
                   int64_t dmax, double *y, uint8_t *delta, double *h0_out)
{
    double *E = (double *)malloc((size_t)n * sizeof(double));
    double *C = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    if (!E || !C || !q) { free(E); free(C); free(q); return -2; }
    for (int64_t i = 0; i < n; ++i) {
        E[i] = -log(u01_open(syn_draw(seed, SYN_STREAM_EVENT, (uint64_t)i, 0)));
        C[i] = 1.0 + (double)(dmax - 1) * u01(syn_draw(seed, SYN_STREAM_CENSOR, (uint64_t)i, 0));
        q[i] = E[i] / (C[i] * exp(eta[i])); /* event iff h0 >= q_i */
    }
    double h0 = split_quantile(q, n, event_frac);
    for (int64_t i = 0; i < n; ++i) {
        double T = E[i] / (h0 * exp(eta[i]));
        double t = T <= C[i] ? T : C[i];
        double d = ceil(t);
        if (d < 1.0) d = 1.0;
        if (d > (double)dmax) d = (double)dmax;
        y[i] = d;
        delta[i] = (uint8_t)(T <= C[i]);
    }
    if (h0_out) *h0_out = h0;
    free(E); free(C); free(q);
    return 0;
}

/* NMF inputs (Section 5.1 experiments: X, V and W drawn uniform on [0, 1)).
 * X entries are drawn on the grid k / 256, k = 0..255, so that they are exact
 * in bf16 (8 significant bits); rows [i0, i0 + ni) of an m x n row-major X. */
void syn_nmf_x(uint64_t seed, int64_t i0, int64_t ni, int64_t n, float *out)
{
    for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < n; ++j) {
            uint64_t h = syn_draw(seed, SYN_STREAM_NMF_X, (uint64_t)(i0 + i), (uint64_t)j);
            out[i * n + j] = (float)(h >> 56) * 0x1.0p-8f;
        }
}

/* count uniform [0, 1) values rounded to FP32; which = 0 for V, 1 for W. */
void syn_nmf_factor(uint64_t seed, int which, int64_t count, float *out)
{
    const uint64_t st = which ? SYN_STREAM_NMF_W : SYN_STREAM_NMF_V;
    for (int64_t t = 0; t < count; ++t) {
        float f = (float)u01(syn_draw(seed, st, (uint64_t)t, 0));
        out[t] = f < 1.0f ? f : 0x1.fffffep-1f;
    }
}
