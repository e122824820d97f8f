/*
 * nmfgb.h -- C ABI of the nonnegative matrix factorisation in libcoxgb.so.
 *
 * Method: Ko, Zhou, Zhou & Won, "DistStat.jl" (arXiv 2010.16114), Section 5.1.
 * X (m x n, nonnegative) is approximated by V W, V (m x r) and W (r x n)
 * nonnegative, minimising f(V, W) = ||X - V W||_F^2.  One iteration updates V
 * from W, then W from the new V, by either
 *   multiplicative (Lee-Seung):
 *     V <- V .* (X W^T) ./ (V W W^T + eps)
 *     W <- W .* (V^T X) ./ (V^T V W + eps)
 *   alternating projected gradient (APG):
 *     V <- max(0, V - sigma (V W W^T - X W^T)),  sigma = 1 / (2 ||W W^T||_F^2 + eps)
 *     W <- max(0, W - tau (V^T V W - V^T X)),     tau   = 1 / (2 ||V^T V||_F^2 + eps)
 * with the W step using the V just computed (Section 5.1's updates and step
 * sizes; eps is added to the denominators as in its listing).
 *
 * Arithmetic: X is held on the device in bf16 (exact for values on a grid of
 * 8 significant bits, e.g. k/256; other values are rounded to nearest, a
 * relative change of at most 2^-9).  V and W are FP32; the products X W^T and
 * V^T X run on tcgen05 tensor cores with each factor split into three bf16
 * limbs (exact for FP32 values) and FP32 accumulation; the r x r Gram matrices
 * W W^T and V^T V are summed in FP64 across blocks.
 *
 * Conventions (those of coxgb.h):
 *   - Return value: COX_OK (0) or a negative COX_ERR_* code of coxgb.h;
 *     cox_strerror() names it.  No call throws or aborts across the boundary.
 *   - Host arrays are row-major: X m x n (entry (i, j) at i n + j), V m x r,
 *     W r x n.  The caller owns them; the library owns the handle and its
 *     device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is ordered on it.  nmf_iterate is asynchronous;
 *     every other call synchronises the stream before it returns, and reports a
 *     device-side error (a wait that ran out its limit, a non-finite factor) met
 *     by earlier asynchronous work.
 *   - A handle is not thread-safe: one host thread at a time.
 */
#ifndef NMFGB_H
#define NMFGB_H

#include <stddef.h>
#include <stdint.h>

#include "coxgb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmf_handle *nmf_h;

#define NMF_MAX_RANK 80

enum {
    NMF_MULTIPLICATIVE = 0, /* Lee-Seung multiplicative updates */
    NMF_APG = 1             /* alternating projected gradient   */
};

typedef struct {
    int64_t m, n;         /* X is m x n                                        */
    int r;                /* rank                                              */
    int limb_cols;        /* N of the tensor-core products: 3 limbs x (r up to
                             a multiple of 8), rounded up to 16             */
    int stages;           /* shared-memory pipeline stages of the products     */
    int sm_count;
    int grid_xwt, grid_vtx;   /* CTAs of the X W^T and V^T X launches          */
    int64_t units_xwt, units_vtx; /* (row tile, 64-wide K chunk) units of each */
    int64_t device_bytes; /* device memory the handle holds                    */
    int64_t launches;     /* kernels launched by the handle so far             */
} nmf_info;

/* Copy X (host, m x n row-major float, nonnegative and finite) to the device
 * in bf16, in both row and column order, and create a handle for rank r
 * (1 .. NMF_MAX_RANK) on `device` (-1: the current device).  V and W start at
 * zero: set them with nmf_set_factors before iterating.
 * Synchronous.  Errors: COX_ERR_ARG (NULL pointers, m or n < 1, r out of
 * range, a negative or non-finite entry of X), COX_ERR_OOM, COX_ERR_CUDA,
 * COX_ERR_UNSUPPORTED (device is not sm_103).  On error *out is NULL. */
int nmf_setup(const float *X_host, int64_t m, int64_t n, int r, int device, nmf_h *out);

/* Free the handle and its device memory; NULL is a no-op. */
int nmf_destroy(nmf_h h);

/* Set V (m x r) and W (r x n) from host arrays (finite, nonnegative), and
 * form their bf16 limbs and Gram matrices.  Synchronous on `stream`.
 * Errors: COX_ERR_ARG for NULL pointers or a negative or non-finite entry. */
int nmf_set_factors(nmf_h h, const float *V_host, const float *W_host, void *stream);

/* Copy V (m x r) and W (r x n) to host arrays.  Synchronous on `stream`. */
int nmf_get_factors(nmf_h h, float *V_host, float *W_host, void *stream);

/* Run `iters` iterations of `algo` (NMF_MULTIPLICATIVE or NMF_APG) with the
 * given eps (>= 0; Section 5.1 uses 1e-10).  One iteration is six kernels
 * (X W^T, the V update, V^T V, V^T X, the W update, W W^T), captured once
 * per (algo, eps) as a CUDA graph and replayed.  Asynchronous on `stream`.
 * Errors: COX_ERR_ARG for iters < 0, an unknown algo or a negative or
 * non-finite eps; COX_ERR_CUDA. */
int nmf_iterate(nmf_h h, int algo, int64_t iters, double eps, void *stream);

/* f(V, W) = ||X - V W||_F^2 of the current factors, from one X W^T product
 * and the identity ||X||^2 - 2 <V, X W^T> + <V^T V, W W^T> (FP64 reductions;
 * ||X||^2 of the bf16 X).  Synchronous on `stream`. */
int nmf_objective(nmf_h h, double *f, void *stream);

/* Wait for the handle's work on `stream` and report a device-side error. */
int nmf_sync(nmf_h h, void *stream);

int nmf_get_info(nmf_h h, nmf_info *out);

/* Measurement: launch each product (X W^T, then X^T V) `reps` times on
 * `stream` between CUDA events and return the mean duration of one launch in
 * milliseconds.  The products overwrite only their partial slots (no factor
 * changes).  Synchronous.  Errors: COX_ERR_ARG for reps < 1 or NULL outputs. */
int nmf_time_products(nmf_h h, int reps, double *ms_xwt, double *ms_vtx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NMFGB_H */
