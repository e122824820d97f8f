// gemv.cu -- CUDA-core kernels of the Cox iteration (arXiv 2010.16114,
// Section 5.3) outside the tensor-core products:
//   * the FP64 path: eta = X beta and X^T V on a dense FP64 design, with the
//     soft-threshold step (Section 4.2) fused after the reduction;
//   * the plain FP32 baseline: one matrix-vector product per penalty on the
//     2-bit tiles (FP32 multiply-add, FP64 across 128-wide chunks) and an
//     unfused soft-threshold kernel;
//   * ||beta||_1 partial sums for the penalised objective.
#include <algorithm>

#include "internal.h"

namespace coxgb {
namespace {

__global__ void k_l1_32(const float *__restrict__ beta, int64_t p, int nb, double *__restrict__ l1p,
                        float *__restrict__ maxp)
{
    __shared__ double sh[8];
    __shared__ float shm[8];
    const int b = blockIdx.x, kk = blockIdx.y;
    // compensated FP32 sum (Knuth's TwoSum per term; the error terms summed
    // apart): ~2^-48 relative, without GB300's slow FP64 pipe in the loop
    float hi = 0.f, lo = 0.f, m = 0.f;
    for (int64_t j = static_cast<int64_t>(b) * blockDim.x + threadIdx.x; j < p; j += static_cast<int64_t>(nb) * blockDim.x) {
        const float v = fabsf(beta[kk * p + j]);
        const float t = hi + v;
        const float bv = t - hi;
        lo += (hi - (t - bv)) + (v - bv);
        hi = t;
        m = fmaxf(m, v);
    }
    double s = static_cast<double>(hi) + static_cast<double>(lo);
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = s;
        shm[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float mm = 0.f;
        for (int w = 0; w < blockDim.x / 32; ++w) {
            t += sh[w];
            mm = fmaxf(mm, shm[w]);
        }
        l1p[kk * nb + b] = t;
        if (maxp) maxp[kk * nb + b] = mm;
    }
}

__global__ void k_l1_64(const double *__restrict__ beta, int64_t p, int nb, double *__restrict__ l1p)
{
    __shared__ double sh[8];
    const int b = blockIdx.x, kk = blockIdx.y;
    double s = 0.0;
    for (int64_t j = static_cast<int64_t>(b) * blockDim.x + threadIdx.x; j < p; j += static_cast<int64_t>(nb) * blockDim.x)
        s += fabs(beta[kk * p + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < blockDim.x / 32; ++w) t += sh[w];
        l1p[kk * nb + b] = t;
    }
}

// y[row] = sum_K A[row][K] x[K] over the 2-bit tiled layout (one thread per row).
// Inside a chunk the products are summed in FP32, chunk sums in FP64.
__global__ void __launch_bounds__(128) k_gemv_tiles(const uint32_t *__restrict__ A, int64_t rows, int64_t KC,
                                                    const float *__restrict__ x, int64_t K_valid,
                                                    float *__restrict__ y)
{
    const int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const int64_t mt = row / TILE;
    const int rit = static_cast<int>(row % TILE);
    const int swap = (rit >> 2) & 1;
    double acc = 0.0;
    for (int64_t kc = 0; kc < KC; ++kc) {
        const uint32_t *blk = A + ((mt * KC + kc) * BLOCK_BYTES + rit * 32) / 4;
        const uint4 h0 = *reinterpret_cast<const uint4 *>(blk + 4 * swap);
        const uint4 h1 = *reinterpret_cast<const uint4 *>(blk + 4 * (1 - swap));
        const uint32_t w[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const int64_t kb = kc * TILE;
        float cs = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t P = w[q];
            if (P == 0) continue;
#pragma unroll
            for (int kap = 0; kap < 16; ++kap) {
                const uint32_t c = (P >> code_bit(kap)) & 3u;
                const int64_t K = kb + 16 * q + kap;
                if (c && K < K_valid) cs = fmaf(static_cast<float>(c), x[K], cs);
            }
        }
        acc += static_cast<double>(cs);
    }
    y[row] = static_cast<float>(acc);
}

// beta_col <- S(beta_col + step g, step lambda), g = (G - mu sum V) / n; or grad = -g.
__global__ void k_prox32(const float *__restrict__ G, int64_t p, const double *__restrict__ mu,
                         const double *__restrict__ sumV, double inv_n, float *beta, float *grad,
                         const double *__restrict__ lam, int col, double step, const int *active)
{
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= p) return;
    const double g = (static_cast<double>(G[j]) - mu[j] * sumV[0]) * inv_n;
    const int64_t bi = static_cast<int64_t>(col) * p + j;
    if (beta) {
        if (active && !active[col]) return;
        const double z = static_cast<double>(beta[bi]) + step * g;
        const double thr = step * lam[col];
        beta[bi] = static_cast<float>(z > thr ? z - thr : (z < -thr ? z + thr : 0.0));
    } else {
        grad[bi] = static_cast<float>(-g);
    }
}

// FP64 path: eta[kk][i] = sum_j X[i][j] beta[kk][j]  (one warp per (i, kk)).
__global__ void k_eta64(const double *__restrict__ Xr, int64_t n, int64_t p, const double *__restrict__ beta,
                        int k, double *__restrict__ eta)
{
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n * k) return;
    const int64_t i = wid % n;
    const int kk = static_cast<int>(wid / n);
    double s = 0.0;
    for (int64_t j = lane; j < p; j += 32) s += Xr[i * p + j] * beta[kk * p + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) eta[kk * n + i] = s;
}

// FP64 path: G_j = sum_i X[i][j] V[kk][i]; then the step or the gradient.
__global__ void k_xtv64(const double *__restrict__ Xc, int64_t n, int64_t p, const double *__restrict__ V, int k,
                        const double *__restrict__ mu, const double *__restrict__ sumV, double *beta, double *grad,
                        const double *__restrict__ lam, double step, const int *active)
{
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= p * k) return;
    const int64_t j = wid % p;
    const int kk = static_cast<int>(wid / p);
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) s += Xc[j * n + i] * V[kk * n + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    const double g = (s - mu[j] * sumV[kk]) / static_cast<double>(n);
    const int64_t bi = static_cast<int64_t>(kk) * p + j;
    if (beta) {
        if (active && !active[kk]) return;
        const double z = beta[bi] + step * g;
        const double thr = step * lam[kk];
        beta[bi] = z > thr ? z - thr : (z < -thr ? z + thr : 0.0);
    } else {
        grad[bi] = -g;
    }
}

__global__ void k_sub_scalar(const float *__restrict__ in, float *__restrict__ out, int64_t len, double sub)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < len) out[i] = static_cast<float>(static_cast<double>(in[i]) - sub);
}

// dots[kk] = sum_j mu_j beta_jk (one block per column, fixed order)
template <typename TB>
__global__ void k_mu_dot(const double *__restrict__ mu, const TB *__restrict__ beta, int64_t p,
                         double *__restrict__ dots)
{
    __shared__ double sh[256];
    const int kk = blockIdx.x;
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += 256) s += mu[j] * static_cast<double>(beta[kk * p + j]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) dots[kk] = sh[0];
}

__global__ void k_eta_out(const double *__restrict__ eta, const double *__restrict__ dots, int64_t n,
                          double *__restrict__ out)
{
    const int kk = blockIdx.y;
    const double d = dots[kk];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[kk * n + i] = eta[kk * n + i] - d;
}

unsigned blocks_for(int64_t n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

} // namespace

int l1_norms32(cox_handle *h, const float *beta, int k, cudaStream_t st, float *maxp)
{
    k_l1_32<<<dim3(h->l1_blocks, k), 256, 0, st>>>(beta, h->p, h->l1_blocks, h->ws.l1p, maxp);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int l1_norms64(cox_handle *h, const double *beta, int k, cudaStream_t st)
{
    k_l1_64<<<dim3(h->l1_blocks, k), 256, 0, st>>>(beta, h->p, h->l1_blocks, h->ws.l1p);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int gemv_tiles(cox_handle *h, const uint32_t *A, int64_t rows, int64_t KC, const float *x, int64_t K_valid,
               float *y, cudaStream_t st)
{
    (void)h;
    k_gemv_tiles<<<blocks_for(rows, 128), 128, 0, st>>>(A, rows, KC, x, K_valid, y);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int prox_or_grad32(cox_handle *h, const float *G, int col, float *beta, float *grad, const double *lam,
                   double step, cudaStream_t st)
{
    k_prox32<<<blocks_for(h->p, 256), 256, 0, st>>>(G, h->p, h->d_mu, h->ws.sumV, 1.0 / static_cast<double>(h->n),
                                                    beta, grad, lam, col, step, h->ws.active);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int eta64(cox_handle *h, const double *beta, int k, double *eta, cudaStream_t st)
{
    const int64_t warps = h->n * k;
    k_eta64<<<blocks_for(warps * 32, 256), 256, 0, st>>>(h->d_Xr, h->n, h->p, beta, k, eta);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int xtv64(cox_handle *h, const double *V, int k, double *beta, double *grad, const double *lam, double step,
          cudaStream_t st)
{
    const int64_t warps = h->p * k;
    k_xtv64<<<blocks_for(warps * 32, 256), 256, 0, st>>>(h->d_Xc, h->n, h->p, V, k, h->d_mu, h->ws.sumV, beta,
                                                         grad, lam, step, h->ws.active);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int center_fix_vec(cox_handle *h, const float *v_in, float *a_out, int64_t len, double sub, cudaStream_t st)
{
    (void)h;
    k_sub_scalar<<<blocks_for(len, 256), 256, 0, st>>>(v_in, a_out, len, sub);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

} // namespace coxgb

namespace coxgb {

int eta_centred_out(cox_handle *h, const void *beta, bool f64, int k, double *out, cudaStream_t st)
{
    if (f64) k_mu_dot<double><<<k, 256, 0, st>>>(h->d_mu, static_cast<const double *>(beta), h->p, h->ws.mub);
    else k_mu_dot<float><<<k, 256, 0, st>>>(h->d_mu, static_cast<const float *>(beta), h->p, h->ws.mub);
    dim3 grid(static_cast<unsigned>(std::min<int64_t>(blocks_for(h->n, 256), 1024)), k);
    k_eta_out<<<grid, 256, 0, st>>>(h->ws.eta, h->ws.mub, h->n, out);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

} // namespace coxgb
