// gemv.cu -- CUDA-core kernels of the Cox iteration (arXiv 2010.16114,
// Section 5.3) outside the tensor-core products:
//   * the FP64 path: eta = X beta and X^T V on a dense FP64 design, with the
//     soft-threshold step (Section 4.2) fused after the reduction;
//   * the plain FP32 baseline: one matrix-vector product per penalty on the
//     2-bit tiles (byte tables of partial sums of x, FP32 throughout) and an
//     unfused soft-threshold kernel;
//   * the power method's matrix-vector product (one thread per row, FP32
//     multiply-add per code, FP64 across 128-wide chunks);
//   * ||beta||_1 partial sums for the penalised objective.
#include <algorithm>
#include <cmath>

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

// ---- the FP32 baseline's matrix-vector product: nibble tables of x ------------
// In the tiled layout nibble np (0, 1) of byte b of word q of half h of a row's
// 32-byte record holds the codes of the two K positions base + 4 (2 np + m)
// (m = 0, 1), base = 128 kc + 64 h + 16 q + b, two bits each.  For one K chunk
// a CTA tabulates, for each of those 64 nibble positions and each of the 16
// nibble values v, the FP32 sum
//   T[v] = sum_m code_m(v) x[base + 4 (2 np + m)],   code_m(v) = (v >> 2m) & 3,
// after which a row's dot product with the chunk is 64 table lookups and FP32
// adds.  Tables are laid out [chunk][q][b][np][h][v], so at every step the 16
// lanes of one half read one 16-entry table in banks 0-15 and the other half's
// lanes another in banks 16-31: lanes that index different entries never
// share a bank, lanes that index the same entry share the word.  A CTA keeps
// the tables of LUT_CW chunks in shared memory and streams the row tiles of its
// split through them with 16-byte coalesced loads, two threads per row (one
// per 16-byte half); every range of chunks leaves one FP32 partial per row, and
// k_gemv_reduce adds the partials with a compensated FP32 sum.
// 16 chunks (64 KB of tables) let two CTAs share an SM (registers allow two of
// 512 threads); measured at full size against 48 (one CTA per SM) and 24 with a
// shift and a mask per lookup: 0.546, 0.477 and 0.529 of the HBM copy bandwidth;
// with the byte-permute lookup below, 0.610.
constexpr int LUT_CW = 16;          // K chunks per CTA (tables: 16 x 4 KB)
constexpr int LUT_THREADS = 512;    // two threads per row, two row tiles per pass
constexpr int LUT_CHUNK = 1024;     // floats per chunk's tables
constexpr int LUT_BATCH = 8;        // chunks whose codes a thread loads before it looks up

// The 32 lookups of one chunk's 16 bytes of codes: nibble j of word q reads the
// table at byte offset 4 (C LUT_CHUNK + ((4 q + j / 2) 2 + j % 2) 32 + v), v the
// nibble, from a 256-byte aligned base.  Per word, lo and hi hold in each byte b
// the low or high nibble of byte b times 4, ORed with this half's 64-byte table
// offset (hm); a lookup's address is then one byte permute, byte 0 from lo or hi
// and bytes 1-3 from the base, with the offset an immediate of the load: a
// permute, the load and the add per nibble, plus four logic operations a word.
#define COX_LUT_NIB(Q, J)                                                                           \
    {                                                                                               \
        const uint32_t a = __byte_perm((J) & 1 ? hi : lo, cb, 0x7650u | ((J) >> 1));                 \
        float t;                                                                                    \
        asm("ld.shared.f32 %0, [%1+%2];"                                                            \
            : "=f"(t)                                                                               \
            : "r"(a), "n"(4 * (C * LUT_CHUNK + (((Q) * 4 + ((J) >> 1)) * 2 + ((J) & 1)) * 32)));    \
        acc[(J) & 3] += t;                                                                          \
    }
#define COX_LUT_WORD(Q)                                                                             \
    {                                                                                               \
        const uint32_t lo = ((ws[Q] << 2) & 0x3C3C3C3Cu) | hm;                                      \
        const uint32_t hi = ((ws[Q] >> 2) & 0x3C3C3C3Cu) | hm;                                      \
        COX_LUT_NIB(Q, 0) COX_LUT_NIB(Q, 1) COX_LUT_NIB(Q, 2) COX_LUT_NIB(Q, 3) COX_LUT_NIB(Q, 4)     \
        COX_LUT_NIB(Q, 5) COX_LUT_NIB(Q, 6) COX_LUT_NIB(Q, 7)                                       \
    }

template <int C>
__device__ __forceinline__ void lut_chunk(uint32_t cb, uint32_t hm, const uint4 &w, float (&acc)[4])
{
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    COX_LUT_WORD(0) COX_LUT_WORD(1) COX_LUT_WORD(2) COX_LUT_WORD(3)
}
#undef COX_LUT_WORD
#undef COX_LUT_NIB

__global__ void __launch_bounds__(LUT_THREADS) k_gemv_lut(const uint32_t *__restrict__ A, int64_t row_tiles,
                                                          int64_t KC, const float *__restrict__ x,
                                                          int64_t K_valid, float *__restrict__ part,
                                                          int64_t rows_pad, int n_ranges, int64_t tiles_per_split)
{
    extern __shared__ __align__(1024) float smem_lut[];
    // tables from the first 256-byte boundary (the launch adds 256 bytes)
    float *tab = reinterpret_cast<float *>(
        smem_lut + ((256u - (static_cast<uint32_t>(__cvta_generic_to_shared(smem_lut)) & 255u)) & 255u) / 4);
    const int range = static_cast<int>(blockIdx.x % n_ranges);
    const int64_t split = blockIdx.x / n_ranges;
    const int64_t kc0 = static_cast<int64_t>(range) * LUT_CW;
    const int ncw = static_cast<int>(min(static_cast<int64_t>(LUT_CW), KC - kc0));
    for (int e = threadIdx.x; e < ncw * LUT_CHUNK; e += LUT_THREADS) {
        const int c = e >> 10, q = (e >> 8) & 3, b = (e >> 6) & 3, np = (e >> 5) & 1, h = (e >> 4) & 1, v = e & 15;
        const int64_t base = (kc0 + c) * TILE + 64 * h + 16 * q + b + 8 * np;
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int64_t K = base + 4 * m;
            const float xv = K < K_valid ? x[K] : 0.f;
            acc = fmaf(static_cast<float>((v >> (2 * m)) & 3), xv, acc);
        }
        tab[e] = acc;
    }
    __syncthreads();
    const int r = (threadIdx.x & 255) >> 1, hh = threadIdx.x & 1;
    const int swp = (r >> 2) & 1;
    // byte address of the tables (256-byte aligned); this half's tables sit 64 bytes
    // in, which hm carries into byte 0 of every lookup's address
    const uint32_t tb = static_cast<uint32_t>(__cvta_generic_to_shared(tab));
    const uint32_t hm = hh ? 0x40404040u : 0u;
    const int64_t mt_begin = split * tiles_per_split;
    const int64_t mt_end = min(row_tiles, mt_begin + tiles_per_split);
    for (int64_t mt = mt_begin + (threadIdx.x >> 8); mt < mt_end; mt += 2) {
        const uint8_t *rec = reinterpret_cast<const uint8_t *>(A) + ((mt * KC + kc0) * BLOCK_BYTES + r * 32 + 16 * (hh ^ swp));
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < ncw; c0 += LUT_BATCH) {
            uint4 w[LUT_BATCH];
#pragma unroll
            for (int c = 0; c < LUT_BATCH; ++c)
                if (c0 + c < ncw) w[c] = __ldcs(reinterpret_cast<const uint4 *>(rec + static_cast<int64_t>(c0 + c) * BLOCK_BYTES));
            // tables of chunk c0 + c start 4 LUT_CHUNK (c0 + c) bytes in: a multiple of 4 KB
            const uint32_t cb = tb + 4u * LUT_CHUNK * static_cast<uint32_t>(c0);
            static_assert(LUT_BATCH == 8, "lut_chunk calls below");
            if (c0 + 0 < ncw) lut_chunk<0>(cb, hm, w[0], acc);
            if (c0 + 1 < ncw) lut_chunk<1>(cb, hm, w[1], acc);
            if (c0 + 2 < ncw) lut_chunk<2>(cb, hm, w[2], acc);
            if (c0 + 3 < ncw) lut_chunk<3>(cb, hm, w[3], acc);
            if (c0 + 4 < ncw) lut_chunk<4>(cb, hm, w[4], acc);
            if (c0 + 5 < ncw) lut_chunk<5>(cb, hm, w[5], acc);
            if (c0 + 6 < ncw) lut_chunk<6>(cb, hm, w[6], acc);
            if (c0 + 7 < ncw) lut_chunk<7>(cb, hm, w[7], acc);
        }
        float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if (hh == 0) part[static_cast<int64_t>(range) * rows_pad + mt * TILE + r] = sum;
    }
}

// y[row] = sum over ranges of part[range][row] (compensated FP32: Knuth's TwoSum
// per term, the error terms summed apart)
__global__ void k_gemv_reduce(const float *__restrict__ part, int n_ranges, int64_t rows_pad, int64_t rows,
                              float *__restrict__ y)
{
    for (int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; row < rows;
         row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < n_ranges; ++q) {
            const float v = part[static_cast<int64_t>(q) * rows_pad + row];
            const float t = hi + v;
            const float bv = t - hi;
            lo += (hi - (t - bv)) + (v - bv);
            hi = t;
        }
        y[row] = hi + lo;
    }
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

int gemv_lut_plan(int64_t rows_pad, int64_t KC, int sm_count, int *n_ranges, int64_t *tiles_per_split,
                  int *grid)
{
    const int64_t row_tiles = rows_pad / TILE;
    const int64_t ranges = (KC + LUT_CW - 1) / LUT_CW;
    // row splits: the grid nearest to whole waves of sm_count CTAs (one per SM)
    int best_s = 1;
    double best = 1e300;
    for (int sp = 1; sp <= 16; ++sp) {
        const int64_t tps = (row_tiles + sp - 1) / sp;
        const int64_t g = ranges * ((row_tiles + tps - 1) / tps);
        const double waves = static_cast<double>(g) / sm_count;
        const double loss = (std::ceil(waves) - waves) / std::ceil(waves) + 0.002 * sp;  // idle share, table builds
        if (loss < best) {
            best = loss;
            best_s = sp;
        }
    }
    *tiles_per_split = (row_tiles + best_s - 1) / best_s;
    *n_ranges = static_cast<int>(ranges);
    *grid = static_cast<int>(ranges * ((row_tiles + *tiles_per_split - 1) / *tiles_per_split));
    return COX_OK;
}

size_t gemv_lut_part_floats(int64_t rows_pad, int64_t KC) { return static_cast<size_t>((KC + LUT_CW - 1) / LUT_CW) * rows_pad; }

int gemv_lut(cox_handle *h, const uint32_t *A, int64_t rows, int64_t KC, const float *x, int64_t K_valid,
             float *part, float *y, cudaStream_t st)
{
    const size_t smem = static_cast<size_t>(LUT_CW) * LUT_CHUNK * sizeof(float) + 256;
    COX_CUDA(cudaFuncSetAttribute(k_gemv_lut, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int n_ranges = 0, grid = 0;
    int64_t tps = 0;
    gemv_lut_plan(rows, KC, h->sm_count, &n_ranges, &tps, &grid);
    k_gemv_lut<<<grid, LUT_THREADS, smem, st>>>(A, rows / TILE, KC, x, K_valid, part, rows, n_ranges, tps);
    k_gemv_reduce<<<blocks_for(rows, 256), 256, 0, st>>>(part, n_ranges, rows, rows, y);
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
