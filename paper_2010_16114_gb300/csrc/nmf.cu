// nmf.cu -- nonnegative matrix factorisation X ~ V W (arXiv 2010.16114,
// Section 5.1): the multiplicative (Lee-Seung) and the alternating projected
// gradient (APG) iterations on one GB300.
//
// An iteration is six kernels:
//   k_nmf_gemm    P = X W^T   (m x r)   tcgen05 kind::f16, A = X row-major
//   k_nmf_update  V from P and W W^T; limbs of V; per-block partials of V^T V
//   k_nmf_gram    V^T V (FP64) from the partials
//   k_nmf_gemm    Q = X^T V   (n x r)   A = X column-major
//   k_nmf_update  W from Q and V^T V; limbs of W; partials of W W^T
//   k_nmf_gram    W W^T
// Both updates have one form.  With F a factor held r x R (V^T, or W), G the
// Gram matrix of the other factor and P the product of X with it,
//   (V W W^T)_ic = sum_d G_cd F_di  and  (V^T V W)_cj = sum_d G_cd F_dj
// (G symmetric), so
//   multiplicative: F_ci <- F_ci P_ci / (sum_d G_cd F_di + eps)
//   APG:            F_ci <- max(0, F_ci - s (sum_d G_cd F_di - P_ci)),
//                   s = 1 / (2 ||G||_F^2 + eps).
//
// Products (nmf_gemm.cuh).  X is stored in bf16 twice (row-major for X W^T,
// column-major for X^T V), so both are K-major A operands of the tensor-core
// product; the factor enters as three bf16 limbs per value (exact for FP32),
// rows l rp + c of an N = 3 rp (rounded up to 16) panel, rp = r rounded up to 8
// so that every limb's columns start 8-aligned in TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "../../include/nmfgb.h"
#include "nmf_gemm.cuh"

struct nmf_handle;

namespace coxgb {
namespace {

struct UpdArgs {
    int r, rp, mode, algo;   // mode 1: update from the product; 0: limbs and Gram partials of F only
    int64_t R;               // factor columns (m for V, n for W)
    float *F;                // r x R, row c at c R
    __nv_bfloat16 *limb;     // NP x ldl: row l rp + c holds limb l of F row c
    int64_t ldl;
    const float *part;       // product partials of this side
    int SL, KC;
    int64_t L;
    const float *Gin;        // r x r Gram of the other factor, FP32
    const double *Gin64;     // and FP64 (its squared Frobenius norm sets the APG step)
    double eps;
    float *gpart;            // Gram partials of the new F: [pair][block], pairs c <= d
    int nblk;                // blocks of this launch
    int *err;
};

// Split f into three bf16 limbs, f = h0 + h1 + h2 (exact for an FP32 f).
__device__ __forceinline__ void split_bf16(float f, __nv_bfloat16 &h0, __nv_bfloat16 &h1, __nv_bfloat16 &h2)
{
    h0 = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
}

// Pair p of the upper triangle (c <= d, row by row) of an r x r matrix.
__device__ __forceinline__ void pair_cd(int p, int r, int &c, int &d)
{
    c = 0;
    while (p >= r - c) {
        p -= r - c;
        ++c;
    }
    d = c + p;
}

constexpr int UPD_ROWS = 32;    // factor columns per block (one per lane)
constexpr int UPD_MAXW = 32;    // warps per block: min(r, 32); warp y takes rank rows c = y, y + W, ...

int upd_warps(int r) { return r < UPD_MAXW ? r : UPD_MAXW; }

// A quarter row tile of a factor per block: lane x of every warp owns column
// i = 128 g + 32 q + x of F (block 4 g + q); warp y of W = min(r, 32) takes
// the rank rows c = y, y + W, ...  Shared memory: G (r x r), the old and the
// new F and the summed product partials ([c][33] each).  The block also
// leaves its partial of the new F's Gram matrix over its 32 columns (FP32),
// one per pair c <= d.  Dot products run in four interleaved FP32 sums (a
// fixed order) to shorten the dependent chains.
__global__ void __launch_bounds__(UPD_ROWS * UPD_MAXW) k_nmf_update(const UpdArgs A)
{
    extern __shared__ float sh[];
    __shared__ double fro_w[UPD_MAXW];
    __shared__ float step_s;
    constexpr int LD = UPD_ROWS + 1;
    const int r = A.r, t = threadIdx.x, x = t % UPD_ROWS, y = t / UPD_ROWS;
    const int W = blockDim.x / UPD_ROWS, nthr = blockDim.x;
    pdl_trigger();
    pdl_wait();  // the product ahead (and everything before it) is complete
    float *Gs = sh;
    float *Fo = Gs + r * r;
    float *Fn = Fo + r * LD;
    float *Pc = Fn + r * LD;
    const int64_t g = blockIdx.x / (NT / UPD_ROWS);
    const int rit = static_cast<int>(blockIdx.x % (NT / UPD_ROWS)) * UPD_ROWS + x;  // row in the tile
    const int64_t i = g * NT + rit;
    const bool valid = i < A.R;
    const bool apg = A.mode && A.algo == NMF_APG;
    if (A.mode) {
        double f = 0.0;  // ||G||_F^2 (APG step): every thread a few entries, then a fixed-order reduction
        for (int e = t; e < r * r; e += nthr) {
            Gs[e] = A.Gin[e];
            if (apg) {
                const double gv = A.Gin64[e];
                f += gv * gv;
            }
        }
        if (apg) {
            for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
            if (x == 0) fro_w[y] = f;
        }
        const int64_t first = (g * A.KC) / A.L, last = (g * A.KC + A.KC - 1) / A.L;
        const int ns = static_cast<int>(last - first + 1);
        const float *pp = A.part + (g * A.SL * r) * NT + rit;
        for (int c = y; c < r; c += W) {
            double acc = 0.0;
#pragma unroll 4
            for (int sl = 0; sl < ns; ++sl) acc += static_cast<double>(pp[(static_cast<int64_t>(sl) * r + c) * NT]);
            Pc[c * LD + x] = static_cast<float>(acc);
        }
    }
    for (int c = y; c < r; c += W) Fo[c * LD + x] = valid ? A.F[c * A.R + i] : 0.f;
    __syncthreads();
    if (apg && t == 0) {  // the step, formed once per block (FP64 division is slow on this part)
        double f2 = 0.0;
        for (int w = 0; w < W; ++w) f2 += fro_w[w];
        step_s = static_cast<float>(1.0 / (2.0 * f2 + A.eps));
    }
    if (apg) __syncthreads();
    const float s = apg ? step_s : 0.f;
    const float eps = static_cast<float>(A.eps);
    bool bad = false;
    for (int c = y; c < r; c += W) {
        const float old = Fo[c * LD + x];
        float v = old;
        if (A.mode && valid) {
            const float pc = Pc[c * LD + x];
            float d4[4] = {0.f, 0.f, 0.f, 0.f};
            const float *gr = Gs + c * r;
            int d = 0;
            for (; d + 4 <= r; d += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d4[q] = fmaf(gr[d + q], Fo[(d + q) * LD + x], d4[q]);
            }
            for (; d < r; ++d) d4[0] = fmaf(gr[d], Fo[d * LD + x], d4[0]);
            const float den = (d4[0] + d4[1]) + (d4[2] + d4[3]);
            v = A.algo == NMF_MULTIPLICATIVE ? old * pc / (den + eps) : fmaxf(0.f, old - s * (den - pc));
            bad |= !isfinite(v);
            A.F[c * A.R + i] = v;
        }
        if (!valid) v = 0.f;
        Fn[c * LD + x] = v;
        if (valid) {
            __nv_bfloat16 h0, h1, h2;
            split_bf16(v, h0, h1, h2);
            A.limb[static_cast<int64_t>(c) * A.ldl + i] = h0;
            A.limb[static_cast<int64_t>(A.rp + c) * A.ldl + i] = h1;
            A.limb[static_cast<int64_t>(2 * A.rp + c) * A.ldl + i] = h2;
        }
    }
    if (bad) atomicOr(A.err, NMF_ERR_NONFINITE);
    __syncthreads();
    // Gram partial over the block's 32 columns (zero for columns past R)
    const int npair = r * (r + 1) / 2;
    for (int p = t; p < npair; p += nthr) {
        int c, d;
        pair_cd(p, r, c, d);
        const float *fc = Fn + c * LD, *fd = Fn + d * LD;
        float a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < UPD_ROWS; j += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a4[q] = fmaf(fc[j + q], fd[j + q], a4[q]);
        }
        A.gpart[static_cast<int64_t>(p) * A.nblk + blockIdx.x] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    }
}

struct GramArgs {
    int r, nblk;
    const float *gpart;      // [pair][block]
    double *G64;             // r x r
    float *G32;
};

// G = F F^T from the update blocks' partials: one warp per pair c <= d, lane
// sums of the blocks b = lane, lane + 32, ... in FP64 and a shuffle tree (a
// fixed order: deterministic).
__global__ void __launch_bounds__(256) k_nmf_gram(const GramArgs A)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int r = A.r;
    pdl_trigger();
    pdl_wait();  // the update ahead is complete
    if (p >= r * (r + 1) / 2) return;
    const float *src = A.gpart + static_cast<int64_t>(p) * A.nblk;
    double v4[4] = {0.0, 0.0, 0.0, 0.0};  // blocks lane + 32 (4 j + q)
    int b = lane;
    for (; b + 96 < A.nblk; b += 128) {
        float u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q] = src[b + 32 * q];
#pragma unroll
        for (int q = 0; q < 4; ++q) v4[q] += static_cast<double>(u[q]);
    }
    for (; b < A.nblk; b += 32) v4[0] += static_cast<double>(src[b]);
    double v = (v4[0] + v4[1]) + (v4[2] + v4[3]);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) {
        int c, d;
        pair_cd(p, r, c, d);
        A.G64[c * r + d] = v;
        A.G64[d * r + c] = v;
        A.G32[c * r + d] = static_cast<float>(v);
        A.G32[d * r + c] = static_cast<float>(v);
    }
}

struct FitArgs {
    int r;
    int64_t R;               // m
    const float *F;          // V^T, r x m
    const float *part;
    int SL, KC;
    int64_t L;
    double *opart;           // per block
    int *counter;
    const double *GV, *GW;
    double xx;
    double *out;
};

// Block sum of one FP64 value per thread in a fixed order: warp shuffles, then
// the warps' sums in warp order by thread 0 (valid there only).
__device__ __forceinline__ double block_sum(double v, double *wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) wsum[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < nw; ++k) s += wsum[k];
    return s;
}

// <V, X W^T> over a quarter row tile per block (lane x: column i of V^T, warp
// y: rank rows c = y, y + W, ...) in FP64, then (last block, all threads) the
// objective by the identity ||X - V W||^2 = ||X||^2 - 2 <V, X W^T> +
// <V^T V, W W^T>.  Fixed orders throughout.
__global__ void __launch_bounds__(UPD_ROWS * UPD_MAXW) k_nmf_fit(const FitArgs A)
{
    __shared__ double wsum[UPD_MAXW];
    __shared__ int is_last;
    const int r = A.r, t = threadIdx.x, x = t % UPD_ROWS, y = t / UPD_ROWS;
    const int W = blockDim.x / UPD_ROWS, nthr = blockDim.x;
    const int64_t g = blockIdx.x / (NT / UPD_ROWS);
    const int rit = static_cast<int>(blockIdx.x % (NT / UPD_ROWS)) * UPD_ROWS + x;
    const int64_t i = g * NT + rit;
    double s = 0.0;
    if (i < A.R) {
        const int64_t first = (g * A.KC) / A.L, last = (g * A.KC + A.KC - 1) / A.L;
        const int ns = static_cast<int>(last - first + 1);
        const float *pp = A.part + (g * A.SL * r) * NT + rit;
        for (int c = y; c < r; c += W) {
            double acc = 0.0;
#pragma unroll 4
            for (int sl = 0; sl < ns; ++sl) acc += static_cast<double>(pp[(static_cast<int64_t>(sl) * r + c) * NT]);
            s += static_cast<double>(A.F[c * A.R + i]) * acc;
        }
    }
    const double bs = block_sum(s, wsum);
    if (t == 0) A.opart[blockIdx.x] = bs;
    __threadfence();
    __syncthreads();
    if (t == 0) is_last = atomicAdd(A.counter, 1) == static_cast<int>(gridDim.x) - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double v = 0.0, tr = 0.0;
    for (int b2 = t; b2 < static_cast<int>(gridDim.x); b2 += nthr) v += __ldcg(A.opart + b2);
    for (int e = t; e < r * r; e += nthr) tr += A.GV[e] * A.GW[e];
    const double vp = block_sum(v, wsum);
    __syncthreads();
    const double trs = block_sum(tr, wsum);
    if (t == 0) {
        *A.out = A.xx - 2.0 * vp + trs;
        *A.counter = 0;
    }
}

// X rows [r0, r0 + nr) (FP32, nr x n) -> bf16 in both orders; 32 x 32 tiles
// through shared memory; squares of the bf16 values summed per block (FP64).
__global__ void k_nmf_pack(const float *__restrict__ x, int64_t r0, int64_t nr, int64_t n, __nv_bfloat16 *Xr,
                           int64_t ldr, __nv_bfloat16 *Xc, int64_t ldc, double *sq, int *err)
{
    __shared__ float tile[32][33];
    __shared__ double red[256];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32, rr0 = static_cast<int64_t>(blockIdx.y) * 32;
    double s = 0.0;
    bool bad = false;
    for (int k = 0; k < 32; k += 8) {
        const int64_t rr = rr0 + ty + k, c = c0 + tx;
        float v = 0.f;
        if (rr < nr && c < n) {
            const float f = x[rr * n + c];
            bad |= !(f >= 0.f) || !isfinite(f);
            const __nv_bfloat16 b = __float2bfloat16_rn(f);
            Xr[(r0 + rr) * ldr + c] = b;
            v = __bfloat162float(b);
            s += static_cast<double>(v) * static_cast<double>(v);
        }
        tile[ty + k][tx] = v;
    }
    __syncthreads();
    for (int k = 0; k < 32; k += 8) {
        const int64_t c = c0 + ty + k, rr = rr0 + tx;
        if (rr < nr && c < n) Xc[c * ldc + r0 + rr] = __float2bfloat16_rn(tile[tx][ty + k]);
    }
    if (bad) atomicOr(err, NMF_ERR_NEGATIVE);
    const int tid = ty * 32 + tx;
    red[tid] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) sq[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn nmf_encoder()
{
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

// 2-D bf16 map: inner extent `inner` (K), `outer` rows, row pitch ld elements
// (a multiple of 8: 16-byte strides), box 64 x box_rows, 128-byte swizzle.
bool encode_bf16(CUtensorMap *m, const void *base, int64_t inner, int64_t outer, int64_t ld, int box_rows)
{
    EncodeFn enc = nmf_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(NK), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

} // namespace

// One product: A (rows x K, bf16, K-major) times the limb panel B (NP x K).
struct NmfSide {
    CUtensorMap tmA, tmB;
    GemmArgs g;
    int grid = 0;
    int MT = 0;         // row tiles
    int64_t rows = 0;   // m for X W^T, n for X^T V
    size_t smem = 0;
};

} // namespace coxgb

using coxgb::NmfSide;

struct nmf_handle {
    int dev = 0, sms = 0;
    int64_t m = 0, n = 0;
    int r = 0, rp = 0, NP = 0;
    cudaStream_t cap = nullptr;   // capture stream
    __nv_bfloat16 *Xr = nullptr, *Xc = nullptr, *Vl = nullptr, *Wl = nullptr;
    int64_t ldr = 0, ldc = 0, ldm = 0, ldn = 0;
    float *Vt = nullptr, *W = nullptr;
    float *part1 = nullptr, *part2 = nullptr;
    NmfSide s1, s2;               // X W^T, X^T V
    float *GV32 = nullptr, *GW32 = nullptr;
    float *gpart = nullptr;    // Gram partials [pair][update block]
    double *GV64 = nullptr, *GW64 = nullptr, *opart = nullptr, *fobj = nullptr;
    int *counters = nullptr, *err = nullptr;
    double xx = 0.0;
    long long wait_cycles = 0;
    int64_t device_bytes = 0, launches = 0;
    cudaGraphExec_t exec = nullptr;
    int g_algo = -1;
    double g_eps = -1.0;
    std::vector<void *> allocs;
};

namespace coxgb {
namespace {

int nmf_alloc(nmf_handle *h, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? COX_ERR_OOM : COX_ERR_CUDA;
    }
    h->allocs.push_back(*p);
    h->device_bytes += static_cast<int64_t>(bytes);
    return COX_OK;
}

int plan_side(nmf_handle *h, NmfSide &sd, const __nv_bfloat16 *A, int64_t rows, int64_t K, int64_t ldA,
              const __nv_bfloat16 *B, int64_t ldB, float **part)
{
    sd.rows = rows;
    sd.MT = static_cast<int>((rows + NT - 1) / NT);
    GemmArgs &g = sd.g;
    g.KC = static_cast<int>((K + NK - 1) / NK);
    g.r = h->r;
    g.rp = h->rp;
    g.NP = h->NP;
    g.stage = A_BYTES + h->NP * 128;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev) != cudaSuccess) return COX_ERR_CUDA;
    g.S = std::min(MAX_STAGES, (optin - 2048 - h->r * NT * static_cast<int>(sizeof(float))) / g.stage);
    if (g.S < 2) return COX_ERR_UNSUPPORTED;
    const int need = h->NP + 3 * h->rp;  // second accumulator: its last limb's columns end before NP + 3 rp
    int tc = 32;
    while (tc < need) tc *= 2;
    if (tc > 512) return COX_ERR_ARG;
    g.tcols = tc;
    g.idesc = idesc_bf16_f32(NT, h->NP);
    g.units = static_cast<int64_t>(sd.MT) * g.KC;
    g.L = (g.units + h->sms - 1) / h->sms;
    sd.grid = static_cast<int>((g.units + g.L - 1) / g.L);
    int SL = 1;
    for (int64_t t = 0; t < sd.MT; ++t) {
        const int64_t f = t * g.KC / g.L, l = (t * g.KC + g.KC - 1) / g.L;
        SL = std::max<int>(SL, static_cast<int>(l - f + 1));
    }
    g.SL = SL;
    g.wait_limit = h->wait_cycles;
    g.err = h->err;
    COX_TRY(nmf_alloc(h, reinterpret_cast<void **>(part),
                      static_cast<size_t>(sd.MT) * SL * h->r * NT * sizeof(float)));
    g.part = *part;
    sd.smem = 1024 + static_cast<size_t>(g.S) * g.stage + 256 + static_cast<size_t>(h->r) * NT * sizeof(float);
    if (!encode_bf16(&sd.tmA, A, K, rows, ldA, NT)) return COX_ERR_CUDA;
    if (!encode_bf16(&sd.tmB, B, K, h->NP, ldB, h->NP)) return COX_ERR_CUDA;
    return COX_OK;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the one ahead of it in the stream finishes (each NMF kernel waits for
// its predecessor with pdl_wait before touching global memory).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

int launch_gemm(nmf_handle *h, const NmfSide &sd, cudaStream_t st)
{
    ++h->launches;
    return launch_pdl(k_nmf_gemm, sd.grid, GEMM_THREADS, sd.smem, st, sd.tmA, sd.tmB, sd.g) == cudaSuccess
               ? COX_OK
               : COX_ERR_CUDA;
}

size_t upd_smem(int r) { return static_cast<size_t>(r * r + 3 * r * (UPD_ROWS + 1)) * sizeof(float); }

int upd_blocks(int64_t R) { return static_cast<int>((R + NT - 1) / NT * (NT / UPD_ROWS)); }

// side 0: V from X W^T (rows m); side 1: W from X^T V (rows n); then the Gram
// matrix of the new factor from the blocks' partials
int launch_update(nmf_handle *h, int side, int mode, int algo, double eps, cudaStream_t st)
{
    UpdArgs a;
    const NmfSide &sd = side == 0 ? h->s1 : h->s2;
    a.r = h->r;
    a.rp = h->rp;
    a.mode = mode;
    a.algo = algo;
    a.R = side == 0 ? h->m : h->n;
    a.F = side == 0 ? h->Vt : h->W;
    a.limb = side == 0 ? h->Vl : h->Wl;
    a.ldl = side == 0 ? h->ldm : h->ldn;
    a.part = sd.g.part;
    a.SL = sd.g.SL;
    a.KC = sd.g.KC;
    a.L = sd.g.L;
    a.Gin = side == 0 ? h->GW32 : h->GV32;
    a.Gin64 = side == 0 ? h->GW64 : h->GV64;
    a.eps = eps;
    a.gpart = h->gpart;
    a.nblk = upd_blocks(a.R);
    a.err = h->err;
    ++h->launches;
    if (launch_pdl(k_nmf_update, a.nblk, UPD_ROWS * upd_warps(h->r), upd_smem(h->r), st, a) != cudaSuccess)
        return COX_ERR_CUDA;
    GramArgs gm;
    gm.r = h->r;
    gm.nblk = a.nblk;
    gm.gpart = h->gpart;
    gm.G64 = side == 0 ? h->GV64 : h->GW64;
    gm.G32 = side == 0 ? h->GV32 : h->GW32;
    const int npair = h->r * (h->r + 1) / 2;
    ++h->launches;
    return launch_pdl(k_nmf_gram, (npair + 7) / 8, 256, 0, st, gm) == cudaSuccess ? COX_OK : COX_ERR_CUDA;
}

int check_err(nmf_handle *h, cudaStream_t st)
{
    int e = 0;
    COX_CUDA(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    COX_CUDA(cudaStreamSynchronize(st));
    if (e) {
        COX_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), st));
        COX_CUDA(cudaStreamSynchronize(st));
    }
    if (e & NMF_ERR_TIMEOUT) return COX_ERR_TIMEOUT;
    if (e & NMF_ERR_NONFINITE) return COX_ERR_NONFINITE;
    if (e & NMF_ERR_NEGATIVE) return COX_ERR_ARG;
    return COX_OK;
}

void release(nmf_handle *h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (void *p : h->allocs) cudaFree(p);
    delete h;
}

int setup_impl(const float *X, int64_t m, int64_t n, int r, int device, nmf_handle **out)
{
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return COX_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return COX_ERR_UNSUPPORTED;
    }
    if (prop.major != 10 || prop.minor != 3) return COX_ERR_UNSUPPORTED;
    DevGuard guard(dev);
    nmf_handle *h = new nmf_handle();
    int rc = COX_OK;
    do {
        h->dev = dev;
        h->sms = prop.multiProcessorCount;
        h->m = m;
        h->n = n;
        h->r = r;
        h->rp = static_cast<int>(rup(r, 8));
        h->NP = static_cast<int>(rup(3 * h->rp, 16));
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
            cudaGetLastError();
            khz = 2100000;
        }
        h->wait_cycles = static_cast<long long>(2.0 * static_cast<double>(khz) * 1000.0);
        if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
        cudaStream_t st = h->cap;
        h->ldr = rup(n, 8);
        h->ldc = rup(m, 8);
        h->ldm = rup(m, 8);
        h->ldn = rup(n, 8);
        auto A = [&](void **p, size_t b) { return nmf_alloc(h, p, b); };
        if ((rc = A(reinterpret_cast<void **>(&h->err), sizeof(int))) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->counters), 4 * sizeof(int))) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->Xr), static_cast<size_t>(m * h->ldr) * 2)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->Xc), static_cast<size_t>(n * h->ldc) * 2)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->Vl), static_cast<size_t>(h->NP * h->ldm) * 2)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->Wl), static_cast<size_t>(h->NP * h->ldn) * 2)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->Vt), static_cast<size_t>(r * m) * 4)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->W), static_cast<size_t>(r * n) * 4)) != COX_OK) break;
        for (float **p : {&h->GV32, &h->GW32})
            if ((rc = A(reinterpret_cast<void **>(p), static_cast<size_t>(r * r) * 4)) != COX_OK) break;
        if (rc) break;
        for (double **p : {&h->GV64, &h->GW64})
            if ((rc = A(reinterpret_cast<void **>(p), static_cast<size_t>(r * r) * 8)) != COX_OK) break;
        if (rc) break;
        if ((rc = A(reinterpret_cast<void **>(&h->fobj), 8)) != COX_OK) break;
        if ((rc = A(reinterpret_cast<void **>(&h->opart), static_cast<size_t>(upd_blocks(std::max(m, n))) * 8)) !=
            COX_OK)
            break;
        if ((rc = A(reinterpret_cast<void **>(&h->gpart), static_cast<size_t>(r * (r + 1) / 2) *
                                                                  upd_blocks(std::max(m, n)) * sizeof(float))) != COX_OK)
            break;
        if (cudaMemsetAsync(h->err, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(h->counters, 0, 4 * sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(h->Vl, 0, static_cast<size_t>(h->NP * h->ldm) * 2, st) != cudaSuccess ||
            cudaMemsetAsync(h->Wl, 0, static_cast<size_t>(h->NP * h->ldn) * 2, st) != cudaSuccess ||
            cudaMemsetAsync(h->Vt, 0, static_cast<size_t>(r * m) * 4, st) != cudaSuccess ||
            cudaMemsetAsync(h->W, 0, static_cast<size_t>(r * n) * 4, st) != cudaSuccess ||
            cudaMemsetAsync(h->GV32, 0, static_cast<size_t>(r * r) * 4, st) != cudaSuccess ||
            cudaMemsetAsync(h->GW32, 0, static_cast<size_t>(r * r) * 4, st) != cudaSuccess ||
            cudaMemsetAsync(h->GV64, 0, static_cast<size_t>(r * r) * 8, st) != cudaSuccess ||
            cudaMemsetAsync(h->GW64, 0, static_cast<size_t>(r * r) * 8, st) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        // X in row blocks of about 64 MB through a staging buffer
        const int64_t rows_blk = std::max<int64_t>(32, ((int64_t(64) << 20) / (4 * n)) / 32 * 32);
        const int64_t nrb = std::min(rows_blk, m);
        float *stage = nullptr;
        if (cudaMalloc(reinterpret_cast<void **>(&stage), static_cast<size_t>(nrb * n) * 4) != cudaSuccess) {
            cudaGetLastError();
            rc = COX_ERR_OOM;
            break;
        }
        const unsigned gx = static_cast<unsigned>((n + 31) / 32);
        double *d_sq = nullptr;
        const size_t nsq = static_cast<size_t>(gx) * ((nrb + 31) / 32);
        if (cudaMalloc(reinterpret_cast<void **>(&d_sq), nsq * 8) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(stage);
            rc = COX_ERR_OOM;
            break;
        }
        std::vector<double> sq(nsq);
        double xx = 0.0;
        for (int64_t r0 = 0; r0 < m && rc == COX_OK; r0 += nrb) {
            const int64_t nr = std::min(nrb, m - r0);
            const unsigned gy = static_cast<unsigned>((nr + 31) / 32);
            if (cudaMemcpyAsync(stage, X + r0 * n, static_cast<size_t>(nr * n) * 4, cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
                rc = COX_ERR_CUDA;
                break;
            }
            k_nmf_pack<<<dim3(gx, gy), dim3(32, 8), 0, st>>>(stage, r0, nr, n, h->Xr, h->ldr, h->Xc, h->ldc, d_sq,
                                                              h->err);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(sq.data(), d_sq, static_cast<size_t>(gx) * gy * 8, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = COX_ERR_CUDA;
                break;
            }
            for (size_t b = 0; b < static_cast<size_t>(gx) * gy; ++b) xx += sq[b];
        }
        cudaFree(stage);
        cudaFree(d_sq);
        if (rc) break;
        h->xx = xx;
        if ((rc = check_err(h, st)) != COX_OK) break;
        if ((rc = plan_side(h, h->s1, h->Xr, m, n, h->ldr, h->Wl, h->ldn, &h->part1)) != COX_OK) break;
        if ((rc = plan_side(h, h->s2, h->Xc, n, m, h->ldc, h->Vl, h->ldm, &h->part2)) != COX_OK) break;
        // the attribute is per function, not per handle: allow the device's
        // largest block, so that handles of any rank can run side by side
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            std::max(h->s1.smem, h->s2.smem) > static_cast<size_t>(optin) ||
            cudaFuncSetAttribute(k_nmf_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
            cudaFuncSetAttribute(k_nmf_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(upd_smem(NMF_MAX_RANK))) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
    } while (false);
    if (rc != COX_OK) {
        cudaGetLastError();
        release(h);
        return rc;
    }
    *out = h;
    return COX_OK;
}

} // namespace
} // namespace coxgb

using namespace coxgb;

extern "C" {

int nmf_setup(const float *X_host, int64_t m, int64_t n, int r, int device, nmf_h *out)
{
    if (!out) return COX_ERR_ARG;
    *out = nullptr;
    if (!X_host || m < 1 || n < 1 || r < 1 || r > NMF_MAX_RANK) return COX_ERR_ARG;
    if (m > (int64_t(1) << 31) - NT || n > (int64_t(1) << 31) - NT) return COX_ERR_ARG;
    return setup_impl(X_host, m, n, r, device, out);
}

int nmf_destroy(nmf_h h)
{
    if (!h) return COX_OK;
    DevGuard guard(h->dev);
    cudaStreamSynchronize(h->cap);
    release(h);
    return COX_OK;
}

int nmf_set_factors(nmf_h h, const float *V, const float *W, void *stream)
{
    if (!h || !V || !W) return COX_ERR_ARG;
    const int64_t m = h->m, n = h->n;
    const int r = h->r;
    for (int64_t e = 0; e < m * r; ++e)
        if (!(V[e] >= 0.f) || !std::isfinite(V[e])) return COX_ERR_ARG;
    for (int64_t e = 0; e < r * n; ++e)
        if (!(W[e] >= 0.f) || !std::isfinite(W[e])) return COX_ERR_ARG;
    DevGuard guard(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<float> vt(static_cast<size_t>(r * m));
    for (int64_t i = 0; i < m; ++i)
        for (int c = 0; c < r; ++c) vt[c * m + i] = V[i * r + c];
    COX_CUDA(cudaMemcpyAsync(h->Vt, vt.data(), vt.size() * 4, cudaMemcpyHostToDevice, st));
    COX_CUDA(cudaMemcpyAsync(h->W, W, static_cast<size_t>(r * n) * 4, cudaMemcpyHostToDevice, st));
    COX_TRY(launch_update(h, 0, 0, 0, 0.0, st));
    COX_TRY(launch_update(h, 1, 0, 0, 0.0, st));
    return check_err(h, st);
}

int nmf_get_factors(nmf_h h, float *V, float *W, void *stream)
{
    if (!h || !V || !W) return COX_ERR_ARG;
    DevGuard guard(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t m = h->m, n = h->n;
    const int r = h->r;
    std::vector<float> vt(static_cast<size_t>(r * m));
    COX_CUDA(cudaMemcpyAsync(vt.data(), h->Vt, vt.size() * 4, cudaMemcpyDeviceToHost, st));
    COX_CUDA(cudaMemcpyAsync(W, h->W, static_cast<size_t>(r * n) * 4, cudaMemcpyDeviceToHost, st));
    COX_TRY(check_err(h, st));
    for (int64_t i = 0; i < m; ++i)
        for (int c = 0; c < r; ++c) V[i * r + c] = vt[c * m + i];
    return COX_OK;
}

int nmf_iterate(nmf_h h, int algo, int64_t iters, double eps, void *stream)
{
    if (!h || iters < 0 || (algo != NMF_MULTIPLICATIVE && algo != NMF_APG) || !(eps >= 0.0) || !std::isfinite(eps))
        return COX_ERR_ARG;
    if (iters == 0) return COX_OK;
    DevGuard guard(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!h->exec || h->g_algo != algo || h->g_eps != eps) {
        if (h->exec) {
            cudaGraphExecDestroy(h->exec);
            h->exec = nullptr;
        }
        const int64_t before = h->launches;
        COX_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        int rc = launch_gemm(h, h->s1, h->cap);
        if (rc == COX_OK) rc = launch_update(h, 0, 1, algo, eps, h->cap);
        if (rc == COX_OK) rc = launch_gemm(h, h->s2, h->cap);
        if (rc == COX_OK) rc = launch_update(h, 1, 1, algo, eps, h->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(h->cap, &graph);
        h->launches = before;
        if (rc == COX_OK && (ec != cudaSuccess || cudaGraphInstantiate(&h->exec, graph, 0) != cudaSuccess))
            rc = COX_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        if (rc != COX_OK) {
            cudaGetLastError();
            h->exec = nullptr;
            return rc;
        }
        h->g_algo = algo;
        h->g_eps = eps;
    }
    for (int64_t t = 0; t < iters; ++t) COX_CUDA(cudaGraphLaunch(h->exec, st));
    h->launches += 6 * iters;
    return COX_OK;
}

int nmf_objective(nmf_h h, double *f, void *stream)
{
    if (!h || !f) return COX_ERR_ARG;
    DevGuard guard(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_TRY(launch_gemm(h, h->s1, st));
    FitArgs a;
    a.r = h->r;
    a.R = h->m;
    a.F = h->Vt;
    a.part = h->s1.g.part;
    a.SL = h->s1.g.SL;
    a.KC = h->s1.g.KC;
    a.L = h->s1.g.L;
    a.opart = h->opart;
    a.counter = h->counters + 2;
    a.GV = h->GV64;
    a.GW = h->GW64;
    a.xx = h->xx;
    a.out = h->fobj;
    k_nmf_fit<<<upd_blocks(h->m), UPD_ROWS * upd_warps(h->r), 0, st>>>(a);
    ++h->launches;
    COX_CUDA(cudaGetLastError());
    COX_CUDA(cudaMemcpyAsync(f, h->fobj, sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_err(h, st);
}

int nmf_sync(nmf_h h, void *stream)
{
    if (!h) return COX_ERR_ARG;
    DevGuard guard(h->dev);
    return check_err(h, static_cast<cudaStream_t>(stream));
}

int nmf_get_info(nmf_h h, nmf_info *o)
{
    if (!h || !o) return COX_ERR_ARG;
    o->m = h->m;
    o->n = h->n;
    o->r = h->r;
    o->limb_cols = h->NP;
    o->stages = h->s1.g.S;
    o->sm_count = h->sms;
    o->grid_xwt = h->s1.grid;
    o->grid_vtx = h->s2.grid;
    o->units_xwt = h->s1.g.units;
    o->units_vtx = h->s2.g.units;
    o->device_bytes = h->device_bytes;
    o->launches = h->launches;
    return COX_OK;
}

int nmf_time_products(nmf_h h, int reps, double *ms_xwt, double *ms_vtx, void *stream)
{
    if (!h || reps < 1 || !ms_xwt || !ms_vtx) return COX_ERR_ARG;
    DevGuard guard(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int rc = COX_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = COX_ERR_CUDA;
    if (rc == COX_OK) {
        cudaEventRecord(ev[0], st);
        for (int i = 0; i < reps && rc == COX_OK; ++i) rc = launch_gemm(h, h->s1, st);
        cudaEventRecord(ev[1], st);
        for (int i = 0; i < reps && rc == COX_OK; ++i) rc = launch_gemm(h, h->s2, st);
        cudaEventRecord(ev[2], st);
    }
    if (rc == COX_OK) rc = check_err(h, st);
    float a = 0.f, b = 0.f;
    if (rc == COX_OK &&
        (cudaEventElapsedTime(&a, ev[0], ev[1]) != cudaSuccess || cudaEventElapsedTime(&b, ev[1], ev[2]) != cudaSuccess))
        rc = COX_ERR_CUDA;
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    *ms_xwt = static_cast<double>(a) / reps;
    *ms_vtx = static_cast<double>(b) / reps;
    return rc;
}

} // extern "C"
