// scans.cu -- Breslow risk-set sums of the Cox iteration in FP64
// (arXiv 2010.16114, Section 5.3: w = exp(eta), W_j = sum_{y_i >= y_j} w_i,
// u = P delta; the paper's remark that sorting by time turns W into a
// cumulative sum; Section 6: Breslow ties).
//
// Subjects are stored in ascending time order, so with R_r = sum_{s >= r} w_s
// (a reverse inclusive scan) and F_r = sum_{s <= r} delta_s / W_s (a forward
// inclusive scan):
//   W_r = R_{head(r)}            head = first position of r's tie group
//   u_r = w_r F_{tail(r)}        tail = last position of r's tie group
//   V_r = delta_r - u_r          (the vector X^T multiplies)
//   f   = (1/n) sum_r delta_r (log W_r - (eta_r - c)),  c = max eta.
// Each scan runs in fixed 2048-subject chunks (block scans with warp
// shuffles), then an exclusive scan of the chunk totals, then a gather; the
// summation order never depends on timing, so results are bit-reproducible.
#include <algorithm>

#include "internal.h"

namespace coxgb {
namespace {

constexpr int NT = 256;
constexpr int PER = SCAN_CH / NT;  // 8

__device__ __forceinline__ double warp_incl_scan(double x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Inclusive scan of one value per thread across the 256-thread block.
__device__ __forceinline__ double block_incl_scan(double x, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = warp_incl_scan(x, lane);
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        double v = lane < NT / 32 ? sh[lane] : 0.0;
        v = warp_incl_scan(v, lane);
        if (lane < NT / 32) sh[lane] = v;
    }
    __syncthreads();
    if (warp > 0) x += sh[warp - 1];
    __syncthreads();
    return x;
}

__device__ __forceinline__ double block_sum(double x, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
    __syncthreads();
    return t;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double x, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    double t = -INFINITY;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t = fmax(t, sh[w]);
    __syncthreads();
    return t;
}

// m (positive, normal) -> m 2^-e in [1, 2); returns e.  Lets a product of
// many positive factors be carried as (mantissa, exponent) without overflow.
__device__ __forceinline__ int renorm(double &m)
{
    const long long b = __double_as_longlong(m);
    m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    return static_cast<int>(b >> 52) - 1023;
}

struct SP {
    int64_t n, n_pad;
    int nch, k;
    int64_t pa, pnb;  // K order of the SNP-major genotype copy (a4_pos)
    const uint8_t *delta;
    const int32_t *head, *tail;
    const int32_t *evhead;  // first positions of the tie groups that hold an event
    int64_t n_evh;
    double *eta, *w, *Rt, *Ft, *cmax, *csw, *csd, *suf, *pre, *lossp, *vsp;
    // unpenalised covariates (q columns; q = 0: none): Z q x n in sorted order,
    // gamma k x q, per-chunk partials of Z^T V (k x q x chunks)
    int q;
    const double *Z, *gamma;
    double *zvp;
};

constexpr int MAXQ = 16;

// (1) eta = sum of the product's partial slots (or a dense copy); chunk maxima.
template <int SRC>
__global__ void k_eta(SP s, const void *src, int64_t slot_stride, int64_t col_stride, int group_rows,
                      int KC, int64_t L)
{
    __shared__ double sh[NT / 32];
    __shared__ int cnt_sh[SCAN_CH / 128];  // partial slots of the row groups of this chunk
    const int c = blockIdx.x, kk = blockIdx.y;
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    if (SRC == ETA_PARTIAL_F32) {
        // group_rows (128 or 256) divides SCAN_CH: the chunk holds whole groups
        if (threadIdx.x < SCAN_CH / group_rows) {
            const int64_t g = i0 / group_rows + threadIdx.x;
            cnt_sh[threadIdx.x] = static_cast<int>((g * KC + KC - 1) / L - (g * KC) / L + 1);
        }
        __syncthreads();
    }
    double mx = -INFINITY;
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        if (i >= s.n) break;
        double v;
        if (SRC == ETA_PARTIAL_F32) {
            const float *part = static_cast<const float *>(src);
            const int cnt = cnt_sh[e / group_rows];
            v = 0.0;
            for (int sl = 0; sl < cnt; ++sl) v += static_cast<double>(part[sl * slot_stride + kk * col_stride + i]);
        } else if (SRC == ETA_DENSE_F32) {
            v = static_cast<double>(static_cast<const float *>(src)[kk * col_stride + i]);
        } else {
            v = static_cast<const double *>(src)[kk * col_stride + i];
        }
        if (s.q) {  // eta += Z gamma (Section 6 unpenalised covariates), in FP64
            double zg = 0.0;
            for (int cq = 0; cq < s.q; ++cq) zg += s.Z[cq * s.n + i] * s.gamma[kk * s.q + cq];
            v += zg;
        }
        s.eta[kk * s.n + i] = v;
        mx = fmax(mx, v);
    }
    const double m = block_max(mx, sh);
    if (threadIdx.x == 0) s.cmax[kk * s.nch + c] = m;
}

__device__ __forceinline__ double column_max(const SP &s, int kk, double *sh)
{
    double m = -INFINITY;
    for (int c = threadIdx.x; c < s.nch; c += NT) m = fmax(m, s.cmax[kk * s.nch + c]);
    m = block_max(m, sh);
    if (threadIdx.x == 0) sh[0] = m;
    __syncthreads();
    m = sh[0];
    __syncthreads();
    return m;
}

// (2) w = exp(eta - c); chunk-local reverse inclusive scan of w; chunk totals.
template <bool EXP64>
__global__ void k_rev(SP s)
{
    __shared__ double sh[NT / 32];
    __shared__ double buf[SCAN_CH];
    const int c = blockIdx.x, kk = blockIdx.y;
    const double cmx = column_max(s, kk, sh);
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        double wv = 0.0;
        if (i < s.n) {
            const double x = s.eta[kk * s.n + i] - cmx;
            wv = EXP64 ? exp(x) : static_cast<double>(expf(static_cast<float>(x)));
            s.w[kk * s.n + i] = wv;
        }
        buf[e] = wv;
    }
    __syncthreads();
    // thread t owns reversed positions [PER t, PER t + PER): elements SCAN_CH-1-(PER t + j)
    double loc[PER];
    double run = 0.0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        run += buf[SCAN_CH - 1 - (PER * threadIdx.x + j)];
        loc[j] = run;
    }
    const double incl = block_incl_scan(run, sh);
    const double excl = incl - run;
#pragma unroll
    for (int j = 0; j < PER; ++j) buf[SCAN_CH - 1 - (PER * threadIdx.x + j)] = loc[j] + excl;
    __syncthreads();
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        if (i < s.n) s.Rt[kk * s.n + i] = buf[e];
    }
    if (threadIdx.x == NT - 1) s.csw[kk * s.nch + c] = incl;
}

// exclusive scans of chunk totals: suffix (reverse) or prefix (forward); one
// warp per column, lane l owning a contiguous run of chunks in scan order.
template <bool SUFFIX>
__global__ void k_chunks(SP s)
{
    const int kk = blockIdx.x, lane = threadIdx.x;
    const double *src = (SUFFIX ? s.csw : s.csd) + static_cast<int64_t>(kk) * s.nch;
    double *dst = (SUFFIX ? s.suf : s.pre) + static_cast<int64_t>(kk) * s.nch;
    const int per = (s.nch + 31) / 32;
    auto at = [&](int q) { return SUFFIX ? s.nch - 1 - q : q; };  // q-th chunk in scan order
    double tot = 0.0;
    for (int j = 0; j < per; ++j) {
        const int q = lane * per + j;
        if (q < s.nch) tot += src[at(q)];
    }
    const double incl = warp_incl_scan(tot, lane);
    double acc = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) acc = 0.0;
    for (int j = 0; j < per; ++j) {
        const int q = lane * per + j;
        if (q < s.nch) {
            dst[at(q)] = acc;
            acc += src[at(q)];
        }
    }
}

// (2b) 1/W in FP64 once per tie group that holds an event: W = R at the
// group's first position (chunk-local reverse scan plus the suffix of later
// chunks), and Rt there is overwritten with 1/W.  Every event of the group
// reads that one value (Breslow: tied events share W), so the FP64 divides
// number the event times (at most a few thousand with times in whole days),
// not the events, and run without divergence.
__global__ void k_inv_w(SP s)
{
    const int kk = blockIdx.y;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < s.n_evh;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t hd = s.evhead[q];
        const double W = s.Rt[kk * s.n + hd] + s.suf[kk * s.nch + hd / SCAN_CH];
        s.Rt[kk * s.n + hd] = 1.0 / W;
    }
}

// (3) D = delta / W (from the group heads' 1/W); loss terms; chunk-local
// forward scan of D, all in FP64.
__global__ void k_fwd(SP s, bool need_loss)
{
    __shared__ double sh[NT / 32];
    __shared__ double buf[SCAN_CH];
    const int c = blockIdx.x, kk = blockIdx.y;
    const double cmx = need_loss ? column_max(s, kk, sh) : 0.0;
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    // The loss terms log W = -log(1/W) are summed as the log of a product:
    // each thread multiplies its 1/W into pm 2^pe (pm in [1, 2)), the warp
    // multiplies its lanes' products, and one log per warp remains (FP64 log is
    // costly and events are sparse, so a per-event log would run in most warps
    // anyway).
    double lsum = 0.0, pm = 1.0;
    int pe = 0;
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        double d = 0.0;
        if (i < s.n && s.delta[i]) {
            d = s.Rt[kk * s.n + s.head[i]];  // 1/W of i's tie group
            if (need_loss) {
                lsum -= s.eta[kk * s.n + i] - cmx;
                if (d >= 0x1p-1000 && d <= 0x1p+1022) {
                    pm *= d;
                    pe += renorm(pm);
                } else {
                    lsum -= log(d);  // zero, huge, subnormal or NaN: as a plain sum of logs
                }
            }
        }
        buf[e] = d;
    }
    __syncthreads();
    double loc[PER];
    double run = 0.0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        run += buf[PER * threadIdx.x + j];
        loc[j] = run;
    }
    const double incl = block_incl_scan(run, sh);
    const double excl = incl - run;
#pragma unroll
    for (int j = 0; j < PER; ++j) buf[PER * threadIdx.x + j] = loc[j] + excl;
    __syncthreads();
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        if (i < s.n) s.Ft[kk * s.n + i] = buf[e];
    }
    if (threadIdx.x == NT - 1) s.csd[kk * s.nch + c] = incl;
    if (need_loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {  // every lane ends with the same product
            pm *= __shfl_xor_sync(0xffffffffu, pm, o);
            pe += __shfl_xor_sync(0xffffffffu, pe, o);
            pe += renorm(pm);
        }
        // sum of log W over this warp's events = -log(product of 1/W)
        if ((threadIdx.x & 31) == 0) lsum -= log(pm) + static_cast<double>(pe) * 0.6931471805599453;
        const double t = block_sum(lsum, sh);
        if (threadIdx.x == 0) s.lossp[kk * s.nch + c] = t;
    }
}

// (4) C = F at the tie tail; u = w C; V = delta - u -> output form; sum of V.
// The FP32 form feeds a product over the SNP-major copy and is written at its
// K positions (a4_pos); the FP64 form stays in sorted order.  For the e4m3
// limbs, V goes to Rt (free after the forward scan) with chunk maxima of |V|,
// and k_vlimbs splits it once the column's scale is known.
template <int VO>
__global__ void k_uv(SP s, void *Vout, int64_t n_pad, double *vmaxp)
{
    __shared__ double sh[NT / 32];
    const int c = blockIdx.x, kk = blockIdx.y;
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    double vs = 0.0;
    float vm32 = 0.f;
    double zv[MAXQ];  // Z^T V over this thread's subjects (unpenalised covariates)
#pragma unroll
    for (int cq = 0; cq < MAXQ; ++cq) zv[cq] = 0.0;
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        if (i >= s.n) break;
        const int64_t tl = s.tail[i];
        const double C = s.Ft[kk * s.n + tl] + s.pre[kk * s.nch + tl / SCAN_CH];
        const double u = s.w[kk * s.n + i] * C;
        const double V = static_cast<double>(s.delta[i]) - u;
        if (s.q) {
#pragma unroll
            for (int cq = 0; cq < MAXQ; ++cq)
                if (cq < s.q) zv[cq] += s.Z[cq * s.n + i] * V;
        }
        // sum V in the form the product reads: X^T V - mu sum V is then
        // exactly the centred product of that V.  (Censored subjects between
        // two event times share one V, so their rounding errors do not
        // cancel; with the exact sum, mu times their sum would remain.)
        if (VO == V_LIMBS_E4M3) {
            // k_vlimbs splits the FP32 value: hand it over in FP32 (the max of
            // the rounded values is the rounded max, so the scale is unchanged)
            const float v32 = static_cast<float>(V);
            reinterpret_cast<float *>(s.Rt)[kk * s.n + i] = v32;
            vm32 = fmaxf(vm32, fabsf(v32));
        } else if (VO == V_DENSE_F64) {
            static_cast<double *>(Vout)[kk * s.n + i] = V;
            vs += V;
        } else {
            const float v32 = static_cast<float>(V);
            static_cast<float *>(Vout)[a4_pos(i, s.pa, s.pnb) + kk * n_pad] = v32;
            vs += static_cast<double>(v32);
        }
    }
    if (VO == V_LIMBS_E4M3) {
        const double m = block_max(static_cast<double>(vm32), sh);
        if (threadIdx.x == 0) vmaxp[kk * s.nch + c] = m;
    } else {
        const double t = block_sum(vs, sh);
        if (threadIdx.x == 0) s.vsp[kk * s.nch + c] = t;
    }
    for (int cq = 0; cq < s.q; ++cq) {  // block-uniform trip count
        double zc = 0.0;
#pragma unroll
        for (int q2 = 0; q2 < MAXQ; ++q2)
            if (q2 == cq) zc = zv[q2];
        const double t = block_sum(zc, sh);
        if (threadIdx.x == 0) s.zvp[(static_cast<int64_t>(kk) * s.q + cq) * s.nch + c] = t;
    }
}

// (4b) V (FP32, in Rt) -> e4m3 limbs at the A4 K positions, one power-of-two
// scale per column (from all chunk maxima); chunk sums of the values the limbs
// hold, exact: each is an integer number of 2^(sc-21) units below 2^30, so
// a chunk's sum is an integer below 2^42, exact in FP64.
__global__ void k_vlimbs(SP s, uint8_t *__restrict__ Vq, int64_t n_pad, const double *__restrict__ vmaxp,
                         int *__restrict__ bs, int *err)
{
    __shared__ double sh[NT / 32];
    __shared__ int s_sh;
    const int c = blockIdx.x, kk = blockIdx.y;
    double m = 0.0;
    for (int q = threadIdx.x; q < s.nch; q += NT) m = fmax(m, vmaxp[kk * s.nch + q]);
    m = block_max(m, sh);
    if (threadIdx.x == 0) {
        float mf = static_cast<float>(m);
        if (!isfinite(mf)) {
            atomicOr(err, DEVERR_NONFINITE);
            mf = 0.f;
        }
        s_sh = limb_scale(mf);
        if (c == 0) bs[kk] = s_sh;
    }
    __syncthreads();
    const int sc = s_sh;
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    const float *V32 = reinterpret_cast<const float *>(s.Rt);
    long long q = 0;
    bool finite = true;
    for (int e = threadIdx.x; e < SCAN_CH; e += NT) {
        const int64_t i = i0 + e;
        if (i >= s.n) break;
        uint8_t d[LIMBS];
        // ldexpf of the FP32 value equals rounding the scaled FP64 value: the
        // scale is a power of two and |V| >= 1/n whenever V is not all zero,
        // so nothing the limbs can hold falls into FP32's subnormal range
        const float r = ldexpf(V32[kk * s.n + i], -sc);
        finite = finite && isfinite(r);
        q += split_e4m3_units(r, d);
        const int64_t pos = a4_pos(i, s.pa, s.pnb);
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) Vq[(LIMBS * kk + l) * n_pad + pos] = d[l];
    }
    const double t = block_sum(finite ? static_cast<double>(q) : NAN, sh);
    if (threadIdx.x == 0) s.vsp[kk * s.nch + c] = ldexp(t, sc - 21);
}

// (5) per column (one warp each): sum V, f, ||beta||_1, F = f + lambda ||beta||_1;
// flag non-finite.
__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// With unpenalised covariates also g_Z = Z^T (delta - u) / n per column, and,
// for a step, gamma <- gamma + step g_Z (Section 6: the covariates take a plain
// gradient step; a frozen column keeps its gamma).
__global__ void k_finalize(SP s, int l1_blocks, const double *l1p, const double *lam, double *sumV,
                           double *f, double *l1, double *Fobj, bool need_loss, int *err, double *gz,
                           double *gamma, const int *active, double step, bool gamma_step)
{
    const int kk = blockIdx.x, lane = threadIdx.x;
    for (int cq = 0; cq < s.q; ++cq) {
        double z = 0.0;
        for (int c = lane; c < s.nch; c += 32) z += s.zvp[(static_cast<int64_t>(kk) * s.q + cq) * s.nch + c];
        z = warp_sum(z) / static_cast<double>(s.n);
        if (lane == 0) {
            gz[kk * s.q + cq] = z;
            if (gamma_step && (!active || active[kk])) gamma[kk * s.q + cq] += step * z;
            if (!isfinite(z)) atomicOr(err, DEVERR_NONFINITE);
        }
    }
    double v = 0.0, lo = 0.0, b1 = 0.0;
    for (int c = lane; c < s.nch; c += 32) v += s.vsp[kk * s.nch + c];
    v = warp_sum(v);
    if (need_loss) {
        for (int c = lane; c < s.nch; c += 32) lo += s.lossp[kk * s.nch + c];
        if (l1p)
            for (int c = lane; c < l1_blocks; c += 32) b1 += l1p[kk * l1_blocks + c];
        lo = warp_sum(lo) / static_cast<double>(s.n);
        b1 = warp_sum(b1);
    }
    if (lane != 0) return;
    sumV[kk] = v;
    if (need_loss) {
        f[kk] = lo;
        l1[kk] = b1;
        Fobj[kk] = lo + (lam ? lam[kk] * b1 : 0.0);
        if (!isfinite(lo)) atomicOr(err, DEVERR_NONFINITE);
    }
    if (!isfinite(v)) atomicOr(err, DEVERR_NONFINITE);
}

} // namespace

int run_scans(cox_handle *h, const ScanArgs &a, cudaStream_t st)
{
    Workspace &ws = h->ws;
    SP s;
    s.n = h->n;
    s.n_pad = h->n_pad;
    s.nch = h->n_chunks;
    s.k = a.k;
    s.pa = h->kperm_a;
    s.pnb = h->kperm_nb;
    s.delta = h->d_delta;
    s.head = h->d_head;
    s.tail = h->d_tail;
    s.evhead = h->d_evhead;
    s.n_evh = h->n_evhead;
    s.q = a.gamma ? h->q : 0;  // no gamma: X_c beta alone (cox_eta)
    s.Z = h->d_Z;
    s.gamma = a.gamma;
    s.zvp = ws.zvp;
    s.eta = ws.eta;
    s.w = ws.w;
    s.Rt = ws.Rt;
    s.Ft = ws.Ft;
    s.cmax = ws.cmax;
    s.csw = ws.csw;
    s.csd = ws.csd;
    s.suf = ws.suf;
    s.pre = ws.pre;
    s.lossp = ws.lossp;
    s.vsp = ws.vsp;
    dim3 grid(h->n_chunks, a.k);
    switch (a.eta_src) {
    case ETA_PARTIAL_F32:
        k_eta<ETA_PARTIAL_F32><<<grid, NT, 0, st>>>(s, a.eta, a.slot_stride, a.col_stride, a.group_rows, a.KC, a.L);
        break;
    case ETA_DENSE_F32:
        k_eta<ETA_DENSE_F32><<<grid, NT, 0, st>>>(s, a.eta, 0, a.col_stride, 1, 1, 1);
        break;
    default:
        k_eta<ETA_DENSE_F64><<<grid, NT, 0, st>>>(s, a.eta, 0, a.col_stride, 1, 1, 1);
        break;
    }
    if (a.eta_only) {
        COX_CUDA(cudaGetLastError());
        return COX_OK;
    }
    if (a.exp64) k_rev<true><<<grid, NT, 0, st>>>(s);
    else k_rev<false><<<grid, NT, 0, st>>>(s);
    k_chunks<true><<<a.k, 32, 0, st>>>(s);
    if (h->n_evhead > 0) {
        const unsigned gx = static_cast<unsigned>(std::min<int64_t>((h->n_evhead + NT - 1) / NT, 64));
        k_inv_w<<<dim3(gx, a.k), NT, 0, st>>>(s);
    }
    k_fwd<<<grid, NT, 0, st>>>(s, a.need_loss);
    k_chunks<false><<<a.k, 32, 0, st>>>(s);
    switch (a.v_out) {
    case V_LIMBS_E4M3:
        k_uv<V_LIMBS_E4M3><<<grid, NT, 0, st>>>(s, a.V, h->n_pad, ws.vmaxp);
        k_vlimbs<<<grid, NT, 0, st>>>(s, static_cast<uint8_t *>(a.V), h->n_pad, ws.vmaxp, ws.bs4, h->d_err);
        break;
    case V_DENSE_F64: k_uv<V_DENSE_F64><<<grid, NT, 0, st>>>(s, a.V, h->n_pad, nullptr); break;
    default: k_uv<V_DENSE_F32><<<grid, NT, 0, st>>>(s, a.V, h->n_pad, nullptr); break;
    }
    k_finalize<<<a.k, 32, 0, st>>>(s, h->l1_blocks, a.need_loss ? ws.l1p : nullptr, a.lam, ws.sumV, ws.f, ws.l1,
                                 ws.F, a.need_loss, h->d_err, a.gz, a.gamma, a.active, a.step, a.gamma_step);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

} // namespace coxgb
