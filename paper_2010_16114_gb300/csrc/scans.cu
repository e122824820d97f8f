// scans.cu -- Breslow risk-set sums of the Cox iteration in FP64
// (arXiv 2010.16114, Section 5.3: w = exp(eta), W_j = sum_{y_i >= y_j} w_i,
// u = P delta; the paper's remark that sorting by time turns W into a
// cumulative sum; Section 6: Breslow ties).
//
// Subjects are stored in ascending time order, so with R_r = sum_{s >= r} w_s
// (a reverse inclusive scan), and the tie groups that hold events numbered
// g = 0, 1, ... in time order (head h_g, e_g events):
//   W_g = R_{h_g}                       the risk-set sum of group g
//   F_g = sum_{g' <= g} e_g' / W_g'     a forward scan over event groups
//   u_r = w_r F_{G(r) - 1}              G(r) = event groups with head <= r's
//                                       tie tail (u_r = 0 when G(r) = 0)
//   V_r = delta_r - u_r                 (the vector X^T multiplies)
//   f   = (1/n) [sum_g e_g log W_g - sum_r delta_r (eta_r - c)],  c = max eta.
// delta / W is nonzero only at events, and tied events share W, so the
// forward scan runs over the event groups (a few thousand with times in whole
// days) instead of the n subjects; the FP64 work that remains per subject is
// the reverse scan of w.  The reverse scan runs in fixed 2048-subject chunks
// (block scans with warp shuffles), then an exclusive scan of the chunk
// totals; the summation order never depends on timing, so results are
// bit-reproducible.
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
    const int32_t *evcnt;   // their event counts
    const int32_t *evidx;   // n: event groups with head <= the subject's tie tail
    const uint8_t *evflag;  // n: 1 at an event group's head
    int64_t n_evh;
    double *eta, *w, *Rt, *Fg, *lossg, *cmax, *csw, *suf, *lossp, *vsp;
    // unpenalised covariates (q columns; q = 0: none): Z q x n in sorted order,
    // gamma k x q, per-chunk partials of Z^T V (k x q x chunks)
    int q;
    const double *Z, *gamma;
    double *zvp;
};

constexpr int MAXQ = 16;

// (1) eta = sum of the product's partial slots (or a dense copy); chunk maxima;
// chunk sums of delta eta (the events' part of the loss).
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
    double mx = -INFINITY, de = 0.0;
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
        if (s.delta[i]) de += v;
    }
    const double m = block_max(mx, sh);
    if (threadIdx.x == 0) s.cmax[kk * s.nch + c] = m;
    const double t = block_sum(de, sh);
    if (threadIdx.x == 0) s.lossp[kk * s.nch + c] = t;
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

// (2) w = exp(eta - c); chunk-local reverse inclusive scan of w, kept at the
// heads of the tie groups that hold events (the only places W is read);
// chunk totals.
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
    for (int j = 0; j < PER; ++j) {
        const int64_t i = i0 + SCAN_CH - 1 - (PER * threadIdx.x + j);
        if (i < s.n && s.evflag[i]) s.Rt[kk * s.n + i] = loc[j] + excl;
    }
    if (threadIdx.x == NT - 1) s.csw[kk * s.nch + c] = incl;
}

// exclusive suffix scans of the chunk totals of w; one warp per column, lane
// l owning a contiguous run of chunks in scan order.
__global__ void k_chunks(SP s)
{
    const int kk = blockIdx.x, lane = threadIdx.x;
    const double *src = s.csw + static_cast<int64_t>(kk) * s.nch;
    double *dst = s.suf + static_cast<int64_t>(kk) * s.nch;
    const int per = (s.nch + 31) / 32;
    auto at = [&](int q) { return s.nch - 1 - q; };  // q-th chunk in scan order
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

// (3) One block per column, over the tie groups that hold events: W_g = the
// chunk-local reverse sum at the group's head plus the suffix of later chunks,
// D_g = e_g / W_g (one FP64 division per event time: tied events share W,
// Breslow), F = the inclusive scan of D over the groups, and the loss term
// sum_g e_g log W_g + (events) c.  Thread t takes a contiguous run of groups;
// the logs are taken of products carried as (mantissa, exponent), one log per
// thread (FP64 log is costly).
__global__ void k_group(SP s, bool need_loss)
{
    __shared__ double sh[NT / 32];
    const int kk = blockIdx.x;
    const int64_t G = s.n_evh;
    const int64_t per = (G + NT - 1) / NT;
    const int64_t g0 = min(G, per * threadIdx.x), g1 = min(G, g0 + per);
    const double cmx = need_loss ? column_max(s, kk, sh) : 0.0;
    double run = 0.0, pm = 1.0, lsum = 0.0;
    int pe = 0;
    long long nev = 0;
    for (int64_t g = g0; g < g1; ++g) {
        const int64_t hd = s.evhead[g];
        const double W = s.Rt[kk * s.n + hd] + s.suf[kk * s.nch + hd / SCAN_CH];
        const int e = s.evcnt[g];
        run += static_cast<double>(e) / W;
        s.Fg[kk * G + g] = run;  // local; the block offset is added below
        if (need_loss) {
            nev += e;
            if (e <= 8 && W >= 0x1p-1000 && W <= 0x1p+1000) {
                for (int q = 0; q < e; ++q) {
                    pm *= W;
                    pe += renorm(pm);
                }
            } else {
                lsum += static_cast<double>(e) * log(W);  // many tied events, or W zero, huge, subnormal, NaN
            }
        }
    }
    const double incl = block_incl_scan(run, sh);
    const double excl = incl - run;
    if (excl != 0.0)
        for (int64_t g = g0; g < g1; ++g) s.Fg[kk * G + g] += excl;
    if (need_loss) {
        lsum += log(pm) + static_cast<double>(pe) * 0.6931471805599453 + static_cast<double>(nev) * cmx;
        const double t = block_sum(lsum, sh);
        if (threadIdx.x == 0) s.lossg[kk] = t;
    }
}

// (4) C = F of the last event group at or before the tie tail; u = w C;
// V = delta - u -> output form; sum of V.
// The FP32 form feeds a product over the SNP-major copy and is written at its
// K positions (a4_pos); the FP64 form stays in sorted order.  For the e4m3
// limbs, V goes to Rt (free once the group kernel read it) with chunk maxima of |V|,
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
        const int32_t gi = s.evidx[i];
        const double C = gi > 0 ? s.Fg[kk * s.n_evh + gi - 1] : 0.0;
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

// (4b, e2m1 form) V -> e2m1 limbs at the A4 K positions: thread e of a chunk
// takes subjects 16 (e / 8) + e mod 8 and that + 8 of the chunk, which share
// one byte per limb row (e2m1_byte); chunk sums of the values the limbs hold,
// exact (integers of 2^(sc-22) units, below 2^35 per chunk).
__global__ void k_vlimbs4(SP s, uint8_t *__restrict__ Vq, int64_t n_pad, const double *__restrict__ vmaxp,
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
        s_sh = limb_scale4(mf);
        if (c == 0) bs[kk] = s_sh;
    }
    __syncthreads();
    const int sc = s_sh;
    const int64_t i0 = static_cast<int64_t>(c) * SCAN_CH;
    const float *V32 = reinterpret_cast<const float *>(s.Rt);
    const int64_t rb = n_pad / 2;
    long long q = 0;
    bool finite = true;
    for (int e = threadIdx.x; e < SCAN_CH / 2; e += NT) {
        const int64_t ia = i0 + ((e >> 3) << 4) + (e & 7);
        if (ia >= s.n) break;
        uint8_t d0[LIMBS4], d1[LIMBS4];
        const float ra = ldexpf(V32[kk * s.n + ia], -sc);
        finite = finite && isfinite(ra);
        q += split_e2m1_units(ra, d0);
        if (ia + 8 < s.n) {
            const float rb8 = ldexpf(V32[kk * s.n + ia + 8], -sc);
            finite = finite && isfinite(rb8);
            q += split_e2m1_units(rb8, d1);
        } else {
#pragma unroll
            for (int l = 0; l < LIMBS4; ++l) d1[l] = 0;
        }
        const int64_t byte = e2m1_byte(a4_pos(ia, s.pa, s.pnb));
#pragma unroll
        for (int l = 0; l < LIMBS4; ++l) Vq[(LIMBS4 * kk + l) * rb + byte] = static_cast<uint8_t>(d0[l] | (d1[l] << 4));
    }
    const double t = block_sum(finite ? static_cast<double>(q) : NAN, sh);
    if (threadIdx.x == 0) s.vsp[kk * s.nch + c] = ldexp(t, sc - (1 + 3 * (LIMBS4 - 1)));
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
        // f = (sum_g e_g log W_g + (events) c - sum_r delta_r eta_r) / n
        for (int c = lane; c < s.nch; c += 32) lo += s.lossp[kk * s.nch + c];
        if (l1p)
            for (int c = lane; c < l1_blocks; c += 32) b1 += l1p[kk * l1_blocks + c];
        lo = (s.lossg[kk] - warp_sum(lo)) / static_cast<double>(s.n);
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
    s.evcnt = h->d_evcnt;
    s.evidx = h->d_evidx;
    s.evflag = h->d_evflag;
    s.n_evh = h->n_evhead;
    s.q = a.gamma ? h->q : 0;  // no gamma: X_c beta alone (cox_eta)
    s.Z = h->d_Z;
    s.gamma = a.gamma;
    s.zvp = ws.zvp;
    s.eta = ws.eta;
    s.w = ws.w;
    s.Rt = ws.Rt;
    s.Fg = ws.Fg;
    s.lossg = ws.lossg;
    s.cmax = ws.cmax;
    s.csw = ws.csw;
    s.suf = ws.suf;
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
    k_chunks<<<a.k, 32, 0, st>>>(s);
    k_group<<<a.k, NT, 0, st>>>(s, a.need_loss);
    switch (a.v_out) {
    case V_LIMBS_E4M3:
        k_uv<V_LIMBS_E4M3><<<grid, NT, 0, st>>>(s, a.V, h->n_pad, ws.vmaxp);
        if (ws.g4.f4)
            k_vlimbs4<<<grid, NT, 0, st>>>(s, static_cast<uint8_t *>(a.V), h->n_pad, ws.vmaxp, ws.bs4, h->d_err);
        else
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
