// gemm_tc.cu -- the two genotype products of the Cox iteration on tcgen05
// tensor cores (arXiv 2010.16114, Section 5.3: X beta, and Delta = X^T (I-P) delta):
//
//   first product : D = X_sorted (n x p) * Bhat (p x 4k)    -> eta partials
//   second product: D = X^T (p x n) * Vhat (n x 4k)         -> X^T V, then the
//                   soft-threshold step (Section 4.2) in the epilogue.
//
// A is the 2-bit genotype matrix in a tiled layout (128 x 128 blocks of 4 KB),
// loaded by TMA into shared memory, decoded by warps into Tensor Memory and
// consumed by tcgen05.mma as the A operand (kind::f8f6f4, e4m3 A from TMEM,
// e4m3 B from 128B-swizzled shared memory, FP32 accumulators in TMEM).
//
// Decode: a genotype code c in {0,1,2} as an e4m3 byte is the subnormal
// c * 2^-9, exact in the tensor core; the packed layout (code_bit) makes one
// shift and one AND produce four such bytes.
//
// B holds each coefficient column c as LIMBS = 4 e4m3 limbs (rows 4c .. 4c+3):
// with r_0 = b 2^-s (s per column, |r_0| <= 256), d_l = RN_e4m3(r_l) and
// r_(l+1) = 16 (r_l - d_l), b = 2^s sum_l d_l 2^-4l to ~16 significant bits.
// The fold adds a column's limb accumulators with their weights 2^-4l and the
// partial is scaled by 2^(s+9).
//
// Pipeline per CTA (one per SM): two TMA warps fill a ring of shared-memory
// stages (T row tiles x CH K chunks of codes, and the matching limb panels);
// groups of four decoder warps turn a stage into e4m3 in a ring of TMEM slots,
// issuing all of a tile's tcgen05.st before one wait; one issuer warp per row
// tile issues the stage's MMAs into its own accumulator and commits.  Decoders
// hand a tile to its issuer through a hardware named barrier (tens of cycles,
// against a few hundred for an mbarrier arrive and wait), and every wait or
// commit serves a whole stage.
//
// Accumulation: each accumulator sums at most one window of K chunks in FP32
// in TMEM, then decoder group 0 adds the window into FP32 sums (round to
// nearest).  The K order of the X^T V product spreads the time order
// (setup.cu), so these running sums stay near the size of the result instead
// of drifting with the time trend of V.
//
// Issue modes.  Per tile (ALT = false): one issuer warp per row tile issues
// that tile's MMAs of every stage (T issuers, 4 CH MMAs per commit).
// Alternating (ALT = true): two issuer warps take alternate stages and each
// issues every tile of its stage into its own accumulators (4 CH T MMAs per
// commit; a commit costs the tensor pipe a few hundred cycles, so longer
// bursts per commit raise the MMA rate).  With two decoder groups, an even
// number of TMEM slots and an even number of shared-memory stages, the stages
// of one parity form a chain of their own: one producer warp, one decoder
// group, one issuer and their own slots and stages.  The window folds add the
// two issuers' accumulators.
//
// Work split: units = (M group, stage) pairs; CTA c takes the contiguous range
// [c L, (c+1) L).  A group that runs entirely in one CTA gets the epilogue
// straight from its sums; a group cut between CTAs gets one partial per CTA
// (slot = CTA - first CTA of the group), and the last CTA to finish it sums
// the slots in slot order (deterministic) and applies the epilogue.
#include <algorithm>

#include "internal.h"
#include "ptx.cuh"

namespace coxgb {
namespace {

struct KParams {
    int KC, F, k, stages, ring, nb_period;
    int pair;           // per-tile issuers commit after every second stage of a window
    const int *bscale;  // k: power-of-two scale of the B limbs
    int64_t units, L;
    int64_t rows_pad, slot_stride;
    float *part;
    int epi;
    int *counters;
    float *beta;
    float *grad;
    const double *lam;
    double step;
    const double *mu;
    const double *sumV;
    const int *active;
    uint8_t *near;      // may be null: SNPs whose |z| came within a quarter of the threshold
    int64_t rows_valid;
    double inv_n;
    long long wait_limit;
    int *err;
};

constexpr long long DRAIN_LIMIT = 4000000000LL;  // ~2 s: copies/MMAs always finish
__device__ int g_never_set = 0;                 // abort flag for drain waits: never raised

// 16 codes of a packed word -> 16 e4m3 bytes (four TMEM columns, K order)
__device__ __forceinline__ void decode16(uint32_t P, uint32_t *o)
{
    o[0] = P & 0x03030303u;
    o[1] = (P >> 2) & 0x03030303u;
    o[2] = (P >> 4) & 0x03030303u;
    o[3] = (P >> 6) & 0x03030303u;
}

__device__ __forceinline__ void fail(volatile int *abort_sm, int *err)
{
    if (!*abort_sm) {
        *abort_sm = 1;
        atomicOr(err, DEVERR_TIMEOUT);
    }
}

// all lanes wait; the warp agrees on the outcome (polling from lane 0 alone,
// with or without sleeping between polls, measured slower)
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, long long lim, volatile int *abort)
{
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, lim, abort));
}

// Warp roles (WARPS = 2 + I + 4 G, I = T issuers, or 2 when alternating):
//   warps 0, 1     TMA producers (lane 0): warp w loads the stages i = w (mod 2);
//                  warp 0 also allocates TMEM
//   warps 2..T+1   MMA issuers: issuer t owns row tile t and accumulates it
//                  into its own TMEM accumulator, 4 CH MMAs (K = 32 each) per
//                  barrier wait and commit.
//   warps T+2..    G decoder groups of four warps (one per TMEM lane quarter);
//                  group gamma decodes the stages i = gamma (mod G) into TMEM
//                  slot i mod R.  Group 0 also adds the accumulators up at window
//                  ends and runs the epilogue.
// Hand-offs of stage i (shared-memory slot s = i mod S, TMEM slot r = i mod R):
//   full[s]        mbarrier, TMA transaction bytes           producer -> decoders
//   named 1+(i%PB)T+t  hardware barrier: tile t of the slot   decoders -> issuer of tile t
//                  written (one barrier per tile, so the issuers of a stage do
//                  not wait for one another)
//   aempty[r]      tcgen05.commit of the T issuers           -> decoders of stage i+R
//   empty[s]       one arrival by the decoders of stage i+R once they have seen
//                  aempty for stage i (its MMAs, which read B and follow the
//                  decoders' reads of X, are complete)       -> producer
// Parity waits must not alias: when a warp waits for a phase, the phase
// before it must be complete (else the wait can return a phase early).  The
// MMAs of a stage complete only after its decoders finished, who had waited
// for its load and arrived on empty for stage - R; issuers go in stage order.
// So the MMAs of stage x being complete means every stage <= x was loaded and
// decoded.  Per barrier (G groups, R slots, S stages, 2 producer warps):
//   aempty, decoders of stage i wait for stage i - R and need stage i - 2R:
//     their own wait at stage i - G completed stage i - G - R: G <= R.
//   full, decoders of stage i wait for the load of stage i and need the load
//     of stage i - S: (a) S >= G + R (the same wait covers it), or (b) S a
//     multiple of G (their own group loaded stage i - S), or (c) R a multiple
//     of G (the load of stage i - G followed the release of stage i - G - S by
//     the decoders of stage i - G - S + R, the group of stage i - S, later).
//   empty, the producer of stage j waits for stage j - S's release and needs
//     stage j - 2S's: S even (one producer warp owns the slot), or S >= R + 2
//     (its load of stage j - 2 followed the release of stage j - 2 - S, so the
//     MMAs of that stage and the releases of every stage <= j - 2 - S - R).
// parity_safe() holds these and the planner keeps to them.  With R < G (two
// slots against three groups, as three K chunks per stage would leave) small
// cases ran exact at S = 4 while a full-size run never finished.
// Alternating issuers (ALT): warps 2, 3 issue the stages i = 0, 1 (mod 2);
// G = 2, and R and S are even, so stage i's producer warp, decoder group,
// issuer, TMEM slot i mod R and shared-memory slot i mod S all belong to the
// parity class i mod 2, and each barrier is only ever used by one class.
// Issuers no longer go in stage order across classes, but within a class they
// do, and every wait above is answered from inside the class: a decoder's
// wait on aempty (stage i - R) follows its own wait for stage i - 2R, its
// wait on full (stage i) its own wait for stage i - S, a producer's wait on
// empty (stage j - S) its own wait for stage j - 2S; a named barrier
// (period PB = lcm(2, R) stages, T per stage) is reused by the decoders of
// stage i + PB only after they saw aempty for stage i + PB - R >= i, which its
// issuer commits after passing the barrier of stage i.  The folds need both
// classes' MMAs of a window, which the issuers commit to accf (count 2).
// PB = lcm(G, R): each use of a named barrier has the same warps, and the
// decoders of stage i+PB cannot arrive before the issuer of stage i has passed
// it (they first wait, through the TMEM slot chain, for MMAs that this issuer
// issues after it).  Decoders arrive on every path, so an issuer's (unbounded)
// hardware-barrier wait always ends.
template <int T, int CH, int NP, int G, bool ALT>
__global__ void __launch_bounds__(32 * (2 + (ALT ? 2 : T) + 4 * G), 1)
    k_packed_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const KParams P)
{
    constexpr int I = ALT ? 2 : T;        // MMA issuers: one per row tile, or two on alternate stages
    static_assert(!ALT || G == 2, "alternating issuers pair with two decoder groups");
    constexpr int KH = NP / LIMBS;        // lambda columns a decoder thread folds (>= k)
    constexpr int B_BYTES = CH * NP * 128;       // CH chunk panels of NP rows x 128 bytes
    constexpr int X_BYTES = T * CH * BLOCK_BYTES;  // [tile][chunk] 4 KB blocks
    constexpr int STAGE = B_BYTES + X_BYTES;
    constexpr int ACC_COLS = (ALT ? 2 * T : T) * NP;  // accumulators: per tile, or per issuer and tile
    constexpr int SLOT_COLS = T * CH * 32;  // 128 e4m3 A values per lane, tile and chunk
    constexpr int DEC0 = 2 + I;           // first decoder warp
    constexpr int NB_COUNT = 32 * 5;      // a decoder group and the tile's issuer warp

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    const int S = P.stages, R = P.ring, PB = P.nb_period;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * STAGE);
    const uint32_t full0 = smem_addr(bars);
    const uint32_t empty0 = full0 + 8 * S;
    const uint32_t aempty0 = empty0 + 8 * S;
    const uint32_t accf = aempty0 + 8 * R;
    const uint32_t acce = accf + 8;
    const uint32_t drainb = acce + 8;
    const uint32_t epib = drainb + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + R + 4);
    volatile int *abort_sm = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *last_sm = reinterpret_cast<volatile int *>(tmem_slot + 2);
    volatile int *armed = reinterpret_cast<volatile int *>(tmem_slot + 4);  // [S] parity of the last TMA into a slot

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
            armed[s] = -1;
        }
        for (int r = 0; r < R; ++r) mbar_init(aempty0 + 8 * r, ALT ? 1 : T);  // commits per stage
        mbar_init(accf, I);
        mbar_init(acce, 4);
        mbar_init(drainb, I);
        mbar_init(epib, 4);
        *abort_sm = 0;
        *last_sm = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), 512);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    const int64_t cta = blockIdx.x;
    const int64_t u0 = cta * P.L;
    const int64_t u1 = min(u0 + P.L, P.units);
    const int64_t nu = u1 > u0 ? u1 - u0 : 0;
    const int KC = P.KC, F = P.F;
    const long long lim = P.wait_limit;
    // position of the first unit; the loops below advance their counters by
    // increments only (no division on the per-stage path)
    const int g0 = static_cast<int>(u0 / KC), kc0 = static_cast<int>(u0 - static_cast<int64_t>(g0) * KC);

    if (warp < 2) {
        // ---------------- TMA producers ----------------
        if (lane == 0) {
            const int w = warp;
            int s = w, kc = kc0 + w, g = g0;
            if (kc >= KC) {
                kc -= KC;
                ++g;
            }
            uint32_t ph = 0;
            for (int64_t i = w; i < nu; i += 2) {
                if (i >= S && !mbar_wait(empty0 + 8 * s, ph ^ 1u, lim, abort_sm)) {
                    fail(abort_sm, P.err);
                    break;
                }
                const uint32_t st = smem_addr(smem + s * STAGE);
                const uint32_t fb = full0 + 8 * s;
                armed[s] = static_cast<int>(ph);
                mbar_arrive_expect_tx(fb, STAGE);
#pragma unroll
                for (int h = 0; h < CH; ++h) tma_load_2d(st + h * NP * 128, &tmB, (kc * CH + h) * TILE, 0, fb);
                tma_load_4d(st + B_BYTES, &tmA, 0, 0, kc * CH, g * T, fb);
                s += 2;
                if (s >= S) {
                    s -= S;
                    ph ^= 1u;
                }
                kc += 2;
                if (kc >= KC) {
                    kc -= KC;
                    ++g;
                }
            }
        }
    } else if (ALT && warp < DEC0) {
        // ------- MMA issuers on alternate stages (whole warp; lane 0 issues) -------
        // Issuer j takes the stages i = j (mod 2) of the CTA's range and issues
        // all T tiles of each into its own accumulators (T NP columns at
        // j T NP), one commit per stage.  Every issuer walks every window (the
        // fold waits for both), zeroing its accumulators with its first MMA in
        // the window; an issuer without a stage in a window commits nothing
        // into it, and the fold then skips its accumulators.
        const int j = warp - 2;
        constexpr uint32_t idesc = idesc_e4m3_f32(128, NP);
        const uint32_t dacc = tbase + static_cast<uint32_t>(j * T * NP);
        const uint64_t desc0 = smem_desc_sw128(smem_addr(smem));
        int s = 0, r = 0, kc = kc0, nb = 0;
        uint64_t dstage = desc0;
        const uint32_t aslot0 = tbase + static_cast<uint32_t>(ACC_COLS);
        uint32_t aslot = aslot0;
        uint32_t eph = 0;
        bool ok = true;
        for (int64_t i = 0, wi = 0; i < nu; ++wi) {
            const int wl = static_cast<int>(min(static_cast<int64_t>(min(F, KC - kc)), nu - i));
            if (wi >= 1) {
                if (ok && !warp_wait(acce, eph, lim, abort_sm)) {
                    ok = false;
                    if (lane == 0) fail(abort_sm, P.err);
                }
                eph ^= 1u;
            }
            bool first = true;
            for (int e = 0; e < wl; ++e) {
                if (((i + e) & 1) == j) {
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        __syncwarp();
                        named_sync(1 + nb * T + t, NB_COUNT);
                        if (ok && lane == 0) {
                            tc_fence_after();
#pragma unroll
                            for (int q = 0; q < 4 * CH; ++q) {
                                const uint64_t bd =
                                    dstage + static_cast<uint64_t>(((q >> 2) * NP * 128 + (q & 3) * 32) >> 4);
                                mma_ts_f8(dacc + static_cast<uint32_t>(t * NP),
                                          aslot + static_cast<uint32_t>(t * CH * 32 + 8 * q), bd, idesc,
                                          (first && q == 0) ? 0u : 1u);
                            }
                        }
                    }
                    if (ok && lane == 0) mma_commit(aempty0 + 8 * r);
                    first = false;
                }
                if (++s == S) {
                    s = 0;
                    dstage = desc0;
                } else {
                    dstage += static_cast<uint64_t>(STAGE >> 4);
                }
                if (++r == R) {
                    r = 0;
                    aslot = aslot0;
                } else {
                    aslot += SLOT_COLS;
                }
                if (++nb == PB) nb = 0;
            }
            i += wl;
            kc += wl;
            if (kc == KC) kc = 0;
            if (ok && lane == 0) mma_commit(accf);
        }
        __syncwarp();
        if (lane == 0) {
            mma_commit(drainb);
            mbar_wait(drainb, 0, DRAIN_LIMIT, &g_never_set);
        }
    } else if (warp < DEC0) {
        // ------- MMA issuers, one per row tile (whole warp; lane 0 issues) -------
        const int t = warp - 2;
        constexpr uint32_t idesc = idesc_e4m3_f32(128, NP);
        const uint32_t d = tbase + static_cast<uint32_t>(t * NP);
        const uint64_t desc0 = smem_desc_sw128(smem_addr(smem));
        // The issuer is the critical thread of the pipeline: per stage it only
        // waits, issues and commits.  Windows (at most F stages, never across
        // a segment end) are sized once when they start.
        const int bid_wrap = PB * T;
        int s = 0, r = 0, kc = kc0, bid = t;  // bid: named barrier id - 1
        uint64_t dstage = desc0;
        uint32_t aslot = tbase + static_cast<uint32_t>(ACC_COLS + t * CH * 32);
        const uint32_t aslot0 = aslot;
        uint32_t eph = 0;
        bool ok = true;
        for (int64_t i = 0, wi = 0; i < nu; ++wi) {
            const int wl = static_cast<int>(min(static_cast<int64_t>(min(F, KC - kc)), nu - i));
            if (wi >= 1) {
                // the accumulator is reused once group 0 has added up the previous window
                if (ok && !warp_wait(acce, eph, lim, abort_sm)) {
                    ok = false;
                    if (lane == 0) fail(abort_sm, P.err);
                }
                eph ^= 1u;
            }
            int pend = -1;  // pair mode: the slot of the stage whose commit waits for the next stage
            for (int e = 0; e < wl; ++e) {
                __syncwarp();
                named_sync(1 + bid, NB_COUNT);
                if (ok && lane == 0) {
                    tc_fence_after();
#pragma unroll
                    for (int q = 0; q < 4 * CH; ++q) {
                        // K = 32 per MMA: 32 bytes of every row of chunk panel q/4, 8 TMEM columns of A
                        const uint64_t bd = dstage + static_cast<uint64_t>(((q >> 2) * NP * 128 + (q & 3) * 32) >> 4);
                        mma_ts_f8(d, aslot + 8 * q, bd, idesc, (e == 0 && q == 0) ? 0u : 1u);
                    }
                    // a commit arrives once all earlier MMAs of this thread are
                    // complete: after every second stage one pair of commits
                    // releases both stages' slots (each slot use still gets one
                    // arrival per issuer, only later)
                    if (!P.pair) {
                        mma_commit(aempty0 + 8 * r);
                    } else if (pend >= 0) {
                        mma_commit(aempty0 + 8 * pend);
                        mma_commit(aempty0 + 8 * r);
                        pend = -1;
                    } else if (e == wl - 1) {
                        mma_commit(aempty0 + 8 * r);
                    } else {
                        pend = r;
                    }
                }
                if (++s == S) {
                    s = 0;
                    dstage = desc0;
                } else {
                    dstage += static_cast<uint64_t>(STAGE >> 4);
                }
                if (++r == R) {
                    r = 0;
                    aslot = aslot0;
                } else {
                    aslot += SLOT_COLS;
                }
                bid += T;
                if (bid >= bid_wrap) bid -= bid_wrap;
            }
            i += wl;
            kc += wl;
            if (kc == KC) kc = 0;
            if (ok && lane == 0) mma_commit(accf);
        }
        __syncwarp();
        if (lane == 0) {
            mma_commit(drainb);
            mbar_wait(drainb, 0, DRAIN_LIMIT, &g_never_set);
        }
    } else {
        // ---------------- decoders (group gamma), folds and epilogue (group 0) ----------------
        const int dw = warp - DEC0;
        const int gamma = dw >> 2;        // decoder group
        const int q = warp & 3;           // TMEM lane quarter
        const int rit = 32 * q + lane;    // row inside a 128-row tile
        const int swp = (rit >> 2) & 1;   // row halves stored swapped
        const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * q) << 16);
        // group 0's running sums of the windows, in shared memory ([column][thread]):
        // registers are the scarce resource of the decoders
        float *accs = reinterpret_cast<float *>(smem + S * STAGE + 1024) + (threadIdx.x - 32 * DEC0);
        auto acc = [&](int tt, int e) -> float & { return accs[(tt * KH + e) * 128]; };
        // per-column constants, loaded once: sum V, step lambda, active (fused
        // step) and the power-of-two scale of the B limbs
        float *colc = reinterpret_cast<float *>(smem + S * STAGE + 1024) + T * KH * 128;
        if (gamma == 0) {
            for (int e = 0; e < T * KH; ++e) accs[e * 128] = 0.f;
            const int tid = threadIdx.x - 32 * DEC0;
            if (tid < P.k) {
                reinterpret_cast<int *>(colc + 3 * KH)[tid] = P.bscale[tid];
                if (P.epi != EPI_PARTIAL) {
                    colc[tid] = static_cast<float>(P.sumV[tid]);
                    if (P.epi == EPI_PROX) {
                        colc[KH + tid] = static_cast<float>(P.step * P.lam[tid]);
                        colc[2 * KH + tid] = (P.active && !P.active[tid]) ? 0.f : 1.f;
                    }
                }
            }
        }
        uint32_t epi_phase = 0, fold_phase = 0;
        bool ok = true;

        // group 0: add the finished window's accumulators into registers; at a
        // segment end write this CTA's partial of group g and, for the last
        // CTA, apply the epilogue.
        // amask (alternating issuers): bit j set when issuer j wrote its
        // accumulators in this window
        auto fold = [&](bool segend, int g, int amask) {
            if (!ok) return;
            if (!warp_wait(accf, fold_phase, lim, abort_sm)) {
                ok = false;
                return;
            }
            fold_phase ^= 1u;
            tc_fence_after();
            {
#pragma unroll
                for (int tt = 0; tt < T; ++tt) {
#pragma unroll
                    for (int cc = 0; cc < NP / 8; ++cc) {
                        float v[8];
                        if (!ALT) {
                            uint32_t u[8];
                            tmem_ld_32x32b_x8(lane_base + static_cast<uint32_t>(tt * NP + cc * 8), u);
                            tmem_wait_ld();
#pragma unroll
                            for (int m = 0; m < 8; ++m) v[m] = __uint_as_float(u[m]);
                        } else {
#pragma unroll
                            for (int m = 0; m < 8; ++m) v[m] = 0.f;
#pragma unroll
                            for (int jj = 0; jj < 2; ++jj) {
                                if (!(amask >> jj & 1)) continue;  // warp-uniform
                                uint32_t u[8];
                                tmem_ld_32x32b_x8(lane_base + static_cast<uint32_t>((jj * T + tt) * NP + cc * 8), u);
                                tmem_wait_ld();
#pragma unroll
                                for (int m = 0; m < 8; ++m) v[m] += __uint_as_float(u[m]);
                            }
                        }
#pragma unroll
                        for (int e = 0; e < 2; ++e) {  // two lambda columns of four limbs
                            float x = v[4 * e + 3];
                            x = fmaf(x, 0.0625f, v[4 * e + 2]);
                            x = fmaf(x, 0.0625f, v[4 * e + 1]);
                            x = fmaf(x, 0.0625f, v[4 * e]);
                            acc(tt, cc * 2 + e) += x;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce);
            if (!segend) return;

            const int64_t first_cta = (static_cast<int64_t>(g) * KC) / P.L;
            const int64_t last_cta = (static_cast<int64_t>(g) * KC + KC - 1) / P.L;
            const int *bsc = reinterpret_cast<const int *>(colc + 3 * KH);
            if (P.epi != EPI_PARTIAL && first_cta == last_cta) {
                // the whole group ran in this CTA: apply the step straight from the
                // sums (the same values the one partial slot would carry)
                const float inv_n = static_cast<float>(P.inv_n), stepf = static_cast<float>(P.step);
                // all loads of a tile (mu and a batch of up to 16 coefficients) are
                // issued before any arithmetic, one round trip per tile and batch
                constexpr int EB = KH < 16 ? KH : 16;
#pragma unroll
                for (int tt = 0; tt < T; ++tt) {
                    const int64_t row = (static_cast<int64_t>(g) * T + tt) * TILE + rit;
                    const bool valid = row < P.rows_valid;
                    const double mud = valid ? P.mu[row] : 0.0;
                    for (int e0 = 0; e0 < P.k; e0 += EB) {
                        float bv[EB];
#pragma unroll
                        for (int u = 0; u < EB; ++u) {
                            const int e = min(e0 + u, P.k - 1);
                            bv[u] = (P.epi == EPI_PROX && valid) ? P.beta[static_cast<int64_t>(e) * P.rows_valid + row] : 0.f;
                        }
                        const float muv = static_cast<float>(mud);
#pragma unroll
                        for (int u = 0; u < EB; ++u) {
                            const int e = e0 + u;
                            if (e >= P.k) break;
                            const float xtv = ldexpf(acc(tt, e), bsc[e] + 9);  // (X^T V)_j
                            acc(tt, e) = 0.f;
                            if (!valid) continue;
                            const float gv = (xtv - muv * colc[e]) * inv_n;
                            const int64_t bi = static_cast<int64_t>(e) * P.rows_valid + row;
                            if (P.epi == EPI_PROX) {
                                if (colc[2 * KH + e] == 0.f) continue;  // converged column: frozen
                                const float thr = colc[KH + e];
                                const float z = fmaf(stepf, gv, bv[u]);
                                P.beta[bi] = z > thr ? z - thr : (z < -thr ? z + thr : 0.f);
                                if (P.near && fabsf(z) > 0.75f * thr) P.near[row] = 1;
                            } else {
                                P.grad[bi] = -gv;
                            }
                        }
                    }
                    for (int e = P.k; e < KH; ++e) acc(tt, e) = 0.f;
                }
                return;
            }
            const int64_t slot = cta - first_cta;
#pragma unroll
            for (int tt = 0; tt < T; ++tt) {
                const int64_t row = (static_cast<int64_t>(g) * T + tt) * TILE + rit;
#pragma unroll
                for (int e = 0; e < KH; ++e) {
                    if (e < P.k) P.part[slot * P.slot_stride + e * P.rows_pad + row] = ldexpf(acc(tt, e), bsc[e] + 9);
                    acc(tt, e) = 0.f;
                }
            }
            if (P.epi == EPI_PARTIAL) return;
            // the last CTA of the group applies the step (Section 5.3: beta <- S(beta + sigma g, sigma lambda))
            __threadfence();
            __syncwarp();
            if (lane == 0) mbar_arrive(epib);
            if (!warp_wait(epib, epi_phase, lim, abort_sm)) {
                ok = false;
                return;
            }
            epi_phase ^= 1u;
            const int cnt = static_cast<int>(last_cta - first_cta + 1);
            if (threadIdx.x == 32 * DEC0) {
                const int old = atomicAdd(&P.counters[g], 1);
                const int is_last = (old == cnt - 1);
                if (is_last) P.counters[g] = 0;
                *last_sm = is_last;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(epib);
            if (!warp_wait(epib, epi_phase, lim, abort_sm)) {
                ok = false;
                return;
            }
            epi_phase ^= 1u;
            if (!*last_sm) return;
            __threadfence();
            // Each thread owns rows tid, tid + 128, ... of the group and walks the
            // lambda columns; the loads of different columns are independent
            // (restrict pointers), so they overlap.  FP32 arithmetic: the
            // partials are FP32 and beta is stored in FP32.
            const int tid = threadIdx.x - 32 * DEC0;
            constexpr int RPT = T * TILE / 128;  // rows per thread
            const float *__restrict__ part = P.part;
            float *__restrict__ beta = P.beta;
            float *__restrict__ grad = P.grad;
            const float inv_n = static_cast<float>(P.inv_n), stepf = static_cast<float>(P.step);
            int64_t rows[RPT];
            float muv[RPT];
#pragma unroll
            for (int rr = 0; rr < RPT; ++rr) {
                rows[rr] = static_cast<int64_t>(g) * (T * TILE) + rr * 128 + tid;
                muv[rr] = rows[rr] < P.rows_valid ? static_cast<float>(P.mu[rows[rr]]) : 0.f;
            }
            // batches of KB columns: all loads of a batch are issued before any
            // arithmetic, so their L2 latencies overlap
            constexpr int KB = 4;
            const int64_t ss = P.slot_stride;
            for (int k0 = 0; k0 < P.k; k0 += KB) {
                float gs[KB][RPT], bv[KB][RPT];
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int kk = min(k0 + u, P.k - 1);
#pragma unroll
                    for (int rr = 0; rr < RPT; ++rr) {
                        const int64_t row = rows[rr] < P.rows_valid ? rows[rr] : 0;
                        const float *pp = part + kk * P.rows_pad + row;
                        float g = __ldcg(pp);
                        if (cnt > 1) g += __ldcg(pp + ss);
                        for (int s2 = 2; s2 < cnt; ++s2) g += __ldcg(pp + s2 * ss);
                        gs[u][rr] = g;
                        bv[u][rr] = P.epi == EPI_PROX ? beta[static_cast<int64_t>(kk) * P.rows_valid + row] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int kk = k0 + u;
                    if (kk >= P.k) break;
                    const float sv = colc[kk];
#pragma unroll
                    for (int rr = 0; rr < RPT; ++rr) {
                        const int64_t row = rows[rr];
                        if (row >= P.rows_valid) continue;
                        const float gv = (gs[u][rr] - muv[rr] * sv) * inv_n;
                        const int64_t bi = static_cast<int64_t>(kk) * P.rows_valid + row;
                        if (P.epi == EPI_PROX) {
                            if (colc[2 * KH + kk] == 0.f) continue;  // converged column: frozen
                            const float thr = colc[KH + kk];
                            const float z = fmaf(stepf, gv, bv[u][rr]);
                            beta[bi] = z > thr ? z - thr : (z < -thr ? z + thr : 0.f);
                            if (P.near && fabsf(z) > 0.75f * thr) P.near[row] = 1;
                        } else {
                            grad[bi] = -gv;
                        }
                    }
                }
            }
        };

        // window bookkeeping (group 0): walk every stage in order and fold each
        // window as soon as its last stage lies behind the stage being decoded
        int wkc = kc0, wg = g0, wlen = 0;
        int64_t wnext = 0;
        auto fold_until = [&](int64_t upto) {  // stages [wnext, upto)
            for (; wnext < upto && wnext < nu && ok; ++wnext) {
                if (wnext == 0 || wkc == 0 || wlen == F) wlen = 0;
                ++wlen;
                const bool seg = (wnext == nu - 1) || (wkc == KC - 1);
                // issuers with a stage in the window [wnext - wlen + 1, wnext]
                const int amask = wlen >= 2 ? 3 : 1 << static_cast<int>(wnext & 1);
                if (seg || wlen == F) fold(seg, wg, amask);
                if (++wkc == KC) {
                    wkc = 0;
                    ++wg;
                }
            }
        };

        int s = gamma % S, r = gamma % R, nbid = gamma % PB;
        uint32_t fph = static_cast<uint32_t>((gamma / S) & 1), aph = static_cast<uint32_t>((gamma / R) & 1);
        for (int64_t i = gamma; i < nu; i += G) {
            bool go = ok;
            if (go && gamma == 0) {
                // windows ending before stage i: every stage of theirs is decoded
                // or owned by another group, so their MMAs complete without us
                fold_until(i);
                go = ok;
            }
            if (go && !warp_wait(full0 + 8 * s, fph, lim, abort_sm)) go = false;
            // TMEM slot r is free once the MMAs of stage i - R are complete
            if (go && i >= R && !warp_wait(aempty0 + 8 * r, aph ^ 1u, lim, abort_sm)) go = false;
            if (go) {
                if (i >= R && q == (DEC0 & 3) && lane == 0) {
                    int se = s - R;
                    if (se < 0) se += S;
                    mbar_arrive(empty0 + 8 * se);
                }
                tc_fence_after();
                const uint8_t *xs = smem + s * STAGE + B_BYTES + rit * 32;
                const uint32_t acol = lane_base + static_cast<uint32_t>(ACC_COLS + r * SLOT_COLS);
#pragma unroll 2
                for (int tc = 0; tc < T * CH; ++tc) {  // tile tc / CH, chunk tc % CH
                    uint32_t o[32];
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(xs + tc * BLOCK_BYTES + 16 * (hh ^ swp));
                        decode16(v.x, o + 16 * hh);
                        decode16(v.y, o + 16 * hh + 4);
                        decode16(v.z, o + 16 * hh + 8);
                        decode16(v.w, o + 16 * hh + 12);
                    }
                    tmem_st_32x32b_x32(acol + tc * 32, o);
                    if (tc % CH == CH - 1) {
                        // tile tc / CH is written: hand it to its issuer
                        tmem_wait_st();
                        tc_fence_before();
                        __syncwarp();
                        named_arrive(1 + nbid * T + tc / CH, NB_COUNT);
                    }
                }
            } else {
                // nothing written (error path): still arrive, so no issuer waits forever
                __syncwarp();
#pragma unroll
                for (int tt = 0; tt < T; ++tt) named_arrive(1 + nbid * T + tt, NB_COUNT);
            }
            if (!go && ok) {
                ok = false;
                if (lane == 0) fail(abort_sm, P.err);
            }
            s += G;
            if (s >= S) {
                s -= S;
                fph ^= 1u;
            }
            r += G;
            while (r >= R) {
                r -= R;
                aph ^= 1u;
            }
            nbid += G;
            if (nbid >= PB) nbid -= PB;
        }
        if (gamma == 0 && ok) fold_until(nu);
        if (!ok && lane == 0) fail(abort_sm, P.err);
    }

    // Lane 0 of the producer and issuer warps may still be loading or draining
    // while lanes 1..31 are already here: reconverge every warp before the
    // CTA-wide (warp-aligned) barrier that precedes the TMEM release.
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        // never leave a copy in flight into shared memory we are about to give
        // up (after an abort, stages may have been loaded that nobody waited for)
        if (lane == 0)
            for (int s = 0; s < S; ++s)
                if (armed[s] >= 0) mbar_wait(full0 + 8 * s, static_cast<uint32_t>(armed[s]), DRAIN_LIMIT, &g_never_set);
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// beta (p x k fp32, column-major) -> e4m3 limbs [NP][p_pad] with one
// power-of-two scale per column (from the max |beta| partials of k_l1_32).
__global__ void k_prep_limbs_beta(const float *__restrict__ beta, int64_t p, int64_t p_pad, int nb,
                                  const float *__restrict__ maxp, uint8_t *__restrict__ Bq,
                                  int *__restrict__ bs, int *err)
{
    __shared__ int s_sh;
    const int kk = blockIdx.y;
    if (threadIdx.x < 32) {
        float m = 0.f;
        for (int b = threadIdx.x; b < nb; b += 32) m = fmaxf(m, maxp[kk * nb + b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) {
            if (!isfinite(m)) {
                atomicOr(err, DEVERR_NONFINITE);
                m = 0.f;
            }
            s_sh = limb_scale(m);
            if (blockIdx.x == 0) bs[kk] = s_sh;
        }
    }
    __syncthreads();
    const int s = s_sh;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < p;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint8_t d[LIMBS];
        split_e4m3(ldexpf(beta[static_cast<int64_t>(kk) * p + j], -s), d);
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) Bq[(LIMBS * kk + l) * p_pad + j] = d[l];
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

using KernelFn = void (*)(const CUtensorMap, const CUtensorMap, const KParams);

// (T row tiles, CH K chunks) per stage for a limb-column class NP.  One issuer
// per tile leaves the most TMEM to the A slot ring (a second issuer per tile
// needs a second accumulator).  N = 256 fills half of TMEM per accumulator,
// so that class takes one tile per stage.
// A stage spans CH K chunks: every hand-off costs a few hundred cycles
// whatever its size, so up to N = 64 a stage takes two chunks (16 KB of codes
// at T = 2), which keeps the same bytes in TMEM with half the hand-offs.
// This is the default; the autotuner times every compiled shape instead.
void shape_for(int NP, int *T, int *CH, int *alt)
{
    *T = NP <= 128 ? 2 : 1;
    *CH = NP <= 64 ? 2 : 1;
    *alt = 0;
}

constexpr int G_ALT = 2;   // decoder groups of the alternating-issuer kernels
constexpr int G_WIDE = 2;  // decoder groups of the 2 x 2 shape at 128 limb columns and 2 x 3 at 64

KernelFn pick_kernel(int T, int CH, int NP, int alt)
{
    switch (((alt ? 100 : 0) + T * 10 + CH) * 1000 + NP) {
    case 22016: return k_packed_gemm<2, 2, 16, DEC_GROUPS, false>;
    case 21016: return k_packed_gemm<2, 1, 16, DEC_GROUPS, false>;
    case 12016: return k_packed_gemm<1, 2, 16, DEC_GROUPS, false>;
    case 22032: return k_packed_gemm<2, 2, 32, DEC_GROUPS, false>;
    case 21032: return k_packed_gemm<2, 1, 32, DEC_GROUPS, false>;
    case 12032: return k_packed_gemm<1, 2, 32, DEC_GROUPS, false>;
    case 22064: return k_packed_gemm<2, 2, 64, DEC_GROUPS, false>;
    case 21064: return k_packed_gemm<2, 1, 64, DEC_GROUPS, false>;
    case 12064: return k_packed_gemm<1, 2, 64, DEC_GROUPS, false>;
    case 21128: return k_packed_gemm<2, 1, 128, DEC_GROUPS, false>;
    case 12128: return k_packed_gemm<1, 2, 128, DEC_GROUPS, false>;
    case 11128: return k_packed_gemm<1, 1, 128, DEC_GROUPS, false>;
    // two decoder groups: 2 tiles x 2 chunks at 128 limb columns, whose two
    // 128-column TMEM slots beside 256 accumulator columns leave no third slot
    case 22128: return k_packed_gemm<2, 2, 128, G_WIDE, false>;
    // two decoder groups: 2 tiles x 3 chunks at 64 limb columns (12 MMAs per
    // commit per issuer; two 192-column slots beside 128 accumulator columns)
    case 23064: return k_packed_gemm<2, 3, 64, G_WIDE, false>;
    case 11256: return k_packed_gemm<1, 1, 256, DEC_GROUPS, false>;
    // alternating issuers: 16 MMAs per commit up to N = 64, 8 at N = 128
    case 122016: return k_packed_gemm<2, 2, 16, G_ALT, true>;
    case 122032: return k_packed_gemm<2, 2, 32, G_ALT, true>;
    case 122064: return k_packed_gemm<2, 2, 64, G_ALT, true>;
    case 112128: return k_packed_gemm<1, 2, 128, G_ALT, true>;
    default: return nullptr;
    }
}

int groups_for(int T, int CH, int NP, int alt)
{
    if (alt) return G_ALT;
    return ((T == 2 && CH == 2 && NP == 128) || (T == 2 && CH == 3 && NP == 64)) ? G_WIDE : DEC_GROUPS;
}
int issuers_for(int T, int alt) { return alt ? 2 : T; }
int threads_for(int T, int G, int alt) { return 32 * (2 + issuers_for(T, alt) + 4 * G); }

int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }

// The conditions under which every parity wait of k_packed_gemm is
// unambiguous, for G decoder groups, R TMEM slots and S shared-memory stages
// (derived with the kernel's hand-off notes).  Alternating issuers need the
// two parity classes apart instead: G = 2 and R, S even.
bool parity_safe(int G, int R, int S, int alt)
{
    if (alt) return G == 2 && R >= 2 && R % 2 == 0 && S % 2 == 0;
    const bool slots = G <= R;                                 // aempty
    const bool stages = S >= G + R || S % G == 0 || R % G == 0; // full
    const bool release = S % 2 == 0 || S >= R + 2;             // empty
    return slots && stages && release;
}
int lcm_i(int a, int b) { return a / gcd_i(a, b) * b; }

} // namespace

int gemm_shapes(int k, int *T, int *CH, int *issue, int max)
{
    const int NP = limb_cols(k);
    int n = 0;
    for (int is = 1; is <= 3; ++is)
        for (int t = 2; t >= 1; --t)
            for (int c = 3; c >= 1; --c)
                if (pick_kernel(t, c, NP, is == 2) && n < max &&
                    !(is == 3 && groups_for(t, c, NP, 0) == G_WIDE)) {
                    T[n] = t;
                    CH[n] = c;
                    issue[n] = is;
                    ++n;
                }
    return n;
}

// Plan one product: A (rows_pad x K_pad, tiled 2-bit) times B limbs (NP x K_pad).
// TMEM budget (512 columns): the accumulators (T of NP columns, twice that with
// alternating issuers) + ring x T CH x 32 A columns.
int plan_shape(GemmPlan &g, int k, int T_req, int CH_req, int stages_req, int issue_req)
{
    if (k < 1 || k > MAX_K_TC) return COX_ERR_ARG;
    if (issue_req < 0 || issue_req > 3) return COX_ERR_ARG;
    const int np_cls = limb_cols(k);
    int T = 2, CH = 1, alt = 0;
    shape_for(np_cls, &T, &CH, &alt);
    if (issue_req > 0) alt = issue_req == 2;
    if (T_req > 0) T = T_req;
    if (CH_req > 0) CH = CH_req;
    if (!pick_kernel(T, CH, np_cls, alt)) return COX_ERR_ARG;  // shape not compiled for this class
    const int G = groups_for(T, CH, np_cls, alt);
    if (G == G_WIDE && !alt && issue_req == 3) return COX_ERR_ARG;  // pair commits: not planned for it
    const int stage = CH * (np_cls * 128 + T * BLOCK_BYTES);
    // group 0's window sums, then four per-column constants
    const int fold_bytes = T * (np_cls / LIMBS) * 128 * 4 + 4 * (np_cls / LIMBS) * 4;
    int S = stages_req > 0 ? stages_req : (225 * 1024 - 2048 - fold_bytes) / stage;
    if (S > 12) S = 12;
    if (alt && stages_req <= 0 && S % 2) --S;  // the parity classes need an even stage ring
    if (S < G + 1) S = G + 1;  // decoder groups step through the stage ring by G
    // TMEM: the accumulators, the rest A slots of T CH x 32 columns;
    // the decoders of stage i free the shared memory of stage i - ring, which
    // the producer needs for stage i - ring + S: ring < S, or the producer of
    // stage i would wait for the decoders of stage i, who wait for it; and
    // the named barriers, one per tile for each stage of the period
    // lcm(G, ring), must fit barriers 1..15
    const int acc_cols = (alt ? 2 * T : T) * np_cls;
    const int ring_max = std::min(8, (512 - acc_cols) / (T * CH * 32));
    // Parity waits need the phase before the awaited one complete; the
    // kernel's hand-off notes derive when the pipeline guarantees that.  With
    // the default depth, one stage more is tried when the rule holds for no
    // ring at the budget's depth and the deeper ring still fits 227 KB (the
    // two-group shape: three stages allow no safe ring of two, four do).
    int ring = 0;
    for (int pass = 0; pass < 2; ++pass) {
        ring = std::min(ring_max, S - 1);
        while (ring >= G && !(lcm_i(G, ring) * T <= 15 && parity_safe(G, ring, S, alt))) --ring;
        if (ring >= G || stages_req > 0 || S >= 12 ||
            static_cast<size_t>(S + 1) * stage + 1024 + 1024 + fold_bytes > 227 * 1024)
            break;
        ++S;
    }
    if (ring < G) return COX_ERR_ARG;
    g.T = T;
    g.CH = CH;
    g.NP = np_cls;
    g.alt = alt;
    g.pair = issue_req == 3;
    g.G = G;
    g.ring = ring;
    g.nb_period = lcm_i(G, ring);
    g.stages = S;
    g.smem = static_cast<size_t>(S) * stage + 1024 + 1024 + fold_bytes;
    if (g.smem < 120 * 1024) g.smem = 120 * 1024;  // one CTA per SM: it owns all 512 TMEM columns
    if (g.smem > 227 * 1024) return COX_ERR_ARG;    // too many stages requested
    return COX_OK;
}

int plan_gemm(cox_handle *h, GemmPlan &g, const uint32_t *A, int64_t rows_pad, int64_t K_pad,
              const uint8_t *B, int k, int T_req, int CH_req, int stages_req, int issue_req)
{
    COX_TRY(plan_shape(g, k, T_req, CH_req, stages_req, issue_req));
    const int64_t m_tiles = rows_pad / TILE;
    const int T = g.T, CH = g.CH, np_cls = g.NP;
    if (m_tiles % T != 0 || (K_pad / TILE) % CH != 0) return COX_ERR_ARG;
    // stages per accumulation window (default 256 K chunks, 1024 MMAs per accumulator)
    const int win = h->opt.window > 0 ? h->opt.window : 256;
    g.F = std::max(1, win / CH);
    g.KC = static_cast<int>(K_pad / (TILE * CH));  // stages per group
    g.n_groups = static_cast<int>(m_tiles / T);
    g.units = static_cast<int64_t>(g.n_groups) * g.KC;
    int grid = h->sm_count;
    if (g.units < grid) grid = static_cast<int>(g.units);
    g.L = (g.units + grid - 1) / grid;
    g.grid = static_cast<int>((g.units + g.L - 1) / g.L);
    int ms = 1;
    for (int64_t gg = 0; gg < g.n_groups; ++gg) {
        const int64_t fc = (gg * g.KC) / g.L, lc = (gg * g.KC + g.KC - 1) / g.L;
        if (lc - fc + 1 > ms) ms = static_cast<int>(lc - fc + 1);
    }
    g.max_slots = ms;
    g.rows_pad = rows_pad;
    {
        // the two products (and the autotuner's candidates) share kernels with
        // different depths: allow the device's largest block allocation once,
        // and let each launch ask for its own size
        KernelFn fn = pick_kernel(g.T, g.CH, g.NP, g.alt);
        if (!fn) return COX_ERR_ARG;
        int optin = 0;
        COX_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
        if (static_cast<size_t>(optin) < g.smem) return COX_ERR_ARG;
        COX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    }

    EncodeTiled enc = get_encoder();
    if (!enc) return COX_ERR_CUDA;
    {
        // a 4 KB block viewed as 4 rows of 1 KB; CH consecutive chunks of T
        // consecutive row tiles per box
        const cuuint64_t kch = static_cast<cuuint64_t>(K_pad / TILE);
        cuuint64_t dims[4] = {256, 4, kch, static_cast<cuuint64_t>(m_tiles)};
        cuuint64_t strides[3] = {1024, BLOCK_BYTES, kch * BLOCK_BYTES};
        cuuint32_t box[4] = {256, 4, static_cast<cuuint32_t>(CH), static_cast<cuuint32_t>(T)};
        cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = enc(&g.tmA, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<uint32_t *>(A), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return COX_ERR_CUDA;
    }
    {
        // one 128-byte row (a K chunk of one limb column) per limb column
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(K_pad), static_cast<cuuint64_t>(np_cls)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(K_pad)};
        cuuint32_t box[2] = {128, static_cast<cuuint32_t>(np_cls)};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(&g.tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(B), dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return COX_ERR_CUDA;
    }
    return COX_OK;
}

int launch_gemm(cox_handle *h, const GemmPlan &g, const EpiArgs &e, int k, cudaStream_t st)
{
    KParams kp;
    kp.KC = g.KC;
    kp.F = g.F;
    kp.k = k;
    kp.stages = g.stages;
    kp.ring = g.ring;
    kp.nb_period = g.nb_period;
    kp.pair = g.pair;
    kp.bscale = e.bscale;
    kp.units = g.units;
    kp.L = g.L;
    kp.rows_pad = g.rows_pad;
    kp.slot_stride = static_cast<int64_t>(k) * g.rows_pad;
    kp.part = e.part;
    kp.epi = e.epi;
    kp.counters = e.counters;
    kp.beta = e.beta;
    kp.grad = e.grad;
    kp.lam = e.lam;
    kp.step = e.step;
    kp.mu = e.mu;
    kp.sumV = e.sumV;
    kp.active = e.active;
    kp.near = e.near;
    kp.rows_valid = e.rows_valid;
    kp.inv_n = e.inv_n;
    kp.wait_limit = h->wait_cycles;
    kp.err = h->d_err;
    KernelFn fn = pick_kernel(g.T, g.CH, g.NP, g.alt);
    if (!fn) return COX_ERR_ARG;
    fn<<<g.grid, threads_for(g.T, g.G, g.alt), g.smem, st>>>(g.tmA, g.tmB, kp);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

int prep_limbs_beta(cox_handle *h, const float *beta, int k, cudaStream_t st)
{
    // about four blocks per SM over all columns; each block strides over p
    const int64_t bx = std::max<int64_t>(1, (4 * static_cast<int64_t>(h->sm_count) + k - 1) / k);
    dim3 grid(static_cast<unsigned>(std::min<int64_t>((h->p + 255) / 256, bx)), k);
    k_prep_limbs_beta<<<grid, 256, 0, st>>>(beta, h->p, h->p_pad, h->l1_blocks, h->ws.bmaxp, h->ws.Bq,
                                            h->ws.bs1, h->d_err);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

} // namespace coxgb
