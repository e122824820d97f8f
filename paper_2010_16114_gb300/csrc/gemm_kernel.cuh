// gemm_kernel.cuh -- the tensor-core kernel of the two genotype products of the
// Cox iteration, shared by the translation units that instantiate its shapes
// (gemm_tc.cu: e4m3 operands, gemm_f4.cu: e2m1 operands).
//
// The products (arXiv 2010.16114, Section 5.3: X beta, and Delta = X^T (I-P) delta):
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
// The e2m1 form (F4 = true; kind::mxf4, K = 64 per MMA): a code c is the e2m1
// nibble c << 1 (value c, exact), two codes per byte, so one MMA instruction
// covers twice the K of an e4m3 one at the same issue cost and a K chunk
// takes 16 TMEM columns per lane instead of 32.  decode16_e2m1 turns a packed
// word into two TMEM words with one shift and one AND each; the limb rows hold
// their K positions in the same order (e2m1_byte).  Coefficients are LIMBS4 = 8
// e2m1 limbs on the grid of halves (r_0 = b 2^-s in [-2, 2), d_l = RN(2 r_l)/2,
// r_(l+1) = 8 (r_l - d_l)), b = 2^s sum_l d_l 8^-l to within 2^-23 of the
// column's largest |b|; the fold weights are 8^-l and the scale 2^s.  The
// block scales are all 1 (ue8m0 127 in every byte of TMEM columns SF_COL ..
// SF_COL + 7, written once per launch), so the scale-factor layout never
// matters.  A limb panel of 128-byte rows covers two K chunks, so the e2m1
// stages hold an even number of chunks.
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
#pragma once
#include <algorithm>

#include "internal.h"
#include "ptx.cuh"

namespace coxgb {

struct KParams {
    int KC, F, k, stages, ring, nb_period;
    int stages2;        // e2m1 form: depth of the limb ring (stages is the code ring's)
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


using GemmKernelFn = void (*)(const CUtensorMap, const CUtensorMap, const KParams);

// The e2m1 shapes (gemm_f4.cu); null when (T, CH, NP) is not compiled.
GemmKernelFn pick_kernel_f4(int T, int CH, int NP);

namespace {

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

// 16 codes of a packed word -> 16 e2m1 nibbles (two TMEM columns): nibble m
// of o[h] is code K = 4h + (m >> 1) + 8 (m & 1) of the word shifted left by
// one (e2m1 0b0010 = 1, 0b0100 = 2), the order of e2m1_pos()
__device__ __forceinline__ void decode16_e2m1(uint32_t P, uint32_t *o)
{
    o[0] = (P << 1) & 0x66666666u;
    o[1] = (P >> 1) & 0x66666666u;
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
template <int T, int CH, int NP, int G, bool ALT, bool F4>
__global__ void __launch_bounds__(32 * (2 + (ALT ? 2 : T) + 4 * G), 1)
    k_packed_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const KParams P)
{
    constexpr int I = ALT ? 2 : T;        // MMA issuers: one per row tile, or two on alternate stages
    static_assert(!ALT || G == 2, "alternating issuers pair with two decoder groups");
    static_assert(!F4 || (!ALT && CH % 2 == 0 && NP % 8 == 0 && LIMBS4 == 8),
                  "e2m1 operands: per-tile issuers, chunk pairs, one coefficient per 8 columns");
    constexpr int NL = F4 ? LIMBS4 : LIMBS;  // limbs per coefficient column
    constexpr int KH = NP / NL;           // lambda columns a decoder thread folds (>= k)
    // B: one panel of NP rows x 128 bytes per K chunk (e4m3), or per two K
    // chunks (e2m1, two values per byte)
    constexpr int B_BYTES = (F4 ? CH / 2 : CH) * NP * 128;
    constexpr int X_BYTES = T * CH * BLOCK_BYTES;  // [tile][chunk] 4 KB blocks
    constexpr int STAGE = B_BYTES + X_BYTES;
    constexpr int ACC_COLS = (ALT ? 2 * T : T) * NP;  // accumulators: per tile, or per issuer and tile
    constexpr int CW = F4 ? 16 : 32;      // TMEM columns of 128 A values (one tile and chunk) per lane
    constexpr int SLOT_COLS = T * CH * CW;
    constexpr int MQ = F4 ? 2 * CH : 4 * CH;  // MMAs per tile and stage (K = 64 e2m1, 32 e4m3)
    constexpr int SH = F4 ? 0 : 9;        // code scale: e2m1 codes are c, e4m3 codes c 2^-9
    constexpr int DEC0 = 2 + I;           // first decoder warp
    constexpr int NB_COUNT = 32 * 5;      // a decoder group and the tile's issuer warp

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    const int S = P.stages, R = P.ring, PB = P.nb_period;
    // e2m1 form: two rings, S code slots (released by the decoders once they have
    // read them) and S2 limb slots (released once the stage's MMAs are complete),
    // so the codes, streamed from HBM, are fetched further ahead than the limbs,
    // which come from L2.  e4m3 form: one ring of S stages of limbs and codes.
    const int S2 = F4 ? P.stages2 : S;
    uint8_t *const lring = smem + static_cast<size_t>(S) * X_BYTES;  // e2m1 limb ring
    const size_t ring_bytes = F4 ? static_cast<size_t>(S) * X_BYTES + static_cast<size_t>(S2) * B_BYTES
                                 : static_cast<size_t>(S) * STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + ring_bytes);
    const uint32_t full0 = smem_addr(bars);
    const uint32_t empty0 = full0 + 8 * S;
    const uint32_t aempty0 = empty0 + 8 * S;
    const uint32_t accf = aempty0 + 8 * R;
    const uint32_t acce = accf + 8;
    const uint32_t drainb = acce + 8;
    const uint32_t epib = drainb + 8;
    const uint32_t lfull0 = epib + 8;          // e2m1: limb slots loaded
    const uint32_t lempty0 = lfull0 + 8 * S2;  // e2m1: limb slots free
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + R + 4 + (F4 ? 2 * S2 : 0));
    volatile int *abort_sm = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *last_sm = reinterpret_cast<volatile int *>(tmem_slot + 2);
    volatile int *armed = reinterpret_cast<volatile int *>(tmem_slot + 4);  // [S] parity of the last TMA into a slot
    volatile int *armed2 = armed + S;                                      // [S2] the same for the limb slots

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, F4 ? 4 : 1);  // e2m1: each warp of the decoding group
            armed[s] = -1;
        }
        if (F4)
            for (int s = 0; s < S2; ++s) {
                mbar_init(lfull0 + 8 * s, 1);
                mbar_init(lempty0 + 8 * s, 1);
                armed2[s] = -1;
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
    if (F4) {
        // unit block scales (ue8m0 127 = 2^0) in every byte of the scale-factor
        // columns, written before the first stage is handed to an issuer
        if (warp >= 2 + I && warp < 2 + I + 4) {
            uint32_t one[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) one[c] = 0x7F7F7F7Fu;
            tmem_st_32x32b_x8(tbase + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + SF_COL, one);
            tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    const int64_t cta = blockIdx.x;
    const int64_t u0 = cta * P.L;
    const int64_t u1 = min(u0 + P.L, P.units);
    const int64_t nu = u1 > u0 ? u1 - u0 : 0;
    const int KC = P.KC, F = P.F;
    const long long lim = P.wait_limit;
    // position of the first unit; the loops below advance their counters by
    // increments only (no division on the per-stage path)
    const int g0 = static_cast<int>(u0 / KC), kc0 = static_cast<int>(u0 - static_cast<int64_t>(g0) * KC);

    if (F4 && warp < 2) {
        // ------- TMA producers of the e2m1 form: warp 0 the codes, warp 1 the limbs -------
        // One thread per ring loads every stage in order, each slot only after its
        // release, so the producers' own waits never see an older phase.  The
        // decoders' waits on the full barriers need the ring depths the planner
        // keeps (at least G + R, or a multiple of G: ring_safe).
        if (lane == 0) {
            const bool codes = warp == 0;
            const int SR = codes ? S : S2;
            int s = 0, kc = kc0, g = g0;
            uint32_t ph = 0;
            for (int64_t i = 0; i < nu; ++i) {
                const uint32_t eb = (codes ? empty0 : lempty0) + 8 * s;
                if (i >= SR && !mbar_wait(eb, ph ^ 1u, lim, abort_sm)) {
                    fail(abort_sm, P.err);
                    break;
                }
                if (codes) {
                    const uint32_t fb = full0 + 8 * s;
                    armed[s] = static_cast<int>(ph);
                    mbar_arrive_expect_tx(fb, X_BYTES);
                    tma_load_4d(smem_addr(smem + static_cast<size_t>(s) * X_BYTES), &tmA, 0, 0, kc * CH, g * T, fb);
                } else {
                    const uint32_t fb = lfull0 + 8 * s;
                    const uint32_t st = smem_addr(lring + static_cast<size_t>(s) * B_BYTES);
                    armed2[s] = static_cast<int>(ph);
                    mbar_arrive_expect_tx(fb, B_BYTES);
#pragma unroll
                    for (int h = 0; h < CH / 2; ++h) tma_load_2d(st + h * NP * 128, &tmB, (kc * (CH / 2) + h) * 128, 0, fb);
                }
                if (++s == SR) {
                    s = 0;
                    ph ^= 1u;
                }
                if (++kc == KC) {
                    kc = 0;
                    ++g;
                }
            }
        }
    } else if (warp < 2) {
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
                for (int h = 0; h < (F4 ? CH / 2 : CH); ++h)
                    tma_load_2d(st + h * NP * 128, &tmB, (F4 ? kc * (CH / 2) + h : kc * CH + h) * 128, 0, fb);
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
        constexpr uint32_t idesc = F4 ? idesc_mxf4_f32(128, NP) : idesc_e4m3_f32(128, NP);
        const uint32_t d = tbase + static_cast<uint32_t>(t * NP);
        // B of stage i: the limb panels at the head of stage slot i mod S, or limb slot i mod S2
        const uint64_t desc0 = smem_desc_sw128(smem_addr(F4 ? lring : smem));
        constexpr uint32_t DSTEP = (F4 ? B_BYTES : STAGE) >> 4;
        // The issuer is the critical thread of the pipeline: per stage it only
        // waits, issues and commits.  Windows (at most F stages, never across
        // a segment end) are sized once when they start.
        const int bid_wrap = PB * T;
        int s = 0, r = 0, kc = kc0, bid = t;  // bid: named barrier id - 1
        uint64_t dstage = desc0;
        uint32_t aslot = tbase + static_cast<uint32_t>(ACC_COLS + t * CH * CW);
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
                    for (int q = 0; q < MQ; ++q) {
                        // 32 bytes of every row of panel q/4 (K = 32 e4m3 or 64 e2m1), 8 TMEM columns of A
                        const uint64_t bd = dstage + static_cast<uint64_t>(((q >> 2) * NP * 128 + (q & 3) * 32) >> 4);
                        if (F4)
                            mma_ts_mxf4(d, aslot + 8 * q, bd, idesc, tbase + SF_COL, tbase + SF_COL + 4,
                                        (e == 0 && q == 0) ? 0u : 1u);
                        else
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
                if (++s == S2) {
                    s = 0;
                    dstage = desc0;
                } else {
                    dstage += static_cast<uint64_t>(DSTEP);
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
        float *accs = reinterpret_cast<float *>(smem + ring_bytes + 1024) + (threadIdx.x - 32 * DEC0);
        auto acc = [&](int tt, int e) -> float & { return accs[(tt * KH + e) * 128]; };
        // per-column constants, loaded once: sum V, step lambda, active (fused
        // step) and the power-of-two scale of the B limbs
        float *colc = reinterpret_cast<float *>(smem + ring_bytes + 1024) + T * KH * 128;
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
            if constexpr (F4) {
                // one lambda column of eight e2m1 limbs (weights 8^-l) per 8 columns
#pragma unroll
                for (int tt = 0; tt < T; ++tt) {
#pragma unroll
                    for (int cc = 0; cc < NP / 8; ++cc) {
                        uint32_t u[8];
                        tmem_ld_32x32b_x8(lane_base + static_cast<uint32_t>(tt * NP + cc * 8), u);
                        tmem_wait_ld();
                        float x = __uint_as_float(u[7]);
#pragma unroll
                        for (int l = 6; l >= 0; --l) x = fmaf(x, 0.125f, __uint_as_float(u[l]));
                        acc(tt, cc) += x;
                    }
                }
            } else {
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
                            const float xtv = ldexpf(acc(tt, e), bsc[e] + SH);  // (X^T V)_j
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
                    if (e < P.k) P.part[slot * P.slot_stride + e * P.rows_pad + row] = ldexpf(acc(tt, e), bsc[e] + SH);
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

        int s = gamma % S, r = gamma % R, nbid = gamma % PB, s2 = gamma % S2;
        uint32_t fph = static_cast<uint32_t>((gamma / S) & 1), aph = static_cast<uint32_t>((gamma / R) & 1);
        uint32_t lph = static_cast<uint32_t>((gamma / S2) & 1);
        for (int64_t i = gamma; i < nu; i += G) {
            bool go = ok;
            if (go && gamma == 0) {
                // windows ending before stage i: every stage of theirs is decoded
                // or owned by another group, so their MMAs complete without us
                fold_until(i);
                go = ok;
            }
            if (go && !warp_wait(full0 + 8 * s, fph, lim, abort_sm)) go = false;
            // e2m1: the stage's limbs too, so that the issuers find them in place
            if (F4 && go && !warp_wait(lfull0 + 8 * s2, lph, lim, abort_sm)) go = false;
            // TMEM slot r is free once the MMAs of stage i - R are complete
            if (go && i >= R && !warp_wait(aempty0 + 8 * r, aph ^ 1u, lim, abort_sm)) go = false;
            if (go) {
                if (i >= R && q == (DEC0 & 3) && lane == 0) {
                    // the MMAs of stage i - R, which read its limbs (and in the
                    // e4m3 form follow the decoders' reads of its codes), are complete
                    if (F4) {
                        int se = s2 - R;
                        if (se < 0) se += S2;
                        mbar_arrive(lempty0 + 8 * se);
                    } else {
                        int se = s - R;
                        if (se < 0) se += S;
                        mbar_arrive(empty0 + 8 * se);
                    }
                }
                tc_fence_after();
                const uint8_t *xs = F4 ? smem + static_cast<size_t>(s) * X_BYTES + rit * 32
                                       : smem + s * STAGE + B_BYTES + rit * 32;
                const uint32_t acol = lane_base + static_cast<uint32_t>(ACC_COLS + r * SLOT_COLS);
                if constexpr (F4) {
                    // two chunks of one tile per store: 16 TMEM columns each
#pragma unroll 2
                    for (int tp = 0; tp < T * CH / 2; ++tp) {
                        uint32_t o[32];
#pragma unroll
                        for (int c2 = 0; c2 < 2; ++c2) {
#pragma unroll
                            for (int hh = 0; hh < 2; ++hh) {
                                const uint4 v = *reinterpret_cast<const uint4 *>(xs + (2 * tp + c2) * BLOCK_BYTES +
                                                                                 16 * (hh ^ swp));
                                uint32_t *oo = o + 16 * c2 + 8 * hh;
                                decode16_e2m1(v.x, oo);
                                decode16_e2m1(v.y, oo + 2);
                                decode16_e2m1(v.z, oo + 4);
                                decode16_e2m1(v.w, oo + 6);
                            }
                        }
                        tmem_st_32x32b_x32(acol + tp * 32, o);
                        if ((2 * tp + 1) % CH == CH - 1) {
                            tmem_wait_st();
                            tc_fence_before();
                            __syncwarp();
                            named_arrive(1 + nbid * T + (2 * tp) / CH, NB_COUNT);
                        }
                    }
                    // every code of the slot has been read into registers (the
                    // stores consumed them): the code slot goes back to its producer
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty0 + 8 * s);
                } else {
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
            s2 += G;
            while (s2 >= S2) {
                s2 -= S2;
                lph ^= 1u;
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
        if (lane == 0) {
            for (int s = 0; s < S; ++s)
                if (armed[s] >= 0) mbar_wait(full0 + 8 * s, static_cast<uint32_t>(armed[s]), DRAIN_LIMIT, &g_never_set);
            if (F4)
                for (int s = 0; s < S2; ++s)
                    if (armed2[s] >= 0)
                        mbar_wait(lfull0 + 8 * s, static_cast<uint32_t>(armed2[s]), DRAIN_LIMIT, &g_never_set);
        }
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

} // namespace
} // namespace coxgb
