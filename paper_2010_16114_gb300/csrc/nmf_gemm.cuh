// nmf_gemm.cuh -- the tensor-core product of the NMF iteration (arXiv
// 2010.16114, Section 5.1: X W^T and X^T V), included by nmf.cu only.
//
// D = A B^T for a bf16 A (rows x K, K-major: X, or X stored column-major) and a
// factor panel B of NP rows = three bf16 limbs of every factor row
// (f = h0 + h1 + h2, exact for FP32 f; row l rp + c holds limb l of row c),
// tcgen05.mma kind::f16 with both operands in 128B-swizzled shared memory and
// FP32 accumulators in Tensor Memory.  The A operand is loaded by TMA in
// 128-row x 64-column boxes (zero-filled past the matrix edges), the panel
// in NP x 64 boxes.
//
// Launched with programmatic stream serialisation, a CTA sets up its barriers
// and TMEM while the kernel ahead finishes, then waits for it (pdl_wait).
//
// Per CTA (one per SM): a TMA warp fills a ring of shared-memory stages, one
// thread issues four M128 x N x K16 MMAs per 64-wide K chunk into one of two
// TMEM accumulators, and four epilogue warps (one per TMEM lane quarter) add
// the three limb columns of each value.  An accumulator takes at most WINDOW
// chunks (512 K); the epilogue then adds it into FP32 running sums in shared
// memory (round to nearest) while the other accumulator fills: the tensor
// cores' own FP32 accumulation over thousands of K came out about 1e-5 low at
// X 10,000 x 10,000, where 512 K keep that bias near 1e-6.  At a row tile's
// end the sums are the CTA's partial of the tile.  Work split: units = (row
// tile, K chunk) in row-tile order; CTA c takes units [c L, (c+1) L), so a
// row tile is cut between at most a few CTAs, each leaving a partial in its
// own slot [tile][slot][r][128]; the update kernel adds the slots in slot
// order (deterministic).
#pragma once
#include <cuda_bf16.h>

#include "ptx.cuh"

namespace coxgb {
namespace {

constexpr int NT = 128;                 // rows per tile (MMA M)
constexpr int NK = 64;                  // K per chunk: 64 bf16 = one 128-byte swizzled row
constexpr int A_BYTES = NT * NK * 2;    // 16 KB A box per stage
constexpr int GEMM_THREADS = 192;       // TMA warp, MMA warp, four epilogue warps
constexpr int MAX_STAGES = 8;
constexpr int WINDOW = 8;               // K chunks one TMEM accumulator sums before the epilogue folds it
constexpr long long NMF_DRAIN = 4000000000LL;  // ~2 s: copies and MMAs always finish
__device__ int g_nmf_never = 0;                // abort flag of drain waits: never raised

enum : int { NMF_ERR_TIMEOUT = 1, NMF_ERR_NONFINITE = 2, NMF_ERR_NEGATIVE = 4 };

struct GemmArgs {
    int KC;             // K chunks per row tile
    int r, rp, NP;      // rank; r rounded up to 8; N of the MMA (3 rp rounded up to 16)
    int S, stage;       // shared-memory stages; bytes per stage (A box + NP x 128 B panel)
    int tcols;          // TMEM columns allocated
    uint32_t idesc;
    int64_t units, L;   // (row tile, chunk) units; units per CTA
    int SL;             // partial slots per row tile
    float *part;        // [tile][slot][r][128] FP32
    long long wait_limit;
    int *err;
};

__device__ __forceinline__ void nmf_fail(volatile int *abort_sm, int *err)
{
    if (!*abort_sm) {
        *abort_sm = 1;
        atomicOr(err, NMF_ERR_TIMEOUT);
    }
}

// Pipeline hand-offs (S stages, two accumulators a = window index mod 2):
//   full[s]   TMA transaction bytes                    producer -> issuer
//   empty[s]  tcgen05.commit after the stage's MMAs    issuer   -> producer
//   accf[a]   tcgen05.commit at a window end           issuer   -> epilogue
//   acce[a]   four arrivals once the epilogue read a   epilogue -> issuer
// Every waiter waits for the completions of a barrier in order, and the
// completion before the awaited one is always one it waited for itself (the
// producer's wait on empty[s] for unit i - S follows its wait for unit i - 2S;
// the issuer's wait on full[s] for unit i follows the one for unit i - S; on
// accf[a] / acce[a] for window w, the waits for window w - 2), so no parity
// wait can return a phase early.  A segment is the CTA's run of units in one
// row tile; a window is at most WINDOW units of a segment.
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_nmf_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs P)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    const int S = P.S, STAGE = P.stage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * STAGE);
    const uint32_t full0 = smem_addr(bars);
    const uint32_t empty0 = full0 + 8 * S;
    const uint32_t accf0 = empty0 + 8 * S;
    const uint32_t acce0 = accf0 + 16;
    const uint32_t drainb = acce0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 5);
    volatile int *abort_sm = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *sums = reinterpret_cast<float *>(smem + S * STAGE + 256);  // [r][128] running sums

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_trigger();
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4);
        }
        mbar_init(drainb, 1);
        *abort_sm = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_addr(tmem_slot), static_cast<uint32_t>(P.tcols));
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
    // everything above touches only this CTA's shared memory, TMEM and the
    // kernel parameters; the kernel ahead (the factor update that wrote the
    // limb panel) must be complete before any global access
    pdl_wait();

    const int64_t u0 = static_cast<int64_t>(blockIdx.x) * P.L;
    const int64_t u1 = min(u0 + P.L, P.units);
    const int64_t nu = u1 > u0 ? u1 - u0 : 0;
    const int KC = P.KC;
    const long long lim = P.wait_limit;
    const int g0 = static_cast<int>(u0 / KC), kc0 = static_cast<int>(u0 - static_cast<int64_t>(g0) * KC);

    if (warp == 0) {
        // ---------------- TMA producer (lane 0) ----------------
        if (lane == 0) {
            int g = g0, kc = kc0, s = 0;
            uint32_t ph = 0;
            int64_t issued = 0;
            for (int64_t i = 0; i < nu; ++i) {
                if (i >= S && !mbar_wait(empty0 + 8 * s, ph ^ 1u, lim, abort_sm)) {
                    nmf_fail(abort_sm, P.err);
                    break;
                }
                const uint32_t st = smem_addr(smem + static_cast<size_t>(s) * STAGE);
                const uint32_t fb = full0 + 8 * s;
                mbar_arrive_expect_tx(fb, static_cast<uint32_t>(STAGE));
                tma_load_2d(st, &tmA, kc * NK, g * NT, fb);
                tma_load_2d(st + A_BYTES, &tmB, kc * NK, 0, fb);
                ++issued;
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
                if (++kc == KC) {
                    kc = 0;
                    ++g;
                }
            }
            // every load issued has landed before the CTA may exit
            for (int64_t i = issued > S ? issued - S : 0; i < issued; ++i)
                mbar_wait(full0 + 8 * static_cast<uint32_t>(i % S), static_cast<uint32_t>((i / S) & 1), NMF_DRAIN,
                          &g_nmf_never);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (lane 0) ----------------
        if (lane == 0) {
            const uint64_t descA = smem_desc_sw128(smem_addr(smem));
            const uint64_t descB = smem_desc_sw128(smem_addr(smem + A_BYTES));
            int s = 0, kc = kc0;
            uint32_t ph = 0;
            bool ok = true;
            int64_t w = 0;  // windows so far
            for (int64_t i = 0; ok && i < nu;) {
                const int64_t seg = min(static_cast<int64_t>(KC - kc), nu - i);
                for (int64_t e0 = 0; ok && e0 < seg; e0 += WINDOW, ++w) {
                    const int64_t wl = min(static_cast<int64_t>(WINDOW), seg - e0);
                    const int a = static_cast<int>(w & 1);
                    if (w >= 2 &&
                        !mbar_wait(acce0 + 8 * a, static_cast<uint32_t>(((w - 2) >> 1) & 1), lim, abort_sm)) {
                        nmf_fail(abort_sm, P.err);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tbase + static_cast<uint32_t>(a * P.NP);
                    for (int64_t e = 0; e < wl; ++e) {
                        if (!mbar_wait(full0 + 8 * s, ph, lim, abort_sm)) {
                            nmf_fail(abort_sm, P.err);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t off = static_cast<uint64_t>(s) * static_cast<uint64_t>(STAGE >> 4);
#pragma unroll
                        for (int kk = 0; kk < NK / 16; ++kk)  // K = 16 per MMA: 32 bytes of every row
                            mma_ss_f16(d, descA + off + 2 * kk, descB + off + 2 * kk, P.idesc,
                                       (e > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(empty0 + 8 * s);
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(accf0 + 8 * a);
                }
                i += seg;
                kc = 0;
            }
            mma_commit(drainb);
            mbar_wait(drainb, 0, NMF_DRAIN, &g_nmf_never);
        }
    } else {
        // ---------------- epilogue: warps 2..5, TMEM lane quarter warp % 4 ----------------
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * quarter) << 16);
        const int r = P.r;
        float *sum = sums + row;
        int g = g0, kc = kc0;
        bool ok = true;
        int64_t w = 0;
        for (int64_t i = 0; ok && i < nu;) {
            const int64_t seg = min(static_cast<int64_t>(KC - kc), nu - i);
            const int64_t slot = static_cast<int64_t>(blockIdx.x) - (static_cast<int64_t>(g) * KC) / P.L;
            float *dst = P.part + ((static_cast<int64_t>(g) * P.SL + slot) * r) * NT + row;
            for (int64_t e0 = 0; e0 < seg; e0 += WINDOW, ++w) {
                const bool first = e0 == 0, last = e0 + WINDOW >= seg;
                const int a = static_cast<int>(w & 1);
                if (!__all_sync(0xffffffffu,
                                mbar_wait(accf0 + 8 * a, static_cast<uint32_t>((w >> 1) & 1), lim, abort_sm))) {
                    if (lane == 0) nmf_fail(abort_sm, P.err);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = lane_base + static_cast<uint32_t>(a * P.NP);
                for (int c0 = 0; c0 < r; c0 += 8) {
                    uint32_t h0[8], h1[8], h2[8];
                    tmem_ld_32x32b_x8(acc + static_cast<uint32_t>(c0), h0);
                    tmem_ld_32x32b_x8(acc + static_cast<uint32_t>(P.rp + c0), h1);
                    tmem_ld_32x32b_x8(acc + static_cast<uint32_t>(2 * P.rp + c0), h2);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int c = c0 + e;
                        if (c < r) {
                            const float v =
                                (__uint_as_float(h0[e]) + __uint_as_float(h1[e])) + __uint_as_float(h2[e]);
                            const float t = first ? v : sum[c * NT] + v;
                            if (last)
                                dst[static_cast<int64_t>(c) * NT] = t;
                            else
                                sum[c * NT] = t;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * a);
            }
            i += seg;
            kc = 0;
            ++g;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, static_cast<uint32_t>(P.tcols));
    }
}

} // namespace
} // namespace coxgb
