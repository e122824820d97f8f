// gemm_tc.cu -- shapes, plans and launches of the two genotype products of the
// Cox iteration (arXiv 2010.16114, Section 5.3); the kernel is in gemm_kernel.cuh.
#include <algorithm>

#include "gemm_kernel.cuh"

namespace coxgb {
namespace {

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

// beta -> e2m1 limbs [NP][p_pad / 2]: thread j of a column writes byte j,
// which holds SNPs 16 (j / 8) + j mod 8 (low nibble) and that + 8 (high).
__global__ void k_prep_limbs_beta4(const float *__restrict__ beta, int64_t p, int64_t p_pad, int nb,
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
            s_sh = limb_scale4(m);
            if (blockIdx.x == 0) bs[kk] = s_sh;
        }
    }
    __syncthreads();
    const int s = s_sh;
    const int64_t rb = p_pad / 2;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < rb;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j0 = ((j >> 3) << 4) + (j & 7);
        if (j0 >= p) continue;
        uint8_t d0[LIMBS4], d1[LIMBS4];
        split_e2m1_units(ldexpf(beta[static_cast<int64_t>(kk) * p + j0], -s), d0);
        if (j0 + 8 < p)
            split_e2m1_units(ldexpf(beta[static_cast<int64_t>(kk) * p + j0 + 8], -s), d1);
        else
            for (int l = 0; l < LIMBS4; ++l) d1[l] = 0;
#pragma unroll
        for (int l = 0; l < LIMBS4; ++l) Bq[(LIMBS4 * kk + l) * rb + j] = static_cast<uint8_t>(d0[l] | (d1[l] << 4));
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

using KernelFn = GemmKernelFn;

// (T row tiles, CH K chunks) per stage for a limb-column class NP.  One issuer
// per tile leaves the most TMEM to the A slot ring (a second issuer per tile
// needs a second accumulator).  N = 256 fills half of TMEM per accumulator,
// so that class takes one tile per stage.
// A stage spans CH K chunks: every hand-off costs a few hundred cycles
// whatever its size, so up to N = 64 a stage takes two chunks (16 KB of codes
// at T = 2), which keeps the same bytes in TMEM with half the hand-offs.
// This is the default; the autotuner times every compiled shape instead.
// The e2m1 form stages chunk pairs (one 128-byte limb panel per pair) of two
// row tiles.
void shape_for(int NP, int *T, int *CH, int *alt, int f4)
{
    *T = NP <= 128 ? 2 : 1;
    *CH = f4 ? 2 : NP <= 64 ? 2 : 1;
    *alt = 0;
}

constexpr int G_ALT = 2;   // decoder groups of the alternating-issuer kernels
constexpr int G_WIDE = 2;  // decoder groups of the 2 x 2 shape at 128 limb columns and 2 x 3 at 64

KernelFn pick_kernel(int T, int CH, int NP, int alt, int f4)
{
    if (f4) return alt ? nullptr : pick_kernel_f4(T, CH, NP);
    switch (((alt ? 100 : 0) + T * 10 + CH) * 1000 + NP) {
    case 22016: return k_packed_gemm<2, 2, 16, DEC_GROUPS, false, false>;
    case 21016: return k_packed_gemm<2, 1, 16, DEC_GROUPS, false, false>;
    case 12016: return k_packed_gemm<1, 2, 16, DEC_GROUPS, false, false>;
    case 22032: return k_packed_gemm<2, 2, 32, DEC_GROUPS, false, false>;
    case 21032: return k_packed_gemm<2, 1, 32, DEC_GROUPS, false, false>;
    case 12032: return k_packed_gemm<1, 2, 32, DEC_GROUPS, false, false>;
    case 22064: return k_packed_gemm<2, 2, 64, DEC_GROUPS, false, false>;
    case 21064: return k_packed_gemm<2, 1, 64, DEC_GROUPS, false, false>;
    case 12064: return k_packed_gemm<1, 2, 64, DEC_GROUPS, false, false>;
    case 21128: return k_packed_gemm<2, 1, 128, DEC_GROUPS, false, false>;
    case 12128: return k_packed_gemm<1, 2, 128, DEC_GROUPS, false, false>;
    case 11128: return k_packed_gemm<1, 1, 128, DEC_GROUPS, false, false>;
    // two decoder groups: 2 tiles x 2 chunks at 128 limb columns, whose two
    // 128-column TMEM slots beside 256 accumulator columns leave no third slot
    case 22128: return k_packed_gemm<2, 2, 128, G_WIDE, false, false>;
    // two decoder groups: 2 tiles x 3 chunks at 64 limb columns (12 MMAs per
    // commit per issuer; two 192-column slots beside 128 accumulator columns)
    case 23064: return k_packed_gemm<2, 3, 64, G_WIDE, false, false>;
    case 11256: return k_packed_gemm<1, 1, 256, DEC_GROUPS, false, false>;
    // alternating issuers: 16 MMAs per commit up to N = 64, 8 at N = 128
    case 122016: return k_packed_gemm<2, 2, 16, G_ALT, true, false>;
    case 122032: return k_packed_gemm<2, 2, 32, G_ALT, true, false>;
    case 122064: return k_packed_gemm<2, 2, 64, G_ALT, true, false>;
    case 112128: return k_packed_gemm<1, 2, 128, G_ALT, true, false>;
    default: return nullptr;
    }
}

int groups_for(int T, int CH, int NP, int alt, int f4)
{
    if (alt) return G_ALT;
    if (f4) return DEC_GROUPS;
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

// A decoder group's parity wait on a slot of a ring of n slots, for stage i,
// is unambiguous once the load of stage i - n is complete.  The group's own
// previous wait was for stage i - G, after the MMAs of stage i - G - R, so
// every load up to stage i - G - R is complete: n >= G + R suffices, and so
// does n a multiple of G (the group itself waited for stage i - n).
bool ring_safe(int G, int R, int n) { return n >= G + R || n % G == 0; }

// The e2m1 form's plan: a ring of S code slots (T CH 4 KB blocks, released by
// the decoders once they have read them) and one of S2 limb slots (CH/2 panels
// of NP 128-byte rows, released once the stage's MMAs are complete), each with
// one producer thread that loads every stage in order and reuses a slot only
// after its release.  Both depths keep ring_safe; S2 > R keeps the limb
// producer of stage i from waiting on the decoders of stage i, and S2 = R + 3
// when it fits gives the limbs (from L2) three stages of look-ahead (R + 2
// measured 0.65 of HBM against 0.84).  The code ring takes the rest of the
// shared memory (at most 12, at least G + 1), the deepest safe depth.  The
// largest TMEM ring for which such depths exist is taken.
int plan_e2m1(GemmPlan &g, int T, int CH, int NP, int G, int stages_req, int fold_bytes)
{
    const int xb = T * CH * BLOCK_BYTES, bb = (CH / 2) * NP * 128;
    const int acc_cols = T * NP;
    // depth of the code ring beside S2 limb slots at TMEM ring R, or 0
    auto code_depth = [&](int R, int S2) {
        if (stages_req > 0) {
            const int S = std::max(stages_req, G + 1);
            const bool fits = S * xb + S2 * bb + 2048 + fold_bytes <= 227 * 1024;
            return ring_safe(G, R, S) && fits ? S : 0;
        }
        int S = std::min(12, (227 * 1024 - (S2 * bb + 2048 + fold_bytes)) / xb);
        while (S >= G + 1 && !ring_safe(G, R, S)) --S;
        return S >= G + 1 ? S : 0;
    };
    int ring = 0, S2 = 0, S = 0;
    for (int R = std::min(8, (SF_COL - acc_cols) / (T * CH * 16)); R >= G && !S; --R) {
        if (lcm_i(G, R) * T > 15) continue;
        for (int L = R + 4; L >= R + 1 && !S; --L) {
            if (!ring_safe(G, R, L)) continue;
            const int d = code_depth(R, L);
            if (d) {
                ring = R;
                S2 = L;
                S = d;
            }
        }
    }
    if (!S) return COX_ERR_ARG;
    const int fixed = S2 * bb + 2048 + fold_bytes;
    g.T = T;
    g.CH = CH;
    g.NP = NP;
    g.f4 = 1;
    g.alt = 0;
    g.pair = 0;
    g.G = G;
    g.ring = ring;
    g.nb_period = lcm_i(G, ring);
    g.stages = S;
    g.stages2 = S2;
    g.smem = static_cast<size_t>(S) * xb + static_cast<size_t>(fixed);
    if (g.smem < 120 * 1024) g.smem = 120 * 1024;  // one CTA per SM: it owns all 512 TMEM columns
    if (g.smem > 227 * 1024) return COX_ERR_ARG;    // too many stages requested
    return COX_OK;
}

} // namespace

int gemm_shapes(int k, int *T, int *CH, int *issue, int max, int f4)
{
    const int NP = f4 ? limb_cols4(k) : limb_cols(k);
    if (NP == 0) return 0;
    int n = 0;
    for (int is = 1; is <= (f4 ? 1 : 3); ++is)
        for (int t = 2; t >= 1; --t)
            for (int c = 4; c >= 1; --c)
                if (pick_kernel(t, c, NP, is == 2, f4) && n < max &&
                    !(is == 3 && groups_for(t, c, NP, 0, f4) == G_WIDE)) {
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
int plan_shape(GemmPlan &g, int k, int T_req, int CH_req, int stages_req, int issue_req, int f4)
{
    if (k < 1 || k > MAX_K_TC) return COX_ERR_ARG;
    if (issue_req < 0 || issue_req > 3) return COX_ERR_ARG;
    if (f4 && (issue_req > 1 || limb_cols4(k) == 0)) return COX_ERR_ARG;  // e2m1: per-tile issuers, k <= 16
    const int np_cls = f4 ? limb_cols4(k) : limb_cols(k);
    int T = 2, CH = 1, alt = 0;
    shape_for(np_cls, &T, &CH, &alt, f4);
    if (issue_req > 0) alt = issue_req == 2;
    if (T_req > 0) T = T_req;
    if (CH_req > 0) CH = CH_req;
    if (!pick_kernel(T, CH, np_cls, alt, f4)) return COX_ERR_ARG;  // shape not compiled for this class
    const int G = groups_for(T, CH, np_cls, alt, f4);
    if (G == G_WIDE && !alt && issue_req == 3) return COX_ERR_ARG;  // pair commits: not planned for it
    // limb panels of 128-byte rows: one per K chunk (e4m3), one per chunk pair (e2m1)
    const int stage = (f4 ? CH / 2 : CH) * np_cls * 128 + CH * T * BLOCK_BYTES;
    const int kh = np_cls / (f4 ? LIMBS4 : LIMBS);  // coefficient columns the fold holds
    // group 0's window sums, then four per-column constants
    const int fold_bytes = T * kh * 128 * 4 + 4 * kh * 4;
    if (f4) return plan_e2m1(g, T, CH, np_cls, G, stages_req, fold_bytes);
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
    const int cw = f4 ? 16 : 32;              // TMEM columns per tile and K chunk
    const int tmem = f4 ? SF_COL : 512;       // the e2m1 form keeps 8 columns of scale factors
    const int ring_max = std::min(8, (tmem - acc_cols) / (T * CH * cw));
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
    g.f4 = f4;
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
    COX_TRY(plan_shape(g, k, T_req, CH_req, stages_req, issue_req, is_e2m1(h)));
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
        KernelFn fn = pick_kernel(g.T, g.CH, g.NP, g.alt, g.f4);
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
        // one 128-byte row (a K chunk of one limb column, or a pair of K chunks
        // in the e2m1 form's two values per byte) per limb column
        const int64_t row_bytes = g.f4 ? K_pad / 2 : K_pad;
        cuuint64_t dims[2] = {static_cast<cuuint64_t>(row_bytes), static_cast<cuuint64_t>(np_cls)};
        cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_bytes)};
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
    kp.stages2 = g.stages2;
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
    KernelFn fn = pick_kernel(g.T, g.CH, g.NP, g.alt, g.f4);
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
    if (h->ws.g1.f4)
        k_prep_limbs_beta4<<<grid, 256, 0, st>>>(beta, h->p, h->p_pad, h->l1_blocks, h->ws.bmaxp, h->ws.Bq,
                                                 h->ws.bs1, h->d_err);
    else
        k_prep_limbs_beta<<<grid, 256, 0, st>>>(beta, h->p, h->p_pad, h->l1_blocks, h->ws.bmaxp, h->ws.Bq,
                                                h->ws.bs1, h->d_err);
    COX_CUDA(cudaGetLastError());
    return COX_OK;
}

} // namespace coxgb
