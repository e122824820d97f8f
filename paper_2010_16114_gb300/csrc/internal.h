// internal.h -- handle layout and cross-file entry points of libcoxgb.
#pragma once
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <vector>

#include "../../include/coxgb.h"

namespace coxgb {

// Device-side error bits (OR-ed into handle->d_err by kernels).
enum : int { DEVERR_TIMEOUT = 1, DEVERR_NONFINITE = 2, DEVERR_CODE3 = 4 };

constexpr int TILE = 128;          // rows per tensor-core tile, K per chunk
constexpr int BLOCK_BYTES = 4096;  // one 128 x 128 block of 2-bit codes
constexpr int PAD = 1024;          // n, p padding of the tiled layouts
constexpr int SCAN_CH = 2048;      // subjects per scan chunk (256 threads x 8)
constexpr int MAX_K_TC = 64;       // largest k of the tensor-core path
constexpr int LIMBS = 4;           // e4m3 limbs per coefficient (4 significant bits each)
constexpr int DEC_GROUPS = 3;      // decoder warp groups of the tensor-core products
constexpr int LIMBS4 = 8;          // e2m1 limbs per coefficient (3 significant bits each)
constexpr int SF_COL = 504;        // TMEM columns 504..511: unit block scales of the e2m1 products

// Limb columns of a k-column product: LIMBS k rounded up to an MMA width class.
inline int limb_cols(int k)
{
    const int n = LIMBS * k;
    return n <= 16 ? 16 : n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256;
}

// Limb columns of the e2m1 form: LIMBS4 k rounded up to 64 or 128 (k <= MAX_K_E2M1);
// 0 beyond.
constexpr int MAX_K_E2M1 = 16;
inline int limb_cols4(int k)
{
    const int n = LIMBS4 * k;
    return n <= 64 ? 64 : n <= 128 ? 128 : 0;
}

// Position of code K (0..15) of a 16-code word: bit 8 (K mod 4) + 2 (K div 4),
// so that (word >> 2q) & 0x03030303 is the four codes 4q..4q+3, one per byte:
// as e4m3 bytes these are the subnormals c 2^-9, exact tensor-core operands.
__host__ __device__ inline int code_bit(int K) { return 8 * (K & 3) + 2 * (K >> 2); }

// ---- e4m3 limbs -----------------------------------------------------------------
// A coefficient column b is held as LIMBS e4m3 numbers: with a power-of-two
// scale 2^s putting max |b| 2^-s in [128, 256) (e4m3 reaches 448),
// r_0 = b 2^-s, d_l = RN_e4m3(r_l), r_(l+1) = 16 (r_l - d_l); each step keeps
// |r| <= 256, and b = 2^s sum_l d_l 2^-4l with about 4 LIMBS significant bits.

__device__ inline float e4m3_value(uint8_t q)
{
    // sign, 4-bit exponent (bias 7), 3-bit mantissa; exponent 0: subnormal m 2^-9
    const int e = (q >> 3) & 15, m = q & 7;
    const float v = e ? ldexpf(1.0f + 0.125f * static_cast<float>(m), e - 7) : ldexpf(static_cast<float>(m), -9);
    return (q & 0x80) ? -v : v;
}

__device__ inline int limb_scale(float mx) { return mx > 0.f ? ilogbf(mx) - 7 : 0; }

// Limbs of r (|r| <= 256) into d[0..LIMBS); returns the value they represent.
__device__ inline float split_e4m3(float r, uint8_t *d)
{
    if (!isfinite(r)) {
        for (int l = 0; l < LIMBS; ++l) d[l] = 0x7F;  // NaN: the products flag it
        return r;
    }
    float rep = 0.f, w = 1.f;
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) {
        const uint8_t q = static_cast<uint8_t>(__nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3));
        const float v = e4m3_value(q);
        d[l] = q;
        rep = fmaf(v, w, rep);
        r = (r - v) * 16.f;
        w *= 0.0625f;
    }
    return rep;
}

// Value of an e4m3 byte in units of 2^-9 (exact: normal values are
// (8 + m) 2^(e - 10), subnormal ones m 2^-9).
__device__ inline int e4m3_units(uint8_t q)
{
    const int e = (q >> 3) & 15, m = q & 7;
    const int u = e ? (8 + m) << (e - 1) : m;
    return (q & 0x80) ? -u : u;
}

// The split of split_e4m3, returning the value the limbs represent times 2^21
// as an exact integer (limb l is a multiple of 2^-9 weighted 16^-l; below
// 2^30 in magnitude for |r| <= 256).  Non-finite r gives NaN limbs and 0.
__device__ inline int split_e4m3_units(float r, uint8_t *d)
{
    if (!isfinite(r)) {
        for (int l = 0; l < LIMBS; ++l) d[l] = 0x7F;
        return 0;
    }
    int q = 0;
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) {
        const uint8_t b = static_cast<uint8_t>(__nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3));
        d[l] = b;
        q = 16 * q + e4m3_units(b);
        r = (r - e4m3_value(b)) * 16.f;
    }
    return q;
}

// ---- e2m1 limbs -----------------------------------------------------------------
// A coefficient column b is held as LIMBS4 e2m1 numbers on the grid of halves in
// [-2, 2]: with a power-of-two scale 2^s putting max |b| 2^-s in [1, 2),
// r_0 = b 2^-s, d_l = RN(2 r_l) / 2, r_(l+1) = 8 (r_l - d_l) (exact; |r| <= 2),
// and b = 2^s sum_l d_l 8^-l to within 2^(1 - 3 LIMBS4) = 2^-23 of max |b|.
// Limb rows hold two K positions per byte, in the order the decoders give the
// codes (decode16_e2m1): positions K and K + 8 of a 16-code group w share byte
// 8 w + (K mod 8), K in the low nibble.
__host__ __device__ inline int64_t e2m1_byte(int64_t K) { return ((K >> 4) << 3) + (K & 7); }

__device__ inline int limb_scale4(float mx) { return mx > 0.f ? ilogbf(mx) : 0; }

// Limbs of r (|r| < 2) as e2m1 nibbles; returns the value they represent in
// units of 2^(-1 - 3 (LIMBS4 - 1)), an exact integer.  Non-finite r gives zero
// limbs (its caller flags it).
__device__ inline int split_e2m1_units(float r, uint8_t *nib)
{
    if (!isfinite(r)) {
        for (int l = 0; l < LIMBS4; ++l) nib[l] = 0;
        return 0;
    }
    int q = 0;
#pragma unroll
    for (int l = 0; l < LIMBS4; ++l) {
        const float t = rintf(2.f * r);  // -4 .. 4
        const int ti = static_cast<int>(t);
        nib[l] = static_cast<uint8_t>((ti < 0 ? 8 : 0) | (ti < 0 ? -ti : ti));
        q = 8 * q + ti;
        r = fmaf(-4.f, t, 8.f * r);  // 8 (r - t / 2), exact
    }
    return q;
}

// 32-bit word index, in a tiled 2-bit layout of KC chunks per row tile, of the
// 16 codes of row rit (0..127) of row tile mt at K offset `within` (a multiple
// of 16) of chunk kc: row records of 32 bytes, two 16-byte halves (K 0-63 and
// 64-127 of the chunk), stored swapped in rows with bit 2 set.
__host__ __device__ inline int64_t word_offset(int64_t mt, int64_t KC, int64_t kc, int rit, int within)
{
    const int hh = within >> 6, w = (within & 63) >> 4;
    const int phys = hh ^ ((rit >> 2) & 1);
    return ((mt * KC + kc) * BLOCK_BYTES + rit * 32 + phys * 16 + w * 4) >> 2;
}

// K order of the SNP-major copy (A4).  Sorted subjects are kept in blocks of
// 16 (one packed word), and sorted block b is stored at block (a b) mod nb,
// nb = n_pad / 16, a odd and prime to nb, near nb (sqrt 5 - 1) / 2.  Any run
// of consecutive K positions then holds subjects spread evenly over the time
// order, so the running sums of x_ij V_i that the tensor cores accumulate do
// not drift with the time trend of V (V = delta - u sums to zero only over all
// subjects); the positions inside a block, and so the K-slot scales, are kept.
__host__ __device__ inline int64_t a4_pos(int64_t i, int64_t a, int64_t nb)
{
    return ((a * (i >> 4)) % nb) * 16 + (i & 15);
}

// One tensor-core product: a 2-bit A (rows x K, tiled) times limb matrix B.
struct GemmPlan {
    int T = 2;         // 128-row tiles per CTA (one M group)
    int CH = 1;        // K chunks (128 each) per stage
    int alt = 0;       // 1: two issuers on alternate stages (else one per row tile)
    int pair = 0;      // 1: per-tile issuers commit after every second stage
    int G = 3;         // decoder groups
    int NP = 16;       // limb columns (limb_cols(k), or limb_cols4(k) in the e2m1 form)
    int f4 = 0;        // 1: e2m1 operands (kind::mxf4), else e4m3 (kind::f8f6f4)
    int stages = 6;    // shared-memory pipeline depth (e2m1 form: code slots)
    int stages2 = 0;   // e2m1 form: limb slots
    int ring = 4;      // TMEM A buffers
    int nb_period = 6; // stage period of the named barriers: lcm(decoder groups, ring)
    int F = 32;        // K chunks per TMEM accumulation window
    int grid = 0;      // CTAs
    int KC = 0;        // stages per M group (K chunks / CH)
    int n_groups = 0;  // M groups
    int64_t units = 0, L = 0;
    int max_slots = 1;
    int64_t rows_pad = 0;  // row stride of the partial buffer
    size_t smem = 0;
    CUtensorMap tmA, tmB;
};

struct Workspace {
    int k = 0;        // columns the workspace is sized for
    int NP = 0;
    // split / gemv / fp64 common (sorted subject order)
    double *eta = nullptr;      // k x n
    double *w = nullptr;        // k x n
    double *Rt = nullptr;       // k x n local reverse scans (at event-group heads); then V in FP32 for k_vlimbs
    double *Fg = nullptr;       // k x event groups: cumulative sum of (events / W) over event groups
    double *lossg = nullptr;    // k: sum over event groups of (events) log W, plus (events) c
    double *cmax = nullptr, *csw = nullptr, *suf = nullptr;
    double *lossp = nullptr, *vsp = nullptr;  // k x chunks (lossp: sum of delta eta per chunk)
    double *l1p = nullptr;                    // k x l1 blocks
    double *sumV = nullptr, *f = nullptr, *F = nullptr, *l1 = nullptr;  // k
    double *mub = nullptr;     // k: mu^T beta (cox_eta)
    double *lam = nullptr;     // k
    int *active = nullptr;     // k
    double *Fring = nullptr;   // lag x k
    // split mode
    uint8_t *Bq = nullptr;     // NP x p_pad e4m3 limbs of beta (row LIMBS c + l: limb l of column c)
    uint8_t *Vq = nullptr;     // NP x n_pad e4m3 limbs of V, A4 K order
    int *bs1 = nullptr;        // k: power-of-two scale of the beta limbs
    int *bs4 = nullptr;        // k: power-of-two scale of the V limbs
    float *bmaxp = nullptr;    // k x l1 blocks: partial max |beta|
    double *vmaxp = nullptr;   // k x chunks: partial max |V|
    float *part1 = nullptr;    // slots x k x rows_pad (eta partials)
    float *part4 = nullptr;    // slots x k x rows_pad (X^T V partials)
    int *cnt4 = nullptr;       // per M group of the second product
    // fp64 / gemv
    double *V64 = nullptr;     // k x n
    float *V32 = nullptr;      // n_pad, A4 K order
    float *eta32 = nullptr;    // n
    float *G32 = nullptr;      // p
    float *gpart = nullptr;    // partials of the FP32 baseline's product
    // unpenalised covariates (q > 0)
    double *gamma = nullptr;   // k x q coefficients (column kk at kk q)
    double *gz = nullptr;      // k x q: Z^T (delta - u) / n at the last evaluation
    double *zvp = nullptr;     // k x q x chunks partials
    GemmPlan g1, g4;
    bool plans_ready = false;
    int part1_slots = 0;       // partial slots part1 holds
    // active-set first product (cox_options.active_set)
    GemmPlan g1a;
    bool g1a_ready = false;
    int64_t g1a_K = 0;
    uint8_t *Bqa = nullptr;    // NP x act_Kpad e4m3 limbs of beta at the active SNPs
};

} // namespace coxgb

struct cox_handle {
    int dev = 0, sm_count = 0;
    int64_t n = 0, p = 0, n_pad = 0, p_pad = 0;
    int64_t kperm_a = 1, kperm_nb = 1;  // K order of A4 (a4_pos)
    int64_t kperm_ainv = 1;             // a^-1 mod nb: A4 block B holds sorted block ainv B mod nb
    int n_chunks = 0, l1_blocks = 0;
    cox_options opt;
    int64_t n_groups_tie = 0;
    // sorted order (host copies)
    std::vector<int64_t> h_order;
    std::vector<double> h_mu;
    // device data
    int32_t *d_head = nullptr, *d_tail = nullptr;
    int32_t *d_evhead = nullptr;  // first positions of the tie groups that hold an event
    int32_t *d_evcnt = nullptr;   // events in each of those groups
    int32_t *d_evidx = nullptr;   // n: event groups whose head is at or before the subject's tie tail
    uint8_t *d_evflag = nullptr;  // n: 1 at the head of a tie group that holds an event
    int64_t n_evhead = 0;
    int q = 0;                    // unpenalised covariates
    double *d_Z = nullptr;        // q x n, sorted order
    // active set of the first product (active.cu)
    uint8_t *d_inA = nullptr, *d_flag = nullptr;  // p: in the active set; in the current support
    uint8_t *d_near = nullptr;    // p: pre-threshold value within a quarter of the threshold
    int32_t *d_Aidx = nullptr;    // active SNPs, ascending
    uint32_t *d_A1act = nullptr;  // subject-major 2-bit copy of the active columns
    unsigned long long *d_actcnt = nullptr;
    int64_t nA = -1, act_cap = 0, act_Kpad = 0, act_rebuilds = 0;
    std::vector<int32_t> h_Aidx;  // the active set (host copy)
    uint8_t *d_delta = nullptr;
    double *d_mu = nullptr;
    uint32_t *d_A1 = nullptr;  // subject-major 2-bit tiles
    uint32_t *d_A4 = nullptr;  // SNP-major 2-bit tiles
    double *d_Xr = nullptr;    // FP64: n x p, sorted rows
    double *d_Xc = nullptr;    // FP64: p x n (columns), sorted subjects
    int *d_err = nullptr;
    int64_t device_bytes = 0;
    long long wait_cycles = 0;
    coxgb::Workspace ws;
    // path / checkpoint state
    int st_k = 0;
    std::vector<float> st_beta32;
    std::vector<double> st_beta64;
    std::vector<int> st_iters;
    std::vector<double> st_F;
    std::vector<int> st_active;
    std::vector<double> st_gamma;  // q x k
    int64_t st_step = 0;
    // autotuned pipeline shapes per k: row tiles, K chunks, stages of each product
    struct TuneChoice {
        int T1, CH1, S1, A1, T4, CH4, S4, A4;  // A: issue mode (1 per tile, 2 alternating)
    };
    std::map<int, TuneChoice> tuned;
    // launch accounting and optional per-kernel-class event timing
    int64_t launches = 0;
    bool prof = false;
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

// The e2m1 form of the tensor-core products (COX_SPLIT_E2M1).
inline bool is_e2m1(const cox_handle *h) { return h->opt.precision == COX_SPLIT_E2M1; }

namespace coxgb {

// ---- error helpers ----------------------------------------------------------
int cuda_status(cudaError_t e);
#define COX_CUDA(x)                                      \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return coxgb::cuda_status(e_); \
    } while (0)
#define COX_TRY(x)            \
    do {                      \
        int r_ = (x);         \
        if (r_ != COX_OK) return r_; \
    } while (0)

int dmalloc(cox_handle *h, void **p, size_t bytes);
void dfree(void *p);

// ---- setup (setup.cu) ----------------------------------------------------------
int setup_genotypes(cox_handle *h, const void *X, int x_format, cudaStream_t st);
int setup_dense64(cox_handle *h, const double *X, cudaStream_t st);

// ---- workspace / plans / one iteration (api.cu) ----------------------------------
int ensure_workspace(cox_handle *h, int k);
int iterate(cox_handle *h, void *beta, int k, int epi, void *grad, double step, cudaStream_t st);
int iterate_from_eta(cox_handle *h, void *beta, const double *eta, int k, double step, cudaStream_t st);
struct ScanArgs;
void set_covariate_args(cox_handle *h, ScanArgs &sa, int col, int epi, double step);

// ---- scans (scans.cu) -------------------------------------------------------------
// Risk-set scans on eta (sorted order, k columns).  eta_src kinds:
enum EtaSrc { ETA_PARTIAL_F32 = 0, ETA_DENSE_F64 = 1, ETA_DENSE_F32 = 2 };
enum VOut { V_LIMBS_E4M3 = 0, V_DENSE_F64 = 1, V_DENSE_F32 = 2 };
struct ScanArgs {
    int k;
    int eta_src;
    const void *eta;      // partial f32 [slot][k][rows_pad] or dense [k][n]
    int64_t slot_stride, col_stride;  // partial layout
    int group_rows, KC;   // partial slot counts: group of a row, K chunks, L
    int64_t L;
    int v_out;
    void *V;              // e4m3 limbs [NP][n_pad] (scales in ws.bs4) or dense
    int NP;
    bool exp64;           // exp in FP64 (FP64 mode) or FP32
    const double *lam;    // k (objective); may be null
    bool need_loss;
    bool eta_only = false;  // stop after eta (cox_eta)
    // unpenalised covariates (the handle's q > 0): gamma (k x q, read for eta,
    // updated when gamma_step), gz (k x q out: Z^T (delta - u) / n), active (k)
    double *gamma = nullptr;
    double *gz = nullptr;
    const int *active = nullptr;
    double step = 0.0;
    bool gamma_step = false;
};
int run_scans(cox_handle *h, const ScanArgs &a, cudaStream_t st);

// ---- tensor-core products (gemm_tc.cu) ---------------------------------------------
// Plan one product; T_req / CH_req / stages_req of 0 take the defaults.
// The shape and depth arithmetic of a product plan (host only, no device):
// T, CH, NP, stages, ring, nb_period and smem of g, or COX_ERR_ARG for a shape
// not compiled for k or a depth the pipeline does not allow.
// issue_req: 0 default, 1 one issuer per row tile, 2 two issuers on alternate
// stages, 3 one issuer per row tile committing after every second stage.
int plan_shape(GemmPlan &g, int k, int T_req, int CH_req, int stages_req, int issue_req, int f4);
int plan_gemm(cox_handle *h, GemmPlan &g, const uint32_t *A, int64_t rows_pad, int64_t K_pad,
              const uint8_t *B, int k, int T_req, int CH_req, int stages_req, int issue_req);
// The compiled (row tiles, K chunks, issue mode) shapes for k columns; returns
// their count.
int gemm_shapes(int k, int *T, int *CH, int *issue, int max, int f4);
enum Epi { EPI_PARTIAL = 0, EPI_PROX = 1, EPI_GRAD = 2 };
struct EpiArgs {
    int epi = EPI_PARTIAL;
    float *part = nullptr;
    int *counters = nullptr;
    float *beta = nullptr;   // p x k (prox: in/out)
    float *grad = nullptr;   // p x k (grad output)
    const double *lam = nullptr;
    double step = 0;
    const double *mu = nullptr;
    const double *sumV = nullptr;
    const int *active = nullptr;
    uint8_t *near = nullptr;      // p: set where |z| > 3/4 of the threshold (active set's headroom)
    const int *bscale = nullptr;  // k: power-of-two scale of the B limbs
    int64_t rows_valid = 0;  // p
    double inv_n = 0;
};
int launch_gemm(cox_handle *h, const GemmPlan &g, const EpiArgs &e, int k, cudaStream_t st);
int prep_limbs_beta(cox_handle *h, const float *beta, int k, cudaStream_t st);

// ---- active-set first product (active.cu) -------------------------------------------
int active_prepare(cox_handle *h, const float *beta, int k, cudaStream_t st, int *use);
void active_free(cox_handle *h);

// ---- CUDA-core paths (gemv.cu) -----------------------------------------------------
// ||beta_c||_1 partials into ws.l1p; with maxp, max |beta_c| partials too
int l1_norms32(cox_handle *h, const float *beta, int k, cudaStream_t st, float *maxp = nullptr);
int l1_norms64(cox_handle *h, const double *beta, int k, cudaStream_t st);
int gemv_tiles(cox_handle *h, const uint32_t *A, int64_t rows, int64_t KC, const float *x,
               int64_t K_valid, float *y, cudaStream_t st);
// The FP32 baseline's product y = A x (byte tables of x; part: the partials,
// gemv_lut_part_floats(rows, KC) floats).  Two kernels.
int gemv_lut(cox_handle *h, const uint32_t *A, int64_t rows, int64_t KC, const float *x, int64_t K_valid,
             float *part, float *y, cudaStream_t st);
size_t gemv_lut_part_floats(int64_t rows_pad, int64_t KC);
int gemv_lut_plan(int64_t rows_pad, int64_t KC, int sm_count, int *n_ranges, int64_t *tiles_per_split, int *grid);
int prox_or_grad32(cox_handle *h, const float *G, int col, float *beta, float *grad,
                   const double *lam, double step, cudaStream_t st);
int eta64(cox_handle *h, const double *beta, int k, double *eta, cudaStream_t st);
int xtv64(cox_handle *h, const double *V, int k, double *beta, double *grad, const double *lam,
          double step, cudaStream_t st);
int center_fix_vec(cox_handle *h, const float *v_in, float *a_out, int64_t len, double sub,
                   cudaStream_t st);
// out (k x n) = ws.eta - mu^T beta per column: X_c beta from the uncentred eta
int eta_centred_out(cox_handle *h, const void *beta, bool f64, int k, double *out, cudaStream_t st);

} // namespace coxgb
