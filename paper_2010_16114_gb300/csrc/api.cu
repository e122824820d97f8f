// api.cu -- the C ABI of libcoxgb: handle life cycle, one proximal-gradient
// iteration (arXiv 2010.16114, Section 5.3), loss and gradient, the power
// method for the step (Section 4.4), the batched path fit with the lag-10
// stopping rule (Section 6) replayed as a CUDA graph, and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace coxgb {

int cuda_status(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return COX_ERR_OOM;
    }
    return COX_ERR_CUDA;
}

int dmalloc(cox_handle *h, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? COX_ERR_OOM : COX_ERR_CUDA;
    }
    if (h) h->device_bytes += static_cast<int64_t>(bytes);
    return COX_OK;
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

namespace {

template <typename T>
int alloc(cox_handle *h, T *&p, size_t count)
{
    void *v = nullptr;
    int r = dmalloc(h, &v, count * sizeof(T));
    p = static_cast<T *>(v);
    return r;
}

void free_workspace(cox_handle *h)
{
    Workspace &w = h->ws;
    void *ptrs[] = {w.eta, w.w, w.Rt, w.Fg, w.lossg, w.cmax, w.csw, w.suf, w.lossp, w.vsp, w.l1p,
                    w.sumV, w.f, w.F, w.l1, w.mub, w.lam, w.active, w.Fring, w.Bq, w.Vq, w.bs1, w.bs4, w.bmaxp,
                    w.vmaxp, w.part1, w.part4, w.cnt4, w.V64, w.V32, w.eta32, w.G32, w.gpart, w.gamma, w.gz, w.zvp};
    for (void *p : ptrs) dfree(p);
    dfree(w.Bqa);
    const GemmPlan g1 = w.g1, g4 = w.g4;
    (void)g1;
    (void)g4;
    h->ws = Workspace();
}

int check_device_error(cox_handle *h, cudaStream_t st)
{
    int e = 0;
    COX_CUDA(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    COX_CUDA(cudaStreamSynchronize(st));
    if (e) {
        COX_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
        COX_CUDA(cudaStreamSynchronize(st));
        if (e & DEVERR_TIMEOUT) return COX_ERR_TIMEOUT;
        if (e & DEVERR_NONFINITE) return COX_ERR_NONFINITE;
        if (e & DEVERR_CODE3) return COX_ERR_CODE3;
    }
    return COX_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool is_split(const cox_handle *h) { return h->opt.precision == COX_SPLIT_E4M3 || is_e2m1(h); }
bool is_fp64(const cox_handle *h) { return h->opt.precision == COX_FP64; }
// tuned shapes are kept per operand form and k (switching forms keeps both)
int tune_key(const cox_handle *h, int k) { return is_e2m1(h) ? k + 4096 : k; }
// largest k of the tensor-core products: 128 e2m1 limb columns hold 16 coefficients
int max_k_tc(const cox_handle *h) { return is_e2m1(h) ? MAX_K_E2M1 : MAX_K_TC; }

cudaEvent_t get_event(cox_handle *h)
{
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// Counts the kernels of one launch site and, when profiling, brackets them
// with events on the launching stream.
struct Site {
    cox_handle *h;
    int cls, nk;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Site(cox_handle *h_, int cls_, int nk_, cudaStream_t st_) : h(h_), cls(cls_), nk(nk_), st(st_)
    {
        h->launches += nk;
        if (h->prof && (a = get_event(h))) cudaEventRecord(a, st);
    }
    ~Site()
    {
        if (!h->prof || !a) return;
        cudaEvent_t b = get_event(h);
        if (!b) return;
        cudaEventRecord(b, st);
        h->prof_recs.push_back({cls * 1000 + nk, a, b});
    }
};

} // namespace

// The unpenalised block of the iteration for columns from `col` on: gamma
// enters eta, and a step (EPI_PROX) moves it by step Z^T (delta - u) / n.
void set_covariate_args(cox_handle *h, ScanArgs &sa, int col, int epi, double step)
{
    Workspace &ws = h->ws;
    if (h->q == 0) return;
    sa.gamma = ws.gamma + static_cast<int64_t>(col) * h->q;
    sa.gz = ws.gz + static_cast<int64_t>(col) * h->q;
    sa.active = ws.active + col;
    sa.step = step;
    sa.gamma_step = epi == EPI_PROX;
}

// One iteration for k columns.  epi: EPI_PROX (update beta) or EPI_GRAD.
int iterate(cox_handle *h, void *beta, int k, int epi, void *grad, double step, cudaStream_t st)
{
    Workspace &ws = h->ws;
    if (is_split(h)) {
        float *b32 = static_cast<float *>(beta);
        int use_active = 0;
        {
            Site s_(h, 3, 1, st);
            COX_TRY(l1_norms32(h, b32, k, st, ws.bmaxp));
            if (h->opt.active_set) COX_TRY(active_prepare(h, b32, k, st, &use_active));
            if (!use_active) {
                COX_TRY(prep_limbs_beta(h, b32, k, st));
                h->launches += 1;
            }
        }
        const GemmPlan &g1 = use_active ? ws.g1a : ws.g1;
        EpiArgs e1;
        e1.epi = EPI_PARTIAL;
        e1.part = ws.part1;
        e1.bscale = ws.bs1;
        {
            Site s_(h, 0, 1, st);
            COX_TRY(launch_gemm(h, g1, e1, k, st));
        }
        ScanArgs sa;
        sa.k = k;
        sa.eta_src = ETA_PARTIAL_F32;
        sa.eta = ws.part1;
        sa.slot_stride = static_cast<int64_t>(k) * h->n_pad;
        sa.col_stride = h->n_pad;
        sa.group_rows = g1.T * TILE;
        sa.KC = g1.KC;
        sa.L = g1.L;
        sa.v_out = V_LIMBS_E4M3;
        sa.V = ws.Vq;
        sa.NP = ws.g4.NP;
        sa.exp64 = false;
        sa.lam = ws.lam;
        sa.need_loss = true;
        set_covariate_args(h, sa, 0, epi, step);
        {
            Site s_(h, 2, 8, st);
            COX_TRY(run_scans(h, sa, st));
        }
        EpiArgs e4;
        e4.epi = epi;
        e4.part = ws.part4;
        e4.counters = ws.cnt4;
        e4.beta = epi == EPI_PROX ? b32 : nullptr;
        e4.grad = epi == EPI_GRAD ? static_cast<float *>(grad) : nullptr;
        e4.lam = ws.lam;
        e4.step = step;
        e4.mu = h->d_mu;
        e4.sumV = ws.sumV;
        e4.active = ws.active;
        e4.near = (h->opt.active_set && epi == EPI_PROX) ? h->d_near : nullptr;
        e4.bscale = ws.bs4;
        e4.rows_valid = h->p;
        e4.inv_n = 1.0 / static_cast<double>(h->n);
        {
            Site s_(h, 1, 1, st);
            COX_TRY(launch_gemm(h, ws.g4, e4, k, st));
        }
        return COX_OK;
    }
    if (is_fp64(h)) {
        double *b64 = static_cast<double *>(beta);
        {
            Site s_(h, 3, 1, st);
            COX_TRY(l1_norms64(h, b64, k, st));
        }
        {
            Site s_(h, 0, 1, st);
            COX_TRY(eta64(h, b64, k, ws.eta, st));
        }
        ScanArgs sa;
        sa.k = k;
        sa.eta_src = ETA_DENSE_F64;
        sa.eta = ws.eta;
        sa.slot_stride = 0;
        sa.col_stride = h->n;
        sa.group_rows = 1;
        sa.KC = 1;
        sa.L = 1;
        sa.v_out = V_DENSE_F64;
        sa.V = ws.V64;
        sa.NP = 0;
        sa.exp64 = true;
        sa.lam = ws.lam;
        sa.need_loss = true;
        set_covariate_args(h, sa, 0, epi, step);
        {
            Site s_(h, 2, 8, st);
            COX_TRY(run_scans(h, sa, st));
        }
        Site s4_(h, 1, 1, st);
        COX_TRY(xtv64(h, ws.V64, k, epi == EPI_PROX ? b64 : nullptr, epi == EPI_GRAD ? static_cast<double *>(grad) : nullptr,
                      ws.lam, step, st));
        return COX_OK;
    }
    // plain FP32 baseline: one column at a time, unfused
    float *b32 = static_cast<float *>(beta);
    for (int c = 0; c < k; ++c) {
        float *bc = b32 + static_cast<int64_t>(c) * h->p;
        {
            Site s_(h, 3, 1, st);
            COX_TRY(l1_norms32(h, bc, 1, st));
        }
        {
            Site s_(h, 0, 2, st);
            COX_TRY(gemv_lut(h, h->d_A1, h->n_pad, h->p_pad / TILE, bc, h->p, ws.gpart, ws.eta32, st));
        }
        ScanArgs sa;
        sa.k = 1;
        sa.eta_src = ETA_DENSE_F32;
        sa.eta = ws.eta32;
        sa.slot_stride = 0;
        sa.col_stride = h->n_pad;
        sa.group_rows = 1;
        sa.KC = 1;
        sa.L = 1;
        sa.v_out = V_DENSE_F32;
        sa.V = ws.V32;
        sa.NP = 0;
        sa.exp64 = false;
        sa.lam = ws.lam + c;
        sa.need_loss = true;
        set_covariate_args(h, sa, c, epi, step);
        {
            Site s_(h, 2, 8, st);
            COX_TRY(run_scans(h, sa, st));
        }
        COX_CUDA(cudaMemcpyAsync(ws.Fring + c, ws.F, sizeof(double), cudaMemcpyDeviceToDevice, st));
        COX_CUDA(cudaMemcpyAsync(ws.Fring + k + c, ws.f, sizeof(double), cudaMemcpyDeviceToDevice, st));
        {
            Site s_(h, 1, 3, st);
            COX_TRY(gemv_lut(h, h->d_A4, h->p_pad, h->n_pad / TILE, ws.V32, h->n_pad, ws.gpart, ws.G32, st));
            float *gc = epi == EPI_GRAD ? static_cast<float *>(grad) : nullptr;
            COX_TRY(prox_or_grad32(h, ws.G32, c, epi == EPI_PROX ? b32 : nullptr, gc, ws.lam, step, st));
        }
    }
    // gather per-column objectives into F / f
    COX_CUDA(cudaMemcpyAsync(ws.F, ws.Fring, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    COX_CUDA(cudaMemcpyAsync(ws.f, ws.Fring + k, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return COX_OK;
}

// One iteration of a column shard from the linear predictor summed over all
// shards (Section 5.3 with X split by columns): eta (k x n doubles, sorted
// order, X part only; the handle adds Z gamma when covariates are set), the
// replicated risk-set scans, then this shard's X_g^T V and the soft-threshold
// step on its coefficients.
int iterate_from_eta(cox_handle *h, void *beta, const double *eta, int k, double step, cudaStream_t st)
{
    Workspace &ws = h->ws;
    ScanArgs sa;
    sa.k = k;
    sa.eta_src = ETA_DENSE_F64;
    sa.eta = eta;
    sa.slot_stride = 0;
    sa.col_stride = h->n;
    sa.group_rows = 1;
    sa.KC = 1;
    sa.L = 1;
    sa.lam = ws.lam;
    sa.need_loss = true;
    set_covariate_args(h, sa, 0, EPI_PROX, step);
    if (is_split(h)) {
        float *b32 = static_cast<float *>(beta);
        {
            Site s_(h, 3, 1, st);
            COX_TRY(l1_norms32(h, b32, k, st));
        }
        sa.v_out = V_LIMBS_E4M3;
        sa.V = ws.Vq;
        sa.NP = ws.g4.NP;
        sa.exp64 = false;
        {
            Site s_(h, 2, 8, st);
            COX_TRY(run_scans(h, sa, st));
        }
        EpiArgs e4;
        e4.epi = EPI_PROX;
        e4.part = ws.part4;
        e4.counters = ws.cnt4;
        e4.beta = b32;
        e4.lam = ws.lam;
        e4.step = step;
        e4.mu = h->d_mu;
        e4.sumV = ws.sumV;
        e4.active = ws.active;
        e4.bscale = ws.bs4;
        e4.rows_valid = h->p;
        e4.inv_n = 1.0 / static_cast<double>(h->n);
        Site s_(h, 1, 1, st);
        return launch_gemm(h, ws.g4, e4, k, st);
    }
    if (is_fp64(h)) {
        double *b64 = static_cast<double *>(beta);
        {
            Site s_(h, 3, 1, st);
            COX_TRY(l1_norms64(h, b64, k, st));
        }
        sa.v_out = V_DENSE_F64;
        sa.V = ws.V64;
        sa.exp64 = true;
        {
            Site s_(h, 2, 8, st);
            COX_TRY(run_scans(h, sa, st));
        }
        Site s4_(h, 1, 1, st);
        return xtv64(h, ws.V64, k, b64, nullptr, ws.lam, step, st);
    }
    return COX_ERR_UNSUPPORTED;
}

namespace {

int validate_k(const cox_handle *h, int k)
{
    if (k < 1) return COX_ERR_ARG;
    if (is_split(h) && k > max_k_tc(h)) return COX_ERR_ARG;
    if (k > 1024) return COX_ERR_ARG;
    return COX_OK;
}

int set_lambdas(cox_handle *h, const double *lambdas, int k, cudaStream_t st)
{
    if (!lambdas) return COX_ERR_ARG;
    for (int c = 0; c < k; ++c)
        if (!(lambdas[c] >= 0.0) || !std::isfinite(lambdas[c])) return COX_ERR_ARG;
    COX_CUDA(cudaMemcpyAsync(h->ws.lam, lambdas, k * sizeof(double), cudaMemcpyHostToDevice, st));
    return COX_OK;
}

int set_all_active(cox_handle *h, int k, cudaStream_t st)
{
    std::vector<int> one(static_cast<size_t>(k), 1);
    COX_CUDA(cudaMemcpyAsync(h->ws.active, one.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    COX_CUDA(cudaStreamSynchronize(st));
    return COX_OK;
}

} // namespace

int ensure_workspace(cox_handle *h, int k)
{
    Workspace &ws = h->ws;
    if (ws.k == k) return COX_OK;
    free_workspace(h);
    const int64_t n = h->n, p = h->p, nch = h->n_chunks;
    const int lag = std::max(1, h->opt.lag);
    int r = COX_OK;
#define A(ptr, cnt)                                 \
    if ((r = alloc(h, ptr, (cnt))) != COX_OK) { \
        free_workspace(h);                          \
        return r;                                   \
    }
    A(ws.eta, k * n);
    A(ws.w, k * n);
    A(ws.Rt, k * n);
    A(ws.Fg, k * std::max<int64_t>(1, h->n_evhead));
    A(ws.lossg, k);
    A(ws.cmax, k * nch);
    A(ws.csw, k * nch);
    A(ws.suf, k * nch);
    A(ws.lossp, k * nch);
    A(ws.vsp, k * nch);
    A(ws.l1p, static_cast<size_t>(k) * h->l1_blocks);
    A(ws.sumV, k);
    A(ws.f, k);
    A(ws.F, k);
    A(ws.l1, k);
    A(ws.mub, k);
    A(ws.lam, k);
    A(ws.active, k);
    A(ws.Fring, static_cast<size_t>(std::max(lag, 2)) * k);
    if (h->q > 0) {
        A(ws.gamma, static_cast<size_t>(k) * h->q);
        A(ws.gz, static_cast<size_t>(k) * h->q);
        A(ws.zvp, static_cast<size_t>(k) * h->q * nch);
        cudaMemset(ws.gamma, 0, static_cast<size_t>(k) * h->q * sizeof(double));
    }
    if (is_split(h)) {
        // limb rows of K_pad e4m3 bytes, or K_pad / 2 bytes of e2m1 pairs
        const int NP = is_e2m1(h) ? limb_cols4(k) : limb_cols(k);
        const int64_t bpk = is_e2m1(h) ? 2 : 1;  // K positions per byte
        A(ws.Bq, static_cast<size_t>(NP) * h->p_pad / bpk);
        A(ws.Vq, static_cast<size_t>(NP) * h->n_pad / bpk);
        A(ws.bs1, k);
        A(ws.bs4, k);
        A(ws.bmaxp, static_cast<size_t>(k) * h->l1_blocks);
        A(ws.vmaxp, k * nch);
        // limb rows past LIMBS k and K positions of padding stay zero
        cudaMemset(ws.Bq, 0, static_cast<size_t>(NP) * h->p_pad / bpk);
        cudaMemset(ws.Vq, 0, static_cast<size_t>(NP) * h->n_pad / bpk);
        ws.NP = NP;
        cudaMemset(ws.bs1, 0, k * sizeof(int));
        cudaMemset(ws.bs4, 0, k * sizeof(int));
        // pipeline shapes: forced by the options, else autotuned for k, else default
        int T1 = h->opt.tile_m, C1 = h->opt.chunks, S1 = h->opt.stages, A1 = h->opt.issue;
        int T4 = T1, C4 = C1, S4 = S1, A4 = A1;
        const auto tc = h->tuned.find(tune_key(h, k));
        if (tc != h->tuned.end() && !T1 && !C1 && !S1 && !A1) {
            T1 = tc->second.T1, C1 = tc->second.CH1, S1 = tc->second.S1, A1 = tc->second.A1;
            T4 = tc->second.T4, C4 = tc->second.CH4, S4 = tc->second.S4, A4 = tc->second.A4;
        }
        if ((r = plan_gemm(h, ws.g1, h->d_A1, h->n_pad, h->p_pad, ws.Bq, k, T1, C1, S1, A1)) != COX_OK ||
            (r = plan_gemm(h, ws.g4, h->d_A4, h->p_pad, h->n_pad, ws.Vq, k, T4, C4, S4, A4)) != COX_OK) {
            free_workspace(h);
            return r;
        }
        A(ws.part1, static_cast<size_t>(ws.g1.max_slots) * k * h->n_pad);
        ws.part1_slots = ws.g1.max_slots;
        A(ws.part4, static_cast<size_t>(ws.g4.max_slots) * k * h->p_pad);
        A(ws.cnt4, static_cast<size_t>(ws.g4.n_groups));
        cudaMemset(ws.cnt4, 0, static_cast<size_t>(ws.g4.n_groups) * sizeof(int));
    } else if (is_fp64(h)) {
        A(ws.V64, k * n);
    } else {
        A(ws.V32, h->n_pad);  // A4 K order; positions of padding stay zero
        cudaMemset(ws.V32, 0, h->n_pad * sizeof(float));
        A(ws.eta32, h->n_pad);
        A(ws.G32, h->p_pad);
        A(ws.gpart, std::max(gemv_lut_part_floats(h->n_pad, h->p_pad / TILE),
                             gemv_lut_part_floats(h->p_pad, h->n_pad / TILE)));
    }
#undef A
    (void)p;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_workspace(h);
        return COX_ERR_CUDA;
    }
    ws.k = k;
    return set_all_active(h, k, 0);
}

} // namespace coxgb

using namespace coxgb;

extern "C" {

void cox_default_options(cox_options *opt)
{
    if (!opt) return;
    opt->precision = COX_SPLIT_E4M3;
    opt->center = 1;
    opt->device = -1;
    opt->tile_m = 0;
    opt->stages = 0;
    opt->chunks = 0;
    opt->window = 0;
    opt->issue = 0;
    opt->active_set = 0;
    opt->lag = 10;
    opt->wait_limit_s = 2.0;
}

const char *cox_strerror(int code)
{
    switch (code) {
    case COX_OK: return "ok";
    case COX_ERR_ARG: return "invalid argument";
    case COX_ERR_CODE3: return "genotype code outside {0,1,2}";
    case COX_ERR_OOM: return "out of memory";
    case COX_ERR_CUDA: return "CUDA runtime error";
    case COX_ERR_TIMEOUT: return "device-side wait timed out";
    case COX_ERR_NONFINITE: return "non-finite value in eta, W or the loss";
    case COX_ERR_NOT_CONVERGED: return "some column reached max_iter before the stopping rule";
    case COX_ERR_STATE: return "state blob does not match the handle";
    case COX_ERR_UNSUPPORTED: return "unsupported device or mode";
    default: return "unknown error";
    }
}

void cox_destroy(cox_h h)
{
    if (!h) return;
    DeviceGuard g(h->dev);
    cudaDeviceSynchronize();
    free_workspace(h);
    active_free(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    void *ptrs[] = {h->d_head, h->d_tail, h->d_evhead, h->d_evcnt, h->d_evidx, h->d_evflag, h->d_delta,
                    h->d_mu, h->d_A1, h->d_A4, h->d_Xr, h->d_Xc, h->d_err, h->d_Z};
    for (void *p : ptrs) dfree(p);
    delete h;
}

int cox_setup(cox_h *out, const void *X, int64_t n, int64_t p, int x_format, const double *time,
              const uint8_t *event, const cox_options *opt_in)
{
    if (!out) return COX_ERR_ARG;
    *out = nullptr;
    cox_options opt;
    cox_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (!X || !time || !event || n < 1 || p < 1 || n > INT32_MAX || p > INT32_MAX) return COX_ERR_ARG;
    if (opt.precision != COX_SPLIT_E4M3 && opt.precision != COX_FP64 && opt.precision != COX_FP32_GEMV &&
        opt.precision != COX_SPLIT_E2M1)
        return COX_ERR_ARG;
    if ((opt.precision == COX_FP64) != (x_format == COX_X_F64_HOST)) return COX_ERR_UNSUPPORTED;
    if (x_format < COX_X_INT8_HOST || x_format > COX_X_PACKED2_DEV) return COX_ERR_ARG;
    if (opt.lag < 1 || !(opt.wait_limit_s >= 0.0)) return COX_ERR_ARG;
    if (opt.tile_m < 0 || opt.tile_m > 2 || opt.chunks < 0 || opt.chunks > 4 || opt.stages < 0 || opt.window < 0 ||
        opt.issue < 0 || opt.issue > 3 || opt.active_set < 0 || opt.active_set > 1)
        return COX_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(time[i])) return COX_ERR_ARG;
        if (event[i] > 1) return COX_ERR_ARG;
    }
    int dev = opt.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return COX_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return COX_ERR_UNSUPPORTED;
    }
    if (prop.major != 10 || prop.minor != 3) return COX_ERR_UNSUPPORTED;
    DeviceGuard guard(dev);

    cox_handle *h = new cox_handle();
    h->dev = dev;
    h->sm_count = prop.multiProcessorCount;
    h->opt = opt;
    h->n = n;
    h->p = p;
    h->n_pad = (n + PAD - 1) / PAD * PAD;
    h->p_pad = (p + PAD - 1) / PAD * PAD;
    h->n_chunks = static_cast<int>((n + SCAN_CH - 1) / SCAN_CH);
    {
        // A4 K order: multiplier near nb (sqrt 5 - 1) / 2, odd, prime to nb
        const int64_t nb = h->n_pad / 16;
        int64_t a = static_cast<int64_t>(std::llround(0.6180339887498949 * static_cast<double>(nb))) | 1;
        while (std::gcd(a, nb) != 1) a += 2;
        h->kperm_nb = nb;
        h->kperm_a = a % nb;
        // inverse of a modulo nb (extended Euclid; a is prime to nb)
        int64_t r0 = nb, r1 = h->kperm_a, t0 = 0, t1 = 1;
        while (r1 != 0) {
            const int64_t q = r0 / r1, r2 = r0 - q * r1, t2 = t0 - q * t1;
            r0 = r1;
            r1 = r2;
            t0 = t1;
            t1 = t2;
        }
        h->kperm_ainv = ((t0 % nb) + nb) % nb;
    }
    h->l1_blocks = static_cast<int>(std::min<int64_t>(64, (p + 4095) / 4096));
    {
        int khz = 0;
        if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
            cudaGetLastError();
            khz = 2100000;  // GB300 boost clock ceiling, 2.07 GHz
        }
        h->wait_cycles = static_cast<long long>(opt.wait_limit_s * static_cast<double>(khz) * 1000.0);
    }

    // stable sort by time; Breslow tie groups
    h->h_order.resize(static_cast<size_t>(n));
    std::iota(h->h_order.begin(), h->h_order.end(), 0);
    std::stable_sort(h->h_order.begin(), h->h_order.end(), [&](int64_t a, int64_t b) { return time[a] < time[b]; });
    std::vector<int32_t> head(static_cast<size_t>(n)), tail(static_cast<size_t>(n));
    std::vector<uint8_t> dsorted(static_cast<size_t>(n));
    int64_t groups = 0;
    std::vector<int32_t> evhead;  // heads of the tie groups with at least one event
    std::vector<int32_t> evcnt;   // and their event counts
    std::vector<int32_t> evidx(static_cast<size_t>(n));  // event groups with head <= the subject's tail
    std::vector<uint8_t> evflag(static_cast<size_t>(n), 0);
    for (int64_t r = 0; r < n;) {
        int64_t e = r;
        while (e + 1 < n && time[h->h_order[e + 1]] == time[h->h_order[r]]) ++e;
        int32_t nev = 0;
        for (int64_t s = r; s <= e; ++s) {
            head[s] = static_cast<int32_t>(r);
            tail[s] = static_cast<int32_t>(e);
            nev += event[h->h_order[s]] != 0;
        }
        if (nev) {
            evhead.push_back(static_cast<int32_t>(r));
            evcnt.push_back(nev);
            evflag[r] = 1;
        }
        for (int64_t s = r; s <= e; ++s) evidx[s] = static_cast<int32_t>(evhead.size());
        ++groups;
        r = e + 1;
    }
    h->n_evhead = static_cast<int64_t>(evhead.size());
    for (int64_t r = 0; r < n; ++r) dsorted[r] = event[h->h_order[r]];
    h->n_groups_tie = groups;

    cudaStream_t st = 0;
    int rc = COX_OK;
    do {
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_err), sizeof(int))) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_head), n * sizeof(int32_t))) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_tail), n * sizeof(int32_t))) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_evhead), evhead.size() * sizeof(int32_t))) != COX_OK)
            break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_evcnt), evcnt.size() * sizeof(int32_t))) != COX_OK)
            break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_evidx), n * sizeof(int32_t))) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_evflag), n)) != COX_OK) break;
        if ((!evhead.empty() &&
             (cudaMemcpy(h->d_evhead, evhead.data(), evhead.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
                  cudaSuccess ||
              cudaMemcpy(h->d_evcnt, evcnt.data(), evcnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
                  cudaSuccess)) ||
            cudaMemcpy(h->d_evidx, evidx.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->d_evflag, evflag.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_delta), n)) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_mu), p * sizeof(double))) != COX_OK) break;
        if (cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess ||
            cudaMemcpy(h->d_head, head.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->d_tail, tail.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->d_delta, dsorted.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        if (opt.precision == COX_FP64) rc = setup_dense64(h, static_cast<const double *>(X), st);
        else rc = setup_genotypes(h, X, x_format, st);
        if (rc != COX_OK) break;
        if (cudaMemcpy(h->d_mu, h->h_mu.data(), p * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
    } while (false);
    if (rc != COX_OK) {
        cox_destroy(h);
        return rc;
    }
    *out = h;
    return COX_OK;
}

int cox_get_info(cox_h h, cox_info *info)
{
    if (!h || !info) return COX_ERR_ARG;
    info->n = h->n;
    info->p = h->p;
    info->n_pad = h->n_pad;
    info->p_pad = h->p_pad;
    info->precision = h->opt.precision;
    info->center = h->opt.center;
    info->tile_m = h->ws.k ? h->ws.g1.T : h->opt.tile_m;
    info->stages = h->ws.k ? h->ws.g1.stages : h->opt.stages;
    info->sm_count = h->sm_count;
    info->device_bytes = h->device_bytes;
    info->n_tie_groups = h->n_groups_tie;
    info->launches = h->launches;
    info->chunks = h->ws.k ? h->ws.g1.CH : h->opt.chunks;
    info->ring = h->ws.k ? h->ws.g1.ring : 0;
    info->issue = h->ws.k ? (h->ws.g1.alt ? 2 : h->ws.g1.pair ? 3 : 1) : h->opt.issue;
    info->issue_xtv = h->ws.k ? (h->ws.g4.alt ? 2 : h->ws.g4.pair ? 3 : 1) : h->opt.issue;
    info->active_cols = h->opt.active_set ? h->nA : -1;
    info->active_rebuilds = h->act_rebuilds;
    return COX_OK;
}

int cox_autotune(cox_h h, int k, int reps, cox_tune_choice *xb, cox_tune_choice *xtv)
{
    if (!h) return COX_ERR_ARG;
    if (!is_split(h)) return COX_ERR_UNSUPPORTED;
    if (k < 1 || k > max_k_tc(h) || reps < 1) return COX_ERR_ARG;
    DeviceGuard guard(h->dev);
    h->tuned.erase(tune_key(h, k));
    COX_TRY(ensure_workspace(h, k));  // limb buffers (zero) and scale arrays for the timing launches
    Workspace &ws = h->ws;
    int Ts[16], Cs[16], As[16];
    const int nshape = gemm_shapes(k, Ts, Cs, As, 16, is_e2m1(h));
    // the planner's depth only: four-stage plans measured 2-3x slower for every
    // shape at full size (the bench's workloads), so they are not timed
    const int depth_req[1] = {0};
    cox_tune_choice best[2];
    int cand[2] = {0, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    COX_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return COX_ERR_CUDA;
    }
    int rc = COX_OK;
    for (int prod = 0; prod < 2 && rc == COX_OK; ++prod) {
        best[prod] = cox_tune_choice{0, 0, 0, 0, 1e300, 0};
        const uint32_t *A = prod == 0 ? h->d_A1 : h->d_A4;
        const int64_t rows = prod == 0 ? h->n_pad : h->p_pad, K = prod == 0 ? h->p_pad : h->n_pad;
        const uint8_t *B = prod == 0 ? ws.Bq : ws.Vq;
        for (int j = 0; j < nshape && rc == COX_OK; ++j) {
            int last_S = -1;
            if (As[j] == 3) continue;  // pair commits: not timed (no faster than per-stage commits)
            for (int dq = 0; dq < 1 && rc == COX_OK; ++dq) {
                GemmPlan g;
                if (plan_gemm(h, g, A, rows, K, B, k, Ts[j], Cs[j], depth_req[dq], As[j]) != COX_OK) continue;
                if (g.stages == last_S) continue;  // the two depths coincide
                last_S = g.stages;
                float *part = nullptr;
                if ((rc = dmalloc(nullptr, reinterpret_cast<void **>(&part),
                                  static_cast<size_t>(g.max_slots) * k * rows * sizeof(float))) != COX_OK)
                    break;
                EpiArgs e;
                e.epi = EPI_PARTIAL;
                e.part = part;
                e.bscale = prod == 0 ? ws.bs1 : ws.bs4;
                float ms = 0.f;
                bool good = launch_gemm(h, g, e, k, 0) == COX_OK;
                good = good && cudaEventRecord(e0, 0) == cudaSuccess;
                for (int q = 0; q < reps && good; ++q) good = launch_gemm(h, g, e, k, 0) == COX_OK;
                good = good && cudaEventRecord(e1, 0) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                       cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                h->launches += reps + 1;
                // every candidate's launches complete, and report, before the next is planned
                good = cudaDeviceSynchronize() == cudaSuccess && good;
                dfree(part);
                if (!good) {
                    rc = COX_ERR_CUDA;
                    break;
                }
                if ((rc = check_device_error(h, 0)) != COX_OK) break;
                ++cand[prod];
                const double m = static_cast<double>(ms) / reps;
                if (m < best[prod].ms) best[prod] = cox_tune_choice{g.T, g.CH, g.stages, 0, m, As[j]};
            }
        }
        best[prod].candidates = cand[prod];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != COX_OK) return rc;
    if (!cand[0] || !cand[1]) return COX_ERR_ARG;
    h->tuned[tune_key(h, k)] = cox_handle::TuneChoice{best[0].tile_m, best[0].chunks, best[0].stages, best[0].issue,
                                         best[1].tile_m, best[1].chunks, best[1].stages, best[1].issue};
    cudaDeviceSynchronize();
    free_workspace(h);  // the next call with k columns plans the chosen shapes
    if (xb) *xb = best[0];
    if (xtv) *xtv = best[1];
    return COX_OK;
}

int cox_rank_by_entry(int64_t p, int L, const double *lambdas, const void *B_host, int dbl,
                      int64_t *order_host, int64_t *entry_host, int64_t *count_out)
{
    if (p < 1 || L < 1 || !lambdas || !B_host || !order_host || !entry_host || !count_out) return COX_ERR_ARG;
    for (int l = 0; l < L; ++l)
        if (!std::isfinite(lambdas[l])) return COX_ERR_ARG;
    auto coef = [&](int l, int64_t j) -> double {
        const int64_t at = static_cast<int64_t>(l) * p + j;
        return dbl ? static_cast<const double *>(B_host)[at]
                   : static_cast<double>(static_cast<const float *>(B_host)[at]);
    };
    struct Key {
        int64_t j;
        int entry;
        double mag;
    };
    std::vector<Key> keys;
    for (int64_t j = 0; j < p; ++j) {
        int best = -1;
        for (int l = 0; l < L; ++l)
            if (coef(l, j) != 0.0 && (best < 0 || lambdas[l] > lambdas[best])) best = l;
        entry_host[j] = best;
        if (best >= 0) keys.push_back(Key{j, best, std::fabs(coef(best, j))});
    }
    // the largest entry lambda first; then the larger |beta| on joining; then the index
    std::sort(keys.begin(), keys.end(), [&](const Key &a, const Key &b) {
        if (lambdas[a.entry] != lambdas[b.entry]) return lambdas[a.entry] > lambdas[b.entry];
        if (a.mag != b.mag) return a.mag > b.mag;
        return a.j < b.j;
    });
    for (size_t c = 0; c < keys.size(); ++c) order_host[c] = keys[c].j;
    *count_out = static_cast<int64_t>(keys.size());
    return COX_OK;
}

int cox_plan_shape(int k, int tile_m, int chunks, int stages, int issue, cox_plan *out)
{
    return cox_plan_shape_prec(COX_SPLIT_E4M3, k, tile_m, chunks, stages, issue, out);
}

int cox_plan_shape_prec(int precision, int k, int tile_m, int chunks, int stages, int issue, cox_plan *out)
{
    if (!out || tile_m < 0 || chunks < 0 || stages < 0 || issue < 0 || issue > 3) return COX_ERR_ARG;
    if (precision != COX_SPLIT_E4M3 && precision != COX_SPLIT_E2M1) return COX_ERR_ARG;
    const int f4 = precision == COX_SPLIT_E2M1;
    GemmPlan g;
    COX_TRY(plan_shape(g, k, tile_m, chunks, stages, issue, f4));
    out->tile_m = g.T;
    out->chunks = g.CH;
    out->stages = g.stages;
    out->ring = g.ring;
    out->decoder_groups = g.G;
    out->named_barriers = g.nb_period * g.T;
    out->limb_cols = g.NP;
    out->tmem_cols = (g.alt ? 2 : 1) * g.T * g.NP + g.ring * g.T * g.CH * (f4 ? 16 : 32) + (f4 ? 8 : 0);
    out->smem_bytes = static_cast<long long>(g.smem);
    out->issue = g.alt ? 2 : g.pair ? 3 : 1;
    out->issuers = g.alt ? 2 : g.T;
    out->mmas_per_commit = (f4 ? 2 : 4) * g.CH * (g.alt ? g.T : g.pair ? 2 : 1);
    out->limb_stages = f4 ? g.stages2 : 0;
    return COX_OK;
}

int cox_set_precision(cox_h h, int precision)
{
    if (!h) return COX_ERR_ARG;
    if (h->opt.precision == COX_FP64 ||
        (precision != COX_SPLIT_E4M3 && precision != COX_FP32_GEMV && precision != COX_SPLIT_E2M1))
        return COX_ERR_UNSUPPORTED;
    if (precision == h->opt.precision) return COX_OK;
    DeviceGuard g(h->dev);
    cudaDeviceSynchronize();
    free_workspace(h);
    h->opt.precision = precision;
    return COX_OK;
}

int cox_set_active_set(cox_h h, int on)
{
    if (!h || on < 0 || on > 1) return COX_ERR_ARG;
    h->opt.active_set = on;
    return COX_OK;
}

int cox_profile(cox_h h, int enable)
{
    if (!h) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    if (enable) {
        cudaDeviceSynchronize();
        h->prof_recs.clear();
        h->ev_used = 0;
    }
    h->prof = enable != 0;
    return COX_OK;
}

int cox_profile_read(cox_h h, double *total_ms, int64_t *launches)
{
    if (!h || !total_ms || !launches) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    for (int c = 0; c < 4; ++c) {
        total_ms[c] = 0.0;
        launches[c] = 0;
    }
    for (const auto &r : h->prof_recs) {
        COX_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        COX_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        const int cls = r.cls / 1000;
        total_ms[cls] += ms;
        launches[cls] += r.cls % 1000;
    }
    return COX_OK;
}

int cox_get_mu_order(cox_h h, double *mu_host, int64_t *order_host)
{
    if (!h) return COX_ERR_ARG;
    if (mu_host) std::memcpy(mu_host, h->h_mu.data(), h->p * sizeof(double));
    if (order_host) std::memcpy(order_host, h->h_order.data(), h->n * sizeof(int64_t));
    return COX_OK;
}

int cox_sync(cox_h h, void *stream)
{
    if (!h) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    return check_device_error(h, static_cast<cudaStream_t>(stream));
}

int cox_loss_grad(cox_h h, const void *beta_dev, int k, double *loss_host, void *grad_dev, void *stream)
{
    if (!h || !beta_dev) return COX_ERR_ARG;
    COX_TRY(validate_k(h, k));
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_TRY(ensure_workspace(h, k));
    std::vector<double> zeros(static_cast<size_t>(k), 0.0);
    COX_TRY(set_lambdas(h, zeros.data(), k, st));
    void *gout = grad_dev;
    void *tmp = nullptr;
    if (!gout) {
        COX_TRY(dmalloc(nullptr, &tmp, static_cast<size_t>(k) * h->p * (is_fp64(h) ? 8 : 4)));
        gout = tmp;
    }
    int rc = iterate(h, const_cast<void *>(beta_dev), k, EPI_GRAD, gout, 0.0, st);
    if (rc == COX_OK) rc = check_device_error(h, st);
    if (rc == COX_OK && loss_host) {
        if (cudaMemcpyAsync(loss_host, h->ws.f, k * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = COX_ERR_CUDA;
    }
    if (tmp) {
        cudaStreamSynchronize(st);
        dfree(tmp);
    }
    return rc;
}

int cox_eta(cox_h h, const void *beta_dev, int k, double *eta_dev, void *stream)
{
    if (!h || !beta_dev || !eta_dev) return COX_ERR_ARG;
    COX_TRY(validate_k(h, k));
    if (h->opt.precision == COX_FP32_GEMV) return COX_ERR_UNSUPPORTED;
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_TRY(ensure_workspace(h, k));
    Workspace &ws = h->ws;
    if (is_split(h)) {
        const float *b32 = static_cast<const float *>(beta_dev);
        COX_TRY(l1_norms32(h, b32, k, st, ws.bmaxp));
        COX_TRY(prep_limbs_beta(h, b32, k, st));
        EpiArgs e1;
        e1.epi = EPI_PARTIAL;
        e1.part = ws.part1;
        e1.bscale = ws.bs1;
        COX_TRY(launch_gemm(h, ws.g1, e1, k, st));
        ScanArgs sa;
        sa.k = k;
        sa.eta_src = ETA_PARTIAL_F32;
        sa.eta = ws.part1;
        sa.slot_stride = static_cast<int64_t>(k) * h->n_pad;
        sa.col_stride = h->n_pad;
        sa.group_rows = ws.g1.T * TILE;
        sa.KC = ws.g1.KC;
        sa.L = ws.g1.L;
        sa.v_out = V_LIMBS_E4M3;
        sa.V = nullptr;
        sa.NP = ws.g4.NP;
        sa.exp64 = false;
        sa.lam = nullptr;
        sa.need_loss = false;
        sa.eta_only = true;
        COX_TRY(run_scans(h, sa, st));
        h->launches += 4;
    } else {
        COX_TRY(eta64(h, static_cast<const double *>(beta_dev), k, ws.eta, st));
        h->launches += 1;
    }
    COX_TRY(eta_centred_out(h, beta_dev, is_fp64(h), k, eta_dev, st));
    h->launches += 2;
    COX_TRY(check_device_error(h, st));
    return COX_OK;
}

int cox_prox_step(cox_h h, void *beta_dev, const double *lambdas, int k, double step, void *stream)
{
    if (!h || !beta_dev || !(step > 0.0) || !std::isfinite(step)) return COX_ERR_ARG;
    COX_TRY(validate_k(h, k));
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_TRY(ensure_workspace(h, k));
    COX_TRY(set_lambdas(h, lambdas, k, st));
    return iterate(h, beta_dev, k, EPI_PROX, nullptr, step, st);
}

int cox_prox_step_host(cox_h h, void *beta_host, const double *lambdas, int k, double step, void *stream)
{
    if (!h || !beta_host) return COX_ERR_ARG;
    COX_TRY(validate_k(h, k));
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = static_cast<size_t>(k) * h->p * (is_fp64(h) ? 8 : 4);
    COX_TRY(ensure_workspace(h, k));
    static thread_local void *dbuf = nullptr;
    static thread_local size_t dcap = 0;
    static thread_local int ddev = -1;
    if (dcap < bytes || ddev != h->dev) {
        if (dbuf) cudaFree(dbuf);
        dbuf = nullptr;
        dcap = 0;
        COX_TRY(dmalloc(nullptr, &dbuf, bytes));
        dcap = bytes;
        ddev = h->dev;
    }
    COX_CUDA(cudaMemcpyAsync(dbuf, beta_host, bytes, cudaMemcpyHostToDevice, st));
    COX_TRY(set_lambdas(h, lambdas, k, st));
    COX_TRY(iterate(h, dbuf, k, EPI_PROX, nullptr, step, st));
    COX_CUDA(cudaMemcpyAsync(beta_host, dbuf, bytes, cudaMemcpyDeviceToHost, st));
    return check_device_error(h, st);
}

int cox_prox_step_eta(cox_h h, void *beta_dev, const double *eta_dev, const double *lambdas, int k, double step,
                      void *stream)
{
    if (!h || !beta_dev || !eta_dev || !(step > 0.0) || !std::isfinite(step)) return COX_ERR_ARG;
    COX_TRY(validate_k(h, k));
    if (h->opt.precision == COX_FP32_GEMV) return COX_ERR_UNSUPPORTED;
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_TRY(ensure_workspace(h, k));
    COX_TRY(set_lambdas(h, lambdas, k, st));
    return iterate_from_eta(h, beta_dev, eta_dev, k, step, st);
}

int cox_last_loss_l1(cox_h h, double *f_host, double *l1_host, int k, void *stream)
{
    if (!h || k != h->ws.k) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (f_host) COX_CUDA(cudaMemcpyAsync(f_host, h->ws.f, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (l1_host) COX_CUDA(cudaMemcpyAsync(l1_host, h->ws.l1, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_device_error(h, st);
}

int cox_last_objective(cox_h h, double *obj_host, int k, void *stream)
{
    if (!h || !obj_host || k != h->ws.k) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    COX_CUDA(cudaMemcpyAsync(obj_host, h->ws.F, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    return check_device_error(h, st);
}

int cox_set_covariates(cox_h h, const double *Z_host, int q)
{
    if (!h || q < 0 || q > COX_MAX_COVARIATES || (q > 0 && !Z_host)) return COX_ERR_ARG;
    const int64_t n = h->n;
    for (int64_t i = 0; i < n * q; ++i)
        if (!std::isfinite(Z_host[i])) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    cudaDeviceSynchronize();
    free_workspace(h);  // gamma and its partials follow q
    dfree(h->d_Z);
    h->d_Z = nullptr;
    h->q = 0;
    if (q == 0) return COX_OK;
    std::vector<double> zs(static_cast<size_t>(q) * n);  // q x n in the sorted order
    for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < q; ++c) zs[static_cast<size_t>(c) * n + r] = Z_host[h->h_order[r] * q + c];
    COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_Z), zs.size() * sizeof(double)));
    COX_CUDA(cudaMemcpy(h->d_Z, zs.data(), zs.size() * sizeof(double), cudaMemcpyHostToDevice));
    h->q = q;
    return COX_OK;
}

int cox_get_gamma(cox_h h, double *gamma_host, int k)
{
    if (!h || !gamma_host || k < 1) return COX_ERR_ARG;
    if (h->q == 0) return COX_OK;
    if (k != h->ws.k) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    COX_CUDA(cudaDeviceSynchronize());
    COX_CUDA(cudaMemcpy(gamma_host, h->ws.gamma, static_cast<size_t>(k) * h->q * sizeof(double),
                        cudaMemcpyDeviceToHost));
    return COX_OK;
}

int cox_set_gamma(cox_h h, const double *gamma_host, int k)
{
    if (!h || k < 1) return COX_ERR_ARG;
    if (h->q == 0) return COX_OK;
    COX_TRY(validate_k(h, k));
    DeviceGuard g(h->dev);
    COX_TRY(ensure_workspace(h, k));
    const size_t bytes = static_cast<size_t>(k) * h->q * sizeof(double);
    if (gamma_host) COX_CUDA(cudaMemcpy(h->ws.gamma, gamma_host, bytes, cudaMemcpyHostToDevice));
    else COX_CUDA(cudaMemset(h->ws.gamma, 0, bytes));
    return COX_OK;
}

int cox_grad_gamma(cox_h h, double *gz_host, int k)
{
    if (!h || !gz_host || k < 1) return COX_ERR_ARG;
    if (h->q == 0) return COX_OK;
    if (k != h->ws.k) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    COX_CUDA(cudaDeviceSynchronize());
    std::vector<double> gz(static_cast<size_t>(k) * h->q);
    COX_CUDA(cudaMemcpy(gz.data(), h->ws.gz, gz.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < gz.size(); ++i) gz_host[i] = -gz[i];  // grad f = -Z^T (delta - u) / n
    return COX_OK;
}

int cox_lambda_max(cox_h h, double *lmax_out)
{
    if (!h || !lmax_out) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    const size_t es = is_fp64(h) ? 8 : 4;
    void *b = nullptr, *gr = nullptr;
    COX_TRY(dmalloc(nullptr, &b, h->p * es));
    if (dmalloc(nullptr, &gr, h->p * es) != COX_OK) {
        dfree(b);
        return COX_ERR_OOM;
    }
    cudaMemset(b, 0, h->p * es);
    int rc = cox_loss_grad(h, b, 1, nullptr, gr, nullptr);
    double m = 0.0;
    if (rc == COX_OK) {
        if (es == 8) {
            std::vector<double> v(static_cast<size_t>(h->p));
            if (cudaMemcpy(v.data(), gr, h->p * 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = COX_ERR_CUDA;
            for (double x : v) m = std::max(m, std::fabs(x));
        } else {
            std::vector<float> v(static_cast<size_t>(h->p));
            if (cudaMemcpy(v.data(), gr, h->p * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = COX_ERR_CUDA;
            for (float x : v) m = std::max(m, static_cast<double>(std::fabs(x)));
        }
    }
    dfree(b);
    dfree(gr);
    *lmax_out = m;
    return rc;
}

} // extern "C"
