// path.cu -- step size by the power method (arXiv 2010.16114, Section 4.4,
// used for the Section 5.3 step), the batched regularisation-path fit with the
// Section 6 stopping rule |F_t - F_{t-lag}| / |F_t + 1| < tol, replayed as a
// CUDA graph of `lag` iterations, and checkpoint / resume of that fit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace coxgb {
namespace {

constexpr int RB = 256;

// out[slot] = sum_j mu_j v_j   (one block, fixed order)
template <typename TV>
__global__ void k_dot_mu(const double *__restrict__ mu, const TV *__restrict__ v, int64_t p, double *out)
{
    __shared__ double sh[RB];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += RB) s += mu[j] * static_cast<double>(v[j]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// a_i -= s for i < n, a_i = 0 for n <= i < len; then out = sum_i a_i
template <typename TV>
__global__ void k_center_sum(TV *a, int64_t n, int64_t len, const double *s, double *out)
{
    __shared__ double sh[RB];
    const double sub = *s;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += RB) {
        if (i < n) {
            const TV v = static_cast<TV>(static_cast<double>(a[i]) - sub);
            a[i] = v;
            acc += static_cast<double>(v);
        } else {
            a[i] = TV(0);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// out[a4_pos(i)] = a[i], i < len: a vector over sorted subjects put in the K
// order of the SNP-major genotype copy
__global__ void k_to_a4(const float *__restrict__ a, int64_t len, int64_t pa, int64_t pnb, float *__restrict__ out)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < len;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[a4_pos(i, pa, pnb)] = a[i];
}

// b_j -= mu_j s (j < p); out = ||b||^2
template <typename TV>
__global__ void k_center_norm(TV *b, const double *__restrict__ mu, int64_t p, const double *s, double *out)
{
    __shared__ double sh[RB];
    const double sa = *s;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += RB) {
        const double v = static_cast<double>(b[j]) - mu[j] * sa;
        b[j] = static_cast<TV>(v);
        acc += v * v;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <typename TV>
__global__ void k_scale(const TV *__restrict__ b, TV *__restrict__ v, int64_t p, double inv)
{
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < p) v[j] = static_cast<TV>(static_cast<double>(b[j]) * inv);
}

// FP64: b_j = sum_i Xc[j][i] a_i (one warp per j)
__global__ void k_xta64(const double *__restrict__ Xc, int64_t n, int64_t p, const double *__restrict__ a,
                        double *__restrict__ b)
{
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= p) return;
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) s += Xc[j * n + i] * a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) b[j] = s;
}

// v = start / ||start|| (start == null: all entries 1/sqrt(p)); one block.
template <typename TV>
__global__ void k_start_vector(const double *__restrict__ start, int64_t p, TV *__restrict__ v)
{
    __shared__ double sh[RB];
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += RB) s += start ? start[j] * start[j] : 1.0;
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double inv = 1.0 / sqrt(sh[0]);
    for (int64_t j = threadIdx.x; j < p; j += RB) v[j] = static_cast<TV>((start ? start[j] : 1.0) * inv);
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

template <typename TV>
int power_method(cox_handle *h, const double *start, double tol, int maxiter, double *L_out)
{
    const int64_t n = h->n, p = h->p;
    const bool f64 = h->opt.precision == COX_FP64;
    const int64_t alen = f64 ? n : h->n_pad, blen = f64 ? p : h->p_pad;
    TV *v = nullptr, *a = nullptr, *b = nullptr, *a4 = nullptr;
    double *sc = nullptr;
    int rc = COX_OK;
    if ((rc = dmalloc(nullptr, reinterpret_cast<void **>(&v), p * sizeof(TV))) != COX_OK) return rc;
    if ((rc = dmalloc(nullptr, reinterpret_cast<void **>(&a), alen * sizeof(TV))) != COX_OK) { dfree(v); return rc; }
    if ((rc = dmalloc(nullptr, reinterpret_cast<void **>(&b), blen * sizeof(TV))) != COX_OK) { dfree(v); dfree(a); return rc; }
    if ((rc = dmalloc(nullptr, reinterpret_cast<void **>(&sc), 4 * sizeof(double))) != COX_OK) { dfree(v); dfree(a); dfree(b); return rc; }
    if (!f64 && (rc = dmalloc(nullptr, reinterpret_cast<void **>(&a4), alen * sizeof(TV))) != COX_OK) {
        dfree(v); dfree(a); dfree(b); dfree(sc);
        return rc;
    }
    // the start vector is normalised on the device, by the same kernel as in
    // cox_lipschitz_noalloc, so that both entry points run one power method
    double *st_dev = nullptr;
    if (start && (rc = dmalloc(nullptr, reinterpret_cast<void **>(&st_dev), p * sizeof(double))) != COX_OK) {
        dfree(v); dfree(a); dfree(b); dfree(sc); dfree(a4);
        return rc;
    }
    cudaStream_t st = 0;
    double s = 0.0, s_prev = 0.0;
    do {
        if (start && cudaMemcpy(st_dev, start, p * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
        k_start_vector<TV><<<1, RB, 0, st>>>(st_dev, p, v);
        for (int it = 1; it <= maxiter; ++it) {
            k_dot_mu<TV><<<1, RB, 0, st>>>(h->d_mu, v, p, sc);
            if (f64) {
                rc = eta64(h, reinterpret_cast<const double *>(v), 1, reinterpret_cast<double *>(a), st);
            } else {
                rc = gemv_tiles(h, h->d_A1, h->n_pad, h->p_pad / TILE, reinterpret_cast<const float *>(v), p,
                                reinterpret_cast<float *>(a), st);
            }
            if (rc != COX_OK) break;
            k_center_sum<TV><<<1, RB, 0, st>>>(a, n, alen, sc, sc + 1);
            if (f64) {
                k_xta64<<<static_cast<unsigned>((p * 32 + 255) / 256), 256, 0, st>>>(h->d_Xc, n, p,
                                                                                     reinterpret_cast<const double *>(a),
                                                                                     reinterpret_cast<double *>(b));
            } else {
                k_to_a4<<<static_cast<unsigned>((alen + 255) / 256), 256, 0, st>>>(
                    reinterpret_cast<const float *>(a), alen, h->kperm_a, h->kperm_nb, reinterpret_cast<float *>(a4));
                rc = gemv_tiles(h, h->d_A4, h->p_pad, h->n_pad / TILE, reinterpret_cast<const float *>(a4), alen,
                                reinterpret_cast<float *>(b), st);
                if (rc != COX_OK) break;
            }
            k_center_norm<TV><<<1, RB, 0, st>>>(b, h->d_mu, p, sc + 1, sc + 2);
            double nb2 = 0.0;
            if (cudaMemcpy(&nb2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
            if (!(nb2 > 0.0) || !std::isfinite(nb2)) { s = 0.0; break; }
            s = std::sqrt(nb2);  // ||X_c^T X_c v|| -> largest eigenvalue of X_c^T X_c
            k_scale<TV><<<static_cast<unsigned>((p + 255) / 256), 256, 0, st>>>(b, v, p, 1.0 / s);
            if (it > 1 && std::fabs(s - s_prev) <= tol * s) break;
            s_prev = s;
        }
        if (cudaDeviceSynchronize() != cudaSuccess && rc == COX_OK) rc = COX_ERR_CUDA;
    } while (false);
    dfree(v);
    dfree(a);
    dfree(b);
    dfree(sc);
    dfree(a4);
    dfree(st_dev);
    if (rc == COX_OK) *L_out = 2.0 * s / static_cast<double>(n);
    return rc;
}

} // namespace
} // namespace coxgb

using namespace coxgb;

extern "C" {

int cox_lipschitz(cox_h h, const double *start_host, double tol, int maxiter, double *L_out)
{
    if (!h || !L_out) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    if (!(tol > 0.0)) tol = 1e-6;
    if (maxiter <= 0) maxiter = 1000;
    if (h->opt.precision == COX_FP64) return power_method<double>(h, start_host, tol, maxiter, L_out);
    return power_method<float>(h, start_host, tol, maxiter, L_out);
}

} // extern "C"

namespace coxgb {
namespace {

// The Section 6 stopping-rule loop for k columns on the handle's device
// buffers (lambdas and active flags already set): CUDA-graph replays of `lag`
// iterations, the host reading the k objectives after each replay; a column
// stops when |F_t - F_{t-lag}| / |F_t + 1| < tol and is frozen.  iters,
// active, hist and t carry the state in and out (resume).
int path_run(cox_handle *h, int k, int max_iter, double tol, double step, void *beta_dev, std::vector<int> &iters,
             std::vector<int> &active, std::vector<std::vector<double>> &hist, int64_t &t)
{
    Workspace &ws = h->ws;
    const int lag = h->opt.lag;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = COX_OK;
    auto one_step = [&](int slot) -> int {
        int r = iterate(h, beta_dev, k, EPI_PROX, nullptr, step, cs);
        if (r != COX_OK) return r;
        if (cudaMemcpyAsync(ws.Fring + static_cast<size_t>(slot) * k, ws.F, k * sizeof(double), cudaMemcpyDeviceToDevice,
                            cs) != cudaSuccess)
            return COX_ERR_CUDA;
        return COX_OK;
    };
    if (cudaMemcpy(ws.active, active.data(), k * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return COX_ERR_CUDA;
    do {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
        // the active-set product decides on the host before each iteration, so
        // those iterations run as plain launches instead of graph replays
        if (max_iter - t >= lag && !(h->opt.active_set && (h->opt.precision == COX_SPLIT_E4M3 || is_e2m1(h)))) {
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
            for (int s = 0; s < lag && rc == COX_OK; ++s) rc = one_step(s);
            cudaError_t ec = cudaStreamEndCapture(cs, &graph);
            if (rc != COX_OK) break;
            if (ec != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
        }
        std::vector<double> ring(static_cast<size_t>(lag) * k);
        while (t < max_iter) {
            bool any = false;
            for (int c = 0; c < k; ++c) any |= active[c] != 0;
            if (!any) break;
            int steps;
            if (exec && max_iter - t >= lag) {
                if (cudaGraphLaunch(exec, cs) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
                steps = lag;
            } else {
                steps = static_cast<int>(std::min<int64_t>(lag, max_iter - t));
                for (int s = 0; s < steps && rc == COX_OK; ++s) rc = one_step(s);
                if (rc != COX_OK) break;
            }
            if (cudaMemcpyAsync(ring.data(), ws.Fring, static_cast<size_t>(steps) * k * sizeof(double),
                                cudaMemcpyDeviceToHost, cs) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
            int e = 0;
            if (cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                cudaStreamSynchronize(cs) != cudaSuccess) { rc = COX_ERR_CUDA; break; }
            if (e) {
                cudaMemset(h->d_err, 0, sizeof(int));
                rc = (e & DEVERR_TIMEOUT) ? COX_ERR_TIMEOUT : COX_ERR_NONFINITE;
                break;
            }
            t += steps;
            bool changed = false;
            for (int c = 0; c < k; ++c) {
                if (!active[c]) continue;
                for (int s = 0; s < steps; ++s) hist[c].push_back(ring[static_cast<size_t>(s) * k + c]);
                iters[c] += steps;
                const size_t L = hist[c].size();
                if (L > static_cast<size_t>(lag)) {
                    const double Fn = hist[c][L - 1], Fo = hist[c][L - 1 - lag];
                    if (std::fabs(Fn - Fo) / std::fabs(Fn + 1.0) < tol) {
                        active[c] = 0;
                        changed = true;
                    }
                }
            }
            if (changed && cudaMemcpy(ws.active, active.data(), k * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = COX_ERR_CUDA;
                break;
            }
        }
    } while (false);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    // restore: later single steps treat every column as active
    std::vector<int> ones(static_cast<size_t>(k), 1);
    cudaMemcpy(ws.active, ones.data(), k * sizeof(int), cudaMemcpyHostToDevice);
    return rc;
}

int check_lambdas(const double *lambdas, int k)
{
    for (int c = 0; c < k; ++c)
        if (!(lambdas[c] >= 0.0) || !std::isfinite(lambdas[c])) return COX_ERR_ARG;
    return COX_OK;
}

} // namespace
} // namespace coxgb

extern "C" {

int cox_path_fit(cox_h h, const double *lambdas, int k, int max_iter, double tol, double step, int warm,
                 void *beta_dev, int *iters_host, double *obj_host, void *stream)
{
    if (!h || !beta_dev || !lambdas || max_iter < 0 || !(tol >= 0.0) || !(step > 0.0) || warm < 0 || warm > 2)
        return COX_ERR_ARG;
    if (k < 1 || (h->opt.precision == COX_SPLIT_E4M3 && k > MAX_K_TC) || (is_e2m1(h) && k > MAX_K_E2M1)) return COX_ERR_ARG;
    COX_TRY(check_lambdas(lambdas, k));
    DeviceGuard g(h->dev);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const size_t es = h->opt.precision == COX_FP64 ? 8 : 4;
    const size_t bbytes = static_cast<size_t>(k) * h->p * es;
    const size_t gbytes = static_cast<size_t>(k) * h->q * sizeof(double);
    COX_TRY(ensure_workspace(h, k));
    Workspace &ws = h->ws;
    COX_CUDA(cudaMemcpy(ws.lam, lambdas, k * sizeof(double), cudaMemcpyHostToDevice));

    // host-side state: iterations, active flags, objective history
    std::vector<int> iters(static_cast<size_t>(k), 0), active(static_cast<size_t>(k), 1);
    std::vector<std::vector<double>> hist(static_cast<size_t>(k));
    int64_t t = 0;
    COX_CUDA(cudaStreamSynchronize(user));
    if (warm == 2) {
        if (h->st_k != k || h->st_gamma.size() != static_cast<size_t>(k) * h->q) return COX_ERR_STATE;
        const void *src = es == 8 ? static_cast<const void *>(h->st_beta64.data()) : static_cast<const void *>(h->st_beta32.data());
        COX_CUDA(cudaMemcpy(beta_dev, src, bbytes, cudaMemcpyHostToDevice));
        if (gbytes) COX_CUDA(cudaMemcpy(ws.gamma, h->st_gamma.data(), gbytes, cudaMemcpyHostToDevice));
        iters = h->st_iters;
        active = h->st_active;
        t = h->st_step;
        hist.assign(static_cast<size_t>(k), {});
        size_t off = 0;
        for (int c = 0; c < k; ++c) {
            const size_t len = static_cast<size_t>(h->st_F[off]);
            hist[c].assign(h->st_F.begin() + off + 1, h->st_F.begin() + off + 1 + len);
            off += 1 + len;
        }
    } else if (warm == 0) {
        COX_CUDA(cudaMemset(beta_dev, 0, bbytes));
        if (gbytes) COX_CUDA(cudaMemset(ws.gamma, 0, gbytes));
    }
    const int rc = path_run(h, k, max_iter, tol, step, beta_dev, iters, active, hist, t);
    if (rc != COX_OK) return rc;

    // checkpoint state
    h->st_k = k;
    h->st_step = t;
    h->st_iters = iters;
    h->st_active = active;
    h->st_F.clear();
    for (int c = 0; c < k; ++c) {
        h->st_F.push_back(static_cast<double>(hist[c].size()));
        h->st_F.insert(h->st_F.end(), hist[c].begin(), hist[c].end());
    }
    h->st_gamma.resize(static_cast<size_t>(k) * h->q);
    if (gbytes) COX_CUDA(cudaMemcpy(h->st_gamma.data(), ws.gamma, gbytes, cudaMemcpyDeviceToHost));
    if (es == 8) {
        h->st_beta64.resize(static_cast<size_t>(k) * h->p);
        COX_CUDA(cudaMemcpy(h->st_beta64.data(), beta_dev, bbytes, cudaMemcpyDeviceToHost));
    } else {
        h->st_beta32.resize(static_cast<size_t>(k) * h->p);
        COX_CUDA(cudaMemcpy(h->st_beta32.data(), beta_dev, bbytes, cudaMemcpyDeviceToHost));
    }
    bool all_conv = true;
    for (int c = 0; c < k; ++c) {
        if (iters_host) iters_host[c] = iters[c];
        if (obj_host) obj_host[c] = hist[c].empty() ? NAN : hist[c].back();
        if (active[c]) all_conv = false;
    }
    return all_conv ? COX_OK : COX_ERR_NOT_CONVERGED;
}

int cox_path_seq(cox_h h, const double *lambdas, int L, int max_iter, double tol, double step, int warm,
                 void *B_dev, double *G_host, int *iters_host, double *obj_host, void *stream)
{
    if (!h || !B_dev || !lambdas || L < 1 || max_iter < 0 || !(tol >= 0.0) || !(step > 0.0) || warm < 0 || warm > 1)
        return COX_ERR_ARG;
    COX_TRY(check_lambdas(lambdas, L));
    DeviceGuard g(h->dev);
    COX_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    const size_t es = h->opt.precision == COX_FP64 ? 8 : 4;
    const size_t cb = static_cast<size_t>(h->p) * es;
    COX_TRY(ensure_workspace(h, 1));
    Workspace &ws = h->ws;
    const size_t gbytes = static_cast<size_t>(h->q) * sizeof(double);
    if (gbytes) COX_CUDA(cudaMemset(ws.gamma, 0, gbytes));
    bool all_conv = true;
    for (int l = 0; l < L; ++l) {
        uint8_t *col = static_cast<uint8_t *>(B_dev) + static_cast<size_t>(l) * cb;
        if (warm && l > 0) {
            COX_CUDA(cudaMemcpy(col, col - cb, cb, cudaMemcpyDeviceToDevice));  // gamma stays: it carries over too
        } else {
            COX_CUDA(cudaMemset(col, 0, cb));
            if (gbytes) COX_CUDA(cudaMemset(ws.gamma, 0, gbytes));
        }
        COX_CUDA(cudaMemcpy(ws.lam, lambdas + l, sizeof(double), cudaMemcpyHostToDevice));
        std::vector<int> iters(1, 0), active(1, 1);
        std::vector<std::vector<double>> hist(1);
        int64_t t = 0;
        COX_TRY(path_run(h, 1, max_iter, tol, step, col, iters, active, hist, t));
        if (iters_host) iters_host[l] = iters[0];
        if (obj_host) obj_host[l] = hist[0].empty() ? NAN : hist[0].back();
        if (G_host && gbytes) COX_CUDA(cudaMemcpy(G_host + static_cast<size_t>(l) * h->q, ws.gamma, gbytes,
                                                  cudaMemcpyDeviceToHost));
        if (active[0]) all_conv = false;
    }
    return all_conv ? COX_OK : COX_ERR_NOT_CONVERGED;
}

int cox_get_state(cox_h h, void *buf, size_t *size)
{
    if (!h || !size) return COX_ERR_ARG;
    const int k = h->st_k;
    if (k == 0) return COX_ERR_STATE;
    const bool f64 = h->opt.precision == COX_FP64;
    const size_t nb = static_cast<size_t>(k) * h->p * (f64 ? 8 : 4);
    const size_t ng = h->st_gamma.size() * sizeof(double);  // q x k unpenalised coefficients
    const size_t need = 8 * sizeof(int64_t) + nb + 2 * k * sizeof(int) + h->st_F.size() * sizeof(double) +
                        sizeof(int64_t) + ng;
    if (!buf) {
        *size = need;
        return COX_OK;
    }
    if (*size < need) return COX_ERR_ARG;
    int64_t hdr[8] = {0x434F5853 /* "COXS" */, 2, h->n, h->p, k, h->opt.precision, h->st_step,
                      static_cast<int64_t>(h->st_F.size())};
    uint8_t *o = static_cast<uint8_t *>(buf);
    std::memcpy(o, hdr, sizeof(hdr));
    o += sizeof(hdr);
    std::memcpy(o, f64 ? static_cast<const void *>(h->st_beta64.data()) : static_cast<const void *>(h->st_beta32.data()), nb);
    o += nb;
    std::memcpy(o, h->st_iters.data(), k * sizeof(int));
    o += k * sizeof(int);
    std::memcpy(o, h->st_active.data(), k * sizeof(int));
    o += k * sizeof(int);
    std::memcpy(o, h->st_F.data(), h->st_F.size() * sizeof(double));
    o += h->st_F.size() * sizeof(double);
    const int64_t q = static_cast<int64_t>(h->st_gamma.size() / static_cast<size_t>(k));
    std::memcpy(o, &q, sizeof(q));
    o += sizeof(q);
    if (ng) std::memcpy(o, h->st_gamma.data(), ng);
    *size = need;
    return COX_OK;
}

int cox_set_state(cox_h h, const void *buf, size_t size)
{
    if (!h || !buf || size < 8 * sizeof(int64_t)) return COX_ERR_ARG;
    int64_t hdr[8];
    std::memcpy(hdr, buf, sizeof(hdr));
    if (hdr[0] != 0x434F5853 || hdr[1] != 2 || hdr[2] != h->n || hdr[3] != h->p || hdr[5] != h->opt.precision)
        return COX_ERR_STATE;
    const int k = static_cast<int>(hdr[4]);
    if (k < 1) return COX_ERR_STATE;
    const bool f64 = h->opt.precision == COX_FP64;
    const size_t nb = static_cast<size_t>(k) * h->p * (f64 ? 8 : 4);
    const size_t nF = static_cast<size_t>(hdr[7]);
    const size_t base = 8 * sizeof(int64_t) + nb + 2 * k * sizeof(int) + nF * sizeof(double);
    if (size < base + sizeof(int64_t)) return COX_ERR_STATE;
    int64_t q = 0;
    std::memcpy(&q, static_cast<const uint8_t *>(buf) + base, sizeof(q));
    if (q != h->q || size < base + sizeof(int64_t) + static_cast<size_t>(q) * k * sizeof(double)) return COX_ERR_STATE;
    const uint8_t *in = static_cast<const uint8_t *>(buf) + sizeof(hdr);
    h->st_k = k;
    h->st_step = hdr[6];
    if (f64) {
        h->st_beta64.resize(static_cast<size_t>(k) * h->p);
        std::memcpy(h->st_beta64.data(), in, nb);
    } else {
        h->st_beta32.resize(static_cast<size_t>(k) * h->p);
        std::memcpy(h->st_beta32.data(), in, nb);
    }
    in += nb;
    h->st_iters.resize(k);
    std::memcpy(h->st_iters.data(), in, k * sizeof(int));
    in += k * sizeof(int);
    h->st_active.resize(k);
    std::memcpy(h->st_active.data(), in, k * sizeof(int));
    in += k * sizeof(int);
    h->st_F.resize(nF);
    std::memcpy(h->st_F.data(), in, nF * sizeof(double));
    in += nF * sizeof(double) + sizeof(int64_t);
    h->st_gamma.resize(static_cast<size_t>(q) * k);
    if (q) std::memcpy(h->st_gamma.data(), in, h->st_gamma.size() * sizeof(double));
    return COX_OK;
}

} // extern "C"

// ---- step size without device allocation ------------------------------------
//
// cox_lipschitz_noalloc runs the same power method as cox_lipschitz, but its
// work vectors live in one file-scope device array instead of memory taken
// with cudaMalloc.  The array is part of the library image: every GPU that
// loads the library holds it until the process exits.  Host code only ever
// sees a host-side stand-in for it under its name, so the device address is
// looked up once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernels.  All calls share the array; calls that
// overlap on the GPU race on it.  Each call writes every element it later
// reads, so nothing left by an earlier call leaks into a result.
namespace coxgb {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = static_cast<size_t>(16) << 20;  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(double)];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on device `dev` (current).  First call
// per device performs the lookup.
int noalloc_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return COX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return COX_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return COX_OK;
}

template <typename TV>
int power_method_noalloc(cox_handle *h, const double *start, double tol, int maxiter, double *L_out)
{
    const int64_t n = h->n, p = h->p;
    const bool f64 = h->opt.precision == COX_FP64;
    const int64_t alen = f64 ? n : h->n_pad, blen = f64 ? p : h->p_pad;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t off_a = up(p * sizeof(TV));
    const size_t off_b = off_a + up(alen * sizeof(TV));
    const size_t off_sc = off_b + up(blen * sizeof(TV));
    const size_t off_a4 = off_sc + 256;
    const size_t off_st = off_a4 + (f64 ? 0 : up(alen * sizeof(TV)));
    const size_t need = off_st + (start ? up(p * sizeof(double)) : 0);
    if (need > NOALLOC_SCRATCH_BYTES) return COX_ERR_ARG;
    void *base = nullptr;
    COX_TRY(noalloc_scratch(h->dev, &base));
    uint8_t *b8 = static_cast<uint8_t *>(base);
    TV *v = reinterpret_cast<TV *>(b8);
    TV *a = reinterpret_cast<TV *>(b8 + off_a);
    TV *b = reinterpret_cast<TV *>(b8 + off_b);
    double *sc = reinterpret_cast<double *>(b8 + off_sc);
    TV *a4 = reinterpret_cast<TV *>(b8 + off_a4);
    double *st_dev = start ? reinterpret_cast<double *>(b8 + off_st) : nullptr;
    cudaStream_t st = 0;
    if (start) COX_CUDA(cudaMemcpyAsync(st_dev, start, p * sizeof(double), cudaMemcpyHostToDevice, st));
    k_start_vector<TV><<<1, RB, 0, st>>>(st_dev, p, v);
    COX_CUDA(cudaGetLastError());
    double s = 0.0, s_prev = 0.0;
    int rc = COX_OK;
    for (int it = 1; it <= maxiter; ++it) {
        k_dot_mu<TV><<<1, RB, 0, st>>>(h->d_mu, v, p, sc);
        if (f64) {
            rc = eta64(h, reinterpret_cast<const double *>(v), 1, reinterpret_cast<double *>(a), st);
        } else {
            rc = gemv_tiles(h, h->d_A1, h->n_pad, h->p_pad / TILE, reinterpret_cast<const float *>(v), p,
                            reinterpret_cast<float *>(a), st);
        }
        if (rc != COX_OK) break;
        k_center_sum<TV><<<1, RB, 0, st>>>(a, n, alen, sc, sc + 1);
        if (f64) {
            k_xta64<<<static_cast<unsigned>((p * 32 + 255) / 256), 256, 0, st>>>(
                h->d_Xc, n, p, reinterpret_cast<const double *>(a), reinterpret_cast<double *>(b));
        } else {
            k_to_a4<<<static_cast<unsigned>((alen + 255) / 256), 256, 0, st>>>(
                reinterpret_cast<const float *>(a), alen, h->kperm_a, h->kperm_nb, reinterpret_cast<float *>(a4));
            rc = gemv_tiles(h, h->d_A4, h->p_pad, h->n_pad / TILE, reinterpret_cast<const float *>(a4), alen,
                            reinterpret_cast<float *>(b), st);
            if (rc != COX_OK) break;
        }
        k_center_norm<TV><<<1, RB, 0, st>>>(b, h->d_mu, p, sc + 1, sc + 2);
        double nb2 = 0.0;
        if (cudaMemcpy(&nb2, sc + 2, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        if (!(nb2 > 0.0) || !std::isfinite(nb2)) {
            s = 0.0;
            break;
        }
        s = std::sqrt(nb2);
        k_scale<TV><<<static_cast<unsigned>((p + 255) / 256), 256, 0, st>>>(b, v, p, 1.0 / s);
        if (it > 1 && std::fabs(s - s_prev) <= tol * s) break;
        s_prev = s;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == COX_OK) rc = COX_ERR_CUDA;
    if (rc == COX_OK) *L_out = 2.0 * s / static_cast<double>(n);
    return rc;
}

} // namespace
} // namespace coxgb

extern "C" int cox_lipschitz_noalloc(cox_h h, const double *start_host, double tol, int maxiter, double *L_out)
{
    if (!h || !L_out) return COX_ERR_ARG;
    DeviceGuard g(h->dev);
    if (!(tol > 0.0)) tol = 1e-6;
    if (maxiter <= 0) maxiter = 1000;
    if (h->opt.precision == COX_FP64) return power_method_noalloc<double>(h, start_host, tol, maxiter, L_out);
    return power_method_noalloc<float>(h, start_host, tol, maxiter, L_out);
}
