// setup.cu -- lays one data set out in device memory for the Cox iteration
// (arXiv 2010.16114, Section 5.3 problem: X, y, delta; the sorting remark;
// Section 6: Breslow ties).
//
// Subjects are put in ascending time order (stable), so the risk sets become
// suffixes of the order.  Genotypes are stored twice as 2-bit codes in
// 128 x 128 blocks of 4 KB: subject-major (A1: rows = sorted subjects,
// K = SNPs, for X beta) and SNP-major (A4: rows = SNPs, K = sorted subjects in
// 16-subject blocks spread by a4_pos, for X^T V), each streamed once per
// iteration by its own product.
//
// Block layout (both copies): row r of a block is 32 bytes = two 16-byte
// halves (K 0-63 and 64-127 of the chunk); the halves of rows with bit 2 of r
// set are stored swapped, which spreads a warp's 16-byte reads over all 32
// banks.  A half is four 32-bit words of 16 codes; inside a word, code K
// (0..15) sits at bit code_bit(K) = 8 (K mod 4) + 2 (K div 4), so one shift
// and one AND give four consecutive codes as four e4m3 bytes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.h"

namespace coxgb {
namespace {

// A1: thread per (sorted row r, 16-SNP word); validates codes.
__global__ void k_pack_a1(const uint8_t *__restrict__ in, int64_t rb, int64_t n, int64_t p,
                          const int32_t *__restrict__ order, uint32_t *__restrict__ A1, int64_t KC1, int *err)
{
    const int64_t W = (p + 15) / 16;
    const int64_t total = n * W;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / W, wq = t - r * W;
        const uint8_t *row = in + static_cast<int64_t>(order[r]) * rb;
        const int64_t j0 = 16 * wq;
        uint32_t P = 0;
        bool bad = false;
#pragma unroll
        for (int kap = 0; kap < 16; ++kap) {
            const int64_t j = j0 + kap;
            if (j < p) {
                const uint32_t c = (row[j >> 2] >> (2 * (j & 3))) & 3u;
                bad |= (c == 3u);
                P |= (c == 3u ? 0u : c) << code_bit(kap);
            }
        }
        if (bad) atomicOr(err, DEVERR_CODE3);
        A1[word_offset(r / TILE, KC1, j0 / TILE, static_cast<int>(r % TILE), static_cast<int>(j0 % TILE))] = P;
    }
}

// A4: thread per (SNP j, 16 sorted subjects), stored at the block's K position
// a4_pos; column sums for mu.
__global__ void k_pack_a4(const uint8_t *__restrict__ in, int64_t rb, int64_t n, int64_t p,
                          const int32_t *__restrict__ order, uint32_t *__restrict__ A4, int64_t KC4,
                          int64_t pa, int64_t pnb, unsigned long long *__restrict__ colsum)
{
    const int64_t R16 = (n + 15) / 16;
    const int64_t total = R16 * p;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t rq = t / p, j = t - rq * p;
        const int64_t r0 = 16 * rq;
        uint32_t P = 0, s = 0;
#pragma unroll
        for (int kap = 0; kap < 16; ++kap) {
            const int64_t r = r0 + kap;
            if (r < n) {
                uint32_t c = (in[static_cast<int64_t>(order[r]) * rb + (j >> 2)] >> (2 * (j & 3))) & 3u;
                if (c == 3u) c = 0u;
                P |= c << code_bit(kap);
                s += c;
            }
        }
        const int64_t k0 = a4_pos(r0, pa, pnb);
        A4[word_offset(j / TILE, KC4, k0 / TILE, static_cast<int>(j % TILE), static_cast<int>(k0 % TILE))] = P;
        if (s) atomicAdd(&colsum[j], static_cast<unsigned long long>(s));
    }
}

unsigned grid_for(int64_t total, int sms)
{
    const int64_t b = (total + 255) / 256;
    return static_cast<unsigned>(std::min<int64_t>(b, static_cast<int64_t>(sms) * 16));
}

} // namespace

int setup_genotypes(cox_handle *h, const void *X, int x_format, cudaStream_t st)
{
    const int64_t n = h->n, p = h->p, rb = (p + 3) / 4;
    const uint8_t *d_in = nullptr;
    uint8_t *d_own = nullptr;
    if (x_format == COX_X_PACKED2_DEV) {
        d_in = static_cast<const uint8_t *>(X);
    } else {
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&d_own), static_cast<size_t>(n * rb)));
        h->device_bytes -= n * rb;  // staging only
        if (x_format == COX_X_PACKED2_HOST) {
            if (cudaMemcpyAsync(d_own, X, static_cast<size_t>(n * rb), cudaMemcpyHostToDevice, st) != cudaSuccess) {
                dfree(d_own);
                return COX_ERR_CUDA;
            }
        } else {  // COX_X_INT8_HOST: pack on the host in row blocks, validate codes
            const uint8_t *x8 = static_cast<const uint8_t *>(X);
            const int64_t rows_blk = std::max<int64_t>(1, (int64_t(64) << 20) / std::max<int64_t>(rb, 1));
            std::vector<uint8_t> buf(static_cast<size_t>(std::min(rows_blk, n) * rb));
            int bad = 0;
            const int nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
            for (int64_t r0 = 0; r0 < n && !bad; r0 += rows_blk) {
                const int64_t nr = std::min(rows_blk, n - r0);
                std::vector<int> badv(nth, 0);
                std::vector<std::thread> th;
                for (int tq = 0; tq < nth; ++tq) {
                    th.emplace_back([&, tq]() {
                        for (int64_t r = tq; r < nr; r += nth) {
                            const uint8_t *src = x8 + (r0 + r) * p;
                            uint8_t *dst = buf.data() + r * rb;
                            std::memset(dst, 0, static_cast<size_t>(rb));
                            for (int64_t j = 0; j < p; ++j) {
                                const uint8_t c = src[j];
                                if (c > 2) badv[tq] = 1;
                                dst[j >> 2] |= static_cast<uint8_t>((c & 3) << (2 * (j & 3)));
                            }
                        }
                    });
                }
                for (auto &t : th) t.join();
                for (int v : badv) bad |= v;
                if (bad) break;
                if (cudaMemcpy(d_own + r0 * rb, buf.data(), static_cast<size_t>(nr * rb), cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                    dfree(d_own);
                    return COX_ERR_CUDA;
                }
            }
            if (bad) {
                dfree(d_own);
                return COX_ERR_CODE3;
            }
        }
        d_in = d_own;
    }

    // sorted order on the device
    int32_t *d_order = nullptr;
    unsigned long long *d_colsum = nullptr;
    int rc = COX_OK;
    std::vector<int32_t> ord32(static_cast<size_t>(n));
    for (int64_t r = 0; r < n; ++r) ord32[r] = static_cast<int32_t>(h->h_order[r]);
    const size_t a1_bytes = static_cast<size_t>(h->n_pad / TILE) * (h->p_pad / TILE) * BLOCK_BYTES;
    do {
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&d_order), n * sizeof(int32_t))) != COX_OK) break;
        h->device_bytes -= n * sizeof(int32_t);
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&d_colsum), p * sizeof(unsigned long long))) != COX_OK) break;
        h->device_bytes -= p * sizeof(unsigned long long);
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_A1), a1_bytes)) != COX_OK) break;
        if ((rc = dmalloc(h, reinterpret_cast<void **>(&h->d_A4), a1_bytes)) != COX_OK) break;
        if (cudaMemcpyAsync(d_order, ord32.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(d_colsum, 0, p * sizeof(unsigned long long), st) != cudaSuccess ||
            cudaMemsetAsync(h->d_A1, 0, a1_bytes, st) != cudaSuccess ||
            cudaMemsetAsync(h->d_A4, 0, a1_bytes, st) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        k_pack_a1<<<grid_for(n * ((p + 15) / 16), h->sm_count), 256, 0, st>>>(d_in, rb, n, p, d_order, h->d_A1,
                                                                                h->p_pad / TILE, h->d_err);
        k_pack_a4<<<grid_for(((n + 15) / 16) * p, h->sm_count), 256, 0, st>>>(d_in, rb, n, p, d_order, h->d_A4,
                                                                                h->n_pad / TILE, h->kperm_a,
                                                                                h->kperm_nb, d_colsum);
        if (cudaGetLastError() != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        std::vector<unsigned long long> cs(static_cast<size_t>(p));
        int herr = 0;
        if (cudaMemcpyAsync(cs.data(), d_colsum, p * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = COX_ERR_CUDA;
            break;
        }
        if (herr & DEVERR_CODE3) {
            rc = COX_ERR_CODE3;
            break;
        }
        h->h_mu.assign(static_cast<size_t>(p), 0.0);
        if (h->opt.center)
            for (int64_t j = 0; j < p; ++j) h->h_mu[j] = static_cast<double>(cs[j]) / static_cast<double>(n);
    } while (false);
    dfree(d_order);
    dfree(d_colsum);
    if (d_own) dfree(d_own);
    return rc;
}

int setup_dense64(cox_handle *h, const double *X, cudaStream_t st)
{
    const int64_t n = h->n, p = h->p;
    std::vector<double> xr(static_cast<size_t>(n * p)), xc(static_cast<size_t>(n * p));
    h->h_mu.assign(static_cast<size_t>(p), 0.0);
    for (int64_t r = 0; r < n; ++r) {
        const double *src = X + h->h_order[r] * p;
        for (int64_t j = 0; j < p; ++j) {
            if (!std::isfinite(src[j])) return COX_ERR_ARG;
            xr[r * p + j] = src[j];
            xc[j * n + r] = src[j];
        }
    }
    if (h->opt.center) {
        for (int64_t j = 0; j < p; ++j) {
            double s = 0.0;
            for (int64_t r = 0; r < n; ++r) s += xc[j * n + r];
            h->h_mu[j] = s / static_cast<double>(n);
        }
    }
    COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_Xr), n * p * sizeof(double)));
    COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_Xc), n * p * sizeof(double)));
    COX_CUDA(cudaMemcpyAsync(h->d_Xr, xr.data(), n * p * sizeof(double), cudaMemcpyHostToDevice, st));
    COX_CUDA(cudaMemcpyAsync(h->d_Xc, xc.data(), n * p * sizeof(double), cudaMemcpyHostToDevice, st));
    COX_CUDA(cudaStreamSynchronize(st));
    return COX_OK;
}

} // namespace coxgb
