// active.cu -- the first product X_c B over the active SNP columns only.
//
// With cox_options.active_set, eta = X B needs only the columns j where some
// penalty's coefficient is nonzero (arXiv 2010.16114, Section 6: along the UK
// Biobank path a few hundred SNPs were selected out of 470,194).  Before each
// X B the library marks the union support of the k coefficient columns; when
// it holds a column outside the current active set A, the host rebuilds A (the
// old set with the support added, and the SNPs the fused step marked as close
// to entering, or without the old set once that union has grown past twice
// the rest), gathers a subject-major 2-bit copy of the columns of A (the tiled
// layout of the full copy, K = position in A), and plans the same tensor-core
// product on it.  A always covers the current support, so the
// product equals the dense one up to the FP32 order of the nonzero terms.
// When the support holds more than a quarter of the (padded) columns the
// dense product runs instead.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace coxgb {
namespace {

// flag[j] = 1 when some column of beta is nonzero at SNP j; counts the
// support and the support outside the active set (cnt[0], cnt[1]).
__global__ void k_support(const float *__restrict__ beta, int k, int64_t p, const uint8_t *__restrict__ inA,
                          uint8_t *__restrict__ flag, unsigned long long *__restrict__ cnt)
{
    unsigned long long sup = 0, out = 0;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < p;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        bool nz = false;
        for (int c = 0; c < k && !nz; ++c) nz = beta[static_cast<int64_t>(c) * p + j] != 0.f;
        flag[j] = nz ? 1 : 0;
        sup += nz;
        out += nz && !inA[j];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sup += __shfl_xor_sync(0xffffffffu, sup, o);
        out += __shfl_xor_sync(0xffffffffu, out, o);
    }
    if ((threadIdx.x & 31) == 0 && (sup || out)) {
        atomicAdd(cnt, sup);
        atomicAdd(cnt + 1, out);
    }
}

// The active copy, one CTA per row tile (thread = row): for each source chunk
// that holds active SNPs (cchunk[c], active positions cstart[c] ..
// cstart[c+1]), the row's 32-byte record of that chunk (coalesced over the
// tile's 128 rows, prefetched GA chunks ahead) yields the codes of all its
// active SNPs, packed in active order into words of 16; positions past nA
// stay 0 (the copy is cleared first).
constexpr int GA = 4;
__global__ void __launch_bounds__(TILE) k_gather_active(const uint32_t *__restrict__ A1, int64_t KC1,
                                                        const int32_t *__restrict__ Aidx,
                                                        const int32_t *__restrict__ cchunk,
                                                        const int32_t *__restrict__ cstart, int nchunks,
                                                        int64_t n, int64_t KCa, uint32_t *__restrict__ out)
{
    const int64_t mt = blockIdx.x;
    const int rit = threadIdx.x;
    if (mt * TILE + rit >= n) return;  // padding rows stay 0
    const int swp = (rit >> 2) & 1;
    int64_t cur = -1;  // word (16 active positions) being built
    uint32_t P = 0;
    for (int c0 = 0; c0 < nchunks; c0 += GA) {
        uint4 rec[GA][2];
#pragma unroll
        for (int g = 0; g < GA; ++g) {
            if (c0 + g >= nchunks) break;
            const uint4 *b = reinterpret_cast<const uint4 *>(
                reinterpret_cast<const uint8_t *>(A1) + (mt * KC1 + cchunk[c0 + g]) * BLOCK_BYTES + rit * 32);
            rec[g][0] = __ldcs(b + swp);      // logical half 0 (K 0..63 of the chunk)
            rec[g][1] = __ldcs(b + (swp ^ 1));  // logical half 1
        }
#pragma unroll
        for (int g = 0; g < GA; ++g) {
            if (c0 + g >= nchunks) break;
            const uint32_t wd[8] = {rec[g][0].x, rec[g][0].y, rec[g][0].z, rec[g][0].w,
                                    rec[g][1].x, rec[g][1].y, rec[g][1].z, rec[g][1].w};
            for (int32_t t = cstart[c0 + g]; t < cstart[c0 + g + 1]; ++t) {
                const int within = static_cast<int>(Aidx[t] % TILE);
                uint32_t word = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q == (within >> 4)) word = wd[q];  // word q = 4 h + (within mod 64) / 16
                const uint32_t code = (word >> code_bit(within & 15)) & 3u;
                const int64_t wq = t >> 4;
                if (wq != cur) {
                    if (cur >= 0)
                        out[word_offset(mt, KCa, (cur * 16) / TILE, rit, static_cast<int>((cur * 16) % TILE))] = P;
                    P = 0;
                    cur = wq;
                }
                P |= code << code_bit(t & 15);
            }
        }
    }
    if (cur >= 0) out[word_offset(mt, KCa, (cur * 16) / TILE, rit, static_cast<int>((cur * 16) % TILE))] = P;
}

// e4m3 limbs of beta at the active SNPs (column t of the limb matrix = SNP
// Aidx[t]), the power-of-two column scale from the max |beta| partials as in
// the dense product's limbs.
__global__ void k_prep_limbs_active(const float *__restrict__ beta, int64_t p, const int32_t *__restrict__ Aidx,
                                    int64_t nA, int64_t Kpad, int nb, const float *__restrict__ maxp,
                                    uint8_t *__restrict__ Bq, int *__restrict__ bs, int *err)
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
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < Kpad;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint8_t d[LIMBS] = {0, 0, 0, 0};
        if (t < nA) split_e4m3(ldexpf(beta[static_cast<int64_t>(kk) * p + Aidx[t]], -s), d);
#pragma unroll
        for (int l = 0; l < LIMBS; ++l) Bq[(LIMBS * kk + l) * Kpad + t] = d[l];
    }
}

unsigned grid_over(int64_t total, int sms)
{
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * sms)));
}

} // namespace

void active_free(cox_handle *h)
{
    void *ptrs[] = {h->d_inA, h->d_flag, h->d_near, h->d_Aidx, h->d_A1act, h->d_actcnt};
    for (void *p : ptrs) dfree(p);
    h->d_inA = h->d_flag = h->d_near = nullptr;
    h->d_Aidx = nullptr;
    h->d_A1act = nullptr;
    h->d_actcnt = nullptr;
    h->nA = -1;
    h->act_cap = 0;
    h->h_Aidx.clear();
}

// Decide the first product of this iteration: *use = 1 with ws.g1a planned on
// the active columns and their limbs prepared, or *use = 0 for the dense one.
// Synchronises `st` once (two counters) and, when the support left the active
// set, rebuilds it.
int active_prepare(cox_handle *h, const float *beta, int k, cudaStream_t st, int *use)
{
    Workspace &ws = h->ws;
    *use = 0;
    const int64_t p = h->p;
    if (!h->d_inA) {
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_inA), p));
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_flag), p));
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_near), p));
        COX_CUDA(cudaMemsetAsync(h->d_near, 0, p, st));
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_actcnt), 2 * sizeof(unsigned long long)));
        COX_CUDA(cudaMemsetAsync(h->d_inA, 0, p, st));
        h->nA = -1;
    }
    COX_CUDA(cudaMemsetAsync(h->d_actcnt, 0, 2 * sizeof(unsigned long long), st));
    k_support<<<grid_over(p, h->sm_count), 256, 0, st>>>(beta, k, p, h->d_inA, h->d_flag, h->d_actcnt);
    COX_CUDA(cudaGetLastError());
    unsigned long long cnt[2] = {0, 0};
    COX_CUDA(cudaMemcpyAsync(cnt, h->d_actcnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    COX_CUDA(cudaStreamSynchronize(st));
    h->launches += 1;
    const int64_t limit = h->p_pad / 4;
    if (static_cast<int64_t>(cnt[0]) > limit) return COX_OK;  // a large support: the dense product
    const bool rebuild = h->nA < 0 || cnt[1] > 0;
    if (rebuild) {
        // the new set: the old one with the current support added (SNPs that
        // leave and re-enter then cost no rebuild), or the support alone once
        // the union has grown past twice the support (plus 4096)
        std::vector<uint8_t> flag(static_cast<size_t>(p)), near(static_cast<size_t>(p));
        COX_CUDA(cudaMemcpyAsync(flag.data(), h->d_flag, p, cudaMemcpyDeviceToHost, st));
        COX_CUDA(cudaMemcpyAsync(near.data(), h->d_near, p, cudaMemcpyDeviceToHost, st));
        COX_CUDA(cudaMemsetAsync(h->d_near, 0, p, st));
        COX_CUDA(cudaStreamSynchronize(st));
        const int64_t sup = static_cast<int64_t>(cnt[0]);
        // headroom: SNPs whose pre-threshold value came within a quarter of the
        // threshold in the steps since the last rebuild (marked by the fused step)
        // are likely to enter next, so the set takes them in now
        int64_t nnear = 0;
        for (int64_t j = 0; j < p; ++j) nnear += near[j] && !flag[j];
        if (sup + nnear <= limit)
            for (int64_t j = 0; j < p; ++j) flag[j] |= near[j];
        if (static_cast<int64_t>(h->h_Aidx.size()) + static_cast<int64_t>(cnt[1]) <= 2 * (sup + nnear) + 4096)
            for (int32_t j : h->h_Aidx) flag[j] = 1;
        std::vector<int32_t> idx;
        for (int64_t j = 0; j < p; ++j)
            if (flag[j]) idx.push_back(static_cast<int32_t>(j));
        const int64_t nA = static_cast<int64_t>(idx.size());
        if (nA > limit) return COX_OK;  // the set in use stays as it was
        // the source chunks that hold active SNPs, and each one's first active position
        std::vector<int32_t> cchunk, cstart;
        for (int64_t t = 0; t < nA; ++t)
            if (cchunk.empty() || idx[t] / TILE != cchunk.back()) {
                cchunk.push_back(idx[t] / TILE);
                cstart.push_back(static_cast<int32_t>(t));
            }
        cstart.push_back(static_cast<int32_t>(nA));
        const int64_t Kpad = std::max<int64_t>(256, (nA + 255) / 256 * 256);
        if (Kpad > h->act_cap) {
            dfree(h->d_Aidx);
            dfree(h->d_A1act);
            h->d_Aidx = nullptr;
            h->d_A1act = nullptr;
            // Aidx then the chunk list (at most one chunk per active SNP) and its starts
            COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_Aidx), (3 * Kpad + 1) * sizeof(int32_t)));
            COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_A1act), static_cast<size_t>(h->n_pad) * Kpad / 4));
            h->act_cap = Kpad;
        }
        int32_t *d_cchunk = h->d_Aidx + h->act_cap, *d_cstart = h->d_Aidx + 2 * h->act_cap;
        const int nchunks = static_cast<int>(cchunk.size());
        if (nA) {
            COX_CUDA(cudaMemcpyAsync(h->d_Aidx, idx.data(), nA * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            COX_CUDA(cudaMemcpyAsync(d_cchunk, cchunk.data(), nchunks * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        }
        COX_CUDA(cudaMemcpyAsync(d_cstart, cstart.data(), cstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        COX_CUDA(cudaMemcpyAsync(h->d_inA, flag.data(), p, cudaMemcpyHostToDevice, st));
        COX_CUDA(cudaMemsetAsync(h->d_A1act, 0, static_cast<size_t>(h->n_pad) * Kpad / 4, st));
        if (nchunks)
            k_gather_active<<<static_cast<unsigned>(h->n_pad / TILE), TILE, 0, st>>>(
                h->d_A1, h->p_pad / TILE, h->d_Aidx, d_cchunk, d_cstart, nchunks, h->n, Kpad / TILE, h->d_A1act);
        COX_CUDA(cudaGetLastError());
        COX_CUDA(cudaStreamSynchronize(st));  // the host lists leave scope
        h->launches += 1;
        h->h_Aidx.swap(idx);
        h->nA = nA;
        h->act_Kpad = Kpad;
        h->act_rebuilds += 1;
        ws.g1a_ready = false;
    }
    if (!ws.g1a_ready || ws.g1a_K != h->act_Kpad) {
        // limbs and plan for this active width (the shape of the dense plan)
        dfree(ws.Bqa);
        ws.Bqa = nullptr;
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&ws.Bqa), static_cast<size_t>(ws.NP) * h->act_Kpad));
        COX_CUDA(cudaMemsetAsync(ws.Bqa, 0, static_cast<size_t>(ws.NP) * h->act_Kpad, st));
        const int issue = ws.g1.alt ? 2 : ws.g1.pair ? 3 : 1;
        COX_TRY(plan_gemm(h, ws.g1a, h->d_A1act, h->n_pad, h->act_Kpad, ws.Bqa, k, ws.g1.T, ws.g1.CH, ws.g1.stages,
                          issue));
        if (ws.g1a.max_slots > ws.part1_slots) {
            dfree(ws.part1);
            ws.part1 = nullptr;
            COX_TRY(dmalloc(h, reinterpret_cast<void **>(&ws.part1),
                            static_cast<size_t>(ws.g1a.max_slots) * k * h->n_pad * sizeof(float)));
            ws.part1_slots = ws.g1a.max_slots;
        }
        ws.g1a_ready = true;
        ws.g1a_K = h->act_Kpad;
    }
    const int64_t gx = std::min<int64_t>((h->act_Kpad + 255) / 256, std::max<int64_t>(1, 4LL * h->sm_count / k));
    k_prep_limbs_active<<<dim3(static_cast<unsigned>(gx), k), 256, 0, st>>>(
        beta, p, h->d_Aidx, h->nA, h->act_Kpad, h->l1_blocks, ws.bmaxp, ws.Bqa, ws.bs1, h->d_err);
    COX_CUDA(cudaGetLastError());
    h->launches += 1;
    *use = 1;
    return COX_OK;
}

} // namespace coxgb
