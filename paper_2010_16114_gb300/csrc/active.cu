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
// layout of the full copy, K = position in A) from the rows of A in the
// SNP-major copy, and plans the same tensor-core product on it.  A always covers the current support, so the
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

// The active copy from the SNP-major copy A4, one CTA of 128 threads per
// (active chunk ca of 128 active positions, A4 K chunk kc of 128 K positions).
// Thread s reads the 32-byte record of active SNP Aidx[128 ca + s] in chunk kc:
// eight words, word u holding the codes of the 16 subjects of K block
// B = 8 kc + u (A4 stores sorted subject block b at block B = (a b) mod nb, so
// b = a^-1 B mod nb).  Per u the 16 threads of a group g (active positions
// 16 g .. 16 g + 15) transpose their 16 words by shuffles into one word per
// subject (the codes of the group's 16 SNPs) and write it to that subject's
// row of the subject-major copy, at active position 16 g of chunk ca: the CTA
// writes whole 32-byte records of 16 rows per u.  Positions past nA read 0.
// Reads are whole 32-byte sectors of the active SNPs' rows only (|A| n / 4
// bytes); every word of the copy is written (no clearing needed).
__global__ void __launch_bounds__(TILE) k_gather_active(const uint32_t *__restrict__ A4, int64_t KC4,
                                                        const int32_t *__restrict__ Aidx, int64_t nA, int64_t KCa,
                                                        int64_t ainv, int64_t nb, uint32_t *__restrict__ out)
{
    const int64_t ca = static_cast<int64_t>(blockIdx.x) % KCa;
    const int64_t kc = static_cast<int64_t>(blockIdx.x) / KCa;
    const int s = threadIdx.x, lane = s & 31, i = s & 15, g = s >> 4;
    const int64_t t = ca * TILE + s;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (t < nA) {
        const int64_t j = Aidx[t];
        const int row = static_cast<int>(j % TILE);
        const int swp = (row >> 2) & 1;
        const uint4 *rec = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(A4) +
                                                           ((j / TILE) * KC4 + kc) * BLOCK_BYTES + row * 32);
        const uint4 h0 = __ldcs(rec + swp), h1 = __ldcs(rec + (swp ^ 1));  // logical halves 0, 1
        w[0] = h0.x; w[1] = h0.y; w[2] = h0.z; w[3] = h0.w;
        w[4] = h1.x; w[5] = h1.y; w[6] = h1.z; w[7] = h1.w;
    }
    const int src0 = lane & 16;  // first lane of this thread's group in the warp
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        uint32_t o = 0;  // subject i of the block: the group's 16 SNP codes
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t wk = __shfl_sync(0xffffffffu, w[u], src0 + k);
            o |= ((wk >> code_bit(i)) & 3u) << code_bit(k);
        }
        const int64_t b = (ainv * (8 * kc + u)) % nb;  // sorted subject block
        out[word_offset(b >> 3, KCa, ca, static_cast<int>((b & 7) * 16 + i), 16 * g)] = o;
    }
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

// e2m1 limbs of beta at the active SNPs: byte t of a limb row holds active
// positions 16 (t / 8) + t mod 8 (low nibble) and that + 8 (e2m1_byte).
__global__ void k_prep_limbs_active4(const float *__restrict__ beta, int64_t p, const int32_t *__restrict__ Aidx,
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
            s_sh = limb_scale4(m);
            if (blockIdx.x == 0) bs[kk] = s_sh;
        }
    }
    __syncthreads();
    const int s = s_sh;
    const int64_t rb = Kpad / 2;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < rb;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t t0 = ((t >> 3) << 4) + (t & 7);
        uint8_t d0[LIMBS4] = {}, d1[LIMBS4] = {};
        if (t0 < nA) split_e2m1_units(ldexpf(beta[static_cast<int64_t>(kk) * p + Aidx[t0]], -s), d0);
        if (t0 + 8 < nA) split_e2m1_units(ldexpf(beta[static_cast<int64_t>(kk) * p + Aidx[t0 + 8]], -s), d1);
#pragma unroll
        for (int l = 0; l < LIMBS4; ++l) Bq[(LIMBS4 * kk + l) * rb + t] = static_cast<uint8_t>(d0[l] | (d1[l] << 4));
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
        // K chunk pairs; groups of four chunks for the e2m1 stages of four chunks
        const int64_t ku = ws.g1.CH == 4 ? 512 : 256;
        const int64_t Kpad = std::max<int64_t>(ku, (nA + ku - 1) / ku * ku);
        if (Kpad > h->act_cap) {
            dfree(h->d_Aidx);
            dfree(h->d_A1act);
            h->d_Aidx = nullptr;
            h->d_A1act = nullptr;
            COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_Aidx), Kpad * sizeof(int32_t)));
            COX_TRY(dmalloc(h, reinterpret_cast<void **>(&h->d_A1act), static_cast<size_t>(h->n_pad) * Kpad / 4));
            h->act_cap = Kpad;
        }
        if (nA) COX_CUDA(cudaMemcpyAsync(h->d_Aidx, idx.data(), nA * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        COX_CUDA(cudaMemcpyAsync(h->d_inA, flag.data(), p, cudaMemcpyHostToDevice, st));
        {
            const int64_t KC4 = h->n_pad / TILE, KCa = Kpad / TILE;
            k_gather_active<<<static_cast<unsigned>(KCa * KC4), TILE, 0, st>>>(
                h->d_A4, KC4, h->d_Aidx, nA, KCa, h->kperm_ainv, h->kperm_nb, h->d_A1act);
        }
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
        const int64_t bpk = ws.g1.f4 ? 2 : 1;  // K positions per limb byte
        COX_TRY(dmalloc(h, reinterpret_cast<void **>(&ws.Bqa), static_cast<size_t>(ws.NP) * h->act_Kpad / bpk));
        COX_CUDA(cudaMemsetAsync(ws.Bqa, 0, static_cast<size_t>(ws.NP) * h->act_Kpad / bpk, st));
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
    if (ws.g1.f4)
        k_prep_limbs_active4<<<dim3(static_cast<unsigned>(gx), k), 256, 0, st>>>(
            beta, p, h->d_Aidx, h->nA, h->act_Kpad, h->l1_blocks, ws.bmaxp, ws.Bqa, ws.bs1, h->d_err);
    else
        k_prep_limbs_active<<<dim3(static_cast<unsigned>(gx), k), 256, 0, st>>>(
            beta, p, h->d_Aidx, h->nA, h->act_Kpad, h->l1_blocks, ws.bmaxp, ws.Bqa, ws.bs1, h->d_err);
    COX_CUDA(cudaGetLastError());
    h->launches += 1;
    *use = 1;
    return COX_OK;
}

} // namespace coxgb
