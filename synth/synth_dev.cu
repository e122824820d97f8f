/*
 * synth_dev.cu -- device-side copy of the genotype draw in synth.c, for
 * workloads too large to generate on the host (hundreds of GB of codes).
 *
 * Input generation only: no Cox arithmetic lives here.  The draw is the
 * SplitMix64 output function keyed by (seed, stream) at counter (i, j), the
 * same integer-only formula as synth.c, so host and device agree bit for bit.
 * Output: row-major packed codes, ceil(p/4) bytes per row, SNP j in bits
 * 2*(j%4)..2*(j%4)+1 of byte j/4, unused tail bits zero.
 */
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void genotypes_packed_kernel(uint64_t key, const uint32_t *__restrict__ thr,
                                        int64_t p, int64_t i0, int64_t ni, uint8_t *__restrict__ out)
{
    const int64_t rb = (p + 3) / 4;
    const int64_t total = ni * rb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / rb, b = t - r * rb;
        const uint64_t ka = mix64(key + (uint64_t)(i0 + r));
        uint32_t byte = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = 4 * b + q;
            if (j < p) {
                const uint64_t h = mix64(ka ^ (uint64_t)j);
                const uint32_t th = thr[j];
                const uint32_t x = ((uint32_t)h < th) + ((uint32_t)(h >> 32) < th);
                byte |= x << (2 * q);
            }
        }
        out[t] = (uint8_t)byte;
    }
}

} // namespace

extern "C" int syn_dev_genotypes_packed(uint64_t seed, const uint32_t *thr_dev, int64_t p,
                                        int64_t i0, int64_t ni, uint8_t *out_dev, void *stream)
{
    if (p <= 0 || ni < 0 || i0 < 0 || !thr_dev || !out_dev) return -1;
    if (ni == 0) return 0;
    /* stream SYN_STREAM_X = 2, key as in synth.c:syn_draw */
    uint64_t z = seed ^ (2ULL * 0xD1B54A32D192ED03ULL);
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    const uint64_t key = z ^ (z >> 31);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    genotypes_packed_kernel<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(key, thr_dev, p, i0, ni, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
