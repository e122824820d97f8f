// gemm_f4.cu -- the e2m1 instantiations of the genotype-product kernel
// (gemm_kernel.cuh): codes as e2m1 nibbles, coefficients as LIMBS4 e2m1 limbs,
// tcgen05.mma kind::mxf4 with unit block scales (K = 64 per instruction).  In a
// translation unit of their own so that the two forms compile in parallel.
#include "gemm_kernel.cuh"

namespace coxgb {

// (T row tiles, CH K chunks, NP limb columns) -> kernel, or null when that
// shape is not compiled.  TMEM (504 columns beside the scale factors): T NP
// accumulator columns and at least G slots of T CH 16 columns.  The limb
// classes stop at 128 columns (k <= 16): a class of N = 192 (six limbs at
// k = 32) faulted on the GPU in its first parity test, and no MMA of N > 128
// is compiled.  One tile x four chunks is compiled at 64 columns only: at 128
// its 32 KB limb slots leave no ring depths that keep every parity wait
// unambiguous (the planner's ring_safe) within 227 KB.
GemmKernelFn pick_kernel_f4(int T, int CH, int NP)
{
    switch ((T * 10 + CH) * 1000 + NP) {
    case 22064: return k_packed_gemm<2, 2, 64, DEC_GROUPS, false, true>;
    case 14064: return k_packed_gemm<1, 4, 64, DEC_GROUPS, false, true>;
    case 22128: return k_packed_gemm<2, 2, 128, DEC_GROUPS, false, true>;
    default: return nullptr;
    }
}

} // namespace coxgb
