// sg_int8_bits_gauss.cu -- instances of the fused int8 kernel for Gaussian
// couplings on the bit-per-chain state in shared memory (half_sweep_bits_gauss:
// work items of 4 sites times chain sets of 8-32 chains, so that the per-site
// index arithmetic and loads are shared by the chains of a set). Same random
// numbers, rule and roundings as the byte-per-chain instances, so the results
// are identical to theirs. A translation unit of its own for parallel
// compilation.
#include "sg_int8_run.cuh"

namespace sg {

namespace {
#define SG_FOR_EACH_BITS_GAUSS_L(X) X(4) X(6) X(8) X(10) X(12) X(14) X(16)
}  // namespace

cudaError_t int8_launch_bits_gauss(int L, const Int8Args &a, const Int8Launch &cfg, cudaStream_t st)
{
#define X(LL) \
    if (L == LL) return launch_t<LL, true, false, false, true>(a, cfg, st);
    SG_FOR_EACH_BITS_GAUSS_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_ctas_per_sm_bits_gauss(int L, int threads, size_t smem)
{
#define X(LL) \
    if (L == LL) return occ_t<LL, true, false, false, true>(threads, smem);
    SG_FOR_EACH_BITS_GAUSS_L(X)
#undef X
    return 0;
}

}  // namespace sg
