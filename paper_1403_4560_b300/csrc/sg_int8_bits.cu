// sg_int8_bits.cu -- bit-parallel instances of the fused int8 kernel for
// +-J couplings (the Gaussian ones are in sg_int8_bits_gauss.cu): the
// sample's chains packed one bit each (the paper's multispin coding of one
// sample's replicas, methods section) and held in
// shared memory; the unsatisfied-bond count of 64 chains is one bit-sliced
// add, while every chain keeps its own Metropolis random words. The random
// numbers, thresholds and summation orders are those of the byte-per-chain
// instances, so the results are identical to theirs. Kept in a translation
// unit of its own so that it compiles in parallel with the other instances.
#include "sg_int8_run.cuh"

namespace sg {

namespace {
#define SG_FOR_EACH_BITS_L(X) X(4) X(6) X(8) X(10) X(12) X(14) X(16)
}  // namespace

bool int8_bits_has(int L)
{
#define X(LL) if (L == LL) return true;
    SG_FOR_EACH_BITS_L(X)
#undef X
    return false;
}

size_t int8_smem_bytes_bits(int L, int Tp, int mchunk, bool gauss)
{
    if (!int8_bits_has(L) || Tp % 32 != 0) return 0;
    const size_t b = carve(nullptr, L, Tp, gauss, mchunk, nullptr, false, true);
    return b <= (size_t)kMaxSmem ? b : 0;
}

cudaError_t int8_launch_bits(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                             cudaStream_t st)
{
    if (gauss) return int8_launch_bits_gauss(L, a, cfg, st);
#define X(LL) \
    if (L == LL) return launch_t<LL, false, false, false, true>(a, cfg, st);
    SG_FOR_EACH_BITS_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_ctas_per_sm_bits(int L, bool gauss, int threads, size_t smem)
{
    if (gauss) return int8_ctas_per_sm_bits_gauss(L, threads, smem);
#define X(LL) \
    if (L == LL) return occ_t<LL, false, false, false, true>(threads, smem);
    SG_FOR_EACH_BITS_L(X)
#undef X
    return 0;
}

}  // namespace sg
