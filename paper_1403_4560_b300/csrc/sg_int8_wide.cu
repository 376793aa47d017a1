// sg_int8_wide.cu -- wide shared-memory instances of the fused int8 kernel
// for L = 10 and 12: the same kernel as the narrow instances, bounded at 512
// threads and one CTA per SM instead of 320 threads and two. With many
// temperatures only one sample fits an SM's shared memory, and the narrow
// bound then leaves the SM with at most ten warps. Kept in a translation unit
// of its own so that it compiles in parallel with the other instances.
#include "sg_int8_run.cuh"

namespace sg {

namespace {
#define SG_FOR_EACH_WIDE_L(X) X(10) X(12)
}  // namespace

bool int8_wide_has(int L)
{
#define X(LL) if (L == LL) return true;
    SG_FOR_EACH_WIDE_L(X)
#undef X
    return false;
}

cudaError_t int8_launch_wide(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                             cudaStream_t st)
{
#define X(LL)                                                                 \
    if (L == LL)                                                              \
        return gauss ? launch_t<LL, true, false, true>(a, cfg, st)            \
                     : launch_t<LL, false, false, true>(a, cfg, st);
    SG_FOR_EACH_WIDE_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_ctas_per_sm_wide(int L, bool gauss, int threads, size_t smem)
{
#define X(LL)                                                                 \
    if (L == LL)                                                              \
        return gauss ? occ_t<LL, true, false, true>(threads, smem)            \
                     : occ_t<LL, false, false, true>(threads, smem);
    SG_FOR_EACH_WIDE_L(X)
#undef X
    return 0;
}

}  // namespace sg
