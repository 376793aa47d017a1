// sg_int8_gst.cu -- global-memory instances of the fused int8 kernel: for
// lattices whose state does not fit one CTA's shared memory (L >= 10 with
// many temperatures, and every L from 18 up to 64), the CTA sweeps its
// sample's state in place in HBM/L2. Kept in a translation unit of its own
// so that it compiles in parallel with the shared-memory instances.
#include "sg_int8_run.cuh"

namespace sg {

namespace {
#define SG_FOR_EACH_GST_L(X) \
    X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32) X(40) X(48) X(64)
}  // namespace

bool int8_gst_has(int L)
{
#define X(LL) if (L == LL) return true;
    SG_FOR_EACH_GST_L(X)
#undef X
    return false;
}

cudaError_t int8_launch_gst(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                            cudaStream_t st)
{
#define X(LL)                                                                          \
    if (L == LL)                                                                       \
        return gauss ? launch_t<LL, true, true>(a, cfg, st) : launch_t<LL, false, true>(a, cfg, st);
    SG_FOR_EACH_GST_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_ctas_per_sm_gst(int L, bool gauss, int threads, size_t smem)
{
#define X(LL) \
    if (L == LL) return gauss ? occ_t<LL, true, true>(threads, smem) : occ_t<LL, false, true>(threads, smem);
    SG_FOR_EACH_GST_L(X)
#undef X
    return 0;
}

}  // namespace sg
