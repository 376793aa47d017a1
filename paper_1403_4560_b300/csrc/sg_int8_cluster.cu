// sg_int8_cluster.cu -- cluster instances of the fused int8 kernel: one
// disorder sample swept by a thread-block cluster of k CTAs (k = 2, 4 or 8),
// for large lattices when there are fewer samples than SMs (the paper cannot
// equilibrate its largest sizes with one sample per unit of hardware; results
// and conclusion sections). With one CTA per sample, 64 samples of L = 24
// would leave 84 of the 148 SMs idle; split over clusters of two they keep
// 128 busy.
//
// Layout and rule are those of the global-memory instances (the sample's
// packed state swept in place in global memory, one byte per site and 4-slot
// group, sg_int8_run.cuh). CTA `rank` of the cluster owns the z-planes
// [rank * L/k, (rank + 1) * L/k) and sweeps only their work items; a
// half-sweep reads the two boundary planes of its neighbours through L2
// (ld.global.cg), since their CTAs store them from other SMs, and a cluster
// barrier (release / acquire at cluster scope) separates the half-sweeps.
// Rank 0 holds the sample's energies and runs what needs the whole lattice:
// the other ranks add their partial bond sums and magnetisations into its
// shared memory (distributed shared memory atomics), it decides the replica
// exchange and publishes the accepted pairs, which every rank applies to its
// own planes, and it sums the ranks' partial overlap marginals before the
// projections and the FP64 accumulation. The random numbers, the order of
// every floating-point operation and the integer counts are those of the
// one-CTA kernel, so the results are identical to it and to the oracle.
//
// Every cluster barrier below sits on control flow that is the same for all
// CTAs of a cluster (sample loop, sweep loop, schedule, the stop decision,
// which rank 0 publishes), so no CTA can wait at a barrier its peers skip,
// and the kernel ends with a barrier so that no CTA exits while a peer may
// still read its shared memory.
#include <cooperative_groups.h>

#include "sg_int8_run.cuh"

namespace sg {

namespace {

namespace cg = cooperative_groups;

#define SG_FOR_EACH_CLUSTER_L(X) X(20) X(24) X(28) X(32) X(40) X(48) X(64)

template <typename T>
__device__ __forceinline__ T *rank0(cg::cluster_group &cl, T *p)
{
    return cl.map_shared_rank(p, 0);
}

// The measurement of one sweep (eq. overlap): energies and the projections
// at rank 0; the marginals of each chunk of 4-slot words summed there from
// every rank's planes.
template <int L>
__device__ __forceinline__ void measure_cluster(cg::cluster_group &cl, const Smem &sm, const Ctx &cx,
                                                const Int8Args &a, int bin)
{
    constexpr int LL = L * L;
    const int rank = (int)cl.block_rank(), k = (int)cl.num_blocks();
    if (rank == 0) measure_energies(sm, cx, a, bin);
    for (int j0 = 0; j0 < cx.WR; j0 += a.mchunk) {
        const int nw = min(a.mchunk, cx.WR - j0);
        measure_marginals<L, true, true>(sm, cx, j0, nw);
        cl.sync();  // every rank's partial marginals are complete
        if (rank == 0) {
            for (int id = threadIdx.x; id < 3 * LL * nw; id += blockDim.x) {
                uint32_t v = sm.marg[id];
                for (int r = 1; r < k; ++r) v += cl.map_shared_rank(sm.marg, r)[id];
                sm.marg[id] = v;  // per byte (or 16-bit) lane at most L: no carries
            }
            __syncthreads();
            measure_projections<L>(sm, cx, a, bin, j0, nw);
        }
        // the next chunk's partial marginals overwrite this chunk's: rank 0
        // must have read them first
        if (j0 + a.mchunk < cx.WR) cl.sync();
    }
}

template <int L, bool GAUSS>
__global__ void __launch_bounds__(KernelBounds<L, true>::threads, 1)
    int8_cluster_kernel(const __grid_constant__ Int8Args a)
{
    constexpr int N = L * L * L;
    constexpr int H = L / 2;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), k = (int)cl.num_blocks();
    Smem sm;
    carve(smem_raw, L, a.Tp, GAUSS, a.mchunk, &sm, true);
    Ctx cx;
    cx.k0r = a.k0r;
    cx.nt = a.nt;
    cx.Tp = a.Tp;
    cx.WR = a.Tp / 4;
    cx.RB = a.Tp / 4;  // packed state: one byte per site and 4-slot group
    cx.seed_lo = a.seed_lo;
    cx.seed_hi = a.seed_hi;
    cx.hq = a.h_f;
    // this CTA's planes; L % 4 == 0 makes each plane's colour sites a whole
    // number of 4-site work items (L * L / 2 divisible by 4)
    const int zs = L / k;
    cx.z0 = rank * zs;
    cx.z1 = cx.z0 + zs;
    cx.u0 = cx.z0 * L * H / kSiteRun;
    cx.u1 = cx.z1 * L * H / kSiteRun;
    const long long t_start = clock64();

    for (int q = threadIdx.x; q < a.Tp; q += blockDim.x) {
        sm.negbeta[q] = a.negbeta[q];
        sm.dbeta[q] = a.dbeta[q];
    }
    for (int q = threadIdx.x; q < 2 * L; q += blockDim.x) sm.twid[q] = a.twid[q];
    if (!GAUSS)
        for (int q = threadIdx.x; q < a.Tp * 16; q += blockDim.x) sm.thr[q] = a.thr[q];
    if (threadIdx.x < 2) sm.ctl[threadIdx.x] = 0;  // stop flags, alternating by sweep
    cl.sync();  // rank 0's flags are cleared before any rank can set one

    const int c = blockIdx.x / k, n_clusters = gridDim.x / k;
    bool stop = false;
    for (int64_t s = a.s_begin + c; s < a.s_end && !stop; s += n_clusters) {
        cx.s = s;
        cx.k1 = (uint32_t)((s + a.s_key0) / a.rng_group);
        sm.spins = a.spins + (size_t)s * N * cx.RB;
        if (!GAUSS)
            sm.J8 = const_cast<uint8_t *>(a.J8) + (size_t)s * N * 8;
        else
            sm.Jg = const_cast<float *>(a.Jg) + (size_t)s * 3 * N;
        for (int q = threadIdx.x; q < 2 * a.Tp; q += blockDim.x) {
            sm.xflag[q] = 0;
            sm.B[q] = rank == 0 ? (unsigned long long)a.B[s * 2 * a.Tp + q] : 0ull;
            sm.M[q] = rank == 0 ? (unsigned long long)a.M[s * 2 * a.Tp + q] : 0ull;
        }
        __syncthreads();
        uint32_t stamp = 0;
        const int64_t sweep0 = a.sweep0_dev ? *a.sweep0_dev : a.sweep0;
        for (int it = 0; it < a.n_sweeps; ++it) {
            const int64_t n = sweep0 + it;
            if (a.watchdog || a.cancel) {  // launch-uniform branch
                // each rank may see its own reason; rank 0's flag for this
                // sweep collects them, and every rank reads it after the
                // barrier, so all ranks stop together
                if (threadIdx.x == 0) {
                    int why = 0;
                    if (a.watchdog && (unsigned long long)(clock64() - t_start) > a.watchdog)
                        why = (int)SG_ETIMEOUT;
                    else if (a.cancel && *a.cancel)
                        why = (int)SG_ECANCELLED;
                    if (why) {
                        atomicCAS(a.status, 0, why);
                        atomicOr(rank0(cl, &sm.ctl[it & 1]), 1);
                    }
                }
                cl.sync();
                int f = 0;
                if (threadIdx.x == 0) f = *rank0(cl, &sm.ctl[it & 1]);
                // the other flag was last read before this barrier by every
                // rank, and is next set after the next one
                if (rank == 0 && threadIdx.x == 0) sm.ctl[(it + 1) & 1] = 0;
                stop = __syncthreads_or(f != 0);
                if (stop) break;
            }
            half_sweep_packed<L, GAUSS, true>(sm, cx, (uint32_t)n, 0);
            for (int q = threadIdx.x; q < 2 * a.Tp; q += blockDim.x) {
                sm.B[q] = 0;
                sm.M[q] = 0;
            }
            cl.sync();  // colour 0 stored everywhere; rank 0's sums are zero
            half_sweep_packed<L, GAUSS, true>(sm, cx, (uint32_t)n, 1);
            __syncthreads();
            if (rank != 0)
                for (int q = threadIdx.x; q < 2 * a.Tp; q += blockDim.x) {
                    atomicAdd(rank0(cl, &sm.B[q]), sm.B[q]);
                    atomicAdd(rank0(cl, &sm.M[q]), sm.M[q]);
                }
            cl.sync();  // colour 1 stored everywhere; rank 0 holds the sample's B and M
            if (a.exchange_every > 0 && (n + 1) % a.exchange_every == 0) {
                const int64_t e = (n + 1) / a.exchange_every - 1;
                ++stamp;
                if (rank == 0 && threadIdx.x < 32)
                    exchange_decide(sm, cx, a, (int)(e & 1), (uint32_t)n, 0u, stamp);
                cl.sync();  // the accepted pairs are published
                if (rank != 0 && threadIdx.x < 2) sm.accm[threadIdx.x] = *rank0(cl, &sm.accm[threadIdx.x]);
                __syncthreads();
                exchange_apply_packed<L>(sm, cx, cx.z0 * L * L, cx.z1 * L * L);
                cl.sync();  // swapped planes stored before anyone reads them
            }
            if (n >= a.n_therm && (n - a.n_therm) % a.measure_every == 0)
                measure_cluster<L>(cl, sm, cx, a, log_bin(n, a.n_bins));
        }
        __syncthreads();
        if (rank == 0)
            for (int q = threadIdx.x; q < 2 * a.Tp; q += blockDim.x) {
                a.B[s * 2 * a.Tp + q] = (int64_t)sm.B[q];
                a.M[s * 2 * a.Tp + q] = (int64_t)sm.M[q];
            }
        // rank 0's shared memory (sums, pairs, marginals) is read by the other
        // ranks within a sample only; the barrier keeps the next sample's
        // writes behind every read of this one
        cl.sync();
    }
    cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

template <int L, bool G>
cudaError_t ensure_cluster_attr()
{
    static cudaError_t done = cudaFuncSetAttribute(
        int8_cluster_kernel<L, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    return done;
}

template <int L, bool G>
cudaError_t launch_cluster_t(const Int8Args &a, const Int8Launch &c, cudaStream_t st)
{
    cudaError_t e = ensure_cluster_attr<L, G>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)c.grid, 1, 1);
    cfg.blockDim = dim3((unsigned)c.threads, 1, 1);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, int8_cluster_kernel<L, G>, a);
}

template <int L, bool G>
int clusters_t(int threads, size_t smem, int k)
{
    if (ensure_cluster_attr<L, G>() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)k, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)k;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, int8_cluster_kernel<L, G>, &cfg) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of a refused shape
        return 0;
    }
    return n;
}

}  // namespace

bool int8_cluster_has(int L)
{
#define X(LL) if (L == LL) return true;
    SG_FOR_EACH_CLUSTER_L(X)
#undef X
    return false;
}

cudaError_t int8_launch_cluster(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                                cudaStream_t st)
{
    if (cfg.cluster < 2 || cfg.grid % cfg.cluster != 0 || L % cfg.cluster != 0)
        return cudaErrorInvalidValue;
#define X(LL)                                                                                \
    if (L == LL)                                                                             \
        return gauss ? launch_cluster_t<LL, true>(a, cfg, st) : launch_cluster_t<LL, false>(a, cfg, st);
    SG_FOR_EACH_CLUSTER_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_active_clusters(int L, bool gauss, int threads, size_t smem, int k)
{
#define X(LL) \
    if (L == LL) return gauss ? clusters_t<LL, true>(threads, smem, k) : clusters_t<LL, false>(threads, smem, k);
    SG_FOR_EACH_CLUSTER_L(X)
#undef X
    return 0;
}

}  // namespace sg
