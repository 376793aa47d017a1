// sg_api.cpp -- host side of the C ABI declared in include/sgmc.h.
//
// Owns ensembles (device arena, tables, stream), builds the per-temperature
// tables on the host (acceptance thresholds from the C library's exp, FP32
// inverse temperatures, DFT twiddles), picks launch shapes and drives the
// fused kernels, alone or batched through a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sg_internal.h"
#include "sg_msc.h"

using namespace sg;

namespace {

thread_local std::string g_last_error;

sg_status fail(sg_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

sg_status cuda_fail(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SG_ENOMEM : SG_ECUDA;
}

#define SG_CUDA(call, where)                           \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// True when every byte is +1 (0x01) or -1 (0xFF); eight bytes per test:
// x = w ^ 0x01.. has bytes 0x00 or 0xFE exactly when the spins are valid.
bool spins_valid(const int8_t *p, size_t n)
{
    const uint64_t ones = 0x0101010101010101ull;
    size_t k = 0;
    for (; k + 8 <= n; k += 8) {
        uint64_t w;
        std::memcpy(&w, p + k, 8);
        const uint64_t x = w ^ ones;
        const uint64_t z = (x >> 1) & 0x7F7F7F7F7F7F7F7Full;  // 0x00 or 0x7F per byte
        if ((x & ones) | ((z + ones) & 0x7E7E7E7E7E7E7E7Eull)) return false;
    }
    for (; k < n; ++k)
        if (p[k] != 1 && p[k] != -1) return false;
    return true;
}

}  // namespace

struct sg_ensemble {
    int L = 0, nt = 0, Tp = 0, layout = 0;
    bool gauss = false;
    int64_t S = 0;
    double h = 0.0, h_used = 0.0;
    uint64_t seed = 0;
    sg_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t branch = nullptr;  // private stream for batched branches
    cudaEvent_t ev = nullptr;
    int device = 0;
    int num_sms = 148;
    // device arena and views
    void *arena = nullptr;
    size_t bytes = 0;
    uint8_t *spins = nullptr, *J8 = nullptr;
    float *Jg = nullptr;
    int64_t *B = nullptr, *M = nullptr;
    double *acc = nullptr;
    unsigned long long *hist = nullptr;  // [nt][n_bins][N+1] or null
    int n_bins = 1;
    size_t acc_bytes = 0, hist_bytes = 0;  // acc, then hist right after it
    uint32_t *thr = nullptr;
    float *negbeta = nullptr, *dbeta = nullptr, *twid = nullptr;
    int *status = nullptr;
    int64_t *sweep_ctr = nullptr;
    unsigned int *work = nullptr;  // int8: segmented-launch counters [1 + S]
    int64_t sweeps_done = 0;
    int64_t exchanges_done = 0;
    std::vector<double> T;
    Int8Launch launch{};
    int mchunk = 1;
    // multispin-coded +-J layout
    bool msc = false;
    uint64_t *W = nullptr, *Jw = nullptr, *masks = nullptr;
    // device staging of canonical host arrays, allocated on first use
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // asynchronous spin uploads: own buffer and copy stream (first use);
    // up_done: the copy has landed; up_free: the import has read the buffer
    void *upload = nullptr;
    void *acc_download = nullptr;  // canonical accumulators for async downloads
    // int8 with global-memory state: the state is packed (a byte per site and
    // 4-slot group); other int8 kernels run on this byte-per-chain copy, part
    // of the arena
    uint8_t *unpacked = nullptr;
    size_t spins_bytes = 0;       // bytes of the state in the arena
    cudaStream_t copy = nullptr;
    cudaEvent_t up_done = nullptr, up_free = nullptr;
};

namespace {

std::mutex g_graph_mu;
struct GraphEntry {
    std::vector<sg_ensemble *> ens;
    cudaGraphExec_t exec = nullptr;
};
std::map<std::string, GraphEntry> g_graphs;

void purge_graphs(sg_ensemble *e)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (std::find(it->second.ens.begin(), it->second.ens.end(), e) != it->second.ens.end()) {
            cudaGraphExecDestroy(it->second.exec);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

struct ArenaPlan {
    size_t spins, unpacked, J, BM, acc, hist, thr, tab, twid, misc, total;
};

int bins_of(const sg_options &o) { return o.log_bins > 1 ? o.log_bins : 1; }

ArenaPlan plan_arena(int L, int nt, int Tp, int64_t S, bool gauss, bool msc, int n_bins,
                     bool hist, bool packed)
{
    const size_t N = (size_t)L * L * L;
    ArenaPlan p{};
    if (msc) {
        // 64 samples per word: W [S/64][nt][2][N], Jw [S/64][3][N], masks [S/64][2][nt]
        p.spins = align256((size_t)(S / 64) * nt * 2 * N * 8);
        p.J = align256((size_t)(S / 64) * 3 * N * 8);
    } else {
        p.spins = align256((size_t)S * N * (packed ? Tp / 4 : 2 * Tp));
        p.unpacked = packed ? align256((size_t)S * N * 2 * Tp) : 0;
        p.J = align256(gauss ? (size_t)S * 3 * N * sizeof(float) : (size_t)S * N * 8);
    }
    p.BM = align256((size_t)S * 2 * Tp * sizeof(int64_t));
    p.acc = align256((size_t)S * nt * n_bins * SG_NACC * sizeof(double));
    p.hist = hist ? align256((size_t)nt * n_bins * (N + 1) * sizeof(uint64_t)) : 0;
    p.thr = align256((size_t)Tp * 16 * sizeof(uint32_t));
    p.tab = align256((size_t)Tp * sizeof(float));
    p.twid = align256((size_t)2 * L * sizeof(float));
    // int8: the segmented launch's unit counter and per-sample progress
    p.misc = 256 + (msc ? align256((size_t)(S / 64) * 2 * nt * 8)
                        : align256((size_t)(1 + S) * sizeof(unsigned int)));
    p.total = p.spins + p.unpacked + p.J + 2 * p.BM + p.acc + p.hist + p.thr + 2 * p.tab + p.twid +
              p.misc;
    return p;
}

int pad_slots(int nt) { return (nt + 3) & ~3; }
// Whether the +-J chains are kept one bit each in shared memory and swept
// bit-parallel (sg_options.state_mode 3, or the library's choice where it
// measured faster than a byte per chain on B300: L >= 14, or L >= 10 with
// more than 16 temperatures; +-J, 1184 samples, attempts/ns byte -> bit:
// L = 10, 24 / 56 T 395 -> 445 / 398 -> 480; L = 12, 24 / 56 T 435 -> 444 /
// 433 -> 463; L = 14, 8 / 56 T 217 -> 259 / 398 -> 501; L = 16, 24 T 388 ->
// 550; slower at L <= 8 and with 8 temperatures below L = 14). The random
// numbers are the same either way, so results do not depend on it.
bool use_bits(int L, int nt, sg_coupling dist, const sg_options &o)
{
    if (o.state_mode == 3) return true;
    return o.state_mode == 0 && o.layout == SG_LAYOUT_INT8 && dist == SG_PM_J && nt <= 64 &&
           int8_bits_has(L) && (L >= 14 || (L >= 10 && nt > 16));
}

// Slots as stored: 4-slot groups, or for the bit-parallel state whole 64-bit
// words of a site row (32 slots of both replicas).
int stored_slots(int L, int nt, sg_coupling dist, const sg_options &o)
{
    return use_bits(L, nt, dist, o) ? (nt + 31) & ~31 : pad_slots(nt);
}

// Autotuned launch shapes per problem shape (L, slots, distribution, mode).
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tuned;  // -> (threads, mchunk)

std::string tune_key(const sg_ensemble *e, const Int8Launch &c)
{
    return std::to_string(e->L) + ":" + std::to_string(e->Tp) + ":" + (e->gauss ? "g" : "j") +
           (c.gst ? ":gst" : c.wide ? ":wide" : ":smem");
}

// Cluster split of the global-memory state (sg_options.cluster): with fewer
// samples than SMs one CTA per sample leaves SMs idle; a cluster of k CTAs
// per sample (each sweeping L/k z-planes) runs S samples in ceil(S / C)
// waves of C resident clusters, each sample k times faster at best. The
// library picks the k in {2, 4, 8} (L % k == 0) with the most effective CTAs
// S * k / ceil(S / C), the smallest on ties (fewer barriers and halo planes
// per sweep), and only when that beats one CTA per sample. (B300, Gaussian,
// 64 samples, 2 x 16 temperatures, attempts/ns at L = 24 / 32: one CTA per
// sample 148 / 158; k = 2 (74 resident clusters) 245 / 273; k = 4, whose 37
// resident clusters leave a ragged second wave, 179 / 231.)
sg_status configure_cluster(sg_ensemble *e, int64_t resident)
{
    const int want = e->opt.cluster;
    if (want == 1) return SG_OK;
    const int L = e->L;
    if (!int8_cluster_has(L)) {
        if (want > 1) return fail(SG_EUNSUPPORTED, "no cluster kernel for this lattice size");
        return SG_OK;
    }
    auto effective = [&](int64_t par, int64_t k) {  // CTAs doing useful work, per wave
        return (double)(e->S * k) / (double)((e->S + par - 1) / par);
    };
    double best_eff = effective(std::max<int64_t>(resident, 1), 1);  // one CTA per sample
    int best_k = 1, best_grid = e->launch.grid;
    for (int k = 2; k <= 8; k *= 2) {
        if (L % k != 0 || (want > 1 && k != want)) continue;
        const int nc = int8_active_clusters(L, e->gauss, e->launch.threads, e->launch.smem, k);
        if (nc <= 0) continue;
        const double eff = effective(nc, k);
        if (want > 1 || (e->S < e->num_sms && eff > best_eff * 1.001)) {
            best_eff = eff;
            best_k = k;
            best_grid = (int)(std::min<int64_t>(e->S, nc) * k);
        }
    }
    if (want > 1 && best_k != want)
        return fail(SG_EUNSUPPORTED, "the requested cluster size cannot run for this lattice");
    e->launch.cluster = best_k;
    e->launch.grid = best_grid;
    return SG_OK;
}

// Launch shape: threads per CTA are a multiple of int8_thread_quantum (each
// thread keeps one (4-slot group, replica) pair for the whole half-sweep); among the candidates the
// one with the best product of work balance and resident warps per SM wins,
// then the largest measurement chunk that keeps that occupancy.
// The bit-parallel instances: one warp per task (32 work items of one word
// of the site row), at most 8 warps per CTA, so that small lattices run more
// CTAs per SM rather than idle warps; the measurement chunk that keeps the
// most CTAs per SM.
// The most CTAs per SM over the measurement chunks, and that chunk.
static int bits_occupancy(const sg_ensemble *e, int threads, int *m_for)
{
    int occ = 0;
    *m_for = 0;
    for (int m = e->Tp / 4; m >= 1; --m) {
        const size_t smem = int8_smem_bytes_bits(e->L, e->Tp, m, e->gauss);
        if (!smem) continue;
        const int o = int8_ctas_per_sm_bits(e->L, e->gauss, threads, smem);
        if (o > occ) {
            occ = o;
            *m_for = m;
        }
    }
    return occ;
}

// Gaussian couplings on the bit-per-chain state: a warp task is 32 work
// items times a chain set of csb 4-slot groups (1, 2 or 4). Larger sets share
// the per-site work of a task (indices, 13 loads per site) among more chains;
// smaller ones make more tasks, which balance the warps of a CTA better. The
// model: a task costs kSetup + (its chains) chain units, warps take tasks
// round-robin, and a shape scores its balance (work over warps x the
// longest warp) x the chain share of the work x the resident warps per SM
// (up to 16, enough to keep the schedulers issuing). A requested
// threads_per_block fixes the warps.
static void bits_gauss_shape(const sg_ensemble *e, int *csb_out, int *warps_out)
{
    constexpr double kSetup = 1.5;
    const int L = e->L, nt = e->nt;
    const int items = (L * L * L / 2) / int8_site_run(L, false);
    const int nub = (items + 31) / 32, ngrp = (nt + 3) / 4;
    const int64_t per_sm = (e->S + e->num_sms - 1) / e->num_sms;
    const int want_w = e->opt.threads_per_block > 0
                           ? std::max(1, std::min(8, e->opt.threads_per_block / 32)) : 0;
    double best = -1.0;
    *csb_out = 1;
    *warps_out = 1;
    for (int csb = 4; csb >= 1; csb /= 2) {
        if (e->opt.chain_set > 0 && csb != e->opt.chain_set) continue;
        const int ncs = (ngrp + csb - 1) / csb;
        std::vector<double> cost((size_t)nub * ncs);
        double work = 0.0, chains = 0.0;
        for (int tk = 0; tk < nub * ncs; ++tk) {
            const int cs = tk % ncs;
            const int t0 = 4 * cs * csb, t1 = std::min(nt, 4 * (cs + 1) * csb);
            const double ch = 2.0 * (t1 - t0);
            cost[tk] = kSetup + ch;
            work += cost[tk];
            chains += ch;
        }
        for (int w = 1; w <= 8; ++w) {
            if (want_w && w != want_w) continue;
            double longest = 0.0;
            for (int k = 0; k < w; ++k) {
                double c = 0.0;
                for (int tk = k; tk < nub * ncs; tk += w) c += cost[tk];
                longest = std::max(longest, c);
            }
            int m = 0;
            const int occ = bits_occupancy(e, 32 * w, &m);
            if (!occ) continue;
            const double resident = (double)std::min<int64_t>(occ, per_sm) * w;
            const double score =
                work / (w * longest) * (chains / work) * std::min(resident, 16.0);
            if (score > best * 1.0001) {
                best = score;
                *csb_out = csb;
                *warps_out = w;
            }
        }
    }
}

sg_status configure_bits(sg_ensemble *e)
{
    const int L = e->L;
    if (!int8_bits_has(L)) return fail(SG_EUNSUPPORTED, "no bit-parallel kernel for this lattice size");
    int t, csb = 0;
    if (e->gauss) {
        int w = 1;
        bits_gauss_shape(e, &csb, &w);
        t = 32 * w;
    } else {
        const int items = (L * L * L / 2) / int8_site_run(L, false);
        const int tasks = ((items + 31) / 32) * (e->Tp / 32);
        t = 32 * std::min(tasks, 8);
    }
    int m_for = 0;
    const int occ = bits_occupancy(e, t, &m_for);
    if (!occ) return fail(SG_EUNSUPPORTED, "the bit-parallel state does not fit shared memory");
    e->mchunk = m_for;
    e->launch = Int8Launch{};
    e->launch.threads = t;
    e->launch.bits = true;
    e->launch.csb = csb;
    e->launch.cluster = 1;
    e->launch.smem = int8_smem_bytes_bits(L, e->Tp, m_for, e->gauss);
    e->launch.grid = (int)std::min<int64_t>(e->S, (int64_t)occ * e->num_sms);
    return SG_OK;
}

sg_status configure_launch(sg_ensemble *e)
{
    if (use_bits(e->L, e->nt, e->gauss ? SG_GAUSS : SG_PM_J, e->opt)) return configure_bits(e);
    const int WR = e->Tp / 4;
    const int L = e->L;
    // shared-memory residency first; the global-memory variant when the
    // sample's state does not fit (large L or many temperatures)
    for (int pass = 0; pass < 2; ++pass) {
        const bool gst = pass == 1;
        if ((e->opt.state_mode == 1 && gst) || (e->opt.state_mode == 2 && !gst)) continue;
        const int Q = int8_thread_quantum(e->Tp, gst);  // thread counts are multiples of Q
        const int items = (L * L * L / 2) / int8_site_run(L, gst) * Q;
        double best_score = -1e300;  // scores of requested sizes are negative
        int best_t = 0, best_m = 0, best_occ = 0;
        bool best_wide = false;
        // in shared memory, L = 10 and 12 have two instances: two CTAs per SM
        // of up to 320 threads, or one of up to 512 (many temperatures, or
        // fewer samples than twice the SMs); the same score picks between them
        for (int v = 0; v < (gst ? 1 : 2); ++v) {
            const bool wide = v == 1;
            if (wide && !int8_wide_has(L)) continue;
            const int maxt = int8_max_threads(e->L, gst, wide);
            for (int t = Q; t <= maxt; t += Q) {
                if (t < 32) continue;  // the measurement needs one full warp
                // a request is clamped to what the instance allows
                const int req = (std::min(e->opt.threads_per_block, maxt) / Q) * Q;
                if (e->opt.threads_per_block > 0 && t != std::max(((32 + Q - 1) / Q) * Q, req))
                    continue;
                int occ = 0, m_for = 0;
                for (int m = WR; m >= 1; --m) {
                    const size_t smem = int8_smem_bytes(L, e->Tp, e->gauss, m, gst);
                    if (!smem) continue;
                    const int o = int8_ctas_per_sm(L, e->gauss, t, smem, gst, wide);
                    if (o > occ) {
                        occ = o;
                        m_for = m;
                    }
                }
                if (!occ) continue;
                // useful threads per SM: work items in flight per round, over the
                // CTAs an SM actually gets (one CTA per sample, so never more than
                // ceil(S / SMs)); ties go to wider CTAs, i.e. fewer rounds of work
                // items between barriers (measured on B300: +-J, L = 14, 16 T,
                // 392 x 1 CTA at 305 attempts/ns against 200 x 2 at 163)
                const int64_t per_sm = (e->S + e->num_sms - 1) / e->num_sms;
                const int eff = (int)std::min<int64_t>(occ, per_sm);
                const int rounds = (items + t - 1) / t;
                const double useful = (double)items / rounds * eff;
                // packed global-memory state: one wide CTA per SM measured best
                // (the whole L1 for one sample's planes, no ragged second wave
                // when samples are not a multiple of the SMs)
                // a requested CTA size: the instance that comes closest to it
                const double score =
                    gst                              ? (double)t
                    : e->opt.threads_per_block > 0 ? -std::abs(t - e->opt.threads_per_block) + 1e-6 * useful
                                                     : std::min(useful, 1024.0) + 1e-3 * t;
                if (score > best_score) {
                    best_score = score;
                    best_t = t;
                    best_m = m_for;
                    best_occ = occ;
                    best_wide = wide;
                }
            }
        }
        if (best_occ == 0) continue;
        Int8Launch cand{};
        cand.gst = gst;
        cand.wide = best_wide;
        if (e->opt.threads_per_block <= 0) {  // a tuned shape for this problem wins
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(tune_key(e, cand));
            if (it != g_tuned.end()) {
                const size_t smem = int8_smem_bytes(L, e->Tp, e->gauss, it->second.second, gst);
                const int occ =
                    smem ? int8_ctas_per_sm(L, e->gauss, it->second.first, smem, gst, best_wide) : 0;
                if (occ > 0) {
                    best_t = it->second.first;
                    best_m = it->second.second;
                    best_occ = occ;
                }
            }
        }
        e->mchunk = best_m;
        e->launch.threads = best_t;
        e->launch.gst = gst;
        e->launch.wide = best_wide;
        e->launch.bits = false;
        e->launch.cluster = 1;
        e->launch.smem = int8_smem_bytes(L, e->Tp, e->gauss, best_m, gst);
        const int64_t resident = (int64_t)best_occ * e->num_sms;
        e->launch.grid = (int)std::min<int64_t>(e->S, resident);
        return gst ? configure_cluster(e, resident) : SG_OK;
    }
    return fail(SG_EUNSUPPORTED, "no int8 kernel serves this lattice size");
}

Int8Args make_args(sg_ensemble *e)
{
    Int8Args a{};
    a.spins = e->spins;
    a.J8 = e->J8;
    a.Jg = e->Jg;
    a.B = e->B;
    a.M = e->M;
    a.acc = e->acc;
    a.hist = e->hist;
    a.n_bins = e->n_bins;
    a.thr = e->thr;
    a.negbeta = e->negbeta;
    a.dbeta = e->dbeta;
    a.twid = e->twid;
    a.status = e->status;
    a.S = e->S;
    a.nt = e->nt;
    a.Tp = e->Tp;
    a.h_f = (float)e->h_used;
    a.qJ_f = e->gauss ? (1.0f / 131072.0f) : 1.0f;
    a.h_d = e->h_used;
    a.qJ_d = e->gauss ? (1.0 / 131072.0) : 1.0;
    a.seed_lo = (uint32_t)e->seed;
    a.seed_hi = (uint32_t)(e->seed >> 32);
    a.rng_group = e->opt.rng_group;
    a.sweep0 = e->sweeps_done;
    a.sweep0_dev = nullptr;
    a.n_sweeps = 0;
    a.exchange_every = e->opt.exchange_every;
    a.measure_every = e->opt.measure_every;
    a.n_therm = e->opt.n_therm;
    a.mchunk = e->mchunk;
    a.watchdog = e->opt.watchdog_cycles;
    a.cancel = nullptr;
    a.s_begin = 0;
    a.s_end = e->S;
    a.s_key0 = e->opt.sample_base;
    a.work = e->work;
    a.n_seg = 1;
    a.seg_wait = 1ull << 30;
    for (int r = 0; r < 10; ++r) a.k0r[r] = (a.seed_lo ^ 0x4D455452u) + (uint32_t)r * 0x9E3779B9u;
    a.csb = e->launch.csb;
    return a;
}

MscArgs make_msc_args(sg_ensemble *e)
{
    MscArgs a{};
    a.W = e->W;
    a.Jw = e->Jw;
    a.B = e->B;
    a.M = e->M;
    a.acc = e->acc;
    a.hist = e->hist;
    a.n_bins = e->n_bins;
    a.thr = e->thr;
    a.dbeta = e->dbeta;
    a.twid = e->twid;
    a.G = e->S / 64;
    a.nt = e->nt;
    a.h_f = (float)e->h_used;
    a.h_d = e->h_used;
    a.seed_lo = (uint32_t)e->seed;
    a.seed_hi = (uint32_t)(e->seed >> 32);
    a.sweep0 = e->sweeps_done;
    a.sweep0_dev = nullptr;
    a.sweep_offset = 0;
    a.exchange_every = e->opt.exchange_every;
    a.measure_every = e->opt.measure_every;
    a.n_therm = e->opt.n_therm;
    a.s_key0 = e->opt.sample_base;
    a.status = e->status;
    for (int r = 0; r < 10; ++r) a.k0r[r] = (a.seed_lo ^ 0x4D455452u) + (uint32_t)r * 0x9E3779B9u;
    return a;
}

// Staging buffer of at least `bytes` for host <-> canonical-layout copies;
// grows on demand (after the stream has drained) and lives with the ensemble.
cudaError_t stage_buffer(sg_ensemble *e, size_t bytes, void **out)
{
    if (e->stage_bytes < bytes) {
        cudaError_t ce = cudaStreamSynchronize(e->stream);
        if (ce != cudaSuccess) return ce;
        if (e->stage) cudaFree(e->stage);
        e->stage = nullptr;
        e->stage_bytes = 0;
        ce = cudaMalloc(&e->stage, bytes);
        if (ce != cudaSuccess) return ce;
        e->stage_bytes = bytes;
    }
    *out = e->stage;
    return cudaSuccess;
}

// The int8 state in the byte-per-chain layout every kernel but the fused one
// works on: the state itself, or (packed state of the global-memory
// instances) the ensemble's scratch copy, unpacked from the state when fill.
cudaError_t unpacked_view(sg_ensemble *e, uint8_t **out, bool fill)
{
    if (!e->unpacked) {
        *out = e->spins;
        return cudaSuccess;
    }
    *out = e->unpacked;
    return fill ? int8_unpack_spins(e->unpacked, e->spins, e->S, e->L, e->Tp, e->stream)
                : cudaSuccess;
}

// After the byte-per-chain view was changed: pack it back into the state
// (a no-op when the view is the state). skip: as for the imports.
cudaError_t commit_unpacked(sg_ensemble *e, const uint8_t *view, const int *skip)
{
    if (view == e->spins) return cudaSuccess;
    return int8_pack_spins(e->spins, view, e->S, e->L, e->Tp, e->stream, skip);
}

// Host tables: +-J thresholds (FP64 exp of the C library), FP32 -beta and
// beta differences, FP32 twiddles of the DFT.
void host_tables(const sg_ensemble *e, std::vector<uint32_t> &thr, std::vector<float> &nb,
                 std::vector<float> &db, std::vector<float> &tw)
{
    thr.assign((size_t)e->Tp * 16, 0u);
    nb.assign((size_t)e->Tp, 0.0f);
    db.assign((size_t)e->Tp, 0.0f);
    for (int t = 0; t < e->nt; ++t) {
        const double beta = 1.0 / e->T[(size_t)t];
        nb[(size_t)t] = -(float)beta;
        if (t + 1 < e->nt) db[(size_t)t] = (float)(beta - 1.0 / e->T[(size_t)t + 1]);
        for (int sb = 0; sb < 2; ++sb)
            for (int u = 0; u <= 6; ++u) {
                const double dE = (double)(12 - 4 * u) + (sb ? -2.0 * e->h_used : 2.0 * e->h_used);
                uint32_t v;
                if (dE <= 0.0) {
                    v = 0xFFFFFFFFu;
                } else {
                    const double p = std::floor(std::exp(-(beta * dE)) * 4294967296.0);
                    v = p >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)p;
                }
                thr[(size_t)t * 16 + sb * 8 + u] = v;
            }
    }
    tw.assign((size_t)2 * e->L, 0.0f);
    for (int d = 0; d < e->L; ++d) {
        const double ang = ((2.0 * M_PI) * (double)d) / (double)e->L;
        tw[(size_t)d] = (float)std::cos(ang);
        tw[(size_t)e->L + d] = (float)std::sin(ang);
    }
}

sg_status validate(int L, const double *T, int nt, sg_coupling dist, int64_t S,
                   const sg_options &o)
{
    if (L < 2 || (L & 1) || L > 64) return fail(SG_EINVAL, "L must be even and in [2, 64]");
    if (nt < 1 || nt > 64) return fail(SG_EINVAL, "n_T must be in [1, 64]");
    if (!T) return fail(SG_EINVAL, "temperature array is NULL");
    for (int t = 0; t < nt; ++t) {
        if (!(T[t] > 0.0) || !std::isfinite(T[t]))
            return fail(SG_EINVAL, "temperatures must be finite and positive");
        if (t > 0 && !(T[t] > T[t - 1]))
            return fail(SG_EINVAL, "temperatures must be strictly ascending");
    }
    if (dist != SG_PM_J && dist != SG_GAUSS) return fail(SG_EINVAL, "unknown coupling distribution");
    if (S < 1 || S > (int64_t)1 << 31) return fail(SG_EINVAL, "n_samples must be in [1, 2^31]");
    if (o.rng_group < 1) return fail(SG_EINVAL, "rng_group must be >= 1");
    if (o.exchange_every < 0) return fail(SG_EINVAL, "exchange_every must be >= 0");
    if (o.measure_every < 1) return fail(SG_EINVAL, "measure_every must be >= 1");
    if (o.layout != SG_LAYOUT_INT8 && o.layout != SG_LAYOUT_MSC64)
        return fail(SG_EINVAL, "unknown layout");
    if (o.sample_base < 0 || o.sample_base + S > ((int64_t)1 << 32))
        return fail(SG_EINVAL, "sample_base + n_samples must be in [0, 2^32]");
    if (o.log_bins < 0 || o.log_bins > 64) return fail(SG_EINVAL, "log_bins must be in [0, 64]");
    if (o.state_mode < 0 || o.state_mode > 3) return fail(SG_EINVAL, "state_mode must be 0, 1, 2 or 3");
    if (o.state_mode == 3 && (o.layout != SG_LAYOUT_INT8 || nt > 64))
        return fail(SG_EINVAL, "state_mode 3 (bit-parallel) needs the INT8 layout and at most 64 "
                               "temperatures");
    if (o.segments < 0) return fail(SG_EINVAL, "segments must be >= 0");
    if (o.chain_set < 0 || o.chain_set == 3 || o.chain_set > 4)
        return fail(SG_EINVAL, "chain_set must be 0, 1, 2 or 4");
    if (o.cluster < 0 || o.cluster == 3 || (o.cluster > 4 && o.cluster != 8))
        return fail(SG_EINVAL, "cluster must be 0, 1, 2, 4 or 8");
    if (o.layout == SG_LAYOUT_MSC64) {
        if (dist != SG_PM_J) return fail(SG_EINVAL, "the MSC64 layout needs +-J couplings");
        if (o.sample_base % 64) return fail(SG_EINVAL, "the MSC64 layout needs sample_base % 64 == 0");
        if (S % 64) return fail(SG_EINVAL, "the MSC64 layout needs n_samples % 64 == 0");
        if (!msc_supported_L(L))
            return fail(SG_EUNSUPPORTED, "the MSC64 layout supports even L <= 16");
    }
    return SG_OK;
}

}  // namespace

extern "C" {

void sg_options_default(sg_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->layout = SG_LAYOUT_INT8;
    o->rng_group = 1;
    o->exchange_every = 1;
    o->measure_every = 1;
    o->n_therm = 0;
}

const char *sg_status_str(sg_status s)
{
    switch (s) {
    case SG_OK: return "ok";
    case SG_EINVAL: return "invalid argument";
    case SG_ENOMEM: return "out of memory";
    case SG_ECUDA: return "CUDA error";
    case SG_ETIMEOUT: return "watchdog timeout";
    case SG_ECANCELLED: return "cancelled";
    case SG_EBUSY: return "busy";
    case SG_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sg_last_error(void) { return g_last_error.c_str(); }

size_t sg_ensemble_bytes(int L, int nt, int64_t S, sg_coupling dist, const sg_options *opt)
{
    sg_options o;
    if (opt) o = *opt; else sg_options_default(&o);
    std::vector<double> T((size_t)std::max(nt, 1));
    for (size_t k = 0; k < T.size(); ++k) T[k] = 1.0 + (double)k;
    if (validate(L, T.data(), nt, dist, S, o) != SG_OK) return 0;
    const bool msc = o.layout == SG_LAYOUT_MSC64;
    const int Tp = msc ? nt : stored_slots(L, nt, dist, o);
    // the global-memory instances (packed state) serve what shared memory
    // cannot hold; the bit-parallel ones keep the packed state too
    const bool packed = !msc && (o.state_mode >= 2 || use_bits(L, nt, dist, o) ||
                                 (o.state_mode == 0 && !int8_smem_bytes(L, Tp, dist == SG_GAUSS, 1, false)));
    return plan_arena(L, nt, Tp, S, dist == SG_GAUSS, msc, bins_of(o), o.pq_hist != 0, packed).total;
}

sg_status sg_create_ensemble(int L, double h, const double *T, int nt, sg_coupling dist,
                             int64_t S, uint64_t seed, const sg_options *opt,
                             const float *J_host, const int8_t *spins_host, void *stream,
                             sg_ensemble **out)
{
    if (!out) return fail(SG_EINVAL, "out is NULL");
    *out = nullptr;
    sg_options o;
    if (opt) o = *opt; else sg_options_default(&o);
    sg_status st = validate(L, T, nt, dist, S, o);
    if (st != SG_OK) return st;
    if (!std::isfinite(h)) return fail(SG_EINVAL, "field must be finite");
    const size_t N = (size_t)L * L * L;
    const bool gauss = dist == SG_GAUSS;
    if (J_host) {
        const size_t nJ = (size_t)S * 3 * N;
        for (size_t k = 0; k < nJ; ++k) {
            const float v = J_host[k];
            if (!gauss) {
                if (v != 1.0f && v != -1.0f) return fail(SG_EINVAL, "+-J couplings must be +1 or -1");
            } else {
                const double q = (double)v * 131072.0;
                if (!(std::fabs(v) <= 16.0f) || q != std::rint(q))
                    return fail(SG_EINVAL, "Gaussian couplings must lie on the 2^-17 grid, |J| <= 16");
            }
        }
    }
    if (spins_host && !spins_valid(spins_host, (size_t)S * 2 * nt * N))
        return fail(SG_EINVAL, "spins must be +1 or -1");

    sg_ensemble *e = new sg_ensemble();
    e->L = L;
    e->nt = nt;
    e->msc = o.layout == SG_LAYOUT_MSC64;
    e->Tp = e->msc ? nt : stored_slots(L, nt, dist, o);  // MSC: B and M are [S][2][nt]
    if (e->msc) o.rng_group = 64;         // the 64 samples of a word share Metropolis numbers
    e->layout = o.layout;
    e->gauss = gauss;
    e->S = S;
    e->h = h;
    e->h_used = gauss ? std::rint(h * 131072.0) / 131072.0 : h;
    e->seed = seed;
    e->opt = o;
    e->stream = (cudaStream_t)stream;
    e->T.assign(T, T + nt);
    auto bail = [&](sg_status s) {
        sg_destroy(e);
        return s;
    };
    cudaError_t ce = cudaGetDevice(&e->device);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaGetDevice"));
    cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    if (!e->msc && (st = configure_launch(e)) != SG_OK) return bail(st);

    e->n_bins = bins_of(o);
    const bool packed = !e->msc && (e->launch.gst || e->launch.bits);
    const ArenaPlan p = plan_arena(L, nt, e->Tp, S, gauss, e->msc, e->n_bins, o.pq_hist != 0,
                                   packed);
    e->spins_bytes = e->msc ? (size_t)(S / 64) * nt * 2 * N * 8
                            : (size_t)S * N * (packed ? e->Tp / 4 : 2 * e->Tp);
    ce = cudaMalloc(&e->arena, p.total);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMalloc(ensemble)"));
    e->bytes = p.total;
    uint8_t *base = (uint8_t *)e->arena;
    size_t off = 0;
    if (e->msc) {
        e->W = (uint64_t *)(base + off); off += p.spins;
        e->Jw = (uint64_t *)(base + off); off += p.J;
    } else {
        e->spins = base + off; off += p.spins;
        if (p.unpacked) e->unpacked = base + off;
        off += p.unpacked;
        if (gauss) e->Jg = (float *)(base + off); else e->J8 = base + off;
        off += p.J;
    }
    e->B = (int64_t *)(base + off); off += p.BM;
    e->M = (int64_t *)(base + off); off += p.BM;
    e->acc = (double *)(base + off); off += p.acc;
    e->acc_bytes = (size_t)S * nt * e->n_bins * SG_NACC * sizeof(double);
    if (p.hist) {
        e->hist = (unsigned long long *)(base + off);
        e->hist_bytes = (size_t)nt * e->n_bins * (N + 1) * sizeof(uint64_t);
    }
    off += p.hist;
    e->thr = (uint32_t *)(base + off); off += p.thr;
    e->negbeta = (float *)(base + off); off += p.tab;
    e->dbeta = (float *)(base + off); off += p.tab;
    e->twid = (float *)(base + off); off += p.twid;
    e->status = (int *)(base + off);
    e->sweep_ctr = (int64_t *)(base + off + 64);
    if (e->msc) e->masks = (uint64_t *)(base + off + 256);
    else e->work = (unsigned int *)(base + off + 256);

    ce = cudaStreamCreateWithFlags(&e->branch, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
    ce = cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaEventCreate"));

    std::vector<uint32_t> thr;
    std::vector<float> nb, db, tw;
    host_tables(e, thr, nb, db, tw);
    cudaStream_t s = e->stream;
    const uint32_t slo = (uint32_t)seed, shi = (uint32_t)(seed >> 32);
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        if ((r = cudaMemsetAsync(e->status, 0, 256, s)) != cudaSuccess) return r;
        if ((r = cudaMemsetAsync(e->acc, 0, p.acc + p.hist, s)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->thr, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->negbeta, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->dbeta, db.data(), db.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return r;
        if ((r = cudaMemcpyAsync(e->twid, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return r;
        if (J_host) {
            float *stage = nullptr;
            const size_t bytes = (size_t)S * 3 * N * sizeof(float);
            if ((r = cudaMalloc(&stage, bytes)) != cudaSuccess) return r;
            r = cudaMemcpyAsync(stage, J_host, bytes, cudaMemcpyHostToDevice, s);
            if (r == cudaSuccess)
                r = e->msc ? msc_import_J(e->Jw, stage, S / 64, L, s)
                           : int8_import_J(e->J8, e->Jg, stage, S, L, gauss, s);
            if (r == cudaSuccess) r = cudaStreamSynchronize(s);
            cudaFree(stage);
            if (r != cudaSuccess) return r;
        } else {
            if (e->msc)
                r = msc_generate(e->Jw, e->W, S / 64, L, nt, slo, shi, o.sample_base, s);
            else
                r = gauss ? int8_gen_gauss(e->Jg, S, L, slo, shi, o.sample_base, s)
                          : int8_gen_pmj(e->J8, S, L, slo, shi, o.sample_base, s);
            if (r != cudaSuccess) return r;
        }
        uint8_t *view = e->spins;  // int8: the byte-per-chain state (or its scratch copy)
        if (!e->msc && (r = unpacked_view(e, &view, false)) != cudaSuccess) return r;
        if (spins_host) {
            int8_t *stage = nullptr;
            const size_t bytes = (size_t)S * 2 * nt * N;
            if ((r = cudaMalloc(&stage, bytes)) != cudaSuccess) return r;
            r = cudaMemcpyAsync(stage, spins_host, bytes, cudaMemcpyHostToDevice, s);
            if (r == cudaSuccess)
                r = e->msc ? msc_import_spins(e->W, stage, S / 64, L, nt, s)
                           : int8_import_spins(view, stage, S, L, nt, e->Tp, s);
            if (r == cudaSuccess) r = cudaStreamSynchronize(s);
            cudaFree(stage);
            if (r != cudaSuccess) return r;
        } else if (!e->msc) {
            if ((r = int8_gen_spins(view, S, L, nt, e->Tp, slo, shi, o.sample_base, s)) != cudaSuccess)
                return r;
        }
        if (e->msc) {
            if ((r = msc_energies(make_msc_args(e), L, s)) != cudaSuccess) return r;
        } else {
            if ((r = commit_unpacked(e, view, nullptr)) != cudaSuccess) return r;
            Int8Args a = make_args(e);
            a.spins = view;
            if ((r = int8_energies(a, L, gauss, s)) != cudaSuccess) return r;
        }
        return cudaStreamSynchronize(s);
    };
    ce = run();
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "ensemble set-up"));
    *out = e;
    return SG_OK;
}

void sg_destroy(sg_ensemble *e)
{
    if (!e) return;
    purge_graphs(e);
    if (e->stream || e->arena) cudaStreamSynchronize(e->stream);
    if (e->branch) cudaStreamSynchronize(e->branch);
    if (e->copy) cudaStreamSynchronize(e->copy);
    if (e->upload) cudaFree(e->upload);
    if (e->acc_download) cudaFree(e->acc_download);
    if (e->copy) cudaStreamDestroy(e->copy);
    if (e->up_done) cudaEventDestroy(e->up_done);
    if (e->up_free) cudaEventDestroy(e->up_free);
    if (e->arena) cudaFree(e->arena);
    if (e->stage) cudaFree(e->stage);
    if (e->branch) cudaStreamDestroy(e->branch);
    if (e->ev) cudaEventDestroy(e->ev);
    delete e;
}

// Segments per sample of an int8 launch of n_sweeps sweeps. Splitting pays
// only when the samples outnumber the resident CTAs (else every sample has a
// CTA to itself) and only for the shared-memory state (the global-memory
// instances read the state through L1, which is not coherent across SMs).
// The library's choice aims at >= 8 units per CTA with segments of 16-64
// sweeps, and splits only when the last wave of samples would leave more
// than 3 % of the CTA slots idle; the cost is one more load and store of
// the sample's state per segment.
static int int8_segments(const sg_ensemble *e, int n_sweeps, int *grid)
{
    *grid = e->launch.grid;
    if (e->launch.gst || n_sweeps < 2) return 1;
    int64_t want;
    if (e->opt.segments > 0) {
        want = e->opt.segments;
    } else {
        if (n_sweeps < 32) return 1;
        if (e->S <= e->launch.grid) {
            // one wave: S CTAs over the SMs leave some SMs one CTA more than
            // others (512 samples: 68 SMs with 4, 80 with 3); k CTAs on every
            // SM that share the samples' segments keep all SMs busy to the end
            // (k >= 3: with fewer CTAs an SM issues too little to win back
            // the extra samples; B300, Gaussian L = 8, 400 samples: 3/2 CTAs
            // per SM 253, 2 per SM with segments 249 attempts/ns)
            const int64_t k = e->S / e->num_sms;
            if (k < 3 || e->S % e->num_sms == 0) return 1;
            const double even = (double)e->S / ((double)(k + 1) * e->num_sms);
            if (even > 0.97) return 1;
            *grid = (int)(k * e->num_sms);
        } else {
            // whole waves of samples (e.g. 1184 samples on 148 CTAs) leave no
            // idle tail: splitting would only add state reloads
            const int64_t waves = (e->S + e->launch.grid - 1) / e->launch.grid;
            if ((double)e->S / ((double)waves * e->launch.grid) > 0.97) return 1;
        }
        // at least 16 units per CTA slot: the last units end at different
        // times, and shorter units shorten that tail (B300, Gaussian L = 12,
        // 512 samples on 296 CTAs, 256-sweep launches, attempts/ns by
        // segments: 5 376.5, 6 382.0, 8 386.0, 11 385.6, 16 385.3; each
        // segment adds one reload of the sample's state)
        const int64_t by_balance = (16 * (int64_t)*grid + e->S - 1) / e->S;
        const int64_t by_length = (n_sweeps + 63) / 64;
        want = std::max(by_balance, by_length);
        want = std::min<int64_t>(want, std::max(1, n_sweeps / 16));
    }
    want = std::min<int64_t>(want, n_sweeps);
    // (segment, sample) units are counted in 32 bits
    while (want > 1 && want * e->S >= (int64_t)1 << 31) --want;
    return (int)std::max<int64_t>(want, 1);
}

// Longest wait of a segment for its sample's previous one. A waited-on unit
// is always held by a running CTA (units are claimed segment-major), so a
// wait lasts at most about two segments: the bound allows 64 clock cycles
// per attempt of a segment (the fused kernel takes about 2 per attempt and
// CTA on B300, more when other kernels share the SMs), at least 2^24 and at
// most 2^30 cycles (about half a second at 2 GHz), so that a lost unit
// cannot hold the GPU for long before the launch reports SG_ETIMEOUT.
static unsigned long long segment_wait_cycles(const sg_ensemble *e, int n_sweeps, int n_seg)
{
    const unsigned long long seg_len = (unsigned long long)((n_sweeps + n_seg - 1) / n_seg);
    const unsigned long long per_sweep = (unsigned long long)e->L * e->L * e->L * 2 * e->Tp;
    const unsigned long long want = 64ull * per_sweep * seg_len;
    return std::min(std::max(want, 1ull << 24), 1ull << 30);
}

// Whether global sweep n of e is measured.
static bool msc_measured(const sg_ensemble *e, int64_t n)
{
    return n >= e->opt.n_therm && (n - e->opt.n_therm) % e->opt.measure_every == 0;
}

static sg_status launch_sweeps(sg_ensemble *e, int64_t n, cudaStream_t s, bool device_counter)
{
    if (e->msc) {
        // one launch per sweep: the exchange pairing alternates between sweeps
        MscArgs a = make_msc_args(e);
        if (device_counter) a.sweep0_dev = e->sweep_ctr;
        const int threads = msc_threads(e->L, e->opt.threads_per_block);
        const bool split = msc_split(e->L, e->opt.threads_per_block);
        for (int64_t k = 0; k < n; ++k) {
            a.sweep_offset = (int)k;
            SG_CUDA(msc_sweep(a, e->L, threads, s, split), "MSC sweep kernel launch");
            // a split sweep is measured by a kernel of its own (with a device
            // sweep counter the host cannot tell, and the kernel decides)
            if (split && (device_counter || msc_measured(e, e->sweeps_done + k)))
                SG_CUDA(msc_measure_split(a, e->L, s), "MSC measurement kernel launch");
        }
        if (device_counter) SG_CUDA(advance_counter(e->sweep_ctr, n, s), "counter");
        return SG_OK;
    }
    int64_t chunk = e->opt.sweeps_per_launch > 0 ? e->opt.sweeps_per_launch : n;
    if (chunk < 1) chunk = 1;
    chunk = std::min<int64_t>(chunk, 1 << 30);
    for (int64_t done = 0; done < n; done += chunk) {
        Int8Args a = make_args(e);
        a.n_sweeps = (int)std::min<int64_t>(chunk, n - done);
        a.sweep0 = e->sweeps_done + done;
        if (device_counter) a.sweep0_dev = e->sweep_ctr;
        Int8Launch cfg = e->launch;
        a.n_seg = int8_segments(e, a.n_sweeps, &cfg.grid);
        a.seg_wait = segment_wait_cycles(e, a.n_sweeps, a.n_seg);
        if (a.n_seg > 1)
            SG_CUDA(cudaMemsetAsync(e->work, 0, (size_t)(1 + e->S) * sizeof(unsigned int), s),
                    "segment counters");
        SG_CUDA(int8_launch(e->L, e->gauss, a, cfg, s), "sweep kernel launch");
        if (device_counter) SG_CUDA(advance_counter(e->sweep_ctr, a.n_sweeps, s), "counter");
    }
    return SG_OK;
}

sg_status sg_sweep(sg_ensemble *e, int64_t n)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    if (n < 0) return fail(SG_EINVAL, "sweep count must be >= 0");
    if (n == 0) return SG_OK;
    sg_status st = launch_sweeps(e, n, e->stream, false);
    if (st != SG_OK) return st;
    e->sweeps_done += n;
    return SG_OK;
}

sg_status sg_sweep_batch(sg_ensemble *const *es, int n_ens, int64_t n, int use_graph)
{
    if (!es || n_ens < 1) return fail(SG_EINVAL, "no ensembles");
    if (n < 0) return fail(SG_EINVAL, "sweep count must be >= 0");
    for (int k = 0; k < n_ens; ++k) {
        if (!es[k]) return fail(SG_EINVAL, "ensemble is NULL");
        if (es[k]->stream != es[0]->stream) return fail(SG_EINVAL, "ensembles must share one stream");
        for (int j = 0; j < k; ++j)
            if (es[j] == es[k]) return fail(SG_EINVAL, "an ensemble appears twice");
    }
    if (n == 0) return SG_OK;
    cudaStream_t main = es[0]->stream;
    if (!use_graph) {
        SG_CUDA(cudaEventRecord(es[0]->ev, main), "event");
        for (int k = 0; k < n_ens; ++k) {
            SG_CUDA(cudaStreamWaitEvent(es[k]->branch, es[0]->ev, 0), "fork");
            sg_status st = launch_sweeps(es[k], n, es[k]->branch, false);
            if (st != SG_OK) return st;
        }
        for (int k = 0; k < n_ens; ++k) {
            SG_CUDA(cudaEventRecord(es[k]->ev, es[k]->branch), "event");
            SG_CUDA(cudaStreamWaitEvent(main, es[k]->ev, 0), "join");
            es[k]->sweeps_done += n;
        }
        return SG_OK;
    }
    // graph path: the sweep index comes from a device counter, so one
    // instantiated graph serves every call with the same ensembles and n
    // (no kernel choice depends on the sweep index: the kernels decide on
    // the device which sweeps they measure)
    std::string key = std::to_string(n);
    for (int k = 0; k < n_ens; ++k) {
        char buf[40];
        std::snprintf(buf, sizeof buf, ":%p", (void *)es[k]);
        key += buf;
    }
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_graph_mu);
        auto it = g_graphs.find(key);
        if (it != g_graphs.end()) exec = it->second.exec;
    }
    for (int k = 0; k < n_ens; ++k)
        SG_CUDA(cudaMemcpyAsync(es[k]->sweep_ctr, &es[k]->sweeps_done, sizeof(int64_t),
                                cudaMemcpyHostToDevice, main), "counter upload");
    if (!exec) {
        cudaStream_t cap = nullptr;
        SG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            ce = cudaEventRecord(es[0]->ev, cap);
            for (int k = 0; k < n_ens && ce == cudaSuccess; ++k) {
                ce = cudaStreamWaitEvent(es[k]->branch, es[0]->ev, 0);
                if (ce == cudaSuccess && launch_sweeps(es[k], n, es[k]->branch, true) != SG_OK)
                    ce = cudaErrorUnknown;
            }
            for (int k = 0; k < n_ens && ce == cudaSuccess; ++k) {
                ce = cudaEventRecord(es[k]->ev, es[k]->branch);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, es[k]->ev, 0);
            }
            cudaError_t ce2 = cudaStreamEndCapture(cap, &graph);
            if (ce == cudaSuccess) ce = ce2;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
        std::lock_guard<std::mutex> lk(g_graph_mu);
        GraphEntry ge;
        ge.ens.assign(es, es + n_ens);
        ge.exec = exec;
        g_graphs[key] = ge;
    }
    SG_CUDA(cudaGraphLaunch(exec, main), "graph launch");
    for (int k = 0; k < n_ens; ++k) es[k]->sweeps_done += n;
    return SG_OK;
}

sg_status sg_exchange(sg_ensemble *e, int parity)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    if (e->msc) {
        SG_CUDA(msc_exchange(make_msc_args(e), e->L, parity & 1, (uint32_t)e->exchanges_done,
                             e->masks, e->stream),
                "exchange");
    } else {
        Int8Args a = make_args(e);
        SG_CUDA(unpacked_view(e, &a.spins, true), "unpack");
        SG_CUDA(int8_exchange(a, e->L, e->gauss, parity & 1, (uint32_t)e->exchanges_done,
                              e->stream),
                "exchange");
        SG_CUDA(commit_unpacked(e, a.spins, nullptr), "pack");
    }
    ++e->exchanges_done;
    return SG_OK;
}

sg_status sg_measure(sg_ensemble *e, const int *k, int nk, float *out)
{
    if (!e || !k || nk < 1 || !out) return fail(SG_EINVAL, "bad measure arguments");
    int *kd = nullptr;
    float *od = nullptr;
    const size_t ob = (size_t)e->S * e->nt * nk * 2 * sizeof(float);
    SG_CUDA(cudaMalloc(&kd, sizeof(int) * 3 * nk), "cudaMalloc");
    cudaError_t ce = cudaMalloc(&od, ob);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(kd, k, sizeof(int) * 3 * nk, cudaMemcpyHostToDevice, e->stream);
    if (ce == cudaSuccess) {
        if (e->msc) {
            ce = msc_measure_k(make_msc_args(e), e->L, kd, nk, od, e->stream);
        } else {
            Int8Args a = make_args(e);
            ce = unpacked_view(e, &a.spins, true);
            if (ce == cudaSuccess) ce = int8_measure_k(a, e->L, kd, nk, od, e->stream);
        }
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, od, ob, cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    cudaFree(kd);
    cudaFree(od);
    if (ce != cudaSuccess) return cuda_fail(ce, "measure");
    return SG_OK;
}

sg_status sg_measure_noalloc(sg_ensemble *e, const int *k, int nk, float *out)
{
    if (!e || !k || nk < 1 || !out) return fail(SG_EINVAL, "bad measure arguments");
    if (e->msc) return fail(SG_EUNSUPPORTED, "sg_measure_noalloc serves the int8 layout");
    // the call copies to and from pageable host memory and waits for the
    // stream, none of which a stream capture accepts: refuse before touching
    // the stream, so that the caller's capture stays valid
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SG_CUDA(cudaStreamIsCapturing(e->stream, &cap), "capture status");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(SG_EUNSUPPORTED, "sg_measure_noalloc cannot run while the ensemble's stream "
                                     "is being captured");
    // the static array's address is per device: the ensemble's device must be
    // the current one
    int cur = -1;
    SG_CUDA(cudaGetDevice(&cur), "current device");
    if (cur != e->device)
        return fail(SG_EINVAL, "sg_measure_noalloc: the ensemble's device is not the current device");
    if (nk > SG_MEASURE_NOALLOC_MAX_K)
        return fail(SG_EINVAL, "sg_measure_noalloc: more than SG_MEASURE_NOALLOC_MAX_K wave vectors");
    const size_t floats = (size_t)e->S * e->nt * nk * 2;
    if (floats > (size_t)SG_MEASURE_NOALLOC_MAX_FLOATS)
        return fail(SG_EINVAL, "sg_measure_noalloc: n_samples * n_T * nk * 2 exceeds "
                               "SG_MEASURE_NOALLOC_MAX_FLOATS");
    // the packed state of large lattices is read through the ensemble's
    // unpacked copy (part of its arena: nothing is allocated here)
    Int8Args a = make_args(e);
    SG_CUDA(unpacked_view(e, &a.spins, true), "unpack");
    SG_CUDA(int8_measure_k_noalloc(a, e->L, k, nk, out, floats, e->stream),
            "measure (no allocation)");
    return SG_OK;
}

// The accumulators' device layouts differ from the canonical one so that the
// measurement's lanes touch consecutive doubles: int8 [S][bins][40][nt] (slot
// fastest), MSC64 [G][nt][bins][40][64] (sample bit fastest).
static cudaError_t acc_layout(sg_ensemble *e, double *dst, const double *src, bool to_dev)
{
    return e->msc ? msc_acc_layout(dst, src, e->S / 64, e->nt, e->n_bins, to_dev, e->stream)
                  : int8_acc_layout(dst, src, e->S, e->nt, e->n_bins, to_dev, e->stream);
}

sg_status sg_get_accumulators(sg_ensemble *e, double *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    double *d = nullptr;  // device layout -> canonical, via the staging buffer
    SG_CUDA(stage_buffer(e, e->acc_bytes, (void **)&d), "staging buffer");
    SG_CUDA(acc_layout(e, d, e->acc, false), "accumulator layout");
    SG_CUDA(cudaMemcpyAsync(out, d, e->acc_bytes, cudaMemcpyDeviceToHost, e->stream),
            "copy accumulators");
    SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
    return SG_OK;
}

sg_status sg_set_accumulators(sg_ensemble *e, const double *in)
{
    if (!e || !in) return fail(SG_EINVAL, "bad arguments");
    double *d = nullptr;  // canonical -> device layout, via the staging buffer
    SG_CUDA(stage_buffer(e, e->acc_bytes, (void **)&d), "staging buffer");
    SG_CUDA(cudaMemcpyAsync(d, in, e->acc_bytes, cudaMemcpyHostToDevice, e->stream),
            "copy accumulators");
    SG_CUDA(acc_layout(e, e->acc, d, true), "accumulator layout");
    SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
    return SG_OK;
}

sg_status sg_reset_accumulators(sg_ensemble *e)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    SG_CUDA(cudaMemsetAsync(e->acc, 0, e->acc_bytes, e->stream), "memset");
    if (e->hist) SG_CUDA(cudaMemsetAsync(e->hist, 0, e->hist_bytes, e->stream), "memset");
    return SG_OK;
}

sg_status sg_get_histogram(sg_ensemble *e, uint64_t *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    if (!e->hist) return fail(SG_EINVAL, "the ensemble keeps no overlap histogram (pq_hist)");
    SG_CUDA(cudaMemcpyAsync(out, e->hist, e->hist_bytes, cudaMemcpyDeviceToHost, e->stream),
            "copy histogram");
    SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
    return SG_OK;
}

sg_status sg_set_histogram(sg_ensemble *e, const uint64_t *in)
{
    if (!e || !in) return fail(SG_EINVAL, "bad arguments");
    if (!e->hist) return fail(SG_EINVAL, "the ensemble keeps no overlap histogram (pq_hist)");
    SG_CUDA(cudaMemcpyAsync(e->hist, in, e->hist_bytes, cudaMemcpyHostToDevice, e->stream),
            "copy histogram");
    SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
    return SG_OK;
}

sg_status sg_get_spins(sg_ensemble *e, int8_t *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    const size_t bytes = (size_t)e->S * 2 * e->nt * e->L * e->L * e->L;
    int8_t *d = nullptr;
    SG_CUDA(stage_buffer(e, bytes, (void **)&d), "staging buffer");
    uint8_t *view = nullptr;
    cudaError_t ce = e->msc ? cudaSuccess : unpacked_view(e, &view, true);
    if (ce == cudaSuccess)
        ce = e->msc ? msc_export_spins(d, e->W, e->S / 64, e->L, e->nt, e->stream)
                    : int8_export_spins(d, view, e->S, e->L, e->nt, e->Tp, e->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "get spins");
    return SG_OK;
}

sg_status sg_set_spins(sg_ensemble *e, const int8_t *in)
{
    if (!e || !in) return fail(SG_EINVAL, "bad arguments");
    const size_t bytes = (size_t)e->S * 2 * e->nt * e->L * e->L * e->L;
    int8_t *d = nullptr;
    SG_CUDA(stage_buffer(e, bytes, (void **)&d), "staging buffer");
    // upload to the staging buffer and check the values there (a pass at HBM
    // speed instead of one host thread); the state is replaced only if every
    // value is +1 or -1
    int *flag = (int *)((uint8_t *)e->status + 128);
    int bad = 0;
    cudaError_t ce = cudaMemsetAsync(flag, 0, sizeof(int), e->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d, in, bytes, cudaMemcpyHostToDevice, e->stream);
    if (ce == cudaSuccess) ce = check_pm1(d, bytes, flag, nullptr, e->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "set spins");
    if (bad) return fail(SG_EINVAL, "spins must be +1 or -1");
    if (e->msc) {
        ce = msc_import_spins(e->W, d, e->S / 64, e->L, e->nt, e->stream);
        if (ce == cudaSuccess) ce = msc_energies(make_msc_args(e), e->L, e->stream);
    } else {
        Int8Args a = make_args(e);
        ce = unpacked_view(e, &a.spins, false);
        if (ce == cudaSuccess) ce = int8_import_spins(a.spins, d, e->S, e->L, e->nt, e->Tp, e->stream);
        if (ce == cudaSuccess) ce = commit_unpacked(e, a.spins, nullptr);
        if (ce == cudaSuccess) ce = int8_energies(a, e->L, e->gauss, e->stream);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "set spins");
    return SG_OK;
}

sg_status sg_set_spins_async(sg_ensemble *e, const int8_t *in)
{
    if (!e || !in) return fail(SG_EINVAL, "bad arguments");
    const size_t bytes = (size_t)e->S * 2 * e->nt * e->L * e->L * e->L;
    if (!e->up_free) {  // first use: each step of the set-up is kept if a later one fails
        SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
        if (!e->upload) SG_CUDA(cudaMalloc(&e->upload, bytes), "upload buffer");
        if (!e->copy)
            SG_CUDA(cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking), "copy stream");
        if (!e->up_done)
            SG_CUDA(cudaEventCreateWithFlags(&e->up_done, cudaEventDisableTiming), "event");
        cudaEvent_t ev = nullptr;
        SG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        const cudaError_t ce = cudaEventRecord(ev, e->stream);
        if (ce != cudaSuccess) {
            cudaEventDestroy(ev);
            return cuda_fail(ce, "event");
        }
        e->up_free = ev;  // set last: its presence marks a complete set-up
    }
    int8_t *d = (int8_t *)e->upload;
    int *flag = (int *)((uint8_t *)e->status + 128);
    // the copy waits only until the previous upload's import has read the
    // buffer, so it overlaps the sweeps enqueued since
    SG_CUDA(cudaStreamWaitEvent(e->copy, e->up_free, 0), "wait");
    SG_CUDA(cudaMemcpyAsync(d, in, bytes, cudaMemcpyHostToDevice, e->copy), "upload");
    SG_CUDA(cudaEventRecord(e->up_done, e->copy), "event");
    // check and import in order with the work already on the ensemble's stream
    SG_CUDA(cudaStreamWaitEvent(e->stream, e->up_done, 0), "wait");
    cudaError_t ce = cudaMemsetAsync(flag, 0, sizeof(int), e->stream);
    if (ce == cudaSuccess) ce = check_pm1(d, bytes, flag, e->status, e->stream);
    if (ce == cudaSuccess) {
        if (e->msc) {
            ce = msc_import_spins(e->W, d, e->S / 64, e->L, e->nt, e->stream, flag);
            if (ce == cudaSuccess) ce = msc_energies(make_msc_args(e), e->L, e->stream);
        } else {
            // packed state: the copy starts as the current state, so that a
            // skipped import leaves the energies of the unchanged state
            Int8Args a = make_args(e);
            ce = unpacked_view(e, &a.spins, true);
            if (ce == cudaSuccess)
                ce = int8_import_spins(a.spins, d, e->S, e->L, e->nt, e->Tp, e->stream, flag);
            if (ce == cudaSuccess) ce = commit_unpacked(e, a.spins, flag);
            if (ce == cudaSuccess) ce = int8_energies(a, e->L, e->gauss, e->stream);
        }
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e->up_free, e->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "set spins (asynchronous)");
    return SG_OK;
}

sg_status sg_get_accumulators_async(sg_ensemble *e, double *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    if (!e->acc_download) {  // canonical copy in a buffer of its own, then the download
        SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
        SG_CUDA(cudaMalloc(&e->acc_download, e->acc_bytes), "download buffer");
    }
    SG_CUDA(acc_layout(e, (double *)e->acc_download, e->acc, false), "accumulator layout");
    SG_CUDA(cudaMemcpyAsync(out, e->acc_download, e->acc_bytes, cudaMemcpyDeviceToHost, e->stream),
            "copy accumulators");
    return SG_OK;
}

sg_status sg_get_energies(sg_ensemble *e, int64_t *Bo, int64_t *Mo)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    std::vector<int64_t> tmp((size_t)e->S * 2 * e->Tp);
    for (int which = 0; which < 2; ++which) {
        int64_t *dst = which == 0 ? Bo : Mo;
        if (!dst) continue;
        SG_CUDA(cudaMemcpyAsync(tmp.data(), which == 0 ? e->B : e->M, tmp.size() * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, e->stream), "copy energies");
        SG_CUDA(cudaStreamSynchronize(e->stream), "sync");
        for (int64_t s = 0; s < e->S; ++s)
            for (int r = 0; r < 2; ++r)
                for (int t = 0; t < e->nt; ++t)
                    dst[(s * 2 + r) * e->nt + t] = tmp[(size_t)(s * 2 + r) * e->Tp + t];
    }
    return SG_OK;
}

sg_status sg_get_couplings(sg_ensemble *e, float *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    const size_t bytes = (size_t)e->S * 3 * e->L * e->L * e->L * sizeof(float);
    float *d = nullptr;
    SG_CUDA(cudaMalloc(&d, bytes), "cudaMalloc");
    cudaError_t ce = e->msc ? msc_export_J(d, e->Jw, e->S / 64, e->L, e->stream)
                            : int8_export_J(d, e->J8, e->Jg, e->S, e->L, e->gauss, e->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    cudaFree(d);
    if (ce != cudaSuccess) return cuda_fail(ce, "get couplings");
    return SG_OK;
}

int64_t sg_sweeps_done(const sg_ensemble *e) { return e ? e->sweeps_done : -1; }

sg_status sg_set_sweeps_done(sg_ensemble *e, int64_t n)
{
    if (!e || n < 0) return fail(SG_EINVAL, "bad arguments");
    e->sweeps_done = n;
    return SG_OK;
}

sg_status sg_synchronize(sg_ensemble *e)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    SG_CUDA(cudaStreamSynchronize(e->stream), "stream synchronize");
    int status = 0;
    SG_CUDA(cudaMemcpy(&status, e->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
    if (status != 0) {
        SG_CUDA(cudaMemset(e->status, 0, sizeof(int)), "status reset");
        return fail((sg_status)status, status == SG_EINVAL
                                           ? "an asynchronous spin upload held values other than "
                                             "+-1; that upload was not applied"
                                           : "device reported an error");
    }
    return SG_OK;
}

sg_status sg_get_info(const sg_ensemble *e, sg_info *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    out->L = e->L;
    out->n_T = e->nt;
    out->layout = e->layout;
    out->dist = e->gauss ? SG_GAUSS : SG_PM_J;
    out->n_samples = e->S;
    out->h = e->h_used;
    out->attempts_per_sweep = (int64_t)e->L * e->L * e->L * 2 * e->nt * e->S;
    out->device_bytes = e->bytes;
    out->log_bins = e->n_bins;
    out->pq_hist = e->hist ? 1 : 0;
    if (e->msc) {
        // the measuring (fused) shape; thermalising launches of L >= 12 run
        // split by replica (sg_launch_plan)
        out->threads_per_block = msc_threads(e->L, e->opt.threads_per_block);
        out->grid = (e->nt / 2 + 1) * (int32_t)(e->S / 64);
        out->state_in_shared = 1;
    } else {
        out->threads_per_block = e->launch.threads;
        out->grid = e->launch.grid;
        out->state_in_shared = e->launch.gst ? 0 : 1;
    }
    out->cluster = e->msc ? 1 : std::max(e->launch.cluster, 1);
    out->chain_set = e->msc ? 0 : e->launch.csb;
    return SG_OK;
}

sg_status sg_launch_plan(const sg_ensemble *e, int64_t n_sweeps, int32_t *grid, int32_t *segments,
                         int32_t *launches)
{
    if (!e || n_sweeps < 0) return fail(SG_EINVAL, "bad arguments");
    int g = 0, seg = 1, nl = 0;
    if (e->msc) {
        const bool split = msc_split(e->L, e->opt.threads_per_block);
        g = (e->nt / 2 + 1) * (int)(e->S / 64) * (split ? 2 : 1);
        int64_t meas = 0;  // measurement launches of split sweeps
        if (split)
            for (int64_t k = 0; k < n_sweeps; ++k) meas += msc_measured(e, e->sweeps_done + k) ? 1 : 0;
        nl = (int)std::min<int64_t>(n_sweeps + meas, INT32_MAX);
    } else if (n_sweeps > 0) {
        int64_t chunk = e->opt.sweeps_per_launch > 0 ? e->opt.sweeps_per_launch : n_sweeps;
        chunk = std::min<int64_t>(std::max<int64_t>(chunk, 1), 1 << 30);
        nl = (int)std::min<int64_t>((n_sweeps + chunk - 1) / chunk, INT32_MAX);
        seg = int8_segments(e, (int)std::min<int64_t>(chunk, n_sweeps), &g);
    } else {
        g = e->launch.grid;
    }
    if (grid) *grid = g;
    if (segments) *segments = seg;
    if (launches) *launches = nl;
    return SG_OK;
}

sg_status sg_threshold_map(const float *x, int n, uint32_t *out)
{
    if (!x || !out || n < 0) return fail(SG_EINVAL, "bad arguments");
    if (n == 0) return SG_OK;
    float *xd = nullptr;
    uint32_t *od = nullptr;
    SG_CUDA(cudaMalloc(&xd, sizeof(float) * (size_t)n), "cudaMalloc");
    cudaError_t ce = cudaMalloc(&od, sizeof(uint32_t) * (size_t)n);
    if (ce == cudaSuccess) ce = cudaMemcpy(xd, x, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = threshold_map(xd, n, od, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(out, od, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(xd);
    cudaFree(od);
    if (ce != cudaSuccess) return cuda_fail(ce, "threshold map");
    return SG_OK;
}

sg_status sg_accept_map(const float *x, const uint32_t *r, int n, uint8_t *out)
{
    if (!x || !r || !out || n < 0) return fail(SG_EINVAL, "bad arguments");
    if (n == 0) return SG_OK;
    float *xd = nullptr;
    uint32_t *rd = nullptr;
    uint8_t *od = nullptr;
    SG_CUDA(cudaMalloc(&xd, sizeof(float) * (size_t)n), "cudaMalloc");
    cudaError_t ce = cudaMalloc(&rd, sizeof(uint32_t) * (size_t)n);
    if (ce == cudaSuccess) ce = cudaMalloc(&od, (size_t)n);
    if (ce == cudaSuccess) ce = cudaMemcpy(xd, x, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(rd, r, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = accept_map(xd, rd, n, od, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(out, od, (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(xd);
    cudaFree(rd);
    cudaFree(od);
    if (ce != cudaSuccess) return cuda_fail(ce, "accept map");
    return SG_OK;
}

sg_status sg_autotune(sg_ensemble *e, int64_t trial_sweeps, sg_tune_report *rep)
{
    if (!e || trial_sweeps < 1) return fail(SG_EINVAL, "bad autotune arguments");
    sg_tune_report r{};
    if (e->msc) {  // a CTA per exchange unit; time the CTA sizes
        const size_t wbytes = (size_t)(e->S / 64) * e->nt * 2 * e->L * e->L * e->L * 8;
        const size_t bm = (size_t)e->S * 2 * e->nt * sizeof(int64_t);
        const size_t ab = e->hist ? (size_t)((uint8_t *)e->hist - (uint8_t *)e->acc) + e->hist_bytes
                                  : e->acc_bytes;
        uint8_t *bk = nullptr;
        SG_CUDA(cudaMalloc(&bk, wbytes + 2 * bm + ab), "autotune backup");
        auto save = [&](bool restore) {
            const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
            void *dst[4] = {bk, bk + wbytes, bk + wbytes + bm, bk + wbytes + 2 * bm};
            void *src[4] = {e->W, e->B, e->M, e->acc};
            const size_t len[4] = {wbytes, bm, bm, ab};
            cudaError_t ce = cudaSuccess;
            for (int q = 0; q < 4 && ce == cudaSuccess; ++q)
                ce = restore ? cudaMemcpyAsync(src[q], dst[q], len[q], k, e->stream)
                             : cudaMemcpyAsync(dst[q], src[q], len[q], k, e->stream);
            return ce;
        };
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const sg_options orig = e->opt;
        const int64_t done0 = e->sweeps_done;
        double best = 1e300, def = 0.0;
        // candidates: the library choice (0: at L >= 12 split by replica, the
        // measured sweeps by the measurement kernel), then fused CTAs of 128,
        // 256 and 512 threads
        int best_t = 0, nc = 0;
        cudaError_t ce = save(false);
        const int cands[4] = {0, 128, 256, 512};
        for (int c = 0; c < 4 && ce == cudaSuccess; ++c) {
            if (c > 0 && !msc_split(e->L, 0) && cands[c] == msc_threads(e->L, 0)) continue;
            e->opt.threads_per_block = cands[c];
            if (launch_sweeps(e, 1, e->stream, false) != SG_OK) break;  // warm-up
            cudaEventRecord(e0, e->stream);
            if (launch_sweeps(e, trial_sweeps, e->stream, false) != SG_OK) break;
            cudaEventRecord(e1, e->stream);
            ce = cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / (double)trial_sweeps;
            if (c == 0) def = per;
            if (per < best) {
                best = per;
                best_t = cands[c];
            }
            ++nc;
            if (ce == cudaSuccess) ce = save(true);
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(bk);
        e->opt = orig;
        e->sweeps_done = done0;
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune");
        e->opt.threads_per_block = best_t;  // 0: the library's choice
        r.threads_per_block = best_t ? best_t : msc_threads(e->L, 0);
        r.n_candidates = nc;
        r.best_ms_per_sweep = best;
        r.default_ms_per_sweep = def;
        if (rep) *rep = r;
        return SG_OK;
    }
    if (e->launch.cluster > 1 || e->launch.bits) {  // a fixed shape: report it, time nothing
        r.threads_per_block = e->launch.threads;
        r.mchunk = e->mchunk;
        r.n_candidates = 1;
        if (rep) *rep = r;
        return SG_OK;
    }
    const size_t N = (size_t)e->L * e->L * e->L;
    const size_t sp_bytes = e->spins_bytes;  // the state as kept (packed or not)
    const size_t bm_bytes = (size_t)e->S * 2 * e->Tp * sizeof(int64_t);
    // the histogram sits right after the accumulators: one copy saves both
    const size_t acc_bytes = e->hist ? (size_t)((uint8_t *)e->hist - (uint8_t *)e->acc) + e->hist_bytes
                                     : e->acc_bytes;
    uint8_t *backup = nullptr;
    SG_CUDA(cudaMalloc(&backup, sp_bytes + 2 * bm_bytes + acc_bytes), "autotune backup");
    auto save = [&](bool restore) {
        const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
        uint8_t *b = backup;
        cudaError_t ce = restore ? cudaMemcpyAsync(e->spins, b, sp_bytes, k, e->stream)
                                 : cudaMemcpyAsync(b, e->spins, sp_bytes, k, e->stream);
        b += sp_bytes;
        if (ce == cudaSuccess)
            ce = restore ? cudaMemcpyAsync(e->B, b, bm_bytes, k, e->stream)
                         : cudaMemcpyAsync(b, e->B, bm_bytes, k, e->stream);
        b += bm_bytes;
        if (ce == cudaSuccess)
            ce = restore ? cudaMemcpyAsync(e->M, b, bm_bytes, k, e->stream)
                         : cudaMemcpyAsync(b, e->M, bm_bytes, k, e->stream);
        b += bm_bytes;
        if (ce == cudaSuccess)
            ce = restore ? cudaMemcpyAsync(e->acc, b, acc_bytes, k, e->stream)
                         : cudaMemcpyAsync(b, e->acc, acc_bytes, k, e->stream);
        return ce;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Int8Launch orig_launch = e->launch;
    const int orig_m = e->mchunk;
    const sg_options orig_opt = e->opt;
    e->opt.sweeps_per_launch = 0;
    const int WR = e->Tp / 4;
    const int Q = int8_thread_quantum(e->Tp, orig_launch.gst);
    double best_ms = 1e300, default_ms = 0.0;
    int best_t = orig_launch.threads, best_m = orig_m, ncand = 0;
    cudaError_t ce = save(false);
    std::vector<std::pair<int, int>> cands;
    cands.push_back({orig_launch.threads, orig_m});
    for (int t = ((32 + Q - 1) / Q) * Q; t <= int8_max_threads(e->L, orig_launch.gst, orig_launch.wide);
         t += Q) {
        int best_occ = 0, m_for = 0;
        for (int m = WR; m >= 1; --m) {
            const size_t smem = int8_smem_bytes(e->L, e->Tp, e->gauss, m, orig_launch.gst);
            const int o =
                smem ? int8_ctas_per_sm(e->L, e->gauss, t, smem, orig_launch.gst, orig_launch.wide) : 0;
            if (o > best_occ) {
                best_occ = o;
                m_for = m;
            }
        }
        if (best_occ > 0 && !(t == orig_launch.threads && m_for == orig_m)) cands.push_back({t, m_for});
    }
    // at most 12 shapes besides the default: spread over the range
    if (cands.size() > 13) {
        std::vector<std::pair<int, int>> pick{cands[0]};
        for (int k = 1; k <= 12; ++k) pick.push_back(cands[1 + (k - 1) * (cands.size() - 2) / 11]);
        cands = pick;
    }
    for (size_t c = 0; c < cands.size() && ce == cudaSuccess; ++c) {
        e->launch.threads = cands[c].first;
        e->mchunk = cands[c].second;
        e->launch.smem = int8_smem_bytes(e->L, e->Tp, e->gauss, e->mchunk, orig_launch.gst);
        const int occ = int8_ctas_per_sm(e->L, e->gauss, e->launch.threads, e->launch.smem,
                                         orig_launch.gst, orig_launch.wide);
        e->launch.grid = (int)std::min<int64_t>(e->S, (int64_t)occ * e->num_sms);
        if (launch_sweeps(e, 1, e->stream, false) != SG_OK) break;  // warm-up
        cudaEventRecord(e0, e->stream);
        if (launch_sweeps(e, trial_sweeps, e->stream, false) != SG_OK) break;
        cudaEventRecord(e1, e->stream);
        ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / (double)trial_sweeps;
        if (c == 0) default_ms = per;
        if (per < best_ms) {
            best_ms = per;
            best_t = cands[c].first;
            best_m = cands[c].second;
        }
        ++ncand;
        if (ce == cudaSuccess) ce = save(true);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(backup);
    e->opt = orig_opt;
    if (ce != cudaSuccess) {
        e->launch = orig_launch;
        e->mchunk = orig_m;
        return cuda_fail(ce, "autotune");
    }
    e->launch = orig_launch;
    e->launch.threads = best_t;
    e->mchunk = best_m;
    e->launch.smem = int8_smem_bytes(e->L, e->Tp, e->gauss, best_m, orig_launch.gst);
    const int occ =
        int8_ctas_per_sm(e->L, e->gauss, best_t, e->launch.smem, orig_launch.gst, orig_launch.wide);
    e->launch.grid = (int)std::min<int64_t>(e->S, (int64_t)occ * e->num_sms);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(e, orig_launch)] = {best_t, best_m};
    }
    r.threads_per_block = best_t;
    r.mchunk = best_m;
    r.n_candidates = ncand;
    r.best_ms_per_sweep = best_ms;
    r.default_ms_per_sweep = default_ms;
    if (rep) *rep = r;
    return SG_OK;
}

// Device bytes of an ensemble's evolving state (spins as kept, B, M, the
// accumulators and the histogram right after them), for the tuners' backup.
static size_t state_backup_bytes(const sg_ensemble *e, size_t part[4])
{
    const size_t N = (size_t)e->L * e->L * e->L;
    part[0] = e->msc ? (size_t)(e->S / 64) * e->nt * 2 * N * 8 : e->spins_bytes;
    part[1] = part[2] = (size_t)e->S * 2 * (e->msc ? e->nt : e->Tp) * sizeof(int64_t);
    part[3] = e->hist ? (size_t)((uint8_t *)e->hist - (uint8_t *)e->acc) + e->hist_bytes
                      : e->acc_bytes;
    return part[0] + part[1] + part[2] + part[3];
}

static cudaError_t state_backup(sg_ensemble *e, uint8_t *buf, bool restore)
{
    size_t part[4];
    state_backup_bytes(e, part);
    void *dev[4] = {e->msc ? (void *)e->W : (void *)e->spins, e->B, e->M, e->acc};
    cudaError_t ce = cudaSuccess;
    for (int q = 0; q < 4 && ce == cudaSuccess; ++q) {
        ce = restore ? cudaMemcpyAsync(dev[q], buf, part[q], cudaMemcpyDeviceToDevice, e->stream)
                     : cudaMemcpyAsync(buf, dev[q], part[q], cudaMemcpyDeviceToDevice, e->stream);
        buf += part[q];
    }
    return ce;
}

sg_status sg_autotune_schedule(sg_ensemble *e, int64_t trial_sweeps, const int32_t *exchange_every,
                               int n_candidates, double tolerance, sg_schedule_report *rep)
{
    if (!e || trial_sweeps < 1 || !exchange_every || n_candidates < 1 ||
        n_candidates > SG_SCHEDULE_MAX_CANDIDATES || !(tolerance >= 0.0))
        return fail(SG_EINVAL, "bad schedule-tuner arguments");
    for (int c = 0; c < n_candidates; ++c)
        if (exchange_every[c] < 0) return fail(SG_EINVAL, "exchange_every candidates must be >= 0");
    size_t part[4];
    const size_t bytes = state_backup_bytes(e, part);
    uint8_t *bk = nullptr;
    SG_CUDA(cudaMalloc(&bk, bytes), "schedule tuner backup");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const sg_options orig = e->opt;
    const int64_t done0 = e->sweeps_done;
    sg_schedule_report r{};
    cudaError_t ce = state_backup(e, bk, false);
    sg_status st = SG_OK;
    for (int c = 0; c < n_candidates && ce == cudaSuccess && st == SG_OK; ++c) {
        e->opt.exchange_every = exchange_every[c];
        st = launch_sweeps(e, 1, e->stream, false);  // warm-up
        if (st != SG_OK) break;
        cudaEventRecord(e0, e->stream);
        st = launch_sweeps(e, trial_sweeps, e->stream, false);
        if (st != SG_OK) break;
        cudaEventRecord(e1, e->stream);
        ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        r.ms_per_sweep[c] = ms / (double)trial_sweeps;
        if (ce == cudaSuccess) ce = state_backup(e, bk, true);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(bk);
    e->opt = orig;
    e->sweeps_done = done0;
    if (st != SG_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(ce, "schedule tuner");
    // the most frequent exchange whose sweeps cost at most (1 + tolerance)
    // times the fastest candidate's; never-exchange (0) only if nothing else
    // qualifies
    double fastest = 1e300;
    for (int c = 0; c < n_candidates; ++c) fastest = std::min(fastest, r.ms_per_sweep[c]);
    int pick = -1;
    for (int c = 0; c < n_candidates; ++c) {
        if (r.ms_per_sweep[c] > fastest * (1.0 + tolerance)) continue;
        const int32_t v = exchange_every[c];
        if (pick < 0) {
            pick = c;
            continue;
        }
        const int32_t w = exchange_every[pick];
        if ((v > 0 && (w == 0 || v < w))) pick = c;
    }
    e->opt.exchange_every = exchange_every[pick];
    purge_graphs(e);  // captured launches carry the old schedule
    r.exchange_every = exchange_every[pick];
    r.n_candidates = n_candidates;
    r.fastest_ms_per_sweep = fastest;
    if (rep) *rep = r;
    return SG_OK;
}

sg_status sg_results_bin(sg_ensemble *e, int bin, const sg_observables *out)
{
    if (!e || !out) return fail(SG_EINVAL, "bad arguments");
    if (bin < 0 || bin >= e->n_bins) return fail(SG_EINVAL, "bin out of range");
    const size_t per = (size_t)e->S * e->nt;
    std::vector<double> acc(per * e->n_bins * SG_NACC);
    sg_status st = sg_get_accumulators(e, acc.data());
    if (st != SG_OK) return st;
    if (e->n_bins > 1) {  // gather the bin into [S][n_T][40]
        for (size_t k = 0; k < per; ++k)
            std::memmove(acc.data() + k * SG_NACC,
                         acc.data() + (k * e->n_bins + bin) * SG_NACC, SG_NACC * sizeof(double));
    }
    return sg_observables_from_acc(acc.data(), e->S, e->nt, e->L, out);
}

sg_status sg_results(sg_ensemble *e, const sg_observables *out)
{
    if (!e) return fail(SG_EINVAL, "ensemble is NULL");
    return sg_results_bin(e, e->n_bins - 1, out);
}

}  // extern "C"
