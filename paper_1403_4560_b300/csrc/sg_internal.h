// sg_internal.h -- declarations shared by the host API and the kernel files
// of the library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sgmc.h"

namespace sg {

// Arguments of the fused int8 sweep kernel (one CTA owns one sample at a time
// and keeps its whole state -- every replica and slot -- in shared memory).
struct Int8Args {
    uint8_t *spins;        // [S][N][2*Tp] bytes, 0 => +1, 1 => -1 (slot_byte layout);
                           // global-memory instances: packed [S][N][Tp/4]
    const uint8_t *J8;     // [S][N][8] +-J bond bits (+x,-x,+y,-y,+z,-z,0,0), 1 => J=-1
    const float *Jg;       // [S][3][N] Gaussian couplings
    int64_t *B;            // [S][2][Tp] bond sums of the current configuration
    int64_t *M;            // [S][2][Tp] magnetisations
    double *acc;           // [S][n_bins][40][nt] measurement accumulators (slot fastest)
    unsigned long long *hist;  // [nt][n_bins][N+1] overlap histogram, or null
    int n_bins;            // logarithmic sweep bins (1 = a single bin)
    const uint32_t *thr;   // [Tp][16] +-J thresholds, entry sb*8 + u
    const float *negbeta;  // [Tp] -(float)beta_t (0 for padding slots)
    const float *dbeta;    // [Tp] (float)(beta_t - beta_{t+1})
    const float *twid;     // [2][L] FP32 cos, sin of 2 pi d / L
    int *status;           // device status word (0 = OK)
    int64_t S;
    int nt, Tp;
    float h_f, qJ_f;       // FP32 field and coupling quantum (exchange rule)
    double h_d, qJ_d;      // FP64 copies (energies in the measurement)
    uint32_t seed_lo, seed_hi;
    int rng_group;
    int64_t sweep0;
    const int64_t *sweep0_dev;   // if set, the first sweep index is read here
    int n_sweeps;
    int exchange_every, measure_every;
    int64_t n_therm;
    int mchunk;            // slot words per measurement pass
    unsigned long long watchdog;
    const volatile int *cancel;  // optional host-mapped cancel flag
    int64_t s_begin, s_end;      // samples handled by this launch
    int64_t s_key0;              // global index of local sample 0 (RNG keys)
    // segmented launch (shared-memory state): n_seg segments of the launch's
    // sweeps per sample; work[0] hands out (segment, sample) units in order,
    // work[1 + s - s_begin] counts the segments of sample s already stored.
    // Zeroed before every launch with n_seg > 1.
    unsigned int *work;
    int n_seg;
    // longest wait (clock64 cycles) for a sample's previous segment when no
    // watchdog budget is set; the launch then stops with SG_ETIMEOUT
    unsigned long long seg_wait;
    // round keys of the Metropolis Philox key word k0 = seed_lo ^ MET:
    // k0r[r] = k0 + r * 0x9E3779B9, fixed per launch, read as constant
    // operands instead of the per-round key increment
    uint32_t k0r[10];
    // bit-parallel state with Gaussian couplings: 4-slot groups (bytes of a
    // site row) in the chain set of one warp task, 1, 2 or 4
    int csb;
};

struct Int8Launch {
    int threads, grid;
    size_t smem;
    bool gst;   // state kept in global memory (large L) instead of shared memory
    bool wide;  // shared-memory state, one CTA of up to 512 threads per SM (L = 10, 12)
    int cluster;  // > 1: global-memory state, each sample swept by a cluster of this many CTAs
    bool bits;    // packed state in shared memory, swept bit-parallel
    int csb;      // bit-parallel Gaussian sweep: 4-slot groups per warp task's chain set
};

// Shared-memory bytes of the fused kernel, or 0 when the state does not fit
// (or no kernel is built for that L and mode).
size_t int8_smem_bytes(int L, int Tp, bool gauss, int mchunk, bool gst);
int int8_max_threads(int L, bool gst, bool wide = false);
// Colour sites per half-sweep work item (items = (L^3 / 2) / run * quantum).
int int8_site_run(int L, bool gst);
// Launch thread counts must be multiples of this (Tp = padded slot count).
int int8_thread_quantum(int Tp, bool gst);
// The global-memory instances keep the state packed, one byte per (site,
// 4-slot group) for the group's 8 chains; every other int8 kernel works on
// the byte-per-chain layout [S][N][2*Tp]. skip: as for the imports.
cudaError_t int8_pack_spins(uint8_t *packed, const uint8_t *unpacked, int64_t S, int L, int Tp,
                            cudaStream_t st, const int *skip = nullptr);
cudaError_t int8_unpack_spins(uint8_t *unpacked, const uint8_t *packed, int64_t S, int L, int Tp,
                              cudaStream_t st);
// Configure and launch the fused kernel.
cudaError_t int8_launch(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                        cudaStream_t st);
// Occupancy of the fused kernel (CTAs per SM), 0 if it cannot launch.
int int8_ctas_per_sm(int L, bool gauss, int threads, size_t smem, bool gst, bool wide = false);
// The global-memory (large lattice) instances, in their own translation unit.
bool int8_gst_has(int L);
cudaError_t int8_launch_gst(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                            cudaStream_t st);
int int8_ctas_per_sm_gst(int L, bool gauss, int threads, size_t smem);
// The bit-parallel instances (packed state in shared memory, slots padded
// to a multiple of 32 so that a site row is whole 64-bit words; +-J and
// Gaussian couplings), in their own translation units.
bool int8_bits_has(int L);
size_t int8_smem_bytes_bits(int L, int Tp, int mchunk, bool gauss);
cudaError_t int8_launch_bits(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                             cudaStream_t st);
int int8_ctas_per_sm_bits(int L, bool gauss, int threads, size_t smem);
cudaError_t int8_launch_bits_gauss(int L, const Int8Args &a, const Int8Launch &cfg, cudaStream_t st);
int int8_ctas_per_sm_bits_gauss(int L, int threads, size_t smem);
// The cluster instances (one sample per thread-block cluster of k = 2, 4 or
// 8 CTAs, each sweeping L/k z-planes of the packed global-memory state), for
// L = 20, 24, 28, 32, 40, 48, 64; in their own translation unit. cfg.grid must be a
// multiple of cfg.cluster and L a multiple of it.
bool int8_cluster_has(int L);
cudaError_t int8_launch_cluster(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                                cudaStream_t st);
// Clusters of k CTAs that can be resident at once (0 if the shape cannot launch).
int int8_active_clusters(int L, bool gauss, int threads, size_t smem, int k);
// The wide shared-memory instances (one sample per SM with up to 512
// threads), for the lattice sizes whose narrow instance is bounded at two
// CTAs per SM; in their own translation unit.
bool int8_wide_has(int L);
cudaError_t int8_launch_wide(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                             cudaStream_t st);
int int8_ctas_per_sm_wide(int L, bool gauss, int threads, size_t smem);

// Instance preparation and state conversion kernels.
cudaError_t int8_gen_pmj(uint8_t *J8, int64_t S, int L, uint32_t seed_lo, uint32_t seed_hi,
                         int64_t key0, cudaStream_t st);
cudaError_t int8_gen_gauss(float *Jg, int64_t S, int L, uint32_t seed_lo, uint32_t seed_hi,
                           int64_t key0, cudaStream_t st);
cudaError_t int8_gen_spins(uint8_t *spins, int64_t S, int L, int nt, int Tp, uint32_t seed_lo,
                           uint32_t seed_hi, int64_t key0, cudaStream_t st);
cudaError_t int8_import_J(uint8_t *J8, float *Jg, const float *Jcanon, int64_t S, int L,
                          bool gauss, cudaStream_t st);
cudaError_t int8_export_J(float *Jcanon, const uint8_t *J8, const float *Jg, int64_t S, int L,
                          bool gauss, cudaStream_t st);
// skip (device, may be null): when *skip is nonzero the import writes nothing
cudaError_t int8_import_spins(uint8_t *spins, const int8_t *canon, int64_t S, int L, int nt,
                              int Tp, cudaStream_t st, const int *skip = nullptr);
cudaError_t int8_export_spins(int8_t *canon, const uint8_t *spins, int64_t S, int L, int nt,
                              int Tp, cudaStream_t st);
cudaError_t int8_energies(const Int8Args &a, int L, bool gauss, cudaStream_t st);
cudaError_t int8_exchange(const Int8Args &a, int L, bool gauss, int parity, uint32_t call_id,
                          cudaStream_t st);
cudaError_t threshold_map(const float *x, int n, uint32_t *out, cudaStream_t st);
cudaError_t accept_map(const float *x, const uint32_t *r, int n, uint8_t *out, cudaStream_t st);
cudaError_t advance_counter(int64_t *ctr, int64_t n, cudaStream_t st);
// Accumulator layouts: canonical [S][nt][nb][40] <-> device [S][nb][40][nt]
// (to_dev: canonical src to device dst; else device src to canonical dst).
cudaError_t int8_acc_layout(double *dst, const double *src, int64_t S, int nt, int nb, bool to_dev,
                            cudaStream_t st);
// Sets *flag (device) when a byte of c[0..n) (device, 8-byte aligned) is not
// +-1, and then also sets *status to SG_EINVAL if status is not null and
// still 0 (asynchronous uploads report through the status word).
cudaError_t check_pm1(const int8_t *c, size_t n, int *flag, int *status, cudaStream_t st);
cudaError_t int8_measure_k_noalloc(const Int8Args &a, int L, const int *k_host, int nk,
                                   float *out_host, size_t out_floats, cudaStream_t st);
cudaError_t int8_measure_k(const Int8Args &a, int L, const int *k_dev, int nk, float *out,
                           cudaStream_t st);

}  // namespace sg
