// sg_msc.h -- internal interface of the multispin-coded +-J path.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sgmc.h"

namespace sg {

struct MscArgs {
    uint64_t *W;          // [G][nt][2][N] spin words, bit b = sample 64g + b
    const uint64_t *Jw;   // [G][3][N] coupling words, bit 1 => J = -1
    int64_t *B, *M;       // [S][2][nt]
    double *acc;          // [G][nt][n_bins][40][64] (sample bit fastest)
    unsigned long long *hist;  // [nt][n_bins][N+1] overlap histogram, or null
    int n_bins;           // logarithmic sweep bins (1 = a single bin)
    const uint32_t *thr;  // [nt][16] thresholds, entry sb*8 + u
    const float *dbeta;   // [nt] (float)(beta_t - beta_{t+1})
    const float *twid;    // [2][L] FP32 cos, sin of 2 pi d / L
    int64_t G;            // word groups (S / 64)
    int nt;
    float h_f;
    double h_d;
    uint32_t seed_lo, seed_hi;
    int64_t sweep0;
    const int64_t *sweep0_dev;  // if set, the base sweep index is read here
    int sweep_offset;           // this launch's sweep = base + sweep_offset
    int exchange_every, measure_every;
    int64_t n_therm;
    int64_t s_key0;             // global index of local sample 0 (multiple of 64)
    int *status;                // device status word (SG_ETIMEOUT if a bulk copy never lands)
    // round keys of the Metropolis key word k0 = seed_lo ^ tag: k0r[r] = k0 +
    // r * 0x9E3779B9, fixed per launch, read from the kernel's parameters
    uint32_t k0r[10];
};

size_t msc_smem_bytes(int L);
bool msc_supported_L(int L);
// Threads per CTA of the sweep kernel: `requested` (0 = library choice for
// L) clamped to [128, 512] and rounded down to a multiple of 128.
int msc_threads(int L, int requested);
// Whether sweeps run split by replica (L >= 12 and no requested CTA size):
// msc_split_sweep_kernel, one replica's chains of an exchange unit per CTA
// (256 threads), which does not measure, followed for a measured sweep by
// msc_measure_split; else the fused msc_sweep_kernel with `threads` threads.
bool msc_split(int L, int requested);
cudaError_t msc_sweep(const MscArgs &a, int L, int threads, cudaStream_t st, bool split);
// The overlap measurement of the sweep base + a.sweep_offset after a split
// sweep (one CTA per slot and word group; returns at once on the device when
// that sweep is not measured).
cudaError_t msc_measure_split(const MscArgs &a, int L, cudaStream_t st);
// skip (device, may be null): when *skip is nonzero the import writes nothing
cudaError_t msc_import_spins(uint64_t *W, const int8_t *canon, int64_t G, int L, int nt,
                             cudaStream_t st, const int *skip = nullptr);
cudaError_t msc_export_spins(int8_t *canon, const uint64_t *W, int64_t G, int L, int nt,
                             cudaStream_t st);
// Accumulator layouts: canonical [S][nt][nb][40] <-> device [G][nt][nb][40][64]
// (to_dev: canonical src to device dst; else device src to canonical dst).
cudaError_t msc_acc_layout(double *dst, const double *src, int64_t G, int nt, int nb, bool to_dev,
                           cudaStream_t st);
cudaError_t msc_import_J(uint64_t *Jw, const float *Jc, int64_t G, int L, cudaStream_t st);
cudaError_t msc_export_J(float *Jc, const uint64_t *Jw, int64_t G, int L, cudaStream_t st);
cudaError_t msc_generate(uint64_t *Jw, uint64_t *W, int64_t G, int L, int nt, uint32_t slo,
                         uint32_t shi, int64_t key0, cudaStream_t st);
cudaError_t msc_energies(const MscArgs &a, int L, cudaStream_t st);
cudaError_t msc_exchange(const MscArgs &a, int L, int parity, uint32_t call_id, uint64_t *masks,
                         cudaStream_t st);
cudaError_t msc_measure_k(const MscArgs &a, int L, const int *k_dev, int nk, float *out,
                          cudaStream_t st);

}  // namespace sg
