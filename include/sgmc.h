/*
 * sgmc.h -- C ABI of the B300 Monte Carlo engine for the three-dimensional
 * Edwards-Anderson spin glass in a uniform field (arXiv:1403.4560).
 *
 * What the engine computes (paper, "Methods and Measured Quantities"):
 *   H = -sum_<ij> J_ij S_i S_j - h sum_i S_i on an L^3 simple cubic lattice
 *   with periodic boundaries (eq. Hamiltonian); couplings bimodal +-1 or
 *   Gaussian N(0,1); two replicas at each of N_T temperatures joined by
 *   parallel tempering (methods section); checkerboard single-spin Metropolis
 *   sweeps; the overlap q(k) (eq. overlap) accumulated per sample and
 *   temperature, from which the Binder ratio (eq. binder), chi_SG(k)
 *   (eq. chi), the correlation length (eq. corr) and R12 (eq. r12) follow.
 *
 * Conventions shared by every call:
 *   - Host arrays use the canonical layouts below; device state is private.
 *       couplings  float  [S][3][N]      J[s][d][i] joins i and i + e_d (mod L),
 *                                        d = 0,1,2 for x,y,z; N = L^3,
 *                                        i = x + L*(y + L*z)
 *       spins      int8   [S][2][n_T][N] +1 / -1 per sample, replica, slot
 *                                        (slot t holds temperature T[t]), site
 *       energies   int64  [S][2][n_T]    B = sum_bonds (J/qJ) s s (qJ = 1 for
 *                                        +-J, 2^-17 for Gaussian couplings);
 *                                        M = sum_i s_i;  E = -(qJ*B + h*M)
 *       accumulators double [S][n_T][B][40] sweep sums of the measurements
 *                                        per logarithmic sweep bin (B =
 *                                        sg_options.log_bins, 1 by default,
 *                                        which is [S][n_T][40]); the index
 *                                        table is listed at SG_ACC_* below
 *       histogram  uint64 [n_T][B][N+1]  optional overlap histogram: entry k
 *                                        counts measurements (all samples)
 *                                        whose two replicas agree on k sites,
 *                                        i.e. q = (2k - N) / N
 *   - Every call that launches work is asynchronous on the ensemble's CUDA
 *     stream (the cudaStream_t passed at creation, 0 = legacy default
 *     stream). Calls that return host data synchronise that stream first.
 *   - No call throws or aborts. Errors come back as sg_status codes; device
 *     faults detected by the kernels are reported through a status word
 *     that sg_synchronize() reads.
 *   - One ensemble must not be used from two host threads at once.
 *   - Results depend only on (instance, seed, sweep count, options): not on
 *     the launch shape, the sweeps-per-launch chunking, or batching.
 */
#ifndef SGMC_H
#define SGMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_ensemble sg_ensemble; /* opaque, owned by the library */

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,       /* invalid argument (message via sg_last_error) */
    SG_ENOMEM = 2,       /* device or host allocation failed */
    SG_ECUDA = 3,        /* a CUDA runtime call failed */
    SG_ETIMEOUT = 4,     /* a kernel gave up after its watchdog budget */
    SG_ECANCELLED = 5,   /* work was cancelled through the cancel flag */
    SG_EBUSY = 6,        /* resource held by other work (serving slots) */
    SG_EUNSUPPORTED = 7  /* valid request this build does not support */
} sg_status;

typedef enum { SG_PM_J = 0, SG_GAUSS = 1 } sg_coupling;

/* Storage of the spins on the device. */
typedef enum {
    SG_LAYOUT_INT8 = 0,  /* one byte per spin; +-J or Gaussian couplings */
    SG_LAYOUT_MSC64 = 1  /* 64 samples per uint64 word; +-J only,
                            n_samples % 64 == 0, rng_group = 64 */
} sg_layout;

/* Accumulator indices (per sample and slot; see sg_get_accumulators). */
enum {
    SG_ACC_COUNT = 0, /* number of measurements                           */
    SG_ACC_Q1 = 1,    /* sum Q, Q = sum_i q_i, q_i = s_i^(0) s_i^(1)      */
    SG_ACC_Q2 = 2,    /* sum Q^2                                          */
    SG_ACC_Q3 = 3,    /* sum Q^3                                          */
    SG_ACC_Q4 = 4,    /* sum (Q^2)^2                                      */
    SG_ACC_E1 = 5,    /* sum E over both replicas                         */
    SG_ACC_E2 = 6,    /* sum E^2 over both replicas                       */
    SG_ACC_M1 = 7,    /* sum M over both replicas                         */
    SG_ACC_M2 = 8,    /* sum M^2 over both replicas                       */
    SG_ACC_K = 9,     /* 9 + 3v + {0,1,2}: sum Re, Im, Re^2+Im^2 of
                         sum_i q_i exp(i k_v . r_i), v = 0..8 with k_v in
                         units 2pi/L: (1,0,0) (0,1,0) (0,0,1) (1,1,0)
                         (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)     */
    SG_NACC = 40
};

typedef struct {
    int32_t layout;            /* sg_layout                                   */
    int32_t rng_group;         /* samples sharing Metropolis random numbers:
                                  1 (independent) or 64 (as the MSC64 path)  */
    int32_t exchange_every;    /* replica exchange after every k-th sweep;
                                  0 = never                                  */
    int32_t measure_every;     /* measure every k-th sweep once measuring     */
    int64_t n_therm;           /* first measured sweep (global sweep index);
                                  the paper thermalises for the first half   */
    int32_t threads_per_block; /* 0 = library choice (autotuned where known);
                                  else rounded down to a multiple of the work
                                  quantum and clamped to the kernel's bound
                                  (int8: 192 for L <= 8, 512 otherwise) */
    int32_t sweeps_per_launch; /* 0 = library choice                          */
    uint64_t watchdog_cycles;  /* 0 = no limit; else per-launch clock64 budget
                                  after which kernels stop and report
                                  SG_ETIMEOUT                                 */
    int64_t sample_base;       /* global index of this ensemble's sample 0: the
                                  key of every random number of sample s is
                                  sample_base + s, so an ensemble split into
                                  shards (one per GPU) reproduces the
                                  unsplit run exactly; 0 by default; a
                                  multiple of 64 for MSC64                   */
    int32_t log_bins;          /* accumulator bins B over the global sweep
                                  index n: 0 or 1 = one bin; B >= 2 sends the
                                  measurement of sweep n to bin
                                  min(floor(log2(n + 1)), B - 1), so bin b
                                  holds sweeps 2^b - 1 .. 2^(b+1) - 2, the
                                  second half of a run of 2^(b+1) sweeps (the
                                  logarithmic-binning equilibration test of
                                  the paper's R12-against-sweeps figure);
                                  at most 64                                 */
    int32_t pq_hist;           /* nonzero: also count the overlap histogram
                                  P(q) per slot and bin (sg_get_histogram)   */
    int32_t state_mode;        /* INT8 layout: where the sweep kernel keeps a
                                  sample's state: 0 = library choice (shared
                                  memory when it fits; for +-J couplings one
                                  bit per chain as in 3 at L >= 14, or at
                                  L >= 10 with more than 16 temperatures,
                                  where it measured faster), 1 = shared
                                  memory, a byte per chain
                                  (SG_EUNSUPPORTED if it does not fit), 2 =
                                  global memory (L >= 10), 3 = shared memory,
                                  one bit per chain (at most 64
                                  temperatures, L = 4..16 even; the paper's
                                  multispin coding of a sample's replicas,
                                  each chain still drawing its own random
                                  numbers): +-J swept bit-parallel, Gaussian
                                  couplings by chain sets (chain_set).
                                  Results do not depend on it.               */
    int32_t segments;          /* INT8 state in shared memory: each launch's
                                  sweeps are split into this many segments per
                                  sample, and the CTAs claim (segment, sample)
                                  units in order, a segment starting once the
                                  sample's previous one is stored, so samples
                                  beyond one wave of CTAs do not leave SMs idle
                                  at the end of a launch. 0 = library choice
                                  for launches of >= 32 sweeps: segments of
                                  16-64 sweeps when the samples outnumber the
                                  resident CTAs and the last wave would leave
                                  more than 3 % of the slots idle, or, when
                                  one wave would give some SMs one CTA more
                                  than others, k = floor(S / SMs) >= 3 CTAs on
                                  every SM sharing the segments (the launch
                                  then runs k * SMs CTAs: sg_launch_plan);
                                  1 = one CTA runs all of a sample's sweeps;
                                  the global-memory state is never split.
                                  Results do not depend on it.               */
    int32_t cluster;           /* INT8 state in global memory, L = 20, 24, 28,
                                  32, 40, 48 or 64: CTAs per sample, each
                                  sweeping L/k of
                                  the z-planes as one thread-block cluster.
                                  0 = library choice (k = 2, 4 or 8 when the
                                  samples are fewer than the SMs and the split
                                  keeps more SMs busy), 1 = one CTA per
                                  sample, 2 / 4 / 8 = that cluster size
                                  (SG_EUNSUPPORTED if it cannot run). Results
                                  do not depend on it.                       */
    int32_t chain_set;         /* one bit per chain (state_mode 3) with
                                  Gaussian couplings: 4-slot groups (8 chains
                                  each) in the chain set of one warp task of
                                  the sweep, 1, 2 or 4: larger sets share a
                                  task's per-site work among more chains,
                                  smaller ones balance the warps; 0 = library
                                  choice (sg_info.chain_set). Results do not
                                  depend on it.                              */
} sg_options;

/* Fill *opt with the defaults: INT8 layout, rng_group 1, exchange and
 * measure every sweep, n_therm 0, library-chosen launch shape, no watchdog,
 * one accumulator bin, no histogram. */
void sg_options_default(sg_options *opt);

/* Number of device bytes sg_create_ensemble allocates for this problem
 * (state, couplings, accumulators, histogram, tables); 0 for invalid
 * arguments. Buffers allocated later on first use come on top: the staging
 * buffer of the host-array getters and setters (the larger of the canonical
 * spins, couplings or accumulators) and the buffers of the asynchronous
 * upload and download (canonical spins, canonical accumulators). */
size_t sg_ensemble_bytes(int L, int n_T, int64_t n_samples, sg_coupling dist,
                         const sg_options *opt);

/*
 * Create an ensemble of n_samples disorder samples on the current device.
 *   L        even, 2 <= L <= 64 (even L keeps the two-colour checkerboard a
 *            proper colouring under periodic boundaries). The INT8 layout
 *            has kernels for every even L up to 32 and for 40, 48 and 64
 *            (SG_EUNSUPPORTED for the other sizes); MSC64 for L <= 16.
 *   h        uniform field (eq. Hamiltonian); rounded to the 2^-17 grid when
 *            dist == SG_GAUSS
 *   T        host array of n_T temperatures, strictly ascending, > 0 (the
 *            paper uses a geometric set, Table I caption); 1 <= n_T <= 64
 *   dist     coupling distribution (+-1 bimodal, model section; or Gaussian)
 *   seed     64-bit key of every random number the engine draws
 *   opt      options (NULL = defaults)
 *   J_host   NULL: couplings drawn on the device from seed (+-J: one Philox
 *            bit per bond; Gaussian: Box-Muller on Philox output, rounded to
 *            the 2^-17 grid, clamped to |J| <= 16). Else a host array in the
 *            canonical layout: +-1 values for SG_PM_J, values on the 2^-17
 *            grid with |J| <= 16 for SG_GAUSS (checked; SG_EINVAL otherwise).
 *   spins_host  NULL: initial spins drawn from seed; else canonical host
 *            array of +-1 (checked).
 *   stream   cudaStream_t for all work of this ensemble (NULL = default).
 *   out      receives the ensemble; *out is NULL on failure.
 * The host arrays are copied before the call returns; the caller keeps
 * ownership. Returns SG_EINVAL for bad arguments, SG_ENOMEM if device memory
 * is short, SG_ECUDA for other CUDA failures.
 */
sg_status sg_create_ensemble(int L, double h, const double *T, int n_T, sg_coupling dist,
                             int64_t n_samples, uint64_t seed, const sg_options *opt,
                             const float *J_host, const int8_t *spins_host, void *stream,
                             sg_ensemble **out);

/* Release every resource of e (synchronises its stream first). NULL is a no-op. */
void sg_destroy(sg_ensemble *e);

/*
 * Run n >= 0 Monte Carlo sweeps (paper: methods section; one sweep = one
 * Metropolis attempt on every site of every replica and slot, colour 0 then
 * colour 1), each followed by the parallel-tempering exchange when the
 * schedule calls for it and by the overlap measurement once the global sweep
 * index reaches n_therm. Asynchronous.
 */
sg_status sg_sweep(sg_ensemble *e, int64_t n);

/*
 * Run n sweeps of several ensembles together: one launch sequence covering all
 * of them, each ensemble's kernels on a branch of one CUDA graph when
 * use_graph != 0 (the graph is cached per ensemble set and n). Results are
 * identical to calling sg_sweep on each. All ensembles must share one stream.
 */
sg_status sg_sweep_batch(sg_ensemble *const *es, int n_ens, int64_t n, int use_graph);

/*
 * One standalone parallel-tempering step (paper: methods section) on the
 * current configurations: energies are recomputed, then pairs (p, p+1) with
 * p = parity, parity+2, ... are offered a swap per replica. Its random numbers
 * are keyed apart from the sweep schedule by the call's own counter.
 */
sg_status sg_exchange(sg_ensemble *e, int parity);

/*
 * Instantaneous overlap at arbitrary wave vectors (eq. overlap):
 * out[s][t][j][0..1] = Re, Im of sum_i q_i exp(i 2pi/L k_j . r_i) for the
 * current configurations, k_j = (k[3j], k[3j+1], k[3j+2]) integers, in FP32,
 * divided by N. out is a host array of n_samples*n_T*nk*2 floats.
 */
sg_status sg_measure(sg_ensemble *e, const int *k, int nk, float *out);

/*
 * sg_measure without any device allocation. The paper has no counterpart;
 * this exists for callers that cannot call cudaMalloc when they measure:
 * serving loops that keep the allocator (and the device-wide synchronisation
 * it can bring) off their latency path, and hosts whose device memory
 * belongs to another framework's pool.
 *   Same arguments and output as sg_measure, for the INT8 layout; MSC64
 *   ensembles get SG_EUNSUPPORTED. The k vectors and the output are staged
 *   in one library-owned static device array of
 *   4096 + 4 * SG_MEASURE_NOALLOC_MAX_FLOATS bytes that every GPU which loads
 *   the library holds until the process exits.
 *   Limits: nk <= SG_MEASURE_NOALLOC_MAX_K and
 *   n_samples * n_T * nk * 2 <= SG_MEASURE_NOALLOC_MAX_FLOATS; larger requests
 *   return SG_EINVAL without touching the device.
 *   The ensemble's device must be the current device (SG_EINVAL otherwise):
 *   the first call on a device looks up the array's device address, once per
 *   device, with that device current.
 *   The call copies from and to pageable host memory and synchronises the
 *   ensemble's stream before it returns, so it cannot be captured: while the
 *   stream is being captured it returns SG_EUNSUPPORTED before any stream
 *   work, and the capture stays valid.
 *   All calls share the one array and it keeps the last call's contents:
 *   calls whose work overlaps on the GPU (other host threads, other streams)
 *   race on it and must be serialised by the caller.
 */
#define SG_MEASURE_NOALLOC_MAX_K 256
#define SG_MEASURE_NOALLOC_MAX_FLOATS (1 << 20)
sg_status sg_measure_noalloc(sg_ensemble *e, const int *k, int nk, float *out);

/* Copy the accumulators (canonical layout, [S][n_T][B][40]) to a host array. */
sg_status sg_get_accumulators(sg_ensemble *e, double *acc_out);
/* Zero the accumulators and the overlap histogram. */
sg_status sg_reset_accumulators(sg_ensemble *e);
/*
 * Overlap histogram (the distribution P(q) the paper's conclusion proposes
 * to analyse), counted in the fused measurement when sg_options.pq_hist was
 * set: host array uint64 [n_T][B][N+1]; entry k of (slot t, bin b) counts the
 * measurements of every sample at temperature T[t] in sweep bin b whose
 * replicas agree on k sites (q = (2k - N)/N). Integer counts, so the result
 * does not depend on the order of the device's atomic additions. SG_EINVAL
 * if the ensemble keeps no histogram. sg_set_histogram restores one
 * (checkpoint); shards of one run add their histograms.
 */
sg_status sg_get_histogram(sg_ensemble *e, uint64_t *hist_out);
sg_status sg_set_histogram(sg_ensemble *e, const uint64_t *hist_host);
/* Copy the current spins (canonical layout, +-1) to a host array. */
sg_status sg_get_spins(sg_ensemble *e, int8_t *spins_out);
/* Replace the current spins from a host array (canonical layout, +-1). */
sg_status sg_set_spins(sg_ensemble *e, const int8_t *spins_host);
/*
 * Stream-ordered variants for pipelined host I/O (the paper has no
 * counterpart; they let a host feed new initial states and read results
 * while the GPU sweeps).
 *
 * sg_set_spins_async: the same replacement as sg_set_spins, enqueued: the
 *   host array (canonical layout) is copied on the ensemble's private copy
 *   stream into a device buffer of its own (allocated on the first call,
 *   which synchronises the stream; do not make that first call inside a
 *   stream capture), so the copy overlaps sweeps enqueued before the call;
 *   the check of the values and the import then run on the ensemble's stream,
 *   after everything enqueued before the call. The host array must stay
 *   valid and unchanged until the next sg_synchronize (page-locked memory
 *   makes the copy truly asynchronous). If a value is not +-1 the state is
 *   left as it was and the next sg_synchronize returns SG_EINVAL.
 * sg_get_accumulators_async: enqueues the copy of the accumulators
 *   ([S][n_T][B][40] doubles) to host memory on the ensemble's stream; the
 *   values are there after sg_synchronize (or any later synchronising call).
 */
sg_status sg_set_spins_async(sg_ensemble *e, const int8_t *spins_host);
sg_status sg_get_accumulators_async(sg_ensemble *e, double *acc_out);

/* Copy B and M ([S][2][n_T] each) of the configuration after the last sweep
 * or exchange; either pointer may be NULL. */
sg_status sg_get_energies(sg_ensemble *e, int64_t *B_out, int64_t *M_out);
/* Copy the couplings on the device back in the canonical layout. */
sg_status sg_get_couplings(sg_ensemble *e, float *J_out);
/* Number of sweeps done so far (the global sweep index of the next sweep). */
int64_t sg_sweeps_done(const sg_ensemble *e);
/* Set the global sweep counter (checkpoint restore together with
 * sg_set_spins and the accumulators; results then continue bit-exactly). */
sg_status sg_set_sweeps_done(sg_ensemble *e, int64_t n);
/* Replace the accumulators from a host array (checkpoint restore). */
sg_status sg_set_accumulators(sg_ensemble *e, const double *acc_host);

/*
 * Autotuner (the paper has no counterpart; it picks launch shapes for this
 * GPU). Times up to 13 candidate launch shapes of the int8 kernel (threads
 * per CTA, measurement chunk) for trial_sweeps sweeps each on the ensemble's
 * own data, restores the state afterwards (spins, energies, accumulators and
 * sweep counter are as before the call, so results do not change), keeps the
 * fastest shape for this ensemble and caches it per (L, slots, distribution,
 * memory mode) for ensembles created later in the process. Synchronises the
 * stream; allocates a device copy of the state while it runs. The
 * multispin-coded layout has one fixed shape (reported, nothing timed).
 */
typedef struct {
    int32_t threads_per_block, mchunk, n_candidates;
    double best_ms_per_sweep, default_ms_per_sweep;
} sg_tune_report;
sg_status sg_autotune(sg_ensemble *e, int64_t trial_sweeps, sg_tune_report *report);

/*
 * Schedule tuner (opt-in; the paper does not say how often to offer
 * replica exchanges, methods section). Times trial_sweeps sweeps of the
 * ensemble, on its own data, for each candidate exchange_every value
 * (sweeps per parallel-tempering exchange, 0 = never; up to
 * SG_SCHEDULE_MAX_CANDIDATES values), restores the state afterwards
 * (spins, energies, accumulators, histogram and sweep counter as before),
 * and sets the ensemble's exchange_every to the most frequent exchange whose
 * time per sweep is at most (1 + tolerance) times the fastest candidate's.
 * Results from then on equal the oracle's run with that exchange_every
 * (the exchange numbering follows the global sweep index, methods section).
 * Cached CUDA graphs of the ensemble are dropped. Synchronises the stream;
 * allocates a device copy of the state while it runs. SG_EINVAL for a
 * negative candidate, no candidates, too many or tolerance < 0.
 */
#define SG_SCHEDULE_MAX_CANDIDATES 16
typedef struct {
    int32_t exchange_every;     /* the value chosen and applied               */
    int32_t n_candidates;
    double fastest_ms_per_sweep;
    double ms_per_sweep[SG_SCHEDULE_MAX_CANDIDATES]; /* per candidate, in order */
} sg_schedule_report;
sg_status sg_autotune_schedule(sg_ensemble *e, int64_t trial_sweeps, const int32_t *exchange_every,
                               int n_candidates, double tolerance, sg_schedule_report *report);

/* Wait for the ensemble's stream and report the first device-side error. */
sg_status sg_synchronize(sg_ensemble *e);

/* Static description of an ensemble. */
typedef struct {
    int32_t L, n_T, layout, dist;
    int64_t n_samples;
    double h;          /* field actually used (rounded for Gaussian)   */
    int64_t attempts_per_sweep; /* N * 2 * n_T * n_samples           */
    size_t device_bytes;
    int32_t log_bins;  /* accumulator bins B (>= 1)                    */
    int32_t pq_hist;   /* 1 if the overlap histogram is kept           */
    int32_t threads_per_block;  /* launch shape of the sweep kernel    */
    int32_t grid;               /* CTAs of an unsplit sweep launch (a
                                   segmented launch may run more:
                                   sg_launch_plan)                     */
    int32_t state_in_shared;    /* 1: state held in shared memory for a
                                   chunk of sweeps; 0: in global memory */
    int32_t cluster;            /* CTAs sweeping one sample together (1
                                   unless sg_options.cluster applies)   */
    int32_t chain_set;          /* bit-parallel Gaussian sweep: 4-slot
                                   groups per warp task (0 otherwise)   */
} sg_info;
sg_status sg_get_info(const sg_ensemble *e, sg_info *out);

/*
 * The launch shape sg_sweep(e, n_sweeps) would use (the paper has no
 * counterpart; it documents what runs). sg_info.grid is the unsplit shape;
 * a launch may run a different number of CTAs: when the samples outnumber
 * the resident CTAs and the last wave would leave slots idle, or when one
 * wave would give some SMs one CTA more than others (then k >= 3 CTAs on
 * every SM), each sample's sweeps are split into segments that the CTAs
 * claim in order (sg_options.segments). MSC64 runs one launch per sweep;
 * at L >= 12 (library CTA size) each exchange unit runs as two CTAs, one per
 * replica (twice the grid), and every measured sweep adds one launch of the
 * overlap measurement (one CTA per slot and word group).
 *   grid      CTAs of each sweep launch (may be NULL)
 *   segments  segments per sample of the first launch, 1 = unsplit (may be NULL)
 *   launches  kernel launches of the call (may be NULL)
 * SG_EINVAL for a NULL ensemble or n_sweeps < 0. Touches no device state.
 */
sg_status sg_launch_plan(const sg_ensemble *e, int64_t n_sweeps, int32_t *grid,
                         int32_t *segments, int32_t *launches);

/*
 * Disorder-averaged observables per slot from the accumulators (paper:
 * eqs. binder, chi, corr, r12; point-group averaging of chi over the three
 * k1 directions and the six k2 directions; delete-one jackknife errors over
 * samples). Every output array has n_T entries and may be NULL.
 */
typedef struct {
    double *g, *g_err;             /* Binder ratio, global centring        */
    double *chi0, *chi0_err;       /* chi_SG(0)                            */
    double *chi1, *chi1_err;       /* chi_SG(k1), mean over 3 directions   */
    double *chi2, *chi2_err;       /* chi_SG(k2), mean over 6 directions   */
    double *xi, *xi_err;           /* xi_L (NaN when chi0/chi1 < 1)        */
    double *r12, *r12_err;         /* chi1 / chi2                          */
    double *e, *e_err;             /* energy per spin                      */
    double *q2, *q2_err;           /* [<q(0)^2>]                           */
    double *q4, *q4_err;           /* [<q(0)^4>]                           */
} sg_observables;
sg_status sg_results(sg_ensemble *e, const sg_observables *out);
/* The same for one sweep bin 0 <= bin < B (sg_results uses the last bin);
 * comparing successive bins is the logarithmic-binning equilibration test. */
sg_status sg_results_bin(sg_ensemble *e, int bin, const sg_observables *out);

/* The same estimators on a host accumulator array [S][n_T][40] (one bin). */
sg_status sg_observables_from_acc(const double *acc, int64_t n_samples, int n_T, int L,
                                  const sg_observables *out);

/*
 * Diagnostics: the device's Metropolis threshold map. out[k] = floor(e^x[k] *
 * 2^32) saturated to [0, 2^32 - 1], with x clamped to [-64, 0] and e^x from
 * the library's own FP32 exponential (Cody-Waite reduction, degree-7 Taylor
 * polynomial): the acceptance rule behind continuous couplings and replica
 * exchange (paper: methods section, Metropolis updates and parallel
 * tempering). x and out are host arrays of n entries; runs on the current
 * device and synchronises it.
 */
sg_status sg_threshold_map(const float *x, int n, uint32_t *out);

/*
 * Diagnostics: the Gaussian sweep's Metropolis decision for n pairs (x[k],
 * r[k]), x = -beta dE (FP32) and r a uniform 32-bit word. The decision is
 * r[k] <= the threshold of sg_threshold_map (paper: methods section,
 * Metropolis updates); the sweep reaches it through a screen against the
 * hardware 2^x with a 2^-12 relative guard band and takes the exact threshold
 * only for draws inside the band. out[k] bit 0: accepted; bit 1: the screen
 * was undecided and the exact threshold decided. x, r and out are host
 * arrays of n entries; runs on the current device and synchronises it.
 */
sg_status sg_accept_map(const float *x, const uint32_t *r, int n, uint8_t *out);

/* Text for a status code, and the message of the last error on this thread. */
const char *sg_status_str(sg_status s);
const char *sg_last_error(void);


/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching on one GPU.
 * The paper has no serving layer; this is the engine's way of running many
 * independent simulation requests (each a full run of the method above)
 * that arrive over time. A worker thread admits queued requests while their
 * ensembles fit the device-memory budget, keeps admitted ensembles resident
 * (lattices, couplings, accumulators, sweep counters), advances each on its
 * own stream in chunks of at most chunk_sweeps sweeps and about 2e9
 * spin-flip attempts (all resident requests share the GPU; streams of
 * smaller requests get higher priority), and releases each as soon as its
 * last chunk completes.
 * A result does not depend on what else ran beside it.
 * ------------------------------------------------------------------------ */
typedef struct sg_server sg_server;

typedef struct {
    size_t memory_budget;  /* device bytes for resident ensembles; 0 = 80% of
                              the free memory when the server starts        */
    int32_t max_active;    /* cap on resident ensembles; 0 = budget only    */
    int64_t chunk_sweeps;  /* sweeps per chunk of a request (default 256)   */
    int32_t use_graph;     /* run chunks through cached CUDA graphs         */
} sg_server_options;

typedef struct {
    int32_t L;              /* as sg_create_ensemble                        */
    double h;
    const double *T;        /* copied at submission                         */
    int32_t n_T;
    int32_t dist;           /* sg_coupling                                  */
    int64_t n_samples;
    uint64_t seed;
    int64_t n_sweeps;       /* total sweeps of the run                      */
    int64_t n_therm;        /* -1: first half thermalises (Table I caption) */
    int32_t layout;         /* -1: MSC64 for +-J with n_samples % 64 == 0
                               and L <= 16, else INT8                       */
    int32_t exchange_every; /* <= 0: every sweep                            */
    int32_t measure_every;  /* <= 0: every sweep                            */
} sg_request;

typedef struct {
    int64_t completed, queued, active, rounds; /* rounds = chunks launched */
    double attempts;        /* spin-flip attempts of all completed chunks   */
    double busy_seconds;    /* wall time with at least one request resident */
    size_t device_bytes_in_use;
    double latency_p50, latency_p99; /* submit-to-result seconds, completed */
} sg_server_stats;

void sg_server_options_default(sg_server_options *opt);
void sg_request_default(sg_request *req);
/* Start a server on the current device. `stream` is unused (each request
 * gets its own stream); it is kept for ABI stability and may be NULL. */
sg_status sg_server_create(const sg_server_options *opt, void *stream, sg_server **out);
/* Queue a request (thread-safe, returns at once); *id receives its handle. */
sg_status sg_server_submit(sg_server *sv, const sg_request *req, int64_t *id);
/* Wait until request id has finished (done, failed or cancelled); a
 * negative timeout waits forever; SG_ETIMEOUT if it has not finished.
 * *state (may be NULL): 0 queued, 1 running, 2 done, 3 failed, 4 cancelled. */
sg_status sg_server_wait(sg_server *sv, int64_t id, double timeout_s, int *state);
/* Accumulators ([n_samples][n_T][40]) and latency of a finished request;
 * SG_EBUSY while it runs, its error code if it failed, SG_ECANCELLED. */
sg_status sg_server_result(sg_server *sv, int64_t id, double *acc_out, double *latency_s);
/* Ask to drop a request; it leaves at the next round boundary. */
sg_status sg_server_cancel(sg_server *sv, int64_t id);
/* Forget a finished request and its stored result. */
sg_status sg_server_release(sg_server *sv, int64_t id);
sg_status sg_server_get_stats(sg_server *sv, sg_server_stats *out);
/* Stop the worker (running requests are cancelled) and free everything. */
void sg_server_destroy(sg_server *sv);

#ifdef __cplusplus
}
#endif
#endif /* SGMC_H */
