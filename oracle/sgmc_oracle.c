/*
 * sgmc_oracle.c -- plain, sequential CPU oracle for the 3D Edwards-Anderson
 * spin glass in a field with parallel tempering (arXiv:1403.4560).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code with
 * the CUDA path: it restates the model and the Monte Carlo chain from the
 * paper's methods section and the frozen RNG / acceptance / accumulator
 * conventions, one site at a time, in the order the method defines.
 *
 * Paper passages followed:
 *   Hamiltonian, eq. (Hamiltonian) and the model paragraph (L^3 periodic
 *   simple cubic lattice, bimodal couplings);
 *   overlap q(k), eq. (overlap);
 *   parallel tempering with two replicas per temperature (methods section);
 *   thermalise-then-measure split (Table I caption);
 *   the logarithmic-binning equilibration test (caption of the figure of R12
 *   against the number of sweeps) and the distribution P(q) of the overlap
 *   (conclusion).
 *
 * Parity pins (tests/): L = 2 exact enumeration of Boltzmann averages and of
 * the one-sweep transition matrix, gauge and global-flip symmetries,
 * local-field dE against Hamiltonian differences, beta = 0 closed forms, and
 * Philox against an independent third-party implementation.
 *
 * Compile with -ffp-contract=off: every fused multiply-add is an explicit
 * fmaf() call.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NACC 40

enum { TAG_MET = 0x4D455452u, TAG_EXC = 0x45584348u,
       TAG_INIT = 0x494E4954u, TAG_BOND = 0x424F4E44u };

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                     */
/* ---------------------------------------------------------------------- */
void orc_philox(const uint32_t key_in[2], const uint32_t ctr_in[4], uint32_t out[4])
{
    uint32_t k0 = key_in[0], k1 = key_in[1];
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t philox_lane(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                            uint32_t c2, uint32_t c3, int lane)
{
    uint32_t key[2] = {k0, k1}, ctr[4] = {c0, c1, c2, c3}, out[4];
    orc_philox(key, ctr, out);
    return out[lane];
}

/* ---------------------------------------------------------------------- */
/* Lattice: site i = x + L*(y + L*z), periodic.                           */
/* ---------------------------------------------------------------------- */
static int site_of(int L, int x, int y, int z)
{
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    z = ((z % L) + L) % L;
    return x + L * (y + L * z);
}

static void coords_of(int L, int i, int *x, int *y, int *z)
{
    *x = i % L;
    *y = (i / L) % L;
    *z = i / (L * L);
}

/* The neighbour of i one step along +d (step = +1) or -d (step = -1). */
static int neighbour(int L, int i, int d, int step)
{
    int x, y, z;
    coords_of(L, i, &x, &y, &z);
    if (d == 0) x += step;
    if (d == 1) y += step;
    if (d == 2) z += step;
    return site_of(L, x, y, z);
}

/* ---------------------------------------------------------------------- */
/* Temperatures and acceptance thresholds.                                */
/* ---------------------------------------------------------------------- */
static double gauss_field(double h) { return rint(h * 131072.0) / 131072.0; }

/* thr[t][sb][u]: +-J Metropolis thresholds; dE = 2 s (b + h) with
 * s b = 6 - 2u, so dE = (12 - 4u) + 2 h s. */
void orc_thresholds(double h, const double *T, int nt, uint32_t *thr)
{
    for (int t = 0; t < nt; ++t) {
        double beta = 1.0 / T[t];
        for (int sb = 0; sb < 2; ++sb)
            for (int u = 0; u <= 6; ++u) {
                double dE = (double)(12 - 4 * u) + (sb ? -2.0 * h : 2.0 * h);
                uint32_t v;
                if (dE <= 0.0) {
                    v = 0xFFFFFFFFu;
                } else {
                    double p = floor(exp(-(beta * dE)) * 4294967296.0);
                    v = p >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)p;
                }
                thr[(t * 2 + sb) * 7 + u] = v;
            }
    }
}

/* exp(x) for x in [-64, 0]: Cody-Waite reduction x = n ln2 + r with a
 * two-part ln2, then the degree-7 Taylor polynomial of e^r in Horner form. */
float orc_mc_exp32(float x)
{
    float t = x * 1.44269502f;
    float n = rintf(t);
    float r = fmaf(-n, 0.693359375f, x);
    r = fmaf(-n, -2.12194440e-4f, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int ni = (int)n;
    uint32_t bits = (uint32_t)(ni + 127) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

uint32_t orc_t32(float x)
{
    if (x < -64.0f) return 0u;
    float v = orc_mc_exp32(x) * 4294967296.0f;
    if (v >= 4294967296.0f) return 0xFFFFFFFFu;
    return (uint32_t)v;
}

/* ---------------------------------------------------------------------- */
/* Instance helpers reproducing the library's own Philox-keyed draws.     */
/* ---------------------------------------------------------------------- */
/* Initial spins of samples s_base .. s_base + S - 1 (stored from index 0). */
void orc_init_spins(uint64_t seed, int64_t s_base, int64_t S, int nt, int L, int8_t *spins)
{
    int N = L * L * L;
    uint32_t slo = (uint32_t)seed, shi = (uint32_t)(seed >> 32);
    for (int64_t sl = 0; sl < S; ++sl) {
        int64_t s = s_base + sl;
        for (int r = 0; r < 2; ++r)
            for (int t = 0; t < nt; ++t)
                for (int i = 0; i < N; ++i) {
                    uint32_t w = philox_lane(slo ^ TAG_INIT, (uint32_t)s, (uint32_t)(i >> 7),
                                             ((uint32_t)r << 16) | (uint32_t)t, 0u, shi,
                                             (i >> 5) & 3);
                    int bit = (w >> (i & 31)) & 1;
                    spins[((sl * 2 + r) * nt + t) * (int64_t)N + i] = (int8_t)(bit ? -1 : 1);
                }
    }
}

/* +-J couplings of samples s_base .. s_base + S - 1 (stored from index 0). */
void orc_pmj_couplings(uint64_t seed, int64_t s_base, int64_t S, int L, float *J)
{
    int N = L * L * L;
    uint32_t slo = (uint32_t)seed, shi = (uint32_t)(seed >> 32);
    for (int64_t sl = 0; sl < S; ++sl) {
        int64_t s = s_base + sl;
        for (int d = 0; d < 3; ++d)
            for (int i = 0; i < N; ++i) {
                uint32_t w = philox_lane(slo ^ TAG_BOND, (uint32_t)s, (uint32_t)(i >> 7),
                                         (uint32_t)d, 0u, shi, (i >> 5) & 3);
                int bit = (w >> (i & 31)) & 1;
                J[(sl * 3 + d) * (int64_t)N + i] = bit ? -1.0f : 1.0f;
            }
    }
}

/* ---------------------------------------------------------------------- */
/* Energy of one configuration, straight from the Hamiltonian:             */
/* B = sum_i sum_d (J[d][i]/qJ) s_i s_{i+d}, M = sum_i s_i.               */
/* ---------------------------------------------------------------------- */
void orc_bond_sum(int L, int gauss, const float *J, const int8_t *s, int64_t *B, int64_t *M)
{
    int N = L * L * L;
    int64_t b = 0, m = 0;
    for (int i = 0; i < N; ++i) {
        m += s[i];
        for (int d = 0; d < 3; ++d) {
            int j = neighbour(L, i, d, +1);
            double Jq = gauss ? (double)J[d * N + i] * 131072.0 : (double)J[d * N + i];
            int64_t ji = (int64_t)llrint(Jq);
            b += ji * s[i] * s[j];
        }
    }
    *B = b;
    *M = m;
}

/* Local field b_i = sum over the 6 bonds of J s_nb, in FP32 (exact for
 * +-J and for couplings on the 2^-17 grid). */
static float local_field(int L, const float *J, const int8_t *s, int i)
{
    int N = L * L * L;
    float b = 0.0f;
    for (int d = 0; d < 3; ++d) {
        int ip = neighbour(L, i, d, +1);
        int im = neighbour(L, i, d, -1);
        b += J[d * N + i] * (float)s[ip];
        b += J[d * N + im] * (float)s[im];
    }
    return b;
}

/* Number of unsatisfied bonds of site i (+-J): bonds with J s_i s_nb < 0. */
static int unsatisfied(int L, const float *J, const int8_t *s, int i)
{
    int N = L * L * L, u = 0;
    for (int d = 0; d < 3; ++d) {
        int ip = neighbour(L, i, d, +1);
        int im = neighbour(L, i, d, -1);
        if (J[d * N + i] * s[i] * s[ip] < 0) ++u;
        if (J[d * N + im] * s[i] * s[im] < 0) ++u;
    }
    return u;
}

/* Acceptance threshold for flipping site i of configuration s at slot t.
 * Exposed for the exact transition-matrix test. */
uint32_t orc_site_threshold(int L, int gauss, double h, double T_t, const uint32_t *thr_t,
                            const float *J, const int8_t *s, int i)
{
    if (!gauss) {
        int u = unsatisfied(L, J, s, i);
        int sb = s[i] < 0;
        return thr_t[sb * 7 + u];
    }
    float hq = (float)gauss_field(h);
    float b = local_field(L, J, s, i);
    float dE = 2.0f * (float)s[i] * (b + hq);
    if (dE <= 0.0f) return 0xFFFFFFFFu;
    float beta_f = (float)(1.0 / T_t);
    float x = -(beta_f * dE);
    return orc_t32(x);
}

/* Energy change of flipping site i, from the local field (FP64). */
double orc_delta_e(int L, double h, const float *J, const int8_t *s, int i)
{
    return 2.0 * (double)s[i] * ((double)local_field(L, J, s, i) + h);
}

/* ---------------------------------------------------------------------- */
/* Measurement of one replica pair (eq. overlap): Q and the 9 projections. */
/* ---------------------------------------------------------------------- */
static const int KV[9][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
    {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};

/* out: Q, then Re_v, Im_v (FP32 values widened) for v = 0..8. */
void orc_overlap(int L, const int8_t *sa, const int8_t *sb, int64_t *Q_out,
                 float *re_out, float *im_out)
{
    int N = L * L * L;
    int64_t Q = 0;
    int64_t *P = (int64_t *)calloc((size_t)9 * L, sizeof(int64_t));
    for (int i = 0; i < N; ++i) {
        int q = sa[i] * sb[i];
        int x, y, z;
        coords_of(L, i, &x, &y, &z);
        Q += q;
        for (int v = 0; v < 9; ++v) {
            int ph = KV[v][0] * x + KV[v][1] * y + KV[v][2] * z;
            int d = ((ph % L) + L) % L;
            P[v * L + d] += q;
        }
    }
    for (int v = 0; v < 9; ++v) {
        float re = 0.0f, im = 0.0f;
        for (int d = 0; d < L; ++d) {
            double ang = ((2.0 * M_PI) * (double)d) / (double)L;
            float c = (float)cos(ang), sn = (float)sin(ang);
            re = fmaf((float)P[v * L + d], c, re);
            im = fmaf((float)P[v * L + d], sn, im);
        }
        re_out[v] = re;
        im_out[v] = im;
    }
    *Q_out = Q;
    free(P);
}

/* ---------------------------------------------------------------------- */
/* The Monte Carlo chain.                                                  */
/* ---------------------------------------------------------------------- */
typedef struct {
    int L, nt, gauss, rng_group, exchange_every, measure_every;
    int slot_shared;       /* 1: the slots of a replica share each Metropolis word */
    int64_t n_therm;
    double h;
    uint64_t seed;
    const double *T;
    const uint32_t *thr;   /* [nt][2][7] */
    const float *db_f;     /* [nt]: (float)(beta_t - beta_{t+1}) */
} chain_params;

static void one_sweep_metropolis(const chain_params *cp, int64_t s, int64_t n,
                                 const float *J, int8_t *sp /* [2][nt][N] */)
{
    int L = cp->L, N = L * L * L, nt = cp->nt;
    uint32_t slo = (uint32_t)cp->seed, shi = (uint32_t)(cp->seed >> 32);
    uint32_t group = (uint32_t)(s / cp->rng_group);
    for (int c = 0; c < 2; ++c)
        for (int r = 0; r < 2; ++r)
            for (int t = 0; t < nt; ++t) {
                int8_t *cfg = sp + ((int64_t)r * nt + t) * N;
                /* the slot field of the counter; with shared slot words every
                 * temperature of the replica reads the word of slot 0, as the
                 * N_T copies packed in the bits of one word share one random
                 * number per site (methods section, multispin coding) */
                uint32_t tw = cp->slot_shared ? 0u : (uint32_t)t;
                for (int i = 0; i < N; ++i) {
                    int x, y, z;
                    coords_of(L, i, &x, &y, &z);
                    if (((x + y + z) & 1) != c) continue;
                    int j = i >> 1;
                    uint32_t rnd = philox_lane(slo ^ TAG_MET, group, (uint32_t)(j >> 2),
                                               (uint32_t)n,
                                               ((uint32_t)c << 24) | ((uint32_t)r << 16) | tw,
                                               shi, j & 3);
                    uint32_t thr = orc_site_threshold(L, cp->gauss, cp->h, cp->T[t],
                                                      cp->thr + (size_t)t * 14, J, cfg, i);
                    if (rnd <= thr) cfg[i] = (int8_t)-cfg[i];
                }
            }
}

static void exchange_step(const chain_params *cp, int64_t s, int parity, uint32_t ctr1,
                          uint32_t rflag, const float *J, int8_t *sp, int64_t *B, int64_t *M)
{
    int L = cp->L, N = L * L * L, nt = cp->nt;
    uint32_t slo = (uint32_t)cp->seed, shi = (uint32_t)(cp->seed >> 32);
    float qJ = cp->gauss ? (1.0f / 131072.0f) : 1.0f;
    float hf = cp->gauss ? (float)gauss_field(cp->h) : (float)cp->h;
    (void)J;
    for (int r = 0; r < 2; ++r)
        for (int p = parity; p + 1 < nt; p += 2) {
            int64_t *Bp = B + r * nt + p, *Mp = M + r * nt + p;
            int64_t dB = Bp[0] - Bp[1];
            int64_t dM = Mp[0] - Mp[1];
            float dE = -((float)dB * qJ + hf * (float)dM);
            float D = cp->db_f[p] * dE;
            uint32_t rnd = philox_lane(slo ^ TAG_EXC, (uint32_t)s, (uint32_t)p, ctr1,
                                       (uint32_t)r | rflag, shi, 0);
            int accept = (D >= 0.0f) || (rnd <= orc_t32(D));
            if (accept) {
                int8_t *a = sp + ((int64_t)r * nt + p) * N;
                int8_t *b = a + N;
                for (int i = 0; i < N; ++i) {
                    int8_t tmp = a[i];
                    a[i] = b[i];
                    b[i] = tmp;
                }
                int64_t tb = Bp[0]; Bp[0] = Bp[1]; Bp[1] = tb;
                int64_t tm = Mp[0]; Mp[0] = Mp[1]; Mp[1] = tm;
            }
        }
}

/* Logarithmic bin of the measurement taken at global sweep n (0-based):
 * floor(log2(n + 1)), the last bin also holding every later sweep. Bin b
 * thus covers sweeps 2^b - 1 ... 2^(b+1) - 2, the second half of a run of
 * 2^(b+1) sweeps. */
static int log_bin(int64_t n, int n_bins)
{
    int b = 0;
    while (b + 1 < n_bins && ((n + 1) >> (b + 1)) != 0) ++b;
    return b;
}

/* One measurement of every slot of one sample at sweep n. acc is the
 * sample's [nt][n_bins][40] block; hist (may be NULL) is [nt][n_bins][N+1]
 * and entry k of a (slot, bin) counts measurements whose replicas agree on
 * exactly k sites, i.e. whose overlap is q = (2k - N) / N. */
static void measure(const chain_params *cp, const int8_t *sp, const int64_t *B,
                    const int64_t *M, int n_bins, int bin, double *acc, uint64_t *hist)
{
    int L = cp->L, N = L * L * L, nt = cp->nt;
    double qJ = cp->gauss ? (1.0 / 131072.0) : 1.0;
    double h = cp->gauss ? gauss_field(cp->h) : cp->h;
    for (int t = 0; t < nt; ++t) {
        double *a = acc + ((size_t)t * n_bins + bin) * ORC_NACC;
        const int8_t *s0 = sp + ((int64_t)0 * nt + t) * N;
        const int8_t *s1 = sp + ((int64_t)1 * nt + t) * N;
        int64_t Q;
        float re[9], im[9];
        orc_overlap(L, s0, s1, &Q, re, im);
        if (hist) {
            int64_t agree = 0;
            for (int i = 0; i < N; ++i) agree += s0[i] == s1[i];
            hist[((size_t)t * n_bins + bin) * (N + 1) + agree] += 1;
        }
        double q = (double)Q;
        a[0] += 1.0;
        a[1] += q;
        a[2] += q * q;
        a[3] += q * q * q;
        a[4] += (q * q) * (q * q);
        for (int r = 0; r < 2; ++r) {
            double e = -((double)B[r * nt + t] * qJ + h * (double)M[r * nt + t]);
            a[5] += e;
            a[6] += e * e;
        }
        for (int r = 0; r < 2; ++r) {
            double m = (double)M[r * nt + t];
            a[7] += m;
            a[8] += m * m;
        }
        for (int v = 0; v < 9; ++v) {
            double dr = (double)re[v], di = (double)im[v];
            a[9 + 3 * v] += dr;
            a[10 + 3 * v] += di;
            a[11 + 3 * v] += dr * dr + di * di;
        }
    }
}

static void energies(const chain_params *cp, const float *J, const int8_t *sp,
                     int64_t *B, int64_t *M)
{
    int N = cp->L * cp->L * cp->L;
    for (int r = 0; r < 2; ++r)
        for (int t = 0; t < cp->nt; ++t)
            orc_bond_sum(cp->L, cp->gauss, J, sp + ((int64_t)r * cp->nt + t) * N,
                         B + r * cp->nt + t, M + r * cp->nt + t);
}

static void make_params(chain_params *cp, int L, int nt, int gauss, double h,
                        const double *T, uint64_t seed, int rng_group, int ee, int me,
                        int64_t n_therm, uint32_t *thr, float *db_f)
{
    cp->L = L; cp->nt = nt; cp->gauss = gauss; cp->h = h; cp->T = T; cp->seed = seed;
    cp->rng_group = rng_group; cp->exchange_every = ee; cp->measure_every = me;
    cp->slot_shared = 0;
    cp->n_therm = n_therm;
    orc_thresholds(h, T, nt, thr);
    for (int t = 0; t < nt; ++t)
        db_f[t] = t + 1 < nt ? (float)(1.0 / T[t] - 1.0 / T[t + 1]) : 0.0f;
    cp->thr = thr;
    cp->db_f = db_f;
}

/*
 * Run sweeps sweep0 .. sweep0 + n_sweeps - 1 for the local samples
 * [s_begin, s_end); local sample k is the global sample s_base + k (the index
 * that keys its random numbers).
 * J [S][3][N] float; spins [S][2][nt][N] int8 in/out; B, M [S][2][nt] out
 * (state after the last sweep); acc [S][nt][n_bins][40] in/out, a sweep's
 * measurement going to its logarithmic bin (n_bins = 1: one bin); hist
 * [nt][n_bins][N+1] in/out or NULL, summed over the samples run here (the
 * caller gives concurrent calls separate arrays). slot_shared: 0 = every
 * (replica, slot) chain draws its own Metropolis words; 1 = the slots of a
 * replica share them (the slot field of the counter is 0).
 * Returns 0, or -1 for invalid arguments.
 */
int orc_run(int L, int nt, int gauss, double h, const double *T, uint64_t seed,
            int rng_group, int exchange_every, int measure_every, int64_t n_therm,
            int64_t sweep0, int64_t n_sweeps, int64_t s_base, int64_t s_begin, int64_t s_end,
            const float *J, int8_t *spins, int64_t *B, int64_t *M, int n_bins, double *acc,
            uint64_t *hist, int slot_shared)
{
    if (L < 2 || (L & 1) || nt < 1 || nt > 4096 || rng_group < 1 || measure_every < 1 ||
        exchange_every < 0 || n_bins < 1 || n_bins > 64)
        return -1;
    int N = L * L * L;
    uint32_t *thr = (uint32_t *)malloc(sizeof(uint32_t) * 14 * (size_t)nt);
    float *db_f = (float *)malloc(sizeof(float) * (size_t)nt);
    chain_params cp;
    make_params(&cp, L, nt, gauss, h, T, seed, rng_group, exchange_every, measure_every,
                n_therm, thr, db_f);
    cp.slot_shared = slot_shared ? 1 : 0;
    for (int64_t s = s_begin; s < s_end; ++s) {
        const float *Js = J + s * 3 * (int64_t)N;
        int8_t *sp = spins + s * 2 * (int64_t)nt * N;
        int64_t *Bs = B + s * 2 * nt, *Ms = M + s * 2 * nt;
        double *as = acc + s * (int64_t)nt * n_bins * ORC_NACC;
        energies(&cp, Js, sp, Bs, Ms);
        for (int64_t n = sweep0; n < sweep0 + n_sweeps; ++n) {
            one_sweep_metropolis(&cp, s_base + s, n, Js, sp);
            energies(&cp, Js, sp, Bs, Ms);
            if (exchange_every > 0 && (n + 1) % exchange_every == 0) {
                int64_t e = (n + 1) / exchange_every - 1;
                exchange_step(&cp, s_base + s, (int)(e & 1), (uint32_t)n, 0u, Js, sp, Bs, Ms);
            }
            if (n >= n_therm && (n - n_therm) % measure_every == 0)
                measure(&cp, sp, Bs, Ms, n_bins, log_bin(n, n_bins), as, hist);
        }
    }
    free(thr);
    free(db_f);
    return 0;
}

/* Standalone exchange call number k with the given pair parity (not part of
 * the sweep schedule; its random numbers are keyed apart from it). */
int orc_exchange(int L, int nt, int gauss, double h, const double *T, uint64_t seed,
                 int64_t k, int parity, int64_t s_base, int64_t s_begin, int64_t s_end,
                 const float *J, int8_t *spins, int64_t *B, int64_t *M)
{
    if (L < 2 || (L & 1) || nt < 1) return -1;
    int N = L * L * L;
    uint32_t *thr = (uint32_t *)malloc(sizeof(uint32_t) * 14 * (size_t)nt);
    float *db_f = (float *)malloc(sizeof(float) * (size_t)nt);
    chain_params cp;
    make_params(&cp, L, nt, gauss, h, T, seed, 1, 1, 1, 0, thr, db_f);
    for (int64_t s = s_begin; s < s_end; ++s) {
        const float *Js = J + s * 3 * (int64_t)N;
        int8_t *sp = spins + s * 2 * (int64_t)nt * N;
        int64_t *Bs = B + s * 2 * nt, *Ms = M + s * 2 * nt;
        energies(&cp, Js, sp, Bs, Ms);
        exchange_step(&cp, s_base + s, parity & 1, (uint32_t)k, 0x100u, Js, sp, Bs, Ms);
    }
    free(thr);
    free(db_f);
    return 0;
}
