// sg_int8_run.cuh -- the fused int8 sweep kernel (templates), shared by the
// translation units that instantiate it for the shared-memory and the
// global-memory (large lattice) variants.
//
// int8-spin path of the EA spin-glass engine on B300 (sm_103a).
//
// One CTA owns one disorder sample at a time and keeps its whole state in
// shared memory for a chunk of sweeps: the 2 x Tp chains (two replicas, Tp
// temperature slots padded to a multiple of 4) of every site, the couplings,
// the threshold table and the energies. The CTA runs the paper's method for
// that sample (methods section: checkerboard single-spin Metropolis sweeps,
// parallel tempering between neighbouring temperatures with two replicas per
// temperature, overlap measurement after thermalisation), then writes the
// state back. HBM is touched only at chunk boundaries, so the sweep loop is
// bound by the SM's integer / FP32 issue rate rather than by HBM.
//
// Shared-memory layout of one sample:
//   spins  [N][2*Tp] bytes   per site, Tp/4 groups of 8 bytes: 4 slots of
//                            replica 0, then the same 4 slots of replica 1;
//                            value 0 => +1, 1 => -1. One 32-bit word holds
//                            four chains (SIMD within a register) and one
//                            64-bit load serves the 8 chains of a group.
//   +-J    [N][8] bytes      bond bits (+x, -x, +y, -y, +z, -z, 0, 0), 1 => J = -1
//   Gauss  [3][N] float      J[d][i] joins i and i + e_d
// Work item of a half-sweep: (run of RUN = lcm(L/2, 4) consecutive sites of
// one colour, one 4-slot group, one replica). RUN is a multiple of 4, so
// the Philox calls (four sites each) never straddle two items.
//
// Global-memory instances (large lattices, or many temperatures): the CTA
// sweeps its sample's state in place in global memory, packed to one byte
// per (site, 4-slot group) -- bit 4r + k is chain (replica r, slot 4j + k) --
// so that rows are 8x smaller and stay in L1; their work item covers both
// replicas of a group (one thread per byte), see half_sweep_packed.
#pragma once
#include <cuda_runtime.h>

#include "sg_device.cuh"
#include "sg_internal.h"

namespace sg {

// Internal linkage: each including translation unit instantiates its own
// kernels.
namespace {


constexpr int kMaxThreads = 512;
constexpr int kBitsThreads = 256;  // bit-parallel instances: up to 8 warps, 2 CTAs per SM
// colour sites per work item of the shared-memory half-sweep
constexpr int kSiteRun = 4;

// Launch bounds of an instance, chosen from B300 measurements of the
// register / resident-warp trade-off:
//   L <= 8 in shared memory: several samples fit per SM, so up to 192
//     threads and four CTAs per SM (at most 80 registers);
//   L = 10, 12 in shared memory: two samples fit per SM; 320 threads and
//     two CTAs per SM (at most 96 registers, no spills with one replica per
//     work item) give up to 20 warps instead of 13.5 (an eleventh warp per
//     CTA would leave two CTAs at most 88 registers, where L = 12 spills);
//   the same lattices with many temperatures (one sample per SM: WIDE),
//     larger lattices (one CTA per SM in shared memory), and the
//     global-memory state: up to 512 threads with 128 registers.
template <int L, bool GST, bool WIDE = false>
struct KernelBounds {
    static constexpr bool kSmall = L <= 8 && !GST;
    static constexpr bool kMid = (L == 10 || L == 12) && !GST && !WIDE;
    static constexpr int threads = kSmall ? 192 : kMid ? 320 : kMaxThreads;
    static constexpr int min_blocks = kSmall ? 4 : kMid ? 2 : 1;
};

// Whether the sweep loop gets one code path per colour (the colour, and so
// the energy bookkeeping of colour 1 only, known at compile time) or one
// path for both colours (half the instruction footprint). From B300
// measurements with the screened Metropolis test: separate paths gained
// 2-6 % for L = 10, 14, 16 and the wide and global-memory instances
// (+-J and Gaussian), but cost 3-5 % for the Gaussian instances bounded at
// 80 registers (L <= 8, where they spill) and nothing for Gaussian L = 12
// at two CTAs per SM.
template <int L, bool GAUSS, bool GST, bool WIDE>
__host__ __device__ constexpr bool unroll_colours()
{
    return !(GAUSS && !GST && !WIDE && (L <= 8 || L == 12));
}


__device__ __forceinline__ uint32_t lds32(const uint8_t *base, int off)
{
    return *reinterpret_cast<const uint32_t *>(base + off);
}
__device__ __forceinline__ void sts32(uint8_t *base, int off, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(base + off) = v;
}

// Byte of (replica r, slot t) inside a site's row: slots come in 4-slot
// words and the two replicas' words of one 4-slot group are adjacent, so one
// 64-bit load reads 8 chains (4 slots x 2 replicas) of a site.
__host__ __device__ __forceinline__ int slot_byte(int r, int t)
{
    return 8 * (t >> 2) + 4 * r + (t & 3);
}

// Packed state (global-memory instances): one byte per (site, 4-slot group)
// holds the group's 8 chains, bit 4r + k = chain (replica r, slot 4j + k), 1
// => -1 (the replicas of one sample packed into bits, as the paper's
// multispin coding does; 8x smaller rows keep a CTA's working planes in L1).
// The sweep computes on the byte-per-chain form: a nibble expands to four
// 0/1 bytes and compresses back. Neither product carries between fields.
__device__ __forceinline__ uint32_t expand4(uint32_t nib)
{
    return (nib * 0x00204081u) & 0x01010101u;  // bit k -> byte k
}
__device__ __forceinline__ uint32_t compress4(uint32_t w)
{
    return (w * 0x01020408u) >> 24;  // byte k (0 or 1) -> bit k
}
__device__ __forceinline__ uint2 load_packed(const uint8_t *p)
{
    const uint32_t b = *p;
    return make_uint2(expand4(b & 15u), expand4(b >> 4));
}
// The same through L2 only: a byte another SM stores during the launch (the
// boundary planes of a neighbouring CTA of the same cluster), which this
// SM's L1 could still hold from before.
__device__ __forceinline__ uint2 load_packed_cg(const uint8_t *p)
{
    const uint32_t b = __ldcg(p);
    return make_uint2(expand4(b & 15u), expand4(b >> 4));
}
__device__ __forceinline__ void store_packed(uint8_t *p, uint2 w)
{
    *p = (uint8_t)(compress4(w.x) | (compress4(w.y) << 4));
}

struct Smem {
    uint8_t *spins;
    uint8_t *J8;
    float *Jg;
    uint32_t *thr;
    float *negbeta, *dbeta, *twid;
    unsigned long long *B, *M;  // [2][Tp], two's complement int64
    uint32_t *xflag;            // [2][Tp] exchange stamps
    uint32_t *sel;              // [2][Tp/4][2] byte-permutation selectors
    int *anyswap;               // [2]
    unsigned long long *accm;   // [2] accepted pairs per replica (bit p: pair p, p+1)
    uint32_t *marg;             // [3][L*L][mchunk] byte counts of q = -1
    int *ctl;                   // [2] the CTA's current unit and a wait-failure flag
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Skewed shared-memory layout of the Gaussian bit-parallel state: site i's
// row of RB bytes starts at bits_row(i) = i RB + 4 floor(i / 8), and its
// couplings at index bits_jidx(i) = i + floor(i / 8) of each of the three
// planes (planes N + N/8 floats apart). The lanes of a warp task take work
// items 8 sites apart, which without the skew would all fall in two banks.
template <bool SKEW>
__host__ __device__ __forceinline__ int bits_row(int i, int RB)
{
    return SKEW ? i * RB + ((i >> 1) & ~3) : i * RB;
}
__host__ __device__ __forceinline__ int bits_jidx(int i) { return i + (i >> 3); }

// Carve the dynamic shared memory; returns the bytes used.
// gst: the sample's spins and couplings stay in global memory (large L);
// only the small tables are carved.
// bits: the packed state (one bit per chain) held in shared memory.
__host__ __device__ inline size_t carve(uint8_t *base, int L, int Tp, bool gauss, int mchunk,
                                        Smem *sm, bool gst = false, bool bits = false)
{
    const size_t N = (size_t)L * L * L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = align16(off + bytes);
        return p;
    };
    Smem s;
    // Gaussian bit-parallel state: rows and coupling planes skewed (bits_row, bits_jidx)
    const bool skew = bits && gauss;
    s.spins = gst ? nullptr : take(bits ? N * (Tp / 4) + (skew ? N / 2 : 0) : N * 2 * Tp);
    s.J8 = (gauss || gst) ? nullptr : take(N * 8);
    s.Jg = (gauss && !gst)
               ? reinterpret_cast<float *>(take((skew ? N + N / 8 : N) * 3 * sizeof(float)))
               : nullptr;
    s.thr = gauss ? nullptr : reinterpret_cast<uint32_t *>(take((size_t)Tp * 16 * 4));
    s.negbeta = reinterpret_cast<float *>(take((size_t)Tp * 4));
    s.dbeta = reinterpret_cast<float *>(take((size_t)Tp * 4));
    s.twid = reinterpret_cast<float *>(take((size_t)2 * L * 4));
    s.B = reinterpret_cast<unsigned long long *>(take((size_t)2 * Tp * 8));
    s.M = reinterpret_cast<unsigned long long *>(take((size_t)2 * Tp * 8));
    s.xflag = reinterpret_cast<uint32_t *>(take((size_t)2 * Tp * 4));
    s.sel = reinterpret_cast<uint32_t *>(take((size_t)2 * (Tp / 4) * 2 * 4));
    s.anyswap = reinterpret_cast<int *>(take(2 * 4));
    s.accm = reinterpret_cast<unsigned long long *>(take(2 * 8));
    s.marg = reinterpret_cast<uint32_t *>(take((size_t)3 * L * L * mchunk * 4));
    s.ctl = reinterpret_cast<int *>(take(2 * 4));
    if (sm) *sm = s;
    return off;
}

struct Ctx {
    int nt, Tp, WR, RB;
    int64_t s;
    uint32_t k1;      // Metropolis Philox key word of the sample (k0 is in k0r)
    uint32_t seed_lo, seed_hi;
    float hq;         // Gaussian: field on the 2^-17 grid
    // cluster instances: this CTA's slab of z-planes [z0, z1) and its work
    // items [u0, u1) of each colour
    int z0, z1, u0, u1;
    const uint32_t *k0r;  // round keys of k0, in the kernel's parameters
};

// Site index and neighbour offsets (in sites) of the colour-COL site with
// colour-compressed index jj (i = 2*jj + parity, i >> 1 == jj).
template <int L>
struct SiteNb {
    int i, x, z, dxp, dxm, dyp, dym, dzp, dzm;
    __device__ __forceinline__ SiteNb(int jj, int COL)
    {
        constexpr int H = L / 2;
        const int row = jj / H;
        const int x2 = jj - row * H;
        const int y = row % L;
        z = row / L;
        x = 2 * x2 + ((COL + y + z) & 1);
        i = x + L * row;
        dxp = (x == L - 1) ? -(L - 1) : 1;
        dxm = (x == 0) ? (L - 1) : -1;
        dyp = (y == L - 1) ? -(L - 1) * L : L;
        dym = (y == 0) ? (L - 1) * L : -L;
        dzp = (z == L - 1) ? -(L - 1) * L * L : L * L;
        dzm = (z == 0) ? (L - 1) * L * L : -L * L;
    }
};

// +-J: Metropolis on 4 chains of one replica word; returns the flip bytes
// (0x01 per flipped chain) and the unsatisfied-bond counts per byte.
__device__ __forceinline__ uint32_t pmj_word(uint32_t s, uint32_t nxp, uint32_t nxm,
                                             uint32_t nyp, uint32_t nym, uint32_t nzp,
                                             uint32_t nzm, const uint32_t (&m)[6],
                                             const uint32_t *thr_w, const uint32_t (&rnd)[4][4],
                                             int lane, uint32_t valid, uint32_t &uw)
{
    uw = (s ^ nxp ^ m[0]) + (s ^ nxm ^ m[1]) + (s ^ nyp ^ m[2]) + (s ^ nym ^ m[3]) +
         (s ^ nzp ^ m[4]) + (s ^ nzm ^ m[5]);
    const uint32_t idx = (s << 3) | uw;  // per byte: sb*8 + u
    uint32_t fm = 0;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t th = thr_w[kk * 16 + ((idx >> (8 * kk)) & 15u)];
        fm |= (uint32_t)(rnd[kk][lane] <= th) << (8 * kk);
    }
    return fm & valid;
}

// Integer products through inline PTX, so that shifts by a runtime amount
// (a multiply by a power of two held in a register) and bit-field adds
// issue on the FMA pipe instead of the ALU pipe, which the sign flips of the
// local field already load.
__device__ __forceinline__ uint32_t mul_lo(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Gaussian: Metropolis on 4 chains of one replica word; nbeta2[kk] = -2 beta
// of the chain's slot. With energy (colour-1 sites), bq[kk] receives
// s_new * b / qJ. The four decisions come from screen_pair for the chain
// pairs (0, 1) and (2, 3), the local-field sums, b + h and -2 beta (s (b + h))
// packed the same way (the roundings of the scalar form); if any draw of the word
// falls in the screen's band, all four are redone with the exact threshold
// (dE <= 0 gives x >= 0, whose threshold is 0xFFFFFFFF).
__device__ __forceinline__ uint32_t gauss_word(uint32_t s, uint32_t nxp, uint32_t nxm,
                                               uint32_t nyp, uint32_t nym, uint32_t nzp,
                                               uint32_t nzm, const float (&j)[6], float hq,
                                               const float (&nbeta2)[4],
                                               const uint32_t (&rnd)[4][4], int lane,
                                               uint32_t valid, bool energy, int (&bq)[4])
{
    const uint32_t nb[6] = {nxp, nxm, nyp, nym, nzp, nzm};
    const unsigned long long hq2 = f2_pack(hq, hq);
    // the sign bit of chain kk's value flipped where bit 8 kk of w is set;
    // for kk = 0, J + w * 2^31 flips exactly bit 31 (one multiply-add)
    auto flip = [](float v, uint32_t w, int kk) {
        return kk == 0 ? __uint_as_float(mad_lo(w, 0x80000000u, __float_as_uint(v)))
                       : __uint_as_float(__float_as_uint(v) ^ ((w << (31 - 8 * kk)) & 0x80000000u));
    };
    bool amb = false;
    float b[4], x[4], u[4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int k0 = 2 * q, k1 = 2 * q + 1;
        unsigned long long t[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) t[d] = f2_pack(flip(j[d], nb[d], k0), flip(j[d], nb[d], k1));
        const unsigned long long bp = f2_add(f2_add(f2_add(t[0], t[1]), f2_add(t[2], t[3])),
                                             f2_add(t[4], t[5]));
        f2_unpack(bp, b[k0], b[k1]);
        float z0, z1;
        f2_unpack(f2_add(bp, hq2), z0, z1);
        const unsigned long long zs = f2_pack(flip(z0, s, k0), flip(z1, s, k1));
        const unsigned long long xp = f2_mul(f2_pack(nbeta2[k0], nbeta2[k1]), zs);
        f2_unpack(xp, x[k0], x[k1]);
        bool b0, b1;
        screen_pair(xp, rnd[k0][lane], rnd[k1][lane], b0, b1, u[k0], u[k1]);
        amb |= b0 | b1;
    }
    // the decisions are the sign bits: the top bytes of the four u gathered
    // into one word, bit 7 of each byte moved to bit 0
    const uint32_t top = __byte_perm(__byte_perm(__float_as_uint(u[0]), __float_as_uint(u[1]), 0x0073),
                                     __byte_perm(__float_as_uint(u[2]), __float_as_uint(u[3]), 0x0073),
                                     0x5410);
    uint32_t fm = (top >> 7) & 0x01010101u;
    if (amb) {
        fm = 0;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            fm |= (rnd[kk][lane] <= thr_of_logp(x[kk]) ? 1u : 0u) << (8 * kk);
    }
    if (energy) {
        const uint32_t sn = s ^ fm;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float e0, e1;
            f2_unpack(f2_mul(f2_pack(b[2 * q], b[2 * q + 1]), f2_pack(131072.0f, 131072.0f)), e0, e1);
            const int q0 = __float2int_rn(e0), q1 = __float2int_rn(e1);
            bq[2 * q] = ((sn >> (16 * q)) & 1u) ? -q0 : q0;
            bq[2 * q + 1] = ((sn >> (16 * q + 8)) & 1u) ? -q1 : q1;
        }
    }
    return fm & valid;
}

// ---------------------------------------------------------------------------
// One checkerboard half-sweep of colour COL over all chains of the sample.
// Work item: (4 consecutive colour-COL sites, i.e. one Philox counter group;
// 4-slot group j; replica r): 16 attempts. A thread keeps (j, r) for every
// item it takes, so its slots' tables are loaded once. One replica per item
// halves the live random numbers and spin words against an item over both
// replicas, which keeps the kernel's registers low enough for more resident
// warps. Short items balance the threads' shares (L = 14, 24 temperatures,
// 504 threads: 4116 items in 8.2 rounds, against 588 items in 1.2 rounds
// with items a row long), so fewer warps idle at the barrier that ends the
// half-sweep, and the partial energy sums of many items share one flush to
// shared memory (B300: L = 8 +14 %, L = 14 +14 %, L = 12 +2 %). For COL == 1 it
// also accumulates B and M of the post-sweep configuration: every bond has
// exactly one colour-1 end, so summing s_i * b_i over colour-1 sites counts
// each bond once; M pairs each colour-1 site with its x^1 partner (colour 0,
// final after the colour-0 half). The byte-wise partial sums run over the
// thread's successive items and go to shared memory every kFlushSites sites.
// ---------------------------------------------------------------------------
template <int L, bool GAUSS>
__device__ __forceinline__ void half_sweep(const Smem &sm, const Ctx &cx, uint32_t n_sweep,
                                        const int COL)
{
    constexpr int N = L * L * L;
    constexpr int RUN = kSiteRun;
    constexpr int U = (N / 2) / RUN;
    // byte-wise sums: at most 6 unsatisfied bonds and 2 for M per site
    constexpr int kFlushSites = 40;
    const int WR = cx.WR, RB = cx.RB;
    const int jr = threadIdx.x % (2 * WR);  // fixed per thread: blockDim.x is a multiple of 2 WR
    const int j = jr >> 1, r = jr & 1;
    const int t0 = 4 * j;

    uint32_t valid = 0;  // bytes of real (not padding) slots in this group
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
        if (t0 + kk < cx.nt) valid |= 1u << (8 * kk);

    float nbeta2[4];  // -2 beta per slot (exact)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) nbeta2[kk] = GAUSS ? __fmul_rn(2.0f, sm.negbeta[t0 + kk]) : 0.0f;
    const uint32_t *thr_w = GAUSS ? nullptr : sm.thr + t0 * 16;
    const int woff = 8 * j + 4 * r;  // byte offset of this (group, replica) word in a site row

    uint32_t eacc = 0, macc = 0;  // byte-wise partial sums
    int bg[4] = {0, 0, 0, 0};
    int nsites = 0;               // colour-1 sites in the partial sums
    // partial sums to shared memory, per slot of this thread's group
    auto flush = [&]() {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int t = t0 + kk;
            if (t < cx.nt) {
                // +-J: s b = 6 - 2u per colour-1 site; M: each pair gives 2 - 2*(#-1)
                const long long usum = (long long)((eacc >> (8 * kk)) & 0xFFu);
                const long long b = GAUSS ? (long long)bg[kk] : 6LL * nsites - 2LL * usum;
                const long long mm = 2LL * nsites - 2LL * ((macc >> (8 * kk)) & 0xFFu);
                atomicAdd(&sm.B[r * cx.Tp + t], (unsigned long long)b);
                atomicAdd(&sm.M[r * cx.Tp + t], (unsigned long long)mm);
            }
            bg[kk] = 0;
        }
        eacc = 0;
        macc = 0;
        nsites = 0;
    };

    // item = u * 2 WR + jr: blockDim.x is a multiple of 2 WR, so a thread's
    // successive items advance u by a fixed step (no division per item)
    const int du = blockDim.x / (2 * WR);
    for (int u = threadIdx.x / (2 * WR); u < U; u += du) {
        if (COL == 1 && nsites + RUN > kFlushSites) flush();
        {
            const uint32_t c0 = (uint32_t)u;
            uint32_t rnd[4][4];
            {
                uint32_t c2[4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    c2[kk] = ((uint32_t)COL << 24) | ((uint32_t)r << 16) | (uint32_t)(t0 + kk);
                u32x4 o[4];
                philox10x4_rk(cx.k0r, cx.k1, c0, n_sweep, c2, cx.seed_hi, o);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                    for (int q = 0; q < 4; ++q) rnd[kk][q] = o[kk].v[q];
            }
#pragma unroll
            for (int lane = 0; lane < 4; ++lane) {
                const SiteNb<L> st(u * RUN + lane, COL);
                const int own = st.i * RB + woff;
                const uint32_t s = lds32(sm.spins, own);
                const uint32_t nxp = lds32(sm.spins, own + st.dxp * RB);
                const uint32_t nxm = lds32(sm.spins, own + st.dxm * RB);
                const uint32_t nyp = lds32(sm.spins, own + st.dyp * RB);
                const uint32_t nym = lds32(sm.spins, own + st.dym * RB);
                const uint32_t nzp = lds32(sm.spins, own + st.dzp * RB);
                const uint32_t nzm = lds32(sm.spins, own + st.dzm * RB);
                uint32_t fm;
                if constexpr (!GAUSS) {
                    const uint2 jb = *reinterpret_cast<const uint2 *>(sm.J8 + 8 * st.i);
                    const uint32_t m[6] = {__byte_perm(jb.x, jb.y, 0x0000),
                                           __byte_perm(jb.x, jb.y, 0x1111),
                                           __byte_perm(jb.x, jb.y, 0x2222),
                                           __byte_perm(jb.x, jb.y, 0x3333),
                                           __byte_perm(jb.x, jb.y, 0x4444),
                                           __byte_perm(jb.x, jb.y, 0x5555)};
                    uint32_t uw;
                    fm = pmj_word(s, nxp, nxm, nyp, nym, nzp, nzm, m, thr_w, rnd, lane, valid, uw);
                    if (COL == 1) {
                        const uint32_t f = fm * 0xFFu;
                        eacc += uw ^ ((uw ^ (0x06060606u - uw)) & f);
                    }
                } else {
                    const float jv[6] = {sm.Jg[st.i], sm.Jg[st.i + st.dxm], sm.Jg[N + st.i],
                                         sm.Jg[N + st.i + st.dym], sm.Jg[2 * N + st.i],
                                         sm.Jg[2 * N + st.i + st.dzm]};
                    int bq[4];
                    fm = gauss_word(s, nxp, nxm, nyp, nym, nzp, nzm, jv, cx.hq, nbeta2, rnd,
                                    lane, valid, COL == 1, bq);
                    if (COL == 1) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) bg[kk] += bq[kk];
                    }
                }
                const uint32_t sn = s ^ fm;
                sts32(sm.spins, own, sn);
                if (COL == 1) {
                    const uint32_t partner = (st.x & 1) ? nxm : nxp;
                    macc += sn + partner;
                }
            }
        }
        nsites += RUN;
    }
    if (COL == 1 && nsites > 0) flush();
}

// ---------------------------------------------------------------------------
// Half-sweep of colour COL on the packed state (global-memory instances).
// Work item: (4 colour-COL sites = one Philox group, 4-slot group j, both
// replicas), i.e. the 8 chains of one byte, which this thread alone writes.
// The rule, random numbers, item order and energy bookkeeping are those of
// half_sweep; only the storage differs (one byte per site and group,
// expanded to 0/1 bytes).
// ---------------------------------------------------------------------------
// SLAB (cluster instances): only the items [cx.u0, cx.u1) of this CTA's
// z-slab, and the z-neighbours in the next or previous slab are read through
// L2 (another CTA of the cluster wrote them).
template <int L, bool GAUSS, bool SLAB = false>
__device__ __forceinline__ void half_sweep_packed(const Smem &sm, const Ctx &cx, uint32_t n_sweep,
                                                  const int COL)
{
    constexpr int N = L * L * L;
    constexpr int RUN = kSiteRun;
    constexpr int U = (N / 2) / RUN;
    constexpr int kFlushSites = 40;    // byte-wise sums: 6 (bonds) and 2 (M) per site
    const int WR = cx.WR, RB = cx.RB;  // packed: RB == WR bytes per site
    const int j = threadIdx.x % WR;    // fixed per thread: blockDim.x is a multiple of WR
    const int t0 = 4 * j;

    uint32_t valid = 0;  // bytes of real (not padding) slots in this group
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
        if (t0 + kk < cx.nt) valid |= 1u << (8 * kk);

    float nbeta2[4];  // -2 beta per slot (exact)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) nbeta2[kk] = GAUSS ? __fmul_rn(2.0f, sm.negbeta[t0 + kk]) : 0.0f;
    const uint32_t *thr_w = GAUSS ? nullptr : sm.thr + t0 * 16;

    uint32_t eacc0 = 0, eacc1 = 0, macc0 = 0, macc1 = 0;  // byte-wise partial sums
    int bg[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    int nsites = 0;  // colour-1 sites in the partial sums
    auto flush = [&]() {
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int t = t0 + kk;
                if (t < cx.nt) {
                    const uint32_t ea = r ? eacc1 : eacc0;
                    const uint32_t ma = r ? macc1 : macc0;
                    const long long usum = (long long)((ea >> (8 * kk)) & 0xFFu);
                    const long long b = GAUSS ? (long long)bg[r][kk] : 6LL * nsites - 2LL * usum;
                    const long long mm = 2LL * nsites - 2LL * ((ma >> (8 * kk)) & 0xFFu);
                    atomicAdd(&sm.B[r * cx.Tp + t], (unsigned long long)b);
                    atomicAdd(&sm.M[r * cx.Tp + t], (unsigned long long)mm);
                }
                bg[r][kk] = 0;
            }
        eacc0 = eacc1 = macc0 = macc1 = 0;
        nsites = 0;
    };

    // item = u * WR + j with a fixed step of u per thread (no division per item)
    const int du = blockDim.x / WR;
    const int u_end = SLAB ? cx.u1 : U;
    for (int u = (SLAB ? cx.u0 : 0) + threadIdx.x / WR; u < u_end; u += du) {
        if (COL == 1 && nsites + RUN > kFlushSites) flush();
        {
            const uint32_t c0 = (uint32_t)u;
            uint32_t rnd[2][4][4];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t c2 = ((uint32_t)COL << 24) | ((uint32_t)r << 16) |
                                        (uint32_t)(t0 + kk);
                    const u32x4 o = philox10_rk(cx.k0r, cx.k1, c0, n_sweep, c2, cx.seed_hi);
                    rnd[r][kk][0] = o.v[0];
                    rnd[r][kk][1] = o.v[1];
                    rnd[r][kk][2] = o.v[2];
                    rnd[r][kk][3] = o.v[3];
                }
#pragma unroll
            for (int lane = 0; lane < 4; ++lane) {
                const SiteNb<L> st(u * RUN + lane, COL);
                const int own = st.i * RB + j;
                const uint2 s = load_packed(sm.spins + own);
                const uint2 nxp = load_packed(sm.spins + own + st.dxp * RB);
                const uint2 nxm = load_packed(sm.spins + own + st.dxm * RB);
                const uint2 nyp = load_packed(sm.spins + own + st.dyp * RB);
                const uint2 nym = load_packed(sm.spins + own + st.dym * RB);
                uint2 nzp, nzm;
                if (SLAB && st.z == cx.z1 - 1)
                    nzp = load_packed_cg(sm.spins + own + st.dzp * RB);
                else
                    nzp = load_packed(sm.spins + own + st.dzp * RB);
                if (SLAB && st.z == cx.z0)
                    nzm = load_packed_cg(sm.spins + own + st.dzm * RB);
                else
                    nzm = load_packed(sm.spins + own + st.dzm * RB);
                uint2 fm;
                if constexpr (!GAUSS) {
                    const uint2 jb = *reinterpret_cast<const uint2 *>(sm.J8 + 8 * st.i);
                    const uint32_t m[6] = {__byte_perm(jb.x, jb.y, 0x0000),
                                           __byte_perm(jb.x, jb.y, 0x1111),
                                           __byte_perm(jb.x, jb.y, 0x2222),
                                           __byte_perm(jb.x, jb.y, 0x3333),
                                           __byte_perm(jb.x, jb.y, 0x4444),
                                           __byte_perm(jb.x, jb.y, 0x5555)};
                    uint32_t uw0, uw1;
                    fm.x = pmj_word(s.x, nxp.x, nxm.x, nyp.x, nym.x, nzp.x, nzm.x, m, thr_w,
                                    rnd[0], lane, valid, uw0);
                    fm.y = pmj_word(s.y, nxp.y, nxm.y, nyp.y, nym.y, nzp.y, nzm.y, m, thr_w,
                                    rnd[1], lane, valid, uw1);
                    if (COL == 1) {
                        const uint32_t f0 = fm.x * 0xFFu, f1 = fm.y * 0xFFu;
                        eacc0 += uw0 ^ ((uw0 ^ (0x06060606u - uw0)) & f0);
                        eacc1 += uw1 ^ ((uw1 ^ (0x06060606u - uw1)) & f1);
                    }
                } else {
                    const float jv[6] = {sm.Jg[st.i], sm.Jg[st.i + st.dxm], sm.Jg[N + st.i],
                                         sm.Jg[N + st.i + st.dym], sm.Jg[2 * N + st.i],
                                         sm.Jg[2 * N + st.i + st.dzm]};
                    int bq0[4], bq1[4];
                    fm.x = gauss_word(s.x, nxp.x, nxm.x, nyp.x, nym.x, nzp.x, nzm.x, jv,
                                      cx.hq, nbeta2, rnd[0], lane, valid, COL == 1, bq0);
                    fm.y = gauss_word(s.y, nxp.y, nxm.y, nyp.y, nym.y, nzp.y, nzm.y, jv,
                                      cx.hq, nbeta2, rnd[1], lane, valid, COL == 1, bq1);
                    if (COL == 1) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            bg[0][kk] += bq0[kk];
                            bg[1][kk] += bq1[kk];
                        }
                    }
                }
                uint2 sn;
                sn.x = s.x ^ fm.x;
                sn.y = s.y ^ fm.y;
                store_packed(sm.spins + own, sn);
                if (COL == 1) {
                    const uint2 partner = (st.x & 1) ? nxm : nxp;
                    macc0 += sn.x + partner.x;
                    macc1 += sn.y + partner.y;
                }
            }
        }
        nsites += RUN;
    }
    if (COL == 1 && nsites > 0) flush();
}

// ---------------------------------------------------------------------------
// Half-sweep of colour COL on the packed state held in shared memory, bit
// parallel (+-J; the paper's multispin coding of one sample's replicas,
// methods section). The site row is read as 64-bit words: word w holds
// the 4-slot groups 8w .. 8w + 7, i.e. slots 32w .. 32w + 31 of both
// replicas, one bit per chain (bit 8g + 4r + k = replica r, slot 4(8w + g)
// + k). For a site the unsatisfied-bond count of all 64 chains is one
// bit-sliced 3-bit add of the six words s ^ s_nb ^ J; then every chain draws
// its own Metropolis word (the random-number layout of half_sweep: Philox
// counter (site group, sweep, colour | replica | slot), lane = site of the
// group) and is accepted iff r <= thr[t][sb][u], the class (sb, u) read off
// the bit planes. Chains never share a random word: sharing one among the
// temperatures of a replica would couple the slots and bias the replica
// exchange.
// Work: a warp task is 32 work items (4 consecutive colour sites each) of
// one word w, so that the lanes' per-chain energy counts (bit-sliced, per
// item) reduce over the warp (the +-J sweep's by a butterfly of bit-sliced
// adds, the Gaussian sweep's M by transposes); the host sizes the CTA to the number of
// tasks (at most 8 warps), so small lattices run more, smaller CTAs per SM.
// (Splitting a word's chains over several warps, which then combine their
// flips with shared-memory atomics, measured slower on B300: L = 10, 24
// temperatures 409 -> 362 attempts/ns, L = 12, 56 temperatures 462 -> 300.)
// For COL == 1 the bond sums and magnetisations of the post-sweep
// configuration go to sm.B and sm.M, which start the half-sweep at 3N and N
// (each of the N/2 colour-1 sites gives 6 - 2 u; its x-pair gives 2 - 2 n(-1)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t lds64(const uint8_t *base, int off)
{
    return *reinterpret_cast<const uint64_t *>(base + off);
}

template <int L>
__device__ __forceinline__ void half_sweep_bits(const Smem &sm, const Ctx &cx, uint32_t n_sweep,
                                                const int COL)
{
    constexpr int N = L * L * L;
    constexpr int U = (N / 2) / kSiteRun;
    constexpr int NUB = (U + 31) / 32;  // blocks of 32 work items
    constexpr int DU = 5, DM = 4;       // counter planes: per item at most 24 and 8
    const int RB = cx.RB;               // bytes per site, a multiple of 8
    const int NW = RB >> 3;             // 64-bit words per site
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    const int nt = cx.nt;
    for (int tk = warp; tk < NUB * NW; tk += nwarp) {
        const int ub = tk / NW, w = tk % NW;
        const int u = ub * 32 + lane;
        uint64_t cu[DU], cm[DM];
#pragma unroll
        for (int k = 0; k < DU; ++k) cu[k] = 0;
#pragma unroll
        for (int k = 0; k < DM; ++k) cm[k] = 0;
        if (u < U) {
            uint64_t s[4], u0[4], u1[4], u2[4], part[4];
            int own[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const SiteNb<L> st(u * kSiteRun + l, COL);
                own[l] = st.i * RB + 8 * w;
                s[l] = lds64(sm.spins, own[l]);
                const uint64_t nxp = lds64(sm.spins, own[l] + st.dxp * RB);
                const uint64_t nxm = lds64(sm.spins, own[l] + st.dxm * RB);
                const uint64_t nyp = lds64(sm.spins, own[l] + st.dyp * RB);
                const uint64_t nym = lds64(sm.spins, own[l] + st.dym * RB);
                const uint64_t nzp = lds64(sm.spins, own[l] + st.dzp * RB);
                const uint64_t nzm = lds64(sm.spins, own[l] + st.dzm * RB);
                const uint2 jb = *reinterpret_cast<const uint2 *>(sm.J8 + 8 * st.i);
                // bond bit 1 (J = -1) -> all-ones mask
                auto jm = [](uint32_t word, int byte) {
                    return (uint64_t)0 - (uint64_t)((word >> (8 * byte)) & 1u);
                };
                const uint64_t d0 = s[l] ^ nxp ^ jm(jb.x, 0), d1 = s[l] ^ nxm ^ jm(jb.x, 1);
                const uint64_t d2 = s[l] ^ nyp ^ jm(jb.x, 2), d3 = s[l] ^ nym ^ jm(jb.x, 3);
                const uint64_t d4 = s[l] ^ nzp ^ jm(jb.y, 0), d5 = s[l] ^ nzm ^ jm(jb.y, 1);
                // u = number of unsatisfied bonds: two full adders and a carry merge
                const uint64_t sa = d0 ^ d1 ^ d2, ca = (d0 & d1) | (d2 & (d0 ^ d1));
                const uint64_t sb = d3 ^ d4 ^ d5, cb = (d3 & d4) | (d5 & (d3 ^ d4));
                u0[l] = sa ^ sb;
                const uint64_t cc = sa & sb;
                u1[l] = ca ^ cb ^ cc;
                u2[l] = (ca & cb) | (cc & (ca ^ cb));
                part[l] = (st.x & 1) ? nxm : nxp;
            }
            uint64_t fl[4] = {0, 0, 0, 0};
            for (int g = 0; g < 8; ++g) {
                const int j = 8 * w + g;  // 4-slot group
                if (4 * j >= nt) break;   // padding groups (the same for the whole warp)
                // per site, the group's class planes as bytes: s | u2 | u1 | u0
                uint32_t X[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const int sh = 8 * g;
                    const uint32_t bs = (uint32_t)(s[l] >> sh) & 0xFFu;
                    const uint32_t b2 = (uint32_t)(u2[l] >> sh) & 0xFFu;
                    const uint32_t b1 = (uint32_t)(u1[l] >> sh) & 0xFFu;
                    const uint32_t b0 = (uint32_t)(u0[l] >> sh) & 0xFFu;
                    X[l] = bs | (b2 << 8) | (b1 << 16) | (b0 << 24);
                }
                uint32_t fb[4] = {0, 0, 0, 0};
#pragma unroll
                for (int k8 = 0; k8 < 8; ++k8) {
                    const int t = 4 * j + (k8 & 3), r = k8 >> 2;
                    if (t >= nt) continue;  // padding slots: never flipped
                    const uint32_t c2 = ((uint32_t)COL << 24) | ((uint32_t)r << 16) | (uint32_t)t;
                    const u32x4 o = philox10_rk(cx.k0r, cx.k1, (uint32_t)u, n_sweep, c2, cx.seed_hi);
                    const uint32_t *thr_t = sm.thr + t * 16;
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        // bit k8 of the four planes gathered into the class
                        // index sb * 8 + u: the four bits sit in bit 0 of the
                        // bytes, and one product moves them to bits 27..24
                        // (no other partial product reaches those bits)
                        const uint32_t v = (X[l] >> k8) & 0x01010101u;
                        const uint32_t idx = (v * 0x08040201u) >> 24;
                        fb[l] |= (uint32_t)(o.v[l] <= thr_t[idx]) << k8;
                    }
                }
#pragma unroll
                for (int l = 0; l < 4; ++l) fl[l] |= (uint64_t)fb[l] << (8 * g);
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint64_t sn = s[l] ^ fl[l];
                *reinterpret_cast<uint64_t *>(sm.spins + own[l]) = sn;
                if (COL == 1) {
                    // unsatisfied bonds after the flip: 6 - u where flipped
                    const uint64_t f = fl[l];
                    const uint64_t n1b = ~(u1[l] ^ u0[l]);
                    const uint64_t n2b = ~u2[l] & ~(u1[l] & u0[l]);
                    const uint64_t un[3] = {u0[l], (u1[l] & ~f) | (n1b & f), (u2[l] & ~f) | (n2b & f)};
                    bs_add<DU, 3>(cu, un);
                    const uint64_t mm[2] = {sn ^ part[l], sn & part[l]};
                    bs_add<DM, 2>(cm, mm);
                }
            }
        }
        if (COL == 1) {
            // per chain, the warp's counts by a bit-sliced butterfly: lane l
            // ends with chain bits b0 = 32 (l >> 4) + (l & 15) and b0 + 16
            uint32_t tu[2], tm[2];
            warp_bs_totals<DU>(cu, tu[0], tu[1]);
            warp_bs_totals<DM>(cm, tm[0], tm[1]);
            const long long vu[2] = {tu[0], tu[1]}, vm[2] = {tm[0], tm[1]};
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int b = 32 * (lane >> 4) + (lane & 15) + 16 * hf;
                const int t = 4 * (8 * w + (b >> 3)) + (b & 3), r = (b >> 2) & 1;
                if (t < nt) {
                    atomicAdd(&sm.B[r * cx.Tp + t], (unsigned long long)(-2 * vu[hf]));
                    atomicAdd(&sm.M[r * cx.Tp + t], (unsigned long long)(-2 * vm[hf]));
                }
            }
        }
    }
}

// Local field of one chain from the neighbour words nb (the six bonds in the
// order +x, -x, +y, -y, +z, -z, couplings j), mp = 2^(31 - p) for the chain
// at bit p: nb * mp moves the chain's bit to bit 31, where it flips the sign
// of the coupling. Exact on the 2^-17 grid in any order, as in gauss_field.
__device__ __forceinline__ float gauss_field_mp(uint32_t mp, const uint32_t (&nb)[6],
                                                const float (&j)[6])
{
    float t[6];
#pragma unroll
    for (int d = 0; d < 6; ++d)
        t[d] = __int_as_float(__float_as_int(j[d]) ^ (mul_lo(nb[d], mp) & 0x80000000u));
    return __fadd_rn(__fadd_rn(__fadd_rn(t[0], t[1]), __fadd_rn(t[2], t[3])), __fadd_rn(t[4], t[5]));
}

// ---------------------------------------------------------------------------
// Half-sweep of colour COL for Gaussian couplings on the bit-per-chain state
// in shared memory (skewed rows, bits_row). A warp task is 32 work items
// (lane = item u: 4 consecutive colour-COL sites, one Philox counter group)
// times one chain set: csb consecutive 4-slot groups (bytes of the site row,
// 8 chains each: slots 4j..4j+3 of replica 0 in bits 0-3, of replica 1 in
// bits 4-7) inside one 32-bit word of the row. The lane loads its four
// sites' words (own spin and six neighbours) and couplings once; then, for
// each chain of a group (the 8 unrolled), one Philox call gives the chain's
// four random words and each site's local field is the six couplings with
// the neighbours' sign bits. The rule, the random numbers and every
// rounding are those of half_sweep (gauss_word: the screened test, the exact
// threshold for draws in the band), so the result is the byte-per-chain
// path's bit for bit; what is shared is the per-site work (indices, loads),
// now spread over 8-32 chains instead of 4. Each decision is kept as a sign
// bit (bit 31 set = flip), which gives both the chain's flip bit and the
// sign of s_new * b. Lanes past the last item take a real item and store
// nothing.
// For COL == 1: each chain's s_new * b over the task's sites (at most
// 128 x 96 x 2^17 < 2^31 in units 2^-17) is one warp reduction, added to
// sm.B (which starts at 0); M by bit-sliced counters and warp transposes
// (sm.M starts at N and each -1 among a colour-1 site and its x-partner
// subtracts 2).
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void half_sweep_bits_gauss(const Smem &sm, const Ctx &cx,
                                                      uint32_t n_sweep, const int COL,
                                                      const int csb)
{
    constexpr int N = L * L * L;
    constexpr int U = (N / 2) / kSiteRun;
    constexpr int NUB = (U + 31) / 32;  // blocks of 32 work items
    constexpr int NJ = N + N / 8;       // skewed coupling plane
    constexpr int DM = 4;               // counter planes: per lane at most 8
    constexpr uint32_t SB = 0x80000000u;
    const int RB = cx.RB, nt = cx.nt;
    const int ngrp = (nt + 3) >> 2;     // 4-slot groups holding real chains
    const int ncs = (ngrp + csb - 1) / csb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarp = blockDim.x >> 5;
    for (int tk = warp; tk < NUB * ncs; tk += nwarp) {
        const int ub = tk / ncs, cs = tk - ub * ncs;
        const bool live = ub * 32 + lane < U;
        const int u = live ? ub * 32 + lane : U - 1;
        const int g0 = cs * csb;          // first group of the set
        const int wb = g0 & ~3;           // byte of the row word holding the set
        const int sh0 = 8 * (g0 & 3);     // bit of the set's first chain in that word
        uint32_t sw[4], nw[4][6];
        float jv[4][6];
        int own[4];
        uint32_t xodd = 0;  // bit l: site l has odd x (its x-partner is the -x neighbour)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const SiteNb<L> st(u * kSiteRun + l, COL);
            xodd |= (uint32_t)(st.x & 1) << l;
            own[l] = bits_row<true>(st.i, RB) + wb;
            sw[l] = lds32(sm.spins, own[l]);
            const int nbi[6] = {st.i + st.dxp, st.i + st.dxm, st.i + st.dyp,
                                st.i + st.dym, st.i + st.dzp, st.i + st.dzm};
#pragma unroll
            for (int d = 0; d < 6; ++d) nw[l][d] = lds32(sm.spins, bits_row<true>(nbi[d], RB) + wb);
            const int ji = bits_jidx(st.i);
            jv[l][0] = sm.Jg[ji];
            jv[l][1] = sm.Jg[bits_jidx(nbi[1])];
            jv[l][2] = sm.Jg[NJ + ji];
            jv[l][3] = sm.Jg[NJ + bits_jidx(nbi[3])];
            jv[l][4] = sm.Jg[2 * NJ + ji];
            jv[l][5] = sm.Jg[2 * NJ + bits_jidx(nbi[5])];
        }
        uint32_t fb[4] = {0u, 0u, 0u, 0u};  // flipped chains per site
        const int gend = min(g0 + csb, ngrp);
#pragma unroll 1
        for (int j = g0; j < gend; ++j) {
            const int pb = sh0 + 8 * (j - g0);    // bit of the group's chain 0
            const uint32_t mpb = 1u << (31 - pb);
            uint32_t gb[4] = {0u, 0u, 0u, 0u};    // the group's flips per site, bit k8
            // the replicas' 4 chains unrolled, the replicas rolled: a body of
            // 4 Philox calls keeps the instruction working set in cache
#pragma unroll 1
            for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k8 = 4 * r + kk;
                const int t = 4 * j + kk;
                if (t < nt) {  // padding slots (the same for the whole warp) never flip
                    const uint32_t mp = mpb >> k8;
                    const uint32_t c2 = ((uint32_t)COL << 24) | ((uint32_t)r << 16) | (uint32_t)t;
                    const u32x4 o = philox10_rk(cx.k0r, cx.k1, (uint32_t)u, n_sweep, c2, cx.seed_hi);
                    const float nbeta2 = __fmul_rn(2.0f, sm.negbeta[t]);
                    float b[4], x[4];
                    uint32_t so[4], dm[4];  // own sign, decision: bit 31
                    bool amb = false;
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        b[l] = gauss_field_mp(mp, nw[l], jv[l]);
                        so[l] = mul_lo(sw[l], mp) & SB;
                        x[l] = __fmul_rn(nbeta2, __int_as_float(__float_as_int(__fadd_rn(b[l], cx.hq)) ^ so[l]));
                        dm[l] = __float_as_uint(screen_logp(x[l], o.v[l], amb)) & SB;
                    }
                    if (amb) {
#pragma unroll
                        for (int l = 0; l < 4; ++l) dm[l] = o.v[l] <= thr_of_logp(x[l]) ? SB : 0u;
                    }
#pragma unroll
                    for (int l = 0; l < 4; ++l) gb[l] = mad_hi(dm[l], 2u << k8, gb[l]);
                    if (COL == 1) {
                        int e = 0;
#pragma unroll
                        for (int l = 0; l < 4; ++l)  // s_new * b: the sign of b flipped where s_new = -1
                            e += __float2int_rn(__fmul_rn(__int_as_float(__float_as_int(b[l]) ^ so[l] ^ dm[l]),
                                                          131072.0f));
                        e = __reduce_add_sync(0xFFFFFFFFu, live ? e : 0);
                        if (lane == 0) atomicAdd(&sm.B[r * cx.Tp + t], (unsigned long long)(long long)e);
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) fb[l] |= gb[l] << pb;
        }
        const uint32_t setm = (csb == 4 ? 0xFFFFFFFFu : ((1u << (8 * csb)) - 1u) << sh0);
        uint32_t cm[DM] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint32_t sn = sw[l] ^ fb[l];
            if (live) {
                if (csb == 4)
                    sts32(sm.spins, own[l], sn);
                else if (csb == 2)
                    *reinterpret_cast<uint16_t *>(sm.spins + own[l] + (g0 & 3)) = (uint16_t)(sn >> sh0);
                else
                    sm.spins[own[l] + (g0 & 3)] = (uint8_t)(sn >> sh0);
            }
            if (COL == 1) {
                // the x-partner of a colour-1 site is its +x or -x neighbour
                const uint32_t part = ((xodd >> l) & 1u) ? nw[l][1] : nw[l][0];
                const uint32_t msk = live ? setm : 0u;
                const uint32_t mm[2] = {(sn ^ part) & msk, (sn & part) & msk};
                bs_add32<DM, 2>(cm, mm);
            }
        }
        if (COL == 1) {
            long long vm = 0;  // lane b: the -1 count of chain bit b of the word
#pragma unroll
            for (int k = 0; k < DM; ++k) vm += (long long)warp_column_popc(cm[k]) << k;
            const int j = (wb + (lane >> 3)), k8 = lane & 7;
            const int t = 4 * j + (k8 & 3), r = k8 >> 2;
            if (((setm >> lane) & 1u) && t < nt)
                atomicAdd(&sm.M[r * cx.Tp + t], (unsigned long long)(-2 * vm));
        }
    }
}

// ---------------------------------------------------------------------------
// Replica exchange between slots p and p+1 of each replica (pairs of one
// parity), then the state swap of accepted pairs as byte permutations of the
// 4-slot words. stamp identifies this exchange in xflag.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void exchange_decide(const Smem &sm, const Ctx &cx, const Int8Args &a,
                                                int parity, uint32_t ctr1, uint32_t rflag,
                                                uint32_t stamp)
{
    // warp 0 only: the pair decisions, then the byte-permutation selectors
    const int lane = threadIdx.x;
    const int nt = cx.nt, Tp = cx.Tp, WR = cx.WR;
    const int np = (nt - parity) / 2;
    if (lane < 2) {
        sm.anyswap[lane] = 0;
        sm.accm[lane] = 0ull;
    }
    __syncwarp();
    for (int id = lane; id < 2 * np; id += 32) {
        const int r = id / np;
        const int p = parity + 2 * (id % np);
        if (p + 1 >= nt) continue;
        unsigned long long *Bp = sm.B + r * Tp + p;
        unsigned long long *Mp = sm.M + r * Tp + p;
        const long long dB = (long long)Bp[0] - (long long)Bp[1];
        const long long dM = (long long)Mp[0] - (long long)Mp[1];
        const float t1 = __fmul_rn(__ll2float_rn(dB), a.qJ_f);
        const float t2 = __fmul_rn(a.h_f, __ll2float_rn(dM));
        const float dE = -__fadd_rn(t1, t2);
        const float D = __fmul_rn(sm.dbeta[p], dE);
        const u32x4 o = philox10(cx.seed_lo ^ kTagExc, (uint32_t)(cx.s + a.s_key0), (uint32_t)p, ctr1,
                                 (uint32_t)r | rflag, cx.seed_hi);
        const bool acc = (D >= 0.0f) || (o.v[0] <= thr_of_logp(D));
        if (acc) {
            const unsigned long long tb = Bp[0];
            Bp[0] = Bp[1];
            Bp[1] = tb;
            const unsigned long long tm = Mp[0];
            Mp[0] = Mp[1];
            Mp[1] = tm;
            sm.xflag[r * Tp + p] = stamp;
            atomicOr(&sm.accm[r], 1ull << p);
        }
    }
    __syncwarp();
    for (int id = lane; id < 2 * WR; id += 32) {
        const int r = id / WR, j = id % WR;
        const uint32_t *fl = sm.xflag + r * Tp;
        uint32_t s1 = 0, s2 = 0;
        bool any = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = 4 * j + k;
            int src = t;
            if (t + 1 < nt && fl[t] == stamp) src = t + 1;
            else if (t >= 1 && t < nt && fl[t - 1] == stamp) src = t - 1;
            any |= (src != t);
            // first permutation over {next word : this word}, second brings in
            // byte 3 of the previous word
            uint32_t n1 = (uint32_t)k, n2 = (uint32_t)k;
            if (src >= 4 * j && src < 4 * j + 4) n1 = (uint32_t)(src - 4 * j);
            else if (src == 4 * j + 4) n1 = 4u;
            else n2 = 7u;  // src == 4j - 1
            s1 |= n1 << (4 * k);
            s2 |= n2 << (4 * k);
        }
        sm.sel[(r * WR + j) * 2 + 0] = s1;
        sm.sel[(r * WR + j) * 2 + 1] = s2;
        if (any) atomicOr(&sm.anyswap[r], 1);
    }
}

// All threads: apply the accepted swaps row by row (after a block barrier
// that publishes the selectors). Up to 8 words per replica row (32 slots),
// a thread keeps one replica (blockDim.x is even) with its selectors in
// registers, and leaves the words that no accepted pair touches unwritten.
template <int L>
__device__ __forceinline__ void exchange_apply(const Smem &sm, const Ctx &cx)
{
    constexpr int N = L * L * L;
    constexpr int kMaxW = 8;
    constexpr uint32_t kIdent = 0x3210u;
    const int WR = cx.WR, RB = cx.RB;
    if (WR <= kMaxW) {
        const int r = threadIdx.x & 1;
        if (!sm.anyswap[r]) return;
        const uint32_t *sel = sm.sel + r * WR * 2;
        uint32_t s1[kMaxW], s2[kMaxW], touched = 0;
#pragma unroll
        for (int jj = 0; jj < kMaxW; ++jj) {
            s1[jj] = jj < WR ? sel[2 * jj] : kIdent;
            s2[jj] = jj < WR ? sel[2 * jj + 1] : kIdent;
            if (s1[jj] != kIdent || s2[jj] != kIdent) touched |= 1u << jj;
        }
        for (int site = threadIdx.x >> 1; site < N; site += blockDim.x >> 1) {
            uint8_t *row = sm.spins + site * RB + 4 * r;  // word j at row + 8j
            uint32_t w[kMaxW];
#pragma unroll
            for (int jj = 0; jj < kMaxW; ++jj) w[jj] = jj < WR ? lds32(row, 8 * jj) : 0u;
#pragma unroll
            for (int jj = 0; jj < kMaxW; ++jj) {
                if (!((touched >> jj) & 1u)) continue;
                const uint32_t next = jj + 1 < kMaxW ? w[jj + 1] : 0u;
                const uint32_t prev = jj > 0 ? w[jj - 1] : 0u;
                sts32(row, 8 * jj, __byte_perm(__byte_perm(w[jj], next, s1[jj]), prev, s2[jj]));
            }
        }
        return;
    }
    for (int id = threadIdx.x; id < 2 * N; id += blockDim.x) {
        const int r = id & 1, site = id >> 1;
        if (!sm.anyswap[r]) continue;
        uint8_t *row = sm.spins + site * RB + 4 * r;  // word j at row + 8j
        const uint32_t *sel = sm.sel + r * WR * 2;
        uint32_t prev = 0, cur = lds32(row, 0);
        for (int jj = 0; jj < WR; ++jj) {
            const uint32_t next = (jj + 1 < WR) ? lds32(row, 8 * (jj + 1)) : 0u;
            const uint32_t tmp = __byte_perm(cur, next, sel[2 * jj]);
            sts32(row, 8 * jj, __byte_perm(tmp, prev, sel[2 * jj + 1]));
            prev = cur;
            cur = next;
        }
    }
}

// Packed state: per site, each replica's slots as one mask (bit t = slot t);
// an accepted pair (p, p+1) swaps bits p and p+1. Pairs of one parity are
// disjoint, so one masked exchange per replica applies them all.
// Sites [site0, site1) (a cluster CTA's slab; the whole lattice by default).
// SKEW: the rows at bits_row (Gaussian bit-parallel state).
template <int L, bool SKEW = false>
__device__ __forceinline__ void exchange_apply_packed(const Smem &sm, const Ctx &cx, int site0 = 0,
                                                      int site1 = L * L * L)
{
    const int WR = cx.WR, RB = cx.RB;
    const unsigned long long a0 = sm.accm[0], a1 = sm.accm[1];
    if (!(a0 | a1)) return;
    for (int site = site0 + threadIdx.x; site < site1; site += blockDim.x) {
        uint8_t *row = sm.spins + bits_row<SKEW>(site, RB);
        unsigned long long w0 = 0, w1 = 0;
        for (int jj = 0; jj < WR; ++jj) {
            const unsigned long long b = row[jj];
            w0 |= (b & 15ull) << (4 * jj);
            w1 |= (b >> 4) << (4 * jj);
        }
        const unsigned long long x0 = (w0 ^ (w0 >> 1)) & a0;
        const unsigned long long x1 = (w1 ^ (w1 >> 1)) & a1;
        w0 ^= x0 | (x0 << 1);
        w1 ^= x1 | (x1 << 1);
        for (int jj = 0; jj < WR; ++jj)
            row[jj] = (uint8_t)(((w0 >> (4 * jj)) & 15ull) | (((w1 >> (4 * jj)) & 15ull) << 4));
    }
}

// Counts of q = -1 per phase d of one wave vector, for the 4 slots of a
// marginal word at once, from the 2D marginal pm[(A*L + B)*nw]: PAT 0: A = d;
// 1: B = d; 2: A + B = d; 3: A - B = d (mod L). This lane takes the phases
// d = part + 4k; the sums stay in byte lanes (one per slot) while L*L <= 255,
// otherwise in two words of 16-bit lanes (lo: slots 0, 2; hi: slots 1, 3).
template <int L, int PAT>
__device__ __forceinline__ void count_phases(const uint32_t *pm, int nw, int part,
                                             uint32_t (&lo)[(L + 3) / 4],
                                             uint32_t (&hi)[(L + 3) / 4])
{
    constexpr bool kWide = L * L > 255;
#pragma unroll
    for (int k = 0; k < (L + 3) / 4; ++k) {
        const int d = part + 4 * k;
        uint32_t a = 0, b = 0;
        if (d < L) {
#pragma unroll 4
            for (int aa = 0; aa < L; ++aa) {
                int A = aa, Bc;
                if (PAT == 0) {
                    A = d;
                    Bc = aa;
                } else if (PAT == 1) {
                    Bc = d;
                } else {
                    Bc = PAT == 2 ? d - aa : aa - d;
                    Bc += (Bc >> 31) & L;  // mod L of a value in (-L, L)
                }
                const uint32_t w = pm[(A * L + Bc) * nw];
                if (kWide) {
                    a += w & 0x00FF00FFu;
                    b += (w >> 8) & 0x00FF00FFu;
                } else {
                    a += w;
                }
            }
        }
        lo[k] = a;
        hi[k] = b;
    }
}

// ---------------------------------------------------------------------------
// Overlap measurement (eq. overlap) for every slot: q = s^(0) s^(1);
// (A) 2D marginals of the q = -1 counts over the xy, xz and yz planes,
// (B) per (slot, v): the integer projections P_v[d] (v over the k1 and k2
// orbits), the FP32 DFT in ascending d and the FP64 accumulation,
// together with Q; E and M per slot before both. Processed mchunk 4-slot
// groups at a time.
// ---------------------------------------------------------------------------
// Per-sample state that another CTA may have written in the same launch (a
// segmented launch hands a sample's segments to whichever CTA is free) is
// read from L2: L1 is not coherent across SMs, and a CTA that ran an earlier
// segment of the sample could still hold its lines.
__device__ __forceinline__ double ld_acc(const double *p, bool seg)
{
    return seg ? __ldcg(p) : *p;
}

// Energies and magnetisations of every slot (one thread per slot).
__device__ __forceinline__ void measure_energies(const Smem &sm, const Ctx &cx, const Int8Args &a,
                                                 int bin)
{
    const int Tp = cx.Tp, nt = cx.nt;
    const bool seg = a.n_seg > 1;  // the accumulators may come from another SM
    // device layout [S][bins][40][nt]: entry k of slot t at accs[k * nt + t],
    // so lanes over consecutive slots touch consecutive doubles
    double *accs = a.acc + ((size_t)cx.s * a.n_bins + bin) * SG_NACC * nt;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        double *ac = accs + t;  // entry k at ac[k * nt]
        double o5 = ld_acc(ac + 5 * nt, seg), o6 = ld_acc(ac + 6 * nt, seg);
        double o7 = ld_acc(ac + 7 * nt, seg), o8 = ld_acc(ac + 8 * nt, seg);
        for (int r = 0; r < 2; ++r) {
            const long long Bv = (long long)sm.B[r * Tp + t];
            const long long Mv = (long long)sm.M[r * Tp + t];
            const double e = -__dadd_rn(__dmul_rn((double)Bv, a.qJ_d), __dmul_rn(a.h_d, (double)Mv));
            o5 = __dadd_rn(o5, e);
            o6 = __dadd_rn(o6, __dmul_rn(e, e));
        }
        for (int r = 0; r < 2; ++r) {
            const double m = (double)(long long)sm.M[r * Tp + t];
            o7 = __dadd_rn(o7, m);
            o8 = __dadd_rn(o8, __dmul_rn(m, m));
        }
        ac[5 * nt] = o5;
        ac[6 * nt] = o6;
        ac[7 * nt] = o7;
        ac[8 * nt] = o8;
    }
}

// (A) 2D marginals of the q = -1 counts of the words j0 .. j0 + nw - 1 into
// sm.marg; the group index varies fastest across lanes. SLAB (cluster
// instances): only the sites of this CTA's z-planes [cx.z0, cx.z1), i.e.
// the partial xy marginal over those planes and the complete xz and yz lines
// inside them (the other lines count 0).
template <int L, bool PACK, bool SLAB = false, bool SKEW = false>
__device__ __forceinline__ void measure_marginals(const Smem &sm, const Ctx &cx, int j0, int nw)
{
    constexpr int LL = L * L;
    const int RB = cx.RB;
    {
        // id / nw by a multiply-high with ceil(2^32 / nw): exact for
        // 2 <= nw <= 16 and id < 3 L^2 nw, L <= 64 (checked exhaustively)
        const uint32_t inv_nw = nw > 1 ? (uint32_t)((0xFFFFFFFFull + (unsigned)nw) / (unsigned)nw) : 0u;
        for (int id = threadIdx.x; id < 3 * LL * nw; id += blockDim.x) {
            const int rest = nw > 1 ? (int)__umulhi((uint32_t)id, inv_nw) : id;
            const int jj = id - rest * nw;
            const int ab = rest % LL;
            const int plane = rest / LL;
            const int A = ab % L, Bc = ab / L;  // A varies fastest
            int base, step;
            if (plane == 0) {        // (x=A, y=Bc), over z
                base = A + L * Bc;
                step = LL;
            } else if (plane == 1) { // (x=A, z=Bc), over y
                base = A + LL * Bc;
                step = L;
            } else {                 // (y=A, z=Bc), over x
                base = L * A + LL * Bc;
                step = 1;
            }
            uint32_t cnt = 0;
            if constexpr (SLAB) {  // packed state, this CTA's planes only
                const bool in = plane == 0 || (Bc >= cx.z0 && Bc < cx.z1);
                const int m0 = plane == 0 ? cx.z0 : 0, m1 = !in ? 0 : plane == 0 ? cx.z1 : L;
                for (int m = m0; m < m1; ++m) {
                    const uint32_t b = sm.spins[(size_t)(base + m * step) * RB + j0 + jj];
                    cnt += expand4((b ^ (b >> 4)) & 15u);
                }
            } else if constexpr (PACK) {  // q of the group's 4 slots: the two nibbles' xor
#pragma unroll 4
                for (int m = 0; m < L; ++m) {
                    const uint32_t b = sm.spins[bits_row<SKEW>(base + m * step, RB) + j0 + jj];
                    cnt += expand4((b ^ (b >> 4)) & 15u);
                }
            } else {
                const int woff = 8 * (j0 + jj);
#pragma unroll 4
                for (int m = 0; m < L; ++m) {
                    const uint2 w = *reinterpret_cast<const uint2 *>(sm.spins + (base + m * step) * RB + woff);
                    cnt += w.x ^ w.y;
                }
            }
            sm.marg[(plane * LL + A * L + Bc) * nw + jj] = cnt;
        }
    }
}

// (B) projections, FP32 DFT and FP64 accumulation of the words j0 .. j0 +
// nw - 1 from the marginals in sm.marg.
template <int L>
__device__ __forceinline__ void measure_projections(const Smem &sm, const Ctx &cx,
                                                    const Int8Args &a, int bin, int j0, int nw)
{
    constexpr int LL = L * L;
    const int nt = cx.nt;
    const bool seg = a.n_seg > 1;
    double *accs = a.acc + ((size_t)cx.s * a.n_bins + bin) * SG_NACC * nt;
    {
        // (B) one warp per wave vector v (v = 0..8; the v = 0 warp also takes
        // Q, whose count is the sum of its phases). Lane = 4 * (word jj) +
        // part: the part counts its phases for the word's 4 slots at once,
        // shuffles then give each lane every phase of slot 4 * jj + part, and
        // the lane runs the FP32 DFT in ascending d and the FP64 accumulation.
        // The accumulators are loaded first, so that their global-memory
        // latency overlaps the counting.
        {
            constexpr int ND = (L + 3) / 4;
            constexpr bool kWide = L * L > 255;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int nwarp = blockDim.x >> 5;  // full warps (shuffles need all lanes)
            const int part = lane & 3;
            for (int v = warp; v < 9 && warp < nwarp; v += nwarp) {
                for (int jb = 0; jb < nw; jb += 8) {
                    const int jj = jb + (lane >> 2);
                    const int t = 4 * (j0 + jj) + part;
                    const bool live = jj < nw && t < nt;
                    const int jc = jj < nw ? jj : 0;  // lanes past the chunk count a real word
                    double *acv = accs + (size_t)(9 + 3 * v) * nt + t;  // entry at acv[q * nt]
                    double *acq = accs + t;                            // Q: entries 0..4
                    double old[3] = {0.0, 0.0, 0.0};
                    if (live) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) old[q] = ld_acc(acv + q * nt, seg);
                    }
                    uint32_t lo[ND], hi[ND];
                    const uint32_t *pm0 = sm.marg + jc;
                    if (v == 0)
                        count_phases<L, 0>(pm0, nw, part, lo, hi);
                    else if (v == 1)
                        count_phases<L, 1>(pm0, nw, part, lo, hi);
                    else if (v == 2)
                        count_phases<L, 1>(pm0 + LL * nw, nw, part, lo, hi);
                    else {
                        const int plane = (v == 3 || v == 4) ? 0 : (v == 5 || v == 6) ? 1 : 2;
                        const uint32_t *pm = pm0 + plane * LL * nw;
                        if (v == 3 || v == 5 || v == 7)
                            count_phases<L, 2>(pm, nw, part, lo, hi);
                        else
                            count_phases<L, 3>(pm, nw, part, lo, hi);
                    }
                    float re = 0.0f, im = 0.0f;
                    int Qi = 0;
                    const int src0 = lane & ~3;
#pragma unroll
                    for (int d = 0; d < L; ++d) {
                        // phase d lives in lane part d & 3, sum index d >> 2
                        const uint32_t xl = __shfl_sync(0xFFFFFFFFu, lo[d >> 2], src0 | (d & 3));
                        int c;
                        if (kWide) {
                            const uint32_t xh = __shfl_sync(0xFFFFFFFFu, hi[d >> 2], src0 | (d & 3));
                            const uint32_t x = (part & 1) ? xh : xl;
                            c = (int)((part & 2) ? (x >> 16) : (x & 0xFFFFu));
                        } else {
                            c = (int)((xl >> (8 * part)) & 0xFFu);
                        }
                        const int P = LL - 2 * c;
                        Qi += P;
                        const float Pf = (float)P;
                        re = __fmaf_rn(Pf, sm.twid[d], re);
                        im = __fmaf_rn(Pf, sm.twid[L + d], im);
                    }
                    if (!live) continue;
                    // (the exact conversions and squares from integer operations)
                    old[0] = __dadd_rn(old[0], f64_of_f32(re));
                    old[1] = __dadd_rn(old[1], f64_of_f32(im));
                    old[2] = __dadd_rn(old[2], __dadd_rn(f64_sq_of_f32(re), f64_sq_of_f32(im)));
#pragma unroll
                    for (int q = 0; q < 3; ++q) acv[q * nt] = old[q];
                    if (v == 0) {
                        if (a.hist)  // P(q): replicas agree on (N + Q) / 2 sites
                            atomicAdd(a.hist + ((size_t)t * a.n_bins + bin) * (L * LL + 1) +
                                          ((L * LL + Qi) >> 1),
                                      1ull);
                        double oq[5];
#pragma unroll
                        for (int q = 0; q < 5; ++q) oq[q] = ld_acc(acq + q * nt, seg);
                        const double Q = (double)Qi;
                        const double Q2 = __dmul_rn(Q, Q);
                        oq[0] = __dadd_rn(oq[0], 1.0);
                        oq[1] = __dadd_rn(oq[1], Q);
                        oq[2] = __dadd_rn(oq[2], Q2);
                        oq[3] = __dadd_rn(oq[3], __dmul_rn(Q2, Q));
                        oq[4] = __dadd_rn(oq[4], __dmul_rn(Q2, Q2));
#pragma unroll
                        for (int q = 0; q < 5; ++q) acq[q * nt] = oq[q];
                    }
                }
            }
        }
    }
}

template <int L, bool PACK, bool SKEW = false>
__device__ __forceinline__ void measure_step(const Smem &sm, const Ctx &cx, const Int8Args &a,
                                             int bin)
{
    // energies and magnetisations first, so that the projection phase reads
    // nothing the next sweep overwrites
    measure_energies(sm, cx, a, bin);
    // only the words holding real slots (the bit-per-chain rows are padded
    // to 32 slots)
    const int WRv = (cx.nt + 3) >> 2;
    for (int j0 = 0; j0 < WRv; j0 += a.mchunk) {
        const int nw = min(a.mchunk, WRv - j0);
        measure_marginals<L, PACK, false, SKEW>(sm, cx, j0, nw);
        __syncthreads();
        measure_projections<L>(sm, cx, a, bin, j0, nw);
        // the next chunk's marginals overwrite this chunk's; after the last
        // chunk the next sweep touches nothing this phase reads (spins, B and
        // M are not read here), so no barrier is needed
        if (j0 + a.mchunk < WRv) __syncthreads();
    }
}

__device__ __forceinline__ void copy16(void *dst, const void *src, size_t bytes)
{
    int4 *d = reinterpret_cast<int4 *>(dst);
    const int4 *s = reinterpret_cast<const int4 *>(src);
    for (size_t k = threadIdx.x; k < bytes / 16; k += blockDim.x) d[k] = s[k];
}

// The same from global memory through L2 only (state another SM may have
// stored in this launch).
__device__ __forceinline__ void copy16_cg(void *dst, const void *src, size_t bytes)
{
    int4 *d = reinterpret_cast<int4 *>(dst);
    const int4 *s = reinterpret_cast<const int4 *>(src);
    for (size_t k = threadIdx.x; k < bytes / 16; k += blockDim.x) d[k] = __ldcg(s + k);
}

// The Gaussian bit-parallel state between its global-memory rows [N][RB]
// and the skewed shared-memory rows (bits_row), 4 bytes per thread and step
// (RB is 8 or 16): IN copies to shared memory (through L2 only with CG).
template <bool IN, bool CG>
__device__ __forceinline__ void copy_rows_skewed(uint8_t *smem, uint8_t *gmem, int N, int RB)
{
    const int lrb = RB == 16 ? 4 : 3;
    for (int k = threadIdx.x; k < N * RB / 4; k += blockDim.x) {
        const int i = (4 * k) >> lrb;
        const int so = bits_row<true>(i, RB) + 4 * k - (i << lrb);
        uint32_t *g = reinterpret_cast<uint32_t *>(gmem) + k;
        uint32_t *sp = reinterpret_cast<uint32_t *>(smem + so);
        if (IN)
            *sp = CG ? __ldcg(g) : *g;
        else
            *g = *sp;
    }
}

// Couplings [3][N] into the skewed planes [3][N + N/8] (bits_jidx).
__device__ __forceinline__ void copy_couplings_skewed(float *smem, const float *gmem, int N)
{
    const int NJ = N + N / 8;
    for (int k = threadIdx.x; k < 3 * N; k += blockDim.x) {
        const int d = k / N, i = k - d * N;
        smem[d * NJ + bits_jidx(i)] = gmem[k];
    }
}


// ---------------------------------------------------------------------------
// The fused kernel: for each sample of this CTA, load, run n_sweeps sweeps
// (half-sweeps, energies, exchange, measurement), store.
// ---------------------------------------------------------------------------
// BITS: the packed state in shared memory, swept bit-parallel (+-J), or by
// chain sets of the bit-per-chain rows (Gaussian couplings).
template <int L, bool GST, bool WIDE, bool BITS>
struct Bounds {
    static constexpr int threads = BITS ? kBitsThreads : KernelBounds<L, GST, WIDE>::threads;
    static constexpr int min_blocks = BITS ? 2 : KernelBounds<L, GST, WIDE>::min_blocks;
};

template <int L, bool GAUSS, bool GST, bool WIDE = false, bool BITS = false>
__global__ void __launch_bounds__(Bounds<L, GST, WIDE, BITS>::threads,
                                  Bounds<L, GST, WIDE, BITS>::min_blocks)
    int8_run_kernel(const __grid_constant__ Int8Args a)
{
    constexpr int N = L * L * L;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Smem sm;
    carve(smem_raw, L, a.Tp, GAUSS, a.mchunk, &sm, GST, BITS);
    Ctx cx;
    cx.k0r = a.k0r;
    cx.nt = a.nt;
    cx.Tp = a.Tp;
    // global-memory instances and the bit-parallel ones keep the packed state
    constexpr bool PACK = GST || BITS;
    constexpr bool SKEW = BITS && GAUSS;  // skewed rows (bits_row)
    cx.WR = a.Tp / 4;
    cx.RB = PACK ? a.Tp / 4 : 2 * a.Tp;
    cx.seed_lo = a.seed_lo;
    cx.seed_hi = a.seed_hi;
    cx.hq = a.h_f;
    const long long t_start = clock64();

    // per-launch tables
    for (int k = threadIdx.x; k < a.Tp; k += blockDim.x) {
        sm.negbeta[k] = a.negbeta[k];
        sm.dbeta[k] = a.dbeta[k];
    }
    for (int k = threadIdx.x; k < 2 * L; k += blockDim.x) sm.twid[k] = a.twid[k];
    if (!GAUSS)
        for (int k = threadIdx.x; k < a.Tp * 16; k += blockDim.x) sm.thr[k] = a.thr[k];

    // units (segment, sample), segment-major: a plain launch (n_seg = 1) takes
    // samples blockIdx.x, + gridDim.x, ...; a segmented one claims units from
    // a counter, and a segment starts once the sample's previous one is
    // stored, so a sample's sweeps still run in order, one CTA at a time
    // (the host keeps n_seg * samples below 2^31)
    const int nS = (int)(a.s_end - a.s_begin);
    const bool segd = a.n_seg > 1;
    int &unit_sh = sm.ctl[0], &wait_fail = sm.ctl[1];
    if (threadIdx.x == 0) unit_sh = blockIdx.x;
    for (;;) {
        __syncthreads();  // every thread has read the previous unit
        if (threadIdx.x == 0 && segd) unit_sh = (int)atomicAdd(a.work, 1u);
        __syncthreads();
        const int unit = unit_sh;
        if (unit >= nS * a.n_seg) break;
        const int segk = unit / nS;
        const int64_t s = a.s_begin + (unit - segk * nS);
        const int seg_len = (a.n_sweeps + a.n_seg - 1) / a.n_seg;
        const int it_begin = segk * seg_len;
        const int n_it = min(seg_len, a.n_sweeps - it_begin);
        if (segk > 0) {
            if (threadIdx.x == 0) {
                int fail = 0;
                const volatile unsigned int *done = a.work + 1 + (s - a.s_begin);
                const unsigned long long limit = a.watchdog ? a.watchdog : a.seg_wait;
                const long long w0 = clock64();
                while (*done < (unsigned int)segk) {
                    if (*(const volatile int *)a.status != 0) {  // stopped elsewhere
                        fail = 1;
                        break;
                    }
                    if ((unsigned long long)(clock64() - w0) > limit) {
                        atomicCAS(a.status, 0, (int)SG_ETIMEOUT);
                        fail = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
                wait_fail = fail;
            }
            __syncthreads();
            if (wait_fail) break;
        }
        cx.s = s;
        cx.k1 = (uint32_t)((s + a.s_key0) / a.rng_group);
        __syncthreads();
        if (GST) {
            // large lattices: the CTA works on the sample's state in place
            sm.spins = a.spins + (size_t)s * N * cx.RB;
            if (!GAUSS)
                sm.J8 = const_cast<uint8_t *>(a.J8) + (size_t)s * N * 8;
            else
                sm.Jg = const_cast<float *>(a.Jg) + (size_t)s * 3 * N;
        } else if (SKEW) {
            if (segd)
                copy_rows_skewed<true, true>(sm.spins, a.spins + (size_t)s * N * cx.RB, N, cx.RB);
            else
                copy_rows_skewed<true, false>(sm.spins, a.spins + (size_t)s * N * cx.RB, N, cx.RB);
            copy_couplings_skewed(sm.Jg, a.Jg + (size_t)s * 3 * N, N);
        } else {
            if (segd)
                copy16_cg(sm.spins, a.spins + (size_t)s * N * cx.RB, (size_t)N * cx.RB);
            else
                copy16(sm.spins, a.spins + (size_t)s * N * cx.RB, (size_t)N * cx.RB);
            if (!GAUSS)
                copy16(sm.J8, a.J8 + (size_t)s * N * 8, (size_t)N * 8);
            else
                copy16(sm.Jg, a.Jg + (size_t)s * 3 * N, (size_t)3 * N * sizeof(float));
        }
        for (int k = threadIdx.x; k < 2 * a.Tp; k += blockDim.x) {
            sm.xflag[k] = 0;
            const int64_t *pb = a.B + s * 2 * a.Tp + k, *pm = a.M + s * 2 * a.Tp + k;
            sm.B[k] = (unsigned long long)(segd ? __ldcg((const long long *)pb) : *pb);
            sm.M[k] = (unsigned long long)(segd ? __ldcg((const long long *)pm) : *pm);
        }
        __syncthreads();

        uint32_t stamp = 0;
        bool stop = false;
        const int64_t sweep0 = (a.sweep0_dev ? *a.sweep0_dev : a.sweep0) + it_begin;
        for (int it = 0; it < n_it; ++it) {
            const int64_t n = sweep0 + it;
            if (a.watchdog || a.cancel) {  // launch-uniform branch
                int why = 0;
                if (threadIdx.x == 0) {
                    if (a.watchdog && (unsigned long long)(clock64() - t_start) > a.watchdog)
                        why = (int)SG_ETIMEOUT;
                    else if (a.cancel && *a.cancel)
                        why = (int)SG_ECANCELLED;
                    if (why) atomicCAS(a.status, 0, why);
                }
                stop = __syncthreads_or(why != 0);
                if (stop) break;
            }
            auto colour = [&](const int col) {
                if constexpr (BITS && GAUSS)
                    half_sweep_bits_gauss<L>(sm, cx, (uint32_t)n, col, a.csb);
                else if constexpr (BITS)
                    half_sweep_bits<L>(sm, cx, (uint32_t)n, col);
                else if constexpr (PACK)
                    half_sweep_packed<L, GAUSS>(sm, cx, (uint32_t)n, col);
                else
                    half_sweep<L, GAUSS>(sm, cx, (uint32_t)n, col);
                if (col == 0)  // the bit-parallel sweep subtracts from 3N and N
                    for (int k = threadIdx.x; k < 2 * a.Tp; k += blockDim.x) {
                        sm.B[k] = (BITS && !GAUSS) ? 3ull * N : 0ull;
                        sm.M[k] = BITS ? (unsigned long long)N : 0ull;
                    }
                __syncthreads();
            };
            // the Gaussian bit-per-chain sweep keeps one code path for both
            // colours (its unrolled chain bodies are large)
            if constexpr (BITS ? !GAUSS : unroll_colours<L, GAUSS, GST, WIDE>()) {
                colour(0);
                colour(1);
            } else {
#pragma unroll 1
                for (int col = 0; col < 2; ++col) colour(col);
            }
            if (a.exchange_every > 0 && (n + 1) % a.exchange_every == 0) {
                const int64_t e = (n + 1) / a.exchange_every - 1;
                ++stamp;
                if (threadIdx.x < 32) exchange_decide(sm, cx, a, (int)(e & 1), (uint32_t)n, 0u, stamp);
                __syncthreads();
                if constexpr (PACK)
                    exchange_apply_packed<L, SKEW>(sm, cx);
                else
                    exchange_apply<L>(sm, cx);
                __syncthreads();
            }
            if (n >= a.n_therm && (n - a.n_therm) % a.measure_every == 0)
                measure_step<L, PACK, SKEW>(sm, cx, a, log_bin(n, a.n_bins));
        }
        __syncthreads();
        if (SKEW)
            copy_rows_skewed<false, false>(sm.spins, a.spins + (size_t)s * N * cx.RB, N, cx.RB);
        else if (!GST)
            copy16(a.spins + (size_t)s * N * cx.RB, sm.spins, (size_t)N * cx.RB);
        for (int k = threadIdx.x; k < 2 * a.Tp; k += blockDim.x) {
            a.B[s * 2 * a.Tp + k] = (int64_t)sm.B[k];
            a.M[s * 2 * a.Tp + k] = (int64_t)sm.M[k];
        }
        // a stopped launch leaves later samples untouched; the status word tells
        if (__syncthreads_or(stop)) break;
        if (segd) {  // publish the stored segment (the barrier above ordered the stores)
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(a.work + 1 + (s - a.s_begin), 1u);
        } else if (threadIdx.x == 0) {
            unit_sh += gridDim.x;
        }
    }
}

constexpr int kMaxSmem = 227 * 1024;

// Raise the kernel's dynamic shared-memory limit once (before any capture).
template <int L, bool G, bool GST, bool WIDE = false, bool BITS = false>
cudaError_t ensure_attr()
{
    static cudaError_t done = cudaFuncSetAttribute(int8_run_kernel<L, G, GST, WIDE, BITS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   kMaxSmem);
    return done;
}

template <int L, bool G, bool GST, bool WIDE = false, bool BITS = false>
cudaError_t launch_t(const Int8Args &a, const Int8Launch &c, cudaStream_t st)
{
    cudaError_t e = ensure_attr<L, G, GST, WIDE, BITS>();
    if (e != cudaSuccess) return e;
    int8_run_kernel<L, G, GST, WIDE, BITS><<<c.grid, c.threads, c.smem, st>>>(a);
    return cudaGetLastError();
}

template <int L, bool G, bool GST, bool WIDE = false, bool BITS = false>
int occ_t(int threads, size_t smem)
{
    auto k = int8_run_kernel<L, G, GST, WIDE, BITS>;
    if (ensure_attr<L, G, GST, WIDE, BITS>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace
}  // namespace sg
