// sg_msc.cu -- multispin-coded +-J path of the EA spin-glass engine (sm_103a).
//
// Multispin coding (paper: methods section, where the replicas of one sample
// were packed into the bits of shared-memory words) is used here across
// disorder samples: bit b of a 64-bit word belongs to sample 64*g + b of word
// group g, so one logical operation updates 64 independent samples. The 64
// samples of a word share the Metropolis random word of each (site, chain,
// sweep) -- the RNG group G = 64 of the frozen random-number layout -- while
// every sample draws its own replica-exchange numbers; the path therefore
// reproduces, bit for bit, the int8 chain run with G = 64.
//
// Device layout (global memory):
//   W   [G][n_T][2][N] uint64   chain (t, r) of word group g; bit 1 => spin -1
//   Jw  [G][3][N] uint64        J[d][i] for the 64 samples; bit 1 => J = -1
//   B,M [S][2][n_T] int64       bond sum and magnetisation per sample and chain
// One launch is one sweep. Its CTAs each own one exchange unit -- a pair of
// neighbouring slots (p, p+1) of the sweep's exchange parity, or a single
// edge slot -- for both replicas, i.e. up to four chains in shared memory:
// both half-sweeps, the per-sample energies, the pair's exchange (a masked
// bit swap) and the overlap measurement of its slots all happen in one CTA.
#include <cuda_runtime.h>

#include "sg_device.cuh"
#include "sg_msc.h"

namespace sg {

namespace {

constexpr int kMscThreads = 512;
// Colour sites one thread visits in a half-sweep when its chain's team has
// at least tpc_min threads: the warps of a team take blocks of 128 colour
// sites (32 Philox groups of four) in turn, a lane one site per block step.
__host__ __device__ constexpr int msc_sites_per_thread(int L, int tpc_min)
{
    return 4 * ((((L * L * L / 8) + 31) / 32 + tpc_min / 32 - 1) / (tpc_min / 32));
}
// Bit planes that hold every count 0..x.
__host__ __device__ constexpr int msc_planes(int x) { return x < 2 ? 1 : 1 + msc_planes(x / 2); }
// Bit planes of a thread's unsatisfied-bond counter (at most 6 per site) and
// (-1)-spin counter (a colour-1 site and its colour-0 x-partner: at most 2
// per site): as few as the counts can reach, since every plane costs each
// site's ripple add and each half-sweep's warp reduction.
__host__ __device__ constexpr int msc_du(int L, int tpc_min)
{
    return msc_planes(6 * msc_sites_per_thread(L, tpc_min));
}
__host__ __device__ constexpr int msc_dm(int L, int tpc_min)
{
    return msc_planes(2 * msc_sites_per_thread(L, tpc_min));
}
static_assert(msc_du(2, 32) >= 5 && msc_dm(2, 32) >= 3, "the pairwise adds reach planes 4 and 2");
static_assert(msc_du(16, 32) == 9 && msc_dm(16, 32) == 8, "L = 16, teams of one warp");
static_assert(msc_du(16, 128) == 7 && msc_dm(16, 128) == 6, "L = 16, teams of four warps");
static_assert(msc_du(10, 32) == 7 && msc_dm(10, 32) == 6, "L = 10, teams of one warp");
// Bit planes of a projection count (0..L^2): the fewest with 2^planes > L^2,
// 9 at L = 16. Fewer planes make the carry chain of the projection sums
// shorter and let more phases share one warp transpose.
__host__ __device__ constexpr int msc_dp(int L)
{
    return L * L < 32 ? 5 : L * L < 64 ? 6 : L * L < 128 ? 7 : L * L < 256 ? 8 : 9;
}
constexpr int kDG = 5;  // bit planes of a 2D marginal entry (<= L <= 16 sites)
// Row stride, in 8-byte words, of the marginal array [3][L][L*kDG]. Padded
// (the measurement kernel) by one word where L * kDG words would put every
// row at the same bank offset (L = 8, 16): at L = 16 the marginal stores
// then take 2 wavefronts per warp instead of 16 and the projection loads 2
// instead of 3.6 on average.
__host__ __device__ constexpr int msc_marg_row(int L, bool pad)
{
    return L * kDG + ((pad && L % 8 == 0) ? 1 : 0);
}



// Add a one-bit carry word of weight 2^F into a bit-sliced counter's planes
// F .. D - 1 (64 lanes).
template <int D, int F>
__device__ __forceinline__ void bs_ripple(uint64_t (&c)[D], uint64_t carry)
{
#pragma unroll
    for (int k = F; k < D; ++k) {
        const uint64_t a = c[k];
        c[k] = a ^ carry;
        carry &= a;
    }
}

// Carry-save adder: three words in, their bitwise sum as (sum, carry).
__device__ __forceinline__ void csa(uint64_t &h, uint64_t &l, uint64_t a, uint64_t b, uint64_t c)
{
    const uint64_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// Bit-sliced population count of 16 words (bitwise, 64 lanes): a carry-save
// adder tree giving the five bit planes of the per-lane count 0..16.
__device__ __forceinline__ void count16(const uint64_t (&x)[16], uint64_t (&c)[5])
{
    uint64_t s1, c1, s2, c2, s3, c3, s4, c4, s5, c5;
    csa(c1, s1, x[0], x[1], x[2]);
    csa(c2, s2, x[3], x[4], x[5]);
    csa(c3, s3, x[6], x[7], x[8]);
    csa(c4, s4, x[9], x[10], x[11]);
    csa(c5, s5, x[12], x[13], x[14]);
    uint64_t s6, c6, s7, c7;
    csa(c6, s6, s1, s2, s3);
    csa(c7, s7, s4, s5, x[15]);
    c[0] = s6 ^ s7;
    const uint64_t c8 = s6 & s7;
    uint64_t t1, d1, t2, d2, t3, d3;  // weight 2: c1..c8
    csa(d1, t1, c1, c2, c3);
    csa(d2, t2, c4, c5, c6);
    csa(d3, t3, c7, c8, t1);
    c[1] = t2 ^ t3;
    const uint64_t d4 = t2 & t3;
    uint64_t f1, e1;  // weight 4: d1..d4
    csa(e1, f1, d1, d2, d3);
    c[2] = f1 ^ d4;
    const uint64_t e2 = f1 & d4;
    c[3] = e1 ^ e2;  // weight 8
    c[4] = e1 & e2;  // weight 16
}


// Small lattices keep the word group's couplings in shared memory too (loaded
// once per launch): the four chain teams of a unit read each bond word six
// times per sweep, which through L1 competed with the chain words.
__host__ __device__ constexpr bool msc_j_shared(int L) { return L <= 8; }

// A coupling word: a plain shared-memory load when the couplings are staged
// there, else a read-only global load.
template <int L>
__device__ __forceinline__ uint64_t ldJ(const uint64_t *p)
{
    if constexpr (msc_j_shared(L))
        return *p;
    else
        return __ldg(p);
}

struct MscSmem {
    uint64_t *w;        // [4][N]   chains: index q = 2*k + r (k = slot in unit)
    uint64_t *J;        // [3][N]   the word group's couplings (small L), else null
    uint32_t *thr;      // [2][16]  +-J thresholds of the unit's slots (sb*8 + u)
    long long *B, *M;   // [4][64]  per-sample energies of the unit's chains
    uint64_t *swap;     // [2]      exchange masks per replica
    uint64_t *marg;     // [ms][3][L][row] bit-sliced 2D marginal counts of q = -1 (msc_marg_row)
    uint64_t *proj;     // [ms][9][L][msc_dp(L)] bit-sliced projection counts of q = -1
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Whether the projections of a two-slot measurement live in the chains'
// space: the measuring CTA writes its chains back to global memory once the
// marginals are counted, so the projection phase can reuse that space. This
// keeps the L = 16 instance at 197 KB of shared memory, inside the 196 KB
// carveout that leaves L1 room for the couplings it reads through the
// cache (at 217 KB the sweeps ran 5 % slower).
__host__ __device__ constexpr bool msc_proj_in_w(int L, int ms)
{
    return ms == 2 && (size_t)2 * 9 * L * msc_dp(L) <= (size_t)4 * L * L * L;
}

// Slots whose overlap one measurement pass covers: both slots of the unit
// for the wide instance, and for the narrow one at L <= 8, where the extra
// shared memory leaves its CTAs per SM unchanged; one slot at a time else.
__host__ __device__ constexpr int msc_measured_slots(int L, bool wide)
{
    return (wide || L <= 8) ? 2 : 1;
}

// ms: slots whose overlap is measured in one pass (msc_measured_slots).
__host__ __device__ inline size_t msc_carve(uint8_t *base, int L, MscSmem *sm, int ms)
{
    const bool jshared = msc_j_shared(L);
    const size_t N = (size_t)L * L * L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = a16(off + bytes);
        return p;
    };
    MscSmem s;
    s.w = reinterpret_cast<uint64_t *>(take(4 * N * 8));
    s.J = jshared ? reinterpret_cast<uint64_t *>(take(3 * N * 8)) : nullptr;
    s.thr = reinterpret_cast<uint32_t *>(take(2 * 16 * 4));
    s.B = reinterpret_cast<long long *>(take(4 * 64 * 8));
    s.M = reinterpret_cast<long long *>(take(4 * 64 * 8));
    s.swap = reinterpret_cast<uint64_t *>(take(2 * 8));
    s.marg = reinterpret_cast<uint64_t *>(take((size_t)ms * 3 * L * L * kDG * 8));
    s.proj = msc_proj_in_w(L, ms) ? s.w
                                  : reinterpret_cast<uint64_t *>(take((size_t)ms * 9 * L * msc_dp(L) * 8));
    if (sm) *sm = s;
    return off;
}

// Exchange unit u of parity par: first slot and slot count (1 or 2).
__device__ __forceinline__ bool unit_slots(int u, int par, int nt, int *t0, int *cnt)
{
    if (par == 0) {
        *t0 = 2 * u;
    } else {
        if (u == 0) {
            *t0 = 0;
            *cnt = 1;
            return nt >= 1;
        }
        *t0 = 2 * u - 1;
    }
    if (*t0 >= nt) return false;
    *cnt = (*t0 + 1 < nt) ? 2 : 1;
    return true;
}

// u >= c for a bit-sliced 3-bit u and a scalar c in 0..7.
__device__ __forceinline__ uint64_t ge_const(uint64_t u0, uint64_t u1, uint64_t u2, int c)
{
    const uint64_t C0 = (c & 1) ? ~0ull : 0ull;
    const uint64_t C1 = (c & 2) ? ~0ull : 0ull;
    const uint64_t C2 = (c & 4) ? ~0ull : 0ull;
    const uint64_t a0 = ~u0 & C0;
    const uint64_t a1 = (~u1 & C1) | (~(u1 ^ C1) & a0);
    const uint64_t lt = (~u2 & C2) | (~(u2 ^ C2) & a1);
    return ~lt;
}

// Number of unsatisfied-bond classes whose threshold rejects r: since the
// threshold grows with u (the energy change falls), r <= thr[u] exactly for
// u >= ustar.
__device__ __forceinline__ int ustar_of(const uint32_t *thr_sb, uint32_t r)
{
    // thr_sb[0..6] does not decrease with u, so {u : r > thr_sb[u]} is the
    // prefix 0 .. ustar - 1, whose length three steps of a binary search find
    int c = r > thr_sb[3] ? 4 : 0;
    c += r > thr_sb[c + 1] ? 2 : 0;
    c += r > thr_sb[c] ? 1 : 0;
    return c;
}

// Site index and periodic neighbour indices of the colour-c site with
// colour-compressed index jj. For L a power of two the coordinates are bit
// fields of the index, and a neighbour is the index with one field stepped
// modulo L (an add and a masked merge); else boundary tests pick the
// wrap-around offsets.
template <int L>
struct MscSite {
    int i, x, ixp, ixm, iyp, iym, izp, izm;
    __device__ __forceinline__ MscSite(int jj, int c)
    {
        constexpr int H = L / 2;
        const int row = jj / H;
        const int x2 = jj - row * H;
        const int y = row % L;
        const int z = row / L;
        x = 2 * x2 + ((c + y + z) & 1);
        i = x + L * row;
        if constexpr ((L & (L - 1)) == 0) {
            constexpr int MX = L - 1, MY = (L - 1) * L, MZ = (L - 1) * L * L;
            ixp = (i & ~MX) | ((i + 1) & MX);
            ixm = (i & ~MX) | ((i - 1) & MX);
            iyp = (i & ~MY) | ((i + L) & MY);
            iym = (i & ~MY) | ((i - L) & MY);
            izp = (i & ~MZ) | ((i + L * L) & MZ);
            izm = (i & ~MZ) | ((i - L * L) & MZ);
        } else {
            ixp = i + ((x == L - 1) ? -(L - 1) : 1);
            ixm = i + ((x == 0) ? (L - 1) : -1);
            iyp = i + ((y == L - 1) ? -(L - 1) * L : L);
            iym = i + ((y == 0) ? (L - 1) * L : -L);
            izp = i + ((z == L - 1) ? -(L - 1) * L * L : L * L);
            izm = i + ((z == 0) ? (L - 1) * L * L : -L * L);
        }
    }
};

// ---------------------------------------------------------------------------
// Half-sweep of colour c for chain q (slot t, replica r) held in sm.w[q].
// Thread team: the threads with (threadIdx.x / tpc) == q, tpc threads per
// chain. For c == 1 the team also accumulates the per-sample unsatisfied-bond
// and (-1)-spin counts of the post-sweep configuration into sm.B / sm.M
// (raw counts; converted to B and M afterwards). CT >= 0 fixes the colour
// at compile time (the split sweep: each colour its own code path, colour 0
// without the energy bookkeeping and its branches; B300, L = 16, +3 %);
// CT = -1 takes it from c_rt (the fused kernel, whose narrow instance ran
// 7 % slower at L = 10 with a code path per colour).
// ---------------------------------------------------------------------------
// w: the chain's words; thr: its slot's 16 thresholds; bm: its row of
// sm.B / sm.M.
// TPC_MIN: a lower bound on tpc, which sizes the energy counters.
template <int L, int TPC_MIN, int CT>
__device__ __forceinline__ void msc_half(const MscSmem &sm, const MscArgs &a, int g, uint64_t *w,
                                         const uint32_t *thr, int bm, int t, int r, int tpc,
                                         int c_rt, uint32_t n_sweep)
{
    const int c = CT >= 0 ? CT : c_rt;
    constexpr int N = L * L * L;
    constexpr int NG = (N / 2) / 4;  // Philox groups of four colour-c sites
    constexpr int kDU = msc_du(L, TPC_MIN), kDM = msc_dm(L, TPC_MIN);
    constexpr bool kPairAdds = TPC_MIN >= 128;
    const int tid = threadIdx.x % tpc;
    const uint64_t *J = msc_j_shared(L) ? sm.J : a.Jw + (size_t)g * 3 * N;
    uint64_t cu[kDU], cm[kDM];
#pragma unroll
    for (int k = 0; k < kDU; ++k) cu[k] = 0;
#pragma unroll
    for (int k = 0; k < kDM; ++k) cm[k] = 0;
    const uint32_t c2 = ((uint32_t)c << 24) | ((uint32_t)r << 16) | (uint32_t)t;
    // A warp of the team takes blocks of 32 Philox groups (128 colour
    // sites): lane l draws the four random words of group 32 blk + l, then
    // the warp updates the block's sites in four steps of 32 consecutive
    // colour sites, each lane taking its site's word by a shuffle from the
    // lane that drew it. Consecutive lanes so read consecutive site words
    // (in shared memory, and the couplings through L1), where a lane per
    // group would put the lanes' words 8 sites apart, in two banks.
    constexpr int NB = (NG + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int blk = tid >> 5; blk < NB; blk += tpc >> 5) {
        const u32x4 rnd = philox10_rk(a.k0r, (uint32_t)(g + a.s_key0 / 64),
                                      (uint32_t)(32 * blk + lane), n_sweep, c2, a.seed_hi);
        // colour 1, teams of 128 threads or more (the split sweep): each
        // site's counts go into the low planes at once; their carry out
        // (weight 8 for u, 2 for the -1 spins) waits for the next site's, and
        // the pair's carries enter the planes above together (one full adder
        // and one ripple per two sites instead of two ripples: B300, L = 16,
        // 4096 samples, 2 x 32 T, 4589 -> 4739 attempts/ns thermalising,
        // 24 bytes of spills notwithstanding). The fused kernel's narrow
        // instance, which measured 1 % slower with it at L = 10, adds each
        // site's counts whole.
        uint64_t k8 = 0, k2m = 0;
        bool pend = false;
#pragma unroll
        for (int step = 0; step < 4; ++step) {
            const int src = 8 * step + (lane >> 2);
            const uint32_t w0 = __shfl_sync(0xFFFFFFFFu, rnd.v[0], src);
            const uint32_t w1 = __shfl_sync(0xFFFFFFFFu, rnd.v[1], src);
            const uint32_t w2 = __shfl_sync(0xFFFFFFFFu, rnd.v[2], src);
            const uint32_t w3 = __shfl_sync(0xFFFFFFFFu, rnd.v[3], src);
            const int jj = 128 * blk + 32 * step + lane;
            if constexpr ((N / 2) % 128 != 0)  // a colour of whole blocks has no tail
                if (jj >= N / 2) continue;
            const int k = lane & 3;  // the site's place in its group = its word
            const uint32_t rr = k == 0 ? w0 : k == 1 ? w1 : k == 2 ? w2 : w3;
            const MscSite<L> st(jj, c);
            const int i = st.i;
            const uint64_t s = w[i];
            const uint64_t n0 = w[st.ixp], n1 = w[st.ixm];
            const uint64_t n2 = w[st.iyp], n3 = w[st.iym];
            const uint64_t n4 = w[st.izp], n5 = w[st.izm];
            // unsatisfied bonds: s ^ s_nb ^ jbit
            const uint64_t d0 = s ^ n0 ^ ldJ<L>(J + i);
            const uint64_t d1 = s ^ n1 ^ ldJ<L>(J + st.ixm);
            const uint64_t d2 = s ^ n2 ^ ldJ<L>(J + N + i);
            const uint64_t d3 = s ^ n3 ^ ldJ<L>(J + N + st.iym);
            const uint64_t d4 = s ^ n4 ^ ldJ<L>(J + 2 * N + i);
            const uint64_t d5 = s ^ n5 ^ ldJ<L>(J + 2 * N + st.izm);
            // 3-bit count u of the six: two full adders and a carry merge
            const uint64_t sa = d0 ^ d1 ^ d2, ca = (d0 & d1) | (d2 & (d0 ^ d1));
            const uint64_t sb = d3 ^ d4 ^ d5, cb = (d3 & d4) | (d5 & (d3 ^ d4));
            const uint64_t u0 = sa ^ sb, cc = sa & sb;
            const uint64_t u1 = ca ^ cb ^ cc, u2 = (ca & cb) | (cc & (ca ^ cb));
            const uint64_t acc0 = ge_const(u0, u1, u2, ustar_of(thr, rr));      // s = +1
            const uint64_t acc1 = ge_const(u0, u1, u2, ustar_of(thr + 8, rr));  // s = -1
            const uint64_t f = (~s & acc0) | (s & acc1);
            const uint64_t sn = s ^ f;
            w[i] = sn;
            if (c == 1) {
                // u after the flip: 6 - u where flipped
                const uint64_t n1b = ~(u1 ^ u0);
                const uint64_t n2b = ~u2 & ~(u1 & u0);
                const uint64_t un1 = (u1 & ~f) | (n1b & f), un2 = (u2 & ~f) | (n2b & f);
                const uint64_t partner = (st.x & 1) ? n1 : n0;
                if constexpr (!kPairAdds) {
                    const uint64_t un[3] = {u0, un1, un2};
                    bs_add<kDU, 3>(cu, un);
                    const uint64_t mm[2] = {sn ^ partner, sn & partner};
                    bs_add<kDM, 2>(cm, mm);
                    continue;
                }
                uint64_t k = cu[0] & u0;  // u into planes 0-2: half, then full adders
                cu[0] ^= u0;
                uint64_t o = cu[1];
                cu[1] = o ^ un1 ^ k;
                k = (o & un1) | (k & (o ^ un1));
                o = cu[2];
                cu[2] = o ^ un2 ^ k;
                k = (o & un2) | (k & (o ^ un2));
                o = cm[0];  // the pair (site, x-partner) into plane 0
                cm[0] = o ^ sn ^ partner;
                const uint64_t km = (o & sn) | (partner & (o ^ sn));
                if ((step & 1) == 0) {
                    k8 = k;
                    k2m = km;
                    pend = true;
                } else {
                    o = cu[3];
                    cu[3] = o ^ k8 ^ k;
                    bs_ripple<kDU, 4>(cu, (o & k8) | (k & (o ^ k8)));
                    o = cm[1];
                    cm[1] = o ^ k2m ^ km;
                    bs_ripple<kDM, 2>(cm, (o & k2m) | (km & (o ^ k2m)));
                    pend = false;
                }
            }
        }
        if (kPairAdds && c == 1 && pend) {  // a block's last site without its pair
            bs_ripple<kDU, 3>(cu, k8);
            bs_ripple<kDM, 1>(cm, k2m);
        }
    }
    if (c == 1) {
        // per-sample warp totals by a bit-sliced butterfly (thread l ends with
        // samples b0 = 32 (l >> 4) + (l & 15) and b0 + 16 of the word)
        uint32_t u0, u1, m0, m1;
        warp_bs_totals<kDU>(cu, u0, u1);
        warp_bs_totals<kDM>(cm, m0, m1);
        const int b0 = 32 * (lane >> 4) + (lane & 15);
        atomicAdd((unsigned long long *)&sm.B[bm * 64 + b0], (unsigned long long)u0);
        atomicAdd((unsigned long long *)&sm.B[bm * 64 + b0 + 16], (unsigned long long)u1);
        atomicAdd((unsigned long long *)&sm.M[bm * 64 + b0], (unsigned long long)m0);
        atomicAdd((unsigned long long *)&sm.M[bm * 64 + b0 + 16], (unsigned long long)m1);
    }
}

// ---------------------------------------------------------------------------
// Overlap measurement of slot k of the unit for the 64 samples (eq. overlap):
// bit-sliced 2D marginals, bit-sliced projections, then per sample the
// integer projections, the FP32 DFT and the FP64 accumulation.
// ---------------------------------------------------------------------------
// QW: sm.w holds the slots' overlap words q = w(r=0) ^ w(r=1) themselves (N
// words per slot) rather than the two replica chains (the measurement
// kernel), and each projection sum is split over two lanes.
template <int L, bool WIDE, bool QW = false>
__device__ __forceinline__ void msc_measure(const MscSmem &sm, const MscArgs &a, int g, int k0,
                                            int nk, int t0, int bin, uint64_t *w_dst, int nw)
{
    constexpr int N = L * L * L;
    constexpr int LL = L * L;
    constexpr int ROW = msc_marg_row(L, QW);
    // the unit's slots k0 .. k0 + nk - 1 (temperatures t0 ..) in one pass: one
    // barrier per phase for all of them, and more independent tasks per phase.
    // The wide instance unrolls the serial loops of (B) and (C) so their
    // independent steps overlap (B300, +-J, 2 x 32 T, 4096 samples: L = 16
    // 1988 -> 2134 attempts/ns with the one-pass slots); the narrow
    // 80-register instance keeps the compiler's choice, which measured faster.
    // (A) marginal counts of q = -1 (bit set) over the summed axis
    for (int id = threadIdx.x; id < nk * 3 * LL; id += blockDim.x) {
        const int kk = id / (3 * LL), pid = id - kk * (3 * LL);
        const uint64_t *w0 = sm.w + (size_t)((QW ? 1 : 2) * (k0 + kk)) * N;
        const uint64_t *w1 = w0 + N;
        uint64_t *margk = sm.marg + (size_t)kk * 3 * L * ROW;
        const int plane = pid / LL, ab = pid % LL;
        const int A = ab % L, Bc = ab / L;  // consecutive lanes: consecutive A
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
        // along x (plane 2) lanes would hit one bank: each lane starts the
        // (order-free) column sum at its own offset
        const int rot = plane == 2 ? (threadIdx.x % L) : 0;
        uint64_t qs[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            int mm = m + rot;
            if (mm >= L) mm -= L;
            const int i = base + mm * step;
            qs[m] = m < L ? (QW ? w0[i] : (w0[i] ^ w1[i])) : 0ull;
        }
        uint64_t cnt[kDG];
        count16(qs, cnt);
#pragma unroll
        for (int p = 0; p < kDG; ++p) margk[((size_t)plane * L + A) * ROW + Bc * kDG + p] = cnt[p];
    }
    __syncthreads();
    // (with QW the projections may take the overlap words' space: the
    // barrier above ends every read of them)
    if constexpr (!QW && msc_proj_in_w(L, msc_measured_slots(L, WIDE))) {
        // the chains are final: store them now (unless they are stored
        // already), their space takes the projections
        if (w_dst)
            for (int k = threadIdx.x; k < nw; k += blockDim.x) w_dst[k] = sm.w[k];
        __syncthreads();
    }
    // (B) projection counts: sum of L marginal entries per (v, d)
    constexpr int DP = msc_dp(L);
    if constexpr (QW) {
        // the measurement kernel: two lanes per (v, d), each adding half of
        // the entries, the halves joined by a shuffle (half the serial adds)
        static_assert(L % 2 == 0, "even L");
        const int items = nk * 9 * L * 2;
        for (int base = 0; base < items; base += blockDim.x) {  // whole warps per pass
            const int id2 = base + (int)threadIdx.x, id = id2 >> 1, hf = id2 & 1;
            const bool valid = id2 < items;
            uint64_t acc[DP];
#pragma unroll
            for (int p = 0; p < DP; ++p) acc[p] = 0;
            if (valid) {
                const int kk = id / (9 * L), pid = id - kk * (9 * L);
                const uint64_t *margk = sm.marg + (size_t)kk * 3 * L * ROW;
                const int v = pid / L, d = pid % L;
                const int plane = (v == 0 || v == 1 || v == 3 || v == 4) ? 0 : (v == 2 || v == 5 || v == 6) ? 1 : 2;
#pragma unroll
                for (int e = 0; e < L / 2; ++e) {
                    const int aa = hf * (L / 2) + e;
                    int A, Bc;
                    if (v == 0) {
                        A = d; Bc = aa;
                    } else if (v == 1 || v == 2) {
                        A = aa; Bc = d;
                    } else if (v == 3 || v == 5 || v == 7) {
                        A = aa; Bc = (d - aa + L) % L;
                    } else {
                        A = aa; Bc = (aa - d + L) % L;
                    }
                    const uint64_t *m = margk + ((size_t)plane * L + A) * ROW + Bc * kDG;
                    const uint64_t x[kDG] = {m[0], m[1], m[2], m[3], m[4]};
                    bs_add<DP, kDG>(acc, x);
                }
            }
            uint64_t oth[DP];
#pragma unroll
            for (int p = 0; p < DP; ++p) oth[p] = __shfl_xor_sync(0xFFFFFFFFu, acc[p], 1);
            if (valid && hf == 0) {
                bs_add<DP, DP>(acc, oth);
#pragma unroll
                for (int p = 0; p < DP; ++p) sm.proj[(size_t)id * DP + p] = acc[p];  // [kk][v][d]
            }
        }
    } else
    for (int id = threadIdx.x; id < nk * 9 * L; id += blockDim.x) {
        const int kk = id / (9 * L), pid = id - kk * (9 * L);
        const uint64_t *margk = sm.marg + (size_t)kk * 3 * L * ROW;
        const int v = pid / L, d = pid % L;
        const int plane = (v == 0 || v == 1 || v == 3 || v == 4) ? 0 : (v == 2 || v == 5 || v == 6) ? 1 : 2;
        uint64_t acc[DP];
#pragma unroll
        for (int p = 0; p < DP; ++p) acc[p] = 0;
        auto add_entry = [&](int aa) {
            int A, Bc;
            if (v == 0) {
                A = d; Bc = aa;
            } else if (v == 1 || v == 2) {
                A = aa; Bc = d;
            } else if (v == 3 || v == 5 || v == 7) {
                A = aa; Bc = (d - aa + L) % L;
            } else {
                A = aa; Bc = (aa - d + L) % L;
            }
            const uint64_t *m = margk + ((size_t)plane * L + A) * ROW + Bc * kDG;
            const uint64_t x[kDG] = {m[0], m[1], m[2], m[3], m[4]};
            bs_add<DP, kDG>(acc, x);
        };
        if constexpr (WIDE) {
#pragma unroll
            for (int aa = 0; aa < L; ++aa) add_entry(aa);
        } else {
            for (int aa = 0; aa < L; ++aa) add_entry(aa);
        }
#pragma unroll
        for (int p = 0; p < DP; ++p) sm.proj[(size_t)id * DP + p] = acc[p];  // [kk][v][d]
    }
    __syncthreads();
    // (C) one warp per (wave vector v, half of the word): lanes j*DP + p load
    // plane p of P_v[d0 + j] for the G = 32 / DP phases of a group, and one
    // bit transpose hands lane b the G counts of sample 32*half + b, packed
    // DP bits each; the lane then runs the FP32 DFT over d in ascending
    // order and the FP64 accumulation. The v = 0 tasks also produce Q and its
    // moments, and the v = 8 tasks (the other round of the task loop, other
    // warps) add E and M straight from the per-sample energies, so no warp
    // carries both extra parts.
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        constexpr int G = 32 / DP;
        const int lj = lane / DP, lp = lane - lj * DP;
        for (int task = warp; task < nk * 2 * 9; task += nwarps) {
            const int kk = task / 18, v = (task % 18) >> 1, half = task & 1;
            const int k = k0 + kk, t = t0 + kk;
            const int b = 32 * half + lane;  // sample 64 g + b
            // device layout [G][nt][bins][40][64]: entry k of this sample at
            // ac[64 k], so the 32 lanes of a warp touch 256 contiguous bytes
            double *ac = a.acc + (((size_t)g * a.nt + t) * a.n_bins + bin) * SG_NACC * 64 + b;
            double *acv = ac + 64 * (9 + 3 * v);
            double o0 = acv[0], o1 = acv[64], o2 = acv[128];
            double q[9];
            if (v == 0) {
#pragma unroll
                for (int k2 = 0; k2 < 5; ++k2) q[k2] = ac[64 * k2];
            } else if (v == 8) {
#pragma unroll
                for (int k2 = 5; k2 < 9; ++k2) q[k2] = ac[64 * k2];
            }
            float re = 0.0f, im = 0.0f;
            int Qi = 0;
            const uint64_t *pv = sm.proj + ((size_t)kk * 9 + v) * L * DP;
            auto add_group = [&](int d0) {
                const int dl = d0 + lj;
                const uint32_t row = (lj < G && dl < L) ? (uint32_t)(pv[dl * DP + lp] >> (32 * half)) : 0u;
                const uint32_t cnts = warp_transpose32(row);
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int d = d0 + j;
                    if (d < L) {
                        const int P = LL - 2 * (int)((cnts >> (j * DP)) & ((1u << DP) - 1));
                        Qi += P;
                        re = __fmaf_rn((float)P, a.twid[d], re);
                        im = __fmaf_rn((float)P, a.twid[L + d], im);
                    }
                }
            };
            if constexpr (WIDE) {
#pragma unroll
                for (int d0 = 0; d0 < L; d0 += G) add_group(d0);
            } else {
                for (int d0 = 0; d0 < L; d0 += G) add_group(d0);
            }
            // (the exact conversions and squares from integer operations)
            acv[0] = __dadd_rn(o0, f64_of_f32(re));
            acv[64] = __dadd_rn(o1, f64_of_f32(im));
            acv[128] = __dadd_rn(o2, __dadd_rn(f64_sq_of_f32(re), f64_sq_of_f32(im)));
            if (v == 0) {
                if (a.hist)  // P(q): replicas agree on (N + Q) / 2 sites
                    atomicAdd(a.hist + ((size_t)t * a.n_bins + bin) * (N + 1) + ((N + Qi) >> 1), 1ull);
                // |Q| <= N <= 4096: Q^2, Q^3 = Q^2 Q and Q^4 = Q^2 Q^2 are
                // integers below 2^53, as exact as their FP64 products
                const long long Q1 = Qi, Q2 = Q1 * Q1;
                q[0] = __dadd_rn(q[0], 1.0);
                q[1] = __dadd_rn(q[1], f64_of_i64(Q1));
                q[2] = __dadd_rn(q[2], f64_of_i64(Q2));
                q[3] = __dadd_rn(q[3], f64_of_i64(Q2 * Q1));
                q[4] = __dadd_rn(q[4], f64_of_i64(Q2 * Q2));
#pragma unroll
                for (int k2 = 0; k2 < 5; ++k2) ac[64 * k2] = q[k2];
            } else if (v == 8) {
                for (int r = 0; r < 2; ++r) {
                    const long long Bv = sm.B[(2 * k + r) * 64 + b];
                    const long long Mv = sm.M[(2 * k + r) * 64 + b];
                    const double e = -__dadd_rn(f64_of_i64(Bv), __dmul_rn(a.h_d, f64_of_i64(Mv)));
                    q[5] = __dadd_rn(q[5], e);
                    q[6] = __dadd_rn(q[6], __dmul_rn(e, e));
                }
                for (int r = 0; r < 2; ++r) {
                    const long long Mv = sm.M[(2 * k + r) * 64 + b];  // |M| <= N: M^2 exact
                    q[7] = __dadd_rn(q[7], f64_of_i64(Mv));
                    q[8] = __dadd_rn(q[8], f64_of_i64(Mv * Mv));
                }
#pragma unroll
                for (int k2 = 5; k2 < 9; ++k2) ac[64 * k2] = q[k2];
            }
        }
    }
    __syncthreads();
}

// MAXT / MINB: launch bounds of the instance. The narrow instance (128
// threads, at least 6 CTAs per SM, so at most 80 registers) serves small
// lattices, where a unit has little work per barrier and several resident
// CTAs hide each other's barrier and memory waits; the wide one (up to 512
// threads) serves large lattices.
template <int L, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) msc_sweep_kernel(const MscArgs a)
{
    constexpr int N = L * L * L;
    extern __shared__ __align__(16) uint8_t msc_smem[];
    constexpr bool WIDE = MAXT == kMscThreads;
    constexpr int MS = msc_measured_slots(L, WIDE);
    MscSmem sm;
    msc_carve(msc_smem, L, &sm, MS);
    const int g = blockIdx.y;
    const int64_t n = (a.sweep0_dev ? *a.sweep0_dev : a.sweep0) + a.sweep_offset;
    const bool xchg = a.exchange_every > 0 && (n + 1) % a.exchange_every == 0;
    const int par = xchg ? (int)(((n + 1) / a.exchange_every - 1) & 1) : 0;
    int t0, cnt;
    if (!unit_slots(blockIdx.x, par, a.nt, &t0, &cnt)) return;
    const bool meas = n >= a.n_therm && (n - a.n_therm) % a.measure_every == 0;
    const int nq = 2 * cnt;

    // the unit's chains (index q = 2k + r is contiguous in W) and, for small
    // lattices, the word group's couplings by bulk copies (sizes multiples of
    // 16 bytes for even L) while the threads set up the tables
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, (uint32_t)((nq + (msc_j_shared(L) ? 3 : 0)) * N * 8));
        bulk_load(sm.w, a.W + ((size_t)g * a.nt + t0) * 2 * N, (uint32_t)(nq * N * 8), &bar);
        if (msc_j_shared(L)) bulk_load(sm.J, a.Jw + (size_t)g * 3 * N, (uint32_t)(3 * N * 8), &bar);
    }
    for (int k = threadIdx.x; k < cnt * 16; k += blockDim.x) sm.thr[k] = a.thr[t0 * 16 + k];
    for (int k = threadIdx.x; k < 4 * 64; k += blockDim.x) {
        sm.B[k] = 0;
        sm.M[k] = 0;
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait(&bar, 0, kBulkWaitCycles))) {
        if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)SG_ETIMEOUT);
        mbar_wait(&bar, 0, kBulkWaitCycles);  // the copies still in flight, bounded again
        return;
    }

    const int tpc = blockDim.x / nq;  // threads per chain
    const int q = threadIdx.x / tpc;
    for (int c = 0; c < 2; ++c) {
        if (q < nq)
            // (at least 128 threads for at most four chains)
            msc_half<L, 32, -1>(sm, a, g, sm.w + (size_t)q * N, sm.thr + (q >> 1) * 16, q,
                                t0 + (q >> 1), q & 1, tpc, c, (uint32_t)n);
        __syncthreads();
    }
    // raw counts -> B = 3N - 2 * (unsatisfied bonds), M = N - 2 * (#-1 spins)
    for (int k = threadIdx.x; k < nq * 64; k += blockDim.x) {
        sm.B[k] = 3LL * N - 2 * sm.B[k];
        sm.M[k] = (long long)N - 2 * sm.M[k];
    }
    if (threadIdx.x < 2) sm.swap[threadIdx.x] = 0;
    __syncthreads();

    if (xchg && cnt == 2) {
        // one thread per (replica, sample): Metropolis on the pair (t0, t0+1)
        if (threadIdx.x < 128) {
            const int r = threadIdx.x >> 6, b = threadIdx.x & 63;
            const int64_t s = 64 * (int64_t)g + b;
            const long long dB = sm.B[(0 + r) * 64 + b] - sm.B[(2 + r) * 64 + b];
            const long long dM = sm.M[(0 + r) * 64 + b] - sm.M[(2 + r) * 64 + b];
            const float t1 = __fmul_rn(__ll2float_rn(dB), 1.0f);
            const float t2 = __fmul_rn(a.h_f, __ll2float_rn(dM));
            const float dE = -__fadd_rn(t1, t2);
            const float D = __fmul_rn(a.dbeta[t0], dE);
            const u32x4 o = philox10(a.seed_lo ^ kTagExc, (uint32_t)(s + a.s_key0), (uint32_t)t0, (uint32_t)n,
                                     (uint32_t)r, a.seed_hi);
            const bool acc = (D >= 0.0f) || (o.v[0] <= thr_of_logp(D));
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, acc);
            if ((threadIdx.x & 31) == 0)
                atomicOr((unsigned long long *)&sm.swap[r],
                         (unsigned long long)bal << (threadIdx.x & 32));
            if (acc) {
                const long long tb = sm.B[r * 64 + b];
                sm.B[r * 64 + b] = sm.B[(2 + r) * 64 + b];
                sm.B[(2 + r) * 64 + b] = tb;
                const long long tm = sm.M[r * 64 + b];
                sm.M[r * 64 + b] = sm.M[(2 + r) * 64 + b];
                sm.M[(2 + r) * 64 + b] = tm;
            }
        }
        __syncthreads();
        for (int id = threadIdx.x; id < 2 * N; id += blockDim.x) {
            const int r = id / N, i = id % N;
            const uint64_t m = sm.swap[r];
            if (!m) continue;
            uint64_t *pa = sm.w + (size_t)r * N + i;         // slot t0
            uint64_t *pb = sm.w + (size_t)(2 + r) * N + i;   // slot t0 + 1
            const uint64_t x = (*pa ^ *pb) & m;
            *pa ^= x;
            *pb ^= x;
        }
        __syncthreads();
    }
    uint64_t *dst = a.W + ((size_t)g * a.nt + t0) * 2 * N;
    if (meas) {
        if constexpr (MS == 2)
            msc_measure<L, WIDE>(sm, a, g, 0, cnt, t0, log_bin(n, a.n_bins), dst, nq * N);
        else
            for (int k = 0; k < cnt; ++k)
                msc_measure<L, WIDE>(sm, a, g, k, 1, t0 + k, log_bin(n, a.n_bins), dst, nq * N);
    }
    // (a measuring two-slot instance whose projections reuse the chains'
    // space has stored the chains already)
    if (!(meas && msc_proj_in_w(L, MS)))
        for (int k = threadIdx.x; k < nq * N; k += blockDim.x) dst[k] = sm.w[k];
    for (int k = threadIdx.x; k < nq * 64; k += blockDim.x) {
        const int qq = k / 64, b = k % 64;
        const int64_t s = 64 * (int64_t)g + b;
        const size_t o = ((size_t)s * 2 + (qq & 1)) * a.nt + t0 + (qq >> 1);
        a.B[o] = sm.B[k];
        a.M[o] = sm.M[k];
    }
}

// ---------------------------------------------------------------------------
// Sweeps of large lattices (L >= 12): the exchange unit split by replica. A
// CTA holds one replica's chains of the unit (the sweep and the exchange
// never mix replicas: methods section, each replica has its own tempering
// ladder), so at L = 16 it needs 64 KB of shared memory instead of 197 KB and
// three CTAs share an SM. It does not measure (the overlap needs both
// replicas): a measured sweep is followed by msc_measure_kernel, which reads
// the stored chains. Same random numbers, decisions and order as
// msc_sweep_kernel: the results are identical. (B300, +-J, 4096 samples,
// 2 x 32 temperatures, attempts/ns, fused -> split: thermalising L = 14
// 2436 -> 2886, L = 16 2969 -> 3117 when first built; with the consecutive-
// site lanes L = 16 3641 split, measuring every sweep 2338 fused -> 2665
// split plus the measurement kernel. At L = 12 the fused 256-thread CTA was
// ahead then (measuring 2234 against 1975 split); with the bulk copies,
// smaller energy counters and padded marginals the split path leads there
// too, measuring 2613 against 2541 fused, thermalising 3664 against 3626,
// while at L = 10 the fused narrow CTAs stay ahead (2 x 56 T, 8192 samples:
// measuring 2510 fused against 2272 split). The replica pair run as a
// cluster, each CTA measuring one slot through the peer's shared memory,
// measured slower than both.)
// ---------------------------------------------------------------------------
constexpr int kMscSplitThreads = 256;

// Whether sweep n walks the word groups from the last: the opposite of
// sweep n - 1 when that one was not measured (in the thermalisation by the
// parity of n), forward after a measured sweep, whose measurement ended on
// the first groups. The order changes no result, only which chains are
// still in L2 when they are read.
__device__ __forceinline__ bool msc_groups_reversed(const MscArgs &a, int64_t n)
{
    if (n - 1 < a.n_therm) return (n & 1) != 0;
    const int64_t m = a.n_therm + a.measure_every * ((n - 1 - a.n_therm) / a.measure_every);
    return ((n - m) & 1) == 0;  // n = m + 1 forward, then alternating
}

__host__ __device__ inline size_t msc_carve_split(uint8_t *base, int L, MscSmem *sm)
{
    const size_t N = (size_t)L * L * L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = a16(off + bytes);
        return p;
    };
    MscSmem s{};
    s.w = reinterpret_cast<uint64_t *>(take(2 * N * 8));
    s.J = nullptr;  // L >= 12: the couplings are read through L1
    s.thr = reinterpret_cast<uint32_t *>(take(2 * 16 * 4));
    s.B = reinterpret_cast<long long *>(take(2 * 64 * 8));
    s.M = reinterpret_cast<long long *>(take(2 * 64 * 8));
    s.swap = reinterpret_cast<uint64_t *>(take(2 * 8));
    if (sm) *sm = s;
    return off;
}

template <int L>
__global__ void __launch_bounds__(kMscSplitThreads, 3) msc_split_sweep_kernel(const MscArgs a)
{
    static_assert(!msc_j_shared(L), "the split kernel reads the couplings through L1");
    constexpr int N = L * L * L;
    extern __shared__ __align__(16) uint8_t msc_smem[];
    MscSmem sm;
    msc_carve_split(msc_smem, L, &sm);
    // word groups outermost (both replicas of a group's units together), so
    // the chains written last are whole groups, which the next reader takes
    // first: the measurement walks the groups in reverse, and a sweep after an
    // unmeasured one walks them opposite to it
    const int64_t n = (a.sweep0_dev ? *a.sweep0_dev : a.sweep0) + a.sweep_offset;
    const int r = blockIdx.y;
    const int g = msc_groups_reversed(a, n) ? (int)(a.G - 1) - (int)blockIdx.z : (int)blockIdx.z;
    const bool xchg = a.exchange_every > 0 && (n + 1) % a.exchange_every == 0;
    const int par = xchg ? (int)(((n + 1) / a.exchange_every - 1) & 1) : 0;
    int t0, cnt;
    if (!unit_slots(blockIdx.x, par, a.nt, &t0, &cnt)) return;

    // chain k of this CTA: slot t0 + k of replica r, brought in by bulk
    // copies (N * 8 bytes each: a multiple of 16 for even L) while the
    // threads set up the rest
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, (uint32_t)(cnt * N * 8));
        for (int k = 0; k < cnt; ++k)
            bulk_load(sm.w + (size_t)k * N, a.W + (((size_t)g * a.nt + t0 + k) * 2 + r) * N,
                      (uint32_t)(N * 8), &bar);
    }
    for (int k = threadIdx.x; k < cnt * 16; k += blockDim.x) sm.thr[k] = a.thr[t0 * 16 + k];
    for (int k = threadIdx.x; k < 2 * 64; k += blockDim.x) {
        sm.B[k] = 0;
        sm.M[k] = 0;
    }
    if (threadIdx.x == 0) sm.swap[0] = 0;
    __syncthreads();
    if (__syncthreads_or(!mbar_wait(&bar, 0, kBulkWaitCycles))) {
        if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)SG_ETIMEOUT);
        mbar_wait(&bar, 0, kBulkWaitCycles);  // the copies still in flight, bounded again
        return;
    }

    const int tpc = blockDim.x / cnt;  // threads per chain: whole warps
    const int k = threadIdx.x / tpc;
    if (k < cnt)
        msc_half<L, kMscSplitThreads / 2, 0>(sm, a, g, sm.w + (size_t)k * N, sm.thr + k * 16, k,
                                             t0 + k, r, tpc, 0, (uint32_t)n);
    __syncthreads();
    if (k < cnt)
        msc_half<L, kMscSplitThreads / 2, 1>(sm, a, g, sm.w + (size_t)k * N, sm.thr + k * 16, k,
                                             t0 + k, r, tpc, 1, (uint32_t)n);
    __syncthreads();
    // raw counts -> B = 3N - 2 * (unsatisfied bonds), M = N - 2 * (#-1 spins)
    for (int q = threadIdx.x; q < cnt * 64; q += blockDim.x) {
        sm.B[q] = 3LL * N - 2 * sm.B[q];
        sm.M[q] = (long long)N - 2 * sm.M[q];
    }
    __syncthreads();

    if (xchg && cnt == 2) {
        // one thread per sample: Metropolis on the pair (t0, t0 + 1) of replica r
        if (threadIdx.x < 64) {
            const int b = threadIdx.x;
            const int64_t s = 64 * (int64_t)g + b;
            const long long dB = sm.B[b] - sm.B[64 + b];
            const long long dM = sm.M[b] - sm.M[64 + b];
            const float t1 = __fmul_rn(__ll2float_rn(dB), 1.0f);
            const float t2 = __fmul_rn(a.h_f, __ll2float_rn(dM));
            const float dE = -__fadd_rn(t1, t2);
            const float D = __fmul_rn(a.dbeta[t0], dE);
            const u32x4 o = philox10(a.seed_lo ^ kTagExc, (uint32_t)(s + a.s_key0), (uint32_t)t0,
                                     (uint32_t)n, (uint32_t)r, a.seed_hi);
            const bool acc = (D >= 0.0f) || (o.v[0] <= thr_of_logp(D));
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, acc);
            if ((threadIdx.x & 31) == 0)
                atomicOr((unsigned long long *)&sm.swap[0], (unsigned long long)bal << (threadIdx.x & 32));
            if (acc) {
                const long long tb = sm.B[b];
                sm.B[b] = sm.B[64 + b];
                sm.B[64 + b] = tb;
                const long long tm = sm.M[b];
                sm.M[b] = sm.M[64 + b];
                sm.M[64 + b] = tm;
            }
        }
        __syncthreads();
        const uint64_t m = sm.swap[0];
        if (m)
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const uint64_t x = (sm.w[i] ^ sm.w[N + i]) & m;
                sm.w[i] ^= x;
                sm.w[N + i] ^= x;
            }
        __syncthreads();
    }
    for (int kk = 0; kk < cnt; ++kk) {
        uint64_t *dst = a.W + (((size_t)g * a.nt + t0 + kk) * 2 + r) * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = sm.w[(size_t)kk * N + i];
    }
    for (int q = threadIdx.x; q < cnt * 64; q += blockDim.x) {
        const int kk = q / 64, b = q % 64;
        const int64_t s = 64 * (int64_t)g + b;
        const size_t o = ((size_t)s * 2 + r) * a.nt + t0 + kk;
        a.B[o] = sm.B[q];
        a.M[o] = sm.M[q];
    }
}

// ---------------------------------------------------------------------------
// Overlap measurement after a split sweep (L >= 12): one CTA per (slot t,
// word group g) reads the slot's two replica chains as stored by
// msc_split_sweep_kernel (after the sweep and the exchange), keeps their
// overlap words q = w(r=0) ^ w(r=1) in shared memory, and runs the three
// phases of msc_measure for that slot, with the energies from B and M as
// stored. The counts, their order and every rounding are those of the fused
// kernel's measurement, so the accumulators are identical. The CTA needs
// the overlap words, the marginals and the energies (about 66 KB at L = 16,
// the projections taking the words' space), so three share an SM and
// overlap one another's phases, where the fused kernel measured inside its
// one 197 KB CTA per SM. Its 9 warps take the 18 DFT tasks of a slot in two
// even rounds, and its projection sums run on two lanes each (the QW form
// of msc_measure). A sweep that is not measured returns at once.
// ---------------------------------------------------------------------------
constexpr int kMscMeasThreads = 288;

__host__ __device__ inline size_t msc_carve_meas(uint8_t *base, int L, MscSmem *sm)
{
    const size_t N = (size_t)L * L * L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off = a16(off + bytes);
        return p;
    };
    MscSmem s{};
    s.w = reinterpret_cast<uint64_t *>(take(N * 8));
    s.B = reinterpret_cast<long long *>(take(2 * 64 * 8));
    s.M = reinterpret_cast<long long *>(take(2 * 64 * 8));
    // the marginals' space first receives replica 1's chain
    const size_t marg = (size_t)3 * L * msc_marg_row(L, true) * 8;
    s.marg = reinterpret_cast<uint64_t *>(take(marg > N * 8 ? marg : N * 8));
    s.proj = s.w;  // [9][L][msc_dp(L)] after the marginals, in the overlap words' space
    if (sm) *sm = s;
    return off;
}

template <int L>
__global__ void __launch_bounds__(kMscMeasThreads, 3) msc_measure_kernel(const MscArgs a)
{
    static_assert((size_t)9 * L * msc_dp(L) <= (size_t)L * L * L, "projections fit the words' space");
    constexpr int N = L * L * L;
    extern __shared__ __align__(16) uint8_t msc_smem[];
    MscSmem sm;
    msc_carve_meas(msc_smem, L, &sm);
    // the word groups in reverse of the sweep's order: the chains stored
    // last by the sweep, still in L2, are read first, and the next sweep
    // starts on the groups read last
    const int t = blockIdx.x, g = (int)(a.G - 1) - (int)blockIdx.y;
    const int64_t n = (a.sweep0_dev ? *a.sweep0_dev : a.sweep0) + a.sweep_offset;
    if (!(n >= a.n_therm && (n - a.n_therm) % a.measure_every == 0)) return;
    const int bin = log_bin(n, a.n_bins);
    // the two chains by bulk copies (replica 0 into the words' space, replica
    // 1 into the marginals'), and this (slot, word group, bin)'s accumulator
    // block on its way to L2 for the last phase
    const uint64_t *w0 = a.W + (((size_t)g * a.nt + t) * 2) * N;
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_expect_tx(&bar, (uint32_t)(2 * N * 8));
        bulk_load(sm.w, w0, (uint32_t)(N * 8), &bar);
        bulk_load(sm.marg, w0 + N, (uint32_t)(N * 8), &bar);
        bulk_prefetch_l2(a.acc + (((size_t)g * a.nt + t) * a.n_bins + bin) * SG_NACC * 64,
                         (uint32_t)(SG_NACC * 64 * sizeof(double)));
    }
    for (int q = threadIdx.x; q < 2 * 64; q += blockDim.x) {
        const int r = q / 64, b = q % 64;
        const int64_t s = 64 * (int64_t)g + b;
        const size_t o = ((size_t)s * 2 + r) * a.nt + t;
        sm.B[q] = a.B[o];
        sm.M[q] = a.M[o];
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait(&bar, 0, kBulkWaitCycles))) {
        if (threadIdx.x == 0) atomicCAS(a.status, 0, (int)SG_ETIMEOUT);
        mbar_wait(&bar, 0, kBulkWaitCycles);  // the copies still in flight, bounded again
        return;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm.w[i] ^= sm.marg[i];
    __syncthreads();
    msc_measure<L, true, true>(sm, a, g, 0, 1, t, bin, nullptr, 0);
}

// ---- conversion, generation and standalone kernels ------------------------

__device__ __forceinline__ int nb_site(int L, int i, int d, int step)
{
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    if (d == 0) x = (x + step + L) % L;
    if (d == 1) y = (y + step + L) % L;
    if (d == 2) z = (z + step + L) % L;
    return x + L * (y + L * z);
}

// Accumulators: canonical [S][nt][bins][40] <-> device [G][nt][bins][40][64]
// (the sample's bit within its word group fastest). to_dev selects the direction.
__global__ void msc_acc_layout_kernel(double *dst, const double *src, int64_t G, int nt, int nb,
                                      int to_dev)
{
    const int64_t total = G * 64 * (int64_t)nt * nb * SG_NACC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        // e runs over the canonical index ((s * nt + t) * nb + bin) * 40 + k
        const int k = (int)(e % SG_NACC);
        const int64_t tb = (e / SG_NACC) % ((int64_t)nt * nb);  // t * nb + bin
        const int64_t s = e / ((int64_t)SG_NACC * nt * nb);
        const int64_t d = (((s / 64) * nt * nb + tb) * SG_NACC + k) * 64 + (s % 64);
        if (to_dev)
            dst[d] = src[e];
        else
            dst[e] = src[d];
    }
}

// canonical int8 [S][2][nt][N] -> W [G][nt][2][N]
__global__ void msc_import_spins_kernel(uint64_t *W, const int8_t *c, int64_t G, int L, int nt,
                                        const int *skip)
{
    if (skip && *skip) return;  // the upload failed its check: keep the state
    const int N = L * L * L;
    const int64_t total = G * nt * 2 * (int64_t)N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int r = (int)((e / N) % 2);
        const int t = (int)((e / (2 * (int64_t)N)) % nt);
        const int64_t g = e / (2 * (int64_t)N * nt);
        uint64_t w = 0;
        for (int b = 0; b < 64; ++b) {
            const int64_t s = 64 * g + b;
            if (c[((s * 2 + r) * nt + t) * N + i] < 0) w |= 1ull << b;
        }
        W[e] = w;
    }
}

__global__ void msc_export_spins_kernel(int8_t *c, const uint64_t *W, int64_t S, int L, int nt)
{
    const int N = L * L * L;
    const int64_t total = S * 2 * (int64_t)nt * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int t = (int)((e / N) % nt);
        const int r = (int)((e / ((int64_t)N * nt)) % 2);
        const int64_t s = e / ((int64_t)2 * nt * N);
        const int64_t g = s / 64;
        const int b = (int)(s % 64);
        const uint64_t w = W[((g * nt + t) * 2 + r) * N + i];
        c[e] = ((w >> b) & 1ull) ? -1 : 1;
    }
}

// canonical float [S][3][N] (+-1) -> Jw [G][3][N]
__global__ void msc_import_J_kernel(uint64_t *Jw, const float *Jc, int64_t G, int L)
{
    const int N = L * L * L;
    const int64_t total = G * 3 * (int64_t)N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int d = (int)((e / N) % 3);
        const int64_t g = e / (3 * (int64_t)N);
        uint64_t w = 0;
        for (int b = 0; b < 64; ++b)
            if (Jc[((64 * g + b) * 3 + d) * N + i] < 0.0f) w |= 1ull << b;
        Jw[e] = w;
    }
}

__global__ void msc_export_J_kernel(float *Jc, const uint64_t *Jw, int64_t S, int L)
{
    const int N = L * L * L;
    const int64_t total = S * 3 * (int64_t)N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int d = (int)((e / N) % 3);
        const int64_t s = e / (3 * (int64_t)N);
        Jc[e] = ((Jw[((s / 64) * 3 + d) * N + i] >> (s % 64)) & 1ull) ? -1.0f : 1.0f;
    }
}

// +-J bonds and initial spins drawn from the seed (same draws as the int8 path)
__global__ void msc_gen_kernel(uint64_t *Jw, uint64_t *W, int64_t G, int L, int nt, uint32_t slo,
                               uint32_t shi, int64_t key0)
{
    const int N = L * L * L;
    const int64_t nJ = G * 3 * (int64_t)N, nW = G * nt * 2 * (int64_t)N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nJ + nW;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w = 0;
        if (e < nJ) {
            const int i = (int)(e % N);
            const int d = (int)((e / N) % 3);
            const int64_t g = e / (3 * (int64_t)N);
            for (int b = 0; b < 64; ++b) {
                const u32x4 o = philox10(slo ^ kTagBond, (uint32_t)(64 * g + b + key0), (uint32_t)(i >> 7),
                                         (uint32_t)d, 0u, shi);
                w |= (uint64_t)((o.v[(i >> 5) & 3] >> (i & 31)) & 1u) << b;
            }
            Jw[e] = w;
        } else {
            const int64_t f = e - nJ;
            const int i = (int)(f % N);
            const int r = (int)((f / N) % 2);
            const int t = (int)((f / (2 * (int64_t)N)) % nt);
            const int64_t g = f / (2 * (int64_t)N * nt);
            for (int b = 0; b < 64; ++b) {
                const u32x4 o = philox10(slo ^ kTagInit, (uint32_t)(64 * g + b + key0), (uint32_t)(i >> 7),
                                         ((uint32_t)r << 16) | (uint32_t)t, 0u, shi);
                w |= (uint64_t)((o.v[(i >> 5) & 3] >> (i & 31)) & 1u) << b;
            }
            W[f] = w;
        }
    }
}

// B and M of every sample and chain straight from the bond sum.
__global__ void msc_energies_kernel(const MscArgs a, int L)
{
    const int N = L * L * L;
    const int64_t S = a.G * 64;
    const int64_t total = S * 2 * a.nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e % a.nt);
        const int r = (int)((e / a.nt) % 2);
        const int64_t s = e / (2 * a.nt);
        const int64_t g = s / 64;
        const int b = (int)(s % 64);
        const uint64_t *w = a.W + ((g * a.nt + t) * 2 + r) * N;
        const uint64_t *J = a.Jw + g * 3 * N;
        long long B = 0, M = 0;
        for (int i = 0; i < N; ++i) {
            const int si = ((w[i] >> b) & 1ull) ? -1 : 1;
            M += si;
            for (int d = 0; d < 3; ++d) {
                const int j = nb_site(L, i, d, +1);
                const int sj = ((w[j] >> b) & 1ull) ? -1 : 1;
                const int jb = ((J[d * N + i] >> b) & 1ull) ? -1 : 1;
                B += jb * si * sj;
            }
        }
        a.B[e] = B;
        a.M[e] = M;
    }
}

// Standalone exchange: one thread per (sample, replica, pair), then the
// masked swaps, on the global-memory state (call after msc_energies_kernel).
__global__ void msc_exchange_decide_kernel(const MscArgs a, int parity, uint32_t call_id,
                                           uint64_t *masks /* [G][2][nt] */)
{
    const int64_t S = a.G * 64;
    const int np = (a.nt - parity) / 2;
    const int64_t total = S * 2 * (int64_t)np;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % np);
        const int r = (int)((e / np) % 2);
        const int64_t s = e / (2 * (int64_t)np);
        const int p = parity + 2 * m;
        int64_t *Bp = a.B + (s * 2 + r) * a.nt + p;
        int64_t *Mp = a.M + (s * 2 + r) * a.nt + p;
        const long long dB = Bp[0] - Bp[1], dM = Mp[0] - Mp[1];
        const float t1 = __fmul_rn(__ll2float_rn(dB), 1.0f);
        const float t2 = __fmul_rn(a.h_f, __ll2float_rn(dM));
        const float dE = -__fadd_rn(t1, t2);
        const float D = __fmul_rn(a.dbeta[p], dE);
        const u32x4 o = philox10(a.seed_lo ^ kTagExc, (uint32_t)(s + a.s_key0), (uint32_t)p, call_id,
                                 (uint32_t)r | 0x100u, a.seed_hi);
        if ((D >= 0.0f) || (o.v[0] <= thr_of_logp(D))) {
            const int64_t tb = Bp[0]; Bp[0] = Bp[1]; Bp[1] = tb;
            const int64_t tm = Mp[0]; Mp[0] = Mp[1]; Mp[1] = tm;
            atomicOr((unsigned long long *)&masks[((s / 64) * 2 + r) * a.nt + p],
                     1ull << (s % 64));
        }
    }
}

__global__ void msc_exchange_apply_kernel(const MscArgs a, int L, const uint64_t *masks)
{
    const int N = L * L * L;
    const int64_t total = a.G * 2 * (int64_t)a.nt * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % N);
        const int p = (int)((e / N) % a.nt);
        const int r = (int)((e / ((int64_t)N * a.nt)) % 2);
        const int64_t g = e / (2 * (int64_t)N * a.nt);
        const uint64_t m = masks[(g * 2 + r) * a.nt + p];
        if (!m || p + 1 >= a.nt) continue;
        uint64_t *pa = a.W + ((g * a.nt + p) * 2 + r) * N + i;
        uint64_t *pb = a.W + ((g * a.nt + p + 1) * 2 + r) * N + i;
        const uint64_t x = (*pa ^ *pb) & m;
        *pa ^= x;
        *pb ^= x;
    }
}

// q(k) for arbitrary integer k, one thread per (sample, slot, k).
__global__ void msc_measure_k_kernel(const MscArgs a, int L, const int *kv, int nk, float *out)
{
    const int N = L * L * L;
    const int64_t S = a.G * 64;
    const int64_t total = S * a.nt * (int64_t)nk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % nk);
        const int t = (int)((e / nk) % a.nt);
        const int64_t s = e / ((int64_t)nk * a.nt);
        const int64_t g = s / 64;
        const int b = (int)(s % 64);
        const uint64_t *w0 = a.W + ((g * a.nt + t) * 2 + 0) * N;
        const uint64_t *w1 = w0 + N;
        float re = 0.0f, im = 0.0f;
        for (int i = 0; i < N; ++i) {
            const int x = i % L, y = (i / L) % L, z = i / (L * L);
            const int q = (((w0[i] ^ w1[i]) >> b) & 1ull) ? -1 : 1;
            int ph = (kv[3 * j] * x + kv[3 * j + 1] * y + kv[3 * j + 2] * z) % L;
            if (ph < 0) ph += L;
            float sn, cs;
            sincospif(2.0f * (float)ph / (float)L, &sn, &cs);
            re += q * cs;
            im += q * sn;
        }
        out[2 * e] = re / (float)N;
        out[2 * e + 1] = im / (float)N;
    }
}

inline int gridn(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 148 * 32) b = 148 * 32;
    return (int)b;
}

constexpr int kMscMaxSmem = 227 * 1024;

constexpr int kMscNarrow = 128;

template <int L>
cudaError_t msc_split_launch_t(const MscArgs &a, cudaStream_t st)
{
    if constexpr (msc_j_shared(L)) {
        return cudaErrorInvalidValue;
    } else {
        // (the kernel's own mbarrier takes a few bytes of static shared memory,
        // so the dynamic size asked for is the carve's, not the SM maximum)
        const size_t smem = msc_carve_split(nullptr, L, nullptr);
        static cudaError_t attr_s = cudaFuncSetAttribute(
            msc_split_sweep_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr_s != cudaSuccess) return attr_s;
        const dim3 grid((unsigned)(a.nt / 2 + 1), 2u, (unsigned)a.G);
        msc_split_sweep_kernel<L><<<grid, kMscSplitThreads, smem, st>>>(a);
        return cudaGetLastError();
    }
}

template <int L>
cudaError_t msc_measure_launch_t(const MscArgs &a, cudaStream_t st)
{
    if constexpr (msc_j_shared(L)) {
        return cudaErrorInvalidValue;
    } else {
        const size_t smem = msc_carve_meas(nullptr, L, nullptr);
        static cudaError_t attr_m = cudaFuncSetAttribute(
            msc_measure_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr_m != cudaSuccess) return attr_m;
        const dim3 grid((unsigned)a.nt, (unsigned)a.G);
        msc_measure_kernel<L><<<grid, kMscMeasThreads, smem, st>>>(a);
        return cudaGetLastError();
    }
}

template <int L>
cudaError_t msc_launch_t(const MscArgs &a, int threads, cudaStream_t st)
{
    // the largest carve of the instance (the kernel's mbarrier takes a few
    // bytes of static shared memory beside it)
    static cudaError_t attr_n = cudaFuncSetAttribute(
        msc_sweep_kernel<L, kMscNarrow, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)msc_carve(nullptr, L, nullptr, msc_measured_slots(L, false)));
    static cudaError_t attr_w = cudaFuncSetAttribute(
        msc_sweep_kernel<L, kMscThreads, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)msc_carve(nullptr, L, nullptr, msc_measured_slots(L, true)));
    if (attr_n != cudaSuccess) return attr_n;
    if (attr_w != cudaSuccess) return attr_w;
    const size_t smem = msc_carve(nullptr, L, nullptr, msc_measured_slots(L, threads != kMscNarrow));
    dim3 grid((unsigned)(a.nt / 2 + 1), (unsigned)a.G);
    if (threads == kMscNarrow)
        msc_sweep_kernel<L, kMscNarrow, 6><<<grid, threads, smem, st>>>(a);
    else
        msc_sweep_kernel<L, kMscThreads, 1><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

#define SG_MSC_FOR_EACH_L(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16)

}  // namespace

size_t msc_smem_bytes(int L)
{
    const size_t b = msc_carve(nullptr, L, nullptr, 2);  // the wide instance's (the larger)
    return b <= (size_t)kMscMaxSmem ? b : 0;
}

bool msc_supported_L(int L)
{
#define X(LL) if (L == LL) return msc_smem_bytes(L) > 0;
    SG_MSC_FOR_EACH_L(X)
#undef X
    return false;
}

int msc_threads(int L, int requested)
{
    // The exchange step uses one thread per (replica, sample), so at least
    // 128; a multiple of 128 splits into whole warps per chain for both unit
    // sizes (2 or 4 chains), which the per-warp energy reduction needs.
    if (requested > 0) {
        const int t = requested < 128 ? 128 : requested > kMscThreads ? kMscThreads : requested;
        return t & ~127;
    }
    // measured on B300 (+-J, 32-56 temperatures, 4096-8192 samples): small
    // lattices run fastest with several narrow CTAs per SM, large ones with
    // one wide CTA
    return L <= 10 ? 128 : L == 12 ? 256 : kMscThreads;
}

bool msc_split(int L, int requested) { return requested <= 0 && L >= 12 && msc_supported_L(L); }

cudaError_t msc_measure_split(const MscArgs &a, int L, cudaStream_t st)
{
#define X(LL) if (L == LL) return msc_measure_launch_t<LL>(a, st);
    SG_MSC_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t msc_sweep(const MscArgs &a, int L, int threads, cudaStream_t st, bool split)
{
    if (split) {
#define X(LL) if (L == LL) return msc_split_launch_t<LL>(a, st);
        SG_MSC_FOR_EACH_L(X)
#undef X
        return cudaErrorInvalidValue;
    }
    if (threads < 128 || threads > kMscThreads || (threads & 127)) return cudaErrorInvalidValue;
#define X(LL) if (L == LL) return msc_launch_t<LL>(a, threads, st);
    SG_MSC_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t msc_import_spins(uint64_t *W, const int8_t *c, int64_t G, int L, int nt, cudaStream_t st,
                             const int *skip)
{
    msc_import_spins_kernel<<<gridn(G * nt * 2 * L * L * L, 256), 256, 0, st>>>(W, c, G, L, nt, skip);
    return cudaGetLastError();
}

cudaError_t msc_export_spins(int8_t *c, const uint64_t *W, int64_t G, int L, int nt, cudaStream_t st)
{
    msc_export_spins_kernel<<<gridn(G * 64 * 2 * nt * L * L * L, 256), 256, 0, st>>>(c, W, G * 64, L,
                                                                                    nt);
    return cudaGetLastError();
}

cudaError_t msc_acc_layout(double *dst, const double *src, int64_t G, int nt, int nb, bool to_dev,
                           cudaStream_t st)
{
    msc_acc_layout_kernel<<<gridn(G * 64 * nt * nb * SG_NACC, 256), 256, 0, st>>>(dst, src, G, nt, nb,
                                                                                  to_dev ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t msc_import_J(uint64_t *Jw, const float *Jc, int64_t G, int L, cudaStream_t st)
{
    msc_import_J_kernel<<<gridn(G * 3 * L * L * L, 256), 256, 0, st>>>(Jw, Jc, G, L);
    return cudaGetLastError();
}

cudaError_t msc_export_J(float *Jc, const uint64_t *Jw, int64_t G, int L, cudaStream_t st)
{
    msc_export_J_kernel<<<gridn(G * 64 * 3 * L * L * L, 256), 256, 0, st>>>(Jc, Jw, G * 64, L);
    return cudaGetLastError();
}

cudaError_t msc_generate(uint64_t *Jw, uint64_t *W, int64_t G, int L, int nt, uint32_t slo,
                         uint32_t shi, int64_t key0, cudaStream_t st)
{
    msc_gen_kernel<<<gridn(G * (3 + 2 * nt) * L * L * L, 128), 128, 0, st>>>(Jw, W, G, L, nt, slo,
                                                                              shi, key0);
    return cudaGetLastError();
}

cudaError_t msc_energies(const MscArgs &a, int L, cudaStream_t st)
{
    msc_energies_kernel<<<gridn(a.G * 64 * 2 * a.nt, 128), 128, 0, st>>>(a, L);
    return cudaGetLastError();
}

cudaError_t msc_exchange(const MscArgs &a, int L, int parity, uint32_t call_id, uint64_t *masks,
                         cudaStream_t st)
{
    cudaError_t e = msc_energies(a, L, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(masks, 0, sizeof(uint64_t) * a.G * 2 * a.nt, st);
    if (e != cudaSuccess) return e;
    const int np = (a.nt - parity) / 2;
    msc_exchange_decide_kernel<<<gridn(a.G * 64 * 2 * (np > 0 ? np : 1), 128), 128, 0, st>>>(
        a, parity, call_id, masks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    msc_exchange_apply_kernel<<<gridn(a.G * 2 * a.nt * L * L * L, 256), 256, 0, st>>>(a, L, masks);
    return cudaGetLastError();
}

cudaError_t msc_measure_k(const MscArgs &a, int L, const int *k_dev, int nk, float *out,
                          cudaStream_t st)
{
    msc_measure_k_kernel<<<gridn(a.G * 64 * a.nt * nk, 128), 128, 0, st>>>(a, L, k_dev, nk, out);
    return cudaGetLastError();
}

}  // namespace sg
