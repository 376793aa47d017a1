// sg_device.cuh -- device-side building blocks of the EA spin-glass engine:
// the counter-based random number generator, the FP32 exponential used for
// continuous acceptance probabilities, the 32-bit threshold map, packed FP32
// pairs, bit-sliced counters and their warp reductions, untiled TMA bulk
// copies on an mbarrier, and exact FP64 values assembled from bit fields.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11). The paper drew its numbers from a
// different generator (XORWOW); a counter-based generator lets every
// (sample, replica, slot, sweep, site) address its own number, so the result
// does not depend on launch shape, and a checkpoint is just the sweep index.
#pragma once
#include <stdint.h>

namespace sg {

constexpr uint32_t kTagMet = 0x4D455452u;
constexpr uint32_t kTagExc = 0x45584348u;
constexpr uint32_t kTagInit = 0x494E4954u;
constexpr uint32_t kTagBond = 0x424F4E44u;

struct u32x4 {
    uint32_t v[4];
};

// Ten Philox rounds: two 32x32->64 multiplies per round, the high halves mixed
// with the other two counter words and the round key, then the Weyl key bump.
__device__ __forceinline__ u32x4 philox10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                          uint32_t c2, uint32_t c3)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c0;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    u32x4 r;
    r.v[0] = c0;
    r.v[1] = c1;
    r.v[2] = c2;
    r.v[3] = c3;
    return r;
}

// The same with the round keys of k0 given (k0r[r] = k0 + r * 0x9E3779B9):
// when k0 is fixed for a launch, the table lives in the kernel's parameters
// and each round's xor takes its key as a constant operand.
__device__ __forceinline__ u32x4 philox10_rk(const uint32_t *k0r, uint32_t k1, uint32_t c0,
                                             uint32_t c1, uint32_t c2, uint32_t c3)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c0;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0r[round];
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
        k1 += 0xBB67AE85u;
    }
    u32x4 r;
    r.v[0] = c0;
    r.v[1] = c1;
    r.v[2] = c2;
    r.v[3] = c3;
    return r;
}

// Four calls of philox10_rk with the same key and counter words c0, c1, c3
// and four values of c2, round by round: the round key of k1 is formed once
// per round for all four, and the first round's product of c0 is shared.
// out[q] equals philox10_rk(k0r, k1, c0, c1, c2[q], c3) bit for bit.
__device__ __forceinline__ void philox10x4_rk(const uint32_t *k0r, uint32_t k1, uint32_t c0,
                                              uint32_t c1, const uint32_t (&c2)[4], uint32_t c3,
                                              u32x4 (&out)[4])
{
    uint32_t a[4], b[4], c[4], d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a[q] = c0;
        b[q] = c1;
        c[q] = c2[q];
        d[q] = c3;
    }
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint64_t pa = (uint64_t)0xD2511F53u * a[q];
            const uint64_t pb = (uint64_t)0xCD9E8D57u * c[q];
            const uint32_t n0 = (uint32_t)(pb >> 32) ^ b[q] ^ k0r[round];
            const uint32_t n2 = (uint32_t)(pa >> 32) ^ d[q] ^ k1;
            b[q] = (uint32_t)pb;
            d[q] = (uint32_t)pa;
            a[q] = n0;
            c[q] = n2;
        }
        k1 += 0xBB67AE85u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        out[q].v[0] = a[q];
        out[q].v[1] = b[q];
        out[q].v[2] = c[q];
        out[q].v[3] = d[q];
    }
}

// e^x * 2^k on [-64, 0] from IEEE basic operations only, so that host and
// device agree bit for bit: Cody-Waite reduction x = n*ln2 + r with ln2 split
// into 0.693359375 + (-2.12194440e-4), then e^r by its degree-7 Taylor
// polynomial (coefficients 1/k! rounded to FP32) in Horner form with fused
// multiply-adds, and the factor 2^(n+k) assembled from exponent bits.
// n = rint(x * log2(e)) is taken with the 1.5 * 2^23 shifter: adding it rounds
// to the nearest integer (ties to even), exactly as rintf does for |t| < 2^22.
template <int K>
__device__ __forceinline__ float exp_cw32_scaled(float x)
{
    const float t = __fmul_rn(x, 1.44269502f);
    const float sh = __fadd_rn(t, 12582912.0f);
    const float n = __fadd_rn(sh, -12582912.0f);
    float r = __fmaf_rn(-n, 0.693359375f, x);
    r = __fmaf_rn(-n, -2.12194440e-4f, r);
    float p = 1.0f / 5040.0f;
    p = __fmaf_rn(p, r, 1.0f / 720.0f);
    p = __fmaf_rn(p, r, 1.0f / 120.0f);
    p = __fmaf_rn(p, r, 1.0f / 24.0f);
    p = __fmaf_rn(p, r, 1.0f / 6.0f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int ni = __float_as_int(sh) - 0x4B400000;
    return __fmul_rn(p, __int_as_float((ni + 127 + K) << 23));
}


// Acceptance threshold for an FP32 log-probability x: a uniform 32-bit word
// r is accepted iff r <= thr, i.e. with probability (thr + 1)/2^32; thr is
// floor(e^x * 2^32) saturated to 0xFFFFFFFF. x >= 0 (an energy decrease)
// gives 0xFFFFFFFF; x < -64 gives 0 (e^-64 * 2^32 < 1, the clamp changes
// nothing). The float-to-unsigned conversion saturates at 2^32 - 1.
__device__ __forceinline__ uint32_t thr_of_logp(float x)
{
    const float xc = fminf(fmaxf(x, -64.0f), 0.0f);
    return __float2uint_rz(exp_cw32_scaled<32>(xc));
}

// Screen of the Metropolis test r <= thr_of_logp(x) that skips the
// exponential for almost every draw. Accepting iff r <= thr_of_logp(x) is
// accepting iff r <= F(x), with F = exp_cw32_scaled<32>(clamped x) (r is an
// integer, and F >= 2^32 saturates the threshold). A = 2^(x log2(e) + 32) from
// the hardware ex2.approx is within 2^-18 (relative) of e^x 2^32 for
// x in [-64, 0], counting the rounding of the exponent; F is within 2^-21 of
// it and the float image of r within 2^-24 of r. So whenever
// |fl(r) - A| > 2^-12 A the sign of fl(r) - A is the sign of r - F, and the
// screen decides exactly as the threshold would; x >= 0 (A >= 2^32) never
// screens as a rejection, and x < -64 leaves only r = 0 accepted, as the clamp
// does. Draws inside the band (probability below 2^-11 per attempt) set amb,
// and the caller redoes them with thr_of_logp. Returns fl(r) - A, whose sign
// bit is the screen's decision (set = accept).
__device__ __forceinline__ float screen_logp(float x, uint32_t r, bool &amb)
{
    const float y = __fmaf_rn(x, 1.44269502f, 32.0f);
    float a;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(y));
    const float u = __fsub_rn(__uint2float_rn(r), a);
    amb |= fabsf(u) <= __fmul_rn(a, 2.44140625e-4f);  // 2^-12 A
    return u;
}

// Two FP32 values in one 64-bit register pair, and the packed FP32
// arithmetic of sm_100-class GPUs on them: one instruction rounds both
// lanes exactly as the scalar operation would (IEEE round to nearest even,
// no flush to zero), so pairs of chains share an issue slot.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// screen_logp for two log-probabilities at once (x of a chain pair, packed
// as by f2_pack), in packed FP32: the same operations and roundings per
// lane. u0, u1 receive fl(r) - A, whose sign bits are the decisions; amb0,
// amb1 are set where the draw falls in the band.
__device__ __forceinline__ void screen_pair(unsigned long long xp, uint32_t r0, uint32_t r1,
                                            bool &amb0, bool &amb1, float &u0, float &u1)
{
    float y0, y1;
    f2_unpack(f2_fma(xp, f2_pack(1.44269502f, 1.44269502f), f2_pack(32.0f, 32.0f)), y0, y1);
    float a0, a1;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a0) : "f"(y0));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(a1) : "f"(y1));
    const unsigned long long ap = f2_pack(a0, a1);
    f2_unpack(f2_sub(f2_pack(__uint2float_rn(r0), __uint2float_rn(r1)), ap), u0, u1);
    float w0, w1;
    f2_unpack(f2_mul(ap, f2_pack(2.44140625e-4f, 2.44140625e-4f)), w0, w1);  // 2^-12 A
    amb0 = fabsf(u0) <= w0;
    amb1 = fabsf(u1) <= w1;
}

// Logarithmic bin of a measurement taken at global sweep n (0-based):
// floor(log2(n + 1)), with every later sweep in the last of n_bins bins. Bin b
// covers sweeps 2^b - 1 .. 2^(b+1) - 2, the second half of a run of 2^(b+1)
// sweeps (the logarithmic-binning equilibration test).
__device__ __forceinline__ int log_bin(int64_t n, int n_bins)
{
    const int b = 63 - __clzll((long long)(n + 1));
    return b < n_bins - 1 ? b : n_bins - 1;
}

// Bit-sliced ripple add of a K-plane number into a D-plane counter (64
// independent lanes, plane k holding bit k of every lane's count).
template <int D, int K>
__device__ __forceinline__ void bs_add(uint64_t (&c)[D], const uint64_t (&x)[K])
{
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const uint64_t a = c[k];
        const uint64_t b = k < K ? x[k] : 0ull;
        c[k] = a ^ b ^ carry;
        carry = (a & b) | (carry & (a ^ b));
    }
}

// The same on 32 lanes.
template <int D, int K>
__device__ __forceinline__ void bs_add32(uint32_t (&c)[D], const uint32_t (&x)[K])
{
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const uint32_t a = c[k];
        const uint32_t b = k < K ? x[k] : 0u;
        c[k] = a ^ b ^ carry;
        carry = (a & b) | (carry & (a ^ b));
    }
}

// 32x32 bit transpose across a warp by five shuffle stages: afterwards bit k
// of lane l's word is bit l of lane k's word before.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x)
{
    const int lane = threadIdx.x & 31;
    uint32_t m = 0x0000FFFFu;
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1, m ^= m << k) {
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, k);
        x = (lane & k) ? ((x & ~m) | ((y & ~m) >> k)) : ((x & m) | ((y & m) << k));
    }
    return x;
}

// Column counts over the 32 lanes of a warp: lane l receives the number of
// lanes whose word has bit l set.
__device__ __forceinline__ int warp_column_popc(uint32_t x) { return __popc(warp_transpose32(x)); }

// Warp totals of a bit-sliced counter over 64 bit lanes (plane k of c holds
// bit k of every bit lane's count). A butterfly of bit-sliced adds: the first
// stage leaves each thread the half of the 64 bit lanes it keeps (threads
// 0-15 bits 0-31, 16-31 bits 32-63) summed with its partner's, the next four
// sum those 32-bit planes over the rest of the threads, one plane wider per
// stage. Afterwards thread l holds, for bit lanes b0 = 32 (l >> 4) + (l & 15)
// and b0 + 16, the sum over the warp's 32 threads of their counts (v0, v1).
// D + 5 planes hold every total, so nothing overflows; the result equals the
// per-plane transpose-and-popcount sums, with fewer shuffles and operations.
template <int D>
__device__ __forceinline__ void warp_bs_totals(const uint64_t (&c)[D], uint32_t &v0, uint32_t &v1)
{
    constexpr int E = D + 5;
    const int lane = threadIdx.x & 31;
    const bool hi = lane & 16;
    uint32_t x[E];
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const uint32_t lo32 = (uint32_t)c[k], hi32 = (uint32_t)(c[k] >> 32);
        const uint32_t keep = hi ? hi32 : lo32;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, hi ? lo32 : hi32, 16);
        x[k] = keep ^ y ^ carry;
        carry = (keep & y) | (carry & (keep ^ y));
    }
    x[D] = carry;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int m = 8 >> s, P = D + 1 + s;  // planes in use before this stage
        uint32_t cy = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const uint32_t a = x[k];
            const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, a, m);
            x[k] = a ^ y ^ cy;
            cy = (a & y) | (cy & (a ^ y));
        }
        x[P] = cy;
    }
    const int j = lane & 15;
    v0 = 0;
    v1 = 0;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        v0 |= ((x[k] >> j) & 1u) << k;
        v1 |= ((x[k] >> (j + 16)) & 1u) << k;
    }
}

// ---- untiled bulk copies (TMA) counted on a shared-memory mbarrier --------
// cp.async.bulk moves one contiguous block from global to shared memory on
// the SM's copy engine, so a CTA has its whole state in flight at once
// instead of one load per thread and loop trip; the barrier's phase
// completes when the bytes announced by mbar_expect_tx have landed. Both
// addresses must be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// One arrival (the thread that announces the bytes) completes a phase.
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst_smem)),
        "l"((unsigned long long)__cvta_generic_to_global(src_gmem)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Ask the copy engine to bring a block into L2 ahead of its plain loads.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src_gmem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     (unsigned long long)__cvta_generic_to_global(src_gmem)),
                 "r"(bytes)
                 : "memory");
}

// Wait until phase `parity` of the barrier has completed; false once `limit`
// clock cycles have passed without it (the caller reports and gives up).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit)
{
    const uint32_t b = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if ((unsigned long long)(clock64() - t0) > limit) return false;
    }
}

// ---- exact FP64 values of the accumulation from integer operations --------
// B300 issues FP64 at a few lanes per cycle, and the accumulation phase of
// the overlap measurement is partly bound by it. The conversions and products below
// are exact in FP64 (24-bit significands and their squares, integers below
// 2^53), so their results are unique: assembled from bit fields they equal
// the FP64 instructions' results bit for bit, and only the rounded sums and
// products stay on the FP64 pipe. Branch-free, with selects for zero.

// (double)f for f zero or normal. The DFT sums of the measurement are: their
// terms are integer multiples of FP32 twiddles, so every nonzero sum is a
// multiple of the smallest twiddle's ulp (far above 2^-126), and |sum| <= L^3.
__device__ __forceinline__ double f64_of_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint64_t bits = ((uint64_t)(u & 0x80000000u) << 32) |
                          ((uint64_t)(((u >> 23) & 0xFFu) + 896u) << 52) |
                          ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double(
        (long long)((u & 0x7FFFFFFFu) ? bits : ((uint64_t)(u & 0x80000000u) << 32)));
}

// (double)f * (double)f for f zero or normal: the 48-bit square of the 24-bit
// significand, its leading bit moved to bit 52.
__device__ __forceinline__ double f64_sq_of_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFFu);
    const uint64_t m = (uint64_t)((u & 0x7FFFFFu) | 0x800000u);
    const uint64_t p = m * m;  // in [2^46, 2^48)
    const uint32_t top = (uint32_t)(p >> 47);
    const uint64_t frac = (p << (6 - top)) & ((1ull << 52) - 1);
    const uint64_t ex = (uint64_t)(2 * e - 300 + 46 + (int)top + 1023);
    return __longlong_as_double((long long)((u & 0x7FFFFFFFu) ? ((ex << 52) | frac) : 0ull));
}

// (double)v for |v| < 2^53.
__device__ __forceinline__ double f64_of_i64(long long v)
{
    const uint64_t a = (uint64_t)(v < 0 ? -v : v);
    const int pos = 63 - __clzll((long long)(a | 1ull));  // leading bit (0 for a = 0, 1)
    const uint64_t bits = (v < 0 ? (1ull << 63) : 0ull) | ((uint64_t)(pos + 1023) << 52) |
                          ((a << (52 - pos)) & ((1ull << 52) - 1));
    return __longlong_as_double((long long)(a ? bits : 0ull));
}

// Bound of a bulk-copy wait: 2^30 cycles, about half a second at 2 GHz, far
// beyond the microseconds a copy of a CTA's state takes.
constexpr unsigned long long kBulkWaitCycles = 1ull << 30;

}  // namespace sg
