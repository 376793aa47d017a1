// sg_int8.cu -- int8-spin path of the EA spin-glass engine on B300 (sm_103a):
// shared-memory instances of the fused kernel (the kernel itself is in
// sg_int8_run.cuh; the large-lattice global-memory instances are in
// sg_int8_gst.cu), instance preparation, conversion and standalone kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "sg_int8_run.cuh"

namespace sg {

namespace {

// ---------------------------------------------------------------------------
// Instance preparation, conversion and standalone kernels (global memory).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int site_nb(int L, int i, int d, int step)
{
    int x = i % L, y = (i / L) % L, z = i / (L * L);
    if (d == 0) x = (x + step + L) % L;
    if (d == 1) y = (y + step + L) % L;
    if (d == 2) z = (z + step + L) % L;
    return x + L * (y + L * z);
}

__global__ void gen_pmj_kernel(uint8_t *J8, int64_t S, int L, uint32_t slo, uint32_t shi,
                               int64_t key0)
{
    const int N = L * L * L;
    const int64_t total = S * N;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / N;
        const int i = (int)(g % N);
        uint8_t out[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            for (int side = 0; side < 2; ++side) {
                const int owner = side == 0 ? i : site_nb(L, i, d, -1);  // bond owner site
                const u32x4 o = philox10(slo ^ kTagBond, (uint32_t)(s + key0), (uint32_t)(owner >> 7),
                                         (uint32_t)d, 0u, shi);
                out[2 * d + side] = (uint8_t)((o.v[(owner >> 5) & 3] >> (owner & 31)) & 1u);
            }
        }
        uint2 v;
        v.x = out[0] | (out[1] << 8) | (out[2] << 16) | ((uint32_t)out[3] << 24);
        v.y = out[4] | (out[5] << 8);
        reinterpret_cast<uint2 *>(J8)[g] = v;
    }
}

__global__ void gen_gauss_kernel(float *Jg, int64_t S, int L, uint32_t slo, uint32_t shi,
                                 int64_t key0)
{
    const int N = L * L * L;
    const int64_t pairs = S * 3 * (int64_t)((N + 1) / 2);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pairs;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int half = (N + 1) / 2;
        const int64_t s = g / (3 * half);
        const int d = (int)((g / half) % 3);
        const int m = (int)(g % half);
        const u32x4 o = philox10(slo ^ kTagBond, (uint32_t)(s + key0), (uint32_t)m, (uint32_t)d, 1u, shi);
        // two uniforms in (0, 1) with 53 bits each, then Box-Muller
        const uint64_t a53 = (((uint64_t)o.v[0] << 21) ^ (o.v[1] >> 11)) & ((1ull << 53) - 1);
        const uint64_t b53 = (((uint64_t)o.v[2] << 21) ^ (o.v[3] >> 11)) & ((1ull << 53) - 1);
        const double u1 = ((double)a53 + 0.5) * 0x1.0p-53;
        const double u2 = ((double)b53 + 0.5) * 0x1.0p-53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const double gv[2] = {rad * cs, rad * sn};
        for (int q = 0; q < 2; ++q) {
            const int i = 2 * m + q;
            if (i >= N) break;
            double v = rint(gv[q] * 131072.0);
            v = fmin(fmax(v, -16.0 * 131072.0), 16.0 * 131072.0);
            Jg[(s * 3 + d) * N + i] = (float)(v / 131072.0);
        }
    }
}

__global__ void gen_spins_kernel(uint8_t *spins, int64_t S, int L, int nt, int Tp, uint32_t slo,
                                 uint32_t shi, int64_t key0)
{
    const int N = L * L * L;
    const int RB = 2 * Tp;
    const int64_t total = S * N * (int64_t)RB;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / ((int64_t)N * RB);
        const int i = (int)((g / RB) % N);
        const int rb = (int)(g % RB);
        const int r = (rb & 7) >> 2, t = 4 * (rb >> 3) + (rb & 3);
        uint8_t v = 0;
        if (t < nt) {
            const u32x4 o = philox10(slo ^ kTagInit, (uint32_t)(s + key0), (uint32_t)(i >> 7),
                                     ((uint32_t)r << 16) | (uint32_t)t, 0u, shi);
            v = (uint8_t)((o.v[(i >> 5) & 3] >> (i & 31)) & 1u);
        }
        spins[g] = v;
    }
}

__global__ void import_J_kernel(uint8_t *J8, float *Jg, const float *Jc, int64_t S, int L,
                                int gauss)
{
    const int N = L * L * L;
    const int64_t total = S * N;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / N;
        const int i = (int)(g % N);
        const float *Js = Jc + s * 3 * N;
        if (gauss) {
            for (int d = 0; d < 3; ++d) Jg[(s * 3 + d) * N + i] = Js[d * N + i];
        } else {
            uint8_t out[6];
            for (int d = 0; d < 3; ++d) {
                out[2 * d] = Js[d * N + i] < 0.0f;
                out[2 * d + 1] = Js[d * N + site_nb(L, i, d, -1)] < 0.0f;
            }
            uint2 v;
            v.x = out[0] | (out[1] << 8) | (out[2] << 16) | ((uint32_t)out[3] << 24);
            v.y = out[4] | (out[5] << 8);
            reinterpret_cast<uint2 *>(J8)[g] = v;
        }
    }
}

__global__ void export_J_kernel(float *Jc, const uint8_t *J8, const float *Jg, int64_t S, int L,
                                int gauss)
{
    const int N = L * L * L;
    const int64_t total = S * 3 * (int64_t)N;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / (3 * N);
        const int d = (int)((g / N) % 3);
        const int i = (int)(g % N);
        Jc[g] = gauss ? Jg[g] : (J8[(s * N + i) * 8 + 2 * d] ? -1.0f : 1.0f);
    }
}

__global__ void import_spins_kernel(uint8_t *spins, const int8_t *c, int64_t S, int L, int nt,
                                    int Tp, const int *skip)
{
    if (skip && *skip) return;  // the upload failed its check: keep the state
    const int N = L * L * L;
    const int RB = 2 * Tp;
    const int64_t total = S * N * (int64_t)RB;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = g / ((int64_t)N * RB);
        const int i = (int)((g / RB) % N);
        const int rb = (int)(g % RB);
        const int r = (rb & 7) >> 2, t = 4 * (rb >> 3) + (rb & 3);
        spins[g] = t < nt ? (uint8_t)(c[((s * 2 + r) * nt + t) * N + i] < 0) : (uint8_t)0;
    }
}

__global__ void export_spins_kernel(int8_t *c, const uint8_t *spins, int64_t S, int L, int nt,
                                    int Tp)
{
    const int N = L * L * L;
    const int64_t total = S * 2 * (int64_t)nt * N;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g % N);
        const int t = (int)((g / N) % nt);
        const int r = (int)((g / ((int64_t)N * nt)) % 2);
        const int64_t s = g / ((int64_t)2 * nt * N);
        c[g] = spins[(s * N + i) * (2 * Tp) + slot_byte(r, t)] ? -1 : 1;
    }
}

// Energies straight from the bond sum, one thread per chain (small helper
// used at creation and by the standalone exchange).
__device__ void chain_energy(const Int8Args &a, int L, bool gauss, int64_t s, int r, int t,
                             long long *Bo, long long *Mo)
{
    const int N = L * L * L;
    const int RB = 2 * a.Tp;
    const uint8_t *sp = a.spins + (size_t)s * N * RB + slot_byte(r, t);
    long long b = 0, m = 0;
    for (int i = 0; i < N; ++i) {
        const int si = sp[(size_t)i * RB] ? -1 : 1;
        m += si;
        for (int d = 0; d < 3; ++d) {
            const int j = site_nb(L, i, d, +1);
            const int sj = sp[(size_t)j * RB] ? -1 : 1;
            long long jq;
            if (gauss)
                jq = __float2ll_rn(__fmul_rn(a.Jg[((size_t)s * 3 + d) * N + i], 131072.0f));
            else
                jq = a.J8[((size_t)s * N + i) * 8 + 2 * d] ? -1 : 1;
            b += jq * si * sj;
        }
    }
    *Bo = b;
    *Mo = m;
}

__global__ void energies_kernel(const Int8Args a, int L, int gauss)
{
    const int64_t total = (a.s_end - a.s_begin) * 2 * a.Tp;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = a.s_begin + g / (2 * a.Tp);
        const int r = (int)((g / a.Tp) % 2), t = (int)(g % a.Tp);
        long long b = 0, m = 0;
        if (t < a.nt) chain_energy(a, L, gauss, s, r, t, &b, &m);
        a.B[s * 2 * a.Tp + r * a.Tp + t] = b;
        a.M[s * 2 * a.Tp + r * a.Tp + t] = m;
    }
}

// Standalone exchange: one CTA per sample, on the global-memory state.
__global__ void exchange_kernel(const Int8Args a, int L, int parity, uint32_t call_id)
{
    const int N = L * L * L;
    const int Tp = a.Tp, nt = a.nt, RB = 2 * Tp;
    __shared__ int accept[2][64];
    for (int64_t s = a.s_begin + blockIdx.x; s < a.s_end; s += gridDim.x) {
        __syncthreads();
        for (int k = threadIdx.x; k < 128; k += blockDim.x) accept[k / 64][k % 64] = 0;
        __syncthreads();
        const int np = (nt - parity) / 2;
        for (int id = threadIdx.x; id < 2 * np; id += blockDim.x) {
            const int r = id / np;
            const int p = parity + 2 * (id % np);
            int64_t *Bp = a.B + s * 2 * Tp + r * Tp + p;
            int64_t *Mp = a.M + s * 2 * Tp + r * Tp + p;
            const long long dB = Bp[0] - Bp[1];
            const long long dM = Mp[0] - Mp[1];
            const float t1 = __fmul_rn(__ll2float_rn(dB), a.qJ_f);
            const float t2 = __fmul_rn(a.h_f, __ll2float_rn(dM));
            const float dE = -__fadd_rn(t1, t2);
            const float D = __fmul_rn(a.dbeta[p], dE);
            const u32x4 o = philox10(a.seed_lo ^ kTagExc, (uint32_t)(s + a.s_key0), (uint32_t)p, call_id,
                                     (uint32_t)r | 0x100u, a.seed_hi);
            if ((D >= 0.0f) || (o.v[0] <= thr_of_logp(D))) {
                accept[r][p] = 1;
                const int64_t tb = Bp[0];
                Bp[0] = Bp[1];
                Bp[1] = tb;
                const int64_t tm = Mp[0];
                Mp[0] = Mp[1];
                Mp[1] = tm;
            }
        }
        __syncthreads();
        uint8_t *sp = a.spins + (size_t)s * N * RB;
        for (int id = threadIdx.x; id < N * 2 * (nt / 2 + 1); id += blockDim.x) {
            const int i = id % N;
            const int rest = id / N;
            const int r = rest % 2;
            const int p = parity + 2 * (rest / 2);
            if (p + 1 >= nt || !accept[r][p]) continue;
            uint8_t *row = sp + (size_t)i * RB;
            const uint8_t tv = row[slot_byte(r, p)];
            row[slot_byte(r, p)] = row[slot_byte(r, p + 1)];
            row[slot_byte(r, p + 1)] = tv;
        }
    }
}

// q(k) for arbitrary integer k: one thread per (sample, slot, k).
__global__ void measure_k_kernel(const Int8Args a, int L, const int *kv, int nk, float *out)
{
    const int N = L * L * L;
    const int RB = 2 * a.Tp;
    const int64_t total = (a.s_end - a.s_begin) * a.nt * (int64_t)nk;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(g % nk);
        const int t = (int)((g / nk) % a.nt);
        const int64_t s = a.s_begin + g / ((int64_t)nk * a.nt);
        const uint8_t *sp = a.spins + (size_t)s * N * RB;
        float re = 0.0f, im = 0.0f;
        for (int i = 0; i < N; ++i) {
            const int x = i % L, y = (i / L) % L, z = i / (L * L);
            const int q = (sp[(size_t)i * RB + slot_byte(0, t)] ^ sp[(size_t)i * RB + slot_byte(1, t)]) ? -1 : 1;
            int ph = (kv[3 * j] * x + kv[3 * j + 1] * y + kv[3 * j + 2] * z) % L;
            if (ph < 0) ph += L;
            float sn, cs;
            sincospif(2.0f * (float)ph / (float)L, &sn, &cs);
            re += q * cs;
            im += q * sn;
        }
        out[2 * g] = re / (float)N;
        out[2 * g + 1] = im / (float)N;
    }
}

__global__ void thr_map_kernel(const float *x, int n, uint32_t *out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = thr_of_logp(x[k]);
}

// Metropolis decision of the Gaussian sweep for (x, r) pairs: the screen,
// and the exact threshold where the screen is undecided. out bit 0: accept;
// bit 1: the screen was undecided.
// The sweep's decision for each (x, r): screen_pair (the packed screen of
// the Gaussian sweep's chain pairs) on the entries 2m and 2m + 1, and the
// exact threshold where the entry's draw falls in the band.
__global__ void accept_map_kernel(const float *x, const uint32_t *r, int n, uint8_t *out)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; 2 * m < n; m += gridDim.x * blockDim.x) {
        const int k[2] = {2 * m, 2 * m + 1 < n ? 2 * m + 1 : 2 * m};
        bool amb[2];
        float u[2];
        screen_pair(f2_pack(x[k[0]], x[k[1]]), r[k[0]], r[k[1]], amb[0], amb[1], u[0], u[1]);
        for (int q = 0; q < 2; ++q) {
            const bool acc = amb[q] ? (r[k[q]] <= thr_of_logp(x[k[q]])) : (__float_as_uint(u[q]) >> 31) != 0u;
            out[k[q]] = (uint8_t)((acc ? 1 : 0) | (amb[q] ? 2 : 0));
        }
    }
}

__global__ void advance_kernel(int64_t *ctr, int64_t n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += n;
}

// Packed state <-> byte per chain: rows = S * N site rows of WR groups; a
// packed byte holds one group's 8 chains (see load_packed / store_packed).
__global__ void pack_spins_kernel(uint8_t *packed, const uint8_t *unpacked, int64_t n_bytes,
                                  const int *skip)
{
    if (skip && *skip) return;  // an upload that failed its check: keep the state
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_bytes;
         g += (int64_t)gridDim.x * blockDim.x)
        store_packed(packed + g, *reinterpret_cast<const uint2 *>(unpacked + 8 * g));
}

__global__ void unpack_spins_kernel(uint8_t *unpacked, const uint8_t *packed, int64_t n_bytes)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_bytes;
         g += (int64_t)gridDim.x * blockDim.x)
        *reinterpret_cast<uint2 *>(unpacked + 8 * g) = load_packed(packed + g);
}

// Accumulators: canonical [S][nt][nb][40] <-> device [S][nb][40][nt].
__global__ void acc_layout_kernel(double *dst, const double *src, int64_t S, int nt, int nb,
                                  int to_dev)
{
    const int64_t total = S * (int64_t)nt * nb * SG_NACC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        // e runs over the canonical index ((s * nt + t) * nb + bin) * 40 + k
        const int k = (int)(e % SG_NACC);
        const int bin = (int)((e / SG_NACC) % nb);
        const int t = (int)((e / ((int64_t)SG_NACC * nb)) % nt);
        const int64_t s = e / ((int64_t)SG_NACC * nb * nt);
        const int64_t d = ((s * nb + bin) * SG_NACC + k) * nt + t;
        if (to_dev)
            dst[d] = src[e];
        else
            dst[e] = src[d];
    }
}

// Sets *flag when any of the n bytes is neither +1 nor -1. Eight bytes per
// step: x = w ^ 0x01.. has every byte 0x00 (for +1) or 0xFE (for -1) exactly
// when all bytes are valid.
__global__ void check_pm1_kernel(const int8_t *c, int64_t n, int *flag, int *status)
{
    const uint64_t ones = 0x0101010101010101ull;
    const int64_t words = n / 8;
    const uint64_t *w = reinterpret_cast<const uint64_t *>(c);
    bool bad = false;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < words;
         g += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = w[g] ^ ones;
        const uint64_t z = (x >> 1) & 0x7F7F7F7F7F7F7F7Full;  // 0x00 or 0x7F per valid byte
        bad |= ((x & ones) | ((z + ones) & 0x7E7E7E7E7E7E7E7Eull)) != 0;
    }
    for (int64_t k = 8 * words + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        bad |= c[k] != 1 && c[k] != -1;
    if (bad) {
        atomicOr(flag, 1);
        if (status) atomicCAS(status, 0, (int)SG_EINVAL);
    }
}

inline int grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 148 * 32) b = 148 * 32;
    return (int)b;
}

#define SG_FOR_EACH_L(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16)

}  // namespace

size_t int8_smem_bytes(int L, int Tp, bool gauss, int mchunk, bool gst)
{
    bool ok = false;
#define X(LL) ok |= (L == LL);
    if (gst) ok = int8_gst_has(L); else { SG_FOR_EACH_L(X) }
#undef X
    if (!ok) return 0;
    size_t b = carve(nullptr, L, Tp, gauss, mchunk, nullptr, gst);
    return b <= (size_t)kMaxSmem ? b : 0;
}

int int8_thread_quantum(int Tp, bool gst)
{
    // a half-sweep thread keeps one (4-slot group, replica) pair, Tp/4 * 2;
    // on the packed state of the global-memory instances one 4-slot group
    // with both replicas, Tp/4
    return gst ? Tp / 4 : Tp / 2;
}

int int8_site_run(int, bool)
{
    return kSiteRun;  // one Philox group, in both state layouts
}

int int8_max_threads(int L, bool gst, bool wide)
{
    if (gst) return KernelBounds<10, true>::threads;  // the same for every L
    if (wide) return int8_wide_has(L) ? KernelBounds<12, false, true>::threads : 0;
    if (L <= 8) return KernelBounds<8, false>::threads;
    if (L <= 12) return KernelBounds<12, false>::threads;
    return KernelBounds<16, false>::threads;
}

cudaError_t int8_launch(int L, bool gauss, const Int8Args &a, const Int8Launch &cfg,
                        cudaStream_t st)
{
    if (cfg.bits) return int8_launch_bits(L, gauss, a, cfg, st);
    if (cfg.gst && cfg.cluster > 1) return int8_launch_cluster(L, gauss, a, cfg, st);
    if (cfg.gst) return int8_launch_gst(L, gauss, a, cfg, st);
    if (cfg.wide) return int8_launch_wide(L, gauss, a, cfg, st);
#define X(LL)                                                                          \
    if (L == LL)                                                                       \
        return gauss ? launch_t<LL, true, false>(a, cfg, st) : launch_t<LL, false, false>(a, cfg, st);
    SG_FOR_EACH_L(X)
#undef X
    return cudaErrorInvalidValue;
}

int int8_ctas_per_sm(int L, bool gauss, int threads, size_t smem, bool gst, bool wide)
{
    if (gst) return int8_ctas_per_sm_gst(L, gauss, threads, smem);
    if (wide) return int8_ctas_per_sm_wide(L, gauss, threads, smem);
#define X(LL) \
    if (L == LL) return gauss ? occ_t<LL, true, false>(threads, smem) : occ_t<LL, false, false>(threads, smem);
    SG_FOR_EACH_L(X)
#undef X
    return 0;
}

cudaError_t int8_gen_pmj(uint8_t *J8, int64_t S, int L, uint32_t slo, uint32_t shi,
                         int64_t key0, cudaStream_t st)
{
    gen_pmj_kernel<<<grid_for(S * L * L * L, 256), 256, 0, st>>>(J8, S, L, slo, shi, key0);
    return cudaGetLastError();
}

cudaError_t int8_gen_gauss(float *Jg, int64_t S, int L, uint32_t slo, uint32_t shi,
                           int64_t key0, cudaStream_t st)
{
    gen_gauss_kernel<<<grid_for(S * 3 * (L * L * L + 1) / 2, 256), 256, 0, st>>>(Jg, S, L, slo,
                                                                                  shi, key0);
    return cudaGetLastError();
}

cudaError_t int8_gen_spins(uint8_t *spins, int64_t S, int L, int nt, int Tp, uint32_t slo,
                           uint32_t shi, int64_t key0, cudaStream_t st)
{
    gen_spins_kernel<<<grid_for(S * L * L * L * 2 * Tp, 256), 256, 0, st>>>(spins, S, L, nt, Tp,
                                                                             slo, shi, key0);
    return cudaGetLastError();
}

cudaError_t int8_import_J(uint8_t *J8, float *Jg, const float *Jc, int64_t S, int L, bool gauss,
                          cudaStream_t st)
{
    import_J_kernel<<<grid_for(S * L * L * L, 256), 256, 0, st>>>(J8, Jg, Jc, S, L, gauss);
    return cudaGetLastError();
}

cudaError_t int8_export_J(float *Jc, const uint8_t *J8, const float *Jg, int64_t S, int L,
                          bool gauss, cudaStream_t st)
{
    export_J_kernel<<<grid_for(S * 3 * L * L * L, 256), 256, 0, st>>>(Jc, J8, Jg, S, L, gauss);
    return cudaGetLastError();
}

cudaError_t int8_import_spins(uint8_t *spins, const int8_t *c, int64_t S, int L, int nt, int Tp,
                              cudaStream_t st, const int *skip)
{
    import_spins_kernel<<<grid_for(S * L * L * L * 2 * Tp, 256), 256, 0, st>>>(spins, c, S, L,
                                                                                nt, Tp, skip);
    return cudaGetLastError();
}

cudaError_t int8_export_spins(int8_t *c, const uint8_t *spins, int64_t S, int L, int nt, int Tp,
                              cudaStream_t st)
{
    export_spins_kernel<<<grid_for(S * 2 * nt * L * L * L, 256), 256, 0, st>>>(c, spins, S, L,
                                                                                nt, Tp);
    return cudaGetLastError();
}

cudaError_t int8_energies(const Int8Args &a, int L, bool gauss, cudaStream_t st)
{
    energies_kernel<<<grid_for((a.s_end - a.s_begin) * 2 * a.Tp, 128), 128, 0, st>>>(a, L, gauss);
    return cudaGetLastError();
}

cudaError_t int8_exchange(const Int8Args &a, int L, bool gauss, int parity, uint32_t call_id,
                          cudaStream_t st)
{
    cudaError_t e = int8_energies(a, L, gauss, st);
    if (e != cudaSuccess) return e;
    const int64_t n = a.s_end - a.s_begin;
    exchange_kernel<<<(int)(n < 148 * 16 ? n : 148 * 16), 256, 0, st>>>(a, L, parity & 1, call_id);
    return cudaGetLastError();
}

cudaError_t threshold_map(const float *x, int n, uint32_t *out, cudaStream_t st)
{
    thr_map_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t accept_map(const float *x, const uint32_t *r, int n, uint8_t *out, cudaStream_t st)
{
    accept_map_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, r, n, out);
    return cudaGetLastError();
}

cudaError_t int8_pack_spins(uint8_t *packed, const uint8_t *unpacked, int64_t S, int L, int Tp,
                            cudaStream_t st, const int *skip)
{
    const int64_t n = S * L * L * L * (int64_t)(Tp / 4);
    pack_spins_kernel<<<grid_for(n, 256), 256, 0, st>>>(packed, unpacked, n, skip);
    return cudaGetLastError();
}

cudaError_t int8_unpack_spins(uint8_t *unpacked, const uint8_t *packed, int64_t S, int L, int Tp,
                              cudaStream_t st)
{
    const int64_t n = S * L * L * L * (int64_t)(Tp / 4);
    unpack_spins_kernel<<<grid_for(n, 256), 256, 0, st>>>(unpacked, packed, n);
    return cudaGetLastError();
}

cudaError_t int8_acc_layout(double *dst, const double *src, int64_t S, int nt, int nb, bool to_dev,
                            cudaStream_t st)
{
    acc_layout_kernel<<<grid_for(S * nt * nb * SG_NACC, 256), 256, 0, st>>>(dst, src, S, nt, nb,
                                                                            to_dev ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t check_pm1(const int8_t *c, size_t n, int *flag, int *status, cudaStream_t st)
{
    // c comes from cudaMalloc (8-byte aligned); one 8-byte word per thread step
    check_pm1_kernel<<<grid_for((int64_t)(n / 8 + 1), 256), 256, 0, st>>>(c, (int64_t)n, flag,
                                                                         status);
    return cudaGetLastError();
}

cudaError_t advance_counter(int64_t *ctr, int64_t n, cudaStream_t st)
{
    advance_kernel<<<1, 32, 0, st>>>(ctr, n);
    return cudaGetLastError();
}

cudaError_t int8_measure_k(const Int8Args &a, int L, const int *k_dev, int nk, float *out,
                           cudaStream_t st)
{
    measure_k_kernel<<<grid_for((a.s_end - a.s_begin) * a.nt * nk, 128), 128, 0, st>>>(a, L, k_dev,
                                                                                        nk, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the arbitrary-k overlap measurement.
//
// Some callers cannot allocate device memory at the point where they want a
// measurement: serving loops that must not touch the allocator (and its
// device-wide synchronisation) on their latency path, and hosts whose device
// memory belongs to another framework's pool, where a stray cudaMalloc
// competes with that pool. For them the k-vector and output staging live in
// this file-scope device array instead of cudaMalloc'd buffers. Every device
// that loads the library holds the array until the process exits.
//
// In host code the array's name is only a host-side stand-in, never a device
// address: the device address comes from cudaGetSymbolAddress, taken once per
// device with that device current (on the first call made on that device;
// the caller has checked that the ensemble's device is the current one).
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocKBytes = 4096;  // room for SG_MEASURE_NOALLOC_MAX_K vectors
constexpr size_t kNoAllocBytes = kNoAllocKBytes + (size_t)SG_MEASURE_NOALLOC_MAX_FLOATS * 4;
static_assert(3 * sizeof(int) * SG_MEASURE_NOALLOC_MAX_K <= kNoAllocKBytes, "k staging");

__device__ __align__(256) unsigned char g_measure_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of g_measure_scratch on the current device (set up once).
cudaError_t scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_measure_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t int8_measure_k_noalloc(const Int8Args &a, int L, const int *k_host, int nk,
                                   float *out_host, size_t out_floats, cudaStream_t st)
{
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return e;
    int *kd = reinterpret_cast<int *>(scratch);
    float *od = reinterpret_cast<float *>(scratch + kNoAllocKBytes);
    e = cudaMemcpyAsync(kd, k_host, sizeof(int) * 3 * (size_t)nk, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    // every output element is written by the kernel, so nothing needs clearing
    measure_k_kernel<<<grid_for((a.s_end - a.s_begin) * a.nt * nk, 128), 128, 0, st>>>(a, L, kd,
                                                                                        nk, od);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out_host, od, sizeof(float) * out_floats, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace sg
