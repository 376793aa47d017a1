// sg_analysis.cpp -- disorder and thermal averages of the measured overlaps.
//
// Paper, methods section: Binder ratio g (eq. binder) with the overlap centred
// on its disorder average; chi_SG(k) = N([<|q(k)|^2>] - |[<q(k)>]|^2)
// (eq. chi); xi_L = sqrt(chi(0)/chi(k_min) - 1) / (2 sin(|k_min|/2))
// (eq. corr); R12 = chi(k1)/chi(k2) (eq. r12). chi at k1 and k2 is averaged
// over the equivalent directions (results section: point-group averaging),
// and every error bar is a delete-one jackknife over disorder samples
// (methods section).
#include <cmath>
#include <vector>

#include "sg_internal.h"

namespace {

struct Means {
    double q1, q2, q3, q4, e;
    double re[9], im[9], ab[9];
};

struct Obs {
    double g, chi0, chi1, chi2, xi, r12, e, q2, q4;
};

Obs from_means(const Means &m, int L)
{
    const double N = (double)L * L * L;
    Obs o;
    const double mu = m.q1;
    const double c2 = m.q2 - 2.0 * mu * m.q1 + mu * mu;
    const double c4 = m.q4 - 4.0 * mu * m.q3 + 6.0 * mu * mu * m.q2 - 4.0 * mu * mu * mu * m.q1 +
                      mu * mu * mu * mu;
    o.g = 0.5 * (3.0 - c4 / (c2 * c2));
    o.chi0 = N * (m.q2 - m.q1 * m.q1);
    double chik[9];
    for (int v = 0; v < 9; ++v) chik[v] = N * (m.ab[v] - (m.re[v] * m.re[v] + m.im[v] * m.im[v]));
    o.chi1 = (chik[0] + chik[1] + chik[2]) / 3.0;
    o.chi2 = (chik[3] + chik[4] + chik[5] + chik[6] + chik[7] + chik[8]) / 6.0;
    const double ratio = o.chi0 / o.chi1;
    o.xi = ratio >= 1.0 ? std::sqrt(ratio - 1.0) / (2.0 * std::sin(M_PI / L)) : NAN;
    o.r12 = o.chi1 / o.chi2;
    o.e = m.e;
    o.q2 = m.q2;
    o.q4 = m.q4;
    return o;
}

// Per-sample thermal means of one slot.
Means sample_means(const double *a, int L)
{
    const double N = (double)L * L * L;
    const double n = a[SG_ACC_COUNT];
    Means m;
    m.q1 = a[SG_ACC_Q1] / n / N;
    m.q2 = a[SG_ACC_Q2] / n / (N * N);
    m.q3 = a[SG_ACC_Q3] / n / (N * N * N);
    m.q4 = a[SG_ACC_Q4] / n / (N * N * N * N);
    m.e = a[SG_ACC_E1] / (2.0 * n) / N;
    for (int v = 0; v < 9; ++v) {
        m.re[v] = a[SG_ACC_K + 3 * v] / n / N;
        m.im[v] = a[SG_ACC_K + 3 * v + 1] / n / N;
        m.ab[v] = a[SG_ACC_K + 3 * v + 2] / n / (N * N);
    }
    return m;
}

void add(Means &s, const Means &x, double w)
{
    s.q1 += w * x.q1;
    s.q2 += w * x.q2;
    s.q3 += w * x.q3;
    s.q4 += w * x.q4;
    s.e += w * x.e;
    for (int v = 0; v < 9; ++v) {
        s.re[v] += w * x.re[v];
        s.im[v] += w * x.im[v];
        s.ab[v] += w * x.ab[v];
    }
}

Means scaled(const Means &x, double f)
{
    Means z = {};
    add(z, x, f);
    return z;
}

}  // namespace

extern "C" sg_status sg_observables_from_acc(const double *acc, int64_t S, int nt, int L,
                                             const sg_observables *out)
{
    if (!acc || !out || S < 1 || nt < 1 || L < 2) return SG_EINVAL;
    for (int t = 0; t < nt; ++t) {
        std::vector<Means> ms((size_t)S);
        Means sum = {};
        for (int64_t s = 0; s < S; ++s) {
            ms[(size_t)s] = sample_means(acc + ((size_t)s * nt + t) * SG_NACC, L);
            add(sum, ms[(size_t)s], 1.0);
        }
        const Obs full = from_means(scaled(sum, 1.0 / (double)S), L);
        double err[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (S > 1) {
            std::vector<Obs> jk((size_t)S);
            Obs mean = {};
            for (int64_t s = 0; s < S; ++s) {
                Means loo = sum;
                add(loo, ms[(size_t)s], -1.0);
                jk[(size_t)s] = from_means(scaled(loo, 1.0 / (double)(S - 1)), L);
                const Obs &o = jk[(size_t)s];
                mean.g += o.g; mean.chi0 += o.chi0; mean.chi1 += o.chi1; mean.chi2 += o.chi2;
                mean.xi += o.xi; mean.r12 += o.r12; mean.e += o.e; mean.q2 += o.q2;
                mean.q4 += o.q4;
            }
            const double f = 1.0 / (double)S;
            mean.g *= f; mean.chi0 *= f; mean.chi1 *= f; mean.chi2 *= f; mean.xi *= f;
            mean.r12 *= f; mean.e *= f; mean.q2 *= f; mean.q4 *= f;
            for (int64_t s = 0; s < S; ++s) {
                const Obs &o = jk[(size_t)s];
                const double d[9] = {o.g - mean.g, o.chi0 - mean.chi0, o.chi1 - mean.chi1,
                                     o.chi2 - mean.chi2, o.xi - mean.xi, o.r12 - mean.r12,
                                     o.e - mean.e, o.q2 - mean.q2, o.q4 - mean.q4};
                for (int k = 0; k < 9; ++k) err[k] += d[k] * d[k];
            }
            for (int k = 0; k < 9; ++k) err[k] = std::sqrt((double)(S - 1) / (double)S * err[k]);
        }
        const double vals[9] = {full.g, full.chi0, full.chi1, full.chi2, full.xi,
                                full.r12, full.e, full.q2, full.q4};
        double *dst[9] = {out->g, out->chi0, out->chi1, out->chi2, out->xi,
                          out->r12, out->e, out->q2, out->q4};
        double *dst_err[9] = {out->g_err, out->chi0_err, out->chi1_err, out->chi2_err,
                              out->xi_err, out->r12_err, out->e_err, out->q2_err, out->q4_err};
        for (int k = 0; k < 9; ++k) {
            if (dst[k]) dst[k][t] = vals[k];
            if (dst_err[k]) dst_err[k][t] = err[k];
        }
    }
    return SG_OK;
}
