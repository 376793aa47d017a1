"""CPU pins of the oracle's logarithmic sweep bins and overlap histogram.

The bins implement the logarithmic-binning equilibration test (figure of R12
against the number of sweeps): the measurement of global sweep n goes to bin
floor(log2(n + 1)), the last bin also taking every later sweep. The histogram
is the distribution P(q) of the overlap the conclusion proposes to analyse.

Pins (none retypes the oracle's code):
  * the bin populations equal a closed-form count made with Python's
    int.bit_length, for several n_therm / measure_every / bin counts;
  * binning does not change the chain, and summed over bins the integer-valued
    accumulators equal the unbinned run's exactly;
  * the histogram, counted from agreeing sites, reproduces the zeroth to
    fourth moments of Q = sum_i q_i that the accumulators hold (Q from the
    marginals), per slot and bin;
  * very high T: each sample's overlap is frozen at its random start, so the
    counts over samples follow Binomial(N, 1/2) (chi-square test);
  * strong field, low T: both replicas align with the field, so all the mass
    sits at q = 1 (k = N), which fixes the orientation of the index.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1403_4560_b300 import inputs

A_N, A_Q1, A_Q2, A_Q3, A_Q4 = 0, 1, 2, 3, 4
A_E1, A_E2, A_M1, A_M2 = 5, 6, 7, 8


def make(L, S, nt, dist="pmj", h=0.3, T=None, seed=5, **kw):
    T = inputs.geometric_ladder(0.6, 1.6, nt) if T is None else np.asarray(T, float)
    J, s0 = inputs.make_instance(dist, L, S, len(T), seed)
    return O.State(L, T, h, dist == "gauss", seed, J, s0, **kw)


def expected_bins(n_sweeps, n_therm, measure_every, n_bins):
    cnt = np.zeros(n_bins, dtype=np.int64)
    for n in range(n_sweeps):
        if n >= n_therm and (n - n_therm) % measure_every == 0:
            cnt[min((n + 1).bit_length() - 1, n_bins - 1)] += 1
    return cnt


@pytest.mark.parametrize("n_sweeps,n_therm,every,bins", [
    (64, 0, 1, 7), (100, 0, 1, 5), (37, 5, 3, 8), (20, 0, 1, 1), (9, 0, 2, 64)])
def test_bin_populations_closed_form(n_sweeps, n_therm, every, bins):
    st = make(2, 3, 2, n_therm=n_therm, measure_every=every, log_bins=bins)
    st.run(n_sweeps // 2)
    st.run(n_sweeps - n_sweeps // 2)  # bins follow the global sweep index
    acc = st.acc.reshape(3, 2, bins, O.NACC)
    want = expected_bins(n_sweeps, n_therm, every, bins)
    for s in range(3):
        for t in range(2):
            np.testing.assert_array_equal(acc[s, t, :, A_N], want)


@pytest.mark.parametrize("dist", ["pmj", "gauss"])
def test_binning_keeps_chain_and_sums(dist):
    a = make(4, 4, 3, dist=dist, n_therm=3)
    b = make(4, 4, 3, dist=dist, n_therm=3, log_bins=6, pq_hist=True)
    a.run(70, threads=2)
    b.run(70, threads=2)
    np.testing.assert_array_equal(a.spins, b.spins)
    np.testing.assert_array_equal(a.B, b.B)
    summed = b.acc.sum(axis=2)
    exact = [A_N, A_Q1, A_Q2, A_Q3, A_Q4, A_M1, A_M2]  # integer-valued sums
    np.testing.assert_array_equal(summed[..., exact], a.acc[..., exact])
    np.testing.assert_allclose(summed, a.acc, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("L,dist,h", [(2, "pmj", 0.5), (4, "gauss", 0.2), (6, "pmj", 0.0)])
def test_histogram_moments_match_accumulators(L, dist, h):
    st = make(L, 5, 4, dist=dist, h=h, n_therm=2, log_bins=4, pq_hist=True)
    st.run(23, threads=3)
    N = L ** 3
    Q = 2.0 * np.arange(N + 1) - N
    for t in range(4):
        for b in range(4):
            hb = st.hist[t, b].astype(np.float64)
            for p, idx in enumerate([A_N, A_Q1, A_Q2, A_Q3, A_Q4]):
                assert np.dot(hb, Q ** p) == st.acc[:, t, b, idx].sum()


def test_high_temperature_histogram_is_binomial():
    L, S = 2, 4000
    N = L ** 3
    st = make(L, S, 1, T=[1e6], h=0.0, seed=11, pq_hist=True)
    st.run(1, threads=8)
    counts = st.hist[0, 0].astype(np.float64)
    assert counts.sum() == S
    p = stats.binom.pmf(np.arange(N + 1), N, 0.5)
    chi2 = ((counts - S * p) ** 2 / (S * p)).sum()
    assert chi2 < stats.chi2.ppf(0.999, N)


def test_strong_field_low_temperature_concentrates_at_q_one():
    L, S = 4, 16
    N = L ** 3
    st = make(L, S, 2, T=[0.2, 0.3], h=8.0, seed=3, n_therm=10, pq_hist=True)
    st.run(30)
    h = st.hist[:, 0]
    assert h[:, N].sum() == h.sum() == 2 * S * 20
