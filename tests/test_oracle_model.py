"""Pins for the oracle's model, Metropolis rule, exchange and measurement.

Every check compares the oracle with something other than itself: the
Hamiltonian evaluated on a 3D numpy array with periodic rolls, closed forms,
exact enumeration of L = 2 lattices, and exact symmetries of the model.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1403_4560_b300 import inputs


def energy_numpy(L, J, s, h):
    """H = -sum_<ij> J s_i s_j - h sum s_i on a periodic L^3 array (eq. Hamiltonian).

    Arrays are indexed [z][y][x] so that site i = x + L*(y + L*z)."""
    S = s.reshape(L, L, L).astype(np.float64)
    Jr = J.reshape(3, L, L, L).astype(np.float64)
    e = 0.0
    for d, axis in ((0, 2), (1, 1), (2, 0)):
        e -= (Jr[d] * S * np.roll(S, -1, axis=axis)).sum()
    return e - h * S.sum()


@pytest.mark.parametrize("L,gauss", [(2, False), (4, False), (6, True), (4, True)])
def test_bond_sum_matches_hamiltonian(L, gauss):
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, 3, 2, seed=5)
    for k in range(3):
        s = s0[k, 1, 1]
        B, M = orc.bond_sum(L, gauss, J[k], s)
        qJ = 2.0 ** -17 if gauss else 1.0
        h = 0.37
        e = -(B * qJ + h * M)
        assert e == pytest.approx(energy_numpy(L, J[k], s, h), rel=1e-12, abs=1e-9)
        assert M == int(s.astype(np.int64).sum())


@pytest.mark.parametrize("L,gauss", [(4, False), (6, False), (4, True), (2, True)])
def test_local_field_delta_e_is_energy_difference(L, gauss):
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, 1, 1, seed=9)
    h = 0.21
    rng = np.random.default_rng(3)
    s = s0[0, 0, 0].copy()
    for _ in range(40):
        i = int(rng.integers(L ** 3))
        flipped = s.copy()
        flipped[i] = -flipped[i]
        want = energy_numpy(L, J[0], flipped, h) - energy_numpy(L, J[0], s, h)
        assert orc.delta_e(L, h, J[0], s, i) == pytest.approx(want, abs=1e-9)
        s = flipped if rng.random() < 0.5 else s


def test_threshold_table_closed_form():
    T = np.array([0.5, 1.0, 2.0])
    h = 0.3
    thr = orc.thresholds(h, T)
    for t, Tt in enumerate(T):
        for sb in (0, 1):
            for u in range(7):
                dE = (12 - 4 * u) + (-2 * h if sb else 2 * h)
                if dE <= 0:
                    assert thr[t, sb, u] == 0xFFFFFFFF
                else:
                    want = math.exp(-dE / Tt) * 2 ** 32
                    assert abs(int(thr[t, sb, u]) - want) <= 1.0
    # infinite temperature: every move accepted
    assert np.all(orc.thresholds(0.7, [1e300]) == 0xFFFFFFFF)


def _all_configs(N):
    return np.array([[1 - 2 * ((c >> i) & 1) for i in range(N)]
                     for c in range(2 ** N)], dtype=np.int8)


def _sweep_matrix(L, gauss, h, T, J):
    """Exact one-sweep transition matrix of one chain at L = 2 (colour 0 then 1),
    built from the oracle's per-site acceptance thresholds: P(accept) =
    (thr + 1)/2^32."""
    N = L ** 3
    cfgs = _all_configs(N)
    index = {tuple(c): k for k, c in enumerate(cfgs)}
    thr_t = orc.thresholds(h, [T])[0]
    colour = [(i % L + (i // L) % L + i // (L * L)) % 2 for i in range(N)]
    P = np.eye(2 ** N)
    for c in (0, 1):
        Pc = np.zeros((2 ** N, 2 ** N))
        for a, cfg in enumerate(cfgs):
            # sites of one colour are independent given the other colour
            sites = [i for i in range(N) if colour[i] == c]
            probs = []
            for i in sites:
                th = orc.site_threshold(L, gauss, h, T, thr_t, J, cfg, i)
                probs.append((th + 1) / 2 ** 32)
            for flips in itertools.product((0, 1), repeat=len(sites)):
                p = 1.0
                new = cfg.copy()
                for f, i, pa in zip(flips, sites, probs):
                    p *= pa if f else (1 - pa)
                    if f:
                        new[i] = -new[i]
                Pc[a, index[tuple(new)]] += p
        P = P @ Pc
    return cfgs, P


@pytest.mark.parametrize("gauss,h,T", [(False, 0.3, 0.9), (True, 0.25, 1.3), (False, 0.0, 0.6)])
def test_l2_sweep_leaves_boltzmann_stationary(gauss, h, T):
    L = 2
    J, _ = inputs.make_instance("gauss" if gauss else "pmj", L, 1, 1, seed=21)
    cfgs, P = _sweep_matrix(L, gauss, h, T, J[0])
    hq = np.rint(h * 2 ** 17) / 2 ** 17 if gauss else h
    E = np.array([energy_numpy(L, J[0], c, hq) for c in cfgs])
    w = np.exp(-(E - E.min()) / T)
    pi = w / w.sum()
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    # acceptance probabilities carry the 2^-32 rounding of the threshold table
    np.testing.assert_allclose(pi @ P, pi, atol=1e-8)


def _exact_l2(J, h, T, gauss):
    """Exact thermal averages of two independent replicas at L = 2."""
    L, N = 2, 8
    cfgs = _all_configs(N)
    hq = np.rint(h * 2 ** 17) / 2 ** 17 if gauss else h
    E = np.array([energy_numpy(L, J, c, hq) for c in cfgs])
    out = []
    coords = np.array([[i % L, (i // L) % L, i // (L * L)] for i in range(N)])
    for Tt in T:
        w = np.exp(-(E - E.min()) / Tt)
        pi = w / w.sum()
        q = (cfgs[:, None, :].astype(np.float64) * cfgs[None, :, :]) / N  # [a][b][i]
        q0 = q.sum(axis=-1)
        pab = pi[:, None] * pi[None, :]
        phase = np.exp(1j * 2 * np.pi / L * coords @ orc.KVECS.T)  # [i][v]
        qk = q @ phase  # [a][b][v]
        out.append({"e": (pi * E).sum() / N, "q2": (pab * q0 ** 2).sum(),
                    "q4": (pab * q0 ** 4).sum(),
                    "qk2": (pab[..., None] * np.abs(qk) ** 2).sum(axis=(0, 1)),
                    "m": (pi * cfgs.sum(axis=1)).sum() / N})
    return out


@pytest.mark.slow
@pytest.mark.parametrize("gauss", [False, True])
def test_l2_parallel_tempering_reproduces_exact_averages(gauss):
    """Monte Carlo with PT on one L = 2 disorder realisation, 48 independent
    chains, against exact enumeration (within 4.5 standard errors)."""
    L, S = 2, 48
    T = inputs.geometric_ladder(0.5, 2.0, 4)
    h = 0.3
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, S, len(T), seed=33,
                                 same_couplings=True)
    st = orc.State(L, T, h, gauss, seed=77, J=J, spins=s0, n_therm=200)
    st.run(2200, threads=4)
    tm = orc.thermal_means(st.acc, L)
    exact = _exact_l2(J[0], h, T, gauss)
    for t in range(len(T)):
        for key, ex in (("e1", exact[t]["e"]), ("q2", exact[t]["q2"]),
                        ("q4", exact[t]["q4"]), ("m1", exact[t]["m"])):
            vals = tm[key][:, t]
            se = vals.std(ddof=1) / math.sqrt(S)
            assert abs(vals.mean() - ex) < 4.5 * se + 1e-12, (key, t, vals.mean(), ex, se)
        vals = tm["qk_abs2"][:, t, :]
        se = vals.std(axis=0, ddof=1) / math.sqrt(S)
        assert np.all(np.abs(vals.mean(axis=0) - exact[t]["qk2"]) < 4.5 * se + 1e-12)


def _run(L, T, h, gauss, seed, J, s0, sweeps, **kw):
    st = orc.State(L, T, h, gauss, seed=seed, J=J, spins=s0, **kw)
    st.run(sweeps)
    return st


@pytest.mark.parametrize("gauss", [False, True])
def test_gauge_symmetry_is_exact_at_zero_field(gauss):
    """J_d[i] -> e_i e_{i+d} J_d[i], s -> e s maps trajectories exactly at h = 0."""
    L = 4
    T = inputs.geometric_ladder(0.5, 1.5, 4)
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, 2, len(T), seed=2)
    rng = np.random.default_rng(4)
    eps = (1 - 2 * rng.integers(0, 2, size=(2, L ** 3))).astype(np.int8)
    Jg = J.copy()
    for s in range(2):
        e3 = eps[s].reshape(L, L, L)
        for d, axis in ((0, 2), (1, 1), (2, 0)):
            Jg[s, d] *= (e3 * np.roll(e3, -1, axis=axis)).reshape(-1)
    s0g = s0 * eps[:, None, None, :]
    a = _run(L, T, 0.0, gauss, 5, J, s0, 60)
    b = _run(L, T, 0.0, gauss, 5, Jg, s0g, 60)
    np.testing.assert_array_equal(b.spins, a.spins * eps[:, None, None, :])
    np.testing.assert_array_equal(b.B, a.B)
    for k in [orc.A_N, orc.A_Q1, orc.A_Q2, orc.A_Q3, orc.A_Q4, orc.A_E1, orc.A_E2] + list(
            range(9, 36)):
        np.testing.assert_array_equal(b.acc[..., k], a.acc[..., k])


@pytest.mark.parametrize("gauss", [False, True])
def test_global_flip_with_reversed_field_is_exact(gauss):
    L = 4
    T = inputs.geometric_ladder(0.4, 1.6, 4)
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, 2, len(T), seed=8)
    a = _run(L, T, 0.3, gauss, 6, J, s0, 50)
    b = _run(L, T, -0.3, gauss, 6, J, -s0, 50)
    np.testing.assert_array_equal(b.spins, -a.spins)
    np.testing.assert_array_equal(b.M, -a.M)
    np.testing.assert_array_equal(b.B, a.B)
    for k in [orc.A_Q1, orc.A_Q2, orc.A_E1, orc.A_E2, orc.A_M2] + list(range(9, 36)):
        np.testing.assert_array_equal(b.acc[..., k], a.acc[..., k])
    np.testing.assert_array_equal(b.acc[..., orc.A_M1], -a.acc[..., orc.A_M1])


def test_infinite_temperature_trajectory_is_deterministic():
    """beta -> 0: every flip is accepted, so one sweep maps s to -s and q is constant."""
    L = 4
    T = np.array([1e30, 2e30])
    J, s0 = inputs.make_instance("pmj", L, 3, 2, seed=12)
    st = _run(L, T, 0.2, False, 1, J, s0, 7, exchange_every=0)
    np.testing.assert_array_equal(st.spins, -s0)
    st2 = _run(L, T, 0.2, True, 1, inputs.make_instance("gauss", L, 3, 2, seed=12)[0], s0, 4,
               exchange_every=0)
    np.testing.assert_array_equal(st2.spins, s0)
    Q = (s0[:, 0].astype(np.int64) * s0[:, 1]).sum(axis=-1)
    np.testing.assert_array_equal(st.acc[..., orc.A_Q1], 7 * Q)


def test_beta_zero_closed_forms_over_independent_spins():
    """i.i.d. spins: E[q0^2] = 1/N, E[q0^4] = (3N-2)/N^3, so g = 1/N, chi(k) = 1,
    xi = 0 and R12 = 1 (eqs. binder, chi, corr, r12), within 4 standard errors."""
    L, S = 4, 3000
    N = L ** 3
    T = np.array([1e30])
    J, s0 = inputs.make_instance("pmj", L, S, 1, seed=99)
    st = _run(L, T, 0.0, False, 3, J, s0, 2, exchange_every=0)
    obs = orc.observables(st.acc, L, jackknife=True)
    err = obs["err"]
    assert abs(obs["q2"][0] - 1 / N) < 4 * err["q2"][0]
    assert abs(obs["q4"][0] - (3 * N - 2) / N ** 3) < 4 * err["q4"][0]
    assert abs(obs["g"][0] - 1 / N) < 4 * err["g"][0]
    assert abs(obs["chi0"][0] - 1) < 4 * err["chi0"][0]
    assert abs(obs["chi_k1"][0] - 1) < 4 * err["chi_k1"][0]
    assert abs(obs["r12"][0] - 1) < 4 * err["r12"][0]


def test_overlap_projections_match_direct_fourier_sum():
    L = 6
    rng = np.random.default_rng(0)
    sa = (1 - 2 * rng.integers(0, 2, L ** 3)).astype(np.int8)
    sb = (1 - 2 * rng.integers(0, 2, L ** 3)).astype(np.int8)
    Q, re, im = orc.overlap(L, sa, sb)
    q = sa.astype(np.float64) * sb
    coords = np.array([[i % L, (i // L) % L, i // (L * L)] for i in range(L ** 3)])
    direct = (q[:, None] * np.exp(1j * 2 * np.pi / L * coords @ orc.KVECS.T)).sum(axis=0)
    assert Q == int(q.sum())
    np.testing.assert_allclose(re, direct.real, atol=2e-4)
    np.testing.assert_allclose(im, direct.imag, atol=2e-4)


def test_rng_group_shares_metropolis_numbers():
    """Samples with equal disorder and start evolve identically iff they share
    the Metropolis random numbers (same key word s / G)."""
    L = 4
    T = inputs.geometric_ladder(0.6, 1.2, 2)
    J, s0 = inputs.make_instance("pmj", L, 1, 2, seed=1)
    J2 = np.repeat(J, 2, axis=0)
    s02 = np.repeat(s0, 2, axis=0)
    shared = _run(L, T, 0.1, False, 4, J2, s02, 20, rng_group=2, exchange_every=0)
    np.testing.assert_array_equal(shared.spins[0], shared.spins[1])
    apart = _run(L, T, 0.1, False, 4, J2, s02, 20, rng_group=1, exchange_every=0)
    assert np.any(apart.spins[0] != apart.spins[1])


def test_exchange_follows_metropolis_rule_statistics():
    """Standalone PT steps between two slots at the same temperature always swap
    (D = 0 accepts) and at very different temperatures match e^D on average."""
    L = 2
    J, s0 = inputs.make_instance("pmj", L, 200, 2, seed=3)
    st = orc.State(L, np.array([1.0, 1.0]), 0.0, False, 5, J, s0)
    before = st.spins.copy()
    st.exchange(0)
    np.testing.assert_array_equal(st.spins[:, :, 0], before[:, :, 1])
    st = orc.State(L, np.array([0.5, 5.0]), 0.0, False, 5, J, s0)
    B = np.array([[orc.bond_sum(L, False, J[s], s0[s, r, t])[0] for t in range(2)]
                  for s in range(200) for r in range(2)]).reshape(200, 2, 2)
    D = (1 / 0.5 - 1 / 5.0) * (-(B[..., 0] - B[..., 1]))
    p = np.minimum(1.0, np.exp(D))
    before = st.spins.copy()
    st.exchange(0)
    swapped = np.all(st.spins[:, :, 0] == before[:, :, 1], axis=-1) & np.any(
        before[:, :, 0] != before[:, :, 1], axis=-1)
    same = np.all(before[:, :, 0] == before[:, :, 1], axis=-1)
    mask = ~same
    k = swapped[mask].sum()
    mu = p[mask].sum()
    sd = math.sqrt((p[mask] * (1 - p[mask])).sum())
    assert abs(k - mu) < 4 * sd + 1


def test_estimators_against_literal_definitions():
    """g, chi(0), chi(k), xi and R12 from the accumulators against a literal
    evaluation of eqs. binder/chi/corr/r12 over explicit per-sample samples."""
    rng = np.random.default_rng(5)
    L, N, S, n = 4, 64, 7, 50
    acc = np.zeros((S, 1, orc.NACC))
    qs = []
    qks = []
    for s in range(S):
        Q = rng.integers(-20, 21, size=n).astype(np.float64) + 2 * s
        qk = rng.normal(size=(n, 9)) * 5 + 1j * rng.normal(size=(n, 9)) * 5
        qs.append(Q / N)
        qks.append(qk / N)
        acc[s, 0, orc.A_N] = n
        acc[s, 0, orc.A_Q1:orc.A_Q4 + 1] = [Q.sum(), (Q ** 2).sum(), (Q ** 3).sum(),
                                           (Q ** 4).sum()]
        for v in range(9):
            acc[s, 0, orc.a_re(v)] = qk[:, v].real.sum()
            acc[s, 0, orc.a_im(v)] = qk[:, v].imag.sum()
            acc[s, 0, orc.a_abs2(v)] = (np.abs(qk[:, v]) ** 2).sum()
    obs = orc.observables(acc, L, jackknife=False)
    mbar = sum(q.mean() for q in qs) / S
    num = sum(((q - mbar) ** 4).mean() for q in qs) / S
    den = sum(((q - mbar) ** 2).mean() for q in qs) / S
    assert obs["g"][0] == pytest.approx(0.5 * (3 - num / den ** 2), rel=1e-10)
    chi0 = N * (sum((q ** 2).mean() for q in qs) / S - (sum(q.mean() for q in qs) / S) ** 2)
    assert obs["chi0"][0] == pytest.approx(chi0, rel=1e-10)
    chik = [N * (sum((np.abs(qk[:, v]) ** 2).mean() for qk in qks) / S
                 - abs(sum(qk[:, v].mean() for qk in qks) / S) ** 2) for v in range(9)]
    c1, c2 = np.mean(chik[:3]), np.mean(chik[3:])
    assert obs["chi_k1"][0] == pytest.approx(c1, rel=1e-10)
    assert obs["r12"][0] == pytest.approx(c1 / c2, rel=1e-10)
    if chi0 / c1 >= 1:
        assert obs["xi"][0] == pytest.approx(math.sqrt(chi0 / c1 - 1) / (2 * math.sin(math.pi / L)))


def test_jackknife_of_a_mean_is_the_standard_error():
    rng = np.random.default_rng(8)
    L, S = 4, 25
    acc = np.zeros((S, 1, orc.NACC))
    acc[:, 0, orc.A_N] = 1
    Q = rng.normal(size=S) * 10
    acc[:, 0, orc.A_Q2] = Q ** 2
    obs = orc.observables(acc, L)
    q2 = Q ** 2 / 64 ** 2
    assert obs["err"]["q2"][0] == pytest.approx(q2.std(ddof=1) / math.sqrt(S), rel=1e-10)


@pytest.mark.parametrize("gauss", [False, True])
def test_high_temperature_energy_follows_the_small_beta_expansion(gauss):
    """ln Z = N ln 2 + (beta^2 / 2)(sum_bonds J^2 + N h^2) + O(beta^4), so
    <E>/N = -beta (sum_bonds J^2 / N + h^2) + O(beta^3). At beta = 0.05 and
    h = 1 the prediction is about -0.2; a sign error, a dropped field term or
    double-counted bonds miss it by far more than the tolerance."""
    L, S, beta, h = 4, 32, 0.05, 1.0
    N = L ** 3
    J, s0 = inputs.make_instance("gauss" if gauss else "pmj", L, S, 1, seed=17)
    st = orc.State(L, np.array([1.0 / beta]), h, gauss, seed=17, J=J, spins=s0, n_therm=20)
    st.run(420, threads=4)
    tm = orc.thermal_means(st.acc, L)
    e_per_spin = tm["e1"][:, 0]                      # per sample, both replicas
    h_used = np.rint(h * 131072.0) / 131072.0 if gauss else h
    pred = -beta * ((J.astype(np.float64) ** 2).sum(axis=(1, 2)) / N + h_used ** 2)
    n = st.acc[:, 0, 0]  # measurements per sample
    # per-measurement spread of E/N, estimated from the accumulated second moment
    var = tm["e2"][:, 0] - e_per_spin ** 2
    se = np.sqrt(var.sum() / (2 * n.sum())) / np.sqrt(S)
    diff = (e_per_spin - pred).mean()
    assert abs(diff) < 4 * se + 3 * beta ** 3 * (3 + h ** 4) * 4, (diff, se)
    assert abs(pred.mean() + 0.2) < 0.02


def test_zero_field_averages_of_m_and_q_vanish():
    """At h = 0 the model is symmetric under s -> -s of one replica (for q) and
    of both (for M): the disorder and thermal averages of M and q(0) vanish
    within their errors."""
    L, S, nt = 4, 48, 2
    T = np.array([1.6, 2.4])
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=23)
    st = orc.State(L, T, 0.0, False, seed=23, J=J, spins=s0, n_therm=100)
    st.run(1100, threads=4)
    tm = orc.thermal_means(st.acc, L)
    for key in ("m1", "q1"):
        per_sample = tm[key]                          # [S][nt]
        mean = per_sample.mean(axis=0)
        se = per_sample.std(axis=0, ddof=1) / np.sqrt(S)
        assert np.all(np.abs(mean) < 4 * se + 1e-12), (key, mean, se)
