"""Pins for the oracle's conventions: the instance generators, the replica
exchange pair schedule and the independence of the Metropolis random words.

None of these is fixed by the paper; they are the readings the engine takes
(the methods section leaves the coupling draw, the initial state, the
exchange schedule and the random-number layout open). What the paper does fix
is what they must achieve: bimodal couplings with p = 1/2 drawn independently
per bond (model paragraph), independent replicas (methods section, two
replicas per temperature), neighbouring temperatures offered a swap in turn
(methods section, parallel tempering), and independent uniform draws for each
spin-flip attempt. Each test checks such a property from the outside, so that
a wrong lane, field or parity in the oracle fails one of them; the planted
mistakes in test_oracle_mutations.py check that they do.
"""
import numpy as np
import pytest

from oracle import oracle as orc


def _corr(a, b):
    a = a.astype(np.float64).ravel()
    b = b.astype(np.float64).ravel()
    return float(np.corrcoef(a, b)[0, 1])


def test_pmj_couplings_are_balanced_and_independent():
    """+-J couplings (model paragraph: J = +-1 with probability 1/2): the
    fraction of -1 bonds is 1/2 overall, per bond direction and per sample
    (chi-square), and bonds are uncorrelated across directions, along the
    site index at lags that would expose a wrong lane or bit (1, 32, 128)
    and across samples."""
    L, S = 8, 48
    N = L ** 3
    J = orc.pmj_couplings(11, S, L)
    assert set(np.unique(J)) == {-1.0, 1.0}
    neg = (J < 0)
    n = neg.size
    assert abs(neg.mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    # chi-square of the -1 counts over the (sample, direction) cells
    cnt = neg.sum(axis=2)
    chi2 = float((((cnt - N / 2) ** 2) / (N / 4)).sum())
    dof = cnt.size
    assert chi2 < dof + 6 * np.sqrt(2 * dof), chi2
    lim = 5 / np.sqrt(S * N)
    for d1, d2 in ((0, 1), (0, 2), (1, 2)):
        assert abs(_corr(J[:, d1], J[:, d2])) < lim
    for lag in (1, 32, 128):
        assert abs(_corr(J[:, :, :-lag], J[:, :, lag:])) < 5 / np.sqrt(S * 3 * (N - lag))
    assert abs(_corr(J[:-1], J[1:])) < 5 / np.sqrt((S - 1) * 3 * N)
    # shards: the draws of a sample depend only on its global index
    np.testing.assert_array_equal(orc.pmj_couplings(11, 5, L, s_base=20), J[20:25])


def test_initial_spins_are_balanced_and_independent():
    """Initial spins: +-1 with probability 1/2, independent across the two
    replicas of a slot (identical replicas would start at q = 1), across
    slots, along the site index and across samples."""
    L, S, nt = 8, 16, 6
    N = L ** 3
    s = orc.init_spins(5, S, nt, L)
    assert set(np.unique(s)) == {-1, 1}
    assert abs((s < 0).mean() - 0.5) < 5 * 0.5 / np.sqrt(s.size)
    cnt = (s < 0).sum(axis=3)
    chi2 = float((((cnt - N / 2) ** 2) / (N / 4)).sum())
    assert chi2 < cnt.size + 6 * np.sqrt(2 * cnt.size), chi2
    lim = 5 / np.sqrt(S * nt * N)
    assert abs(_corr(s[:, 0], s[:, 1])) < lim
    assert abs(_corr(s[:, :, :-1], s[:, :, 1:])) < 5 / np.sqrt(S * 2 * (nt - 1) * N)
    for lag in (1, 32, 128):
        assert abs(_corr(s[..., :-lag], s[..., lag:])) < 5 / np.sqrt(S * 2 * nt * (N - lag))
    assert abs(_corr(s[:-1], s[1:])) < 5 / np.sqrt((S - 1) * 2 * nt * N)
    np.testing.assert_array_equal(orc.init_spins(5, 3, nt, L, s_base=7), s[7:10])


# Slots holding initial slot k's configuration after each sweep, when every
# offered swap is accepted: exchange after sweep n when (n + 1) % ee == 0,
# exchange number e = (n + 1)/ee - 1 offers the pairs (p, p+1) with p of the
# parity of e, each replica on its own ladder.
TRACES = {
    # (n_T, exchange_every): permutation after sweeps 0, 1, 2, 3
    (4, 1): [[1, 0, 3, 2], [1, 3, 0, 2], [3, 1, 2, 0], [3, 2, 1, 0]],
    (3, 1): [[1, 0, 2], [1, 2, 0], [2, 1, 0], [2, 0, 1]],
    (4, 2): [[0, 1, 2, 3], [1, 0, 3, 2], [1, 0, 3, 2], [1, 3, 0, 2]],
    (5, 1): [[1, 0, 3, 2, 4], [1, 3, 0, 4, 2], [3, 1, 4, 0, 2], [3, 4, 1, 2, 0]],
}


@pytest.mark.parametrize("nt,ee", sorted(TRACES))
def test_exchange_pair_schedule_trace(nt, ee):
    """At infinite temperature in every slot, a sweep flips every spin
    (every threshold is 2^32 - 1) and every offered swap is accepted (the
    exponent (beta_p - beta_{p+1}) dE is 0), so the slot each configuration
    sits in traces the pair schedule: even pairs (0,1), (2,3), ... at even
    exchanges, odd pairs (1,2), (3,4), ... at odd ones (methods section:
    neighbouring temperatures offered a swap in turn). The expected
    permutations are written out above."""
    L = 4
    N = L ** 3
    rng = np.random.default_rng(nt * 10 + ee)
    s0 = rng.choice(np.array([-1, 1], dtype=np.int8), size=(1, 2, nt, N))
    J = rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(1, 3, N))
    T = np.full(nt, np.inf)
    st = orc.State(L, T, 0.2, False, seed=3, J=J, spins=s0, exchange_every=ee)
    for n, perm in enumerate(TRACES[(nt, ee)]):
        st.run(1)
        sign = -1 if n % 2 == 0 else 1  # every spin flips once per sweep
        for r in range(2):
            for t in range(nt):
                np.testing.assert_array_equal(
                    st.spins[0, r, t], sign * s0[0, r, perm[t]],
                    err_msg=f"sweep {n}, replica {r}, slot {t}")
        # energies follow their configurations
        for r in range(2):
            for t in range(nt):
                assert (st.B[0, r, t], st.M[0, r, t]) == orc.bond_sum(L, False, J[0],
                                                                      st.spins[0, r, t])


def _twins(L=4, nt=4, S=2, sweeps=20, rng_group=1, T=1.0):
    """Zero couplings (every site an independent two-state chain in the field
    h = 0.5), every chain of every sample started at all +1, equal
    temperatures and no exchange, so any two chains see the same law; only
    their random words tell them apart."""
    N = L ** 3
    J = np.zeros((S, 3, N), dtype=np.float32)
    s0 = np.ones((S, 2, nt, N), dtype=np.int8)
    st = orc.State(L, np.full(nt, T), 0.5, True, seed=9, J=J, spins=s0, exchange_every=0,
                   rng_group=rng_group)
    st.run(sweeps)
    return st.spins


def _agree(a, b):
    return float((a == b).mean())


def _same_colour_pairs(L, delta):
    """Sites (a, b) of one checkerboard colour whose colour-compressed
    indices (i >> 1) differ by delta."""
    col = lambda i: (i % L + (i // L) % L + i // (L * L)) & 1
    a, b = [], []
    for i in range(L ** 3):
        j = (i >> 1) + delta
        for k in (2 * j, 2 * j + 1):
            if k < L ** 3 and col(k) == col(i):
                a.append(i)
                b.append(k)
    return np.array(a), np.array(b)


def test_metropolis_words_differ_between_colours_replicas_slots_and_sites():
    """Each attempt draws its own uniform word. With zero couplings at
    beta = 1, h = 0.5, each site flips + -> - with probability e^-1 and
    - -> + always; two chains driven by independent words agree on a site
    with probability p^2 + (1 - p)^2 ~ 0.61 (p = 1/(1 + e^-1)), while chains
    fed the same words stay identical forever. So: the x-neighbours 2j, 2j+1
    (different colours, same colour-compressed index j), the two replicas of
    a slot, two slots, two sites of one Philox group (j, j+1) and of
    neighbouring groups (j, j+4), and two samples must all disagree somewhere;
    only samples inside one RNG group share their words. The fraction of +1
    spins is the stationary p, not the 1 that a word reused every sweep
    would give after an even number of sweeps."""
    L = 6
    sp = _twins(L=L)
    p = 1.0 / (1.0 + np.exp(-1.0))
    indep = p * p + (1 - p) ** 2
    even, odd = sp[..., 0::2], sp[..., 1::2]
    # sites 2j and 2j+1: different colours, same j = i >> 1
    assert _agree(even, odd) < indep + 0.12
    assert _agree(sp[:, 0], sp[:, 1]) < indep + 0.12
    assert _agree(sp[:, :, 0], sp[:, :, 1]) < indep + 0.12
    for delta in (1, 4):  # neighbouring lanes of a Philox group; neighbouring groups
        a, b = _same_colour_pairs(L, delta)
        assert _agree(sp[..., a], sp[..., b]) < indep + 0.12, delta
    assert _agree(sp[0], sp[1]) < indep + 0.12
    assert abs((sp > 0).mean() - p) < 0.06
    # samples of one RNG group share every Metropolis word
    grouped = _twins(L=L, rng_group=2)
    np.testing.assert_array_equal(grouped[0], grouped[1])


def test_slot_shared_words_keep_the_slots_of_a_replica_together():
    """Shared slot words (the N_T temperatures of a replica packed in the
    bits of one word draw one random number per site; methods section,
    multispin coding): chains of one replica at equal temperatures, started
    equal, stay identical forever, while the two replicas (separate words)
    still decorrelate and the stationary +1 fraction is unchanged."""
    L, nt, S = 6, 4, 2
    N = L ** 3
    J = np.zeros((S, 3, N), dtype=np.float32)
    s0 = np.ones((S, 2, nt, N), dtype=np.int8)
    st = orc.State(L, np.full(nt, 1.0), 0.5, True, seed=9, J=J, spins=s0, exchange_every=0,
                   slot_shared=True)
    st.run(20)
    sp = st.spins
    for t in range(1, nt):
        np.testing.assert_array_equal(sp[:, :, t], sp[:, :, 0])
    p = 1.0 / (1.0 + np.exp(-1.0))
    assert _agree(sp[:, 0], sp[:, 1]) < p * p + (1 - p) ** 2 + 0.12
    assert _agree(sp[0], sp[1]) < p * p + (1 - p) ** 2 + 0.12
    assert abs((sp > 0).mean() - p) < 0.06


@pytest.mark.slow
def test_shared_slot_words_bias_parallel_tempering():
    """Why every chain draws its own Metropolis words. Packing the N_T
    temperatures of a replica into the bits of one word and updating them
    with one random number per site (the cheap reading of the methods
    section's multispin coding) couples the slots' moves: each slot's sweep
    still leaves its own Boltzmann law invariant, but the joint law of
    neighbouring slots is no longer the product that the replica-exchange
    rule assumes, and exchange then moves the slots' marginals away from
    equilibrium. At L = 2 (exact enumeration), 96 chains over 2000 sweeps:
    with independent words every temperature's energy agrees within 3
    standard errors; with shared words at least one is off by more than 10."""
    import math
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from paper_1403_4560_b300 import inputs
    from test_oracle_model import _exact_l2
    L, S, h = 2, 96, 0.3
    T = inputs.geometric_ladder(0.5, 2.0, 4)
    J, s0 = inputs.make_instance("pmj", L, S, len(T), seed=33, same_couplings=True)
    exact = _exact_l2(J[0], h, T, False)
    z = {}
    for shared in (False, True):
        st = orc.State(L, T, h, False, seed=77, J=J, spins=s0, n_therm=200, slot_shared=shared)
        st.run(2200, threads=4)
        tm = orc.thermal_means(st.acc, L)
        z[shared] = [abs(tm["e1"][:, t].mean() - exact[t]["e"]) /
                     (tm["e1"][:, t].std(ddof=1) / math.sqrt(S)) for t in range(len(T))]
    assert max(z[False]) < 3.0, z[False]
    assert max(z[True]) > 10.0, z[True]
