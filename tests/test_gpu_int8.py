"""GPU parity of the int8 path against the CPU oracle, through the C ABI.

+-J and Gaussian couplings both reproduce the oracle bit for bit: spins,
energies and every FP64 accumulator (the acceptance rule, RNG layout and
summation orders are frozen on both sides). Sizes span several work units
and ragged slot counts; the full-size check samples a few disorder samples of
the bench workload in the bench's own launch configuration.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    sgbuild.build()
    torch.cuda.init()


def oracle_state(L, T, h, dist, seed, J, s0, **opt):
    return orc.State(L, T, h, dist == "gauss", seed=seed, J=J, spins=s0,
                     rng_group=opt.get("rng_group", 1),
                     exchange_every=opt.get("exchange_every", 1),
                     measure_every=opt.get("measure_every", 1), n_therm=opt.get("n_therm", 0))


def assert_same(ens, st, samples=None):
    sl = slice(None) if samples is None else samples
    np.testing.assert_array_equal(ens.spins()[sl], st.spins[sl])
    B, M = ens.energies()
    np.testing.assert_array_equal(B[sl], st.B[sl])
    np.testing.assert_array_equal(M[sl], st.M[sl])
    np.testing.assert_array_equal(ens.accumulators()[sl], st.acc[sl])


def test_library_generated_pmj_instance_matches_oracle_generators():
    L, S, nt, seed = 4, 16, 8, 1
    T = inputs.geometric_ladder(0.4, 1.6, nt)
    with sgmc.Ensemble(L, 0.3, T, "pmj", S, seed) as ens:
        np.testing.assert_array_equal(ens.couplings(), orc.pmj_couplings(seed, S, L))
        np.testing.assert_array_equal(ens.spins(), orc.init_spins(seed, S, nt, L))
        B, M = ens.energies()
        for s in (0, 7):
            for r in (0, 1):
                for t in (0, nt - 1):
                    b, m = orc.bond_sum(L, False, orc.pmj_couplings(seed, S, L)[s],
                                        orc.init_spins(seed, S, nt, L)[s, r, t])
                    assert (B[s, r, t], M[s, r, t]) == (b, m)


def test_plain_pmj_config_is_bit_exact():
    """L=4, +-J, h=0.3, 2 x 8 temperatures geometric 0.4-1.6, exchange every
    sweep, 16 samples, seed 1 (the small plain configuration), library-drawn
    instance reproduced by the oracle's own generators."""
    L, S, nt, seed, h = 4, 16, 8, 1, 0.3
    T = inputs.geometric_ladder(0.4, 1.6, nt)
    sweeps, n_therm = 1200, 600
    with sgmc.Ensemble(L, h, T, "pmj", S, seed, n_therm=n_therm) as ens:
        ens.sweep(sweeps)
        ens.synchronize()
        st = oracle_state(L, T, h, "pmj", seed, orc.pmj_couplings(seed, S, L),
                          orc.init_spins(seed, S, nt, L), n_therm=n_therm)
        st.run(sweeps, threads=THREADS)
        assert_same(ens, st)


@pytest.mark.parametrize("L,nt,dist,ee,me,rg", [
    (2, 3, "pmj", 1, 1, 1), (2, 5, "gauss", 2, 1, 1), (4, 5, "gauss", 1, 2, 1),
    (6, 6, "pmj", 1, 1, 2), (6, 4, "gauss", 3, 1, 1), (8, 7, "pmj", 2, 3, 1),
    (8, 9, "gauss", 1, 1, 1), (10, 6, "gauss", 1, 1, 1), (10, 4, "pmj", 0, 1, 1),
    (12, 5, "pmj", 1, 1, 4), (12, 8, "gauss", 1, 1, 1), (14, 4, "pmj", 1, 1, 1),
    (16, 4, "gauss", 1, 2, 1), (4, 1, "pmj", 1, 1, 1), (14, 5, "gauss", 1, 1, 1),
    # state kept in global memory: large L, or too many slots for shared memory
    (18, 3, "pmj", 1, 1, 1), (20, 2, "gauss", 1, 1, 1), (22, 2, "pmj", 1, 1, 1),
    (24, 2, "gauss", 1, 1, 1), (12, 64, "gauss", 1, 1, 1)])
def test_int8_paths_are_bit_exact(L, nt, dist, ee, me, rg):
    S, seed, h = 4, 1234 + L, 0.25
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=L * 100 + nt)
    sweeps = 12 if (L >= 18 or nt > 32) else 60 if L >= 12 else 150
    opt = dict(exchange_every=ee, measure_every=me, n_therm=sweeps // 3, rng_group=rg)
    with sgmc.Ensemble(L, h, T, dist, S, seed, J=J, spins=s0, **opt) as ens:
        ens.sweep(sweeps)
        ens.synchronize()
        st = oracle_state(L, T, h, dist, seed, J, s0, **opt)
        st.run(sweeps, threads=THREADS)
        assert_same(ens, st)


@pytest.mark.parametrize("dist", ["pmj", "gauss"])
def test_chunking_and_launch_shape_do_not_change_results(dist):
    L, S, nt = 6, 5, 6
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=3)
    ref = None
    for opt in (dict(), dict(sweeps_per_launch=1), dict(sweeps_per_launch=7, threads_per_block=96),
                dict(threads_per_block=480)):
        with sgmc.Ensemble(L, 0.1, T, dist, S, 77, J=J, spins=s0, n_therm=5, **opt) as ens:
            ens.sweep(20)
            ens.sweep(13)
            got = (ens.spins(), ens.energies(), ens.accumulators())
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1][0], ref[1][0])
            np.testing.assert_array_equal(got[2], ref[2])


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_uneven_ensembles_match_single_runs(use_graph):
    specs = [(4, "pmj", 3, 6), (6, "gauss", 2, 5), (8, "gauss", 4, 4)]
    Ts = {nt: inputs.geometric_ladder(0.5, 1.5, nt) for _, _, _, nt in specs}
    insts = [inputs.make_instance(d, L, S, nt, seed=L) for L, d, S, nt in specs]
    singles = []
    for (L, d, S, nt), (J, s0) in zip(specs, insts):
        with sgmc.Ensemble(L, 0.2, Ts[nt], d, S, 5, J=J, spins=s0) as e:
            e.sweep(25)
            e.sweep(25)
            singles.append((e.spins(), e.accumulators()))
    ens = [sgmc.Ensemble(L, 0.2, Ts[nt], d, S, 5, J=J, spins=s0)
           for (L, d, S, nt), (J, s0) in zip(specs, insts)]
    try:
        sgmc.sweep_batch(ens, 25, use_graph=use_graph)
        sgmc.sweep_batch(ens, 25, use_graph=use_graph)  # second call replays the cached graph
        for e, (sp, acc) in zip(ens, singles):
            e.synchronize()
            assert e.sweeps_done == 50
            np.testing.assert_array_equal(e.spins(), sp)
            np.testing.assert_array_equal(e.accumulators(), acc)
    finally:
        for e in ens:
            e.close()


@pytest.mark.parametrize("dist", ["pmj", "gauss"])
def test_standalone_exchange_matches_oracle(dist):
    L, S, nt = 4, 6, 7
    T = inputs.geometric_ladder(0.3, 3.0, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=11)
    with sgmc.Ensemble(L, 0.4, T, dist, S, 21, J=J, spins=s0) as ens:
        st = oracle_state(L, T, 0.4, dist, 21, J, s0)
        for parity in (0, 1, 1, 0):
            ens.exchange(parity)
            st.exchange(parity)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        B, M = ens.energies()
        np.testing.assert_array_equal(B, st.B)
        np.testing.assert_array_equal(M, st.M)


def test_measure_arbitrary_wavevectors():
    L, S, nt = 6, 3, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=2)
    k = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [2, -1, 3]])
    with sgmc.Ensemble(L, 0.0, T, "pmj", S, 3, J=J, spins=s0) as ens:
        got = ens.measure(k)
    coords = np.array([[i % L, (i // L) % L, i // (L * L)] for i in range(L ** 3)])
    q = s0[:, 0].astype(np.float64) * s0[:, 1]
    want = (q[..., None] * np.exp(2j * np.pi / L * coords @ k.T)).mean(axis=-2)
    np.testing.assert_allclose(got[..., 0], want.real, atol=2e-6)
    np.testing.assert_allclose(got[..., 1], want.imag, atol=2e-6)


def test_results_match_oracle_estimators():
    L, S, nt = 4, 24, 4
    T = inputs.geometric_ladder(0.6, 1.6, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=8)
    with sgmc.Ensemble(L, 0.1, T, "gauss", S, 4, J=J, spins=s0, n_therm=50) as ens:
        ens.sweep(300)
        got = ens.results()
        acc = ens.accumulators()
    want = orc.observables(acc, L)
    for kl, ko in [("g", "g"), ("chi0", "chi0"), ("chi1", "chi_k1"), ("r12", "r12"), ("e", "e")]:
        np.testing.assert_allclose(got[kl], want[ko], rtol=1e-10, equal_nan=True)
        np.testing.assert_allclose(got[kl + "_err"], want["err"][ko], rtol=1e-7, equal_nan=True)


@pytest.mark.parametrize("L", [8, 12])
def test_full_size_gaussian_workload_sampled_parity(L):
    """512 samples, 2 x 24 temperatures geometric 0.5-1.6, Gaussian couplings,
    h = 0.2, exchange every sweep, measuring from sweep 0, default (bench)
    launch configuration; three samples are re-run by the oracle."""
    S, nt, h, seed, sweeps = 512, 24, 0.2, 2024, 6
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=31 + L)
    with sgmc.Ensemble(L, h, T, "gauss", S, seed, J=J, spins=s0) as ens:
        ens.sweep(sweeps)
        ens.synchronize()
        st = oracle_state(L, T, h, "gauss", seed, J, s0)
        picks = [0, 255, 511]
        for s in picks:
            st.run(sweeps, s_range=(s, s + 1))
        assert_same(ens, st, samples=picks)


@pytest.mark.parametrize("L,dist,S,nt", [(8, "gauss", 700, 8), (12, "pmj", 400, 8),
                                         (6, "gauss", 90, 5), (8, "gauss", 520, 8)])
def test_segmented_launches_match_one_cta_per_sample(L, dist, S, nt):
    """Launches whose sweeps are split into segments that the CTAs claim one
    by one (consecutive segments of a sample may run on different SMs, each
    waiting for the previous one to be stored) give the chain of one CTA per
    sample bit for bit: library choice (more samples than resident CTAs, or
    one wave that would load some SMs with one CTA more than others, here
    520 samples as 3 CTAs on every SM) and a forced split; the oracle agrees
    on sampled samples."""
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=50 + L)
    opt = dict(n_therm=10, log_bins=3, pq_hist=1)
    outs = []
    for seg in (1, 0, 5):
        with sgmc.Ensemble(L, 0.2, T, dist, S, 8, J=J, spins=s0, segments=seg, **opt) as ens:
            ens.sweep(48)
            ens.sweep(40)
            ens.synchronize()
            outs.append((ens.spins(), ens.energies()[0], ens.energies()[1], ens.accumulators(),
                         ens.histogram()))
    for out in outs[1:]:
        for got, want in zip(out, outs[0]):
            np.testing.assert_array_equal(got, want)
    st = oracle_state(L, T, 0.2, dist, 8, J, s0, n_therm=10)
    picks = [0, S // 2, S - 1]
    for s in picks:
        st.run(88, s_range=(s, s + 1))
    np.testing.assert_array_equal(outs[0][0][picks], st.spins[picks])
    with pytest.raises(sgmc.SgError):
        sgmc.Ensemble(L, 0.2, T, dist, 4, 8, segments=-1)


def test_segmented_launches_in_a_replayed_graph_match_single_runs():
    """Ensembles with more samples than resident CTAs, batched through one
    CUDA graph (counters zeroed by captured memset nodes, the sweep index from
    the device counter) and the graph replayed, equal single runs with one CTA
    per sample bit for bit."""
    specs = [(8, "gauss", 700, 8), (12, "pmj", 400, 8)]
    T = inputs.geometric_ladder(0.5, 1.6, 8)
    insts = [inputs.make_instance(d, L, S, nt, seed=70 + L) for L, d, S, nt in specs]
    singles = []
    for (L, d, S, nt), (J, s0) in zip(specs, insts):
        with sgmc.Ensemble(L, 0.3, T, d, S, 6, J=J, spins=s0, n_therm=5, segments=1) as e:
            e.sweep(96)
            singles.append((e.spins(), e.accumulators()))
    ens = [sgmc.Ensemble(L, 0.3, T, d, S, 6, J=J, spins=s0, n_therm=5)
           for (L, d, S, nt), (J, s0) in zip(specs, insts)]
    try:
        sgmc.sweep_batch(ens, 48, use_graph=True)
        sgmc.sweep_batch(ens, 48, use_graph=True)
        for e, (sp, acc) in zip(ens, singles):
            e.synchronize()
            np.testing.assert_array_equal(e.spins(), sp)
            np.testing.assert_array_equal(e.accumulators(), acc)
    finally:
        for e in ens:
            e.close()


def test_library_gaussian_couplings_are_standard_normal_on_grid():
    from scipy import stats
    L, S = 8, 64
    with sgmc.Ensemble(L, 0.0, [1.0], "gauss", S, 99) as ens:
        J = ens.couplings().astype(np.float64).ravel()
    assert np.all(np.rint(J * 2 ** 17) == J * 2 ** 17)
    n = J.size
    assert abs(J.mean()) < 5 / np.sqrt(n)
    assert abs(J.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(J, "norm").pvalue > 1e-4


def test_edge_cases_and_argument_errors():
    T = [0.7]
    with sgmc.Ensemble(2, 0.5, T, "pmj", 1, 3) as ens:   # one sample, one temperature
        ens.sweep(0)
        ens.sweep(10)
        ens.synchronize()
        st = oracle_state(2, np.array(T), 0.5, "pmj", 3, orc.pmj_couplings(3, 1, 2),
                          orc.init_spins(3, 1, 1, 2))
        st.run(10)
        assert_same(ens, st)
    for bad in (dict(L=5), dict(L=4, T=[1.0, 0.5]), dict(L=4, T=[0.0, 1.0])):
        with pytest.raises(sgmc.SgError) as ei:
            sgmc.Ensemble(bad["L"], 0.1, bad.get("T", [1.0]), "pmj", 2, 1)
        assert ei.value.status == sgmc.SG_EINVAL
    J = np.full((1, 3, 64), 0.5, dtype=np.float32)
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(4, 0.1, [1.0], "pmj", 1, 1, J=J)
    assert ei.value.status == sgmc.SG_EINVAL


def test_watchdog_stops_a_long_launch_with_a_status():
    """A launch whose clock budget runs out stops between sweeps and reports
    SG_ETIMEOUT through the status word; the context stays usable."""
    L, S, nt = 8, 4, 8
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.1, T, "gauss", S, 1, watchdog_cycles=20000) as ens:
        ens.sweep(2000)
        with pytest.raises(sgmc.SgError) as ei:
            ens.synchronize()
        assert ei.value.status == sgmc.SG_ETIMEOUT
    with sgmc.Ensemble(4, 0.1, [1.0, 2.0], "pmj", 2, 1) as ens:
        ens.sweep(5)
        ens.synchronize()


def test_device_threshold_map_matches_oracle_bit_for_bit():
    """The device exponential/threshold map equals the oracle's on a dense grid
    (all FP32 values in [-1, 0] of one binade sample, and a uniform grid over
    [-70, 1])."""
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-70.0, 1.0, 400001, dtype=np.float32),
                        -rng.random(200000).astype(np.float32),
                        -(rng.random(100000) * 23).astype(np.float32),
                        np.array([0.0, -0.0, -1e-30, -64.0, -64.0001, -22.18, -22.19],
                                 dtype=np.float32)])
    got = sgmc.threshold_map(x)
    want = np.array([orc.t32(float(v)) if v < 0 else 0xFFFFFFFF for v in x], dtype=np.uint32)
    np.testing.assert_array_equal(got, want)


def test_screened_metropolis_decision_is_the_threshold_rule():
    """The Gaussian sweep decides r <= t32(x) through a screen (hardware 2^x
    with a 2^-12 guard band) and the exact threshold inside the band. Its
    decisions equal the oracle's rule at every threshold, one above and one
    below it, and on uniform draws; draws at the threshold of a large
    threshold must go to the exact path, uniform draws almost never do."""
    rng = np.random.default_rng(11)
    x = np.concatenate([np.linspace(-70.0, 2.0, 150001, dtype=np.float32),
                        -(rng.random(100000) * 23).astype(np.float32),
                        -rng.random(50000).astype(np.float32) * 1e-3,
                        np.array([0.0, -0.0, 1e-30, -1e-30, -64.0, -64.0001, -22.18, -22.19,
                                  -88.0, -100.0, 5.0, 60.0], dtype=np.float32)])
    thr = np.array([orc.t32(float(v)) if v < 0 else 0xFFFFFFFF for v in x], dtype=np.int64)
    uniform = rng.integers(0, 2 ** 32, x.size, dtype=np.int64)
    for name, r in (("at", thr), ("above", thr + 1), ("below", thr - 1), ("uniform", uniform),
                    ("zero", np.zeros_like(thr)), ("max", np.full_like(thr, 2 ** 32 - 1))):
        r = np.clip(r, 0, 2 ** 32 - 1)
        got = sgmc.accept_map(x, r.astype(np.uint32))
        np.testing.assert_array_equal(got & 1, (r <= thr).astype(np.uint8), err_msg=name)
        if name == "at":
            # the band is wider than one unit of r (x > 0 screens as a sure accept)
            big = (thr >= 2 ** 14) & (x <= 0)
            assert np.all(got[big] & 2), "draws at a large threshold skipped the exact path"
        if name == "uniform":
            assert np.mean(got & 2) / 2 < 2.0 ** -10


@pytest.mark.parametrize("dist,L,nt", [("gauss", 8, 20), ("pmj", 12, 8)])
def test_autotune_changes_speed_not_results(dist, L, nt):
    S = 40
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=6)
    with sgmc.Ensemble(L, 0.2, T, dist, S, 4, J=J, spins=s0, n_therm=3) as ref:
        ref.sweep(10)
        want = (ref.spins(), ref.accumulators(), ref.energies()[0])
    with sgmc.Ensemble(L, 0.2, T, dist, S, 4, J=J, spins=s0, n_therm=3) as ens:
        ens.sweep(4)
        rep = ens.autotune(trial_sweeps=3)
        assert rep["n_candidates"] > 1 and rep["best_ms_per_sweep"] <= rep["default_ms_per_sweep"]
        assert ens.sweeps_done == 4
        ens.sweep(6)
        np.testing.assert_array_equal(ens.spins(), want[0])
        np.testing.assert_array_equal(ens.accumulators(), want[1])
        np.testing.assert_array_equal(ens.energies()[0], want[2])


@pytest.mark.parametrize("layout,dist,S,cut,L", [(0, "gauss", 12, 5, 6), (0, "pmj", 9, 4, 8),
                                                 (1, "pmj", 192, 64, 6)])
def test_shards_with_sample_base_reproduce_the_unsplit_run(layout, dist, S, cut, L):
    """Library-drawn instance; one ensemble against two shards whose samples
    carry their global indices (the multi-GPU split)."""
    nt, seed = 5, 31
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, dist, S, seed, layout=layout, n_therm=4) as whole, \
            sgmc.Ensemble(L, 0.2, T, dist, cut, seed, layout=layout, n_therm=4) as a, \
            sgmc.Ensemble(L, 0.2, T, dist, S - cut, seed, layout=layout, n_therm=4,
                          sample_base=cut) as b:
        for e in (whole, a, b):
            e.sweep(20)
        np.testing.assert_array_equal(np.concatenate([a.couplings(), b.couplings()]),
                                      whole.couplings())
        np.testing.assert_array_equal(np.concatenate([a.spins(), b.spins()]), whole.spins())
        np.testing.assert_array_equal(np.concatenate([a.accumulators(), b.accumulators()]),
                                      whole.accumulators())


@pytest.mark.parametrize("layout,dist,S", [(0, "gauss", 6), (1, "pmj", 64)])
def test_checkpoint_and_resume_is_bit_exact(layout, dist, S):
    L, nt = 6, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=2)
    with sgmc.Ensemble(L, 0.1, T, dist, S, 8, J=J, spins=s0, layout=layout, n_therm=5) as ref:
        ref.sweep(30)
        want = (ref.spins(), ref.accumulators())
    with sgmc.Ensemble(L, 0.1, T, dist, S, 8, J=J, spins=s0, layout=layout, n_therm=5) as e:
        e.sweep(12)
        ckpt = (e.spins(), e.accumulators(), e.sweeps_done)
    with sgmc.Ensemble(L, 0.1, T, dist, S, 8, J=J, spins=s0, layout=layout, n_therm=5) as r:
        r.set_spins(ckpt[0])
        r.set_accumulators(ckpt[1])
        r.set_sweeps_done(ckpt[2])
        r.sweep(18)
        np.testing.assert_array_equal(r.spins(), want[0])
        np.testing.assert_array_equal(r.accumulators(), want[1])


@pytest.mark.parametrize("layout", [0, sgmc.SG_LAYOUT_MSC64])
def test_set_spins_rejects_values_other_than_pm1_and_keeps_the_state(layout):
    """The values are checked on the device after the upload; a bad array
    (a 0, a 2, in the middle or in the ragged tail) leaves the state as it was."""
    L, nt, S = 4, 3, 64
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 5, layout=layout) as ens:
        ens.sweep(3)
        before, (B0, M0) = ens.spins(), ens.energies()
        for pos, val in ((0, 0), (S * 2 * nt * L ** 3 // 2 + 3, 2), (S * 2 * nt * L ** 3 - 1, 0)):
            bad = before.copy().reshape(-1)
            bad[pos] = val
            with pytest.raises(sgmc.SgError) as ei:
                ens.set_spins(bad.reshape(before.shape))
            assert ei.value.status == sgmc.SG_EINVAL
            np.testing.assert_array_equal(ens.spins(), before)
            np.testing.assert_array_equal(ens.energies()[0], B0)
        flipped = -before
        ens.set_spins(flipped)
        np.testing.assert_array_equal(ens.spins(), flipped)


@pytest.mark.parametrize("layout", [0, sgmc.SG_LAYOUT_MSC64])
def test_async_uploads_and_downloads_match_the_synchronous_calls(layout):
    """A pipelined loop (upload the next state while the previous sweeps run,
    download each step's accumulators) gives the same results bit for bit as
    the synchronous calls, with a different initial state every step."""
    import torch
    L, nt, S, steps, n = 6, 4, 64, 3, 7
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    states = [inputs.make_instance("pmj", L, S, nt, seed=20 + k)[1] for k in range(steps)]
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 9, layout=layout) as a, \
            sgmc.Ensemble(L, 0.2, T, "pmj", S, 9, layout=layout) as b:
        want = []
        for x in states:
            a.set_spins(x)
            a.sweep(n)
            want.append(a.accumulators())
        pinned = [torch.from_numpy(x).pin_memory().numpy() for x in states]
        outs = [torch.zeros(want[0].shape, dtype=torch.float64).pin_memory().numpy()
                for _ in range(steps)]
        for x, o in zip(pinned, outs):
            b.set_spins_async(x)
            b.sweep(n)
            b.accumulators_async(o)
        b.synchronize()
        for w, o in zip(want, outs):
            np.testing.assert_array_equal(o, w)
        np.testing.assert_array_equal(b.spins(), a.spins())


@pytest.mark.parametrize("layout", [0, sgmc.SG_LAYOUT_MSC64])
def test_async_upload_with_bad_values_is_skipped_and_reported(layout):
    L, nt, S = 4, 3, 64
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 5, layout=layout) as a, \
            sgmc.Ensemble(L, 0.2, T, "pmj", S, 5, layout=layout) as ref:
        bad = a.spins().copy()
        bad.reshape(-1)[-1] = 0
        a.set_spins_async(bad)
        a.sweep(5)
        with pytest.raises(sgmc.SgError) as ei:
            a.synchronize()
        assert ei.value.status == sgmc.SG_EINVAL
        a.synchronize()  # the status word was reported once and cleared
        ref.sweep(5)
        np.testing.assert_array_equal(a.spins(), ref.spins())
        np.testing.assert_array_equal(a.accumulators(), ref.accumulators())
