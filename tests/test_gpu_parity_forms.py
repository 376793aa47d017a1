"""The batched, benchmarked and served forms of the engine against the CPU
oracle, element by element, through the C ABI.

Each test runs the library exactly the way its production form runs it and
re-runs sampled disorder samples with the oracle (each sample alone, keyed by
its global index), comparing spins, B, M and every FP64 accumulator bit for
bit:
  * the uneven batch (L = 6..16 with 2048..256 Gaussian samples, 2 x 20
    temperatures, h = 0.2) through one CUDA graph replayed twice, every
    ensemble's fused kernel on a graph branch with segmented launches;
  * the benchmark's own ensembles (Gaussian, 512 samples, 2 x 24
    temperatures geometric 0.5-1.6) in one 256-sweep sg_sweep: the library
    splits L = 12 into segments that the CTAs claim across SMs, and runs
    L = 8 as k = 3 CTAs on every SM sharing the segments (one-wave split);
  * requests submitted to a running server (int8 +-J, multispin-coded +-J,
    +-J with the state in global memory), whose accumulators come back from
    sg_server_result.
Paper: methods section (checkerboard Metropolis sweeps, parallel tempering
with two replicas per temperature), eq. overlap, Table I caption (first half
thermalises).
"""
import os
import time
from concurrent.futures import ThreadPoolExecutor

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


def oracle_one(L, T, h, gauss, seed, J, s0, s, sweeps, **opt):
    """The oracle's run of global sample s alone (its random numbers keyed by s)."""
    st = orc.State(L, T, h, gauss, seed=seed, J=J[s:s + 1], spins=s0[s:s + 1], s_base=s,
                   rng_group=opt.get("rng_group", 1), n_therm=opt.get("n_therm", 0),
                   exchange_every=opt.get("exchange_every", 1),
                   measure_every=opt.get("measure_every", 1))
    st.run(sweeps)
    return st


def assert_sample(got, st, s, what):
    spins, B, M, acc = got
    np.testing.assert_array_equal(spins[s], st.spins[0], err_msg=f"{what}: spins of sample {s}")
    np.testing.assert_array_equal(B[s], st.B[0], err_msg=f"{what}: B of sample {s}")
    np.testing.assert_array_equal(M[s], st.M[0], err_msg=f"{what}: M of sample {s}")
    np.testing.assert_array_equal(acc[s], st.acc[0], err_msg=f"{what}: accumulators of sample {s}")


def snapshot(ens):
    B, M = ens.energies()
    return ens.spins(), B, M, ens.accumulators()


UNEVEN = [(6, 2048), (8, 1024), (10, 1024), (12, 512), (16, 256)]


def test_graph_batched_uneven_ensemble_matches_oracle():
    """The uneven batch: L = 6, 8, 10, 12, 16 with 2048, 1024, 1024, 512, 256
    Gaussian samples, h = 0.2, 2 x 20 temperatures geometric 0.5-1.5,
    exchange and measurement every sweep, one graph of five branches replayed
    twice (2 x 48 sweeps, segmented launches); samples 0, S/2 and S-1 of every
    ensemble against the oracle."""
    nt, h, n, seed = 20, 0.2, 48, 5
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    insts = [inputs.make_instance("gauss", L, S, nt, seed=40 + L) for L, S in UNEVEN]
    ens = [sgmc.Ensemble(L, h, T, "gauss", S, seed + L, J=J, spins=s0)
           for (L, S), (J, s0) in zip(UNEVEN, insts)]
    try:
        plans = [e.launch_plan(n) for e in ens]
        assert all(p["segments"] > 1 for p in plans), plans  # the split path is what runs
        sgmc.sweep_batch(ens, n, use_graph=True)
        sgmc.sweep_batch(ens, n, use_graph=True)  # replays the cached graph
        got = []
        for e in ens:
            e.synchronize()
            assert e.sweeps_done == 2 * n
            got.append(snapshot(e))
    finally:
        for e in ens:
            e.close()
    jobs = [(k, s) for k, (L, S) in enumerate(UNEVEN) for s in (0, S // 2, S - 1)]

    def work(job):
        k, s = job
        (L, S), (J, s0) = UNEVEN[k], insts[k]
        return job, oracle_one(L, T, h, True, seed + L, J, s0, s, 2 * n)

    with ThreadPoolExecutor(THREADS) as ex:
        for (k, s), st in ex.map(work, jobs):
            assert_sample(got[k], st, s, f"batched L={UNEVEN[k][0]}")


@pytest.mark.parametrize("L", [8, 12])
def test_benchmark_launch_matches_oracle(L):
    """The benchmark's ensemble shape: Gaussian, 512 samples, 2 x 24
    temperatures geometric 0.5-1.6, h = 0.2, exchange and measurement every
    sweep, one sg_sweep of 256 sweeps in the library's own launch choice
    (L = 12: more samples than resident CTAs, segments claimed across SMs;
    L = 8: one wave run as 3 CTAs on every SM sharing the segments); four
    samples against the oracle."""
    S, nt, h, seed, sweeps = 512, 24, 0.2, 2024, 256
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=31 + L)
    with sgmc.Ensemble(L, h, T, "gauss", S, seed, J=J, spins=s0) as ens:
        plan = ens.launch_plan(sweeps)
        assert plan["segments"] > 1 and plan["launches"] == 1, plan
        if L == 8:
            assert plan["grid"] % 148 == 0 or plan["grid"] > ens.info().grid, plan
        ens.sweep(sweeps)
        ens.synchronize()
        got = snapshot(ens)
    picks = [0, 1, S // 2, S - 1]
    with ThreadPoolExecutor(min(THREADS, len(picks))) as ex:
        sts = list(ex.map(lambda s: oracle_one(L, T, h, True, seed, J, s0, s, sweeps), picks))
    for s, st in zip(picks, sts):
        assert_sample(got, st, s, f"bench L={L}")


SERVED = [  # L, h, nt, samples, sweeps, layout: +-J requests the oracle re-draws from the seed
    (12, 0.2, 5, 10, 40, 0),      # int8 +-J, state in shared memory
    (8, 0.1, 6, 64, 64, 1),       # multispin-coded +-J (RNG group 64)
    (20, 0.05, 3, 2, 8, 0),       # int8 +-J, state in global memory
    (4, 0.3, 8, 128, 90, 1),      # multispin-coded, two words
]


@pytest.mark.parametrize("use_graph", [False, True])
def test_served_requests_match_oracle(use_graph):
    """Requests admitted into a running server (a long Gaussian request keeps
    the GPU busy while they arrive) return accumulators equal to the oracle's
    run of the same instance: couplings and initial spins re-drawn by the
    oracle's own generators from the request's seed, first half thermalising."""
    with sgmc.Server(chunk_sweeps=16, use_graph=use_graph) as sv:
        busy = sv.submit(16, 0.2, inputs.geometric_ladder(0.5, 1.6, 16), "gauss", 256, seed=7,
                         n_sweeps=400)
        time.sleep(0.05)
        ids = []
        for k, (L, h, nt, S, sweeps, layout) in enumerate(SERVED):
            ids.append(sv.submit(L, h, inputs.geometric_ladder(0.5, 1.6, nt), "pmj", S,
                                 seed=300 + k, n_sweeps=sweeps, layout=layout))
            time.sleep(0.01)
        results = []
        for rid in ids:
            assert sv.wait(rid, timeout=300) == 2
            results.append(sv.result(rid)[0])
        assert sv.wait(busy, timeout=300) == 2
    for k, ((L, h, nt, S, sweeps, layout), acc) in enumerate(zip(SERVED, results)):
        seed = 300 + k
        T = inputs.geometric_ladder(0.5, 1.6, nt)
        st = orc.State(L, T, h, False, seed=seed, J=orc.pmj_couplings(seed, S, L),
                       spins=orc.init_spins(seed, S, nt, L), rng_group=64 if layout else 1,
                       n_therm=sweeps // 2)
        st.run(sweeps, threads=THREADS)
        np.testing.assert_array_equal(acc, st.acc, err_msg=f"served request {k} (L={L})")


@pytest.mark.parametrize("dist,layout", [("gauss", 0), ("pmj", 1)])
def test_schedule_tuner_applies_its_choice_and_matches_oracle(dist, layout):
    """sg_autotune_schedule times each sweeps-per-exchange candidate on the
    ensemble's own data, restores the state, and applies its pick: with a
    wide tolerance the most frequent exchange (3 of {0, 3, 8}); the run that
    follows equals the oracle's at that schedule, bit for bit."""
    L, nt, S, sweeps = 6, 6, 64, 40
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=12)
    extra = dict(layout=sgmc.SG_LAYOUT_MSC64) if layout else {}
    with sgmc.Ensemble(L, 0.2, T, dist, S, 13, J=J, spins=s0, n_therm=10, **extra) as ens:
        rep = ens.autotune_schedule([0, 3, 8], trial_sweeps=4, tolerance=10.0)
        assert rep["exchange_every"] == 3
        assert all(v > 0 for v in rep["ms_per_sweep"])
        assert ens.sweeps_done == 0
        np.testing.assert_array_equal(ens.spins(), s0)
        assert not ens.accumulators().any()
        ens.sweep(sweeps)
        ens.synchronize()
        st = orc.State(L, T, 0.2, dist == "gauss", seed=13, J=J, spins=s0, n_therm=10,
                       exchange_every=3, rng_group=64 if layout else 1)
        st.run(sweeps, threads=THREADS)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        np.testing.assert_array_equal(ens.accumulators(), st.acc)
        # tolerance 0: the fastest candidate wins; bad arguments are refused
        rep0 = ens.autotune_schedule([1, 4], trial_sweeps=2, tolerance=0.0)
        best = [1, 4][int(np.argmin(rep0["ms_per_sweep"]))]
        assert rep0["exchange_every"] == best
        for bad in ([], [-1, 2]):
            with pytest.raises(sgmc.SgError) as ei:
                ens.autotune_schedule(bad)
            assert ei.value.status == sgmc.SG_EINVAL
