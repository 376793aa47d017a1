"""GPU parity of the logarithmic sweep bins and the overlap histogram P(q)
against the CPU oracle, through the C ABI: binned FP64 accumulators and the
integer histogram agree bit for bit on the int8 path (+-J and Gaussian, shared
and global-memory state), the multispin-coded path, batched graph launches and
a checkpoint/restore; the per-bin estimators match the host estimators on the
bin's slice."""
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


def oracle_for(L, T, h, dist, seed, J, s0, **opt):
    return orc.State(L, T, h, dist == "gauss", seed=seed, J=J, spins=s0,
                     rng_group=opt.get("rng_group", 1), exchange_every=opt.get("exchange_every", 1),
                     measure_every=opt.get("measure_every", 1), n_therm=opt.get("n_therm", 0),
                     s_base=opt.get("sample_base", 0), log_bins=opt.get("log_bins", 1),
                     pq_hist=bool(opt.get("pq_hist", 0)))


def check(ens, st):
    np.testing.assert_array_equal(ens.spins(), st.spins)
    np.testing.assert_array_equal(ens.accumulators(), st.acc)
    if st.hist is not None:
        np.testing.assert_array_equal(ens.histogram(), st.hist)


@pytest.mark.parametrize("L,nt,dist,S,bins,therm,every", [
    (4, 6, "pmj", 5, 6, 0, 1), (6, 5, "gauss", 3, 5, 2, 2), (8, 3, "pmj", 2, 64, 0, 1),
    (2, 4, "gauss", 7, 3, 1, 1), (20, 2, "gauss", 1, 4, 0, 1)])
def test_int8_bins_and_histogram_bit_exact(L, nt, dist, S, bins, therm, every):
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=40 + L)
    opt = dict(log_bins=bins, pq_hist=1, n_therm=therm, measure_every=every)
    sweeps = 9 if L >= 20 else 70
    with sgmc.Ensemble(L, 0.25, T, dist, S, 3 + L, J=J, spins=s0, **opt) as ens:
        ens.sweep(sweeps // 3)
        ens.sweep(sweeps - sweeps // 3)
        st = oracle_for(L, T, 0.25, dist, 3 + L, J, s0, **opt)
        st.run(sweeps, threads=THREADS)
        check(ens, st)


@pytest.mark.parametrize("L,nt,S", [(4, 4, 64), (8, 3, 128)])
def test_msc_bins_and_histogram_bit_exact(L, nt, S):
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=70 + L)
    opt = dict(log_bins=5, pq_hist=1, n_therm=1)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 5 + L, J=J, spins=s0,
                       layout=sgmc.SG_LAYOUT_MSC64, **opt) as ens:
        ens.sweep(45)
        st = oracle_for(L, T, 0.2, "pmj", 5 + L, J, s0, rng_group=64, **opt)
        st.run(45, threads=THREADS)
        check(ens, st)


def test_batched_graph_launches_bin_by_global_sweep():
    """Graph replays read the sweep index on the device; bins must follow it."""
    T = inputs.geometric_ladder(0.5, 1.5, 4)
    cases = [(4, "pmj", 6), (6, "gauss", 3)]
    ens, sts = [], []
    for L, dist, S in cases:
        J, s0 = inputs.make_instance(dist, L, S, 4, seed=L)
        opt = dict(log_bins=7, pq_hist=1)
        ens.append(sgmc.Ensemble(L, 0.1, T, dist, S, 11 * L, J=J, spins=s0, **opt))
        sts.append(oracle_for(L, T, 0.1, dist, 11 * L, J, s0, **opt))
    try:
        for _ in range(5):
            sgmc.sweep_batch(ens, 13, use_graph=True)
        for e, st in zip(ens, sts):
            st.run(65, threads=THREADS)
            check(e, st)
    finally:
        for e in ens:
            e.close()


def test_checkpoint_restore_continues_bins_and_histogram():
    L, nt, S = 6, 4, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=9)
    opt = dict(log_bins=8, pq_hist=1, n_therm=3)
    with sgmc.Ensemble(L, 0.3, T, "gauss", S, 21, J=J, spins=s0, **opt) as a:
        a.sweep(30)
        spins, acc, hist, done = a.spins(), a.accumulators(), a.histogram(), a.sweeps_done
        a.sweep(50)
        with sgmc.Ensemble(L, 0.3, T, "gauss", S, 21, J=J, spins=spins, **opt) as b:
            b.set_accumulators(acc)
            b.set_histogram(hist)
            b.set_sweeps_done(done)
            b.sweep(50)
            np.testing.assert_array_equal(b.accumulators(), a.accumulators())
            np.testing.assert_array_equal(b.histogram(), a.histogram())
            b.reset_accumulators()
            assert not b.histogram().any() and not b.accumulators().any()


def test_results_per_bin_match_host_estimators_on_the_slice():
    L, nt, S, bins = 4, 5, 24, 6
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 4, log_bins=bins) as ens:
        ens.sweep(63)
        acc = ens.accumulators()
        assert acc.shape == (S, nt, bins, sgmc.NACC)
        for b in (2, bins - 1):
            want = sgmc.observables_from_acc(np.ascontiguousarray(acc[:, :, b]), L)
            got = ens.results(b)
            for k in ("g", "chi0", "xi", "r12", "e"):
                np.testing.assert_array_equal(got[k], want[k])
        last = ens.results()
        np.testing.assert_array_equal(last["g"], ens.results(bins - 1)["g"])
        info = ens.info()
        assert info.log_bins == bins and info.pq_hist == 0


def test_bad_bin_and_histogram_requests_are_rejected():
    T = inputs.geometric_ladder(0.5, 1.5, 3)
    with sgmc.Ensemble(4, 0.2, T, "pmj", 2, 1) as ens:
        with pytest.raises(sgmc.SgError) as ei:
            ens.histogram()
        assert ei.value.status == sgmc.SG_EINVAL
        with pytest.raises(sgmc.SgError):
            ens.results(1)
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(4, 0.2, T, "pmj", 2, 1, log_bins=65)
    assert ei.value.status == sgmc.SG_EINVAL


def test_autotune_leaves_bins_and_histogram_untouched():
    L, nt, S = 6, 8, 40
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    opt = dict(log_bins=5, pq_hist=1)
    with sgmc.Ensemble(L, 0.2, T, "gauss", S, 8, **opt) as a, \
            sgmc.Ensemble(L, 0.2, T, "gauss", S, 8, **opt) as b:
        a.sweep(20)
        b.sweep(20)
        b.autotune(3)
        a.sweep(20)
        b.sweep(20)
        np.testing.assert_array_equal(a.accumulators(), b.accumulators())
        np.testing.assert_array_equal(a.histogram(), b.histogram())
