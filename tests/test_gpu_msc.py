"""GPU parity of the multispin-coded +-J path (64 samples per word) against the
CPU oracle run with RNG group 64, through the C ABI: spins, energies and
every FP64 accumulator must agree bit for bit."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))
MSC = dict(layout=sgmc.SG_LAYOUT_MSC64)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    sgbuild.build()


def oracle_state(L, T, h, seed, J, s0, s_base=0, **opt):
    return orc.State(L, T, h, False, seed=seed, J=J, spins=s0, rng_group=64,
                     exchange_every=opt.get("exchange_every", 1),
                     measure_every=opt.get("measure_every", 1), n_therm=opt.get("n_therm", 0),
                     s_base=s_base)


def assert_same(ens, st, samples=None):
    sl = slice(None) if samples is None else samples
    np.testing.assert_array_equal(ens.spins()[sl], st.spins)
    B, M = ens.energies()
    np.testing.assert_array_equal(B[sl], st.B)
    np.testing.assert_array_equal(M[sl], st.M)
    np.testing.assert_array_equal(ens.accumulators()[sl], st.acc)


@pytest.mark.parametrize("L,nt,h,ee,me,S", [
    (2, 3, 0.3, 1, 1, 64), (4, 4, 0.3, 1, 1, 64), (4, 5, 0.0, 2, 3, 128),
    (6, 1, 0.5, 1, 1, 64), (6, 6, 0.1, 1, 2, 64), (8, 4, 0.2, 0, 1, 64),
    (10, 3, 0.7, 1, 1, 64), (12, 2, 0.3, 1, 1, 64), (16, 2, 0.05, 1, 1, 64),
    # wide instance, both slots of a unit measured in one pass: several units,
    # single-slot edge units and two word groups
    (14, 3, 0.2, 1, 1, 64), (16, 5, 0.15, 1, 1, 128)])
def test_msc_is_bit_exact_against_int8_oracle_with_rng_group_64(L, nt, h, ee, me, S):
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=100 + L + nt)
    sweeps = 40 if L >= 12 else 90
    opt = dict(exchange_every=ee, measure_every=me, n_therm=sweeps // 3)
    with sgmc.Ensemble(L, h, T, "pmj", S, 9 + L, J=J, spins=s0, **MSC, **opt) as ens:
        ens.sweep(sweeps)
        ens.synchronize()
        st = oracle_state(L, T, h, 9 + L, J, s0, **opt)
        st.run(sweeps, threads=THREADS)
        assert_same(ens, st)


def test_msc_library_instance_and_int8_layout_agree():
    """Library-drawn couplings and spins are the same draws in both layouts,
    and the MSC run equals the int8 run with RNG group 64."""
    L, S, nt, seed = 4, 64, 4, 3
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, seed, **MSC) as m, \
            sgmc.Ensemble(L, 0.2, T, "pmj", S, seed, rng_group=64) as b:
        np.testing.assert_array_equal(m.couplings(), orc.pmj_couplings(seed, S, L))
        np.testing.assert_array_equal(m.spins(), orc.init_spins(seed, S, nt, L))
        np.testing.assert_array_equal(m.spins(), b.spins())
        m.sweep(30)
        b.sweep(30)
        np.testing.assert_array_equal(m.spins(), b.spins())
        np.testing.assert_array_equal(m.accumulators(), b.accumulators())
        np.testing.assert_array_equal(m.energies()[0], b.energies()[0])


def test_msc_full_size_sampled_parity():
    """L = 16, 4096 samples (64 words), 2 x 32 temperatures 0.4-1.5, h = 0.1,
    exchange and measurement every sweep, library-drawn instance; four samples
    re-run by the oracle from its own generators."""
    L, S, nt, h, seed, sweeps = 16, 4096, 32, 0.1, 77, 3
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    with sgmc.Ensemble(L, h, T, "pmj", S, seed, **MSC) as ens:
        ens.sweep(sweeps)
        ens.synchronize()
        spins, (B, M), acc = ens.spins(), ens.energies(), ens.accumulators()
    for s in (0, 63, 2047, 4095):
        J = orc.pmj_couplings(seed, 1, L, s_base=s)
        s0 = orc.init_spins(seed, 1, nt, L, s_base=s)
        st = oracle_state(L, T, h, seed, J, s0, s_base=s)
        st.run(sweeps)
        np.testing.assert_array_equal(spins[s:s + 1], st.spins)
        np.testing.assert_array_equal(B[s:s + 1], st.B)
        np.testing.assert_array_equal(M[s:s + 1], st.M)
        np.testing.assert_array_equal(acc[s:s + 1], st.acc)


def _paper_ladder():
    """The 56 temperatures of the paper's geometry as bench.py draws them."""
    return np.ascontiguousarray((1.0 / (0.1 * 18.0 ** (np.arange(56) / 55.0)))[::-1])


@pytest.mark.parametrize("L,S,ladder", [(16, 4096, "bench"), (10, 8192, "paper")])
def test_msc_bench_form_graph_replays_full_size_sampled_parity(L, S, ladder):
    """The multispin-coded ensembles as bench.py times them: a library-drawn
    instance, h = 0.1, exchange and measurement every sweep, sweeps through a
    replayed CUDA graph (device sweep counter; at L = 16 split sweeps whose
    measurement kernels decide on the device which sweeps they measure, at
    L = 10 the fused narrow kernel). Sampled samples, from each end of the
    word groups and the middle, against the oracle from its own generators."""
    h, seed, reps = 0.1, 5, 2
    T = inputs.geometric_ladder(0.4, 1.5, 32) if ladder == "bench" else _paper_ladder()
    with sgmc.Ensemble(L, h, T, "pmj", S, seed, n_therm=0, **MSC) as e:
        for _ in range(reps):
            sgmc.sweep_batch([e], 4, use_graph=True)
        e.synchronize()
        assert e.sweeps_done == 4 * reps
        spins, (B, M), acc = e.spins(), e.energies(), e.accumulators()
    for s in (0, 65, S // 2 + 31, S - 1):
        J = orc.pmj_couplings(seed, 1, L, s_base=s)
        s0 = orc.init_spins(seed, 1, len(T), L, s_base=s)
        st = oracle_state(L, T, h, seed, J, s0, s_base=s)
        st.run(4 * reps)
        np.testing.assert_array_equal(spins[s:s + 1], st.spins)
        np.testing.assert_array_equal(B[s:s + 1], st.B)
        np.testing.assert_array_equal(M[s:s + 1], st.M)
        np.testing.assert_array_equal(acc[s:s + 1], st.acc)


def test_msc_standalone_exchange_and_measure():
    L, S, nt = 4, 64, 5
    T = inputs.geometric_ladder(0.3, 3.0, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=12)
    with sgmc.Ensemble(L, 0.4, T, "pmj", S, 21, J=J, spins=s0, **MSC) as ens:
        st = oracle_state(L, T, 0.4, 21, J, s0)
        for parity in (0, 1, 1, 0):
            ens.exchange(parity)
            st.exchange(parity)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        np.testing.assert_array_equal(ens.energies()[0], st.B)
        k = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0]])
        got = ens.measure(k)
        sp = ens.spins()
    coords = np.array([[i % L, (i // L) % L, i // (L * L)] for i in range(L ** 3)])
    q = sp[:, 0].astype(np.float64) * sp[:, 1]
    want = (q[..., None] * np.exp(2j * np.pi / L * coords @ k.T)).mean(axis=-2)
    np.testing.assert_allclose(got[..., 0], want.real, atol=2e-6)
    np.testing.assert_allclose(got[..., 1], want.imag, atol=2e-6)


def test_msc_graph_batch_with_int8_matches_single_runs():
    L, S, nt = 6, 64, 3
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=5)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 8, J=J, spins=s0, **MSC) as ref:
        ref.sweep(12)
        want = (ref.spins(), ref.accumulators())
    a = sgmc.Ensemble(L, 0.2, T, "pmj", S, 8, J=J, spins=s0, **MSC)
    b = sgmc.Ensemble(4, 0.2, T, "gauss", 3, 8)
    try:
        sgmc.sweep_batch([a, b], 6, use_graph=True)
        sgmc.sweep_batch([a, b], 6, use_graph=True)
        a.synchronize()
        np.testing.assert_array_equal(a.spins(), want[0])
        np.testing.assert_array_equal(a.accumulators(), want[1])
    finally:
        a.close()
        b.close()


def test_msc_argument_checks():
    T = [1.0, 2.0]
    for kw in (dict(S=63, dist="pmj"), dict(S=64, dist="gauss")):
        with pytest.raises(sgmc.SgError) as ei:
            sgmc.Ensemble(4, 0.1, T, kw["dist"], kw["S"], 1, **MSC)
        assert ei.value.status == sgmc.SG_EINVAL
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(20, 0.1, T, "pmj", 64, 1, **MSC)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED


@pytest.mark.parametrize("L,nt", [(4, 5), (8, 4), (12, 3)])
def test_msc_cta_size_changes_speed_not_results(L, nt):
    """The narrow (128-thread) and wide (256, 512) kernel instances give the
    same chain, energies, accumulators and histogram bit for bit."""
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, 128, nt, seed=3 + L)
    ref = None
    for th in (128, 256, 512):
        with sgmc.Ensemble(L, 0.2, T, "pmj", 128, 17, J=J, spins=s0, threads_per_block=th,
                           log_bins=4, pq_hist=1, **MSC) as ens:
            ens.sweep(21)
            out = (ens.spins(), ens.energies(), ens.accumulators(), ens.histogram())
        if ref is None:
            ref = out
            continue
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1][0], ref[1][0])
        np.testing.assert_array_equal(out[2], ref[2])
        np.testing.assert_array_equal(out[3], ref[3])


def test_msc_autotune_changes_speed_not_results():
    L, nt, S = 6, 6, 128
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=12)
    with sgmc.Ensemble(L, 0.1, T, "pmj", S, 5, J=J, spins=s0, **MSC) as a, \
            sgmc.Ensemble(L, 0.1, T, "pmj", S, 5, J=J, spins=s0, **MSC) as b:
        a.sweep(10)
        b.sweep(10)
        rep = b.autotune(trial_sweeps=4)
        assert rep["threads_per_block"] in (128, 256, 512) and rep["n_candidates"] >= 2
        a.sweep(15)
        b.sweep(15)
        np.testing.assert_array_equal(a.spins(), b.spins())
        np.testing.assert_array_equal(a.accumulators(), b.accumulators())
        assert a.sweeps_done == b.sweeps_done == 25


@pytest.mark.parametrize("L,nt,ee,me,S", [(12, 5, 1, 1, 128), (14, 5, 1, 1, 128), (14, 6, 2, 3, 64),
                                          (16, 4, 1, 1, 64), (16, 3, 0, 2, 128)])
def test_replica_split_sweep_equals_fused_kernel_and_oracle(L, nt, ee, me, S):
    """At L >= 12 the sweeps run split by replica (one replica's chains of an
    exchange unit per CTA), and each measured sweep is measured by a kernel
    of its own (one CTA per slot and word group, from the stored chains). A
    run of a thermalising then a measuring call must equal the fused kernel
    throughout (an explicit CTA size selects it) bit for bit, through plain
    launches and a replayed CUDA graph (whose measurement kernels decide on
    the device which sweeps they measure), and the oracle on sample 0."""
    T = inputs.geometric_ladder(0.4, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=300 + L + nt)
    opt = dict(exchange_every=ee, measure_every=me, n_therm=9, log_bins=3, pq_hist=1)
    outs = []
    for tpb, graph in ((0, False), (0, True), (512, False)):
        with sgmc.Ensemble(L, 0.2, T, "pmj", S, 4, J=J, spins=s0, threads_per_block=tpb, **MSC,
                           **opt) as e:
            plan = e.launch_plan(18)
            assert plan["grid"] == (2 if tpb == 0 else 1) * e.info().grid
            n_meas = sum(1 for n in range(9, 18) if (n - 9) % me == 0)
            assert plan["launches"] == 18 + (n_meas if tpb == 0 else 0)
            if graph:
                sgmc.sweep_batch([e], 9, use_graph=True)
                sgmc.sweep_batch([e], 9, use_graph=True)
            else:
                e.sweep(9)
                e.sweep(9)
            e.synchronize()
            outs.append((e.spins(), e.energies()[0], e.energies()[1], e.accumulators(),
                         e.histogram()))
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)
    st = oracle_state(L, T, 0.2, 4, J[:1], s0[:1], exchange_every=ee, measure_every=me, n_therm=9)
    st.run(18)
    np.testing.assert_array_equal(outs[0][0][:1], st.spins)
    np.testing.assert_array_equal(outs[0][1][:1], st.B)
