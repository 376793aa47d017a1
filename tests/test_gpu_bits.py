"""The bit-per-chain state (one bit per chain in shared memory, the paper's
multispin coding of one sample's replicas; methods section) against the CPU
oracle through the C ABI: +-J swept bit-parallel, Gaussian couplings by
chain sets.

Every chain keeps its own Metropolis random words, so the path must
reproduce the oracle's standard run bit for bit (spins, B, M, every FP64
accumulator, the overlap histogram) for every lattice size it serves, one
word or two per site row (up to 32 or 64 temperatures), ragged slot counts
and segmented launches; and it must equal the byte-per-chain path.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))
BITS = dict(state_mode=3)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    sgbuild.build()


def snapshot(e):
    B, M = e.energies()
    return e.spins(), B, M, e.accumulators(), (e.histogram() if e.has_hist else None)


@pytest.mark.parametrize("L,nt,h,ee,me", [(4, 1, 0.3, 1, 1), (4, 8, 0.3, 1, 1), (6, 5, 0.0, 2, 1),
                                          (8, 32, 0.2, 1, 2), (8, 33, 0.1, 1, 1),
                                          (10, 56, 0.1, 1, 1), (12, 7, 0.25, 3, 1),
                                          (14, 4, 0.2, 1, 1), (16, 64, 0.05, 1, 1)])
def test_bit_parallel_sweeps_are_bit_exact_against_oracle(L, nt, h, ee, me):
    S, seed = 3, 500 + L + nt
    T = inputs.geometric_ladder(0.4, 1.8, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=L * 7 + nt)
    sweeps = 24 if L >= 12 else 60
    opt = dict(exchange_every=ee, measure_every=me, n_therm=sweeps // 3, log_bins=3, pq_hist=1)
    with sgmc.Ensemble(L, h, T, "pmj", S, seed, J=J, spins=s0, **BITS, **opt) as ens:
        ens.sweep(sweeps // 2)
        ens.sweep(sweeps - sweeps // 2)
        ens.synchronize()
        got = snapshot(ens)
    st = orc.State(L, T, h, False, seed=seed, J=J, spins=s0, exchange_every=ee, measure_every=me,
                   n_therm=sweeps // 3, log_bins=3, pq_hist=True)
    st.run(sweeps, threads=THREADS)
    np.testing.assert_array_equal(got[0], st.spins)
    np.testing.assert_array_equal(got[1], st.B)
    np.testing.assert_array_equal(got[2], st.M)
    np.testing.assert_array_equal(got[3], st.acc)
    np.testing.assert_array_equal(got[4], st.hist)


@pytest.mark.parametrize("L,S,nt", [(6, 700, 8), (10, 400, 56)])
def test_bit_parallel_equals_byte_path_with_segmented_launches(L, S, nt):
    """More samples than resident CTAs: the library splits launches into
    segments; the bit-parallel state gives the byte-per-chain run bit for
    bit, and the oracle agrees on sampled samples."""
    T = inputs.geometric_ladder(0.4, 1.8, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=91 + L)
    outs = []
    for mode in (3, 0):
        with sgmc.Ensemble(L, 0.1, T, "pmj", S, 17, J=J, spins=s0, state_mode=mode, n_therm=8) as e:
            if mode == 3:
                assert e.launch_plan(64)["segments"] > 1
            e.sweep(64)
            outs.append(snapshot(e)[:4])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    for s in (0, S - 1):
        st = orc.State(L, T, 0.1, False, seed=17, J=J[s:s + 1], spins=s0[s:s + 1], s_base=s,
                       n_therm=8)
        st.run(64)
        np.testing.assert_array_equal(outs[0][0][s], st.spins[0])
        np.testing.assert_array_equal(outs[0][3][s], st.acc[0])


@pytest.mark.parametrize("L,nt,h,ee,me,cs", [(4, 1, 0.3, 1, 1, 0), (4, 8, 0.3, 1, 1, 1),
                                             (6, 5, 0.0, 2, 1, 2), (8, 24, 0.2, 1, 1, 2),
                                             (8, 33, 0.1, 1, 2, 4), (10, 56, 0.1, 1, 1, 0),
                                             (12, 24, 0.25, 3, 1, 1), (12, 24, 0.2, 1, 1, 4),
                                             (14, 4, 0.2, 1, 1, 0), (16, 64, 0.05, 1, 1, 2)])
def test_gaussian_bit_parallel_sweeps_are_bit_exact_against_oracle(L, nt, h, ee, me, cs):
    """Gaussian couplings on the bit-per-chain state, every chain-set size:
    the screened Metropolis test, the exact threshold in its band and the
    2^-17 energy sums reproduce the oracle bit for bit."""
    S, seed = 3, 900 + L + nt
    T = inputs.geometric_ladder(0.4, 1.8, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=L * 11 + nt)
    sweeps = 24 if L >= 12 else 60
    opt = dict(exchange_every=ee, measure_every=me, n_therm=sweeps // 3, log_bins=3, pq_hist=1,
               chain_set=cs)
    with sgmc.Ensemble(L, h, T, "gauss", S, seed, J=J, spins=s0, **BITS, **opt) as ens:
        if cs:
            assert ens.info().chain_set == cs
        assert ens.info().chain_set in (1, 2, 4)
        ens.sweep(sweeps // 2)
        ens.sweep(sweeps - sweeps // 2)
        ens.synchronize()
        got = snapshot(ens)
    st = orc.State(L, T, h, True, seed=seed, J=J, spins=s0, exchange_every=ee, measure_every=me,
                   n_therm=sweeps // 3, log_bins=3, pq_hist=True)
    st.run(sweeps, threads=THREADS)
    np.testing.assert_array_equal(got[0], st.spins)
    np.testing.assert_array_equal(got[1], st.B)
    np.testing.assert_array_equal(got[2], st.M)
    np.testing.assert_array_equal(got[3], st.acc)
    np.testing.assert_array_equal(got[4], st.hist)


@pytest.mark.parametrize("L,S,nt,threads", [(8, 700, 24, 0), (12, 512, 24, 0), (10, 300, 20, 96)])
def test_gaussian_bit_parallel_equals_byte_path_in_segmented_launches(L, S, nt, threads):
    """Launches of 64 sweeps over more samples than one wave (segmented):
    the Gaussian bit-per-chain state gives the byte-per-chain run bit for
    bit, and the oracle agrees on the first, a middle and the last sample."""
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=41 + L)
    outs = []
    for mode in (3, 0):
        with sgmc.Ensemble(L, 0.2, T, "gauss", S, 23, J=J, spins=s0, state_mode=mode, n_therm=8,
                           threads_per_block=threads if mode == 3 else 0) as e:
            e.sweep(64)
            outs.append(snapshot(e)[:4])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    for s in (0, S // 2, S - 1):
        st = orc.State(L, T, 0.2, True, seed=23, J=J[s:s + 1], spins=s0[s:s + 1], s_base=s,
                       n_therm=8)
        st.run(64)
        np.testing.assert_array_equal(outs[0][0][s], st.spins[0])
        np.testing.assert_array_equal(outs[0][1][s], st.B[0])
        np.testing.assert_array_equal(outs[0][3][s], st.acc[0])


def test_bit_parallel_state_round_trips_and_options_are_checked():
    L, nt, S = 8, 40, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=3)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, 5, J=J, spins=s0, **BITS) as e:
        np.testing.assert_array_equal(e.spins(), s0)
        e.sweep(7)
        e.exchange(1)
        got = e.spins()
        e.set_spins(-got)
        np.testing.assert_array_equal(e.spins(), -got)
        assert e.info().state_in_shared == 1
    for bad in (dict(nt=65), dict(layout=sgmc.SG_LAYOUT_MSC64), dict(dist="gauss", chain_set=3),
                dict(dist="gauss", chain_set=8)):
        n = bad.get("nt", 4)
        with pytest.raises(sgmc.SgError) as ei:
            sgmc.Ensemble(8, 0.1, inputs.geometric_ladder(0.5, 1.5, n), bad.get("dist", "pmj"),
                          64, 1, state_mode=3, layout=bad.get("layout", 0),
                          chain_set=bad.get("chain_set", 0))
        assert ei.value.status == sgmc.SG_EINVAL
    # Gaussian couplings on the bit-per-chain state round-trip too
    Jg, sg0 = inputs.make_instance("gauss", L, S, nt, seed=4)
    with sgmc.Ensemble(L, 0.2, T, "gauss", S, 5, J=Jg, spins=sg0, **BITS) as e:
        np.testing.assert_array_equal(e.spins(), sg0)
        e.sweep(5)
        e.exchange(0)
        got = e.spins()
        e.set_spins(-got)
        np.testing.assert_array_equal(e.spins(), -got)
        assert e.info().state_in_shared == 1 and e.info().chain_set in (1, 2, 4)
