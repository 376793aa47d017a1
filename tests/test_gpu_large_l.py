"""Large lattices (L = 26 .. 64) on the int8 path with the state in global
memory, against the CPU oracle through the C ABI: spins, energies, binned
accumulators and the overlap histogram agree bit for bit. L = 26 has the
longest run of colour sites (lcm(13, 4) = 52), where the byte-wise sums of
unsatisfied +-J bonds are flushed every four sites."""
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


@pytest.mark.parametrize("L,nt,dist,S,sweeps", [
    (26, 3, "pmj", 2, 6), (28, 2, "gauss", 1, 5), (32, 5, "pmj", 2, 4), (32, 2, "gauss", 2, 4),
    (40, 2, "gauss", 1, 3), (64, 1, "pmj", 1, 2)])
def test_large_lattice_is_bit_exact(L, nt, dist, S, sweeps):
    T = inputs.geometric_ladder(0.6, 1.5, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=L)
    opt = dict(log_bins=3, pq_hist=1)
    with sgmc.Ensemble(L, 0.15, T, dist, S, 100 + L, J=J, spins=s0, **opt) as ens:
        ens.sweep(sweeps - 1)
        ens.sweep(1)
        st = orc.State(L, T, 0.15, dist == "gauss", seed=100 + L, J=J, spins=s0, log_bins=3,
                       pq_hist=True)
        st.run(sweeps, threads=THREADS)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        B, M = ens.energies()
        np.testing.assert_array_equal(B, st.B)
        np.testing.assert_array_equal(M, st.M)
        np.testing.assert_array_equal(ens.accumulators(), st.acc)
        np.testing.assert_array_equal(ens.histogram(), st.hist)


def test_library_drawn_large_instance_matches_oracle_generators():
    L, S, nt, seed = 32, 2, 3, 9
    T = inputs.geometric_ladder(0.6, 1.5, nt)
    with sgmc.Ensemble(L, 0.2, T, "pmj", S, seed) as ens:
        np.testing.assert_array_equal(ens.couplings(), orc.pmj_couplings(seed, S, L))
        np.testing.assert_array_equal(ens.spins(), orc.init_spins(seed, S, nt, L))


def test_unbuilt_lattice_sizes_are_rejected():
    T = inputs.geometric_ladder(0.6, 1.5, 2)
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(34, 0.2, T, "pmj", 1, 1)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(66, 0.2, T, "pmj", 1, 1)
    assert ei.value.status == sgmc.SG_EINVAL


def test_few_large_samples_get_wide_ctas():
    """One CTA per sample: with fewer samples than the SMs could hold CTAs,
    the launch must use wide CTAs, not many narrow ones that never come."""
    T = inputs.geometric_ladder(0.5, 1.6, 32)
    with sgmc.Ensemble(16, 0.1, T, "gauss", 256, 1) as ens:
        info = ens.info()
        assert info.state_in_shared == 0 and info.grid <= 256
        assert info.threads_per_block >= 256, info.threads_per_block
    with sgmc.Ensemble(12, 0.1, inputs.geometric_ladder(0.5, 1.6, 24), "gauss", 512, 1) as ens:
        info = ens.info()
        assert info.state_in_shared == 1 and info.threads_per_block >= 64


# the narrow shared-memory instance of L = 10, 12 is bounded at 320 threads
NARROW_MAX = 320


@pytest.mark.parametrize("L,nt,dist,S", [(10, 56, "gauss", 3), (10, 56, "pmj", 2), (12, 40, "pmj", 2),
                                         (12, 24, "gauss", 2)])
def test_wide_shared_memory_instance_is_bit_exact(L, nt, dist, S):
    """Many temperatures (one sample per SM's shared memory) or fewer samples
    than SMs: L = 10, 12 run the wide instance (one CTA of up to 512 threads
    per SM), which must give the oracle's chain bit for bit."""
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=L + nt)
    with sgmc.Ensemble(L, 0.2, T, dist, S, 31, J=J, spins=s0, state_mode=1, log_bins=2,
                       pq_hist=1) as ens:
        info = ens.info()
        assert info.state_in_shared == 1 and info.threads_per_block > NARROW_MAX, info.threads_per_block
        ens.sweep(3)
        ens.sweep(2)
        st = orc.State(L, T, 0.2, dist == "gauss", seed=31, J=J, spins=s0, log_bins=2, pq_hist=True)
        st.run(5, threads=THREADS)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        B, M = ens.energies()
        np.testing.assert_array_equal(B, st.B)
        np.testing.assert_array_equal(M, st.M)
        np.testing.assert_array_equal(ens.accumulators(), st.acc)
        np.testing.assert_array_equal(ens.histogram(), st.hist)


def test_instance_choice_follows_occupancy_and_requests():
    """Many samples with few temperatures keep two narrow CTAs per SM; many
    temperatures (one sample per SM) take the wide instance; a requested CTA
    size above the narrow bound selects the wide instance, and both give the
    same chain."""
    many = inputs.geometric_ladder(0.5, 1.6, 56)
    few = inputs.geometric_ladder(0.5, 1.6, 24)
    with sgmc.Ensemble(12, 0.1, few, "gauss", 1024, 1) as ens:
        assert ens.info().threads_per_block <= NARROW_MAX
    with sgmc.Ensemble(10, 0.1, many, "gauss", 1024, 1) as ens:
        assert ens.info().threads_per_block > NARROW_MAX
    J, s0 = inputs.make_instance("gauss", 12, 3, 24, seed=5)
    got = []
    for req in (120, 480):
        with sgmc.Ensemble(12, 0.1, few, "gauss", 3, 8, J=J, spins=s0, threads_per_block=req) as ens:
            assert ens.info().threads_per_block == req
            ens.sweep(6)
            got.append((ens.spins(), ens.accumulators()))
    np.testing.assert_array_equal(got[0][0], got[1][0])
    np.testing.assert_array_equal(got[0][1], got[1][1])


@pytest.mark.parametrize("L,dist", [(10, "gauss"), (12, "pmj")])
def test_state_in_shared_or_global_memory_gives_the_same_chain(L, dist):
    T = inputs.geometric_ladder(0.5, 1.6, 6)
    J, s0 = inputs.make_instance(dist, L, 5, 6, seed=L)
    out = []
    for mode in (1, 2):
        with sgmc.Ensemble(L, 0.2, T, dist, 5, 3, J=J, spins=s0, state_mode=mode, log_bins=3,
                           pq_hist=1) as ens:
            assert ens.info().state_in_shared == (1 if mode == 1 else 0)
            ens.sweep(25)
            out.append((ens.spins(), ens.accumulators(), ens.histogram()))
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_state_mode_requests_that_cannot_be_met_are_rejected():
    T = inputs.geometric_ladder(0.5, 1.6, 32)
    with pytest.raises(sgmc.SgError) as ei:  # 262 KB of spins per sample
        sgmc.Ensemble(16, 0.2, T, "gauss", 4, 1, state_mode=1)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED
    with pytest.raises(sgmc.SgError) as ei:  # no global-memory kernel below L = 10
        sgmc.Ensemble(8, 0.2, T, "gauss", 4, 1, state_mode=2)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED
    with pytest.raises(sgmc.SgError) as ei:  # one bit per chain: L = 4..16 only
        sgmc.Ensemble(18, 0.2, T, "gauss", 4, 1, state_mode=3)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED


@pytest.mark.parametrize("nt,dist", [(64, "pmj"), (1, "gauss"), (9, "gauss")])
def test_packed_state_edge_slot_counts_are_bit_exact(nt, dist):
    """Global-memory (packed) state with 64 temperatures (the exchange masks
    use all 64 bits), a single temperature (one 4-slot group) and a ragged
    group, against the oracle."""
    L, S = 10, 2
    T = inputs.geometric_ladder(0.4, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=nt)
    with sgmc.Ensemble(L, 0.2, T, dist, S, 31, J=J, spins=s0, state_mode=2, log_bins=2,
                       pq_hist=1) as ens:
        assert ens.info().state_in_shared == 0
        ens.sweep(6)
        st = orc.State(L, T, 0.2, dist == "gauss", seed=31, J=J, spins=s0, log_bins=2, pq_hist=True)
        st.run(6, threads=THREADS)
        np.testing.assert_array_equal(ens.spins(), st.spins)
        np.testing.assert_array_equal(ens.energies()[0], st.B)
        np.testing.assert_array_equal(ens.accumulators(), st.acc)
        np.testing.assert_array_equal(ens.histogram(), st.hist)


def test_standalone_calls_on_packed_state_match_shared_memory_state():
    """Calls that read or change the state outside the fused kernel (standalone
    exchange and measurement, spin get/set, a rejected asynchronous upload)
    go through the ensemble's unpacked copy; they must give what the same
    calls give on the shared-memory state."""
    L, nt, S = 12, 6, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=77)
    kv = [[1, 0, 0], [0, 2, 1], [3, 1, -1]]
    out = {}
    for mode in (1, 2):
        with sgmc.Ensemble(L, 0.2, T, "gauss", S, 13, J=J, spins=s0, state_mode=mode) as e:
            e.sweep(7)
            e.exchange(1)
            e.sweep(3)
            m = e.measure(kv)
            bad = e.spins().copy()
            bad.reshape(-1)[5] = 0
            e.set_spins_async(bad)
            with pytest.raises(sgmc.SgError):
                e.synchronize()
            e.sweep(2)
            flipped = -e.spins()
            e.set_spins(flipped)
            e.sweep(2)
            out[mode] = (m, e.spins(), e.energies()[0], e.accumulators())
    for a, b in zip(out[1], out[2]):
        np.testing.assert_array_equal(a, b)
