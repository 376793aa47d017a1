"""Large lattices with each sample swept by a thread-block cluster (the paper
cannot equilibrate its largest sizes with one sample per unit of hardware;
results and conclusion sections), against the CPU oracle through the C ABI.

The cluster instances split a sample's z-planes over k = 2, 4 or 8 CTAs that
exchange their boundary planes through L2 and gather energies, exchange
decisions and overlap marginals at rank 0. They must reproduce the oracle
bit for bit: spins, B, M, every FP64 accumulator and the overlap histogram,
for +-J and Gaussian couplings, whatever the cluster size; the library picks
a cluster when the samples are fewer than the SMs; a watchdog stop ends
every CTA of a cluster together.
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


def snapshot(e):
    B, M = e.energies()
    return e.spins(), B, M, e.accumulators(), (e.histogram() if e.has_hist else None)


@pytest.mark.parametrize("L,k,dist,nt", [(24, 2, "gauss", 4), (24, 4, "pmj", 5), (24, 8, "gauss", 3),
                                         (32, 2, "pmj", 4), (32, 4, "gauss", 6), (32, 8, "pmj", 2),
                                         (20, 4, "gauss", 9), (28, 2, "pmj", 4),
                                         (40, 8, "gauss", 2), (48, 4, "pmj", 3)])
def test_cluster_split_is_bit_exact_against_oracle(L, k, dist, nt):
    S, h, seed, sweeps = 3, 0.15, 40 + L + k, 10
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=L * 10 + k)
    opt = dict(n_therm=3, log_bins=3, pq_hist=1)
    with sgmc.Ensemble(L, h, T, dist, S, seed, J=J, spins=s0, cluster=k, **opt) as ens:
        info = ens.info()
        assert info.cluster == k and info.grid % k == 0 and not info.state_in_shared
        ens.sweep(6)
        ens.sweep(sweeps - 6)
        ens.synchronize()
        got = snapshot(ens)
    st = orc.State(L, T, h, dist == "gauss", seed=seed, J=J, spins=s0, n_therm=3, log_bins=3,
                   pq_hist=True)
    st.run(sweeps, threads=THREADS)
    np.testing.assert_array_equal(got[0], st.spins)
    np.testing.assert_array_equal(got[1], st.B)
    np.testing.assert_array_equal(got[2], st.M)
    np.testing.assert_array_equal(got[3], st.acc)
    np.testing.assert_array_equal(got[4], st.hist)


def test_cluster_measurement_in_several_chunks_matches_oracle():
    """L = 64 with 24 temperatures: the overlap marginals of a sample's six
    4-slot words do not fit one CTA's shared memory at once, so each
    measurement runs in chunks, every chunk's partial marginals gathered at
    rank 0 between cluster barriers; one sample over 4 CTAs, against the
    oracle bit for bit."""
    L, S, nt, h, seed, sweeps = 64, 1, 24, 0.1, 3, 2
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=64)
    with sgmc.Ensemble(L, h, T, "pmj", S, seed, J=J, spins=s0, cluster=4) as ens:
        assert ens.info().cluster == 4
        ens.sweep(sweeps)
        got = snapshot(ens)
    st = orc.State(L, T, h, False, seed=seed, J=J, spins=s0)
    st.run(sweeps)
    np.testing.assert_array_equal(got[0], st.spins)
    np.testing.assert_array_equal(got[1], st.B)
    np.testing.assert_array_equal(got[3], st.acc)


def test_library_picks_a_cluster_for_few_samples_and_results_do_not_change():
    """12 samples of L = 24 (fewer than the SMs): the library sweeps each
    with a cluster; the run equals the one-CTA-per-sample run bit for bit,
    and sampled samples equal the oracle."""
    L, S, nt, h, seed, sweeps = 24, 12, 4, 0.2, 5, 8
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("gauss", L, S, nt, seed=77)
    outs = []
    for cl in (0, 1):
        with sgmc.Ensemble(L, h, T, "gauss", S, seed, J=J, spins=s0, cluster=cl) as ens:
            if cl == 0:
                assert ens.info().cluster > 1
            else:
                assert ens.info().cluster == 1
            ens.sweep(sweeps)
            outs.append(snapshot(ens)[:4])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    for s in (0, S - 1):
        st = orc.State(L, T, h, True, seed=seed, J=J[s:s + 1], spins=s0[s:s + 1], s_base=s)
        st.run(sweeps)
        np.testing.assert_array_equal(outs[0][0][s], st.spins[0])
        np.testing.assert_array_equal(outs[0][3][s], st.acc[0])


def test_clusters_taking_several_samples_each_match_one_cta_per_sample():
    """More samples than resident clusters (L = 24, 180 samples, clusters of
    2 CTAs, at most ~74 resident): each cluster loops over several samples,
    rank 0's shared sums and flags reused between them; the run equals one
    CTA per sample bit for bit, and the last sample equals the oracle."""
    L, S, nt, h, seed, sweeps = 24, 180, 2, 0.3, 9, 4
    T = inputs.geometric_ladder(0.5, 1.6, nt)
    J, s0 = inputs.make_instance("pmj", L, S, nt, seed=180)
    outs = []
    for cl in (2, 1):
        with sgmc.Ensemble(L, h, T, "pmj", S, seed, J=J, spins=s0, cluster=cl, n_therm=1) as e:
            if cl == 2:
                assert e.info().grid < 2 * S  # fewer clusters than samples
            e.sweep(sweeps)
            outs.append(snapshot(e)[:4])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    s = S - 1
    st = orc.State(L, T, h, False, seed=seed, J=J[s:s + 1], spins=s0[s:s + 1], s_base=s,
                   n_therm=1)
    st.run(sweeps)
    np.testing.assert_array_equal(outs[0][0][s], st.spins[0])
    np.testing.assert_array_equal(outs[0][3][s], st.acc[0])


def test_cluster_options_are_checked():
    T = inputs.geometric_ladder(0.5, 1.6, 4)
    for bad in (3, 5, -1):
        with pytest.raises(sgmc.SgError) as ei:
            sgmc.Ensemble(24, 0.1, T, "pmj", 2, 1, cluster=bad)
        assert ei.value.status == sgmc.SG_EINVAL
    # no cluster kernel for L = 18 (not a multiple of 4) or a shared-memory state
    with pytest.raises(sgmc.SgError) as ei:
        sgmc.Ensemble(18, 0.1, T, "pmj", 2, 1, cluster=2)
    assert ei.value.status == sgmc.SG_EUNSUPPORTED
    with sgmc.Ensemble(8, 0.1, T, "pmj", 2, 1, cluster=0) as e:
        assert e.info().cluster == 1


def test_watchdog_stops_every_cta_of_a_cluster_with_a_status():
    """A launch whose clock budget runs out stops all CTAs of each cluster at
    the same sweep (rank 0 collects the ranks' reasons before the barrier)
    and reports SG_ETIMEOUT; the context stays usable."""
    L, S, nt = 24, 4, 8
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.1, T, "gauss", S, 1, cluster=4, watchdog_cycles=20000) as ens:
        ens.sweep(500)
        with pytest.raises(sgmc.SgError) as ei:
            ens.synchronize()
        assert ei.value.status == sgmc.SG_ETIMEOUT
    with sgmc.Ensemble(L, 0.1, T, "pmj", 2, 1, cluster=2) as ens:
        ens.sweep(3)
        ens.synchronize()
