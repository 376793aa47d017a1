"""The allocation-free measurement entry point, through the C ABI.

sg_measure_noalloc is for callers that cannot call cudaMalloc when they
measure (a serving loop that keeps the allocator off its latency path, a host
whose device memory belongs to another framework's pool). It must give what
sg_measure gives, call after call, although every call reuses the same static
device array; it refuses a capturing stream without spoiling the capture.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

pytestmark = pytest.mark.gpu

ATOL = 2e-6  # the tolerance of the sg_measure parity test


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    sgbuild.build()


@pytest.mark.parametrize("dist", ["pmj", "gauss"])
def test_noalloc_measure_matches_allocating_measure_on_consecutive_calls(dist):
    L, S, nt = 6, 5, 7
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    J, s0 = inputs.make_instance(dist, L, S, nt, seed=17)
    k1 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [2, -1, 3]])
    k2 = np.array([[1, 1, 0], [0, 0, 1]])
    with sgmc.Ensemble(L, 0.2, T, dist, S, 5, J=J, spins=s0) as ens:
        a1 = ens.measure_noalloc(k1)
        np.testing.assert_allclose(a1, ens.measure(k1), atol=ATOL, rtol=0)
        ens.sweep(7)
        # second call in a row: new configuration, new k-set, same static array
        a2 = ens.measure_noalloc(k2)
        np.testing.assert_allclose(a2, ens.measure(k2), atol=ATOL, rtol=0)
        a3 = ens.measure_noalloc(k1)
        np.testing.assert_allclose(a3, ens.measure(k1), atol=ATOL, rtol=0)
        assert not np.array_equal(a1, a3)  # the configuration moved on


def test_noalloc_measure_rejects_requests_beyond_its_array():
    L, S, nt = 4, 8, 4
    T = inputs.geometric_ladder(0.5, 1.5, nt)
    with sgmc.Ensemble(L, 0.1, T, "pmj", S, 3) as ens:
        too_many_k = np.zeros((257, 3), dtype=np.int32)
        with pytest.raises(sgmc.SgError) as ei:
            ens.measure_noalloc(too_many_k)
        assert ei.value.status == sgmc.SG_EINVAL
        ok = ens.measure_noalloc(np.array([[1, 0, 0]]))
        np.testing.assert_allclose(ok, ens.measure(np.array([[1, 0, 0]])), atol=ATOL, rtol=0)
    # output larger than SG_MEASURE_NOALLOC_MAX_FLOATS floats
    with sgmc.Ensemble(2, 0.1, [1.0], "pmj", 2 ** 13, 3) as big:
        with pytest.raises(sgmc.SgError) as ei:
            big.measure_noalloc(np.zeros((65, 3), dtype=np.int32))
        assert ei.value.status == sgmc.SG_EINVAL


def test_noalloc_measure_status_for_msc_and_for_a_capturing_stream():
    """The multispin-coded layout is not served (SG_EUNSUPPORTED). A call
    made while the ensemble's stream is being captured returns
    SG_EUNSUPPORTED before it touches the stream: the capture completes and
    replays, and the next call outside the capture measures as before."""
    import torch
    T = inputs.geometric_ladder(0.5, 1.5, 4)
    with sgmc.Ensemble(4, 0.1, T, "pmj", 64, 3, layout=sgmc.SG_LAYOUT_MSC64) as msc:
        with pytest.raises(sgmc.SgError) as ei:
            msc.measure_noalloc(np.array([[1, 0, 0]]))
        assert ei.value.status == sgmc.SG_EUNSUPPORTED
    side = torch.cuda.Stream()
    k = np.array([[1, 0, 0], [0, 1, 1]])
    with sgmc.Ensemble(4, 0.1, T, "pmj", 3, 3, stream=side) as ens:
        want = ens.measure(k)
        np.testing.assert_allclose(ens.measure_noalloc(k), want, atol=ATOL, rtol=0)
        x = torch.zeros(16, device="cuda")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            with pytest.raises(sgmc.SgError) as ei:
                ens.measure_noalloc(k)
            y = x + 1.0
        assert ei.value.status == sgmc.SG_EUNSUPPORTED
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, torch.ones(16, device="cuda"))
        np.testing.assert_allclose(ens.measure_noalloc(k), want, atol=ATOL, rtol=0)
