"""Serving loop (continuous batching) on the GPU, through the C ABI: every
request's result equals the same run alone, whatever ran beside it; memory
admission, cancellation and the latency statistics work."""
import threading
import time

import numpy as np
import pytest

from paper_1403_4560_b300 import build as sgbuild
from paper_1403_4560_b300 import inputs, sgmc

pytestmark = pytest.mark.gpu

REQS = [  # L, h, nt, dist, samples, sweeps
    (8, 0.1, 6, "pmj", 64, 60),     # multispin-coded
    (6, 0.3, 5, "gauss", 7, 45),
    (12, 0.2, 4, "pmj", 10, 30),
    (20, 0.05, 3, "gauss", 2, 8),   # state in global memory
    (4, 0.4, 8, "pmj", 128, 100),   # multispin-coded, two words
    (10, 0.2, 6, "gauss", 5, 37),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for the gpu-marked tests")
    sgbuild.build()


def alone(L, h, nt, dist, S, sweeps, seed, T=None):
    T = inputs.geometric_ladder(0.5, 1.6, nt) if T is None else T
    layout = sgmc.SG_LAYOUT_MSC64 if (dist == "pmj" and S % 64 == 0 and L <= 16) else 0
    with sgmc.Ensemble(L, h, T, dist, S, seed, layout=layout, n_therm=sweeps // 2) as e:
        e.sweep(sweeps)
        return e.accumulators()


@pytest.mark.parametrize("use_graph", [False, True])
def test_results_are_the_same_alone_and_in_the_mix(use_graph):
    with sgmc.Server(chunk_sweeps=16, use_graph=use_graph) as sv:
        ids = []
        # submit from two host threads, staggered, so requests join mid-flight
        def submit(lst):
            for k in lst:
                L, h, nt, dist, S, sweeps = REQS[k]
                ids.append((k, sv.submit(L, h, inputs.geometric_ladder(0.5, 1.6, nt), dist, S,
                                         seed=100 + k, n_sweeps=sweeps)))
                time.sleep(0.01)
        th = [threading.Thread(target=submit, args=(lst,)) for lst in ([0, 2, 4], [1, 3, 5])]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for k, rid in ids:
            assert sv.wait(rid, timeout=300) == 2
            acc, lat = sv.result(rid)
            assert lat > 0
            L, h, nt, dist, S, sweeps = REQS[k]
            np.testing.assert_array_equal(acc, alone(L, h, nt, dist, S, sweeps, 100 + k))
        st = sv.stats()
        assert st["completed"] == len(REQS)
        assert st["latency_p99"] >= st["latency_p50"] > 0
        assert st["attempts"] > 0 and st["device_bytes_in_use"] == 0


def test_memory_admission_queues_and_completes():
    T = inputs.geometric_ladder(0.5, 1.5, 4)
    one = sgmc.lib().sg_ensemble_bytes(8, 4, 16, sgmc.SG_GAUSS, None)
    with sgmc.Server(memory_budget=int(one * 1.5), chunk_sweeps=8) as sv:
        rids = [sv.submit(8, 0.2, T, "gauss", 16, seed=s, n_sweeps=24) for s in range(4)]
        seen_queue = False
        for _ in range(200):
            st = sv.stats()
            seen_queue |= st["queued"] > 0 and st["active"] <= 1
            if st["completed"] == 4:
                break
            time.sleep(0.01)
        for r in rids:
            assert sv.wait(r, timeout=300) == 2
        assert seen_queue
        acc, _ = sv.result(rids[2])
        np.testing.assert_array_equal(acc, alone(8, 0.2, 4, "gauss", 16, 24, 2, T=T))
        # a request that can never fit fails instead of blocking the queue
        big = sv.submit(16, 0.2, T, "gauss", 4096, seed=1, n_sweeps=4)
        assert sv.wait(big, timeout=60) == 3
        with pytest.raises(sgmc.SgError) as ei:
            sv.result(big)
        assert ei.value.status == sgmc.SG_ENOMEM


def test_cancel_a_running_request():
    T = inputs.geometric_ladder(0.5, 1.5, 8)
    with sgmc.Server(chunk_sweeps=4) as sv:
        rid = sv.submit(12, 0.2, T, "gauss", 64, seed=3, n_sweeps=1_000_000)
        time.sleep(0.3)
        sv.cancel(rid)
        assert sv.wait(rid, timeout=120) == 4
        with pytest.raises(sgmc.SgError) as ei:
            sv.result(rid)
        assert ei.value.status == sgmc.SG_ECANCELLED
        ok = sv.submit(4, 0.2, T, "pmj", 3, seed=4, n_sweeps=10)
        assert sv.wait(ok, timeout=120) == 2
