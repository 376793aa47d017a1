"""Multi-rank path on CPU (gloo, world size 2): sample shards keyed by their
global index reproduce the unsplit run, the accumulator gather rebuilds the
full (sweep-binned) array in rank order and the histogram reduction gives the
unsplit histogram. The per-shard compute here is the oracle (no
GPU); the sharding and gather logic under test is the product's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as orc
from paper_1403_4560_b300 import inputs, shard

L, S, NT, SEED, SWEEPS, BINS = 4, 11, 3, 21, 40, 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T = inputs.geometric_ladder(0.5, 1.5, NT)
    J, s0 = inputs.make_instance("pmj", L, S, NT, seed=5)
    b, e = shard.shard_bounds(S, world, rank)
    st = orc.State(L, T, 0.2, False, seed=SEED, J=J[b:e], spins=s0[b:e], s_base=b, n_therm=10,
                   log_bins=BINS, pq_hist=True)
    st.run(SWEEPS)
    full = shard.gather_accumulators(st.acc)
    hist = shard.reduce_histogram(st.hist)
    if rank == 0:
        np.save(out_path, full)
        np.save(out_path + ".hist.npy", hist)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_partition_the_samples():
    for n, w, a in [(11, 2, 1), (256, 3, 64), (64, 4, 64), (5, 8, 1)]:
        parts = [shard.shard_bounds(n, w, r, a) for r in range(w)]
        assert parts[0][0] == 0 and parts[-1][1] == n
        assert all(p[1] == q[0] for p, q in zip(parts, parts[1:]))
        assert all((p[0] % a) == 0 for p in parts)


def test_two_gloo_ranks_reproduce_the_single_process_run(tmp_path):
    out = str(tmp_path / "acc.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    T = inputs.geometric_ladder(0.5, 1.5, NT)
    J, s0 = inputs.make_instance("pmj", L, S, NT, seed=5)
    st = orc.State(L, T, 0.2, False, seed=SEED, J=J, spins=s0, n_therm=10, log_bins=BINS,
                   pq_hist=True)
    st.run(SWEEPS)
    np.testing.assert_array_equal(np.load(out), st.acc)
    np.testing.assert_array_equal(np.load(out + ".hist.npy"), st.hist)
