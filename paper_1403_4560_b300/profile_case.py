"""Run one ensemble for profiling (ncu) or quick timing of a single kernel shape.

  python -m paper_1403_4560_b300.profile_case --L 12 --dist gauss --samples 148 \
      --nt 24 --sweeps 16 [--chunks 2]

Creates the ensemble from the seeded inputs, runs `chunks` launches of
`sweeps` sweeps each (exchange and measurement every sweep) and prints the
CUDA-event time of the last launch.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=12)
    ap.add_argument("--dist", default="gauss")
    ap.add_argument("--samples", type=int, default=148)
    ap.add_argument("--nt", type=int, default=24)
    ap.add_argument("--sweeps", type=int, default=16)
    ap.add_argument("--chunks", type=int, default=2)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--layout", type=int, default=0)
    ap.add_argument("--n-therm", type=int, default=0)
    ap.add_argument("--exchange-every", type=int, default=1)
    ap.add_argument("--measure-every", type=int, default=1)
    ap.add_argument("--state-mode", type=int, default=0)
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--chain-set", type=int, default=0)
    ap.add_argument("--h", type=float, default=0.2)
    args = ap.parse_args()

    import torch

    from paper_1403_4560_b300 import inputs, sgmc

    T = inputs.geometric_ladder(0.5, 1.6, args.nt)
    J, s0 = inputs.make_instance(args.dist, args.L, args.samples, args.nt, seed=7)
    stream = torch.cuda.current_stream()
    opt = dict(threads_per_block=args.threads, layout=args.layout, n_therm=args.n_therm,
               exchange_every=args.exchange_every, measure_every=args.measure_every,
               state_mode=args.state_mode, cluster=args.cluster, chain_set=args.chain_set)
    if args.layout == sgmc.SG_LAYOUT_MSC64:
        opt["rng_group"] = 64
    with sgmc.Ensemble(args.L, args.h, T, args.dist, args.samples, 7, J=J, spins=s0,
                       stream=stream, **opt) as ens:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for c in range(args.chunks):
            if c == args.chunks - 1:
                ev[0].record(stream)
            ens.sweep(args.sweeps)
        ev[1].record(stream)
        ens.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        att = ens.info().attempts_per_sweep * args.sweeps
        print(json.dumps({"L": args.L, "dist": args.dist, "samples": args.samples,
                          "nt": args.nt, "sweeps": args.sweeps, "n_therm": args.n_therm,
                          "exchange_every": args.exchange_every,
                          "threads": ens.info().threads_per_block,
                          "chain_set": ens.info().chain_set, "state_mode": args.state_mode,
                          "ms": ms,
                          "attempts_per_ns": att / (ms * 1e6)}))


if __name__ == "__main__":
    main()
