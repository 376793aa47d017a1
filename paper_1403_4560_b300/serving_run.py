"""Finite Poisson request streams through the serving loop (sg_server_*).

Each request is one full run of the method (paper: methods section; first
half of the sweeps thermalising, Table I caption) drawn uniformly from
L in {8, 12, 16, 20, 24}, h in {0.05, 0.10, ..., 0.40}, 16-32 temperatures
geometric in 0.5-1.6, 64-1024 samples (multiples of 64) and +-J or Gaussian
couplings. Requests are submitted at their Poisson arrival times; the server
admits them by device memory, keeps their state resident and runs the
resident requests' chunks concurrently. Reported: submit-to-result latency
(queueing included) p50 / p99 / max, and the aggregate spin-flip attempts per
ns over the stream's wall time and over the server's busy time.

  python -m paper_1403_4560_b300.serving_run --requests 24 --rate 50 \
      --sweeps 16384 [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

UNIT = "spin-flip attempts/ns"


def draw_requests(n_req: int, rate: float, seed: int = 1) -> list[dict]:
    """n_req requests with exponential inter-arrival times of mean 1/rate."""
    rng = np.random.default_rng(seed)
    reqs, t = [], 0.0
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate)
        reqs.append(dict(at=t, L=int(rng.choice([8, 12, 16, 20, 24])),
                         h=float(rng.choice(np.arange(1, 9) * 0.05)),
                         nt=int(rng.integers(16, 33)), S=int(64 * rng.integers(1, 17)),
                         dist=str(rng.choice(["pmj", "gauss"]))))
    return reqs


def run_stream(reqs: list[dict], sweeps: int, chunk_sweeps: int = 256, use_graph: bool = False,
               stream=None) -> dict:
    """Submit `reqs` at their arrival times, wait for all, summarise."""
    from paper_1403_4560_b300 import inputs, sgmc

    att = [r["L"] ** 3 * 2 * r["nt"] * r["S"] * sweeps for r in reqs]
    with sgmc.Server(chunk_sweeps=chunk_sweeps, use_graph=use_graph, stream=stream) as sv:
        t0 = time.perf_counter()
        ids = []
        for k, r in enumerate(reqs):
            delay = r["at"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(sv.submit(r["L"], r["h"], inputs.geometric_ladder(0.5, 1.6, r["nt"]),
                                 r["dist"], r["S"], seed=1000 + k, n_sweeps=sweeps))
        states = [sv.wait(rid) for rid in ids]
        wall = time.perf_counter() - t0
        lat = np.array([sv.result(rid)[1] for rid in ids])
        st = sv.stats()
    span = reqs[-1]["at"] - reqs[0]["at"]
    return {"requests": len(reqs), "rate_per_s": (len(reqs) - 1) / span if span > 0 else None,
            "sweeps_per_request": sweeps, "completed": int(sum(s == 2 for s in states)),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "mean_s": float(lat.mean()),
            "attempts_total": float(sum(att)),
            "attempts_per_ns_wall": sum(att) / (wall * 1e9),
            "attempts_per_ns_busy": st["attempts"] / (st["busy_seconds"] * 1e9),
            "wall_s": wall, "unit": UNIT}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--sweeps", type=int, default=16384)
    ap.add_argument("--chunk-sweeps", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    import torch

    from paper_1403_4560_b300 import build as sgbuild
    if not torch.cuda.is_available():
        raise SystemExit("serving_run needs a CUDA GPU")
    sgbuild.build()
    reqs = draw_requests(args.requests, args.rate, args.seed)
    out = run_stream(reqs, args.sweeps, chunk_sweeps=args.chunk_sweeps)
    out["nominal_rate_per_s"] = args.rate
    out["seed"] = args.seed
    out["mix"] = {"pmj": sum(r["dist"] == "pmj" for r in reqs),
                  "gauss": sum(r["dist"] == "gauss" for r in reqs),
                  "mean_attempts_per_request": out["attempts_total"] / len(reqs)}
    print(json.dumps(out), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"config": vars(args), "result": out, "requests": reqs}, fh, indent=1)


if __name__ == "__main__":
    main()
