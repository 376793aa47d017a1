#!/usr/bin/env python3
"""Throughput benchmark of the EA spin-glass Monte Carlo engine on B300.

Workload: Gaussian couplings, L = 8 and L = 12, h in {0.1, 0.2, 0.3}, 512
disorder samples per (L, h), 2 replicas x 24 temperatures geometric in
0.5-1.6, replica exchange and overlap measurement after every sweep. All six
ensembles run batched (one CUDA graph launch per step, one persistent fused
kernel per ensemble on parallel graph branches). A step is SWEEPS_PER_STEP
sweeps of every chain of every sample, exchange and measurement included.

Metric: spin-flip attempts per ns (one attempt = one Metropolis proposal on
one site of one chain). Printed as one JSON line by rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain sequential restatement of the
method) on the host cores for the same metric, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/ns on 1 B300, batched vs plain, oracle-matched; p50/p99 lat"
UNIT = "spin-flip attempts/ns"
LS = (8, 12)
HS = (0.1, 0.2, 0.3)
N_SAMPLES = 512
N_T = 24
T_MIN, T_MAX = 0.5, 1.6
SWEEPS_PER_STEP = 256
B_ALG_CONST = 2.0     # int8 spin read + write per attempt, bytes
B_ALG_COUPLING = 12.0  # three FP32 bonds per site, shared by the 2*N_T chains
WORKLOAD = ("gaussian EA 3D, L=8 and 12 x h=0.1,0.2,0.3, 512 samples each, "
            "2 replicas x 24 T geometric 0.5-1.6, exchange+measure every sweep")
# DRAM bytes (read + write) of one launch of the dominant kernel in this
# workload (L = 12, 512 samples, 256 sweeps), from the one-pass ncu capture
# summarised under profiles/. Must be reset to
# None whenever the kernel changes, until it is captured again.
TRAFFIC_BYTES_PER_LAUNCH = 65.9e6
# Thread instructions per attempt of the same kernel in the same launch shape
# (ncu smsp__thread_inst_executed.sum over the launch's attempts, captured on
# the bench's own 512-sample, 256-sweep segmented launch;
# its ncu summary is kept under profiles/). Reset to None whenever
# the kernel changes, until it is captured again.
INSTR_PER_ATTEMPT = 66.7
# SM issue peak: 148 SMs x 4 schedulers x 1 warp instruction per cycle x 32
# threads x 2.032 GHz (maximum SM clock), in thread instructions per second.
ISSUE_PEAK = 148 * 4 * 32 * 2.032e9


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sweeps-per-step", type=int, default=SWEEPS_PER_STEP)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads (uneven batch, MSC, serving)")
    return ap.parse_args()


def attempts_per_sweep() -> int:
    return sum(L ** 3 * 2 * N_T * N_SAMPLES for L in LS for _ in HS)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, f in enumerate(flags)
                          if f.lower() == "active"})
        loaded = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def make_ensembles(sgmc, inputs, rank, stream, **opt):
    """One ensemble per (L, h). Rank r holds the global samples
    [r * N_SAMPLES, (r + 1) * N_SAMPLES) of each: couplings and initial spins
    are drawn on the device keyed by the global sample index (sample_base),
    so N ranks run one N-times-larger ensemble split by samples. The host
    copy of the initial spins feeds the end-to-end uploads."""
    T = inputs.geometric_ladder(T_MIN, T_MAX, N_T)
    ens, host = [], []
    for li, L in enumerate(LS):
        for hi, h in enumerate(HS):
            seed = 10 * li + hi + 1
            e = sgmc.Ensemble(L, h, T, "gauss", N_SAMPLES, seed, stream=stream, n_therm=0,
                              sample_base=rank * N_SAMPLES, **opt)
            ens.append(e)
            host.append(e.spins())
    return ens, host


def cpu_baseline(budget_s: float):
    """The oracle, as it stands, on a bounded sample of the workload: L = 12,
    Gaussian, h = 0.2, 2 x 24 temperatures, one sample per host core."""
    from oracle import oracle as orc
    from paper_1403_4560_b300 import inputs

    cores = os.cpu_count() or 1
    L = 12
    T = inputs.geometric_ladder(T_MIN, T_MAX, N_T)
    J, s0 = inputs.make_instance("gauss", L, cores, N_T, seed=99)
    st = orc.State(L, T, 0.2, True, seed=99, J=J, spins=s0, n_therm=0)
    st.run(1, threads=cores)  # warm-up (library load, thread start)
    # two-point calibration: each call pays a fixed start-up (worker threads),
    # so the per-sweep cost is the difference of two call lengths
    t0 = time.perf_counter()
    st.run(4, threads=cores)
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    st.run(20, threads=cores)
    tb = time.perf_counter() - t0
    per_sweep = max((tb - ta) / 16, 1e-4)
    n = max(1, min(20000, int(budget_s / per_sweep)))
    t0 = time.perf_counter()
    st.run(n, threads=cores)  # the timed sample: one call
    dt = time.perf_counter() - t0
    att = L ** 3 * 2 * N_T * cores * n
    # one core: one sample in the calling thread, a quarter of the budget
    one = orc.State(L, T, 0.2, True, seed=99, J=J[:1], spins=s0[:1], n_therm=0)
    one.run(1)  # warm-up
    t0 = time.perf_counter()
    one.run(4)
    per1 = max((time.perf_counter() - t0) / 4, 1e-4)
    n1 = max(1, min(20000, int(0.25 * budget_s / per1)))
    t0 = time.perf_counter()
    one.run(n1)
    dt1 = time.perf_counter() - t0
    v1 = L ** 3 * 2 * N_T * n1 / (dt1 * 1e9)
    return {"value": att / (dt * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": v1,
            "sample": f"L=12 gaussian, 2x24 T, h=0.2, {cores} samples x {n} sweeps "
                      f"(exchange+measure every sweep) in one call, {dt:.1f} s; 1 core: "
                      f"1 sample x {n1} sweeps, {dt1:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_seconds)
    steps = []
    from oracle import oracle as orc
    from paper_1403_4560_b300 import inputs
    cores = cb["cores"]
    T = inputs.geometric_ladder(T_MIN, T_MAX, N_T)
    J, s0 = inputs.make_instance("gauss", 12, cores, N_T, seed=5)
    st = orc.State(12, T, 0.2, True, seed=5, J=J, spins=s0, n_therm=0)
    per_step = 16  # sweeps per step: one call, so thread start-up is amortised
    for _ in range(args.warmup):
        st.run(per_step, threads=cores)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st.run(per_step, threads=cores)
        steps.append(time.perf_counter() - t0)
    att = 12 ** 3 * 2 * N_T * cores * per_step
    value = att * len(steps) / (sum(steps) * 1e9)
    cb["value"] = value
    cb["sample"] = (f"each step: {per_step} sweeps of {cores} L=12 gaussian samples, 2x24 T, "
                    f"exchange+measure, on {cores} host cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(steps) / len(steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "CPU oracle (plain sequential C)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


CFG4 = [(6, 2048), (8, 1024), (10, 1024), (12, 512), (16, 256)]


def extra_uneven_batch(sgmc, inputs, stream, torch):
    """Uneven-L Gaussian ensemble (L = 6..16 with 2048..256 samples, h = 0.2,
    2 x 20 T in 0.5-1.5): autotuned, batched through one CUDA graph per step,
    against plain per-sweep launches of the ensembles one after another."""
    T = inputs.geometric_ladder(0.5, 1.5, 20)
    insts = [inputs.make_instance("gauss", L, S, 20, seed=40 + L) for L, S in CFG4]
    att_sweep = sum(L ** 3 * 40 * S for L, S in CFG4)
    ens = [sgmc.Ensemble(L, 0.2, T, "gauss", S, 40 + L, J=J, spins=s0, stream=stream, n_therm=0)
           for (L, S), (J, s0) in zip(CFG4, insts)]
    tune = {f"L{e.L}": e.autotune(trial_sweeps=16)["threads_per_block"] for e in ens}
    # sweeps per exchange: the most frequent exchange within 3 % of the fastest
    sched = {f"L{e.L}": e.autotune_schedule([1, 2, 4], trial_sweeps=8,
                                            tolerance=0.03)["exchange_every"] for e in ens}
    n = 64
    sgmc.sweep_batch(ens, n, use_graph=True)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(2):
        sgmc.sweep_batch(ens, n, use_graph=True)
    ev[1].record(stream)
    torch.cuda.synchronize()
    batched = att_sweep * 2 * n / (ev[0].elapsed_time(ev[1]) * 1e6)
    for e in ens:
        e.close()
    pens = [sgmc.Ensemble(L, 0.2, T, "gauss", S, 40 + L, J=J, spins=s0, stream=stream,
                          n_therm=0, sweeps_per_launch=1, exchange_every=sched[f"L{L}"])
            for (L, S), (J, s0) in zip(CFG4, insts)]
    for e in pens:
        e.sweep(1)
    torch.cuda.synchronize()
    npl = 16
    ev[0].record(stream)
    for e in pens:
        e.sweep(npl)
    ev[1].record(stream)
    torch.cuda.synchronize()
    plain = att_sweep * npl / (ev[0].elapsed_time(ev[1]) * 1e6)
    for e in pens:
        e.close()
    return {"batched": batched, "plain": plain, "unit": UNIT, "tuned_threads": tune,
            "tuned_exchange_every": sched,
            "workload": "gaussian, L=6,8,10,12,16 x 2048,1024,1024,512,256 samples, h=0.2, "
                        "2x20 T 0.5-1.5, measure every sweep, exchange every "
                        "tuned_exchange_every sweeps (both arms)"}


def extra_msc(sgmc, stream, torch, L=16, S=4096, T=None, h=0.1):
    """+-J multispin-coded path, by default L = 16, 4096 samples (64 words),
    h = 0.1, 2 x 32 T in 0.4-1.5; one launch per sweep (graph-captured batch)."""
    from paper_1403_4560_b300 import inputs
    T = inputs.geometric_ladder(0.4, 1.5, 32) if T is None else T
    out = {}
    for name, n_therm in (("measuring", 0), ("thermalising", 10 ** 9)):
        with sgmc.Ensemble(L, h, T, "pmj", S, 5, stream=stream, n_therm=n_therm,
                           layout=sgmc.SG_LAYOUT_MSC64) as e:
            sgmc.sweep_batch([e], 4, use_graph=True)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(4):
                sgmc.sweep_batch([e], 4, use_graph=True)
            ev[1].record(stream)
            torch.cuda.synchronize()
            out[name] = e.info().attempts_per_sweep * 16 / (ev[0].elapsed_time(ev[1]) * 1e6)
    out["unit"] = UNIT
    return out


def extra_int8(sgmc, stream, torch, L, S, T, h, dist="gauss", sweeps=32, **opt):
    """The fused int8 path on one ensemble (measurement every sweep), timed
    over `sweeps` sweeps after a warm-up launch."""
    with sgmc.Ensemble(L, h, T, dist, S, 7, stream=stream, n_therm=0, **opt) as e:
        e.sweep(4)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        e.sweep(sweeps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        info = e.info()
        return {"value": info.attempts_per_sweep * sweeps / (ev[0].elapsed_time(ev[1]) * 1e6),
                "unit": UNIT, "threads": info.threads_per_block, "grid": info.grid,
                "workload": f"{dist}, L={L}, {S} samples, 2x{len(T)} T, h={h}"}


def extra_cluster(sgmc, stream, torch, sweeps=16):
    """Large lattices with fewer samples than SMs (64 samples, Gaussian, 2 x
    16 temperatures geometric 0.5-1.6, h = 0.2, measuring every sweep): each
    sample swept by a thread-block cluster (library choice) against one CTA
    per sample."""
    from paper_1403_4560_b300 import inputs
    T = inputs.geometric_ladder(0.5, 1.6, 16)
    out = {"unit": UNIT}
    for L in (24, 32):
        row = {}
        for name, cl in (("cluster", 0), ("k2", 2), ("k4", 4), ("one_cta_per_sample", 1)):
            with sgmc.Ensemble(L, 0.2, T, "gauss", 64, 11, stream=stream, n_therm=0,
                               cluster=cl) as e:
                e.sweep(2)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(stream)
                e.sweep(sweeps)
                ev[1].record(stream)
                torch.cuda.synchronize()
                row[name] = e.info().attempts_per_sweep * sweeps / (ev[0].elapsed_time(ev[1]) * 1e6)
                if cl == 0:
                    row["ctas_per_sample"] = e.info().cluster
        out[f"L{L}_64_samples"] = row
    return out


def extra_serving(stream, n_req=24, rate=50.0, sweeps=256):
    """A finite Poisson stream (mean 50 requests/s, seed 1) of requests drawn
    uniformly from L in {8,12,16,20,24}, h in {0.05,...,0.40}, 16-32
    temperatures geometric in 0.5-1.6, 64-1024 samples (multiples of 64),
    +-J or Gaussian couplings; each request runs `sweeps` sweeps (the full
    2^14-sweep stream takes minutes: python -m
    paper_1403_4560_b300.serving_run, results committed separately)."""
    from paper_1403_4560_b300 import serving_run
    return serving_run.run_stream(serving_run.draw_requests(n_req, rate, seed=1), sweeps,
                                  chunk_sweeps=64, stream=stream)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_1403_4560_b300 import build as sgbuild
    from paper_1403_4560_b300 import inputs, sgmc

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        sgbuild.build()
    if dist is not None:
        dist.barrier()
    sgmc.lib()
    stream = torch.cuda.current_stream()
    K, W, nsw = args.steps, args.warmup, args.sweeps_per_step
    ens, host_spins = make_ensembles(sgmc, inputs, rank, stream)
    n_launch_per_step = 2 * len(ens)  # fused kernel + sweep-counter update per ensemble

    def step():
        sgmc.sweep_batch(ens, nsw, use_graph=True)

    for _ in range(W):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(K):
            step()
        stop.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = start.elapsed_time(stop)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    for e in ens:
        e.synchronize()
    att_total = attempts_per_sweep() * nsw * K * world
    value = att_total / (ms * 1e6)

    # dominant kernel alone: L = 12 fused kernel, timed on its launch stream
    dom = ens[len(HS)]
    dom_att = dom.info().attempts_per_sweep * nsw
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    reps = 3
    dom.sweep(nsw)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        dom.sweep(nsw)
    ev[1].record(stream)
    torch.cuda.synchronize()
    dom_ms = ev[0].elapsed_time(ev[1]) / reps
    b_alg = B_ALG_CONST + B_ALG_COUPLING / (2 * N_T)
    achieved = b_alg * dom_att / (dom_ms * 1e6)  # GB/s
    peak, peak_kind = peaks()
    # HBM-equivalent roofline: the bytes a sweep would move if the state were
    # streamed through HBM every sweep (B_alg per attempt), against the
    # measured copy bandwidth
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_LAUNCH,
           "algorithmic_bytes_per_launch": b_alg * dom_att,
           "kernel": "int8_run_kernel<L=12, gauss>",
           "b_alg_bytes_per_attempt": b_alg, "peak_kind": peak_kind,
           "attempts_per_ns": dom_att / (dom_ms * 1e6)}
    # The roofline is the HBM-equivalent one above (B_alg x attempts / time
    # against the measured copy bandwidth). What binds is instruction issue:
    # the state stays on chip, so at I thread instructions per attempt the
    # kernel cannot pass ISSUE_PEAK / I attempts/s. That ceiling, and the
    # share of it reached, are reported beside the roofline.
    roofline = hbm
    issue = None
    if INSTR_PER_ATTEMPT:
        inst = INSTR_PER_ATTEMPT * dom_att / (dom_ms * 1e-3) / 1e12
        ceiling = ISSUE_PEAK / INSTR_PER_ATTEMPT / 1e9  # attempts/ns at 100 % issue
        issue = {"bound": "alu", "achieved": inst, "peak": ISSUE_PEAK / 1e12,
                 "unit": "T thread-instructions/s", "frac": inst / (ISSUE_PEAK / 1e12),
                 "instructions_per_attempt": INSTR_PER_ATTEMPT,
                 "issue_ceiling_attempts_per_ns": ceiling,
                 "issue_ceiling_hbm_frac": ceiling * b_alg / peak,
                 "peak_kind": "derived: 148 SMs x 4 schedulers x 32 lanes x 2.032 GHz",
                 "kernel": "int8_run_kernel<L=12, gauss>"}

    plain = None
    if not args.no_plain and rank == 0:
        pens, _ = make_ensembles(sgmc, inputs, rank, stream, sweeps_per_launch=1)
        for e in pens:
            e.sweep(1)
        torch.cuda.synchronize()
        nplain = 16
        ev[0].record(stream)
        for e in pens:
            e.sweep(nplain)
        ev[1].record(stream)
        torch.cuda.synchronize()
        pms = ev[0].elapsed_time(ev[1])
        plain = {"value": attempts_per_sweep() * nplain / (pms * 1e6), "unit": UNIT,
                 "how": "one launch per sweep per ensemble, ensembles one after another"}
        for e in pens:
            e.close()

    e2e = None
    if not args.no_e2e:
        # per step: upload that step's initial spins from page-locked host
        # memory (the copies overlap the previous step's sweeps), the batched
        # sweeps, and the download of every ensemble's accumulators
        pinned = [torch.from_numpy(s).pin_memory().numpy() for s in host_spins]
        acc_out = [torch.zeros(e.accumulators().shape, dtype=torch.float64).pin_memory().numpy()
                   for e in ens]
        n_e2e = max(2, min(K, 6))

        def e2e_step():
            for e, s in zip(ens, pinned):
                e.set_spins_async(s)
            step()
            for e, o in zip(ens, acc_out):
                e.accumulators_async(o)

        e2e_step()  # first call allocates the upload buffers
        for e in ens:
            e.synchronize()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        for e in ens:
            e.synchronize()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": attempts_per_sweep() * nsw * n_e2e * world / (dt * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(s.nbytes for s in pinned)),
               "d2h_bytes_per_step": int(sum(o.nbytes for o in acc_out)), "steps": n_e2e,
               "how": "per step: sg_set_spins_async from page-locked host spins for all 6 "
                      "ensembles (copies overlap the previous step's sweeps), batched sweeps, "
                      "sg_get_accumulators_async to page-locked host memory; one "
                      "synchronisation after the last step"}

    extras = None
    if rank == 0 and not args.no_extras:
        # the paper's own geometry (Table I): L = 10, 56 temperatures
        # geometric in beta 0.1-1.8, h = 0.1
        t_paper = np.ascontiguousarray((1.0 / (0.1 * 18.0 ** (np.arange(56) / 55.0)))[::-1])
        extras = {"uneven_batch": extra_uneven_batch(sgmc, inputs, stream, torch),
                  "msc_L16": extra_msc(sgmc, stream, torch),
                  "msc_paper_L10_56T": extra_msc(sgmc, stream, torch, L=10, S=8192, h=0.1,
                                                 T=t_paper),
                  # the same geometry with Gaussian couplings on the int8 path
                  "int8_paper_L10_56T_gauss": extra_int8(sgmc, stream, torch, L=10, S=1184,
                                                         T=t_paper, h=0.1),
                  # +-J at the same geometry: a byte per chain, and one bit per
                  # chain swept bit-parallel (each chain its own random words)
                  "int8_paper_L10_56T_pmj": extra_int8(sgmc, stream, torch, L=10, S=1184,
                                                       T=t_paper, h=0.1, dist="pmj",
                                                       state_mode=1),
                  "bits_paper_L10_56T_pmj": extra_int8(sgmc, stream, torch, L=10, S=1184,
                                                       T=t_paper, h=0.1, dist="pmj",
                                                       state_mode=3),
                  "cluster": extra_cluster(sgmc, stream, torch),
                  "serving": extra_serving(stream)}

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "sweeps_per_step": nsw,
                           "parallelism": f"sample shards (sample_base), {world} GPU(s), no collective in the timed region",
                           "l2": "state+couplings 206 MB per GPU, larger than L2",
                           "batched": "one CUDA graph per step, 6 parallel branches"},
                "gpu_launches": n_launch_per_step * K,
                "roofline": roofline, "issue": issue, "plain": plain, "e2e": e2e,
                "cpu_baseline": cb,
                "clocks": clk.summary(), "extras": extras}
        print(json.dumps(line), flush=True)
    for e in ens:
        e.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
