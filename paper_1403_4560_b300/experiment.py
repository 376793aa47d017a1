"""Finite-size runs of the paper's observables, with the equilibration test.

For each lattice size L this runs one ensemble of disorder samples (the
multispin-coded layout for +-J couplings when the sample count allows it),
with the accumulators split into logarithmic sweep bins, and reports:
  * g, xi_L / L and R12 per temperature of the last bin (the second half of
    the run, the paper's thermalise-then-measure split, Table I caption),
    with jackknife errors, and where the curves of successive L cross, with a
    block-jackknife error of each crossing;
  * the logarithmic-binning test (caption of the paper's R12-against-sweeps
    figure): the observables of the last bins must agree within errors;
  * the overlap distribution P(q) at the lowest temperature (conclusion).

Presets:
  h0     +-J at h = 0, T 0.8..1.6: the curves of g and xi_L / L cross near the
         zero-field transition T_c ~ 1.10 the paper quotes (results section),
         the benchmark the paper itself ran;
  paper  the paper's field runs at reduced sample count: +-J, h = 0.1,
         L = 6, 8, 10, 56 temperatures geometric in beta from 0.1 to 1.8
         (Table I).

  python -m paper_1403_4560_b300.experiment --preset h0 [--Ls ...] [--samples S]
      [--log2-sweeps K] [--json out.json]
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

PRESETS = {
    "h0": dict(h=0.0, Ls=[4, 6, 8, 10, 12], T=("T", 0.8, 1.6), nt=16, samples=4096,
               log2_sweeps=16),
    "paper": dict(h=0.1, Ls=[6, 8, 10], T=("beta", 0.1, 1.8), nt=56, samples=8192,
                  log2_sweeps=18),
}
KEYS = (("g", "g"), ("xi_over_L", "xi"), ("R12", "r12"))


def crossing(T, a, b):
    """Temperatures where the piecewise-linear curves a(T) and b(T) cross."""
    d = np.asarray(a) - np.asarray(b)
    out = []
    for k in range(len(T) - 1):
        if np.isfinite(d[k]) and np.isfinite(d[k + 1]) and d[k] * d[k + 1] < 0:
            out.append(float(T[k] + (T[k + 1] - T[k]) * d[k] / (d[k] - d[k + 1])))
    return out


def _curve(o, key, L):
    return o["xi"] / L if key == "xi" else o[key]


def crossing_error(T, accs, La, Lb, key, x0, blocks=32):
    """Block-jackknife error of the crossing nearest x0 of observable `key`
    between sizes La and Lb: delete one of `blocks` blocks of samples, redo
    the estimators and the crossing, and take the jackknife spread."""
    from paper_1403_4560_b300 import sgmc
    ests = []
    for b in range(blocks):
        curves = []
        for L in (La, Lb):
            acc = accs[L]
            S = acc.shape[0]
            keep = np.ones(S, bool)
            keep[b * S // blocks:(b + 1) * S // blocks] = False
            curves.append(_curve(sgmc.observables_from_acc(acc[keep], L), key, L))
        cs = crossing(T, curves[0], curves[1])
        if not cs:
            return float("nan")
        ests.append(min(cs, key=lambda c: abs(c - x0)))
    ests = np.asarray(ests)
    n = len(ests)
    return float(np.sqrt((n - 1) / n * np.sum((ests - ests.mean()) ** 2)))


def log_binning_test(per_bin, L, last=3, keys=("g", "xi", "r12", "e")):
    """Largest deviation, in combined standard errors, between the last bin
    and each of the `last - 1` bins before it, per observable (over all
    temperatures). Bins share samples, so adding their errors in quadrature
    overstates the error of the difference: a small number here is a
    necessary, not a sufficient, sign of equilibrium."""
    B = len(per_bin)
    out = {}
    for key in keys:
        ref = _curve(per_bin[B - 1], key, L)
        rerr = _curve({key: per_bin[B - 1][key + "_err"]}, key, L)
        worst = 0.0
        for b in range(max(0, B - last), B - 1):
            x = _curve(per_bin[b], key, L)
            xe = _curve({key: per_bin[b][key + "_err"]}, key, L)
            with np.errstate(invalid="ignore", divide="ignore"):
                z = np.abs(x - ref) / np.sqrt(xe ** 2 + rerr ** 2)
            z = z[np.isfinite(z)]
            if z.size:
                worst = max(worst, float(z.max()))
        out[key] = worst
    return out


def temperatures(spec, nt):
    from paper_1403_4560_b300 import inputs
    kind, a, b = spec
    if kind == "T":
        return inputs.geometric_ladder(a, b, nt)
    # geometric in beta from beta_min = a to beta_max = b, as ascending T
    beta = a * (b / a) ** (np.arange(nt) / (nt - 1))
    return np.ascontiguousarray((1.0 / beta)[::-1])


def run(Ls, h, T, samples, log2_sweeps, seed=2014, dist="pmj"):
    from paper_1403_4560_b300 import sgmc
    res, accs = {}, {}
    for L in Ls:
        t0 = time.time()
        msc = dist == "pmj" and samples % 64 == 0 and L <= 16
        opt = dict(log_bins=log2_sweeps, pq_hist=1, n_therm=0)
        if msc:
            opt["layout"] = sgmc.SG_LAYOUT_MSC64
        with sgmc.Ensemble(L, h, T, dist, samples, seed + L, **opt) as e:
            e.sweep(2 ** log2_sweeps)
            e.synchronize()
            acc = e.accumulators()
            hist = e.histogram()
        # the library's estimators on each bin's slice (one device copy in all)
        per_bin = [sgmc.observables_from_acc(np.ascontiguousarray(acc[:, :, b]), L)
                   for b in range(log2_sweeps)]
        accs[L] = np.ascontiguousarray(acc[:, :, -1])
        r = per_bin[-1]
        N = L ** 3
        res[L] = {
            "g": r["g"].tolist(), "g_err": r["g_err"].tolist(),
            "xi_over_L": (r["xi"] / L).tolist(), "xi_over_L_err": (r["xi_err"] / L).tolist(),
            "R12": r["r12"].tolist(), "R12_err": r["r12_err"].tolist(),
            "chi0": r["chi0"].tolist(), "e": r["e"].tolist(),
            "log_binning_z": log_binning_test(per_bin, L),
            "bins_R12_lowest_T": [float(pb["r12"][0]) for pb in per_bin],
            "pq_lowest_T": {"q": ((2 * np.arange(N + 1) - N) / N).tolist(),
                            "p": (hist[0, -1] / max(hist[0, -1].sum(), 1)).tolist()},
            "layout": "msc64" if msc else "int8",
            "seconds": time.time() - t0,
        }
        print(f"L={L}: {res[L]['seconds']:.1f} s, log-binning z (last 3 bins): "
              + ", ".join(f"{k} {v:.2f}" for k, v in res[L]["log_binning_z"].items()), flush=True)
    cross = {}
    for a, b in zip(Ls, Ls[1:]):
        c = {}
        for name, key in KEYS:
            xs = crossing(T, res[a][name], res[b][name])
            c[name] = xs
            c[name + "_err"] = [crossing_error(T, accs, a, b, key, x0) for x0 in xs]
        cross[f"{a}-{b}"] = c
    return res, cross


def fmt(xs):
    return "[" + ", ".join(f"{x:.4f}" for x in xs) + "]"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", choices=sorted(PRESETS), default="h0")
    ap.add_argument("--Ls", type=int, nargs="+")
    ap.add_argument("--samples", type=int)
    ap.add_argument("--log2-sweeps", type=int)
    ap.add_argument("--h", type=float)
    ap.add_argument("--seed", type=int, default=2014)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    cfg = dict(PRESETS[args.preset])
    for k in ("Ls", "samples", "log2_sweeps", "h"):
        if getattr(args, k) is not None:
            cfg[k] = getattr(args, k)
    T = temperatures(cfg["T"], cfg["nt"])
    res, cross = run(cfg["Ls"], cfg["h"], T, cfg["samples"], cfg["log2_sweeps"], args.seed)
    Ls = cfg["Ls"]
    head = f"{'T':>7s} " + "   ".join(
        " ".join(f"{name + ' L=' + str(L):>16s}" for L in Ls) for name, _ in KEYS)
    print(head)
    for k, t in enumerate(T):
        cols = []
        for name, _ in KEYS:
            cols.append(" ".join(f"{res[L][name][k]:8.4f}({res[L][name + '_err'][k]:.4f})"
                                 for L in Ls))
        print(f"{t:7.4f} " + "   ".join(cols))
    for pair, c in cross.items():
        print(f"crossings L={pair}: " + ", ".join(
            f"{name} at {fmt(c[name])} +- {fmt(c[name + '_err'])}" for name, _ in KEYS))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"preset": args.preset, "config": {**cfg, "T": T.tolist()},
                       "results": res, "crossings": cross}, fh, indent=1)


if __name__ == "__main__":
    main()
