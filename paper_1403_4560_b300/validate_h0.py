"""Zero-field check of the whole engine: Binder ratio, xi_L / L and R12 crossings.

The paper benchmarks its code at h = 0 (results section), where the 3D +-J
Edwards-Anderson model has a spin-glass transition near T_c ~ 1.10 (the value
it cites). At h = 0 the curves g(T) and xi_L(T)/L of different L cross close
to T_c, and the paper finds that R12 crosses there as well (results
section, zero-field runs). This script runs +-J ensembles at h = 0 for several L with the
multispin-coded path (parallel tempering, thermalise for the first half of
the sweeps, measure in the second), computes g, xi_L/L and R12 with jackknife
errors through the library's estimators, and reports where the curves of
successive L cross.

  python -m paper_1403_4560_b300.validate_h0 [--Ls 4 6 8 10] [--samples 256]
      [--sweeps 16384] [--nt 16] [--tmin 0.8] [--tmax 1.6] [--json out.json]
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


def crossing(T, a, b):
    """Temperatures where the piecewise-linear curves a(T) and b(T) cross."""
    d = np.asarray(a) - np.asarray(b)
    out = []
    for k in range(len(T) - 1):
        if np.isfinite(d[k]) and np.isfinite(d[k + 1]) and d[k] * d[k + 1] < 0:
            out.append(float(T[k] + (T[k + 1] - T[k]) * d[k] / (d[k] - d[k + 1])))
    return out


def fmt(xs):
    return "[" + ", ".join(f"{x:.4f}" for x in xs) + "]"


def crossing_errors(T, accs, La, Lb, key, x0, blocks=32):
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
            o = sgmc.observables_from_acc(acc[keep], L)
            curves.append(o["xi"] / L if key == "xi_over_L" else o[key])
        cs = crossing(T, curves[0], curves[1])
        if not cs:
            return float("nan")
        ests.append(min(cs, key=lambda c: abs(c - x0)))
    ests = np.asarray(ests)
    n = len(ests)
    return float(np.sqrt((n - 1) / n * np.sum((ests - ests.mean()) ** 2)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--Ls", type=int, nargs="+", default=[4, 6, 8, 10])
    ap.add_argument("--samples", type=int, default=256)
    ap.add_argument("--sweeps", type=int, default=16384)
    ap.add_argument("--nt", type=int, default=16)
    ap.add_argument("--tmin", type=float, default=0.8)
    ap.add_argument("--tmax", type=float, default=1.6)
    ap.add_argument("--seed", type=int, default=2014)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()

    from paper_1403_4560_b300 import inputs, sgmc

    T = inputs.geometric_ladder(args.tmin, args.tmax, args.nt)
    res = {}
    accs = {}
    for L in args.Ls:
        t0 = time.time()
        with sgmc.Ensemble(L, 0.0, T, "pmj", args.samples, args.seed + L,
                           layout=sgmc.SG_LAYOUT_MSC64, n_therm=args.sweeps // 2) as e:
            e.sweep(args.sweeps)
            e.synchronize()
            r = e.results()
            accs[L] = e.accumulators()
        res[L] = {"g": r["g"].tolist(), "g_err": r["g_err"].tolist(),
                  "xi_over_L": (r["xi"] / L).tolist(), "xi_over_L_err": (r["xi_err"] / L).tolist(),
                  "R12": r["r12"].tolist(), "R12_err": r["r12_err"].tolist(),
                  "seconds": time.time() - t0}
        print(f"L={L}: {time.time() - t0:.1f} s", flush=True)
    print(f"{'T':>7s} " + " ".join(f"{'g L=' + str(L):>14s}" for L in args.Ls) + "   " +
          " ".join(f"{'xi/L L=' + str(L):>14s}" for L in args.Ls) + "   " +
          " ".join(f"{'R12 L=' + str(L):>14s}" for L in args.Ls))
    for k, t in enumerate(T):
        gs = " ".join(f"{res[L]['g'][k]:7.4f}({res[L]['g_err'][k]:.4f})" for L in args.Ls)
        xs = " ".join(f"{res[L]['xi_over_L'][k]:7.4f}({res[L]['xi_over_L_err'][k]:.4f})"
                      for L in args.Ls)
        rs = " ".join(f"{res[L]['R12'][k]:7.4f}({res[L]['R12_err'][k]:.4f})" for L in args.Ls)
        print(f"{t:7.4f} {gs}   {xs}   {rs}")
    cross = {}
    for a, b in zip(args.Ls, args.Ls[1:]):
        cross[f"{a}-{b}"] = {"g": crossing(T, res[a]["g"], res[b]["g"]),
                             "xi_over_L": crossing(T, res[a]["xi_over_L"], res[b]["xi_over_L"]),
                             "R12": crossing(T, res[a]["R12"], res[b]["R12"])}
        c = cross[f"{a}-{b}"]
        for key, lib_key in (("g", "g"), ("xi_over_L", "xi_over_L"), ("R12", "r12")):
            c[key + "_err"] = [crossing_errors(T, accs, a, b, lib_key, x0) for x0 in c[key]]
        print(f"crossings L={a},{b}: g at {fmt(c['g'])} +- {fmt(c['g_err'])}, "
              f"xi/L at {fmt(c['xi_over_L'])} +- {fmt(c['xi_over_L_err'])}, "
              f"R12 at {fmt(c['R12'])} +- {fmt(c['R12_err'])}")
    out = {"T": T.tolist(), "results": res, "crossings": cross,
           "config": vars(args)}
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
