"""CPU oracle: ctypes front end of sgmc_oracle.c plus the paper's estimators.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the product path never imports it.

The Monte Carlo chain lives in sgmc_oracle.c (plain sequential C). This module
adds the disorder/thermal averages of the paper's methods section in FP64
numpy, written from the definitions:
  Binder ratio g             eq. (binder)
  chi(k)                     eq. (chi)
  correlation length xi_L    eq. (corr)
  R12 = chi(k1)/chi(k2)      eq. (r12)
  point-group averaging over equivalent wave vectors (results section,
  averaging chi over the three axis directions) and jackknife errors over
  disorder samples (methods section).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_PATH = os.path.join(HERE, "sgmc_oracle.c")
# SGMC_ORACLE_LIB names a prebuilt oracle library to load instead (the
# mutation tests point the pins at deliberately broken builds this way)
LIB_OVERRIDE = os.environ.get("SGMC_ORACLE_LIB", "")
LIB_PATH = LIB_OVERRIDE or os.path.join(HERE, "liboracle.so")
NACC = 40

# accumulator indices (frozen layout)
A_N, A_Q1, A_Q2, A_Q3, A_Q4, A_E1, A_E2, A_M1, A_M2 = range(9)


def a_re(v):
    return 9 + 3 * v


def a_im(v):
    return 10 + 3 * v


def a_abs2(v):
    return 11 + 3 * v


KVECS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 0],
                  [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]], dtype=np.int64)


def compile_oracle(src: str, out: str) -> str:
    """gcc the oracle source into a shared library (no FP contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile sgmc_oracle.c into liboracle.so (plain gcc, no FP contraction)."""
    if LIB_OVERRIDE:
        return LIB_PATH
    if force or not os.path.exists(LIB_PATH) or \
            os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC_PATH):
        compile_oracle(SRC_PATH, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u32, u64, f64, f32 = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_float)
        L.orc_philox.argtypes = [P, P, P]
        L.orc_thresholds.argtypes = [f64, P, i32, P]
        L.orc_mc_exp32.argtypes = [f32]
        L.orc_mc_exp32.restype = f32
        L.orc_t32.argtypes = [f32]
        L.orc_t32.restype = u32
        L.orc_init_spins.argtypes = [u64, i64, i64, i32, i32, P]
        L.orc_pmj_couplings.argtypes = [u64, i64, i64, i32, P]
        L.orc_bond_sum.argtypes = [i32, i32, P, P, P, P]
        L.orc_site_threshold.argtypes = [i32, i32, f64, f64, P, P, P, i32]
        L.orc_site_threshold.restype = u32
        L.orc_delta_e.argtypes = [i32, f64, P, P, i32]
        L.orc_delta_e.restype = f64
        L.orc_overlap.argtypes = [i32, P, P, P, P, P]
        L.orc_run.argtypes = [i32, i32, i32, f64, P, u64, i32, i32, i32, i64, i64, i64,
                              i64, i64, i64, P, P, P, P, i32, P, P, i32]
        L.orc_run.restype = i32
        L.orc_exchange.argtypes = [i32, i32, i32, f64, P, u64, i64, i32, i64, i64, i64, P, P,
                                   P, P]
        L.orc_exchange.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------
def philox(key, ctr) -> np.ndarray:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(k), _p(c), _p(out))
    return out


def thresholds(h: float, T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    thr = np.zeros((len(T), 2, 7), dtype=np.uint32)
    lib().orc_thresholds(float(h), _p(T), len(T), _p(thr))
    return thr


def mc_exp32(x: float) -> float:
    return lib().orc_mc_exp32(float(x))


def t32(x: float) -> int:
    return lib().orc_t32(float(x))


def init_spins(seed: int, S: int, n_t: int, L: int, s_base: int = 0) -> np.ndarray:
    """Seed-drawn initial spins of samples s_base .. s_base + S - 1."""
    out = np.zeros((S, 2, n_t, L ** 3), dtype=np.int8)
    lib().orc_init_spins(seed, s_base, S, n_t, L, _p(out))
    return out


def pmj_couplings(seed: int, S: int, L: int, s_base: int = 0) -> np.ndarray:
    """Seed-drawn +-J couplings of samples s_base .. s_base + S - 1."""
    out = np.zeros((S, 3, L ** 3), dtype=np.float32)
    lib().orc_pmj_couplings(seed, s_base, S, L, _p(out))
    return out


def bond_sum(L: int, gauss: bool, J: np.ndarray, s: np.ndarray):
    J = np.ascontiguousarray(J, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    B = np.zeros(1, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    lib().orc_bond_sum(L, int(gauss), _p(J), _p(s), _p(B), _p(M))
    return int(B[0]), int(M[0])


def site_threshold(L, gauss, h, T_t, thr_t, J, s, i) -> int:
    thr_t = np.ascontiguousarray(thr_t, dtype=np.uint32)
    J = np.ascontiguousarray(J, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib().orc_site_threshold(L, int(gauss), float(h), float(T_t), _p(thr_t), _p(J),
                                    _p(s), int(i))


def delta_e(L, h, J, s, i) -> float:
    J = np.ascontiguousarray(J, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return lib().orc_delta_e(L, float(h), _p(J), _p(s), int(i))


def overlap(L, sa, sb):
    sa = np.ascontiguousarray(sa, dtype=np.int8)
    sb = np.ascontiguousarray(sb, dtype=np.int8)
    Q = np.zeros(1, dtype=np.int64)
    re = np.zeros(9, dtype=np.float32)
    im = np.zeros(9, dtype=np.float32)
    lib().orc_overlap(L, _p(sa), _p(sb), _p(Q), _p(re), _p(im))
    return int(Q[0]), re, im


class State:
    """Host-side state of one oracle ensemble (canonical layouts)."""

    def __init__(self, L, T, h, gauss, seed, J, spins, rng_group=1, exchange_every=1,
                 measure_every=1, n_therm=0, s_base=0, log_bins=1, pq_hist=False,
                 slot_shared=False):
        """Local sample k is the global sample s_base + k (its RNG key).

        slot_shared: the temperature slots of a replica share each Metropolis
        random word (the slot field of the counter is 0), as when the N_T
        copies of a sample are packed in the bits of one word (methods
        section, multispin coding).

        log_bins: accumulators per logarithmic sweep bin (acc then has shape
        [S][n_T][log_bins][40]; 1 keeps [S][n_T][40]). pq_hist: also count
        the overlap histogram hist[n_T][log_bins][N+1] (entry k: replicas
        agree on k sites)."""
        self.s_base = int(s_base)
        self.L, self.h, self.gauss, self.seed = L, float(h), bool(gauss), int(seed)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.nt = len(self.T)
        self.J = np.ascontiguousarray(J, dtype=np.float32)
        self.spins = np.array(spins, dtype=np.int8, order="C", copy=True)
        self.S = self.spins.shape[0]
        self.rng_group, self.exchange_every = rng_group, exchange_every
        self.measure_every, self.n_therm = measure_every, n_therm
        self.slot_shared = bool(slot_shared)
        self.B = np.zeros((self.S, 2, self.nt), dtype=np.int64)
        self.M = np.zeros((self.S, 2, self.nt), dtype=np.int64)
        self.log_bins = int(log_bins)
        shape = (self.S, self.nt, NACC) if self.log_bins == 1 else (self.S, self.nt, self.log_bins, NACC)
        self.acc = np.zeros(shape, dtype=np.float64)
        N = L ** 3
        self.hist = (np.zeros((self.nt, self.log_bins, N + 1), dtype=np.uint64) if pq_hist
                     else None)
        self.sweeps_done = 0
        self.exchanges_done = 0

    def run(self, n_sweeps: int, threads: int = 1, s_range=None):
        """Advance samples (all, or s_range) by n_sweeps sweeps."""
        s0, s1 = s_range if s_range is not None else (0, self.S)
        L = lib()

        def work(a, b):
            # each call counts into its own histogram; the parts are summed below
            h = None if self.hist is None else np.zeros_like(self.hist)
            rc = L.orc_run(self.L, self.nt, int(self.gauss), self.h, _p(self.T), self.seed,
                           self.rng_group, self.exchange_every, self.measure_every,
                           self.n_therm, self.sweeps_done, n_sweeps, self.s_base, a, b, _p(self.J),
                           _p(self.spins), _p(self.B), _p(self.M), self.log_bins, _p(self.acc),
                           None if h is None else _p(h), int(self.slot_shared))
            if rc != 0:
                raise ValueError("oracle rejected its arguments")
            return h

        if threads <= 1:
            parts = [work(s0, s1)]
        else:
            cuts = np.linspace(s0, s1, threads + 1).astype(np.int64)
            with ThreadPoolExecutor(threads) as ex:
                parts = list(ex.map(lambda ab: work(int(ab[0]), int(ab[1])),
                                    zip(cuts[:-1], cuts[1:])))
        if self.hist is not None:
            for h in parts:
                self.hist += h
        if s_range is None:
            self.sweeps_done += n_sweeps

    def exchange(self, parity: int):
        rc = lib().orc_exchange(self.L, self.nt, int(self.gauss), self.h, _p(self.T), self.seed,
                                self.exchanges_done, parity, self.s_base, 0, self.S, _p(self.J),
                                _p(self.spins), _p(self.B), _p(self.M))
        if rc != 0:
            raise ValueError("oracle rejected its arguments")
        self.exchanges_done += 1


# ---------------------------------------------------------------------------
# estimators (FP64 numpy, from the paper's definitions)
# ---------------------------------------------------------------------------
def thermal_means(acc: np.ndarray, L: int) -> dict:
    """Per (sample, slot) thermal averages from the accumulators."""
    N = float(L ** 3)
    n = acc[..., A_N]
    out = {
        "q1": acc[..., A_Q1] / n / N,
        "q2": acc[..., A_Q2] / n / N ** 2,
        "q3": acc[..., A_Q3] / n / N ** 3,
        "q4": acc[..., A_Q4] / n / N ** 4,
        "e1": acc[..., A_E1] / (2 * n) / N,       # energy per spin, both replicas
        "e2": acc[..., A_E2] / (2 * n) / N ** 2,
        "m1": acc[..., A_M1] / (2 * n) / N,
        "m2": acc[..., A_M2] / (2 * n) / N ** 2,
    }
    re = np.stack([acc[..., a_re(v)] for v in range(9)], axis=-1) / n[..., None] / N
    im = np.stack([acc[..., a_im(v)] for v in range(9)], axis=-1) / n[..., None] / N
    ab = np.stack([acc[..., a_abs2(v)] for v in range(9)], axis=-1) / n[..., None] / N ** 2
    out["qk_re"], out["qk_im"], out["qk_abs2"] = re, im, ab
    return out


def _observables_from_means(tm: dict, L: int) -> dict:
    """Disorder averages over axis 0 (samples) of the thermal means."""
    N = float(L ** 3)
    mean = lambda a: a.mean(axis=0)
    m = mean(tm["q1"])
    # central moments about the disorder mean m (global centring), binomial expansion
    c2 = tm["q2"] - 2 * m * tm["q1"] + m ** 2
    c4 = (tm["q4"] - 4 * m * tm["q3"] + 6 * m ** 2 * tm["q2"] - 4 * m ** 3 * tm["q1"]
          + m ** 4)
    g = 0.5 * (3.0 - mean(c4) / mean(c2) ** 2)
    chi0 = N * (mean(tm["q2"]) - mean(tm["q1"]) ** 2)
    chik = N * (mean(tm["qk_abs2"]) - (mean(tm["qk_re"]) ** 2 + mean(tm["qk_im"]) ** 2))
    chi1 = chik[..., 0:3].mean(axis=-1)
    chi2 = chik[..., 3:9].mean(axis=-1)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = chi0 / chi1
        xi = np.where(ratio >= 1.0, np.sqrt(np.maximum(ratio - 1.0, 0.0)), np.nan) / (
            2.0 * np.sin(np.pi / L))
        r12 = chi1 / chi2
    return {"g": g, "chi0": chi0, "chik": chik, "chi_k1": chi1, "chi_k2": chi2,
            "xi": xi, "xi_over_L": xi / L, "r12": r12,
            "e": mean(tm["e1"]), "q2": mean(tm["q2"]), "q4": mean(tm["q4"]),
            "m": mean(tm["m1"])}


def observables(acc: np.ndarray, L: int, jackknife: bool = True) -> dict:
    """Paper observables per slot, with delete-one jackknife standard errors."""
    tm = thermal_means(acc, L)
    est = _observables_from_means(tm, L)
    if not jackknife:
        return est
    S = acc.shape[0]
    reps = []
    for i in range(S):
        keep = np.ones(S, dtype=bool)
        keep[i] = False
        reps.append(_observables_from_means({k: v[keep] for k, v in tm.items()}, L))
    err = {}
    for k in est:
        th = np.stack([r[k] for r in reps], axis=0)
        with np.errstate(invalid="ignore"):  # xi is NaN where chi0/chi1 < 1; its error too
            err[k] = np.sqrt((S - 1) / S * ((th - th.mean(axis=0)) ** 2).sum(axis=0))
    est["err"] = err
    return est
