"""Thin Python binding of libsgmc.so (the C ABI in include/sgmc.h).

Argument marshalling only: every step of the Monte Carlo runs in the library's
CUDA kernels. Importing this module does not need a GPU; creating an ensemble
does, and fails loudly (RuntimeError) when the library or the GPU is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgmc.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ETIMEOUT, SG_ECANCELLED, SG_EBUSY, \
    SG_EUNSUPPORTED = range(8)
SG_PM_J, SG_GAUSS = 0, 1
SG_LAYOUT_INT8, SG_LAYOUT_MSC64 = 0, 1
NACC = 40


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sgmc error {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("rng_group", ctypes.c_int32),
                ("exchange_every", ctypes.c_int32), ("measure_every", ctypes.c_int32),
                ("n_therm", ctypes.c_int64), ("threads_per_block", ctypes.c_int32),
                ("sweeps_per_launch", ctypes.c_int32), ("watchdog_cycles", ctypes.c_uint64),
                ("sample_base", ctypes.c_int64), ("log_bins", ctypes.c_int32),
                ("pq_hist", ctypes.c_int32), ("state_mode", ctypes.c_int32),
                ("segments", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("chain_set", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_T", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("dist", ctypes.c_int32), ("n_samples", ctypes.c_int64), ("h", ctypes.c_double),
                ("attempts_per_sweep", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("log_bins", ctypes.c_int32), ("pq_hist", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("state_in_shared", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("chain_set", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("mchunk", ctypes.c_int32),
                ("n_candidates", ctypes.c_int32), ("best_ms_per_sweep", ctypes.c_double),
                ("default_ms_per_sweep", ctypes.c_double)]


class ScheduleReport(ctypes.Structure):
    _fields_ = [("exchange_every", ctypes.c_int32), ("n_candidates", ctypes.c_int32),
                ("fastest_ms_per_sweep", ctypes.c_double),
                ("ms_per_sweep", ctypes.c_double * 16)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("chunk_sweeps", ctypes.c_int64), ("use_graph", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("h", ctypes.c_double),
                ("T", ctypes.POINTER(ctypes.c_double)), ("n_T", ctypes.c_int32),
                ("dist", ctypes.c_int32), ("n_samples", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("n_sweeps", ctypes.c_int64),
                ("n_therm", ctypes.c_int64), ("layout", ctypes.c_int32),
                ("exchange_every", ctypes.c_int32), ("measure_every", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("active", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("attempts", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("device_bytes_in_use", ctypes.c_size_t), ("latency_p50", ctypes.c_double),
                ("latency_p99", ctypes.c_double)]


_OBS_FIELDS = ["g", "chi0", "chi1", "chi2", "xi", "r12", "e", "q2", "q4"]


class Observables(ctypes.Structure):
    _fields_ = [(f, ctypes.POINTER(ctypes.c_double)) for name in _OBS_FIELDS
                for f in (name, name + "_err")]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsgmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run python -m paper_1403_4560_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64, f64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_double)
    st = ctypes.c_int
    sigs = {
        "sg_options_default": (None, [P]),
        "sg_ensemble_bytes": (ctypes.c_size_t, [i32, i32, i64, i32, P]),
        "sg_create_ensemble": (st, [i32, f64, P, i32, i32, i64, u64, P, P, P, P, P]),
        "sg_destroy": (None, [P]),
        "sg_sweep": (st, [P, i64]),
        "sg_sweep_batch": (st, [P, i32, i64, i32]),
        "sg_exchange": (st, [P, i32]),
        "sg_measure": (st, [P, P, i32, P]),
        "sg_measure_noalloc": (st, [P, P, i32, P]),
        "sg_get_accumulators": (st, [P, P]),
        "sg_set_accumulators": (st, [P, P]),
        "sg_reset_accumulators": (st, [P]),
        "sg_get_histogram": (st, [P, P]),
        "sg_set_histogram": (st, [P, P]),
        "sg_get_spins": (st, [P, P]),
        "sg_set_spins": (st, [P, P]),
        "sg_set_spins_async": (st, [P, P]),
        "sg_get_accumulators_async": (st, [P, P]),
        "sg_get_energies": (st, [P, P, P]),
        "sg_get_couplings": (st, [P, P]),
        "sg_sweeps_done": (i64, [P]),
        "sg_set_sweeps_done": (st, [P, i64]),
        "sg_synchronize": (st, [P]),
        "sg_get_info": (st, [P, P]),
        "sg_launch_plan": (st, [P, i64, P, P, P]),
        "sg_results": (st, [P, P]),
        "sg_results_bin": (st, [P, i32, P]),
        "sg_observables_from_acc": (st, [P, i64, i32, i32, P]),
        "sg_threshold_map": (st, [P, i32, P]),
        "sg_accept_map": (st, [P, P, i32, P]),
        "sg_server_options_default": (None, [P]),
        "sg_request_default": (None, [P]),
        "sg_server_create": (st, [P, P, P]),
        "sg_server_submit": (st, [P, P, P]),
        "sg_server_wait": (st, [P, i64, f64, P]),
        "sg_server_result": (st, [P, i64, P, P]),
        "sg_server_cancel": (st, [P, i64]),
        "sg_server_release": (st, [P, i64]),
        "sg_server_get_stats": (st, [P, P]),
        "sg_server_destroy": (None, [P]),
        "sg_autotune": (st, [P, i64, P]),
        "sg_autotune_schedule": (st, [P, i64, P, i32, f64, P]),
        "sg_status_str": (ctypes.c_char_p, [i32]),
        "sg_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != SG_OK:
        msg = lib().sg_last_error().decode(errors="replace")
        raise SgError(status, msg)


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def default_options(**kw) -> Options:
    o = Options()
    lib().sg_options_default(ctypes.byref(o))
    names = {f for f, _ in Options._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown sg_options field {k!r}")
        setattr(o, k, v)
    return o


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    return int(getattr(stream, "cuda_stream", stream))


class Ensemble:
    """One ensemble of disorder samples (see sg_create_ensemble)."""

    def __init__(self, L: int, h: float, T, dist: str = "pmj", n_samples: int = 1,
                 seed: int = 1, J: np.ndarray | None = None, spins: np.ndarray | None = None,
                 stream=None, **options):
        self.L, self.n_samples = int(L), int(n_samples)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.n_T = len(self.T)
        self.dist = SG_GAUSS if dist in ("gauss", SG_GAUSS) else SG_PM_J
        self.opt = default_options(**options)
        self.n_bins = max(int(self.opt.log_bins), 1)
        self.has_hist = bool(self.opt.pq_hist)
        self._keep = []
        self._inflight = []  # host arrays of enqueued copies, kept until synchronize
        Jp = None
        sp = None
        if J is not None:
            J = np.ascontiguousarray(J, dtype=np.float32)
            assert J.shape == (n_samples, 3, L ** 3)
            Jp = _ptr(J)
        if spins is not None:
            spins = np.ascontiguousarray(spins, dtype=np.int8)
            assert spins.shape == (n_samples, 2, self.n_T, L ** 3)
            sp = _ptr(spins)
        h_ = ctypes.c_void_p()
        self._h = None
        _check(lib().sg_create_ensemble(self.L, float(h), _ptr(self.T), self.n_T, self.dist,
                                        self.n_samples, int(seed) & (2 ** 64 - 1),
                                        ctypes.byref(self.opt), Jp, sp,
                                        ctypes.c_void_p(_stream_handle(stream)),
                                        ctypes.byref(h_)))
        self._h = h_

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.sg_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- work ------------------------------------------------------------
    def sweep(self, n: int):
        _check(lib().sg_sweep(self._h, int(n)))

    def exchange(self, parity: int = 0):
        _check(lib().sg_exchange(self._h, int(parity)))

    def synchronize(self):
        try:
            _check(lib().sg_synchronize(self._h))
        finally:
            self._inflight.clear()

    # ---- data ------------------------------------------------------------
    def _acc_shape(self):
        if self.n_bins == 1:
            return (self.n_samples, self.n_T, NACC)
        return (self.n_samples, self.n_T, self.n_bins, NACC)

    def accumulators(self) -> np.ndarray:
        """[S][n_T][40], or [S][n_T][log_bins][40] with logarithmic bins."""
        out = np.zeros(self._acc_shape(), dtype=np.float64)
        _check(lib().sg_get_accumulators(self._h, _ptr(out)))
        return out

    def set_accumulators(self, acc: np.ndarray):
        acc = np.ascontiguousarray(acc, dtype=np.float64)
        if acc.shape != self._acc_shape():
            raise ValueError(f"accumulators must have shape {self._acc_shape()}")
        _check(lib().sg_set_accumulators(self._h, _ptr(acc)))

    def set_spins_async(self, s: np.ndarray):
        """sg_set_spins_async: enqueue the replacement of the spins; the array
        (best page-locked) is kept referenced until synchronize()."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        if s.shape != (self.n_samples, 2, self.n_T, self.L ** 3):
            raise ValueError("spins must have shape [S][2][n_T][N]")
        self._inflight.append(s)
        _check(lib().sg_set_spins_async(self._h, _ptr(s)))

    def accumulators_async(self, out: np.ndarray) -> np.ndarray:
        """sg_get_accumulators_async into `out` (float64, the accumulators'
        shape, best page-locked); valid after synchronize()."""
        if out.dtype != np.float64 or out.shape != self._acc_shape() or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous float64 array of shape {self._acc_shape()}")
        self._inflight.append(out)
        _check(lib().sg_get_accumulators_async(self._h, _ptr(out)))
        return out

    def histogram(self) -> np.ndarray:
        """Overlap histogram uint64 [n_T][log_bins][N+1]: entry k counts the
        measurements whose replicas agree on k sites (q = (2k - N) / N)."""
        out = np.zeros((self.n_T, self.n_bins, self.L ** 3 + 1), dtype=np.uint64)
        _check(lib().sg_get_histogram(self._h, _ptr(out)))
        return out

    def set_histogram(self, hist: np.ndarray):
        hist = np.ascontiguousarray(hist, dtype=np.uint64)
        if hist.shape != (self.n_T, self.n_bins, self.L ** 3 + 1):
            raise ValueError("histogram must have shape [n_T][log_bins][N+1]")
        _check(lib().sg_set_histogram(self._h, _ptr(hist)))

    def reset_accumulators(self):
        _check(lib().sg_reset_accumulators(self._h))

    def spins(self) -> np.ndarray:
        out = np.zeros((self.n_samples, 2, self.n_T, self.L ** 3), dtype=np.int8)
        _check(lib().sg_get_spins(self._h, _ptr(out)))
        return out

    def set_spins(self, s: np.ndarray):
        s = np.ascontiguousarray(s, dtype=np.int8)
        _check(lib().sg_set_spins(self._h, _ptr(s)))

    def energies(self):
        B = np.zeros((self.n_samples, 2, self.n_T), dtype=np.int64)
        M = np.zeros_like(B)
        _check(lib().sg_get_energies(self._h, _ptr(B), _ptr(M)))
        return B, M

    def couplings(self) -> np.ndarray:
        out = np.zeros((self.n_samples, 3, self.L ** 3), dtype=np.float32)
        _check(lib().sg_get_couplings(self._h, _ptr(out)))
        return out

    def measure(self, k) -> np.ndarray:
        k = np.ascontiguousarray(k, dtype=np.int32).reshape(-1, 3)
        out = np.zeros((self.n_samples, self.n_T, len(k), 2), dtype=np.float32)
        _check(lib().sg_measure(self._h, _ptr(k), len(k), _ptr(out)))
        return out

    def autotune(self, trial_sweeps: int = 8) -> dict:
        """sg_autotune: pick the fastest launch shape; state is unchanged."""
        r = TuneReport()
        _check(lib().sg_autotune(self._h, int(trial_sweeps), ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in TuneReport._fields_}

    def autotune_schedule(self, exchange_every, trial_sweeps: int = 8,
                          tolerance: float = 0.03) -> dict:
        """sg_autotune_schedule: time each exchange_every candidate and apply
        the most frequent exchange within `tolerance` of the fastest."""
        c = np.ascontiguousarray(exchange_every, dtype=np.int32)
        r = ScheduleReport()
        _check(lib().sg_autotune_schedule(self._h, int(trial_sweeps), _ptr(c), len(c),
                                          float(tolerance), ctypes.byref(r)))
        self.opt.exchange_every = r.exchange_every
        return {"exchange_every": r.exchange_every, "fastest_ms_per_sweep": r.fastest_ms_per_sweep,
                "ms_per_sweep": list(r.ms_per_sweep[:len(c)])}

    def measure_noalloc(self, k) -> np.ndarray:
        """sg_measure_noalloc: the same result, staged in the library's static
        device array instead of freshly allocated device memory."""
        k = np.ascontiguousarray(k, dtype=np.int32).reshape(-1, 3)
        out = np.zeros((self.n_samples, self.n_T, len(k), 2), dtype=np.float32)
        _check(lib().sg_measure_noalloc(self._h, _ptr(k), len(k), _ptr(out)))
        return out

    @property
    def sweeps_done(self) -> int:
        return int(lib().sg_sweeps_done(self._h))

    def set_sweeps_done(self, n: int):
        _check(lib().sg_set_sweeps_done(self._h, int(n)))

    def info(self) -> Info:
        i = Info()
        _check(lib().sg_get_info(self._h, ctypes.byref(i)))
        return i

    def launch_plan(self, n_sweeps: int) -> dict:
        """sg_launch_plan: grid, segments per sample and launches of sg_sweep(n_sweeps)."""
        g, seg, nl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sg_launch_plan(self._h, int(n_sweeps), ctypes.byref(g), ctypes.byref(seg),
                                    ctypes.byref(nl)))
        return {"grid": g.value, "segments": seg.value, "launches": nl.value}

    def results(self, bin: int | None = None) -> dict:
        """Observables of the last sweep bin, or of bin `bin`."""
        if bin is None:
            return _observables(lambda o: lib().sg_results(self._h, ctypes.byref(o)), self.n_T)
        return _observables(lambda o: lib().sg_results_bin(self._h, int(bin), ctypes.byref(o)),
                            self.n_T)


def _observables(call, nt: int) -> dict:
    arrays = {}
    o = Observables()
    for name in _OBS_FIELDS:
        for f in (name, name + "_err"):
            arrays[f] = np.zeros(nt, dtype=np.float64)
            setattr(o, f, arrays[f].ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(call(o))
    return arrays


def observables_from_acc(acc: np.ndarray, L: int) -> dict:
    """Library estimators (host C++) on an accumulator array [S][n_T][40]."""
    acc = np.ascontiguousarray(acc, dtype=np.float64)
    S, nt, _ = acc.shape
    return _observables(lambda o: lib().sg_observables_from_acc(_ptr(acc), S, nt, L,
                                                                 ctypes.byref(o)), nt)


def threshold_map(x) -> np.ndarray:
    """Device Metropolis threshold map on an FP32 array (diagnostics)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape, dtype=np.uint32)
    _check(lib().sg_threshold_map(_ptr(x), x.size, _ptr(out)))
    return out


def accept_map(x, r) -> np.ndarray:
    """Device Metropolis decision of the Gaussian sweep for (x, r) pairs
    (diagnostics): bit 0 accept, bit 1 decided by the exact threshold."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    if x.shape != r.shape:
        raise ValueError("x and r must have the same shape")
    out = np.zeros(x.shape, dtype=np.uint8)
    _check(lib().sg_accept_map(_ptr(x), _ptr(r), x.size, _ptr(out)))
    return out


def sweep_batch(ensembles, n: int, use_graph: bool = True):
    arr = (ctypes.c_void_p * len(ensembles))(*[e.handle.value for e in ensembles])
    _check(lib().sg_sweep_batch(arr, len(ensembles), int(n), int(bool(use_graph))))


class Server:
    """Request loop with continuous batching (sg_server_*)."""

    def __init__(self, memory_budget: int = 0, max_active: int = 0, chunk_sweeps: int = 256,
                 use_graph: bool = False, stream=None):
        o = ServerOptions()
        lib().sg_server_options_default(ctypes.byref(o))
        o.memory_budget, o.max_active = int(memory_budget), int(max_active)
        o.chunk_sweeps, o.use_graph = int(chunk_sweeps), int(bool(use_graph))
        h = ctypes.c_void_p()
        _check(lib().sg_server_create(ctypes.byref(o), ctypes.c_void_p(_stream_handle(stream)),
                                      ctypes.byref(h)))
        self._h = h
        self._meta = {}

    def submit(self, L, h, T, dist="pmj", n_samples=64, seed=1, n_sweeps=256, n_therm=-1,
               layout=-1, exchange_every=1, measure_every=1) -> int:
        r = Request()
        lib().sg_request_default(ctypes.byref(r))
        T = np.ascontiguousarray(T, dtype=np.float64)
        r.L, r.h, r.n_T = int(L), float(h), len(T)
        r.T = T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.dist = SG_GAUSS if dist in ("gauss", SG_GAUSS) else SG_PM_J
        r.n_samples, r.seed, r.n_sweeps = int(n_samples), int(seed), int(n_sweeps)
        r.n_therm, r.layout = int(n_therm), int(layout)
        r.exchange_every, r.measure_every = int(exchange_every), int(measure_every)
        rid = ctypes.c_int64()
        _check(lib().sg_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._meta[rid.value] = (int(n_samples), len(T))
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> int:
        state = ctypes.c_int()
        _check(lib().sg_server_wait(self._h, int(rid), float(timeout), ctypes.byref(state)))
        return state.value

    def result(self, rid: int):
        S, nt = self._meta[rid]
        acc = np.zeros((S, nt, NACC), dtype=np.float64)
        lat = ctypes.c_double()
        _check(lib().sg_server_result(self._h, int(rid), _ptr(acc), ctypes.byref(lat)))
        return acc, lat.value

    def cancel(self, rid: int):
        _check(lib().sg_server_cancel(self._h, int(rid)))

    def release(self, rid: int):
        _check(lib().sg_server_release(self._h, int(rid)))
        self._meta.pop(rid, None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().sg_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.sg_server_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
