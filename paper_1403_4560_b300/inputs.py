"""Seeded synthetic inputs for the EA spin-glass engine.

This module holds only random draws and input recipes: disorder couplings,
initial spin configurations and temperature ladders. It contains none of the
Monte Carlo arithmetic (no energies, no acceptance rule, no RNG layout of the
sweep); both the CUDA path and the CPU oracle receive what it produces as
plain arrays.

Canonical array layouts (shared interface, host memory):
  J      float32 [S][3][N]      J[s][d][i] couples site i to i + e_d (mod L),
                                d = 0, 1, 2 for x, y, z; N = L**3 and
                                i = x + L*(y + L*z).
  spins  int8    [S][2][n_T][N] +1 / -1, indexed [sample][replica][slot][site];
                                slot t holds temperature T[t] (ascending T).

The coupling distributions follow the paper's model section: bimodal +-1 with
probability 1/2 each, and zero-mean unit-variance Gaussian couplings (the
continuous distribution the paper names for the critical field and proposes
as future work). Gaussian couplings are rounded to the grid 2**-17 and clamped
to |J| <= 16 so that every local field is exact in FP32; the distortion of
N(0, 1) from the rounding is below 4e-6.
"""
from __future__ import annotations

import numpy as np

GAUSS_QUANTUM = 2.0 ** -17
GAUSS_CLAMP = 16.0


def n_sites(L: int) -> int:
    return L * L * L


def geometric_ladder(t_min: float, t_max: float, n_t: int) -> np.ndarray:
    """Ascending temperatures with a constant ratio between neighbours.

    The paper's Table I caption defines beta_n = beta_min * alpha**(n-1) with
    alpha = (beta_max/beta_min)**(1/(N_T-1)); a geometric set in beta is a
    geometric set in T, listed here in ascending T.
    """
    if n_t == 1:
        return np.array([t_min], dtype=np.float64)
    n = np.arange(n_t, dtype=np.float64)
    return t_min * (t_max / t_min) ** (n / (n_t - 1))


def pm_j_couplings(rng: np.random.Generator, n_samples: int, L: int) -> np.ndarray:
    """Bimodal couplings: +1 or -1 with probability 1/2 each (model section)."""
    bits = rng.integers(0, 2, size=(n_samples, 3, n_sites(L)), dtype=np.int8)
    return (1 - 2 * bits).astype(np.float32)


def gaussian_couplings(rng: np.random.Generator, n_samples: int, L: int) -> np.ndarray:
    """N(0, 1) couplings rounded to the 2**-17 grid, clamped to |J| <= 16."""
    g = rng.standard_normal(size=(n_samples, 3, n_sites(L)))
    q = np.clip(np.rint(g / GAUSS_QUANTUM), -GAUSS_CLAMP / GAUSS_QUANTUM,
                GAUSS_CLAMP / GAUSS_QUANTUM)
    return (q * GAUSS_QUANTUM).astype(np.float32)


def random_spins(rng: np.random.Generator, n_samples: int, n_t: int, L: int) -> np.ndarray:
    """Independent uniform +-1 spins for every sample, replica, slot and site."""
    bits = rng.integers(0, 2, size=(n_samples, 2, n_t, n_sites(L)), dtype=np.int8)
    return (1 - 2 * bits).astype(np.int8)


def make_instance(dist: str, L: int, n_samples: int, n_t: int, seed: int,
                  same_couplings: bool = False):
    """Couplings and initial spins for one ensemble.

    dist: "pmj" or "gauss". With same_couplings every sample shares the first
    sample's couplings (independent chains of one disorder realisation).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    if dist == "pmj":
        J = pm_j_couplings(rng, 1 if same_couplings else n_samples, L)
    elif dist == "gauss":
        J = gaussian_couplings(rng, 1 if same_couplings else n_samples, L)
    else:
        raise ValueError(f"unknown coupling distribution {dist!r}")
    if same_couplings:
        J = np.repeat(J, n_samples, axis=0)
    s0 = random_spins(rng, n_samples, n_t, L)
    return np.ascontiguousarray(J), np.ascontiguousarray(s0)
