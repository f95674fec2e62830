"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it only draws numbers.  The
initial state of a simulation is made by each side's own init (both implement
the same published counter-based generator); arrays drawn here are used where a
test wants arbitrary population sets.
"""
import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_array(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    """FP64 array of independent uniform draws in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=shape)


def perturbed(base: np.ndarray, seed: int, rel: float) -> np.ndarray:
    """base * (1 + rel * U(-1, 1)), elementwise."""
    return base * (1.0 + rel * rng(seed).uniform(-1.0, 1.0, size=base.shape))


def ensemble_draws(master_seed: int, n: int, sizes=(129, 257, 513, 1025),
                   log_ra=(5.0, 8.0), prs=(0.71, 7.0)):
    """(N, Ra, Pr, seed) draws for an ensemble of square 2D cells."""
    r = rng(master_seed)
    out = []
    for i in range(n):
        N = int(r.choice(sizes))
        Ra = float(10.0 ** r.uniform(*log_ra))
        Pr = float(r.choice(prs))
        out.append((N, Ra, Pr, 1000 + i))
    return out
