"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers; it holds none of the method's
arithmetic (no quadrature, no equilibrium).  Callers multiply the drawn
factors into their own equilibrium populations.
"""
from __future__ import annotations

import numpy as np

PARITY_SEED = 12345
BATCH_SEED = 1708_05944
TRAIN_SEED = 1708_05945
HELDOUT_SEED = 1708_05946


def perturbation(shape, seed: int = PARITY_SEED, amplitude: float = 0.01) -> np.ndarray:
    """Multiplicative factors 1 + amplitude * U(-1, 1), float64."""
    rng = np.random.default_rng(seed)
    return 1.0 + amplitude * rng.uniform(-1.0, 1.0, size=shape)


def perturbation32(shape, seed: int = PARITY_SEED, amplitude: float = 0.01) -> np.ndarray:
    """Multiplicative factors 1 + amplitude * U(-1, 1) drawn in float32 (for inputs of
    gigabytes, where a float64 draw would double the host memory)."""
    rng = np.random.default_rng(seed)
    out = rng.random(size=shape, dtype=np.float32)
    out *= np.float32(2.0 * amplitude)
    out += np.float32(1.0 - amplitude)
    return out


def couette_instances(n_inst: int, seed: int = BATCH_SEED, n_min: int = 64, n_max: int = 1024,
                      log10_kn=(-3.0, 1.0)):
    """Circular Couette instances: cells ~ U{n_min..n_max}, log10 Kn ~ U[log10_kn],
    inner wall speed ~ U[0.01, 0.5], R_out/R_in ~ U[1.5, 4] with R_in = 1."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        out.append(dict(
            n_cells=int(rng.integers(n_min, n_max + 1)),
            kn=float(10.0 ** rng.uniform(*log10_kn)),
            u_wall=float(rng.uniform(0.01, 0.5)),
            r_in=1.0,
            r_out=float(rng.uniform(1.5, 4.0)),
        ))
    return out
