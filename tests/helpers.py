"""Shared helpers of the test-suite: layout conversion between the oracle
(field, cell, i, j) and the library (cell, field, i, j), and context builders."""
import numpy as np

from oracle.couette import CouetteGrid, CouetteOracle, Wall
from paper_1708_05944_gb300.inputs import perturbation


def to_lib(F):
    return np.ascontiguousarray(np.asarray(F).transpose(1, 0, 2, 3))


def to_oracle(F):
    return np.ascontiguousarray(np.asarray(F).transpose(1, 0, 2, 3))


def make_case(spec, n_cells, u_in=0.1, u_out=0.0, T_in=1.0, T_out=1.0, kn=0.1, tau_mode=1, A=0.0, delta=0.5,
              r_in=1.0, r_out=2.0, seed=12345, amplitude=0.01):
    """Oracle instance and a seeded perturbed-equilibrium input (oracle layout)."""
    o = CouetteOracle(spec, CouetteGrid(n_cells, r_in, r_out, A, delta), Wall(u_in, T_in), Wall(u_out, T_out), kn,
                      tau_mode)
    F0 = o.initial_equilibrium()
    F0 = F0 * perturbation(F0.shape, seed=seed, amplitude=amplitude)
    grid = dict(n_cells=n_cells, r_in=r_in, r_out=r_out, stretch_A=A, stretch_delta=delta)
    return o, F0, grid


def rel_err(got, ref):
    return float(np.abs(np.asarray(got, dtype=np.float64) - ref).max() / np.abs(ref).max())
