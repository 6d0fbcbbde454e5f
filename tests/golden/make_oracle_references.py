"""Write the oracle references that take too long to recompute inside a test.

Every value written here comes from oracle/ alone (the fp64 CPU oracle); the
GPU tests compare the library's results with them.  Run from the repository
root:  python tests/golden/make_oracle_references.py

* couette_config1_10000_steps.json -- the circular Couette workload of 32
  equidistant cells between R_in = 1 and R_out = 2, HH(3;4)xH(3;4), inner wall
  speed 0.1, outer wall at rest, T_w = 1, Kn = 0.1 (Aoki tau), dt = 1e-3,
  10^4 TVD-RK3 steps from the seeded perturbed equilibrium of tests/helpers.py
  (seed 12345): the final populations and moments.
* couette_steady_16x320.json -- 16 cells, HH(4;8)xH(4;20), R in [1, 2], inner
  wall speed 0.2, Kn = 0.1 (Aoki tau), from f_eq(1, 0, 1) for 13340 steps of
  dt = 1.5e-3 (20 time units of 667 steps; the residual of Eq. msites_steady between the last
  two time units is recorded): the steady moments.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.couette import TAU_AOKI, CouetteGrid, CouetteOracle, Wall  # noqa: E402
from paper_1708_05944_gb300.inputs import perturbation  # noqa: E402


def config1():
    o = CouetteOracle("HH(3;4)xH(3;4)", CouetteGrid(32), Wall(0.1), Wall(0.0), 0.1, TAU_AOKI)
    F = o.initial_equilibrium()
    F = F * perturbation(F.shape, seed=12345, amplitude=0.01)
    for _ in range(10000):
        F = o.step(F, 1e-3)
    n, u0, u1, T = o.m.moments(F)
    return {"F": F.tolist(), "n": n.tolist(), "u0": u0.tolist(), "u1": u1.tolist(), "T": T.tolist(),
            "nw": list(o.last_nw)}


def steady():
    o = CouetteOracle("HH(4;8)xH(4;20)", CouetteGrid(16), Wall(0.2), Wall(0.0), 0.1, TAU_AOKI)
    F = o.initial_equilibrium()
    dt, per_unit = 1.5e-3, 667
    prev = o.m.moments(F)
    res = None
    for unit in range(20):
        for _ in range(per_unit):
            F = o.step(F, dt)
        mom = o.m.moments(F)
        res = max(o.residual(mom, prev, 0.2))
        prev = mom
    n, u0, u1, T = prev
    return {"n": n.tolist(), "u0": u0.tolist(), "u1": u1.tolist(), "T": T.tolist(), "steps": 20 * per_unit,
            "dt": dt, "last_residual": res}


if __name__ == "__main__":
    for name, fn in (("couette_config1_10000_steps.json", config1), ("couette_steady_16x320.json", steady)):
        t0 = time.time()
        out = fn()
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(out, f)
        print(name, f"{time.time() - t0:.0f} s", flush=True)
