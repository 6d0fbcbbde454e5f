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
* couette_residual_floor.json -- the norms of Eq. (msites_steady) between
  checks 300 steps apart over 120 checks for two instances of HH(4;8)xH(4;20)
  started from f_eq(1, 0, 1): 24 cells, R in [1, 1.5], Kn = 5, inner wall speed
  0.1; and 32 cells, R in [1, 2], Kn = 2, inner wall speed 0.3 (Aoki tau, dt =
  min(CFL 0.4 on the radial spacing, half the relaxation time at n = 1.2)).
  With the epsilon-free weights the norms stop falling near 1e-5 and wander
  there (the weights switch between the stencils from one check to the next).

Usage: python tests/golden/make_oracle_references.py [name ...] (all by default).
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


FLOOR_INSTANCES = [dict(n_cells=24, kn=5.0, u_wall=0.1, r_in=1.0, r_out=1.5),
                   dict(n_cells=32, kn=2.0, u_wall=0.3, r_in=1.0, r_out=2.0)]
PMAX = 5.2128  # largest |p^R| of the half-range rule of order 8


def residual_floor(checks=120, every=300):
    out = []
    for inst in FLOOR_INSTANCES:
        dr = (inst["r_out"] - inst["r_in"]) / inst["n_cells"]
        dt = min(0.4 * dr / PMAX, 0.5 * np.sqrt(np.pi / 8) * inst["kn"] / 1.2)
        o = CouetteOracle("HH(4;8)xH(4;20)", CouetteGrid(inst["n_cells"], inst["r_in"], inst["r_out"]),
                          Wall(inst["u_wall"]), Wall(0.0), inst["kn"], TAU_AOKI)
        F = o.initial_equilibrium()
        prev = o.m.moments(F)
        hist = []
        for _ in range(checks):
            for _ in range(every):
                F = o.step(F, dt)
            mom = o.m.moments(F)
            hist.append(list(o.residual(mom, prev, inst["u_wall"])))
            prev = mom
        out.append({"instance": inst, "dt": dt, "every": every, "norms": hist})
    return out


ALL = {"couette_config1_10000_steps.json": config1, "couette_steady_16x320.json": steady,
       "couette_residual_floor.json": residual_floor}

if __name__ == "__main__":
    names = sys.argv[1:] or list(ALL)
    for name, fn in ((n, ALL[n]) for n in names):
        t0 = time.time()
        out = fn()
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(out, f)
        print(name, f"{time.time() - t0:.0f} s", flush=True)
