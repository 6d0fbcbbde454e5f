"""Learned warm start of batched circular Couette runs.

The paper starts every run from the rest state f_eq(n = 1, u = 0, T = 1)
(Sec. VI.A).  Here a neural operator (vlb.NeuralOperator), trained on steady
states that the solver itself computed, predicts n, u^phi, T and q^R from
(Kn, inner wall speed, R_out/R_in); the prediction is seeded into the solver
with vlb_init_from_moments and the run continues to the same steady state.

Every numerical step runs in libvlb: the stepping and seeding kernels, and the
network's forward, backward and Adam kernels.  This module sequences the calls
and does bookkeeping on small host arrays (per-instance slicing, the density
rescaling of `seed_fields`, error norms of read-back profiles).
"""
from __future__ import annotations

import numpy as np

from . import vlb

MODEL = "HH(4;8)xH(4;20)"
NO_SHAPE = dict(width=64, modes=32, layers=4, hidden=128)
TRAIN_POINTS = 64


def _model(model):
    return vlb.vlb_parse_model(model) if isinstance(model, str) else model


def p_max(model):
    p, _ = vlb.vlb_quadrature(_model(model), 0)
    return float(np.abs(p).max())


def force_radius(model):
    """Spectral radius of the momentum-space force operator of Eq. (boltz_couette_kom) at
    R = 1, (p^phi)^2 K^R - p^R Kt^phi on the model's populations.  Its eigenvalues lie
    near the imaginary axis and grow with the quadrature orders (about 656 for
    HH(4;8)xH(4;20)), so on coarse radial grids they, not the advection CFL, bound the
    time step of the third-order Runge-Kutta scheme (stable up to sqrt(3) there)."""
    m = _model(model)
    p0, _, K0, _ = vlb.vlb_axis_tables(m, 0)
    p1, _, _, Kt1 = vlb.vlb_axis_tables(m, 1)
    A = np.kron(K0, np.diag(p1 ** 2)) - np.kron(np.diag(p0), Kt1)
    return float(np.abs(np.linalg.eigvals(A)).max())


def stable_dt(inst, pmax, rho, cfl=0.4, cforce=1.2):
    """The smallest of: CFL `cfl` on the radial spacing; cforce R_in / rho for the
    force term (rho from force_radius; 1 / R is largest at the inner wall); half
    the relaxation time sqrt(pi/8) Kn / n at n = 1.2 (the stiff BGK term)."""
    dr = (inst["r_out"] - inst["r_in"]) / inst["n_cells"]
    tau = np.sqrt(np.pi / 8) * inst["kn"] / 1.2
    return min(cfl * dr / pmax, cforce * inst["r_in"] / rho, 0.5 * tau)


def conditions(insts):
    """(B, 3): Kn, inner wall speed, R_out / R_in."""
    return np.array([[i["kn"], i["u_wall"], i["r_out"] / i["r_in"]] for i in insts], dtype=np.float64)


def make_context(insts, model=MODEL, precision=vlb.VLB_FP32_BULK):
    grids = [dict(n_cells=i["n_cells"], r_in=i["r_in"], r_out=i["r_out"]) for i in insts]
    c = vlb.Couette(model, precision, grids, [(i["u_wall"], 1.0) for i in insts], [(0.0, 1.0)] * len(insts),
                    [i["kn"] for i in insts], [vlb.VLB_TAU_AOKI] * len(insts))
    pm, rho = p_max(model), force_radius(model)
    c.set_dt([stable_dt(i, pm, rho) for i in insts])
    return c


def offsets(insts):
    return np.concatenate([[0], np.cumsum([i["n_cells"] for i in insts])])


def volumes(inst):
    """Cell volumes R_{s+1/2}^2 - R_{s-1/2}^2 of the uniform grid (up to a common factor)."""
    f = np.linspace(inst["r_in"], inst["r_out"], inst["n_cells"] + 1)
    return f[1:] ** 2 - f[:-1] ** 2


def profiles(ctx, insts):
    """Per instance an (n_cells, 4) array of n, u^phi, T, q^R."""
    n, _, u1, T, _, q = ctx.read_moments(full=True)
    o = offsets(insts)
    return [np.stack([n[a:b], u1[a:b], T[a:b], q[a:b, 0]], axis=1) for a, b in zip(o[:-1], o[1:])]


def steady_states(insts, model=MODEL, precision=vlb.VLB_FP32_BULK, check_steps=200, threshold=1e-4,
                  max_steps=200_000):
    """Cold-started steady states: (profiles, first converged step per instance)."""
    c = make_context(insts, model, precision)
    c.init_equilibrium()
    _, _, conv = c.run_to_steady(0.0, check_steps, threshold, max_steps)
    out = profiles(c, insts)
    c.close()
    return out, conv


class WarmStart:
    """The network, its target scaling and the grids it is evaluated on."""

    def __init__(self, shape=None, train_points=TRAIN_POINTS):
        self.shape = dict(NO_SHAPE if shape is None else shape)
        self.train_points = train_points
        self.net = vlb.NeuralOperator(train_points, **self.shape)
        self.mean = np.zeros(4)
        self.std = np.ones(4)
        self._eval = {}

    def init_params(self, seed=0):
        """He-style normal initialisation (biases zero), drawn on the host."""
        rng = np.random.default_rng(seed)
        C, K, L, H = self.shape["width"], self.shape["modes"], self.shape["layers"], self.shape["hidden"]
        parts = [rng.normal(0, 1 / 2, (4, C)), np.zeros(C)]
        for _ in range(L):
            parts += [rng.normal(0, 1 / np.sqrt(2 * C * K), (K, 2 * C, 2 * C)), rng.normal(0, 1 / np.sqrt(C), (C, C)),
                      np.zeros(C)]
        parts += [rng.normal(0, 1 / np.sqrt(C), (C, H)), np.zeros(H), rng.normal(0, 1 / np.sqrt(H), (H, 4)),
                  np.zeros(4)]
        theta = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
        assert theta.size == self.net.size
        self.net.set_params(theta)

    def fit(self, conds, targets, steps=2000, batch=64, lr=2e-3, seed=0):
        """Adam on the mean squared error of normalised targets (B, train_points, 4);
        the learning rate decays by cosine to 5 % of `lr`.  Returns the loss history."""
        targets = np.asarray(targets, dtype=np.float64)
        self.mean = targets.reshape(-1, 4).mean(axis=0)
        self.std = targets.reshape(-1, 4).std(axis=0) + 1e-12
        self.net.set_target_scaling(self.mean, self.std)
        rng = np.random.default_rng(seed)
        B = len(conds)
        hist = []
        for s in range(steps):
            idx = rng.choice(B, size=min(batch, B), replace=False)
            rate = lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * s / steps)))
            hist.append(self.net.train_step(conds[idx], targets[idx], rate))
        self._eval.clear()
        return np.array(hist)

    def predict(self, conds, n_points):
        """(B, n_points, 4) on n_points uniform cells: the same parameters on another grid."""
        if n_points == self.train_points:
            net = self.net
        else:
            net = self._eval.get(n_points)
            if net is None:
                net = vlb.NeuralOperator(n_points, **self.shape)
                net.set_params(self.net.get_params())
                net.set_target_scaling(self.mean, self.std)
                self._eval[n_points] = net
        return net.predict(conds)

    def predict_instances(self, insts):
        out = [None] * len(insts)
        cond = conditions(insts)
        by_size = {}
        for k, i in enumerate(insts):
            by_size.setdefault(i["n_cells"], []).append(k)
        for n_points, ks in by_size.items():
            pred = self.predict(cond[ks], n_points)
            for j, k in enumerate(ks):
                out[k] = pred[j]
        return out

    def close(self):
        for net in self._eval.values():
            net.close()
        self._eval.clear()
        self.net.close()


def seed_fields(insts, preds):
    """Concatenated n, u^R, u^phi, T, q^R for vlb_init_from_moments.  The density
    is rescaled per instance to the mass of the rest state n = 1 (the walls
    conserve mass, so the run keeps the mass it starts with); u^R = 0; T is
    floored at 0.05 and n at 1e-3 of its mean."""
    n, u0, u1, T, q = [], [], [], [], []
    for inst, p in zip(insts, preds):
        V = volumes(inst)
        ni = np.maximum(p[:, 0], 1e-3 * max(np.abs(p[:, 0]).mean(), 1e-12))
        ni = ni * V.sum() / (ni * V).sum()
        n.append(ni)
        u0.append(np.zeros(len(V)))
        u1.append(p[:, 1])
        T.append(np.maximum(p[:, 2], 0.05))
        q.append(p[:, 3])
    return tuple(np.concatenate(a) for a in (n, u0, u1, T, q))


def profile_error(prof, ref, inst):
    """max over n, u^phi, T of the volume-weighted RMS deviation from a reference
    profile: relative for n and T, in units of the wall speed for u^phi."""
    V = volumes(inst)
    V = V / V.sum()
    en = np.sqrt((V * (prof[:, 0] / ref[:, 0] - 1) ** 2).sum())
    eu = np.sqrt((V * (prof[:, 1] - ref[:, 1]) ** 2).sum()) / inst["u_wall"]
    eT = np.sqrt((V * (prof[:, 2] / ref[:, 2] - 1) ** 2).sum())
    return max(en, eu, eT)


def trajectory(ctx, insts, chunk, n_chunks):
    """Profiles after every `chunk` steps (n_chunks + 1 snapshots, the first at step 0)."""
    snaps = [profiles(ctx, insts)]
    for _ in range(n_chunks):
        ctx.step_graph(0.0, chunk)
        snaps.append(profiles(ctx, insts))
    return snaps


def steps_to_tolerance(snaps, ref, insts, chunk, tol):
    """Per instance the first step after which the profile stays within tol of ref
    (-1 if it never gets there)."""
    out = np.full(len(insts), -1, dtype=np.int64)
    for k, inst in enumerate(insts):
        err = np.array([profile_error(s[k], ref[k], inst) for s in snaps])
        bad = np.nonzero(err >= tol)[0]
        last_bad = bad[-1] if len(bad) else -1
        if last_bad < len(err) - 1:
            out[k] = (last_bad + 1) * chunk
    return out


def compare(insts, ws, chunk=500, n_chunks=200, tol=1e-3, model=MODEL, precision=vlb.VLB_FP32_BULK):
    """Cold start against the learned warm start on the same instances.

    Both runs take chunk * n_chunks steps; the reference is the cold run's last
    state.  Returns (cold steps, warm steps, initial warm error, reference)."""
    cold = make_context(insts, model, precision)
    cold.init_equilibrium()
    cold_snaps = trajectory(cold, insts, chunk, n_chunks)
    cold.close()
    ref = cold_snaps[-1]
    warm = make_context(insts, model, precision)
    warm.init_from_moments(*seed_fields(insts, ws.predict_instances(insts)))
    warm_snaps = trajectory(warm, insts, chunk, n_chunks)
    warm.close()
    e0 = np.array([profile_error(warm_snaps[0][k], ref[k], i) for k, i in enumerate(insts)])
    return (steps_to_tolerance(cold_snaps, ref, insts, chunk, tol),
            steps_to_tolerance(warm_snaps, ref, insts, chunk, tol), e0, ref)
