"""FP64 reference of the learned warm-start operator (oracle; test infrastructure only).

The paper has no learned component; this is the reference the GPU training
and inference kernels are checked against.  Architecture (a 1D spectral
neural operator over the normalised radius s in (0, 1)):

* input per grid point: f = [(log10 Kn + 1)/2, (u_w - 0.255)/0.245,
  (R_out/R_in - 2.75)/1.25, 2 s - 1];
* lift: h = f W_in + b_in (width C);
* L layers: h <- act(S_l(h) + h W_l + b_l), act = GELU (exact erf form) on all
  but the last layer, where the spectral part S_l is a truncated real DFT
  along the points (modes 0..K-1, rows ordered (mode, Re/Im)), a general real
  linear map per mode on its (Re, Im) pair of channel vectors (2C x 2C), and
  the inverse truncated DFT;
* projection: y = GELU(h P1 + c1) P2 + c2, four outputs per point
  (n, u^phi, T, q^R in normalised units);
* loss: mean of squared differences to normalised targets.

Parameters are one flat vector in this order: W_in (4 x C), b_in (C), then per
layer Wspec (K x 2C x 2C), W (C x C), b (C), then P1 (C x H), c1 (H),
P2 (H x 4), c2 (4); every matrix is [in][out], row-major.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def dft_matrices(M: int, K: int):
    m = np.arange(M)
    D = np.zeros((2 * K, M))
    Dinv = np.zeros((M, 2 * K))
    for k in range(K):
        th = 2.0 * math.pi * k * m / M
        D[2 * k] = np.cos(th)
        D[2 * k + 1] = -np.sin(th)
        ck = 1.0 if k == 0 else 2.0
        Dinv[:, 2 * k] = ck * np.cos(th) / M
        Dinv[:, 2 * k + 1] = -ck * np.sin(th) / M
    return D, Dinv


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def dgelu(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def features(cond, M):
    """cond (B, 3) = (Kn, u_w, R_out/R_in) -> (B, M, 4)."""
    cond = np.asarray(cond, dtype=np.float64)
    s = (np.arange(M) + 0.5) / M
    B = cond.shape[0]
    f = np.empty((B, M, 4))
    f[:, :, 0] = ((np.log10(cond[:, 0]) + 1.0) / 2.0)[:, None]
    f[:, :, 1] = ((cond[:, 1] - 0.255) / 0.245)[:, None]
    f[:, :, 2] = ((cond[:, 2] - 2.75) / 1.25)[:, None]
    f[:, :, 3] = (2.0 * s - 1.0)[None, :]
    return f


class NeuralOperator:
    def __init__(self, M=64, C=64, K=32, L=4, H=128):
        self.M, self.C, self.K, self.L, self.H = M, C, K, L, H
        self.D, self.Dinv = dft_matrices(M, K)
        shapes = [("W_in", (4, C)), ("b_in", (C,))]
        for l in range(L):
            shapes += [(f"S{l}", (K, 2 * C, 2 * C)), (f"W{l}", (C, C)), (f"b{l}", (C,))]
        shapes += [("P1", (C, H)), ("c1", (H,)), ("P2", (H, 4)), ("c2", (4,))]
        self.shapes = shapes
        self.size = sum(int(np.prod(s)) for _, s in shapes)

    def unpack(self, theta):
        out, o = {}, 0
        for name, s in self.shapes:
            n = int(np.prod(s))
            out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(s)
            o += n
        return out

    def init_params(self, seed=0):
        rng = np.random.default_rng(seed)
        parts = []
        for name, s in self.shapes:
            if len(s) == 1:
                parts.append(np.zeros(s))
            else:
                fan_in = s[-2]
                parts.append(rng.normal(0.0, 1.0 / math.sqrt(fan_in), size=s))
        return np.concatenate([p.ravel() for p in parts])

    def _spectral(self, h, S):
        """h (B, M, C) -> (B, M, C)."""
        B, M, C = h.shape
        Hh = np.einsum("km,bmc->bkc", self.D, h)                      # (B, 2K, C), rows (mode, Re/Im)
        Hm = Hh.reshape(B, self.K, 2 * C)                             # per mode the (Re, Im) channel pair
        Om = np.einsum("bki,kio->bko", Hm, S)                         # per-mode linear map
        return np.einsum("mk,bkc->bmc", self.Dinv, Om.reshape(B, 2 * self.K, C)), Hm

    def forward(self, theta, cond, keep=False):
        p = self.unpack(theta)
        x = features(cond, self.M)
        h = x @ p["W_in"] + p["b_in"]
        cache = [dict(x=x)]
        for l in range(self.L):
            s, Hm = self._spectral(h, p[f"S{l}"])
            z = s + h @ p[f"W{l}"] + p[f"b{l}"]
            cache.append(dict(h=h, Hm=Hm, z=z))
            h = gelu(z) if l < self.L - 1 else z
        a = h @ p["P1"] + p["c1"]
        y = gelu(a) @ p["P2"] + p["c2"]
        cache.append(dict(h=h, a=a))
        return (y, cache) if keep else y

    def loss_and_grad(self, theta, cond, target):
        """Mean squared error to normalised targets (B, M, 4) and its gradient."""
        p = self.unpack(theta)
        y, cache = self.forward(theta, cond, keep=True)
        n = y.size
        loss = float(((y - target) ** 2).sum() / n)
        dy = 2.0 * (y - target) / n
        g = {}
        last = cache[-1]
        ga = gelu(last["a"])
        g["P2"] = np.einsum("bmh,bmo->ho", ga, dy)
        g["c2"] = dy.sum(axis=(0, 1))
        da = (dy @ p["P2"].T) * dgelu(last["a"])
        g["P1"] = np.einsum("bmc,bmh->ch", last["h"], da)
        g["c1"] = da.sum(axis=(0, 1))
        dh = da @ p["P1"].T
        for l in reversed(range(self.L)):
            c = cache[l + 1]
            dz = dh * dgelu(c["z"]) if l < self.L - 1 else dh
            h_in = c["h"]
            g[f"W{l}"] = np.einsum("bmc,bmo->co", h_in, dz)
            g[f"b{l}"] = dz.sum(axis=(0, 1))
            B = dz.shape[0]
            dOm = np.einsum("mk,bmc->bkc", self.Dinv, dz).reshape(B, self.K, 2 * self.C)
            g[f"S{l}"] = np.einsum("bki,bko->kio", c["Hm"], dOm)
            dHm = np.einsum("bko,kio->bki", dOm, p[f"S{l}"]).reshape(B, 2 * self.K, self.C)
            dh = dz @ p[f"W{l}"].T + np.einsum("km,bkc->bmc", self.D, dHm)
        g["W_in"] = np.einsum("bmi,bmc->ic", cache[0]["x"], dh)
        g["b_in"] = dh.sum(axis=(0, 1))
        grad = np.concatenate([g[name].ravel() for name, _ in self.shapes])
        return loss, grad
