"""GPU forward and backward of the learned warm-start operator (BF16 tensor-core
GEMMs, FP32 accumulation) against the FP64 CPU reference, the seeding kernel
against the oracle's truncated equilibrium, and a training run that lowers the loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.couette import CouetteGrid, CouetteOracle, Wall  # noqa: E402
from oracle import seeding  # noqa: E402
from oracle.neural_operator import NeuralOperator as RefNO  # noqa: E402
from paper_1708_05944_gb300 import vlb  # noqa: E402
from tests.helpers import to_oracle  # noqa: E402

SHAPE = dict(M=64, C=64, K=32, L=4, H=128)


def make_pair(seed=1, scale=0.5):
    ref = RefNO(**SHAPE)
    theta = ref.init_params(seed) * scale
    gpu = vlb.NeuralOperator(SHAPE["M"], SHAPE["C"], SHAPE["K"], SHAPE["L"], SHAPE["H"])
    assert gpu.size == ref.size
    gpu.set_params(theta.astype(np.float32))
    gpu.set_target_scaling(np.zeros(4), np.ones(4))
    return ref, gpu, theta


def conds(B, seed):
    rng = np.random.default_rng(seed)
    return np.stack([10 ** rng.uniform(-3, 1, B), rng.uniform(0.01, 0.5, B), rng.uniform(1.5, 4, B)], axis=1)


def test_forward_matches_fp64_reference():
    ref, gpu, theta = make_pair()
    c = conds(16, 2)
    y_ref = ref.forward(theta, c)
    y = gpu.predict(c)
    err = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert err < 2e-2, err  # BF16 operands (8-bit mantissa), FP32 accumulation
    gpu.close()


def test_gradient_matches_fp64_reference():
    ref, gpu, theta = make_pair(seed=4)
    c = conds(12, 5)
    tgt = np.random.default_rng(6).normal(size=(12, 64, 4))
    loss_ref, g_ref = ref.loss_and_grad(theta, c, tgt)
    loss, g = gpu.loss_and_grad(c, tgt)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    g = g.astype(np.float64)
    cos = g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 5e-2
    # every parameter block agrees, not only the largest
    o = 0
    for name, s in ref.shapes:
        n = int(np.prod(s))
        a, b = g[o:o + n], g_ref[o:o + n]
        if np.linalg.norm(b) > 1e-8:
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-1, name
        o += n
    gpu.close()


def test_training_lowers_the_loss():
    ref, gpu, theta = make_pair(seed=9, scale=1.0)
    c = conds(32, 11)
    s = (np.arange(64) + 0.5) / 64
    # smooth targets of the conditions (a stand-in task for the check)
    tgt = np.stack([np.outer(np.log10(c[:, 0]), 1 - s), np.outer(c[:, 1], np.sin(np.pi * s)),
                    np.outer(c[:, 2], s ** 2), np.outer(c[:, 1] * c[:, 2], s)], axis=-1)
    first = gpu.train_step(c, tgt, 1e-3)
    for _ in range(200):
        last = gpu.train_step(c, tgt, 1e-3)
    assert last < 0.2 * first, (first, last)
    gpu.close()


@pytest.mark.parametrize("prec", [vlb.VLB_FP64, vlb.VLB_FP32_BULK])
@pytest.mark.parametrize("spec", ["HH(4;8)xH(4;20)", "H(4;6)xHH(3;5)"])
@pytest.mark.parametrize("with_q", [False, True])
def test_seed_from_moments_matches_oracle(prec, spec, with_q):
    N = 40
    o = CouetteOracle(spec, CouetteGrid(N), Wall(0.1), Wall(0.0), 0.1)
    rng = np.random.default_rng(3)
    n = 1 + 0.1 * rng.uniform(-1, 1, N)
    u1 = 0.2 * rng.uniform(-1, 1, N)
    u0 = 0.05 * rng.uniform(-1, 1, N)
    T = 1 + 0.1 * rng.uniform(-1, 1, N)
    q0 = 0.05 * rng.uniform(-1, 1, N) if with_q else None
    f1, f2 = seeding.seed(o.m, n, u0, u1, T, q0)
    c = vlb.Couette(spec, prec, [dict(n_cells=N)], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    c.init_from_moments(n, u0, u1, T, q0=q0)
    got = to_oracle(c.read_f())
    ref = np.stack([f1, f2])
    tol = 1e-13 if prec == vlb.VLB_FP64 else 1e-6
    assert np.abs(got - ref).max() / np.abs(ref).max() < tol
    if with_q:
        mom = o.m.full_moments(got.astype(np.float64))
        assert np.abs(mom["q0"] - q0).max() < (1e-13 if prec == vlb.VLB_FP64 else 1e-6)
    c.close()


def test_seed_rejects_invalid_fields():
    c = vlb.Couette("HH(3;4)xH(4;8)", vlb.VLB_FP64, [dict(n_cells=8)], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    ones, zeros = np.ones(8), np.zeros(8)
    with pytest.raises(vlb.VlbError):
        c.init_from_moments(ones, zeros, zeros, -ones)
    with pytest.raises(vlb.VlbError):
        c.init_from_moments(zeros, zeros, zeros, ones)
    c.close()
