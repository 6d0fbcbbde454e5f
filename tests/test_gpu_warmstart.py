"""The learned warm start against the paper's cold start (rest state) on held-out
Couette instances: a network trained on the GPU by the project's own kernels,
on steady states the solver computed, seeds runs that reach the steady state
in fewer steps than runs started from rest.

Scaled to run in about a minute: 192 training states on 64 cells, 48 held-out
instances on 64..96 cells (another resolution than the training grid), Kn in
[0.1, 10], FP32-bulk stepping.  Below Kn = 0.1 the viscous time grows as 1/Kn
and a run to steady state takes millions of steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1708_05944_gb300 import warmstart as W  # noqa: E402
from paper_1708_05944_gb300.inputs import HELDOUT_SEED, TRAIN_SEED, couette_instances  # noqa: E402

KN = (-1.0, 1.0)
CHUNK, N_CHUNKS, TOL = 400, 200, 1e-3


def test_learned_warm_start_reaches_steady_state_sooner():
    train = couette_instances(192, seed=TRAIN_SEED, n_min=64, n_max=64, log10_kn=KN)
    c = W.make_context(train)
    c.init_equilibrium()
    c.step_graph(0.0, 80_000)
    targets = np.stack(W.profiles(c, train))
    c.close()
    assert np.all(np.isfinite(targets))

    ws = W.WarmStart()
    ws.init_params(0)
    hist = ws.fit(W.conditions(train), targets, steps=1500, batch=64, lr=2e-3)
    assert hist[-50:].mean() < 1e-2 * hist[:10].mean(), (hist[:10], hist[-50:])

    held = couette_instances(48, seed=HELDOUT_SEED, n_min=64, n_max=96, log10_kn=KN)
    cold, warm, e0, ref = W.compare(held, ws, chunk=CHUNK, n_chunks=N_CHUNKS, tol=TOL)
    ws.close()
    horizon = CHUNK * N_CHUNKS
    cold_c = np.where(cold < 0, horizon, cold)
    warm_c = np.where(warm < 0, horizon, warm)
    # the seed starts within a few per cent of the steady state ...
    assert np.median(e0) < 0.05, e0
    # ... and the runs it seeds arrive sooner, by a clear margin on average
    assert warm_c.mean() < 0.75 * cold_c.mean(), (cold, warm)
    assert np.mean(warm_c <= cold_c) > 0.8, (cold, warm)
    # and to the same steady state: every warm run settles within TOL of the cold one
    assert np.all(warm >= 0), warm
