"""vlb_step_static_scratch, the entry point for callers that cannot allocate
device memory when they step: its output must equal vlb_step's on the same
input, on two calls in a row (the second call starts from the first call's
output while the static scratch still holds the first call's stage buffers).
This file is collected last so that a failure here comes after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1708_05944_gb300 import vlb  # noqa: E402
from tests.helpers import make_case, rel_err, to_lib  # noqa: E402


@pytest.mark.parametrize("spec,n,prec", [("HH(3;4)xH(3;4)", 32, vlb.VLB_FP64),
                                         ("HH(4;8)xH(4;20)", 300, vlb.VLB_FP32_BULK),
                                         ("HH(4;8)xH(4;20)", 128, vlb.VLB_FP64)])
def test_static_scratch_step_matches_vlb_step(spec, n, prec):
    o, F0, grid = make_case(spec, n, u_in=0.15, kn=0.2)
    c = vlb.Couette(spec, prec, [grid], [(0.15, 1.0)], [(0.0, 1.0)], [0.2], [1])
    dtype = torch.float64 if prec == vlb.VLB_FP64 else torch.float32
    f_in = torch.from_numpy(to_lib(F0)).to(dtype=dtype, device="cuda").contiguous()
    dt = 2e-4
    tol = 1e-13 if prec == vlb.VLB_FP64 else 1e-6
    # reference: the context's own buffers and vlb_step
    c.set_f(f_in)
    c.step(dt, 1)
    ref1 = c.read_f().astype(np.float64)
    c.step(dt, 2)
    ref2 = c.read_f().astype(np.float64)
    # no-allocation path, two calls in a row
    out1 = torch.empty_like(f_in)
    c.step_static_scratch(f_in, out1, dt, 1)
    torch.cuda.synchronize()
    assert rel_err(out1.cpu().numpy(), ref1) <= tol
    out2 = torch.empty_like(f_in)
    c.step_static_scratch(out1, out2, dt, 2)
    torch.cuda.synchronize()
    assert rel_err(out2.cpu().numpy(), ref2) <= tol
    # the input buffer is only read
    assert torch.equal(f_in.cpu(), torch.from_numpy(to_lib(F0)).to(dtype))
    c.close()


def test_static_scratch_rejects_oversize_and_aliasing():
    spec = "HH(4;8)xH(4;20)"
    c = vlb.Couette(spec, vlb.VLB_FP64, [dict(n_cells=8000)], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    f = torch.zeros((8000, 2, 16, 20), dtype=torch.float64, device="cuda")
    g = torch.zeros_like(f)
    with pytest.raises(vlb.VlbError) as e:
        c.step_static_scratch(f, g, 1e-4, 1)
    assert e.value.status == vlb.VLB_ERR_UNSUPPORTED
    with pytest.raises(vlb.VlbError) as e:
        c.step_static_scratch(f, f, 1e-4, 1)
    assert e.value.status == vlb.VLB_ERR_INVALID
    c.close()


def test_static_scratch_rejects_channel_contexts():
    """The entry point steps Couette contexts only: a channel context (small
    enough for the scratch) gets VLB_ERR_UNSUPPORTED before anything runs, and
    its own state is untouched."""
    ch = vlb.Channel("HH(4;8)xH(4;12)", vlb.VLB_FP32_BULK, n_lambda=8, n_xi=16, kn=0.05)
    before = ch.read_f()
    f = torch.zeros((8 * 16, 2, 16, 12), dtype=torch.float32, device="cuda")
    g = torch.zeros_like(f)
    with pytest.raises(vlb.VlbError) as e:
        ch.step_static_scratch(f, g, 1e-4, 1)
    assert e.value.status == vlb.VLB_ERR_UNSUPPORTED
    assert torch.count_nonzero(g).item() == 0
    assert np.array_equal(ch.read_f(), before)
    ch.close()


def test_static_scratch_rejects_non_finite_dt():
    spec = "HH(3;4)xH(3;4)"
    c = vlb.Couette(spec, vlb.VLB_FP64, [dict(n_cells=16)], [(0.1, 1.0)], [(0.0, 1.0)], [0.1], [1])
    f = torch.zeros((16, 2, 8, 4), dtype=torch.float64, device="cuda")
    g = torch.zeros_like(f)
    for dt in (float("inf"), float("nan"), 0.0, -1e-4):
        with pytest.raises(vlb.VlbError) as e:
            c.step_static_scratch(f, g, dt, 1)
        assert e.value.status == vlb.VLB_ERR_INVALID
    c.close()
