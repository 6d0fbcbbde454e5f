"""Host-side helpers of bench.py on the CPU: the algorithmic bytes per stage launch, the L2
note's threshold, the kernel-source key of the recorded DRAM traffic (comments do not change
it, code does) and the host CPU model beside the oracle baseline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stage_bytes_is_the_three_stage_mean():
    # stage 1: F read, F^(1) written (2 fields each); stages 2, 3: F_l read too
    units, esize = 1000, 4
    assert bench.stage_bytes(units, esize) == units * esize * (4 + 6 + 6) / 3.0
    # the headline's 21.33 B per cell-velocity in FP32, 42.67 B in FP64
    assert abs(bench.stage_bytes(1, 4) - 21.333333) < 1e-5 and abs(bench.stage_bytes(1, 8) - 42.666667) < 1e-5


def test_l2_note_threshold():
    assert "larger than L2" in bench.l2_note(bench.L2_BYTES + 1)
    assert "smaller than L2" in bench.l2_note(bench.L2_BYTES // 2)
    # the headline copy: 2048 x 512 cells x 192 velocities x two 4-byte fields
    assert "1.61 GB" in bench.l2_note(2048 * 512 * 192 * 8)


def test_kernel_source_key_ignores_comments(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_1708_05944_gb300", "csrc", "vlb_channel.cuh")
    text = open(src, encoding="utf-8").read()
    base = bench.kernel_source_sha()
    fake = tmp_path / "paper_1708_05944_gb300" / "csrc"
    fake.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (fake / "vlb_channel.cuh").write_text("// a new comment line\n" + text.replace("\n}", "  // trailing\n}", 1) + "\n\n")
    assert bench.kernel_source_sha() == base
    (fake / "vlb_channel.cuh").write_text(text + "\nint x;\n")  # a line of code
    assert bench.kernel_source_sha() != base


def test_cpu_model_is_named():
    m = bench.cpu_model()
    assert isinstance(m, str) and m
