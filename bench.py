"""Benchmark of the vielbein lattice Boltzmann TVD-RK3 step on GB300.

Headline workload (one "step" = one full TVD-RK3 step, three stage launches):
the gradually expanding channel on its body-fitted grid, 2048 (xi) x 512
(lambda, tanh-stretched) cells, model HH(4;8)xH(4;12) (16 x 12 = 192
velocities), Kn = 0.05, particle reservoirs n_in / n_out = 2 / 1 at T0 = 1,
FP32-bulk storage and stencil arithmetic, compensated density sums and an FP64
wall-flux balance.  Input: seeded perturbed equilibrium, synthetic.  One
distribution copy is 1.6 GB, larger than L2, so no flush is needed.

Metric: cell-velocity updates per second (cells x velocities advanced by one RK3
step / time), each stage timed with CUDA events on the launching stream.  Beside
it: the end-to-end rate through the C ABI with pinned host buffers, the stage
kernel's roofline, the circular Couette scale-up batch (the L2-resident case,
FP32 and FP64), the batched Couette case (HBM-scale), a bounded time-to-steady
measurement, the measured FP64 FMA peak and the oracle on the host cores.

--impl reference times the fp64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MODEL = "HH(4;8)xH(4;20)"
N_CELLS = 1024
KNS = [1e-3, 1e-2, 0.1, 1.0, 10.0]
U_WALL = 0.1
DT = 5e-5  # CFL 0.4 with max |p^R| = 5.21 and dR = 1/1024, and below tau_min
METRIC = "cell-velocity updates/s"
L2_BYTES = 129 * 1024 * 1024  # GB300 L2
# floating-point operations of one stage per cell-velocity (both fields) of the Couette
# scale-up model, counted from the equations: WENO-5 2 x 60, force 2 x 2 (2 Q_R + Q_phi) = 144,
# moments 10, equilibrium + BGK + RK3 combine 16 (the per-cell equilibrium factors are O(cells))
FLOP_PER_CELL_VELOCITY_STAGE = 290
BATCH_N = 256  # instances of the batched Couette measurement
BATCH_F_SEED = 4  # seed of its perturbed initial populations
CH_MODEL = "HH(4;8)xH(4;12)"
CH_KN, CH_NIN, CH_NOUT = 0.05, 2.0, 1.0
CH_DT = 2e-5  # CFL 0.4 on the wall-adjacent cell of the stretched lambda grid (d lambda = 3.7e-4)
COUETTE_WORKLOAD = ("circular Couette scale-up: 1024 cells x HH(4;8)xH(4;20) (320 velocities), "
                    "Kn in {1e-3,1e-2,0.1,1,10}")
CH_NL, CH_NX = 512, 2048
CH_VEL = 192
CH_SEED = 12  # seed of the channel's perturbed initial populations
WORKLOAD = (f"gradually expanding channel: {CH_NX} (xi) x {CH_NL} (lambda) cells x {CH_MODEL} ({CH_VEL} velocities), "
            f"Kn={CH_KN}, reservoirs n_in/n_out = {CH_NIN}/{CH_NOUT}, FP32 bulk")
# DRAM bytes (read + write) per launch of the channel stage kernel from one ncu capture, keyed by
# the SHA-256 of the kernel's code at the time of the capture (a changed kernel reports null):
# see profiles/ for the command and the scaling to the full grid
CH_TRAFFIC = {"2136950b3e5fe6b7": 4.449e9, "430a6d91e4dc5596": 4.397e9, "70feb0c42dc71e10": 4.385e9,
              "26f60cccea2d0a70": 4.395e9}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_rate(local_ms, units_per_rank, steps, world):
    """(whole-job rate, the slowest rank's milliseconds).  Every rank timed
    `steps` steps of `units_per_rank` cell-velocities in `local_ms`; the job
    takes as long as its slowest rank (all-reduce MAX over the process group
    when world > 1), and the rate counts the units of all ranks."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return units_per_rank * world * steps / (total_ms * 1e-3), total_ms


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def channel_inputs(vlb, nl=CH_NL, nx=CH_NX):
    """Perturbed equilibrium f_eq(1, 0, 1) * (1 + 0.01 U(-1, 1)) of the headline channel in the
    library's caller layout (cell p * n_lambda + s, then f', f'', then the 16 x 12 nodes),
    float32; the weights come from the library's own quadrature."""
    from paper_1708_05944_gb300.inputs import perturbation32
    m = vlb.vlb_parse_model(CH_MODEL)
    _, w0 = vlb.vlb_quadrature(m, 0)
    _, w1 = vlb.vlb_quadrature(m, 1)
    F = perturbation32((nl * nx, 2, 16, 12), seed=CH_SEED)
    F *= np.outer(w0, w1).astype(np.float32)
    return F


def kernel_source_sha():
    """SHA-256 prefix of the channel kernel's code (comments and blank lines left out), the
    key of the DRAM traffic recorded for it: a changed kernel has no recorded traffic."""
    import hashlib
    import re
    path = os.path.join(ROOT, "paper_1708_05944_gb300", "csrc", "vlb_channel.cuh")
    with open(path, encoding="utf-8") as f:
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in f]
    code = "\n".join(ln for ln in lines if ln)
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def stage_bytes(units, esize):
    """Algorithmic bytes of one stage launch, averaged over the three stages: stage 1
    reads F and writes F^(1) (4 values per cell-velocity: two fields), stages 2 and 3
    also read F_l (6 values)."""
    return units * esize * (4 + 6 + 6) / 3.0


def channel_oracle_sample(seconds_target=12.0, nx_sample=8):
    """The fp64 CPU oracle, as it stands, on a bounded sample of the headline workload: a
    channel of the same model and lambda grid with nx_sample xi-columns (the whole lambda
    extent, walls and reservoirs included), whole RK3 steps until the target time."""
    from oracle.channel import ChannelGrid, ChannelOracle
    from paper_1708_05944_gb300.inputs import perturbation
    o = ChannelOracle(CH_MODEL, ChannelGrid(CH_NL, nx_sample), CH_KN, n_in=CH_NIN, n_out=CH_NOUT)
    F = o.initial_state()
    F = F * perturbation(F.shape, seed=CH_SEED)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds_target or steps == 0:
        F = o.step(F, CH_DT)
        steps += 1
    dt = time.perf_counter() - t0
    units = CH_NL * nx_sample * CH_VEL * steps
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return units / dt, steps, dt, cores


def _oracle_worker(seconds):
    v, steps, dt, _ = channel_oracle_sample(seconds_target=seconds)
    return v, steps, dt


def oracle_all_cores(seconds):
    """The same oracle sample run as one single-threaded process per visible host core, at
    once (processes started with spawn): the summed rate is the all-core CPU figure."""
    import multiprocessing as mp
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [seconds] * n)
    return float(sum(r[0] for r in res)), n, int(sum(r[1] for r in res)), float(max(r[2] for r in res))


def make_inputs(dtype):
    """Perturbed equilibrium f_eq(1, 0, 1) * (1 + 0.01 U(-1, 1)) in the library layout.
    f_eq(1, 0, 1) has weighted populations w_i w_j (f'') and w_i w_j (f'); the
    weights come from the library's own quadrature."""
    from paper_1708_05944_gb300 import vlb
    from paper_1708_05944_gb300.inputs import perturbation
    m = vlb.vlb_parse_model(MODEL)
    _, w0 = vlb.vlb_quadrature(m, 0)
    _, w1 = vlb.vlb_quadrature(m, 1)
    ww = np.outer(w0, w1)
    cells = N_CELLS * len(KNS)
    F = np.broadcast_to(ww, (cells, 2) + ww.shape) * perturbation((cells, 2) + ww.shape)
    return np.ascontiguousarray(F.astype(dtype))


def make_ctx(prec, stream_ptr):
    from paper_1708_05944_gb300 import vlb
    n = len(KNS)
    return vlb.Couette(MODEL, prec, [dict(n_cells=N_CELLS)] * n, [(U_WALL, 1.0)] * n, [(0.0, 1.0)] * n, KNS,
                       [vlb.VLB_TAU_AOKI] * n, stream=stream_ptr)


def evict_l2(flush, sink):
    """Write the flush buffer (larger than L2), then read it back into sink, so that
    the dirty lines the write leaves are written back before the next timed region."""
    flush.fill_(1.0)
    sink.copy_(flush.sum())


def time_device(ctx, torch, stream, steps, warmup, flush, dt=DT):
    """Per-step device times with CUDA events on the launching stream around one
    vlb_step call (its three stage launches, queued by the library back to back),
    and the mean stage-launch time, a third of each step (it carries the gaps
    between the launches too).  Events between the stages would put the host's
    work between them into the timed region."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        sink = torch.zeros((), dtype=flush.dtype, device=flush.device)
        for _ in range(warmup):
            ctx.step(dt, 1)
        stream.synchronize()
        step_ms = []
        for _ in range(steps):
            evict_l2(flush, sink)  # outside the events
            t0, t1 = ev(), ev()
            t0.record(stream)
            ctx.step(dt, 1)
            t1.record(stream)
            stream.synchronize()
            step_ms.append(t0.elapsed_time(t1))
    step_ms = np.array(step_ms)
    return step_ms, step_ms / 3.0


def cpu_model():
    """The host CPU's model from /proc/cpuinfo: the model name (x86), else the Arm part (Grace is
    Neoverse V2, part 0xd4f)."""
    names = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1", "0xd49": "Neoverse N2"}
    try:
        with open("/proc/cpuinfo", encoding="utf-8") as f:
            info = f.read().splitlines()
    except OSError:
        return "unknown"
    for ln in info:
        if ln.lower().startswith("model name"):
            return ln.split(":", 1)[1].strip()
    for ln in info:
        if ln.startswith("CPU part"):
            part = ln.split(":", 1)[1].strip()
            return f"Arm {names.get(part, 'part ' + part)}"
    return "unknown"


def threads_used():
    # numpy element-wise work and einsum without BLAS run on one thread
    return 1


def run_reference(args):
    """The reference arm: the oracle, as it stands, timed on the host cores on bounded
    samples of the headline workload; rank 0 alone."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        channel_oracle_sample(seconds_target=0.0, nx_sample=4)
    per = []
    for _ in range(args.steps):  # each step: one RK3 step of the 512 x 8 sample (about 3 s)
        v, steps, dt, _ = channel_oracle_sample(seconds_target=0.0)
        per.append((v, steps, dt))
    value = float(np.mean([p[0] for p in per]))
    units = CH_NL * CH_NX * CH_VEL
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-velocity updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * units / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{CH_NL} x 8 cells (all lambda rows, 8 xi-columns), "
                                                      "whole RK3 steps", "model": CH_MODEL},
            "cpu_baseline": {"value": value, "unit": "cell-velocity updates/s", "cores": threads_used(),
                             "kind": "oracle",
                             "sample": f"{sum(p[1] for p in per)} RK3 steps of a {CH_NL} x 8-cell sample of the "
                                       "channel"},
            "e2e": {"value": value, "unit": "cell-velocity updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched(args, torch, stream, vlb, flush):
    """The batched Couette workload: BATCH_N instances from the seeded sampler (cells
    U{64..1024}, log10 Kn U[-3, 1], inner wall speed U[0.01, 0.5], R_out/R_in U[1.5, 4]),
    HH(4;8)xH(4;20), FP32 bulk, each instance with its own stable time step, one
    launch per stage over all of them.  One distribution copy (~360 MB) is larger
    than L2: the Couette case measured against HBM."""
    from paper_1708_05944_gb300 import warmstart as W
    from paper_1708_05944_gb300.inputs import couette_instances, perturbation
    insts = couette_instances(BATCH_N)
    n = len(insts)
    grids = [dict(n_cells=i["n_cells"], r_in=i["r_in"], r_out=i["r_out"]) for i in insts]
    ctx = vlb.Couette(MODEL, vlb.VLB_FP32_BULK, grids, [(i["u_wall"], 1.0) for i in insts], [(0.0, 1.0)] * n,
                      [i["kn"] for i in insts], [vlb.VLB_TAU_AOKI] * n, stream=stream.cuda_stream)
    pm, rho = W.p_max(MODEL), W.force_radius(MODEL)
    ctx.set_dt([W.stable_dt(i, pm, rho) for i in insts])
    m = vlb.vlb_parse_model(MODEL)
    _, w0 = vlb.vlb_quadrature(m, 0)
    _, w1 = vlb.vlb_quadrature(m, 1)
    cells = sum(i["n_cells"] for i in insts)
    F = np.broadcast_to(np.outer(w0, w1), (cells, 2, 16, 20)) * perturbation((cells, 2, 16, 20), seed=BATCH_F_SEED)
    ctx.set_f(np.ascontiguousarray(F.astype(np.float32)))
    del F
    tuned, _ = ctx.autotune(0.0, reps=5)
    shape = ctx.variants()[tuned]
    step_ms, stage_ms = time_device(ctx, torch, stream, args.batch_steps, 3, flush, dt=0.0)
    nmom = ctx.read_moments()[0]
    ctx.close()
    units = cells * 320
    bytes_per_launch = stage_bytes(units, 4)
    launch_ms = float(stage_ms.mean())
    hbm, kind = peaks()
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    return {"workload": f"batched circular Couette: {n} instances, {cells} cells in total (64..1024 each), "
                        f"{MODEL} (320 velocities), log10 Kn in [-3, 1], FP32 bulk, per-instance dt",
            "value": units / (float(step_ms.mean()) * 1e-3), "unit": "cell-velocity updates/s",
            "ms_per_step": float(step_ms.mean()), "steps": len(step_ms),
            "launch_shape": {"cells_per_cta": shape[0], "threads": shape[1], "persistent": bool(shape[2]),
                             "autotuned": True},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": f"couette_stage_kernel<float, TC={shape[0]}, NT={shape[1]}>",
                         "peak_source": f"{kind} hbm_gbs", "algorithmic_bytes_per_launch": bytes_per_launch,
                         "launch_ms": launch_ms},
            "density_finite": bool(np.all(np.isfinite(nmom)))}


def bench_channel(args, torch, stream, vlb, world):
    """The headline: the gradually expanding channel, FP32 bulk, one RK3 step per timed
    step, each stage launch bracketed by CUDA events on the launching stream (the
    launches are milliseconds long, so the host's enqueueing between them is hidden).
    Then the same metric end to end through the C ABI from pinned host buffers."""
    nl, nx = (int(x) for x in args.channel_cells.split("x"))
    ctx = vlb.Channel(CH_MODEL, vlb.VLB_FP32_BULK, nl, nx, CH_KN, n_in=CH_NIN, n_out=CH_NOUT,
                      stream=stream.cuda_stream)
    host_in = torch.from_numpy(channel_inputs(vlb, nl, nx)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ctx.set_f(host_in)
    if args.channel_shape is None:
        tuned, _ = ctx.autotune(CH_DT, reps=3)
    else:
        tuned = args.channel_shape
        ctx.set_variant(tuned)
    shape = ctx.channel_variants()[tuned]
    tensor_cores = ctx.channel_variant_tensor_cores(tuned)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.step(CH_DT, 1)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        marks = []
        for _ in range(args.steps):
            m = [ev() for _ in range(4)]
            m[0].record(stream)
            for k in (1, 2, 3):
                ctx.stage(CH_DT, k)
                m[k].record(stream)
            marks.append(m)
        stream.synchronize()
        clocks = sampler.stop()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        step_ms = np.array([m[0].elapsed_time(m[3]) for m in marks])
        stage_ms = np.array([m[k - 1].elapsed_time(m[k]) for m in marks for k in (1, 2, 3)])
        # end to end: H2D of the step's input, one RK3 step, D2H of the result; one untimed
        # round first (the first copies from and to the pinned buffers carry one-off costs)
        e2e_steps = args.e2e_steps
        if e2e_steps > 0:
            ctx.set_f(host_in)
            ctx.step(CH_DT, 1)
            ctx.read_f(host_out)
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.set_f(host_in)
            ctx.step(CH_DT, 1)
            ctx.read_f(host_out)
        stream.synchronize()
        e2e_s = time.perf_counter() - t0
    nmom = ctx.read_moments()[0]
    ctx.close()
    units = nl * nx * CH_VEL
    value, total_ms = whole_job_rate(float(step_ms.sum()), units, args.steps, world)
    e2e_value, _ = whole_job_rate(e2e_s * 1e3, units, max(e2e_steps, 1), world)
    bytes_per_launch = stage_bytes(units, 4)
    launch_ms = float(stage_ms.mean())
    hbm, kind = peaks()
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    sha = kernel_source_sha()
    # the recorded traffic is for the full grid and the autotuned shape
    traffic = CH_TRAFFIC.get(sha) if (nl, nx) == (CH_NL, CH_NX) and args.channel_shape is None else None
    return {
        "value": value, "ms_per_step": total_ms / args.steps, "units": units, "clocks": clocks,
        "launches": 3 * args.steps,
        "launch_shape": {"rows_per_segment": shape[0], "columns_per_strip": shape[1], "threads": shape[2],
                         "force": "tensor cores (mma.sync TF32, hi/lo split)" if tensor_cores
                                  else "CUDA cores (packed FP32x2, reflection-split matrices)",
                         "autotuned": True},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "kernel": f"channel_stage_kernel<float, 16, 12, {shape[1]}, "
                                                   f"{'true' if tensor_cores else 'false'}>",
                     "kernel_source_sha": sha, "peak_source": f"{kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                     "launch_ms_by_stage": [float(stage_ms[k::3].mean()) for k in range(3)]},
        "e2e": {"value": e2e_value, "unit": "cell-velocity updates/s", "steps": e2e_steps,
                "h2d_bytes_per_step": int(host_in.numel() * 4), "d2h_bytes_per_step": int(host_out.numel() * 4)},
        "density_finite": bool(np.all(np.isfinite(nmom))),
        "variant": tuned,
    }


def time_steps(ctx, torch, stream, steps, warmup, dt, flush=None):
    """Per-step device times (CUDA events on the launching stream around each vlb_step), after
    warmup untimed steps; L2 written over before each step when flush is given."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = []
    with torch.cuda.stream(stream):
        sink = torch.zeros((), dtype=torch.float32, device="cuda")
        for _ in range(warmup):
            ctx.step(dt, 1)
        stream.synchronize()
        for _ in range(steps):
            if flush is not None:
                evict_l2(flush, sink)
            t0, t1 = ev(), ev()
            t0.record(stream)
            ctx.step(dt, 1)
            t1.record(stream)
            stream.synchronize()
            out.append(t0.elapsed_time(t1))
    return np.array(out)


def bench_next(args, torch, stream, vlb, flush, head):
    """The extensions beyond the vielbein BGK stage, each timed on its own workload: the
    channel with the paper's flow-rate ends and the Cartesian-split channel (both on the
    headline grid), the Couette scale-up batch in the f~ formulation, and the ballistic
    Couette case with 8000 velocities (the multi-kernel large-set path)."""
    hbm, kind = peaks()
    out = {}
    nl, nx = (int(x) for x in args.channel_cells.split("x"))
    units = nl * nx * CH_VEL
    for name, setup in (("channel_flow_rate", lambda c: (c.set_variant(head["variant"]), c.set_flow_rate(0.1))),
                        ("cartesian_split_channel", lambda c: c.set_formulation(vlb.VLB_CARTESIAN))):
        ctx = vlb.Channel(CH_MODEL, vlb.VLB_FP32_BULK, nl, nx, CH_KN, n_in=CH_NIN, n_out=CH_NOUT,
                          stream=stream.cuda_stream)
        ctx.set_f(channel_inputs(vlb, nl, nx))
        setup(ctx)
        ms = time_steps(ctx, torch, stream, 3, 1, CH_DT)
        ctx.close()
        launch = float(ms.mean()) / 3.0
        achieved = stage_bytes(units, 4) / (launch * 1e-3) / 1e9
        out[name] = {"value": units / (float(ms.mean()) * 1e-3), "unit": "cell-velocity updates/s",
                     "ms_per_step": float(ms.mean()), "steps": len(ms),
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                  "frac": achieved / hbm, "peak_source": f"{kind} hbm_gbs",
                                  "algorithmic_bytes_per_stage": stage_bytes(units, 4),
                                  "stage_ms": launch}}
    out["channel_flow_rate"]["workload"] = (f"the headline channel with the flow-rate ends of Sec. VII.C.1-2 "
                                            f"(Q0 = 0.1), the same stage kernel and launch shape")
    out["cartesian_split_channel"]["workload"] = ("the headline channel in the Cartesian split of Sec. VII.G: "
                                                  "per stage a cell pass (moments, equilibrium), a wall pass "
                                                  "(n_w per column) and an update pass; the cell pass reads F "
                                                  "once more than the algorithmic bytes count")
    # the Couette scale-up batch in the f~ formulation (multi-kernel stage)
    ctx = make_ctx(vlb.VLB_FP32_BULK, stream.cuda_stream)
    ctx.set_f(make_inputs(np.float32))
    ctx.set_formulation(vlb.VLB_FTILDE)
    tuned_ft, _ = ctx.autotune(DT, reps=10)
    ms = time_steps(ctx, torch, stream, 10, 2, DT, flush)
    ctx.close()
    cu = N_CELLS * len(KNS) * 320
    out["ftilde_couette"] = {"workload": COUETTE_WORKLOAD + ", FP32 bulk, f~ formulation (Sec. VI.B); L2 flushed "
                                                          "before each timed step", "value": cu / (float(ms.mean()) * 1e-3),
                             "unit": "cell-velocity updates/s", "ms_per_step": float(ms.mean()), "steps": len(ms),
                             "launch_shape": {"variant": tuned_ft, "kernel": "the fused stage kernel's f~ instance"},
                             "l2": "L2-resident copies (13 MB): a rate, not an HBM figure"}
    # the ballistic case: HH(4;200) x HH(4;10), 16 stretched cells, Kn = 1000
    spec, n = "HH(4;200)xHH(4;10)", 16
    grid = dict(n_cells=n, r_in=1.0, r_out=2.0, stretch_A=0.95, stretch_delta=0.75)
    ctx = vlb.Couette(spec, vlb.VLB_FP32_BULK, [grid], [(0.1, 1.0)], [(0.0, 1.0)], [1000.0], [vlb.VLB_TAU_KN_OVER_NT],
                      stream=stream.cuda_stream)
    ctx.init_equilibrium(1.0, 0.0, 0.0, 1.0)
    ms = time_steps(ctx, torch, stream, 50, 5, 2e-5)
    # the same steps replayed from a CUDA graph (vlb_step_graph), 200 at a time
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ctx.step_graph(2e-5, 200)
        stream.synchronize()
        t0, t1 = ev(), ev()
        t0.record(stream)
        ctx.step_graph(2e-5, 1000)
        t1.record(stream)
        stream.synchronize()
    graph_ms = t0.elapsed_time(t1) / 1000
    ctx.close()
    bu = n * 400 * 20
    out["ballistic_couette"] = {"workload": f"circular Couette, {spec} (8000 velocities), {n} stretched cells "
                                            "(A = 0.95, delta = 0.75), Kn = 1000, FP32 bulk, the multi-kernel "
                                            "large-set stage (Sec. VI.D.2)",
                                "value": bu / (float(ms.mean()) * 1e-3), "unit": "cell-velocity updates/s",
                                "ms_per_step": float(ms.mean()), "steps": len(ms),
                                "graph": {"value": bu / (graph_ms * 1e-3), "unit": "cell-velocity updates/s",
                                          "ms_per_step": graph_ms, "steps": 1000},
                                "l2": "1 MB copies: launch- and latency-bound, a rate"}
    return out


def l2_note(copy_bytes):
    """How the headline treats L2: a distribution copy larger than L2 needs no flush."""
    gb = copy_bytes / 1e9
    if copy_bytes > L2_BYTES:
        return f"inputs larger than L2 ({gb:.2f} GB per distribution copy); no flush"
    return f"inputs smaller than L2 ({gb:.3f} GB per distribution copy), not flushed: a profiling size only"


def bench_couette(args, torch, stream, vlb, flush):
    """The circular Couette scale-up batch (5 x 1024 cells x 320 velocities, one instance
    per Kn), FP32 bulk and FP64.  Its 13 MB copies fit in L2, so L2 is flushed before
    each timed step; it is reported as a rate, the L2-resident case."""
    units = N_CELLS * len(KNS) * 320
    ctx = make_ctx(vlb.VLB_FP32_BULK, stream.cuda_stream)
    ctx.set_f(make_inputs(np.float32))
    tuned32, _ = ctx.autotune(DT, reps=20)
    shape32 = ctx.variants()[tuned32]
    step_ms, stage_ms = time_device(ctx, torch, stream, args.couette_steps, 3, flush)
    # the same batch with the Shakhov collision (Pr = 2/3): the BGK stage plus its correction pass
    ctx.set_collision(vlb.VLB_SHAKHOV, 2.0 / 3.0)
    shk_ms, _ = time_device(ctx, torch, stream, max(3, min(args.couette_steps, 20)), 2, flush)
    ctx.close()
    ctx64 = make_ctx(vlb.VLB_FP64, stream.cuda_stream)
    ctx64.set_f(make_inputs(np.float64))
    tuned64, _ = ctx64.autotune(DT, reps=5)
    shape64 = ctx64.variants()[tuned64]
    s64, st64 = time_device(ctx64, torch, stream, max(3, min(args.couette_steps, 20)), 2, flush)
    ctx64.close()
    launch_ms = float(stage_ms.mean())
    b32 = stage_bytes(units, 4)
    try:
        fp64_tflops = vlb.vlb_peak_fp64()
    except Exception:
        fp64_tflops = None
    flops_per_launch = units * FLOP_PER_CELL_VELOCITY_STAGE
    launch64 = float(st64.mean())
    fp64_achieved = flops_per_launch / (launch64 * 1e-3) / 1e12
    return {
        "workload": COUETTE_WORKLOAD + ", FP32 bulk; L2 flushed before each timed step (512 MB written, then read)",
        "value": units / (float(step_ms.mean()) * 1e-3), "unit": "cell-velocity updates/s",
        "ms_per_step": float(step_ms.mean()), "steps": len(step_ms), "launch_ms": launch_ms,
        "achieved_GBps_algorithmic": b32 / (launch_ms * 1e-3) / 1e9,
        "launch_shape": {"cells_per_cta": shape32[0], "threads": shape32[1], "persistent": bool(shape32[2])},
        "shakhov": {"value": units / (float(shk_ms.mean()) * 1e-3), "unit": "cell-velocity updates/s",
                    "ms_per_step": float(shk_ms.mean()), "prandtl": 2.0 / 3.0,
                    "note": "FP32 bulk; each stage is the BGK stage kernel and the Shakhov correction kernel "
                            "(the moments of F_prev and the heat-flux term in one pass)"},
        "fp64": {"value": units / (float(s64.mean()) * 1e-3), "unit": "cell-velocity updates/s",
                 "ms_per_step": float(s64.mean()), "launch_shape": {"cells_per_cta": shape64[0], "threads": shape64[1]},
                 "roofline": {"bound": "alu", "achieved": fp64_achieved, "peak": fp64_tflops, "unit": "TFLOP/s",
                              "frac": (fp64_achieved / fp64_tflops) if fp64_tflops else None,
                              "peak_source": "measured FP64 fma throughput (vlb_peak_fp64, this run)",
                              "flops_per_cell_velocity_stage": FLOP_PER_CELL_VELOCITY_STAGE,
                              "kernel": f"couette_stage_kernel<double, TC={shape64[0]}, NT={shape64[1]}>",
                              "launch_ms": launch64}},
    }


def time_to_steady(args, torch):
    """The second metric: how long a batch of held-out Couette instances takes to reach a
    steady state, judged as the paper does by the L2 norms of Eq. (msites_steady) between
    checks (here every 500 steps, about one time unit at these time steps) falling below a
    threshold (1e-6, the metric's).  Three solvers run the same batch to the same criterion,
    each timed as a whole: the plain FP64 GPU solver from rest (the paper's start), the
    FP32-bulk batched solver from rest, and the FP32-bulk solver seeded by the learned warm
    start.  The network is trained first on steady states the solver computes (its cost is
    reported apart).  With the epsilon-free weights some instances never get below ~1e-5
    (the oracle shows the same floor); they count as not converged within the horizon."""
    from paper_1708_05944_gb300 import vlb, warmstart as W
    from paper_1708_05944_gb300.inputs import HELDOUT_SEED, TRAIN_SEED, couette_instances
    kn_range = (-1.0, 1.0)
    t0 = time.perf_counter()
    train = couette_instances(args.tts_train, seed=TRAIN_SEED, n_min=64, n_max=64, log10_kn=kn_range)
    c = W.make_context(train)
    c.init_equilibrium()
    c.step_graph(0.0, 80_000)
    targets = np.stack(W.profiles(c, train))
    c.close()
    t_data = time.perf_counter() - t0
    ws = W.WarmStart()
    ws.init_params(0)
    t1 = time.perf_counter()
    hist = ws.fit(W.conditions(train), targets, steps=1500, batch=64, lr=2e-3)
    t_train = time.perf_counter() - t1
    held = couette_instances(args.tts_instances, seed=HELDOUT_SEED, n_min=64, n_max=96, log10_kn=kn_range)
    t2 = time.perf_counter()
    seeds = W.seed_fields(held, ws.predict_instances(held))
    t_seed = time.perf_counter() - t2
    ws.close()
    check, threshold, horizon = 500, args.tts_threshold, args.tts_steps
    runs, convs = {}, {}
    for name, prec, warm in (("plain_fp64", vlb.VLB_FP64, False), ("batched_fp32", vlb.VLB_FP32_BULK, False),
                             ("warm_fp32", vlb.VLB_FP32_BULK, True)):
        ctx = W.make_context(held, precision=prec)
        if warm:
            ctx.init_from_moments(*seeds)
        else:
            ctx.init_equilibrium()
        torch.cuda.synchronize()
        a = time.perf_counter()
        taken, res, conv = ctx.run_to_steady(0.0, check, threshold, horizon)
        secs = time.perf_counter() - a
        ctx.close()
        ok = conv > 0
        convs[name] = conv
        runs[name] = {"seconds": secs + (t_seed if warm else 0.0), "steps_taken": int(taken),
                      "seconds_per_step": secs / max(taken, 1), "converged": int(ok.sum()),
                      "steps_mean_converged": float(conv[ok].mean()) if ok.any() else None,
                      "steps_max_converged": int(conv[ok].max()) if ok.any() else None,
                      "residual_median_at_end": float(np.median(res))}
    cells = sum(i["n_cells"] for i in held)
    # the instances every run brought below the threshold: each solver's time to converge
    # all of them (its last converged check times its seconds per step, plus the seed)
    common = np.all([convs[k] > 0 for k in convs], axis=0)
    to_common = {}
    for k in runs:
        if common.any():
            to_common[k] = float(convs[k][common].max()) * runs[k]["seconds_per_step"] + (
                t_seed if k == "warm_fp32" else 0.0)
    return {
        "workload": f"{len(held)} held-out Couette instances, {cells} cells in total (64..96 each), HH(4;8)xH(4;20), "
                    "log10 Kn ~ U[-1, 1], inner wall speed ~ U[0.01, 0.5], R_out/R_in ~ U[1.5, 4]; network trained on "
                    f"{len(train)} solver steady states on 64 cells",
        "criterion": f"max(L2_u, L2_n, L2_T) of Eq. (msites_steady) between checks {check} steps apart < {threshold:g}; "
                     f"horizon {horizon} steps",
        "runs": runs,
        "instances_converged_by_all": int(common.sum()),
        "seconds_to_steady_common": to_common,
        "speedup_vs_plain_fp64": {k: to_common["plain_fp64"] / to_common[k] for k in to_common},
        "warm_start_cost_s": {"training_data": t_data, "training": t_train, "seed": t_seed,
                              "final_loss": float(hist[-50:].mean())},
    }


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1708_05944_gb300 import vlb

    stream = torch.cuda.Stream()
    head = bench_channel(args, torch, stream, vlb, world)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    couette = bench_couette(args, torch, stream, vlb, flush) if args.workload in ("all", "couette") else None
    batched = bench_batched(args, torch, stream, vlb, flush) if args.workload in ("all", "batched") else None
    nxt = bench_next(args, torch, stream, vlb, flush, head) if (args.workload == "all" and not args.no_next) else None
    del flush
    steady = time_to_steady(args, torch) if (not args.no_time_to_steady and rank == 0) else None

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, steps, dt, cores = channel_oracle_sample(seconds_target=args.cpu_seconds)
        cpu = {"value": v, "unit": "cell-velocity updates/s", "cores": threads_used(), "kind": "oracle",
               "sample": f"{steps} RK3 steps of a {CH_NL} x 8-cell sample of the channel (all lambda rows, 8 "
                         f"xi-columns) in {dt:.1f} s ({cores} host cores visible, numpy single-threaded)",
               "cpu_model": cpu_model()}
        if not args.no_all_cores:
            va, na, sa, da = oracle_all_cores(args.cpu_seconds)
            cpu["all_cores"] = {"value": va, "unit": "cell-velocity updates/s", "cores": na, "kind": "oracle",
                                "sample": f"the same sample in {na} single-threaded processes at once, "
                                          f"{sa} RK3 steps in all within {da:.1f} s"}
    line = {
        "metric": METRIC, "value": head["value"], "unit": "cell-velocity updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.channel_cells == f"{CH_NL}x{CH_NX}" else
                   WORKLOAD.replace(f"{CH_NX} (xi) x {CH_NL} (lambda)", "{1} (xi) x {0} (lambda)".format(
                       *args.channel_cells.split("x"))),
                   "model": CH_MODEL, "cells": [int(x) for x in args.channel_cells.split("x")[::-1]],
                   "velocities": CH_VEL,
                   "grid": "xi in [-10, 40] equidistant, lambda tanh-stretched (A = 0.95), Re_c = 100, H/2 = 1",
                   "kn": CH_KN, "reservoirs": {"n_in": CH_NIN, "n_out": CH_NOUT, "T0": 1.0}, "dt": CH_DT,
                   "precision": "fp32-bulk (compensated density sums, fp64 wall flux)",
                   "l2": l2_note(head["units"] * 8),  # two fields of four bytes per cell-velocity
                   "launch_shape": head["launch_shape"], "replicas_per_gpu": 1},
        "roofline": head["roofline"],
        "cpu_baseline": cpu,
        "e2e": head["e2e"],
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "couette_scaleup": couette,
        "batched": batched,
        "extensions": nxt,
    }
    if steady is not None:
        line["time_to_steady"] = steady
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed RK3 steps of the headline channel")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="all", choices=["all", "channel", "couette", "batched"],
                    help="all: the channel line with the Couette scale-up and batched measurements beside it")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end steps (host buffers) of the headline")
    ap.add_argument("--channel-cells", default=f"{CH_NL}x{CH_NX}",
                    help="lambda x xi cells of the channel (another size than the headline's is for profiling)")
    ap.add_argument("--channel-shape", type=int, default=None,
                    help="channel launch shape index instead of the autotuner's choice (for profiling)")
    ap.add_argument("--couette-steps", type=int, default=100, help="timed steps of the Couette scale-up batch")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed steps of the batched Couette measurement")
    ap.add_argument("--no-time-to-steady", action="store_true", help="leave out the time-to-steady measurement")
    ap.add_argument("--no-next", action="store_true", help="leave out the extension measurements")
    ap.add_argument("--no-all-cores", action="store_true", help="leave out the all-core oracle figure")
    ap.add_argument("--tts-instances", type=int, default=24, help="held-out instances of the time-to-steady batch")
    ap.add_argument("--tts-train", type=int, default=192, help="solver steady states the warm start is trained on")
    ap.add_argument("--tts-threshold", type=float, default=1e-6, help="residual threshold of the time to steady")
    ap.add_argument("--tts-steps", type=int, default=20000, help="step horizon of the time-to-steady runs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
