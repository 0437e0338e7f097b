"""Benchmark of the stencil hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--headline-only]

Workload (one "step"): the 3D 7-point heat sweep on a 512^3 periodic grid,
u <- u + 0.1 (sum of 6 neighbours - 6u), 100 sweeps, FP32 storage and
arithmetic, followed by the FP64 interior reduction (sum, sum of squares,
max |u|) of the result.  Inputs are the seeded synthetic heat3d field (8 sine
modes + N(0, 0.01) noise), resident in HBM before timing; each buffer is
512 MiB, larger than the 129 MB L2, so no flush is needed between steps.

Metric: grid-point updates per second (GLUP/s = 1e9 interior updates / s)
and the fraction of the HBM roofline of the dominant kernel (the sweep):
algorithmic bytes = 8 per point per sweep (one FP32 read, one FP32 write).

Printed: one JSON line (rank 0).  Also measured in the same run unless
--headline-only: the FP64 variant, the 2D 5-point FP64 256^2 case, the
radius-4 leapfrog wave, the variable-coefficient forward and adjoint, and the
batched 512-grid form, each with its own roofline numbers.

--impl reference times the CPU oracle (plain C loops, double precision) on
the host cores on the same workload, a bounded slab per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N3 = 512
SWEEPS = 100
# FP64 issue rate of the GB300 (nominal 1.25 TFLOP/s FP64, an FMA counting two
# FLOPs): the bound of the FP64 sweeps, which need more DP instructions per
# point than their bytes allow at HBM speed.
FP64_INSTR_PER_S = 1.25e12 / 2
WORKLOAD = "heat3d 7-point periodic 512^3, 100 sweeps per step, FP32 + FP64 reduction"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # the samples are kept next to other run outputs when BENCH_CLOCKS_DIR
        # names a directory, else in the system temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"stencil_bench_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def aggregate_ms(ms: float, pg, device=None) -> float:
    """Job time of a replicas-only run: the slowest rank's time (all-reduce
    MAX over the process group; no data-path collective exists)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(points_per_rank_step: float, steps: int, world: int, ms_total: float) -> float:
    """Whole-job GLUP/s: the updates of all ranks divided by the job time."""
    return world * points_per_rank_step * steps / (ms_total * 1e-3) / 1e9


def source_sha(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2512_19851_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(key: str, sha: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[key]
        return float(e["dram_bytes_per_launch"]) if e.get("source_sha") == sha else None
    except Exception:
        return None


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_2512_19851_gb300 import abi, inputs
    from paper_2512_19851_gb300.grid import Grid

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the GPU arm has no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    hbm_peak, peak_kind = peaks()

    h = inputs.heat3d(n=N3)
    u0 = h.u0
    w = [0.4] + [0.1] * 6
    g = Grid((N3, N3, N3), inputs.OFFSETS_7PT, w, periodic=True, dtype=torch.float32, device=dev)
    g.set_field(u0)
    stream = torch.cuda.Stream(device=dev)
    red = torch.empty(3, dtype=torch.float64, device=dev)

    # a step: 100 sweeps and the FP64 reduction of the result, the reduction
    # fused into the last sweep (stencil_step_reduce); the first 99 sweeps are
    # issued apart so that events time them on their own
    def one_step():
        abi.stencil_step(g.h, SWEEPS - 1, stream)
        abi.stencil_step_reduce(g.h, 1, red.data_ptr(), stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            abi.stencil_step(g.h, SWEEPS - 1, stream)
            ev[i][1].record(stream)
            abi.stencil_step_reduce(g.h, 1, red.data_ptr(), stream)
            ev[i][2].record(stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ms_total = t0.elapsed_time(t1)
    sweep_ms = [a.elapsed_time(b) for a, b, _ in ev]
    last_ms = [b.elapsed_time(c) for _, b, c in ev]  # the last sweep with the fused reduction
    ms_total = aggregate_ms(ms_total, pg, dev)
    ms_step = ms_total / args.steps
    pts = N3 ** 3 * SWEEPS
    value = job_value(pts, args.steps, ws, ms_total)
    per_sweep_s = statistics.mean(sweep_ms) * 1e-3 / (SWEEPS - 1)
    # the standalone reduction of the same field, for comparison (after the timed region)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = g.bufs[g.current_slot()]
    abi.stencil_reduce(g.h, cur.data_ptr(), 0, red.data_ptr(), stream)
    r0.record(stream)
    for _ in range(5):
        abi.stencil_reduce(g.h, cur.data_ptr(), 0, red.data_ptr(), stream)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    red_alone_us = r0.elapsed_time(r1) / 5 * 1e3
    achieved = 8.0 * N3 ** 3 / per_sweep_s / 1e9
    kname = g.kernel
    sha = source_sha("k_star3d.cu")
    traffic = ncu_traffic("heat3d_f32", sha)
    clocks = clk.summary()
    result = float(red[1].item())
    assert np.isfinite(result)

    # ---------------- end to end through the public API (host buffers)
    src = torch.from_numpy(u0.astype(np.float32)).pin_memory()
    dst = torch.empty((N3, N3, N3), dtype=torch.float32).pin_memory()
    # every step is a job: its field copied in from pinned host memory, 100
    # sweeps, the result copied out; one pipelined call runs the steps, so a
    # job's copies overlap its neighbours' sweeps (the first input and the
    # last output are exposed)
    e_steps = max(3, args.steps)  # as many steps as the device-resident timing
    abi.stencil_run_host_many(g.h, SWEEPS, [src.data_ptr()] * 2, [dst.data_ptr()] * 2, stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    abi.stencil_run_host_many(g.h, SWEEPS, [src.data_ptr()] * e_steps, [dst.data_ptr()] * e_steps, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = aggregate_ms(e0.elapsed_time(e1) / e_steps, pg, dev)
    # the same through the one-job call, copies not overlapped
    abi.stencil_run_host(g.h, SWEEPS, src.data_ptr(), dst.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(3):
        abi.stencil_run_host(g.h, SWEEPS, src.data_ptr(), dst.data_ptr(), stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e1_ms = aggregate_ms(e0.elapsed_time(e1) / 3, pg, dev)
    e2e = {"value": job_value(pts, 1, ws, e_ms), "unit": "GLUP/s", "h2d_bytes_per_step": int(src.numel() * 4),
           "d2h_bytes_per_step": int(dst.numel() * 4), "ms_per_step": e_ms, "jobs": e_steps,
           "api": "stencil_run_host_many (one call for all timed steps; per step a pinned host field in by the "
                  "copy engines, 100 sweeps, the result out to pinned host memory)",
           "single_job_call": {"value": job_value(pts, 1, ws, e1_ms), "ms_per_step": e1_ms,
                               "api": "stencil_run_host (pack kernels read and write the pinned host buffers; "
                                      "nothing overlaps)"}}
    g.close()
    del src, dst

    line = {
        "metric": "grid-point updates/s (GLUP/s) and % of HBM roofline, forward and adjoint",
        "value": value,
        "unit": "GLUP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded heat3d: 8 sine modes + N(0,0.01) noise)",
        "config": {"workload": WORKLOAD, "grid": [N3, N3, N3], "sweeps_per_step": SWEEPS, "boundary": "periodic",
                   "l2": "inputs larger than L2 (512 MiB per buffer), no flush", "parallelism":
                   "replicas only" if ws > 1 else "single GPU", "kernel": kname},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": kname, "algorithmic_bytes_per_launch": 8 * N3 ** 3,
                     "sweep_us": per_sweep_s * 1e6,
                     # the FP64 reduction of each step, fused into its last sweep: its cost is
                     # that sweep's time beyond a plain sweep's
                     "reduce_us": statistics.mean(last_ms) * 1e3 - per_sweep_s * 1e6,
                     "last_sweep_with_reduction_us": statistics.mean(last_ms) * 1e3,
                     "reduce": "fused into the step's last sweep (stencil_step_reduce)",
                     # the same reduction as a separate pass over the field (reads 4 B per point)
                     "reduce_alone_us": red_alone_us,
                     "reduce_alone_frac": 4.0 * N3 ** 3 / (red_alone_us * 1e-6) / 1e9 / hbm_peak},
        "e2e": e2e,
        "gpu_launches": args.steps * (SWEEPS + 1),  # 100 sweeps (the last fused) + the final combination
        "clocks": clocks,
    }
    if rank == 0 and not args.headline_only:
        line["extra"] = extra_configs(dev, hbm_peak)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def _time(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps * 1e-3


def _time_after(setup, fn, reps, stream):
    """Mean device time of fn over reps runs (after one untimed run), each
    run preceded by an untimed setup() on the same stream."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for r in range(reps + 1):
        setup()
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            total += a.elapsed_time(b) * 1e-3
    return total / reps


def normwise(x, ref) -> float:
    """max |x - ref| / max |ref| of two device tensors, in double precision."""
    d = (x.double() - ref.double()).abs().max()
    return float(d / ref.double().abs().max())


def extra_configs(dev, hbm_peak):
    """The other workloads, each timed with CUDA events (seconds per call),
    and the measured error of each FP32 workload: its FP32 result against
    the FP64 run of the same workload on the GPU (whose kernels match the
    FP64 oracle to 1e-12 in the parity tests), normwise."""
    import numpy as np
    import torch

    from paper_2512_19851_gb300 import abi, inputs, stencils
    from paper_2512_19851_gb300.grid import Batch, Grid, VarCoefProblem

    out = {}
    s = torch.cuda.Stream(device=dev)
    # heat3d FP64 (same workload, double)
    h = inputs.heat3d(n=N3)
    g = Grid((N3,) * 3, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, periodic=True, dtype=torch.float64, device=dev)
    g.set_field(h.u0)
    t = _time(lambda: abi.stencil_step(g.h, SWEEPS, s), 2, s)
    per = t / SWEEPS
    glups = N3 ** 3 * SWEEPS / t / 1e9
    out["heat3d_f64"] = {"glups": glups, "us_per_sweep": per * 1e6,
                         "hbm_gbs": 16 * N3 ** 3 / per / 1e9, "hbm_frac": 16 * N3 ** 3 / per / 1e9 / hbm_peak,
                         "bound": "alu", "alu_peak_glups": FP64_INSTR_PER_S / 7 / 1e9,
                         "alu_frac": glups / (FP64_INSTR_PER_S / 7 / 1e9), "kernel": g.kernel}
    # FP32 error of the workload (100 sweeps from u0) against FP64
    g.set_field(h.u0)
    g.step(SWEEPS, s)
    g32 = Grid((N3,) * 3, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, periodic=True, dtype=torch.float32, device=dev)
    g32.set_field(h.u0)
    g32.step(SWEEPS, s)
    torch.cuda.synchronize()
    out["heat3d_f32_error"] = {"normwise_vs_fp64": normwise(g32.current(), g.current()), "steps": SWEEPS,
                               "grid": [N3] * 3, "bound_tested": 1e-5}
    g32.close()
    g.close()
    del h
    torch.cuda.empty_cache()
    # heat2d FP64 256^2 Dirichlet, 100 steps
    u0 = inputs.heat2d()
    g = Grid((256, 256), inputs.OFFSETS_5PT, [0.2] * 5, dtype=torch.float64, device=dev)
    g.set_field(u0)
    cfg = g.tune(100)
    t = _time(lambda: abi.stencil_step(g.h, 100, s), 20, s)
    alu_us = 256 * 256 * 5 / FP64_INSTR_PER_S * 1e6
    out["heat2d_f64"] = {"glups": 256 * 256 * 100 / t / 1e9, "us_per_step": t / 100 * 1e6,
                         "us_per_run": t * 1e6, "kernel": g.kernel, "config": list(cfg),
                         "bound": "alu", "alu_bound_us_per_step": alu_us, "alu_frac": alu_us / (t / 100 * 1e6)}
    g.close()
    # wave, radius-4 leapfrog FP32, 1000 steps
    wv = inputs.wave3d(n=N3, steps=1000)
    offs, alpha, beta = stencils.wave25()
    g = Grid((N3,) * 3, offs, alpha, beta, periodic=False, dtype=torch.float32, time_levels=2,
             device=dev)
    g.set_coeff(wv.m)
    z = np.zeros((N3,) * 3, dtype=np.float32)
    g.set_levels(z, z)
    g.set_source(wv.src, wv.amps)
    del wv, z

    def wave_run():
        g.set_step_index(0)
        abi.stencil_step(g.h, 1000, s)

    t = _time(wave_run, 1, s)
    per = t / 1000
    out["wave3d_f32"] = {"glups": N3 ** 3 * 1000 / t / 1e9, "us_per_step": per * 1e6,
                         "hbm_gbs": 16 * N3 ** 3 / per / 1e9, "hbm_frac": 16 * N3 ** 3 / per / 1e9 / hbm_peak,
                         "kernel": g.kernel, "bytes_per_point": 16}
    # FP32 error of the full run (1000 steps from rest) against FP64
    wv = inputs.wave3d(n=N3, steps=1000)
    z = np.zeros((N3,) * 3, dtype=np.float32)
    g.set_levels(z, z)
    g.set_step_index(0)
    g.step(1000, s)
    g64 = Grid((N3,) * 3, offs, alpha, beta, periodic=False, dtype=torch.float64, time_levels=2, device=dev)
    g64.set_coeff(wv.m)
    g64.set_levels(z, z)
    g64.set_source(wv.src, wv.amps)
    del wv, z
    g64.step(1000, s)
    torch.cuda.synchronize()
    out["wave3d_f32_error"] = {"normwise_vs_fp64": normwise(g.current(), g64.current()), "steps": 1000,
                               "grid": [N3] * 3, "bound_tested": 1e-3, "fp64_kernel": g64.kernel}
    g64.close()
    g.close()
    torch.cuda.empty_cache()
    # variable-coefficient forward + adjoint, 256^3, 200 steps, ckpt 20
    v = inputs.varcoef3d(n=256)
    g = Grid((256,) * 3, inputs.OFFSETS_7PT, [1.0] + [0.0] * 6, [-6.0] + [1.0] * 6, dtype=torch.float32, device=dev)
    p = VarCoefProblem(g, 200, 20)
    g.set_field(v.u0)
    g.set_coeff(v.kappa)
    t_fwd = _time(lambda: abi.stencil_step(g.h, 200, s), 3, s)
    tgt = g.new_field()
    g.interior(tgt).copy_(torch.as_tensor(v.target, dtype=torch.float32))
    del v

    def fwd_ckpt():
        abi.stencil_set_current(g.h, 0)
        abi.stencil_step_ckpt(g.h, 200, 20, p.ws.data_ptr(), s)

    def adj():
        cur = g.bufs[g.current_slot()]
        abi.stencil_residual(g.h, cur.data_ptr(), tgt.data_ptr(), p.lam.data_ptr(), p.loss.data_ptr(), s)
        abi.stencil_adjoint(g.h, 200, 20, p.ws.data_ptr(), p.lam.data_ptr(), p.lam_tmp.data_ptr(),
                            p.gk.data_ptr(), s)

    # the reverse pass that follows a checkpointed forward run (which keeps
    # the last two segments' states), each timed rep after its own forward
    # run; and a second reverse pass on the same record, which recomputes
    # every segment but the last
    t_adj = _time_after(fwd_ckpt, adj, 2, s)
    t_adj_again = _time(adj, 2, s)
    # the same reverse pass when the forward run keeps every state (one
    # 200-step segment, about 13 GB of workspace): no recomputation
    del p
    torch.cuda.empty_cache()
    p = VarCoefProblem(g, 200, 200)
    abi.stencil_set_current(g.h, 0)
    abi.stencil_step_ckpt(g.h, 200, 200, p.ws.data_ptr(), s)

    def adj_all():
        cur = g.bufs[g.current_slot()]
        abi.stencil_residual(g.h, cur.data_ptr(), tgt.data_ptr(), p.lam.data_ptr(), p.loss.data_ptr(), s)
        abi.stencil_adjoint(g.h, 200, 200, p.ws.data_ptr(), p.lam.data_ptr(), p.lam_tmp.data_ptr(),
                            p.gk.data_ptr(), s)

    t_all = _time(adj_all, 2, s)
    n4 = 256 ** 3
    out["varcoef3d_f32"] = {"fwd_glups": n4 * 200 / t_fwd / 1e9, "fwd_us_per_step": t_fwd / 200 * 1e6,
                            "fwd_hbm_frac": 12 * n4 / (t_fwd / 200) / 1e9 / hbm_peak,
                            "adj_glups": n4 * 200 / t_adj / 1e9, "adj_us_per_step": t_adj / 200 * 1e6,
                            "adj_over_fwd": t_adj / t_fwd, "ckpt_every": 20,
                            "adj_repeat_us_per_step": t_adj_again / 200 * 1e6,
                            "adj_repeat_over_fwd": t_adj_again / t_fwd,
                            "adj_keep_all_us_per_step": t_all / 200 * 1e6, "adj_keep_all_over_fwd": t_all / t_fwd,
                            "kernel": g.kernel}
    g.close()
    del p
    torch.cuda.empty_cache()
    # FP32 errors of the forward, lambda_0 and the gradient (200 steps,
    # checkpoint every 20) against FP64
    v = inputs.varcoef3d(n=256)
    res = {}
    for dt in (torch.float32, torch.float64):
        gg = Grid((256,) * 3, inputs.OFFSETS_7PT, [1.0] + [0.0] * 6, [-6.0] + [1.0] * 6, dtype=dt, device=dev)
        pp = VarCoefProblem(gg, 200, 20)
        pp.forward(v.u0, v.kappa, s)
        torch.cuda.synchronize()
        uT = gg.current().clone()
        lam0, gk, loss = pp.backward_from(target=v.target, stream=s)
        torch.cuda.synchronize()
        res[dt] = (uT, lam0.clone(), gk.clone(), float(loss[0]))
        gg.close()
        del pp
    del v
    a32, a64 = res[torch.float32], res[torch.float64]
    out["varcoef3d_f32_error"] = {"forward_normwise_vs_fp64": normwise(a32[0], a64[0]),
                                  "lambda0_normwise_vs_fp64": normwise(a32[1], a64[1]),
                                  "gradient_normwise_vs_fp64": normwise(a32[2], a64[2]),
                                  "loss_rel_vs_fp64": abs(a32[3] - a64[3]) / abs(a64[3]),
                                  "steps": 200, "ckpt_every": 20, "grid": [256] * 3,
                                  "bounds_tested": {"forward": 1e-5, "lambda0": 1e-3, "gradient": 1e-3}}
    del res, a32, a64
    torch.cuda.empty_cache()
    # the same diffusion in conservative face-averaged form (one thread per
    # point), 256^3 FP32, 200 steps, checkpoint every 20
    v = inputs.varcoef3d(n=256)
    g = Grid((256,) * 3, None, None, dtype=torch.float32, device=dev, conservative=True)
    p = VarCoefProblem(g, 200, 20)
    g.set_field(v.u0)
    g.set_coeff(v.kappa)
    t_fwd = _time(lambda: abi.stencil_step(g.h, 200, s), 3, s)
    tgt = g.new_field()
    g.interior(tgt).copy_(torch.as_tensor(v.target, dtype=torch.float32))
    del v

    def fwd_ckpt_c():
        abi.stencil_set_current(g.h, 0)
        abi.stencil_step_ckpt(g.h, 200, 20, p.ws.data_ptr(), s)

    def adj_c():
        cur = g.bufs[g.current_slot()]
        abi.stencil_residual(g.h, cur.data_ptr(), tgt.data_ptr(), p.lam.data_ptr(), p.loss.data_ptr(), s)
        abi.stencil_adjoint(g.h, 200, 20, p.ws.data_ptr(), p.lam.data_ptr(), p.lam_tmp.data_ptr(),
                            p.gk.data_ptr(), s)

    t_adj = _time_after(fwd_ckpt_c, adj_c, 2, s)
    out["conservative3d_f32"] = {"fwd_glups": n4 * 200 / t_fwd / 1e9, "fwd_us_per_step": t_fwd / 200 * 1e6,
                                 "fwd_hbm_frac": 12 * n4 / (t_fwd / 200) / 1e9 / hbm_peak,
                                 "adj_us_per_step": t_adj / 200 * 1e6, "adj_over_fwd": t_adj / t_fwd,
                                 "ckpt_every": 20, "kernel": g.kernel}
    g.close()
    del p
    torch.cuda.empty_cache()
    # batched 512 grids, FP32, 50 steps
    b = inputs.batch2d()
    bt = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=torch.float32, device=dev)
    bt.set_fields(b.fields)
    npts = int((b.shapes[:, 0] * b.shapes[:, 1]).sum())
    cfg = bt.tune(50, s)
    t = _time(lambda: bt.step(50, s), 3, s)
    out["batch2d_f32"] = {"glups": npts * 50 / t / 1e9, "ms_per_run": t * 1e3,
                          "nominal_hbm_frac": 8 * npts * 50 / t / 1e9 / hbm_peak, "config": list(cfg)}
    # the comparison the workload asks for: 512 separate plain FP64 launches
    # per step (one-thread-per-point kernel, 25,600 launches in one graph)
    bp = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=torch.float64, generic=True, device=dev)
    bp.set_fields(b.fields)
    t64 = _time(lambda: bp.step(50, s), 1, s)
    # accuracy of one 50-step FP32 batched run against the FP64 plain run
    bt.set_fields(b.fields)
    bp.set_fields(b.fields)
    bt.step(50, s)
    bp.step(50, s)
    torch.cuda.synchronize()
    err = 0.0
    for i in range(len(b.fields)):
        a32 = bt.current(i).double()
        a64 = bp.current(i)
        err = max(err, float((a32 - a64).abs().max() / a64.abs().max()))
    out["batch2d_f32"].update({"plain_f64_ms_per_run": t64 * 1e3, "speedup_vs_plain_f64": t64 / t,
                               "max_normwise_err_vs_plain_f64": err})
    # actual DRAM bytes of one 50-step launch (ncu counters of the committed
    # capture, valid while k_batch.cu is unchanged): temporal blocking keeps
    # tiles in shared memory for several steps, so they are far below the
    # nominal 8 bytes per point and step
    tr = ncu_traffic("batch2d_f32", source_sha("k_batch.cu"))
    out["batch2d_f32"].update({"nominal_bytes_per_run": 8 * npts * 50, "dram_bytes_per_run": tr,
                               "dram_gbs": tr / t / 1e9 if tr else None,
                               "dram_frac": tr / t / 1e9 / hbm_peak if tr else None})
    bp.close()
    bt.close()
    del bp, bt
    torch.cuda.empty_cache()
    out.update(frontend_laplace(dev, hbm_peak))
    out.update(cavity_flow(dev, hbm_peak))
    return out


def cavity_flow(dev, hbm_peak, n=16384, steps=3, nit=50):
    """The paper's cavity-flow benchmark at its per-GPU size: 16384^2 arrays,
    50 pressure iterations per time step, unit lid velocity, rho = 1,
    nu = 0.1 on [0, 2]^2, dt = 0.25 min(dx, dx^2 / (4 nu)) (stable at this
    resolution); from rest.  One untimed step, then `steps` timed steps."""
    import torch

    from paper_2512_19851_gb300.grid import Cavity

    out = {}
    dx = 2.0 / (n - 1)
    dt = 0.25 * min(dx, dx * dx / 0.4)
    s = torch.cuda.Stream(device=dev)
    for dtype, name in ((torch.float64, "cavity2d_f64"), (torch.float32, "cavity2d_f32")):
        c = Cavity(n, n, dx, dx, dt, 1.0, 0.1, nit, 1.0, dtype=dtype, device=dev)
        t = _time(lambda: c.step(steps, s), 1, s)
        pts = (n - 2) ** 2
        sweeps = steps * (nit + 2)
        esz = 8 if dtype == torch.float64 else 4
        # algorithmic bytes per sweep and point: pressure 2 reads (p, b) + 1 write;
        # source 2 reads + 1 write; velocity 3 reads + 2 writes
        bytes_step = esz * pts * (3 * nit + 3 + 5)
        out[name] = {"glups": pts * sweeps / t / 1e9, "ms_per_time_step": t / steps * 1e3,
                     "time_steps_per_s": steps / t, "grid": [n, n], "pressure_iterations": nit,
                     "hbm_frac": bytes_step * steps / t / 1e9 / hbm_peak,
                     "count": "interior points x (pressure iterations + 2) per time step"}
        if dtype == torch.float64:
            # FP64 instructions per cell counted by ncu
            # (smsp__sass_thread_inst_executed_op_fp64_pred_on.sum over the
            # cells of an 8192^2 step): source term 15, each pressure
            # iteration 6, fused velocity update 30.  Every cell of the
            # array runs them (boundary cells recompute clamped updates).
            dp_step = n * n * (15 + 6 * nit + 30)
            bound_s = dp_step / FP64_INSTR_PER_S
            out[name].update({"bound": "alu", "dp_instr_per_cell_step": 15 + 6 * nit + 30,
                              "alu_bound_ms_per_time_step": bound_s * 1e3,
                              "alu_frac": bound_s * steps / t})
        c.close()
        del c
        torch.cuda.empty_cache()
    return out


def frontend_laplace(dev, hbm_peak, n=16384, iters=1000):
    """Example 1 of the paper (2D Laplace/Jacobi written as slice assignments,
    boundary ring 1, interior 0) at the paper's per-GPU size, 16384^2 and
    1000 iterations, recorded and executed through the frontend.  Wall time
    of recording the 1000 assignments plus sync(), after one untimed
    identical run (array placement, graph capture)."""
    import numpy as np
    import torch

    from paper_2512_19851_gb300.frontend import Program

    out = {}
    for dt, name in ((np.float64, "laplace2d_frontend_f64"), (np.float32, "laplace2d_frontend_f32")):
        p = Program(device=dev)
        u1, u2 = p.create_array((n, n), dt), p.create_array((n, n), dt)
        u1[0, :] = u1[-1, :] = u1[:, 0] = u1[:, -1] = 1
        u2[0, :] = u2[-1, :] = u2[:, 0] = u2[:, -1] = 1
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            for _ in range(iters):
                u2[1:-1, 1:-1] = 0.25 * (u1[:-2, 1:-1] + u1[2:, 1:-1] + u1[1:-1, :-2] + u1[1:-1, 2:])
                u1, u2 = u2, u1
            t_rec = time.perf_counter() - t
            e0.record(stream)
            p.sync()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t
        dev_s = e0.elapsed_time(e1) * 1e-3
        pts = (n - 2) ** 2
        esz = np.dtype(dt).itemsize
        per = dev_s / iters
        out[name] = {"glups": pts * iters / dev_s / 1e9, "us_per_iteration": per * 1e6,
                     "glups_wall_incl_recording": pts * iters / wall / 1e9, "recording_s": t_rec,
                     "hbm_frac": 2 * esz * pts / per / 1e9 / hbm_peak, "grid": [n, n], "iterations": iters,
                     "timing": "CUDA events around sync() (the 1000 sweeps), second of two identical runs; "
                               "glups_wall_incl_recording adds the Python recording of the 1000 assignments",
                     "kernel": _fe_kernel(p), "config": _fe_config(p)}
        if dt == np.float64:
            # four DP instructions per point (a chain of four FMAs), the FP64 pipe's rate
            out[name].update({"bound": "alu", "alu_peak_glups": FP64_INSTR_PER_S / 4 / 1e9,
                              "alu_frac": pts * iters / dev_s / (FP64_INSTR_PER_S / 4)})
        p.close()
        del u1, u2, p
        torch.cuda.empty_cache()
    return out


def _fe_kernel(p):
    from paper_2512_19851_gb300 import abi
    for key, h in p._handles.items():
        if key[0] == "grid":
            return abi.stencil_info(h.h)[2]
    return None


def _fe_config(p):
    from paper_2512_19851_gb300 import abi
    for key, h in p._handles.items():
        if key[0] == "grid":
            return list(abi.stencil_tune_config(h.h))
    return None


# ----------------------------------------------------------------------------- CPU oracle
def cpu_baseline(target_s: float = 12.0, single_s: float = 6.0):
    """The oracle on the host cores: 7-point periodic sweeps of the 512^3
    workload field, double precision, on resident arrays (no copies in the
    timed region), with OpenMP over every core in the affinity mask; and the
    same oracle single-threaded on a slab of the field (all 512x512 points of
    a few planes), whose result must equal the multi-threaded one bit for bit
    (the sweep has no reductions, so the thread count cannot change it)."""
    import numpy as np

    import oracle
    from paper_2512_19851_gb300 import inputs

    cores = oracle.default_threads()
    u = np.ascontiguousarray(inputs.heat3d(n=N3).u0, dtype=np.float64)
    tmp = np.empty_like(u)
    w = [0.4] + [0.1] * 6
    t = time.perf_counter()
    oracle.sweep_const_into(u, tmp, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=cores)
    rate = 2 * u.size / (time.perf_counter() - t)
    sweeps = int(max(2, min(100, target_s * rate / u.size))) // 2 * 2
    t = time.perf_counter()
    oracle.sweep_const_into(u, tmp, inputs.OFFSETS_7PT, w, True, 0.0, sweeps, threads=cores)
    dt = time.perf_counter() - t
    # single thread on a slab sized from the multi-threaded rate
    nz = int(max(2, min(N3, single_s * rate / cores / (N3 * N3) / 2)))
    slab = np.ascontiguousarray(u[:nz])
    one = slab.copy()
    t1 = np.empty_like(slab)
    t = time.perf_counter()
    oracle.sweep_const_into(one, t1, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=1)
    dt1 = time.perf_counter() - t
    many = slab.copy()
    oracle.sweep_const_into(many, t1, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=cores)
    return {"value": u.size * sweeps / dt / 1e9, "unit": "GLUP/s", "cores": cores, "kind": "oracle",
            "sample": f"{sweeps} periodic 7-point sweeps of the 512^3 heat3d field, FP64, resident arrays, "
                      f"{cores} OpenMP threads, {dt:.1f} s",
            "single_thread": {"value": 2 * slab.size / dt1 / 1e9, "unit": "GLUP/s", "cores": 1,
                              "sample": f"2 periodic sweeps of a {nz}x512x512 slab, FP64, {dt1:.1f} s",
                              "bitwise_equal_to_multithread": bool(np.array_equal(one, many))}}


def run_reference(args):
    """The CPU oracle as the reference arm, on rank 0 only: per step, two
    periodic 7-point sweeps of a slab of the 512^3 workload (all 512x512
    points of nz planes, nz sized so the whole run takes about two minutes),
    on resident arrays, OpenMP over every core."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2512_19851_gb300 import inputs

    cores = oracle.default_threads()
    w = [0.4] + [0.1] * 6
    probe = np.ascontiguousarray(inputs.heat3d(shape=(16, N3, N3)).u0)
    ptmp = np.empty_like(probe)
    t = time.perf_counter()
    oracle.sweep_const_into(probe, ptmp, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=cores)
    rate = 2 * probe.size / (time.perf_counter() - t)
    budget = 120.0 / max(1, args.steps + args.warmup)  # seconds per step
    nz = int(max(2, min(N3, budget * rate / (2 * N3 * N3))))
    slab = np.ascontiguousarray(inputs.heat3d(shape=(nz, N3, N3)).u0)
    tmp = np.empty_like(slab)
    for _ in range(args.warmup):
        oracle.sweep_const_into(slab, tmp, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.sweep_const_into(slab, tmp, inputs.OFFSETS_7PT, w, True, 0.0, 2, threads=cores)
    dt = time.perf_counter() - t
    val = 2 * slab.size * args.steps / dt / 1e9
    sample = (f"per step: 2 periodic 7-point sweeps of a {nz}x512x512 slab of the 512^3 workload, FP64, "
              f"resident arrays")
    line = {"impl": "reference", "metric": "grid-point updates/s (GLUP/s) and % of HBM roofline, forward and adjoint",
            "value": val, "unit": "GLUP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded heat3d)",
            "config": {"workload": WORKLOAD, "grid": [N3, N3, N3]},
            "cpu_baseline": {"value": val, "unit": "GLUP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(case: str, launches: int = 3):
    """A small fixed case for ncu captures: two warm-up launches, then
    `launches` launches of the kernel under study, nothing else.  Sizes keep
    every buffer above L2 (129 MB) and the device footprint near 1 GB."""
    import numpy as np
    import torch

    from paper_2512_19851_gb300 import abi, inputs, stencils
    from paper_2512_19851_gb300.grid import Grid, VarCoefProblem

    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    if case in ("heat3d_f32", "heat3d_f64", "heat3d_f32_512"):
        dt = torch.float64 if case == "heat3d_f64" else torch.float32
        # the 512^3 case is the headline sweep itself (about 1.1 GB on the
        # device), for single-pass counter captures
        shape = (512, 512, 512) if case == "heat3d_f32_512" else (256, 512, 512)
        offs, w, _ = stencils.heat3d()
        g = Grid(shape, offs, w, periodic=True, dtype=dt)
        g.set_field(inputs.heat3d(shape=shape).u0)
        red = torch.empty(3, dtype=torch.float64, device="cuda")
        for _ in range(2 + launches):
            abi.stencil_step(g.h, 1, s)
            abi.stencil_reduce(g.h, g.bufs[g.current_slot()].data_ptr(), 0, red.data_ptr(), s)
        if dt == torch.float32:
            for _ in range(2):  # the sweep with the fused reduction
                abi.stencil_step_reduce(g.h, 1, red.data_ptr(), s)
    elif case == "laplace2d_f64":
        # Example 1's update in FP64 on a 6144^2 interior (302 MB per buffer)
        n = 6144
        g = Grid((n, n), [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4, bc_value=1.0, dtype=torch.float64)
        g.set_field(np.random.default_rng(0).random((n, n)))
        for _ in range(2 + launches):
            abi.stencil_step(g.h, 1, s)
    elif case == "heat2d":
        # the configuration stencil_tune picks for this workload (k_tb2d,
        # 16 x 14 tiles, 3 steps per launch), fixed so that no tuning
        # launches precede the captured ones
        os.environ["ST_TB2D_CFG"] = "16,14,3"
        offs, w, _ = stencils.heat2d()
        g = Grid((256, 256), offs, w, dtype=torch.float64)
        os.environ.pop("ST_TB2D_CFG")
        g.set_field(inputs.heat2d())
        for _ in range(2 + launches):
            abi.stencil_step(g.h, 100, s)
    elif case == "wave":
        n = 384
        wv = inputs.wave3d(n=n, steps=8)
        offs, alpha, beta = stencils.wave25()
        g = Grid((n,) * 3, offs, alpha, beta, periodic=False, dtype=torch.float32, time_levels=2)
        g.set_coeff(wv.m)
        z = np.zeros((n,) * 3)
        g.set_levels(z, z)
        g.set_source(wv.src, wv.amps)
        for _ in range(2 + launches):
            abi.stencil_step(g.h, 1, s)
    elif case in ("varcoef_fwd", "varcoef_adj"):
        n = 256
        v = inputs.varcoef3d(n=n)
        offs, alpha, beta = stencils.varcoef7()
        g = Grid((n,) * 3, offs, alpha, beta, dtype=torch.float32)
        g.set_field(v.u0)
        g.set_coeff(v.kappa)
        if case == "varcoef_fwd":
            for _ in range(2 + launches):
                abi.stencil_step(g.h, 1, s)
        else:
            p = VarCoefProblem(g, 2 + launches, 2 + launches)
            p.forward(v.u0, v.kappa)
            p.backward_from(target=v.target)
    elif case in ("cons_fwd", "cons_adj"):
        # the conservative face-averaged operator, 256 x 512 x 512 FP32
        shape = (256, 512, 512)
        rng = np.random.default_rng(3)
        u0 = rng.random(shape, dtype=np.float32)
        kappa = np.clip(0.05 * np.exp(0.5 * rng.standard_normal(shape, dtype=np.float32)), 0, 0.16)
        g = Grid(shape, None, None, dtype=torch.float32, conservative=True)
        g.set_field(u0)
        g.set_coeff(kappa)
        if case == "cons_fwd":
            for _ in range(2 + launches):
                abi.stencil_step(g.h, 1, s)
        else:
            p = VarCoefProblem(g, 2 + launches, 2 + launches)
            p.forward(u0, kappa)
            p.backward_from(target=u0)
    elif case in ("cavity_f32", "cavity_f64"):
        # the cavity flow's kernels on 8192^2 arrays (268 or 537 MB each)
        from paper_2512_19851_gb300.grid import Cavity
        n = 8192
        dx = 2.0 / (n - 1)
        g = Cavity(n, n, dx, dx, 0.25 * min(dx, dx * dx / 0.4), 1.0, 0.1, 10,
                   dtype=torch.float32 if case == "cavity_f32" else torch.float64)
        g.kernel = "k_cav_*"
        g.step(launches, s)
    elif case == "batch":
        from paper_2512_19851_gb300.grid import Batch
        b = inputs.batch2d()
        g = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=torch.float32)
        g.set_fields(b.fields)
        g.kernel = "k_batch"
        for _ in range(1 + launches):
            g.step(50, s)
    else:
        raise SystemExit(f"unknown profile case {case}")
    torch.cuda.synchronize()
    print(f"profile case {case} done ({g.kernel})")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline-only", action="store_true")
    ap.add_argument("--profile", default=None, help="run one small case for ncu (heat3d_f32, heat3d_f32_512, heat3d_f64, laplace2d_f64, cons_fwd, cons_adj, cavity_f32, cavity_f64, wave, "
                                                      "varcoef_fwd, varcoef_adj) and exit")
    args = ap.parse_args()
    if args.profile:
        run_profile(args.profile)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
