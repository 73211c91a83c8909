"""Benchmark of the implicit photochemical step on the 594-species,
7,720-reaction, 150-layer column (the size of the paper's XODIAC-2025 network
on a 150-layer hot-Jupiter profile), synthetic inputs.

One step = one pass of the whole path: Gibbs energies and rate coefficients,
photolysis, reaction rates and derivatives, residual, Jacobian blocks, block
factorization, solve (FP64 sweeps, or FGMRES around the FP32 factorization in
mixed mode), and the accept/reject update.

Prints one JSON line.  `value` is implicit steps/s of the mixed-precision
path summed over ranks (each rank solves its own column: replicas, weak
scaling); the plain FP64 path is timed on the same steps beside it.
`--impl reference` times the CPU oracle instead (bounded layer sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "implicit steps/s at 594 sp x 150 layers (mixed FP32 LU + FP64 FGMRES; FP64 path beside it)"
UNIT = "steps/s"
WORKLOAD = "xodiac-594sp-7720rx-150L"
SAMPLE_LAYERS = 24          # CPU oracle sample: this many layers of the same column


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _alu_peaks(peaks):
    """Peaks of the SIMT pipes the block inversion runs on, derived from the
    measured bf16 tensor peak and NVIDIA's nominal ratios for GB300
    (bf16 dense 2.25 PF; FP64 1.25 TF; FP32 SIMT 152 SMs x 128 lanes x 2 x 2.07 GHz)."""
    scale = peaks["bf16_tflops"] / 2250.0
    return {"f64": 1.25 * scale, "f32": 152 * 128 * 2 * 2.07e9 / 1e12 * scale}


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1])); mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nme, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nme)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample_step_time(prob, layers=SAMPLE_LAYERS, steps=1):
    """CPU oracle, single thread: seconds per implicit step on `layers` layers
    of the column (same network, same profile slice), steps repeated."""
    from oracle.oracle import Oracle
    sub = prob.replace(P_bar=prob.P_bar[:layers].copy(), T=prob.T[:layers].copy(),
                       Kzz=prob.Kzz[:layers].copy(), f0=prob.f0[:layers].copy())
    o = Oracle(sub)
    n = o.initial_state()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step_delta(n, 1e-2)
        times.append(time.perf_counter() - t0)
    return times


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2512_06729_gb300 import synth
    prob = synth.full_column()
    times = oracle_sample_step_time(prob, SAMPLE_LAYERS, args.warmup + args.steps)[args.warmup:]
    per_step_full = statistics.mean(times) * prob.L / SAMPLE_LAYERS
    value = 1.0 / per_step_full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step_full * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "species": prob.S, "reactions": prob.R, "layers": prob.L,
                   "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"one implicit step on {SAMPLE_LAYERS} of the {prob.L} layers per timed step, "
                                   f"scaled by {prob.L}/{SAMPLE_LAYERS} (block Thomas is linear in layers)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_steps(col, K, stream, prof=True):
    """Device time of K controlled steps (CUDA events on the library's stream)."""
    import torch
    if prof:
        col.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    n0 = col.lib_launches()
    torch.cuda.synchronize()
    start.record(stream)
    info = col.run_to_steady(0.0, K)
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    launches = col.lib_launches() - n0
    phases = col.profile_read() if prof else {}
    if prof:
        col.profile(False)
    return ms, info, phases, launches


def run_ours(args):
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import build as xkbuild
    from paper_2512_06729_gb300 import synth, xk

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    xkbuild.build()
    prob = synth.full_column(seed=2 + rank)
    stream = torch.cuda.current_stream(dev)
    peaks, peak_kind = _peaks()
    alu = _alu_peaks(peaks)

    from paper_2512_06729_gb300 import autotune
    results = {}
    tuning = {}
    for prec in ("mixed", "fp64"):
        params = autotune.tuned(prob.S, prec)
        if not params:
            nb, ctas, _ = autotune.tune(prob, prec)
            params = {"panel_width": nb, "factor_ctas": ctas}
        tuning[prec] = params
    for prec in ("mixed", "fp64"):
        col = xk.Column(prob, prec, device=local, **tuning[prec])
        col.set_mixing_ratios(prob.f0)
        col.step(1e-8)
        for _ in range(max(args.warmup - 1, 0)):
            col.step(0.0)
        K = args.steps if prec == "mixed" else max(3, args.steps // 4)
        _barrier(ws)
        torch.cuda.synchronize()
        if prec == "mixed":
            with ClockSampler(local) as cs:
                ms, info, phases, launches = time_steps(col, K, stream)
            clocks = cs.summary()
        else:
            ms, info, phases, launches = time_steps(col, K, stream)
        _barrier(ws)
        ms = _max_over_ranks(ms, ws, dev)
        steps_done = max(int(info.steps), 1)
        results[prec] = dict(ms=ms, steps=steps_done, phases=phases, launches=launches, info=info,
                             col=col if prec == "mixed" else None)
        if prec == "fp64":
            del col
            torch.cuda.empty_cache()

    mixed = results["mixed"]
    fp64 = results["fp64"]
    S, L = prob.S, prob.L
    ms_step = mixed["ms"] / mixed["steps"]
    value = 1e3 / ms_step * ws
    fp64_ms_step = fp64["ms"] / fp64["steps"]

    def roofline(res, dtype):
        ph = res["phases"]
        fac_ms, fac_calls = ph["factor"]
        flops = 2.0 * S ** 3 * L + 3.0 * S * S * (L - 1)      # Gauss-Jordan inversions + Schur updates
        avg_s = fac_ms / max(fac_calls, 1) * 1e-3
        achieved = flops / avg_s / 1e12
        peak = alu[dtype]
        return {"kernel": f"k_factor<{'double' if dtype == 'f64' else 'float'}>", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": f"derived from {peak_kind} bf16 x nominal ratio",
                "flops_per_launch": flops, "launch_ms": avg_s * 1e3}

    # end to end through the C-ABI with host buffers: host state in, step, host state out
    col = mixed["col"]
    n_host = col.get_state()
    Ke = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        col.set_state(n_host)
        col.step(0.0)
        n_host = col.get_state()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / Ke
    e2e_s = _max_over_ranks(e2e_s, ws, dev)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        t = oracle_sample_step_time(prob, SAMPLE_LAYERS, 1)[0]
        cpu = {"value": 1.0 / (t * L / SAMPLE_LAYERS), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one implicit step on {SAMPLE_LAYERS} of the {L} layers ({t:.1f} s), "
                         f"scaled by {L}/{SAMPLE_LAYERS}"}

    if rank == 0:
        ph = {k: {"ms_total": v[0], "calls": v[1]} for k, v in mixed["phases"].items()}
        ph64 = {k: {"ms_total": v[0], "calls": v[1]} for k, v in fp64["phases"].items()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": mixed["steps"],
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "species": S, "reactions": prob.R, "layers": L,
                       "precision": "mixed: FP32 block inversions, FP64 FGMRES on the FP64 operator",
                       "l2": "inputs larger than L2: FP32 blocks 217 MB per step (FP64 433 MB)",
                       "start": "initial state, dt0 1e-8 s, adaptive dt", "parallelism": f"replicas x{ws}",
                       "factorization": tuning},
            "fp64": {"value": 1e3 / fp64_ms_step * ws, "unit": UNIT, "ms_per_step": fp64_ms_step,
                     "steps": fp64["steps"], "speedup_mixed_over_fp64": fp64_ms_step / ms_step},
            "roofline": roofline(mixed, "f32"),
            "roofline_fp64": roofline(fp64, "f64"),
            "phases_ms": ph, "phases_ms_fp64": ph64,
            "solver_iters_per_step": mixed["info"].solver_iters / mixed["steps"],
            "cpu_baseline": cpu,
            "e2e": {"value": ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": L * S * 8,
                    "d2h_bytes_per_step": L * S * 8},
            "gpu_launches": int(mixed["launches"]),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
