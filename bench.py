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
# many columns on their own streams (batch, serving, parcel sweeps): 32 hardware work queues
# instead of the default 8, so that streams do not share one queue (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "implicit steps/s at 594 sp x 150 layers (mixed FP32 LU + FP64 FGMRES; FP64 path beside it)"
UNIT = "steps/s"
WORKLOAD = "xodiac-594sp-7720rx-150L"
SAMPLE_LAYERS = 24          # CPU oracle sample: this many layers of the same column


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
# kernels, from the ncu captures summarized in profiles/, for the configuration captured there;
# a run in another configuration reports null.
PROFILED_TRAFFIC = {
    ("mixed", 16, 8, 1): (371.3e6, "k_factor_cluster<8>, two-chain launch (profiles/k_factor_cluster_594x150.txt)"),
    ("fp64", 152, 8, 0, 0): (833.5e6, "k_factor<double, 8> (profiles/k_factor_fp64_594x150.txt)"),
    ("fp64", 152, 8, 0, 1): (818.6e6, "k_factor<double, 8>, two-chain launch (profiles/k_factor_fp64_594x150.txt)"),
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _derived_peaks(peaks, kind):
    """Peaks of the other pipes from the bf16 tensor peak and NVIDIA's nominal GB300 ratios
    (dense bf16 2.25 PF, TF32 1.1 PF, FP64 1.25 TF; FP32 SIMT 152 SMs x 128 lanes x 2 x 2.07 GHz)."""
    scale = peaks["bf16_tflops"] / 2250.0
    return {"tf32": 1100.0 * scale, "f64": 1.25 * scale, "f32": 152 * 128 * 2 * 2.07e9 / 1e12 * scale,
            "kind": f"{kind} bf16 x nominal ratio"}


def live_peaks():
    """Matrix-product throughput of this GPU measured now with torch.matmul (CUDA events, best of 5):
    FP64, FP32 with TF32 tensor cores, FP32 without (SIMT).  Seconds of work in total."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, N, tf32 in (("f64", torch.float64, 4096, False), ("tf32", torch.float32, 8192, True),
                              ("f32", torch.float32, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(N, N, device="cuda", dtype=dt)
        b = torch.randn(N, N, device="cuda", dtype=dt)
        c = torch.empty(N, N, device="cuda", dtype=dt)
        best = None
        for i in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            if i >= 2:
                t = e0.elapsed_time(e1) / 1e3
                best = t if best is None else min(best, t)
        out[name] = 2.0 * N ** 3 / best / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


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


def whole_job_rate(ms_per_step, ws, device):
    """Steps/s of the whole job: every rank solves its own column (replicas),
    so the job's rate is ws steps per slowest rank's step time."""
    ms = _max_over_ranks(ms_per_step, ws, device)
    return ws * 1e3 / ms, ms


def replica_seed(rank):
    """Seed of the column a rank solves (distinct per rank)."""
    return 2 + rank


def _sample_column(prob, layers):
    return prob.replace(P_bar=prob.P_bar[:layers].copy(), T=prob.T[:layers].copy(),
                        Kzz=prob.Kzz[:layers].copy(), f0=prob.f0[:layers].copy())


def oracle_sample_step_time(prob, layers=SAMPLE_LAYERS, steps=1):
    """CPU oracle, single thread: seconds per implicit step on `layers` layers
    of the column (same network, same profile slice), steps repeated."""
    from oracle.oracle import Oracle
    o = Oracle(_sample_column(prob, layers))
    n = o.initial_state()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        o.step_delta(n, 1e-2)
        times.append(time.perf_counter() - t0)
    return times


def _oracle_worker(args):
    seed, layers, lo = args
    from oracle.oracle import Oracle
    from paper_2512_06729_gb300 import synth
    prob = synth.full_column(seed=seed)
    sub = prob.replace(P_bar=prob.P_bar[lo:lo + layers].copy(), T=prob.T[lo:lo + layers].copy(),
                       Kzz=prob.Kzz[lo:lo + layers].copy(), f0=prob.f0[lo:lo + layers].copy())
    o = Oracle(sub)
    n = o.initial_state()
    t0 = time.perf_counter()
    o.step_delta(n, 1e-2)
    return time.perf_counter() - t0


def oracle_all_cores(L, layers=SAMPLE_LAYERS, seed=2):
    """The oracle on every host core at once (spawned processes, each one step on its own
    `layers`-layer slice of the column): full-column steps/s of the whole host, and the cores."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(seed, layers, (i * layers) % max(L - layers, 1)) for i in range(cores)]
    # spawned (not forked) workers: the parent holds a CUDA context; a dead worker raises instead of hanging
    with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_oracle_worker, jobs, timeout=600))       # interpreter and library start-up, untimed
        t0 = time.perf_counter()
        list(pool.map(_oracle_worker, jobs, timeout=600))
        wall = time.perf_counter() - t0
    # cores x layers layer-steps in `wall` seconds; a full step is L layer-steps
    return cores * layers / L / wall, cores, wall


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
    """Device time of K controlled steps (CUDA events on the library's stream).  Without tracing
    the steps replay as captured CUDA graphs (one graph launch per 16 steps); with tracing every
    kernel is launched from the host between event pairs."""
    import torch
    if prof:
        col.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    n0 = col.lib_launches()
    g0 = col.graph_launches()
    torch.cuda.synchronize()
    start.record(stream)
    info = col.run_to_steady(0.0, K)
    end.record(stream)
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    launches = col.lib_launches() - n0
    graphs = col.graph_launches() - g0
    phases = col.profile_read() if prof else {}
    if prof:
        col.profile(False)
    return ms, info, phases, launches, graphs


def err_vs_oracle(prob, tuning, dt=1e-8):
    """Element-wise error of the mixed and FP64 steps against the oracle's step on the bench's
    first step (initial state, dt0), relative to n on every species above 1e-20 mixing ratio."""
    import numpy as np
    import torch
    from oracle.oracle import Oracle
    from paper_2512_06729_gb300 import xk
    o = Oracle(prob)
    n = o.initial_state()
    ng = o.grid()[0]
    keep = n > 1e-20 * ng[:, None]
    t0 = time.perf_counter()
    od = o.step_delta(n, dt)
    oracle_s = time.perf_counter() - t0
    out = {"dt": dt, "oracle_step_s": round(oracle_s, 2), "entries": int(keep.sum())}
    for prec in ("mixed", "fp64"):
        col = xk.Column(prob, prec, **tuning.get(prec, {}))
        d, iters, _ = col.step_delta(torch.as_tensor(n, device="cuda"), dt)
        rel = np.abs(d.cpu().numpy() - od)[keep] / n[keep]
        out[prec] = {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)),
                     "median": float(np.median(rel)), "within_1e-6": float((rel <= 1e-6).mean()),
                     "solver_iters": int(iters)}
        col.close()
        del col
        torch.cuda.empty_cache()
    return out


def steady_runs(prob, tuning, caps):
    """Time to steady state from the initial state (dt0 1e-8 s) for each path, in chunks of 50
    steps, each path stopped at its time cap (then reported as not converged, with how far it got).
    A key "<path>_from_equilibrium" starts that path from the chemical-equilibrium composition of
    the same elements (Sec. 2.5 option (i); computed on the device, its time included)."""
    import torch
    from paper_2512_06729_gb300 import xk
    out = {}
    for name, cap in caps.items():
        prec = name.split("_")[0]
        kw = dict(tuning.get(prec, {}))
        if prec == "mixed":
            kw["reuse_factorization"] = 1
        col = xk.Column(prob, prec, **kw)
        col.set_mixing_ratios(prob.f0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name.endswith("_from_equilibrium"):
            col.equilibrium(set_state=True)
        steps = fp64_steps = refactors = iters = 0
        t_model = 0.0
        info = None
        while time.perf_counter() - t0 < cap:
            info = col.run_to_steady(1e-8 if steps == 0 else 0.0, 50)
            steps += int(info.steps)
            fp64_steps += int(info.fp64_steps)
            refactors += int(info.refactors)
            iters += int(info.solver_iters)
            t_model += float(info.t)
            if info.converged or info.steps == 0:
                break
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[name] = {"s": round(wall, 2), "converged": bool(info and info.converged), "steps": steps,
                     "steps_per_s": round(steps / wall, 2), "fp64_route_steps": fp64_steps,
                     "fp64_refactors": refactors, "fgmres_iters": iters, "t_model_s": t_model,
                     "dt_last": float(info.dt) if info else None, "time_cap_s": cap}
        col.close()
        del col
        torch.cuda.empty_cache()
    return out


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
    prob = synth.full_column(seed=replica_seed(rank))
    stream = torch.cuda.current_stream(dev)
    peaks, peak_kind = _peaks()
    derived = _derived_peaks(peaks, peak_kind)
    live = live_peaks()

    from paper_2512_06729_gb300 import autotune
    results = {}
    tuning = {}
    tables = {}
    for prec in ("mixed", "fp64"):
        if args.no_tune:
            tuning[prec] = {}
            continue
        tuning[prec] = autotune.tuned(prob.S, prec)
        if not tuning[prec]:
            tuning[prec], table = autotune.tune(prob, prec)
            tables[prec] = [[params, round(ms, 4)] for ms, params in table]
    clocks = None
    for prec in ("mixed", "fp64"):
        col = xk.Column(prob, prec, device=local, **tuning[prec])
        col.set_mixing_ratios(prob.f0)
        info_w = col.step(1e-8)
        for _ in range(max(args.warmup - 1, 0)):
            info_w = col.step(0.0)
        # where the timed steps start: the end-to-end run repeats the same steps from here
        start_state, start_dt = col.get_state(), float(info_w.dt_next)
        K = args.steps if prec == "mixed" else max(3, args.steps // 4)
        _barrier(ws)
        torch.cuda.synchronize()
        # the headline: K steps replayed from CUDA graphs, untraced; then K more steps traced
        # (every launch between event pairs) for the per-phase times
        if prec == "mixed":
            with ClockSampler(local) as cs:
                ms, info, _, launches, graphs = time_steps(col, K, stream, prof=False)
            clocks = cs.summary()
        else:
            ms, info, _, launches, graphs = time_steps(col, K, stream, prof=False)
        _barrier(ws)
        ms_traced, info_traced, phases, _, _ = time_steps(col, K, stream, prof=True)
        steps_done = max(int(info.steps), 1)
        t = tuning[prec]
        col_cfg = {"bcr": t.get("fp32_bcr", 1) if prec == "mixed" else 0, "cluster": t.get("cluster_size", 16),
                   "nb": t.get("panel_width", 8) or 8, "twisted": t.get("twisted", 1),
                   "ctas": t.get("factor_ctas", 152) or 152, "panel": t.get("fp64_panel", 0)}
        work = col.factor_work() if (prec == "mixed" and col_cfg["bcr"]) else None
        results[prec] = dict(ms=ms, steps=steps_done, phases=phases, launches=launches, info=info, graphs=graphs,
                             start_state=start_state, start_dt=start_dt, K=K,
                             ms_traced=ms_traced, steps_traced=max(int(info_traced.steps), 1),
                             col=col if prec == "mixed" else None, col_cfg=col_cfg, work=work)
        if prec == "fp64":
            del col
            torch.cuda.empty_cache()

    mixed = results["mixed"]
    fp64 = results["fp64"]
    S, L = prob.S, prob.L
    value, ms_step = whole_job_rate(mixed["ms"] / mixed["steps"], ws, dev)
    fp64_value, fp64_ms_step = whole_job_rate(fp64["ms"] / fp64["steps"], ws, dev)
    a7_flops = 8.0 / 3.0 * S ** 3 * L            # LU + Schur work of block Thomas per step (the survey's count)

    def per_launch(ph, name):
        ms_, calls = ph.get(name, (0.0, 0))
        return ms_ / max(calls, 1), calls

    def rooflines(res):
        """Per-kernel rooflines of the mixed step's FP32 factorization and the FP64 one."""
        ph = res["phases"]
        steps = res["steps"]
        out = {}
        if res["work"]:
            mma, leaf = res["work"]
            tc_ms, tc_calls = ph["tc"]
            lf_ms, lf_calls = ph["leaf"]
            nfac = max(ph["factor"][1], 1)            # factorizations timed
            tc_s = tc_ms / nfac * 1e-3
            lf_s = lf_ms / nfac * 1e-3
            ach = 3.0 * mma / tc_s / 1e12            # the tensor pipe executes head x head, head x tail, tail x head
            out["tc"] = {"kernel": "k_tc_gemm (tcgen05 kind::tf32, head/tail split)", "bound": "tensor",
                         "achieved": ach, "peak": derived["tf32"], "unit": "TFLOP/s", "frac": ach / derived["tf32"],
                         "peak_kind": derived["kind"] + " (tf32 1.1 / bf16 2.25)",
                         "peak_live_tf32_matmul": live["tf32"], "frac_of_live": ach / live["tf32"],
                         "useful_tflops": mma / tc_s / 1e12, "flops_per_factorization": mma,
                         "ms_per_factorization": tc_s * 1e3, "launches_per_factorization": tc_calls / nfac,
                         "ms_per_step": tc_ms / steps, "traffic": 5.011e6,
                         "traffic_launch": "one 72-tile launch (A and B operands first touched from DRAM)",
                         "traffic_source": "profiles/k_tc_gemm_594x150.txt"}
            ach = leaf / lf_s / 1e12
            out["leaf"] = {"kernel": "k_leaf_inverse (FP32 Gauss-Jordan, partial pivoting, one CTA per block)",
                           "bound": "alu", "achieved": ach, "peak": derived["f32"], "unit": "TFLOP/s",
                           "frac": ach / derived["f32"], "peak_kind": derived["kind"],
                           "peak_live_f32_matmul": live["f32"], "flops_per_factorization": leaf,
                           "ms_per_factorization": lf_s * 1e3, "launches_per_factorization": lf_calls / nfac,
                           "ms_per_step": lf_ms / steps, "traffic": 7.843e6,
                           "traffic_launch": "one level-0 launch of 75 blocks of 160 (7.68 MB algorithmic read)",
                           "traffic_source": "profiles/k_leaf_inverse_594x150.txt"}
        fac_ms, fac_calls = per_launch(ph, "factor")
        out["a7"] = {"flops_per_factorization": a7_flops, "ms_per_factorization": fac_ms,
                     "tflops": a7_flops / (fac_ms * 1e-3) / 1e12,
                     "note": "8/3 S^3 L (block Thomas LU + Schur) over the whole FP32 factorization phase"}
        return out

    def roofline_fp64(res):
        ph = res["phases"]
        fac_ms, fac_calls = per_launch(ph, "factor")
        avg_s = fac_ms * 1e-3
        flops = 2.0 * S ** 3 * L + 3.0 * S * S * (L - 1)     # Gauss-Jordan inversions + Schur updates
        achieved = flops / avg_s / 1e12
        cfg = res["col_cfg"]
        twisted = int(cfg["twisted"] and not cfg["panel"] and L >= 3)
        key = ("fp64", cfg["ctas"], cfg["nb"], cfg["panel"], twisted)
        traffic, source = PROFILED_TRAFFIC.get(key, (None, None))
        return {"kernel": f"k_factor<double, {cfg['nb']}>" + (" (two grid halves, then the middle layer)" if twisted else ""),
                "bound": "alu", "achieved": achieved, "peak": live["f64"], "unit": "TFLOP/s",
                "frac": achieved / live["f64"], "peak_kind": "FP64 matmul measured live (torch.matmul float64)",
                "peak_derived": derived["f64"], "flops_per_factorization": flops,
                "a7_survey_tflops": a7_flops / avg_s / 1e12, "ms_per_factorization": avg_s * 1e3,
                "traffic": traffic, "traffic_source": source}

    roof = rooflines(mixed)
    dom = max((k for k in ("tc", "leaf") if k in roof), key=lambda k: roof[k]["ms_per_step"], default=None)

    # end to end through the C-ABI with host buffers, over the same K steps as the timed region (same
    # starting state and dt): the state from pinned host memory in, one step, the state back into
    # pinned host memory, every step
    col = mixed["col"]
    n_host = torch.empty((L, S), dtype=torch.float64, pin_memory=True)
    n_host.copy_(torch.from_numpy(mixed["start_state"]))
    Ke = mixed["K"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = 0
    for i in range(Ke):
        col.set_state(n_host)
        col.step(mixed["start_dt"] if i == 0 else 0.0)
        col.get_state(out=n_host)
        e2e_steps += 1
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = _max_over_ranks(e2e_s, ws, dev)
    col.close()
    del col
    mixed["col"] = None
    torch.cuda.empty_cache()

    cpu = errs = steady = None
    if rank == 0 and ws == 1:
        if not args.no_cpu:
            t = oracle_sample_step_time(prob, SAMPLE_LAYERS, 1)[0]
            rate, cores, wall = oracle_all_cores(L)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"one implicit step on a {SAMPLE_LAYERS}-layer slice of the {L}-layer column per "
                             f"process, {cores} processes at once ({wall:.1f} s), as full-column steps/s",
                   "single_core": {"value": 1.0 / (t * L / SAMPLE_LAYERS), "cores": 1,
                                   "sample": f"one step on {SAMPLE_LAYERS} of {L} layers ({t:.1f} s), "
                                             f"scaled by {L}/{SAMPLE_LAYERS}"}}
            errs = err_vs_oracle(prob, tuning)
            # the error leg runs the oracle's step on the whole 150-layer column once: its time is the
            # unscaled single-core figure (rates, Jacobian, block solve and its refinement)
            if errs and errs.get("oracle_step_s"):
                cpu["single_core_full_column"] = {"value": 1.0 / errs["oracle_step_s"], "cores": 1,
                                                  "sample": f"one step of the whole {L}-layer column "
                                                            f"({errs['oracle_step_s']:.1f} s)"}
        if not args.no_steady:
            steady = steady_runs(prob, tuning, {"mixed": args.steady_cap, "fp64": args.steady_cap_fp64,
                                                "mixed_from_equilibrium": args.steady_cap})
    batch = serving_obj = parcel = analysis = radiation = bdf = None
    if rank == 0 and ws == 1:
        if not args.no_batch:
            batch = batch_object(args.columns, steps=5, warmup=3, tune=not args.no_tune)
        if not args.no_serving:
            serving_obj = serving_object(args.requests, args.rate, args.slots, args.serving_deadline)
        if not args.no_parcel:
            parcel = parcel_object(live, cpu=not args.no_cpu)
        if not args.no_analysis:
            analysis = analysis_object(live, cpu=not args.no_cpu)
            radiation = radiation_object(live, cpu=not args.no_cpu)
            bdf = bdf_object(cpu=not args.no_cpu)
    if rank == 0:
        ph = {k: {"ms_total": v[0], "calls": v[1]} for k, v in mixed["phases"].items() if v[1]}
        ph64 = {k: {"ms_total": v[0], "calls": v[1]} for k, v in fp64["phases"].items() if v[1]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": mixed["steps"],
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "species": S, "reactions": prob.R, "layers": L,
                       "precision": "mixed: FP32 factorization (tensor-core block cyclic reduction), "
                                    "FP64 FGMRES on the FP64 operator",
                       "l2": "inputs larger than L2: FP32 blocks 222 MB per step (FP64 433 MB)",
                       "start": "initial state, dt0 1e-8 s, adaptive dt", "parallelism": f"replicas x{ws}",
                       "factorization": tuning, "tuning_ms_per_layer": tables},
            "fp64": {"value": fp64_value, "unit": UNIT, "ms_per_step": fp64_ms_step,
                     "steps": fp64["steps"], "speedup_mixed_over_fp64": fp64_ms_step / ms_step},
            "roofline": roof.get(dom) if dom else roof["a7"],
            "rooflines": roof,
            "roofline_fp64": roofline_fp64(fp64),
            "peaks": {"measured_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
                      "derived": derived, "live_matmul_tflops": live},
            "phases_ms": ph, "phases_ms_fp64": ph64,
            "solver_iters_per_step": mixed["info"].solver_iters / mixed["steps"],
            "fp64_fallback_steps": int(mixed["info"].fp64_steps),
            "err_vs_oracle": errs,
            "steady": steady,
            "cpu_baseline": cpu,
            "e2e": {"value": ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": L * S * 8,
                    "d2h_bytes_per_step": L * S * 8},
            "gpu_launches": int(mixed["launches"]),
            "graph_launches": int(mixed["graphs"]),
            "batch": batch,
            "serving": serving_obj,
            "parcel": parcel,
            "analysis": analysis,
            "radiation": radiation,
            "bdf": bdf,
            "traced": {"ms_per_step": mixed["ms_traced"] / mixed["steps_traced"],
                       "note": "the next steps with every kernel launched from the host between CUDA event "
                               "pairs (phases_ms comes from this run)"},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_problems(n=64, seed=0):
    """64 uneven columns: S from {96, 250, 594}, L uniform in 80..200, T_eq U[800, 2500] K."""
    import numpy as np
    from paper_2512_06729_gb300 import synth
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        S = int(rng.choice([96, 250, 594]))
        L = int(rng.integers(80, 201))
        T_eq = float(rng.uniform(800.0, 2500.0))
        out.append(synth.sweep_column(S, L, T_eq, 1.0, 1.0, seed=100 + i))
    return out


def batch_object(columns=64, steps=5, warmup=3, tune=True, budget=200 << 30):
    """Config-3 batch: `columns` uneven columns advanced together, every round (one controlled step
    of every unfinished column) replayed as one CUDA graph with a branch per column.  Returns the
    bench's `batch` object: column-steps/s of the whole batch over `steps` timed rounds."""
    import torch
    from paper_2512_06729_gb300 import autotune
    from paper_2512_06729_gb300 import xk
    probs = batch_problems(columns)
    tuning, tables = {}, {}
    t_tune = time.perf_counter()
    for p in probs:
        if p.S in tuning:
            continue
        if not tune:
            tuning[p.S] = {}
            continue
        got = autotune.tuned(p.S, "mixed")
        if not got:
            got, table = autotune.tune(p, "mixed")
            tables[str(p.S)] = [[params, round(ms, 4)] for ms, params in table]
        tuning[p.S] = got
    t_tune = time.perf_counter() - t_tune
    b = xk.Batch(budget, len(probs))
    cols = []
    footprint = 0
    for p in probs:
        kw = {k: v for k, v in tuning[p.S].items() if k != "factor_ctas"}   # the batch shares the SMs
        c = xk.Column(p, "mixed", reuse_factorization=1, allocate=False, **kw)
        if not b.fits(c.workspace_bytes):
            raise RuntimeError(f"batch budget exhausted at column {len(cols)}")
        c.allocate()
        c.set_mixing_ratios(p.f0)
        assert b.add(c, 1e-8) is not None
        footprint += c.workspace_bytes
        cols.append(c)
    t_cap = time.perf_counter()
    b.step(1)                       # the first round captures the round's graph
    torch.cuda.synchronize()
    t_cap = time.perf_counter() - t_cap
    for _ in range(max(warmup - 1, 0)):
        b.step(1)
    torch.cuda.synchronize()
    n0, g0 = xk.Column.lib_launches(), xk.Column.graph_launches()
    with ClockSampler(0) as cs:
        t0 = time.perf_counter()
        for _ in range(steps):
            b.step(1)
        wall = time.perf_counter() - t0
    launches = xk.Column.lib_launches() - n0
    graphs = xk.Column.graph_launches() - g0
    done = sum(1 for i in range(len(cols)) if b.poll(i)[1])
    sizes = {}
    for p in probs:
        sizes[str(p.S)] = sizes.get(str(p.S), 0) + 1
    b.close()
    for c in cols:
        c.close()
    del cols
    torch.cuda.empty_cache()
    col_steps = len(probs) * steps
    return {
        "metric": f"column-steps/s, {len(probs)} uneven columns (S in {{96, 250, 594}}, L 80..200) on one GPU",
        "value": col_steps / wall, "unit": "column-steps/s", "rounds": steps, "warmup": warmup,
        "ms_per_round": wall * 1e3 / steps, "columns": len(probs), "species_counts": sizes,
        "layers_total": int(sum(p.L for p in probs)), "footprint_gb": footprint / 1e9,
        "precision": "mixed (FP32 factorization, FP64 FGMRES, FP64 reuse)",
        "graph_launches_per_round": graphs / steps, "kernel_nodes_per_round": launches / steps,
        "first_round_s_with_capture": t_cap, "tune_s": t_tune, "finished_columns": done,
        "factorization": {str(k): v for k, v in tuning.items()}, "tuning_ms_per_layer": tables or None,
        "clocks": cs.summary(),
    }


def run_batch(args):
    """Batched uneven columns: column-steps/s of the whole batch (mixed precision)."""
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    obj = batch_object(args.columns, args.steps, args.warmup, tune=not args.no_tune)
    line = {"metric": obj["metric"], "value": obj["value"], "unit": obj["unit"], "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": obj["ms_per_round"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "batch-64-uneven"}, "batch": obj,
            "gpu_launches": int(obj["kernel_nodes_per_round"] * args.steps), "clocks": obj["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def serving_object(requests=16, rate=0.25, slots=16, deadline=120.0, precisions=("mixed", "fp64"), seed=0,
                   equilibrium=True):
    """Config-4 serving: Poisson-arriving steady-state requests from the planet-parameter sweep
    (60/30/10 % of 96/250/594 species on 150 layers), admitted by HBM footprint and kept on the
    device, served once by the mixed path and once by the plain FP64 path on the same requests.
    Returns the bench's `serving` object (p50/p99 time to steady state of the finished requests,
    solves/s, and how many did not finish before the deadline)."""
    import torch
    from paper_2512_06729_gb300 import serving
    reqs = serving.sweep_requests(requests, rate, seed=seed)
    reqs_eq = serving.sweep_requests(requests, rate, seed=seed, initial="equilibrium")
    out = {"requests": requests, "rate_per_s": rate, "slots": slots, "deadline_s": deadline, "layers": 150,
           "species": [r.problem.S for r in reqs]}
    runs = [(prec, prec, reqs) for prec in precisions]
    if equilibrium and "mixed" in precisions:
        # the same sweep started from the chemical-equilibrium composition (Sec. 2.5 option (i))
        runs.append(("mixed_from_equilibrium", "mixed", reqs_eq))
    for name, prec, rq in runs:
        kw = dict(reuse_factorization=1) if prec == "mixed" else {}
        srv = serving.Server(200 << 30, slots, precision=prec, chunk=8, column_kw=kw)
        t0 = time.perf_counter()
        res = srv.run(rq, deadline=deadline)
        wall = time.perf_counter() - t0
        srv.close()
        torch.cuda.empty_cache()
        summ = serving.summarize(res, wall)
        summ["wall_s"] = wall
        summ["unfinished"] = summ["requests"] - summ["finished"]
        summ["per_request"] = [{"S": q.problem.S, "arrival_s": round(x.arrival, 3),
                                "latency_s": None if x.finished is None else round(x.latency, 3),
                                "steps": x.steps, "fp64_steps": x.fp64_steps} for q, x in zip(rq, res)]
        out[name] = summ
    if "mixed" in out and "fp64" in out:
        fm, ff = out["mixed"]["solves_per_s"], out["fp64"]["solves_per_s"]
        out["solves_per_s_mixed_over_fp64"] = fm / ff if ff > 0 else None
    return out


def run_serving(args):
    """Continuous batching of steady-state requests from a planet-parameter sweep."""
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    obj = serving_object(args.requests, args.rate, args.slots, args.time_limit,
                         precisions=tuple(args.variants.split(",")))
    first = obj[args.variants.split(",")[0]]
    line = {
        "metric": "serving: time to steady state p50/p99 (s) and solves/s, sweep requests 60/30/10 % of 96/250/594 sp",
        "value": first["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": first["steps_total"],
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic", "config": {"workload": "serving-sweep"}, "serving": obj,
    }
    print(json.dumps(line), flush=True)
    return 0


def parcel_object(live, iterations=3, cpu=True, columns=152):
    """The paper's Lagrangian parcel scheme (Sec. 2, Fig. 2) on the 96-species, 150-layer column:
    device time of a global iteration (one CTA sweeps the parcel bottom to top and back, an FP64
    partial-pivot LU per implicit step), after one untimed iteration from the initial state; the
    oracle's time for the same first iteration on one host core, and the element-wise error of
    that iteration against it; then `columns` copies of the column swept at once, one CTA each on
    its own stream (iterations/s of the whole GPU)."""
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import synth, xk
    prob = synth.chons_column()
    S, L = prob.S, prob.L
    col = xk.Column(prob, "fp64")
    col.set_mixing_ratios(prob.f0)
    n0 = col.get_state()
    first = col.parcel_iteration(h=1e-8)
    n1 = col.get_state()
    h = first.h
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 0
    ms = 0.0
    for _ in range(iterations):
        torch.cuda.synchronize()
        start.record(stream)
        info = col.parcel_iteration(h=h)
        end.record(stream)
        torch.cuda.synchronize()
        ms += start.elapsed_time(end)
        h = info.h
        steps += int(info.steps + info.rejected)
    ms_it = ms / iterations
    steps_it = steps / iterations
    # FP64 work of one implicit step: elimination 2/3 S^3 plus the two triangular solves 2 S^2
    flops_step = 2.0 / 3.0 * S ** 3 + 2.0 * S ** 2
    achieved = flops_step * steps_it / (ms_it * 1e-3) / 1e12
    peak_sm = live["f64"] / 152.0
    out = {
        "workload": f"{S} species x {L} layers, {2 * L - 1} visits per global iteration",
        "iterations_per_s": 1e3 / ms_it, "ms_per_iteration": ms_it, "implicit_steps_per_iteration": steps_it,
        "first_iteration": {"steps": int(first.steps), "rejected": int(first.rejected),
                            "max_change": float(first.max_change)},
        "roofline": {"kernel": "k_parcel_iteration (one CTA, FP64 Gaussian elimination per implicit step)",
                     "bound": "alu", "achieved": achieved, "peak": peak_sm, "unit": "TFLOP/s",
                     "frac": achieved / peak_sm,
                     "peak_kind": "FP64 matmul measured live / 152 SMs (the sweep is sequential: one SM)"},
    }
    col.close()
    # many parcels at once: one column per SM, each on its own stream (the sweep of one column is
    # sequential, so throughput comes from independent columns, one CTA each)
    if columns > 0:
        streams = [torch.cuda.Stream() for _ in range(columns)]
        cols = []
        for st in streams:
            cc = xk.Column(prob, "fp64", stream=st)
            cc.set_mixing_ratios(prob.f0)
            cols.append(cc)
        for cc in cols:
            cc.parcel_begin(h=1e-8)
        firsts = [cc.parcel_end() for cc in cols]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for cc, fi in zip(cols, firsts):
            cc.parcel_begin(h=fi.h)
        seconds = [cc.parcel_end() for cc in cols]
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        steps_all = sum(int(x.steps + x.rejected) for x in seconds)
        ach = flops_step * steps_all / wall / 1e12
        out["columns_at_once"] = {
            "columns": columns, "iterations_per_s": columns / wall, "wall_s": wall,
            "roofline": {"bound": "alu", "achieved": ach, "peak": live["f64"], "unit": "TFLOP/s",
                         "frac": ach / live["f64"], "peak_kind": "FP64 matmul measured live (whole GPU)"},
            "note": "the second global iteration of each column, all columns begun before any is awaited"}
        for cc in cols:
            cc.close()
        del cols
        torch.cuda.empty_cache()
    if cpu:
        from oracle.oracle import Oracle
        o = Oracle(prob)
        t0 = time.perf_counter()
        N, oi = o.parcel_iteration(n0, h=1e-8)
        dt = time.perf_counter() - t0
        ngas = o.grid()[0]
        keep = N > 1e-20 * ngas[:, None]
        out["cpu_oracle_first_iteration_s"] = dt
        # the sweep's own sensitivity: the oracle from the same state perturbed by 1e-13 relative
        Np, pi = o.parcel_iteration(n0 * (1.0 + 1e-13 * np.random.default_rng(7).standard_normal(n0.shape)), h=1e-8)
        out["gpu_vs_oracle_first_iteration"] = {
            "max_rel": float(np.max(np.abs(n1[keep] - N[keep]) / N[keep])),
            "median_rel": float(np.median(np.abs(n1[keep] - N[keep]) / N[keep])),
            "steps_equal": bool(oi.steps == first.steps and oi.rejected == first.rejected),
            "oracle_vs_itself_perturbed_1e-13": {
                "max_rel": float(np.max(np.abs(Np[keep] - N[keep]) / N[keep])),
                "median_rel": float(np.median(np.abs(Np[keep] - N[keep]) / N[keep])),
                "steps_equal": bool(oi.steps == pi.steps and oi.rejected == pi.rejected)}}
    return out


def run_parcel(args):
    """The parcel-scheme object alone (the command the parcel kernel's profile runs)."""
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    out = parcel_object(live_peaks(), iterations=max(args.steps, 1), cpu=not args.no_cpu)
    print(json.dumps({"mode": "parcel", "parcel": out}), flush=True)
    return 0


def analysis_object(live, calls=5, cpu=True, sources=8):
    """Equilibrium initial state (Sec. 2.5) and reaction-pathway analyser (Sec. 4) on the
    594-species, 7,720-reaction, 150-layer column from its initial state: device time of one
    equilibrium solve of all layers (one CTA per layer) and of Dijkstra searches from `sources`
    species in every layer (one warp each), each the mean of `calls` calls after one untimed call;
    errors against the oracle (equilibrium: every layer; pathways: bitwise on the oracle's rates)."""
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import synth, xk
    prob = synth.full_column()
    S, L, E, R = prob.S, prob.L, prob.E, prob.R
    col = xk.Column(prob, "fp64")
    col.set_mixing_ratios(prob.f0)
    n0 = col.get_state(device=True)
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(calls):
            res = fn()
        end.record(stream)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / calls, res

    ms_eq, (x, info) = timed(lambda: col.equilibrium())
    # FP64 work per Newton iteration and layer: the system's sparse sums (a multiply-add per species
    # and pair of its elements, three flops per species and element for the two element sums), the
    # species' potentials and updates (a multiply-add per element), and the totals
    ne = np.count_nonzero(prob.elem, axis=1).astype(float)
    flops_it = L * (2.0 * np.sum(ne * (ne + 1) / 2) + 3.0 * np.sum(ne) + 2.0 * np.sum(ne) + 6.0 * S)
    ach = flops_it * info.iters_max / (ms_eq * 1e-3) / 1e12
    src = list(range(2, 2 + sources))
    q = col.reaction_fluxes(n0)
    ms_path, out = timed(lambda: col.pathways(q, src))
    edges = sum(len({a for a in (prob.reac[r] if d == 0 else prob.prod[r]) if a >= 0}) *
                len({a for a in (prob.prod[r] if d == 0 else prob.reac[r]) if a >= 0}) for r in range(R) for d in (0, 1)
                if not (d == 1 and prob.rtype[r] == synth.RX_PHOTO))
    res = {
        "workload": f"{S} species x {R} reactions x {L} layers, initial state",
        "equilibrium": {"ms_per_call": ms_eq, "layers_per_s": L / (ms_eq * 1e-3),
                        "newton_iters_max": int(info.iters_max),
                        "roofline": {"kernel": "k_equilibrium (one CTA per layer)", "bound": "alu",
                                     "achieved": ach, "peak": live["f64"], "unit": "TFLOP/s",
                                     "frac": ach / live["f64"],
                                     "peak_kind": "FP64 matmul measured live; the solve is latency-bound "
                                                  "(150 CTAs, a barrier-separated chain per Newton iteration)"}},
        "pathways": {"sources": sources, "searches": sources * L, "ms_per_call": ms_path,
                     "searches_per_s": sources * L / (ms_path * 1e-3), "edges_per_layer": edges,
                     "edge_relaxations_per_s": sources * L * edges / (ms_path * 1e-3)},
    }
    if cpu:
        from oracle.oracle import Oracle
        o = Oracle(prob)
        nh = n0.cpu().numpy()
        t0 = time.perf_counter()
        ref, _, _ = o.equilibrium(o.element_totals(nh))
        res["equilibrium"]["cpu_oracle_s"] = time.perf_counter() - t0
        xg = x.cpu().numpy()
        m = ref > 1e-250
        res["equilibrium"]["err_vs_oracle"] = {"max_rel": float(np.max(np.abs(xg[m] - ref[m]) / ref[m])),
                                               "species_compared": int(m.sum())}
        qo = o.fluxes(nh)
        got = col.pathways(torch.as_tensor(qo, device=q.device), src[:1])
        d = got["dist"].cpu().numpy()
        pe = got["pred_edge"].cpu().numpy()
        same, t_cpu = True, 0.0
        for k in (0, L // 2, L - 1):
            t0 = time.perf_counter()
            r = o.pathways(qo[k], src[0])
            t_cpu += time.perf_counter() - t0
            same &= bool(np.array_equal(r["dist"], d[0, k]) and np.array_equal(r["pred_edge"], pe[0, k]))
        res["pathways"]["bitwise_equal_to_oracle"] = same
        res["pathways"]["cpu_oracle_s_per_search"] = t_cpu / 3
    col.close()
    return res


def run_analysis(args):
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    out = analysis_object(live_peaks(), calls=max(args.steps, 1), cpu=not args.no_cpu)
    print(json.dumps({"mode": "analysis", "analysis": out}), flush=True)
    return 0


def radiation_object(live, calls=5, cpu=True):
    """Photolysis rates with the extinction and diffuse field of Sec. 2.3.3 on the 594-species,
    150-layer column: the 1,000-bin direct beam of the headline workload beside Rayleigh scattering
    plus the two-stream diffuse field on the paper's 10,000-bin grid (1-10,000 A).  Device time of
    one evaluation (extinction sums, beam and diffuse recursion, rate integrals), mean of `calls`
    after one untimed call; the FP64 work of the two contractions (extinction sum_i sigma_i n_i per
    layer and bin, and sum_w J sigma dlambda per layer and reaction) over that time; error against
    the oracle on every rate."""
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import synth, xk
    out = {}
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, prob in (("direct_1000", synth.full_column()),
                       ("scattering_diffuse_10000", synth.with_scattering(synth.full_column(), bins=10000))):
        col = xk.Column(prob, "fp64")
        col.set_mixing_ratios(prob.f0)
        n = col.get_state(device=True)
        col.eval_photolysis(n)
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(calls):
            kph = col.eval_photolysis(n)
        end.record(stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end) / calls
        S, L, W, Rph = prob.S, prob.L, prob.W, prob.Rph
        n_abs = int(np.count_nonzero(np.any(prob.sigma_abs != 0, axis=1)))
        n_sca = 0 if prob.sigma_s is None else int(np.count_nonzero(np.any(prob.sigma_s != 0, axis=1)))
        flops = 2.0 * L * W * (n_abs + n_sca) + 3.0 * L * Rph * W
        ach = flops / (ms * 1e-3) / 1e12
        o = {"bins": W, "absorbers": n_abs, "scatterers": n_sca, "diffuse": int(prob.diffuse),
             "ms_per_evaluation": ms,
             "roofline": {"kernels": "k_photo_alpha + k_photo_J + k_photo_k", "bound": "alu", "achieved": ach,
                          "peak": live["f64"], "unit": "TFLOP/s", "frac": ach / live["f64"],
                          "peak_kind": "FP64 matmul measured live; work = the two FP64 contractions"}}
        if cpu:
            from oracle.oracle import Oracle
            nh = n.cpu().numpy()
            t0 = time.perf_counter()
            ref = Oracle(prob).photolysis(nh)
            o["cpu_oracle_s"] = time.perf_counter() - t0
            g = kph.cpu().numpy()
            m = ref > 1e-300
            o["err_vs_oracle_max_rel"] = float(np.max(np.abs(g[m] - ref[m]) / ref[m]))
        out[name] = o
        col.close()
    # one linear step of the mixed path with the direct beam's rates differentiated (photo_jacobian:
    # FGMRES on the fully coupled operator, the block-tridiagonal factorization as preconditioner)
    # beside the same step with lagged rates
    prob = synth.full_column()
    steps = {}
    for flag in (0, 1):
        col = xk.Column(prob, "mixed", photo_jacobian=flag)
        col.set_mixing_ratios(prob.f0)
        n = col.get_state(device=True)
        col.step_delta(n, 1e-2)
        torch.cuda.synchronize()
        start.record(stream)
        d, iters, res = col.step_delta(n, 1e-2)
        end.record(stream)
        torch.cuda.synchronize()
        steps["coupled" if flag else "lagged"] = {"ms": start.elapsed_time(end), "fgmres_iters": int(iters),
                                                  "residual": float(res)}
        col.close()
    out["step_photo_jacobian_594"] = dict(steps, dt_s=1e-2)
    return out


def run_radiation(args):
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    out = radiation_object(live_peaks(), calls=max(args.steps, 1), cpu=not args.no_cpu)
    print(json.dumps({"mode": "radiation", "radiation": out}), flush=True)
    return 0


def bdf_object(attempts=40, cpu=True):
    """The variable-order BDF integrator (the DLSODES family of Sec. 2.1) from the initial state:
    wall time per attempt on the 594-species, 150-layer column (mixed precision; every attempt is
    one block-tridiagonal solve plus the predictor and error kernels, synchronised with the host
    controller), the orders it reaches, and on the 96-species column the end state after the same
    number of attempts against the oracle's BDF."""
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import synth, xk
    out = {}
    prob = synth.full_column()
    col = xk.Column(prob, "mixed")
    col.set_mixing_ratios(prob.f0)
    col.bdf_run(h0=1e-8, max_steps=3)                      # warm-up (rates, plans)
    col.set_mixing_ratios(prob.f0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, rc = col.bdf_run(h0=1e-8, max_steps=attempts, rtol=1e-3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out["full_mixed"] = {"attempts": int(info.steps), "accepted": int(info.accepted), "rejected": int(info.rejected),
                         "order_steps": [int(x) for x in info.order_steps], "t_reached_s": info.t,
                         "ms_per_attempt": 1e3 * wall / max(int(info.steps), 1),
                         "solver_iters": int(info.solver_iters)}
    # the same from the chemical-equilibrium initial state (Sec. 2.5 option (i)) of the same elements
    col.set_mixing_ratios(prob.f0)
    col.equilibrium(set_state=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, rc = col.bdf_run(h0=1e-8, max_steps=attempts, rtol=1e-3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out["full_mixed_from_equilibrium"] = {"attempts": int(info.steps), "accepted": int(info.accepted),
                                          "order_steps": [int(x) for x in info.order_steps], "t_reached_s": info.t,
                                          "ms_per_attempt": 1e3 * wall / max(int(info.steps), 1)}
    col.close()
    small = synth.chons_column()
    c2 = xk.Column(small, "fp64")
    c2.set_mixing_ratios(small.f0)
    n0 = c2.get_state()
    gi, _ = c2.bdf_run(h0=1e-8, max_steps=attempts, rtol=1e-3)
    res = {"attempts": int(gi.steps), "order_steps": [int(x) for x in gi.order_steps], "t_reached_s": gi.t}
    if cpu:
        from oracle.oracle import Oracle
        o = Oracle(small)
        t0 = time.perf_counter()
        ref, ri, _ = o.bdf_run(n0, h0=1e-8, max_steps=attempts, rtol=1e-3)
        res["cpu_oracle_s"] = time.perf_counter() - t0
        ngas = o.grid()[0]
        g = c2.get_state()
        keep = ref > 1e-20 * ngas[:, None]
        res["same_steps_as_oracle"] = bool(ri.steps == gi.steps and ri.accepted == gi.accepted
                                           and list(ri.order_steps) == list(gi.order_steps))
        res["err_vs_oracle_max_rel"] = float(np.max(np.abs(g[keep] - ref[keep]) / ref[keep]))
    out["chons_fp64"] = res
    c2.close()
    return out


def run_extras(args):
    """The analysis and radiation objects in one process (the command behind their kernel profiles)."""
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    live = live_peaks()
    out = {"analysis": analysis_object(live, calls=max(args.steps, 1), cpu=not args.no_cpu),
           "radiation": radiation_object(live, calls=max(args.steps, 1), cpu=not args.no_cpu)}
    print(json.dumps({"mode": "extras", **out}), flush=True)
    return 0


def run_bdf(args):
    from paper_2512_06729_gb300 import build as xkbuild
    xkbuild.build()
    out = bdf_object(attempts=max(args.steps, 1), cpu=not args.no_cpu)
    print(json.dumps({"mode": "bdf", "bdf": out}), flush=True)
    return 0


def run_steady(args):
    """Time to steady state of the 594 x 150 column: mixed path (FP64 factorization reused as the
    FGMRES preconditioner once steps go to FP64) against the plain FP64 path, the two end states
    compared, and the oracle's own linear step at the FP64 end state as a check of the fixed point."""
    import numpy as np
    import torch
    from paper_2512_06729_gb300 import build as xkbuild
    from paper_2512_06729_gb300 import synth, xk
    xkbuild.build()
    prob = synth.full_column()
    stream = torch.cuda.current_stream()
    runs = {}
    extra = json.loads(args.column_kw) if args.column_kw else {}
    variants = {"mixed": ("mixed", dict(reuse_factorization=1, **extra)), "fp64": ("fp64", {}),
                "mixed_from_equilibrium": ("mixed", dict(reuse_factorization=1, **extra))}
    for name in args.variants.split(","):
        prec, kw = variants[name]
        col = xk.Column(prob, prec, **kw)
        col.set_mixing_ratios(prob.f0)
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        t0 = time.perf_counter()
        if name.endswith("_from_equilibrium"):
            col.equilibrium(set_state=True)   # the chemical-equilibrium start (Sec. 2.5 option (i)), timed
        steps = acc = fp64_steps = iters = refactors = 0
        t_model = 0.0
        info = None
        # in chunks, so that a run that would exceed the time limit stops and reports how far it got
        while steps < args.max_steps and time.perf_counter() - t0 < args.time_limit:
            info = col.run_to_steady(1e-8 if steps == 0 else 0.0, min(50, args.max_steps - steps))
            steps += int(info.steps)
            acc += int(info.accepted)
            fp64_steps += int(info.fp64_steps)
            iters += int(info.solver_iters)
            refactors += int(info.refactors)
            t_model += float(info.t)            # each call starts its model clock at 0
            if info.converged or info.steps == 0:
                break
        end.record(stream)
        torch.cuda.synchronize()
        runs[name] = dict(s=start.elapsed_time(end) / 1e3, wall=time.perf_counter() - t0, steps=steps,
                          accepted=acc, converged=int(info.converged), t_model=t_model, dt=float(info.dt),
                          fp64_steps=fp64_steps, refactors=refactors, iters=iters, n=col.get_state())
        col.close()
        del col
        torch.cuda.empty_cache()
    rel = None
    if "mixed" in runs and "fp64" in runs:
        nm, nf = runs["mixed"]["n"], runs["fp64"]["n"]
        ng = nf.sum(axis=1)
        keep = nf > 1e-20 * ng[:, None]
        rel = float(np.max(np.abs(nm - nf)[keep] / nf[keep]))
    check = None
    nf = runs["fp64"]["n"] if "fp64" in runs else next(iter(runs.values()))["n"]
    if not args.no_cpu and any(r["converged"] for r in runs.values()):
        from oracle.oracle import Oracle
        o = Oracle(prob)
        ong = o.grid()[0]
        t0 = time.perf_counter()
        d = o.step_delta(nf, 1e8)
        s = np.maximum(nf, 1e-20 * ong[:, None])
        okeep = nf > 1e-20 * ong[:, None]
        check = {"oracle_step_max_rel_change": float(np.max(np.abs(d)[okeep] / s[okeep])),
                 "steady_tol": 1e-3, "oracle_s": time.perf_counter() - t0}
    first = next(iter(runs.values()))
    line = {
        "metric": "time to steady state (s), 594 sp x 150 layers, mixed (FP64 reuse) vs FP64",
        "value": first["s"] if first["converged"] else None, "unit": "s", "n_gpus": 1, "steps": first["steps"],
        "warmup": 0, "ms_per_step": first["s"] * 1e3 / max(first["steps"], 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "species": prob.S, "reactions": prob.R, "layers": prob.L,
                   "start": "initial state, dt0 1e-8 s", "steady": "dt >= 1e8 s and max relative change < 1e-3"},
        "runs": {k: {kk: vv for kk, vv in v.items() if kk != "n"} for k, v in runs.items()},
        "mixed_vs_fp64_max_rel": rel,
        "oracle_check": check,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_kernels(args):
    """Linear steps (rates to solve, no step control) of one precision on the 594 x 150 column at
    library defaults: per-phase device times for the rooflines, and a short command to profile."""
    import torch
    from paper_2512_06729_gb300 import build as xkbuild
    from paper_2512_06729_gb300 import synth, xk
    xkbuild.build()
    prob = synth.full_column()
    col = xk.Column(prob, args.precision)
    col.set_mixing_ratios(prob.f0)
    n = col.get_state(device=True)
    for _ in range(args.warmup):
        col.step_delta(n, args.dt)
    col.profile(True)
    n0 = xk.Column.lib_launches()
    iters = []
    for _ in range(args.steps):
        iters.append(col.step_delta(n, args.dt)[1])
    torch.cuda.synchronize()
    ph = col.profile_read()
    line = {"mode": "kernels", "precision": args.precision, "dt": args.dt, "steps": args.steps,
            "launches": xk.Column.lib_launches() - n0, "solver_iters": iters,
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in ph.items()},
            "phase_calls": {k: v[1] for k, v in ph.items()}}
    print(json.dumps(line), flush=True)
    col.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle legs (baseline, error vs oracle)")
    ap.add_argument("--no-steady", action="store_true", help="skip the time-to-steady-state runs")
    ap.add_argument("--steady-cap", type=float, default=300.0, help="seconds allowed to the mixed run to steady state")
    ap.add_argument("--steady-cap-fp64", type=float, default=60.0,
                    help="seconds allowed to the plain FP64 run to steady state")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch object of the default line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving object of the default line")
    ap.add_argument("--no-parcel", action="store_true", help="skip the parcel-scheme object of the default line")
    ap.add_argument("--no-analysis", action="store_true",
                    help="skip the equilibrium and pathway-analyser object of the default line")
    ap.add_argument("--serving-deadline", type=float, default=75.0,
                    help="seconds each serving run (mixed, then FP64) may take in the default line")
    ap.add_argument("--no-tune", action="store_true",
                    help="library defaults instead of the autotuned factorization (shorter runs for profiling)")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serving", "steady", "kernels", "parcel", "analysis", "radiation", "bdf", "extras"],
                    help="step: one 594 x 150 column (the headline); batch: 64 uneven columns; serving: sweep "
                         "requests; steady: time to steady state of the 594 x 150 column")
    ap.add_argument("--max-steps", type=int, default=5000)
    ap.add_argument("--variants", default="mixed,fp64", help="--mode steady / serving: paths to run, in order")
    ap.add_argument("--time-limit", type=float, default=600.0,
                    help="--mode steady: seconds per path; --mode serving: deadline of the serving loop")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="--mode kernels")
    ap.add_argument("--dt", type=float, default=1e-2, help="--mode kernels: step size of the linear steps")
    ap.add_argument("--columns", type=int, default=64)
    ap.add_argument("--column-kw", default="", help="--mode steady: JSON of extra config fields of the mixed path")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--rate", type=float, default=0.25)
    ap.add_argument("--slots", type=int, default=16)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serving":
        return run_serving(args)
    if args.mode == "steady":
        return run_steady(args)
    if args.mode == "kernels":
        return run_kernels(args)
    if args.mode == "parcel":
        return run_parcel(args)
    if args.mode == "analysis":
        return run_analysis(args)
    if args.mode == "radiation":
        return run_radiation(args)
    if args.mode == "bdf":
        return run_bdf(args)
    if args.mode == "extras":
        return run_extras(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
