"""Continuous batching of steady-state solves on one GPU.

Requests (one atmospheric column each) arrive over time; the server admits
them into an xk batch as slots and HBM budget free up, advances every active
column together (their work overlaps on the device), retires the ones that
reach steady state and admits waiting ones between batch steps.  Columns keep
their state on the device from admission to retirement.  Reports the time to
steady state of every request (completion minus arrival), p50/p99 and solves/s.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import synth, xk


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    problem: synth.Problem
    dt0: float = 1e-8
    initial: str = "user"       # "user": the problem's mixing ratios; "equilibrium": the chemical-
                                # equilibrium composition of the same elements (Sec. 2.5 option (i)),
                                # computed on the device at admission


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float | None      # None: never admitted before the deadline
    finished: float | None      # None: not finished before the deadline
    converged: bool
    steps: int
    fp64_steps: int
    state: np.ndarray | None

    @property
    def latency(self):
        return self.finished - self.arrival


def sweep_requests(n, rate, seed=0, mix=((96, 0.6), (250, 0.3), (594, 0.1)), layers=150, initial="user"):
    """Poisson arrivals (rate per second) from a planet-parameter sweep:
    T_eq U[800, 2500] K, metallicity log-U[1, 100] x solar, Kzz scale
    log-U[1e6, 1e11] / 1e8 (the profile's Kzz is 1e7 .. 1e10 cm^2/s), and the
    species mix 60 / 30 / 10 % of 96 / 250 / 594-species networks."""
    rng = np.random.default_rng(seed)
    sizes = np.array([m[0] for m in mix])
    probs = np.array([m[1] for m in mix], float)
    probs /= probs.sum()
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        S = int(rng.choice(sizes, p=probs))
        T_eq = rng.uniform(800.0, 2500.0)
        met = 10.0 ** rng.uniform(0.0, 2.0)
        kzz = 10.0 ** rng.uniform(6.0, 11.0) / 1e8
        prob = synth.sweep_column(S, layers, T_eq, met, kzz, seed=1000 + i)
        out.append(Request(i, t, prob, initial=initial))
    return out


class Server:
    """Admission by HBM footprint into a fixed number of slots; each admitted
    column gets `chunk` controlled steps at a time on its own stream, the next
    chunk as soon as the previous one has run, so that small columns are not
    paced by large ones."""

    def __init__(self, budget_bytes, max_slots, precision="mixed", device=0, chunk=4, max_steps=4000,
                 keep_states=False, column_kw=None):
        import torch
        self.torch = torch
        self.batch = xk.Batch(budget_bytes, max_slots, device)
        self.precision = precision
        self.device = device
        self.chunk = chunk
        self.max_steps = max_steps
        self.keep_states = keep_states
        self.column_kw = column_kw or {}
        self.budget = budget_bytes

    def run(self, requests, clock=None, deadline=None):
        """Serve all requests; arrival times are honoured against a wall clock
        that starts now.  Returns the list of Results in request order; with a
        deadline (seconds) the loop stops there and the requests not finished
        by then are returned with finished=None."""
        clock = clock or time.perf_counter
        t0 = clock()
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting = []
        active = {}            # slot -> (request, column, admitted time)
        inflight = set()       # slots with submitted steps not yet seen done
        results = {}
        while pending or waiting or active:
            now = clock() - t0
            if deadline is not None and now >= deadline:
                for slot in list(active):
                    req, col, adm = active.pop(slot)
                    while slot in inflight and not self.batch.query(slot):
                        time.sleep(0.0005)
                    inflight.discard(slot)
                    info, _, _ = self.batch.poll(slot)
                    self.batch.remove(slot)
                    results[req.rid] = Result(req.rid, req.arrival, adm, None, False, int(info.steps),
                                              int(info.fp64_steps), None)
                    col.close()
                for req in waiting + pending:
                    results[req.rid] = Result(req.rid, req.arrival, None, None, False, 0, 0, None)
                break
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # admit in arrival order while slots and budget allow: the footprint is checked against
            # the batch before the column's workspace is allocated
            while waiting:
                req = waiting[0]
                col = xk.Column(req.problem, self.precision, device=self.device, allocate=False, **self.column_kw)
                if not self.batch.fits(col.workspace_bytes):
                    col.close()
                    del col
                    break
                col.allocate()
                col.set_mixing_ratios(req.problem.f0)
                if req.initial == "equilibrium":
                    col.equilibrium(set_state=True)
                slot = self.batch.add(col, req.dt0)
                if slot is None:
                    col.close()
                    del col
                    break
                waiting.pop(0)
                active[slot] = (req, col, clock() - t0)
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - (clock() - t0))))
                continue
            # every column advances at its own pace: a slot whose last chunk has run gets the next
            for slot in active:
                if slot not in inflight:
                    self.batch.submit(slot, self.chunk)
                    inflight.add(slot)
            progressed = False
            for slot in list(active):
                if not self.batch.query(slot):
                    continue
                inflight.discard(slot)
                progressed = True
                info, finished, status = self.batch.poll(slot)
                if finished or info.steps >= self.max_steps:
                    req, col, adm = active.pop(slot)
                    self.batch.remove(slot)
                    state = col.get_state() if self.keep_states else None
                    results[req.rid] = Result(req.rid, req.arrival, adm, clock() - t0, bool(info.converged),
                                              int(info.steps), int(info.fp64_steps), state)
                    col.close()
                    del col
            if not progressed:
                time.sleep(0.0005)
        return [results[r.rid] for r in requests]

    def close(self):
        self.batch.close()


def summarize(results, wall):
    done = [r for r in results if r.finished is not None]
    lat = np.array([r.latency for r in done]) if done else np.array([np.nan])
    return {
        "requests": len(results),
        "finished": len(done),
        "converged": int(sum(r.converged for r in results)),
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "solves_per_s": len(done) / wall,
        "steps_total": int(sum(r.steps for r in results)),
        "fp64_steps_total": int(sum(r.fp64_steps for r in results)),
    }
