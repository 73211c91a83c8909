"""Host logic of the serving loop with a fake batch (no GPU): admission in
arrival order by footprint and slots, retirement when finished, latency
accounting."""
import types

import numpy as np

from paper_2512_06729_gb300 import serving


ALLOCATED = []
STARTS = []


class FakeColumn:
    def __init__(self, prob, precision, device=0, allocate=True, **kw):
        self.prob = prob
        self.workspace_bytes = prob.S * 100
        self.bytes = self.workspace_bytes
        self.closed = False
        self.allocated = False
        if allocate:
            self.allocate()

    def allocate(self):
        self.allocated = True
        ALLOCATED.append(self.prob.name)

    def set_mixing_ratios(self, f):
        self.start = "user"

    def equilibrium(self, set_state=False):
        assert self.allocated and self.start == "user"      # after the workspace and the user state
        if set_state:
            self.start = "equilibrium"
        STARTS.append(self.prob.name)
        return None, None

    def get_state(self):
        return np.zeros((1, 1))

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self, budget, slots, device=0):
        self.budget, self.slots, self.used = budget, slots, 0
        self.active = {}
        self.admissions = []

    def fits(self, nbytes):
        return len(self.active) < self.slots and self.used + nbytes <= self.budget

    def add(self, col, dt0=1e-8):
        assert col.allocated
        if not self.fits(col.bytes):
            return None
        slot = min(set(range(self.slots)) - set(self.active))
        self.active[slot] = [col, 0]
        self.used += col.bytes
        self.admissions.append(col.prob.name)
        return slot

    def step(self, n):
        for v in self.active.values():
            v[1] += n

    def submit(self, slot, n):
        self.active[slot][1] += n

    def query(self, slot):
        return True

    def poll(self, slot):
        col, steps = self.active[slot]
        need = col.prob.S // 10          # fake work: proportional to the size
        info = types.SimpleNamespace(steps=steps, converged=steps >= need, fp64_steps=0)
        return info, steps >= need, 0

    def remove(self, slot):
        col, _ = self.active.pop(slot)
        self.used -= col.bytes
        return col

    def close(self):
        pass


def test_admission_order_budget_and_latency(monkeypatch):
    monkeypatch.setattr(serving.xk, "Column", FakeColumn)
    monkeypatch.setattr(serving.xk, "Batch", FakeBatch)
    probs = [types.SimpleNamespace(name=f"r{i}", S=s, f0=None) for i, s in enumerate([40, 80, 40, 120, 40])]
    reqs = [serving.Request(i, 0.0, p) for i, p in enumerate(probs)]
    t = [0.0]

    def clock():
        t[0] += 0.001
        return t[0]

    srv = serving.Server(budget_bytes=16000, max_slots=2, chunk=2)
    ALLOCATED.clear()
    res = srv.run(reqs, clock=clock)
    # arrival order is kept; never more than 2 slots or 16000 bytes at once
    assert srv.batch.admissions == ["r0", "r1", "r2", "r3", "r4"]
    # a workspace is allocated only for a column the batch admits: once per request
    assert ALLOCATED == ["r0", "r1", "r2", "r3", "r4"]
    assert all(r.converged for r in res)
    assert all(r.finished > r.admitted >= r.arrival for r in res)
    s = serving.summarize(res, t[0])
    assert s["requests"] == 5 and s["p99_s"] >= s["p50_s"]


def test_sweep_requests_shape():
    import paper_2512_06729_gb300.synth as synth
    calls = []

    def fake_sweep(S, L, T_eq, met, kzz, seed):
        calls.append((S, L, T_eq, met, kzz))
        return types.SimpleNamespace(S=S)

    orig = synth.sweep_column
    synth.sweep_column = fake_sweep
    try:
        reqs = serving.sweep_requests(400, rate=10.0, seed=1)
    finally:
        synth.sweep_column = orig
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert abs(arr[-1] / 400 - 0.1) < 0.02                 # mean inter-arrival 1 / rate
    sizes = np.array([c[0] for c in calls])
    assert abs((sizes == 96).mean() - 0.6) < 0.08 and abs((sizes == 594).mean() - 0.1) < 0.05
    T = np.array([c[2] for c in calls])
    assert T.min() >= 800 and T.max() <= 2500
    met = np.array([c[3] for c in calls])
    assert met.min() >= 1 and met.max() <= 100


def test_deadline_reports_unfinished(monkeypatch):
    """With a deadline the loop stops there: finished requests keep their
    latency, active and waiting ones are returned unfinished, and the summary
    counts only the finished ones."""
    monkeypatch.setattr(serving.xk, "Column", FakeColumn)
    monkeypatch.setattr(serving.xk, "Batch", FakeBatch)
    probs = [types.SimpleNamespace(name=f"r{i}", S=s, f0=None) for i, s in enumerate([40, 10 ** 6, 40, 40])]
    reqs = [serving.Request(i, 0.0, p) for i, p in enumerate(probs)]
    t = [0.0]

    def clock():
        t[0] += 0.001
        return t[0]

    srv = serving.Server(budget_bytes=10 ** 9, max_slots=1, chunk=2)
    res = srv.run(reqs, clock=clock, deadline=0.5)
    assert res[0].finished is not None and res[0].converged
    assert res[1].finished is None and res[1].admitted is not None     # the long one was running
    assert res[2].finished is None and res[2].admitted is None         # never admitted
    s = serving.summarize(res, t[0])
    assert s["requests"] == 4 and s["finished"] == 1


def test_equilibrium_start_is_set_before_admission(monkeypatch):
    """A request marked to start from the equilibrium composition gets it on the device after its
    workspace exists and before the batch admits it; the others keep their mixing ratios."""
    monkeypatch.setattr(serving.xk, "Column", FakeColumn)
    monkeypatch.setattr(serving.xk, "Batch", FakeBatch)
    probs = [types.SimpleNamespace(name=f"r{i}", S=40, f0=None) for i in range(4)]
    reqs = [serving.Request(i, 0.0, p, initial="equilibrium" if i % 2 else "user") for i, p in enumerate(probs)]
    t = [0.0]

    def clock():
        t[0] += 0.001
        return t[0]

    STARTS.clear()
    srv = serving.Server(budget_bytes=10 ** 9, max_slots=2, chunk=2)
    res = srv.run(reqs, clock=clock)
    assert STARTS == ["r1", "r3"]
    assert all(r.converged for r in res)
