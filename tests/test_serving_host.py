"""Host logic of the continuous-batching server, on the CPU: the admission loop, budget
accounting, chunking and retirement run against a stand-in for the library (simulations
that only count their steps, batches that enforce the C library's budget rule and report
completion at once).  Every request must be served exactly once with its own step count,
the resident bytes must stay within the budget except for a lone oversize request, and the
loop must end."""
import threading

import pytest

from paper_2002_09217_gb300 import inputs, serving


class FakeSim:
    def __init__(self, w, precision):
        self.nodes = w.nodes
        self.precision = precision
        self.steps = 0
        self.flags = []
        self.closed = False

    def device_bytes(self):
        return serving.footprint_bytes(self.nodes, self.precision)

    def init_fields(self, *fields):
        pass

    def moments(self):
        return {"steps": self.steps}

    def stats(self):
        return {"steps": self.steps, "nonfinite": 0}

    def get_state(self):
        return None

    def close(self):
        self.closed = True


class FakeBatch:
    """Budget rule of pond_batch_add: refuse a member that would exceed the budget unless
    the batch is empty."""

    def __init__(self, stream=None):
        self.members = []
        self.budget = 0

    def set_budget(self, nbytes):
        self.budget = nbytes

    def add(self, sim):
        used = sum(m.device_bytes() for m in self.members)
        if self.budget and self.members and used + sim.device_bytes() > self.budget:
            raise FakePond.PondError(2, "over budget")
        self.members.append(sim)

    def remove(self, sim):
        self.members.remove(sim)

    def step(self, n):
        for m in self.members:
            m.steps += n

    def poll(self):
        return True

    def synchronize(self):
        pass

    def close(self):
        self.members = []


class FakePond:
    class PondError(RuntimeError):
        def __init__(self, status, msg):
            super().__init__(msg)
            self.status = status

    Batch = FakeBatch

    @staticmethod
    def from_workload(w, precision="mixed", stream=None):
        return FakeSim(w, precision)


class FakeStream:
    def __init__(self, priority=0):
        self.priority = priority


@pytest.fixture
def server_cls(monkeypatch):
    import torch
    monkeypatch.setattr(serving, "pond", FakePond)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    return serving.Server


def _run(server, reqs, timeout=60.0):
    out = {}

    def target():
        out["results"] = server.run(reqs, time_scale=0.0)

    t = threading.Thread(target=target, daemon=True)
    t.start()
    t.join(timeout)
    assert not t.is_alive(), "the serving loop did not end"
    return out["results"]


@pytest.mark.parametrize("budget_mib", [16, 256, 4096])
def test_every_request_is_served_once_with_its_own_steps(server_cls, budget_mib):
    reqs = inputs.serving_requests(n=40, rate=100.0)
    server = server_cls(hbm_budget=budget_mib << 20, chunk=37)
    res = _run(server, reqs)
    assert sorted(r.rid for r in res) == sorted(r.rid for r in reqs)
    want = {r.rid: r.steps for r in reqs}
    for r in res:
        assert r.fields["steps"] == want[r.rid] == r.steps
    assert server.refused == 0
    biggest = max(serving.footprint_bytes(r.side * r.side, r.precision) for r in reqs)
    assert server.peak_bytes <= max(budget_mib << 20, biggest)


def test_request_larger_than_the_budget_runs_alone(server_cls):
    reqs = inputs.serving_requests(n=6, rate=100.0)
    server = server_cls(hbm_budget=1 << 20, chunk=500)   # smaller than any request
    res = _run(server, reqs)
    assert len(res) == len(reqs)
    assert server.peak_bytes == max(serving.footprint_bytes(r.side * r.side, r.precision) for r in reqs)
