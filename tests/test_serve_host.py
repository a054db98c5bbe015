"""Host-side tests of the continuous-batching server with a fake solver factory:
budget and slot admission, first-come-first-served order, overlap, latency
accounting (no GPU)."""
import math

import pytest

from paper_1403_1661_gb300.serve import Request, Server


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeJob:
    def __init__(self, clock, req, rounds_per_step):
        self.clock = clock
        self.macro_period = 4
        self.busy_until = 0.0
        self.steps = 0
        self.dt = rounds_per_step

    def step(self, n):
        self.steps += n
        self.busy_until = self.clock() + self.dt * n

    def idle(self):
        self.clock.t += 1e-4        # the host loop itself takes time
        return self.clock() >= self.busy_until

    def finish(self):
        return None, 100 * self.steps


class FakeFactory:
    def __init__(self, clock, sizes, step_time):
        self.clock = clock
        self.sizes = sizes
        self.step_time = step_time
        self.started = []

    def prepare(self, req):
        return {"bytes": self.sizes[req.rid]}

    def bytes(self, prep):
        return prep["bytes"]

    def start(self, req, prep):
        self.started.append(req.rid)
        return FakeJob(self.clock, req, self.step_time)


def _run(sizes, arrivals, budget, slots, substeps=40, step_time=10.0):
    # fake device time per macro step is large against the host loop's own time,
    # so admission order does not depend on how fast the preparation threads run
    clock = FakeClock()
    fac = FakeFactory(clock, sizes, step_time)
    srv = Server(budget_bytes=budget, max_slots=slots, macro_per_round=2, prep_workers=1, factory=fac,
                 clock=clock, sleep=clock.sleep)
    reqs = [Request(rid=i, arrival=a, scenario=None, substeps=substeps) for i, a in enumerate(arrivals)]
    return srv, fac, srv.run(reqs)


def test_all_requests_finish_fifo_within_budget():
    sizes = [30, 50, 40, 10, 60, 20]
    srv, fac, out = _run(sizes, [0.0, 0.01, 0.02, 0.03, 0.04, 0.05], budget=100, slots=3)
    assert out["requests"] == 6
    assert fac.started == sorted(fac.started)            # first come, first served
    assert out["peak_bytes"] <= 100
    assert out["peak_running"] <= 3
    for r in out["done"]:
        assert r.admitted >= r.arrival and r.finished > r.admitted
        assert r.dof_updates == 100 * math.ceil(40 / 4)
    lat = sorted(r.finished - r.arrival for r in out["done"])
    assert out["p50_s"] <= out["p99_s"] <= lat[-1] + 1e-12


def test_work_overlaps_when_memory_allows():
    # four equal requests arriving together: with room for all they finish together
    _, _, wide = _run([10] * 4, [0.0] * 4, budget=1000, slots=8)
    _, _, narrow = _run([10] * 4, [0.0] * 4, budget=10, slots=8)
    assert wide["peak_running"] == 4 and narrow["peak_running"] == 1
    assert wide["wall_s"] < 0.5 * narrow["wall_s"]


def test_request_over_budget_is_rejected():
    with pytest.raises(MemoryError):
        _run([10, 500], [0.0, 0.0], budget=100, slots=2)
