"""Host-side tests of the continuous-batching server with a fake solver factory:
budget and slot admission, first-come-first-served order, overlap, latency
accounting, and failures that stay with their request: rejection, a solve whose
state turns non-finite, a failed start, cancellation (no GPU)."""
import math
import threading

from paper_1403_1661_gb300.serve import Request, Server


class FakeClock:
    def __init__(self, limit=1e6):
        self.t = 0.0
        self.limit = limit     # fake seconds: a loop that never drains fails instead of hanging

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt
        if self.t > self.limit:
            raise RuntimeError("fake clock ran past its limit")


class FakeJob:
    def __init__(self, clock, req, rounds_per_step, bad_after=None, raises=None):
        self.clock = clock
        self.macro_period = 4
        self.busy_until = 0.0
        self.steps = 0
        self.dt = rounds_per_step
        self.bad_after = bad_after     # macro steps after which the state is non-finite
        self.raises = raises or {}     # method name -> macro steps after which it raises
        self.aborted = False
        self.health_checks = 0

    def _maybe_raise(self, what):
        if what in self.raises and self.steps >= self.raises[what]:
            raise RuntimeError(f"{what}: launch refused")

    def step(self, n):
        self._maybe_raise("step")
        self.steps += n
        self.busy_until = self.clock() + self.dt * n

    def idle(self):
        self.clock.t += 1e-4        # the host loop itself takes time
        self._maybe_raise("idle")
        return self.clock() >= self.busy_until

    def healthy(self):
        self.health_checks += 1
        self._maybe_raise("healthy")
        return self.bad_after is None or self.steps < self.bad_after

    def finish(self):
        self._maybe_raise("finish")
        return None, 100 * self.steps

    def abort(self):
        self.aborted = True


class FakeFactory:
    def __init__(self, clock, sizes, step_time, bad_prepare=(), bad_start=(), bad_after=None, raises=None):
        self.clock = clock
        self.sizes = sizes
        self.step_time = step_time
        self.started = []
        self.jobs = {}
        self.bad_prepare = set(bad_prepare)
        self.bad_start = set(bad_start)
        self.bad_after = bad_after or {}
        self.raises = raises or {}      # rid -> {method: macro steps after which it raises}

    def prepare(self, req):
        if req.rid in self.bad_prepare:
            raise ValueError("mesh is not conforming")
        return {"bytes": self.sizes[req.rid]}

    def bytes(self, prep):
        return prep["bytes"]

    def start(self, req, prep):
        if req.rid in self.bad_start:
            raise RuntimeError("workspace refused")
        self.started.append(req.rid)
        job = FakeJob(self.clock, req, self.step_time, self.bad_after.get(req.rid), self.raises.get(req.rid))
        self.jobs[req.rid] = job
        return job


def _run(sizes, arrivals, budget, slots, substeps=40, step_time=10.0, cancel_at=None, server_cancel=(),
         health_every=2, start_workers=0, **faults):
    # fake device time per macro step is large against the host loop's own time,
    # so admission order does not depend on how fast the preparation threads run
    clock = FakeClock()
    fac = FakeFactory(clock, sizes, step_time, **faults)
    srv = Server(budget_bytes=budget, max_slots=slots, macro_per_round=2, prep_workers=1, factory=fac,
                 clock=clock, sleep=clock.sleep, health_every=health_every, start_workers=start_workers)
    cancel_at = cancel_at or {}
    reqs = [Request(rid=i, arrival=a, scenario=None, substeps=substeps, cancel_at=cancel_at.get(i))
            for i, a in enumerate(arrivals)]
    for rid in server_cancel:
        srv.cancel(rid)
    return srv, fac, srv.run(reqs)


def _status(out):
    return {r.rid: r.status for r in out["done"] + out["ended"]}


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


def test_request_over_budget_is_rejected_and_the_rest_are_served():
    _, fac, out = _run([10, 500, 20], [0.0, 0.0, 0.0], budget=100, slots=2)
    st = _status(out)
    assert st == {0: "done", 1: "rejected", 2: "done"}
    assert 1 not in fac.started and "over the whole budget" in out["ended"][0].error
    assert out["requests"] == 2 and out["rejected"] == 1


def test_failed_preparation_or_start_stays_with_its_request():
    _, fac, out = _run([10, 10, 10, 10], [0.0] * 4, budget=100, slots=4, bad_prepare={1}, bad_start={2})
    st = _status(out)
    assert st == {0: "done", 1: "rejected", 2: "failed", 3: "done"}
    errs = {r.rid: r.error for r in out["ended"]}
    assert "not conforming" in errs[1] and "workspace refused" in errs[2]
    assert out["failed"] == 1 and out["rejected"] == 1


def test_threaded_start_serves_all_and_keeps_failures_with_their_request():
    # solves created on two threads: admission stays first come first served, a
    # failed creation gives its memory back and the others are served
    _, fac, out = _run([10] * 6, [0.0] * 6, budget=20, slots=3, bad_start={2}, start_workers=2)
    st = _status(out)
    assert st == {0: "done", 1: "done", 2: "failed", 3: "done", 4: "done", 5: "done"}
    assert "workspace refused" in [r.error for r in out["ended"] if r.rid == 2][0]
    assert out["peak_bytes"] <= 20 and out["peak_running"] <= 2
    admitted = [r.admitted for r in sorted(out["done"], key=lambda r: r.rid)]
    assert admitted == sorted(admitted)
    for r in out["done"]:
        assert r.dof_updates == 100 * math.ceil(40 / 4)


def test_nonfinite_solve_is_stopped_and_its_memory_admits_the_next():
    # room for one solve at a time: request 0 goes non-finite after 4 macro steps,
    # is stopped at the next check (every 2 rounds), and request 1 then runs
    _, fac, out = _run([60, 60], [0.0, 0.0], budget=100, slots=2, bad_after={0: 4})
    st = _status(out)
    assert st == {0: "failed", 1: "done"}
    j0 = fac.jobs[0]
    assert j0.aborted and j0.steps < 10 and out["ended"][0].error == "non-finite state"
    assert fac.jobs[1].steps == 10 and not fac.jobs[1].aborted
    assert out["peak_bytes"] <= 100
    assert out["requests"] == 1 and out["dof_updates"] == 1000


def test_health_checked_before_a_result_is_returned():
    # non-finite only after the last macro step: caught by the check at retirement
    _, fac, out = _run([10], [0.0], budget=100, slots=1, bad_after={0: 10}, health_every=0)
    assert _status(out) == {0: "failed"} and fac.jobs[0].steps == 10


def test_cancellation_before_start_and_while_running():
    # request 0 runs alone (budget) and is cancelled mid-run; request 1 waits
    # behind it and is cancelled before it could start; request 2 is cancelled
    # through Server.cancel before the run; request 3 is served
    _, fac, out = _run([60, 60, 10, 10], [0.0, 0.0, 0.0, 0.0], budget=100, slots=4,
                       cancel_at={0: 25.0, 1: 5.0}, server_cancel=(2,))
    st = _status(out)
    assert st == {0: "cancelled", 1: "cancelled", 2: "cancelled", 3: "done"}
    assert 1 not in fac.started and 2 not in fac.started
    assert fac.jobs[0].aborted and 0 < fac.jobs[0].steps < 10
    assert out["cancelled"] == 3 and out["requests"] == 1


def test_cancel_from_another_thread():
    clock = FakeClock()
    fac = FakeFactory(clock, [10, 10], 10.0)
    srv = Server(budget_bytes=100, max_slots=2, macro_per_round=2, prep_workers=1, factory=fac,
                 clock=clock, sleep=clock.sleep)
    th = threading.Thread(target=srv.cancel, args=(1,))
    th.start()
    th.join()
    out = srv.run([Request(rid=i, arrival=0.0, scenario=None, substeps=40) for i in range(2)])
    assert _status(out) == {0: "done", 1: "cancelled"}


def test_step_check_or_readback_error_stays_with_its_request():
    # room for two solves at a time; four of six raise in a different place (a step
    # launch, the stream query, the non-finite check, the final read-back): each of
    # them fails alone and gives its memory back, so the last request is still served
    raises = {1: {"step": 4}, 2: {"finish": 0}, 3: {"healthy": 2}, 4: {"idle": 6}}
    _, fac, out = _run([10] * 6, [0.0] * 6, budget=20, slots=6, raises=raises)
    st = _status(out)
    assert st == {0: "done", 1: "failed", 2: "failed", 3: "failed", 4: "failed", 5: "done"}
    errs = {r.rid: r.error for r in out["ended"]}
    assert errs[1].startswith("step failed") and errs[2].startswith("finish failed")
    assert errs[3].startswith("health check failed") and errs[4].startswith("device error")
    assert all(fac.jobs[i].aborted for i in (1, 2, 3, 4))
    assert not fac.jobs[0].aborted and not fac.jobs[5].aborted
    assert out["peak_bytes"] <= 20 and out["failed"] == 4 and out["requests"] == 2


def test_loop_exception_closes_every_created_solve():
    # the loop is left by an exception (here the host's sleep) while solves run and
    # others are being created on worker threads: every solve created is closed
    clock = FakeClock(limit=25.0)
    fac = FakeFactory(clock, [10] * 8, 10.0)
    srv = Server(budget_bytes=40, max_slots=8, macro_per_round=2, prep_workers=1, factory=fac,
                 clock=clock, sleep=clock.sleep, start_workers=2)
    reqs = [Request(rid=i, arrival=0.0, scenario=None, substeps=40) for i in range(8)]
    try:
        srv.run(reqs)
        raise AssertionError("the run should have raised")
    except RuntimeError as ex:
        assert "past its limit" in str(ex)
    assert len(fac.jobs) >= 4
    assert all(j.aborted for j in fac.jobs.values())
