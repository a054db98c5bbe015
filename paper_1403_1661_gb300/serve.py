"""Continuous-batching server for tsunami-scenario solves.

Requests (a scenario and a number of finest MRAB substeps) arrive over time.
Host-side preparation (mesh, connectivity, nodal inputs, level grouping) runs on
a thread pool; a request is admitted, first come first served, as soon as its
device workspace fits in the HBM budget and a slot is free. Every admitted solve
keeps its state and Adams-Bashforth history resident in its own workspace and
advances on its own CUDA stream a few macro steps at a time (graph replays), so
the work of all running requests overlaps on the GPU. Finished requests return
their state to the host and free their memory immediately, which admits the next
ones. Latency is completion time minus arrival time. Optionally (GpuFactory's
regroup_every) each solve is regrouped into CFL levels every few macro steps, the
remedy Section 4 gives for levels that no longer fit the state.

Solves never interact (no shared buffers, deterministic kernels), so a result
does not depend on what else is running.

Failures stay with their request: a request whose preparation fails (an invalid
mesh, say) or whose workspace exceeds the whole budget is rejected, one whose
solver cannot be created fails, and a running solve whose state turned
non-finite (the device flag that swe_stats reports, checked every few rounds
while the solve is idle and again before its result is returned), or whose step,
check or read-back raises, is stopped and fails; its memory is released and the
others carry on. If the loop itself is left by an exception, every solve it had
created is closed before the exception propagates. A request can be
cancelled from any thread (Server.cancel) or at a scripted time
(Request.cancel_at): one that has not started is dropped, a running one is
retired at its next idle point without a result.
"""
from __future__ import annotations

import collections
import contextlib
import concurrent.futures as cf
import dataclasses
import math
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    scenario: object
    substeps: int = 500
    admitted: float | None = None
    finished: float | None = None
    dof_updates: int = 0
    bytes: int = 0
    result: object = None
    cancel_at: float | None = None   # cancel at this many seconds after the start (scripted clients)
    status: str = "waiting"          # then "done", "rejected", "failed" or "cancelled"
    error: str | None = None


class GpuFactory:
    """Builds real solvers (used by the server; tests may pass a fake).

    regroup_every: every this many macro steps (0: never) a running solve is
    regrouped into MRAB levels by the CFL rule at its current state (Section 4:
    elements may be regrouped every few steps), keeping its history; if an
    element's CFL step has fallen below the finest step dt_min, the solve restarts
    its levels from its current state instead (a new dt_min, history from AB1). A
    solve whose shoreline layers speed up then stays within its CFL bound instead of
    outrunning the levels it was given at t = 0."""

    def __init__(self, precision="fp32tc", keep_state=False, tuned=None, regroup_every=0):
        self.precision = precision
        self.keep_state = keep_state
        self.tuned = tuned or {}
        self.regroup_every = int(regroup_every)

    def prepare(self, req):
        from .solver import Mesh, scenario_inputs
        from . import _native as nat
        import ctypes as C
        scn = req.scenario
        vx, vy, E = scn.build_mesh()
        mesh = Mesh(vx, vy, E)
        B, h, hu, hv = scenario_inputs(scn, mesh)
        lev, dtm = mesh.levels(scn.N, h, hu, hv, scn.g, scn.cfl, scn.nlevels)
        prm = nat.swe_params(scn.g, scn.h0, 0.0, scn.tvb_M, scn.tvb_nu, scn.cfl, scn.N, scn.nlevels,
                             {"fp64": 0, "fp32": 1, "fp32tc": 2}[self.precision], scn.limiter_mask,
                             scn.dry_mode, nat.SWE_SCHEME_CUBATURE)
        nb = C.c_size_t()
        nat.check(nat.lib().swe_workspace_bytes(mesh.handle, C.byref(prm), C.byref(nb)), "swe_workspace_bytes")
        return {"mesh": mesh, "inputs": (B, h, hu, hv), "levels": (lev, dtm), "bytes": int(nb.value) + 256}

    def bytes(self, prepared):
        return prepared["bytes"]

    def start(self, req, prepared):
        return _GpuJob(self, req, prepared)


class _GpuJob:
    def __init__(self, factory, req, prepared):
        import torch
        from .solver import Solver
        scn = req.scenario
        self.factory = factory
        self.s = Solver(prepared["mesh"], scn.N, g=scn.g, h0=scn.h0, cfl=scn.cfl, nlevels_max=scn.nlevels,
                        precision=factory.precision, limiter_mask=scn.limiter_mask, tvb_M=scn.tvb_M,
                        tvb_nu=scn.tvb_nu, dry_mode=scn.dry_mode)
        try:
            if scn.N in factory.tuned:
                self.s.set_launch_config(factory.tuned[scn.N])
            B, h, hu, hv = prepared["inputs"]
            lev, dtm = prepared["levels"]
            self.s.set_bathymetry(B)
            self.s.set_levels(lev, dtm)      # before the state: no re-ordering of uploaded data
            self.s.set_state(h, hu, hv)
        except BaseException:
            self.s.close()                   # a failed start gives its workspace back at once
            raise
        L = int(np.max(lev))
        self.macro_period = 2 ** (L - 1)
        self.substeps_left = int(req.substeps)   # finest substeps still to take
        self.event = torch.cuda.Event()
        self.pending = False
        self.since_regroup = 0      # macro steps since the last regroup
        self.since_restart = 0      # macro steps since the levels were last set up
        self.regroups = 0
        self.restarts = 0

    def remaining_macro(self):
        return -(-self.substeps_left // self.macro_period)

    def step(self, n):
        every = self.factory.regroup_every
        # a regroup needs three Adams-Bashforth values of every level since the last restart
        if every and self.since_regroup >= every and self.since_restart >= 3:
            _, margin = self.s.regroup()
            self.regroups += 1
            self.since_regroup = 0
            if margin < 1.0:
                self.s.setup_levels()
                self.restarts += 1
                self.since_restart = 0
                self.macro_period = 2 ** (self.s.level_info()[0] - 1)
            n = min(n, self.remaining_macro())
        self.s.step(n)
        self.substeps_left -= n * self.macro_period
        self.since_regroup += n
        self.since_restart += n
        self.event.record(self.s.stream)
        self.pending = True

    def idle(self):
        return (not self.pending) or self.event.query()

    def healthy(self):
        """False once the device has flagged a non-finite value (call when idle)."""
        return not self.s.stats()["nonfinite"]

    def finish(self):
        try:
            st = self.s.stats()
            out = self.s.get_state() if self.factory.keep_state else None
        finally:
            self.s.close()
        return out, st["dof_updates"]

    def abort(self):
        self.s.close()


class Server:
    def __init__(self, budget_bytes=150e9, max_slots=64, macro_per_round=2, prep_workers=4, factory=None,
                 clock=time.perf_counter, sleep=time.sleep, health_every=16, start_workers=0):
        self.budget = float(budget_bytes)
        self.max_slots = int(max_slots)
        self.macro_per_round = int(macro_per_round)
        self.prep_workers = int(prep_workers)
        # start_workers > 0: admitted solves are created (device workspace, inputs,
        # levels) on that many threads, so the loop that issues the running solves'
        # steps never waits for a creation; 0 creates them in the loop itself
        self.start_workers = int(start_workers)
        self.factory = factory if factory is not None else GpuFactory()
        self.clock = clock
        self.sleep = sleep
        self.health_every = int(health_every)    # rounds of a solve between non-finite checks
        self._cancel = set()
        self._lock = threading.Lock()

    def cancel(self, rid):
        """Cancel request ``rid`` (callable from any thread, before or during run)."""
        with self._lock:
            self._cancel.add(rid)

    def _cancelled(self, r, now):
        if r.cancel_at is not None and now >= r.cancel_at:
            return True
        with self._lock:
            return r.rid in self._cancel

    def run(self, requests):
        """Serve the requests (sorted by arrival); returns a summary dict. Latencies
        and throughput count the completed requests; the others are listed with
        their status and error under "ended"."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque(reqs)
        preparing = collections.deque()          # (req, future) in arrival order
        ready = collections.deque()               # (req, prepared), FIFO
        starting = collections.deque()            # (req, future of the job), admitted
        running = []                              # [req, job, remaining_macro, rounds]
        used = 0.0
        peak_used = 0.0
        peak_running = 0
        done = []
        ended = []
        t0 = self.clock()

        def end(r, status, error=None):
            r.status, r.error = status, error
            r.finished = self.clock() - t0
            ended.append(r)

        def admit(r, job):
            r.admitted = self.clock() - t0
            running.append([r, job, int(math.ceil(r.substeps / job.macro_period)), 0])

        def drop(r, job, status, error=None):
            """Retire a running solve without a result and give its memory back."""
            nonlocal used
            try:
                job.abort()
            except Exception as ex:
                error = f"{error}; abort failed: {ex}" if error else f"abort failed: {ex}"
            used -= r.bytes
            end(r, status, error)

        def release_all():
            """On leaving the loop by an exception: close the solves still running and
            those whose creation had finished (the pools have shut down by then)."""
            for item in running:
                with contextlib.suppress(Exception):
                    item[1].abort()
            for _, fut in starting:
                if fut.done() and not fut.cancelled() and fut.exception() is None:
                    with contextlib.suppress(Exception):
                        fut.result().abort()

        with contextlib.ExitStack() as pools:   # both pools shut down however the loop ends
            pools.callback(release_all)          # runs last: after the pools' shutdown
            pool = pools.enter_context(cf.ThreadPoolExecutor(max_workers=self.prep_workers))
            starter = (pools.enter_context(cf.ThreadPoolExecutor(max_workers=self.start_workers))
                       if self.start_workers > 0 else None)
            while pending or preparing or ready or starting or running:
                now = self.clock() - t0
                progressed = False
                while pending and pending[0].arrival <= now:
                    r = pending.popleft()
                    if self._cancelled(r, now):
                        end(r, "cancelled")
                    else:
                        preparing.append((r, pool.submit(self.factory.prepare, r)))
                    progressed = True
                while preparing and preparing[0][1].done():
                    r, fut = preparing.popleft()
                    progressed = True
                    try:
                        prep = fut.result()
                    except Exception as ex:          # e.g. an invalid mesh
                        end(r, "rejected", f"preparation failed: {ex}")
                        continue
                    r.bytes = self.factory.bytes(prep)
                    if r.bytes > self.budget:
                        end(r, "rejected", f"needs {r.bytes} B, over the whole budget of {self.budget:.0f} B")
                        continue
                    ready.append((r, prep))
                if any(self._cancelled(r, now) for r, _ in ready):
                    keep = collections.deque()
                    for r, prep in ready:
                        if self._cancelled(r, now):
                            end(r, "cancelled")
                        else:
                            keep.append((r, prep))
                    ready = keep
                    progressed = True
                # admission: first come first served, by budget and slots
                while (ready and len(running) + len(starting) < self.max_slots
                       and used + ready[0][0].bytes <= self.budget):
                    r, prep = ready.popleft()
                    progressed = True
                    if starter is not None:
                        used += r.bytes
                        peak_used = max(peak_used, used)
                        starting.append((r, starter.submit(self.factory.start, r, prep)))
                        continue
                    try:
                        job = self.factory.start(r, prep)
                    except Exception as ex:          # e.g. the device refused the workspace
                        end(r, "failed", f"start failed: {ex}")
                        continue
                    used += r.bytes
                    peak_used = max(peak_used, used)
                    admit(r, job)
                # solves whose creation finished join the running ones, in admission order
                while starting and starting[0][1].done():
                    r, fut = starting.popleft()
                    progressed = True
                    try:
                        job = fut.result()
                    except Exception as ex:
                        used -= r.bytes
                        end(r, "failed", f"start failed: {ex}")
                        continue
                    admit(r, job)
                peak_running = max(peak_running, len(running))
                # issue work and retire finished, failed or cancelled solves
                still = []
                for item in running:
                    r, job, rem, rounds = item
                    try:
                        idle = job.idle()
                    except Exception as ex:          # the solve's stream reported an error
                        drop(r, job, "failed", f"device error: {ex}")
                        progressed = True
                        continue
                    if not idle:
                        still.append(item)
                        continue
                    progressed = True
                    if self._cancelled(r, self.clock() - t0):
                        drop(r, job, "cancelled")
                        continue
                    if hasattr(job, "remaining_macro"):   # the job counts its own substeps
                        rem = item[2] = job.remaining_macro()
                    check = rem == 0 or (self.health_every > 0 and rounds > 0 and rounds % self.health_every == 0)
                    try:
                        ok = not check or getattr(job, "healthy", lambda: True)()
                    except Exception as ex:          # e.g. the device reported an error
                        drop(r, job, "failed", f"health check failed: {ex}")
                        continue
                    if not ok:
                        drop(r, job, "failed", "non-finite state")
                        continue
                    if rem > 0:
                        n = min(rem, self.macro_per_round)
                        try:
                            job.step(n)
                        except Exception as ex:      # e.g. a refused regroup or graph launch
                            drop(r, job, "failed", f"step failed: {ex}")
                            continue
                        item[2] = rem - n
                        item[3] = rounds + 1
                        still.append(item)
                    else:
                        try:
                            r.result, r.dof_updates = job.finish()
                        except Exception as ex:      # finish closes the solve in any case
                            drop(r, job, "failed", f"finish failed: {ex}")
                            continue
                        r.status = "done"
                        r.finished = self.clock() - t0
                        used -= r.bytes
                        done.append(r)
                running = still
                if not progressed:
                    nxt = pending[0].arrival - (self.clock() - t0) if pending else 0.0
                    self.sleep(max(0.0002, min(nxt, 0.002)))
        wall = self.clock() - t0
        lat = np.array([r.finished - r.arrival for r in done]) if done else np.zeros(1)
        dofs = sum(r.dof_updates for r in done)
        count = collections.Counter(r.status for r in ended)
        return {"requests": len(done), "wall_s": wall, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "aggregate_dof_per_s": dofs / wall if wall > 0 else 0.0, "dof_updates": int(dofs),
                "peak_running": peak_running, "peak_bytes": peak_used, "done": done,
                "rejected": count["rejected"], "failed": count["failed"], "cancelled": count["cancelled"],
                "ended": ended}


def requests_from_stream(stream, substeps=500):
    """workloads.scenarios.served_stream() output -> Request list."""
    return [Request(rid=i, arrival=t, scenario=scn, substeps=substeps) for i, (t, scn) in enumerate(stream)]
