"""Batched scenarios (one graph launch advances many solvers) and the launch-shape
autotuner. Argument marshalling only: the work runs in the native library."""
from __future__ import annotations

import contextlib
import ctypes as C
import hashlib
import json
import os
import tempfile
import time

import numpy as np

from . import _native as nat
from .build import BUILD
from .solver import own_stream, release_stream


class Batch:
    """Many independent solvers advanced together: per (tier, order) group one
    persistent kernel over a device ticket queue, one CUDA-graph replay per step."""

    def __init__(self, solvers, stream=None, max_macro=8):
        import torch
        self.solvers = list(solvers)
        if not self.solvers:
            raise ValueError("empty batch")
        self.max_macro = int(max_macro)
        dev = self.solvers[0].device
        n = len(self.solvers)
        handles = (C.c_void_p * n)(*[s.handle.value for s in self.solvers])
        nbytes = C.c_size_t()
        nat.check(nat.lib().swe_batch_workspace_bytes(handles, n, self.max_macro, C.byref(nbytes)),
                  "swe_batch_workspace_bytes")
        self._own_stream = None
        with torch.cuda.device(dev):
            self.stream = own_stream(self) if stream is None else stream
            self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        with torch.cuda.device(dev):
            nat.check(nat.lib().swe_batch_create(handles, n, self.max_macro, C.c_void_p(self.workspace.data_ptr()),
                                                 self.workspace.numel(), C.c_void_p(self.stream.cuda_stream),
                                                 C.byref(h)), "swe_batch_create")
        self.handle = h
        self.last_status = np.zeros(n, np.int32)

    def step(self, n_macro=1, check=True):
        """Advance every solver by n_macro macro steps (an int, or one count per
        solver). Returns the per-solver status codes of the last batch step; with
        check, a timed-out solver raises."""
        n = len(self.solvers)
        counts = np.broadcast_to(np.asarray(n_macro, np.int32), (n,)).copy()
        status = np.zeros(n, np.int32)
        while counts.max(initial=0) > 0:
            now = np.minimum(counts, self.max_macro).astype(np.int32)
            rc = nat.lib().swe_batch_step(self.handle, nat.iptr(now), nat.iptr(status))
            if rc not in (nat.SWE_OK, nat.SWE_ETIMEOUT):
                nat.check(rc, "swe_batch_step")
            counts -= now
            if rc == nat.SWE_ETIMEOUT:
                break
        self.last_status = status
        if check and (status != nat.SWE_OK).any():
            raise nat.SWEError(int(status[status != nat.SWE_OK][0]), "swe_batch_step")
        return status

    def set_wait_limit(self, seconds):
        nat.check(nat.lib().swe_batch_set_wait_limit(self.handle, float(seconds)), "swe_batch_set_wait_limit")

    def hold(self, i, hold=True):
        nat.check(nat.lib().swe_batch_hold(self.handle, int(i), 1 if hold else 0), "swe_batch_hold")

    def launches(self):
        v = C.c_int64()
        nat.check(nat.lib().swe_batch_launches(self.handle, C.byref(v)), "swe_batch_launches")
        return v.value

    def close(self):
        if getattr(self, "handle", None):
            nat.lib().swe_batch_destroy(self.handle)
            self.handle = None
            self.workspace = None
        release_stream(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autotuner: launch shapes per (order, precision, GPU) -- CTAs per SM of the
# grid-stride kernels and, on the tensor-core tier, warps per CTA of the
# tensor-core stage and batch kernels

CACHE = os.path.join(BUILD, "autotune.json")
CTAS = (1, 2, 3, 4, 0)            # CTAs per SM (0 = as many as fit)
TC_WARPS = (2, 3, 4, 5, 6, 7, 8)  # warps per CTA of the tensor-core kernels


def candidates_for(precision):
    """Every launch shape the tuner tries: (ctas_per_sm, tc_warps), tc_warps None
    off the tensor-core tier."""
    if precision == "fp32tc":
        return tuple((c, w) for w in TC_WARPS for c in CTAS)
    return tuple((c, None) for c in CTAS)


def _gpu_key():
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def _sources_key():
    """Hash of the native sources: a cached shape is used only with the kernels it
    was measured on."""
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".inc", ".hpp", ".cpp")):
            h.update(f.encode())
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:       # absent, or unreadable: tune again
        return {}


def _store_cache(cache):
    """Write the cache by an atomic rename, so a concurrent reader never sees a
    partial file (a concurrent writer may drop the other's entry: it is re-tuned)."""
    d = os.path.dirname(CACHE)
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune.", suffix=".json")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(cache, f, indent=1, default=str)
        os.replace(tmp, CACHE)
    except BaseException:
        with contextlib.suppress(OSError):
            os.unlink(tmp)
        raise


def tune(N, precision, candidates=None, reps=3, force=False, verbose=False):
    """Time one macro step of a seeded sample problem of order N (an 80,000-triangle
    beach, 4 levels) for every candidate launch shape and return the fastest as
    {"ctas_per_sm": c, "tc_warps": w}. Shapes that do not fit on an SM are skipped.
    Only a search over the full candidate set reads or writes the cache, so a
    narrower search never stands in for it; a cached shape is used only with the
    native sources it was measured on."""
    import torch
    from workloads import scenarios as sc
    from .solver import solver_from_scenario
    full_set = candidates_for(precision)
    cands = full_set if candidates is None else tuple(candidates)
    key = f"{_gpu_key()}/N{N}/{precision}/shape"
    full = cands == full_set
    src = _sources_key()
    cache = _load_cache()
    hit = cache.get(key)
    if full and not force and isinstance(hit, dict) and hit.get("sources") == src:
        return dict(hit["shape"])
    s = solver_from_scenario(sc.tsunami(nx=400, ny=100, N=N, nlevels=4), precision=precision)
    timings = {}
    try:
        for c, w in cands:
            try:
                s.set_launch_config({"ctas_per_sm": c, "tc_warps": w})
            except nat.SWEError as ex:
                if ex.code == nat.SWE_EINVAL:     # that many warps' tiles do not fit on an SM
                    continue
                raise
            s.step(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.step(reps)
            e1.record(s.stream)
            torch.cuda.synchronize()
            timings[(c, w)] = e0.elapsed_time(e1) / reps
    finally:
        s.close()
    if not timings:
        raise ValueError(f"tune: none of the launch shapes {cands} fits order {N} on this GPU")
    c, w = min(timings, key=timings.get)
    best = {"ctas_per_sm": c, "tc_warps": w}
    if full:
        cache = _load_cache()            # re-read: another process may have added entries
        cache[key] = {"shape": best, "ms_per_macro_step": {f"{k[0]}/{k[1]}": v for k, v in timings.items()},
                      "sources": src, "when": time.time()}
        _store_cache(cache)
    if verbose:
        print(f"autotune {key}: {timings} -> {best}")
    return best


def apply_tuning(solver, precision):
    """Set the cached (or freshly tuned) launch shape on a solver."""
    best = tune(solver.N, precision)
    solver.set_launch_config(best)
    return best
