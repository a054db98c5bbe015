"""Write tests/golden/full_config_oracle.json: the FP64 oracle's results on two
benchmark configurations at their full sizes and full run lengths, too long to
recompute inside a GPU test session (test infrastructure; calls only ``oracle/``
and the seeded input generators in ``workloads/``).

* ``dam_break``: the 20,480-triangle wet/dry dam break (N = 3, [0,20] x [0,2],
  320 x 32 x 2 triangles, positivity-preserving + TVB limiter with M = 0 every
  stage, AB3 single rate at CFL 0.5), 2000 steps. The problem is one-dimensional
  up to the triangulation, so the state is summarised per column of the 320
  square cells (area-weighted averages of the element means of h, hu, hv), plus
  the element means of a seeded sample of elements and the global mass, the
  injected mass of dry resets (Algorithm 3) and the smallest nodal depth seen
  after any step.
* ``dam_break_ulp``: the same run from an initial depth perturbed by one unit in
  the last place (h (1 + 2^-52)): the oracle's own response to a rounding-level
  change, which bounds how closely a differently rounded FP64 implementation can
  follow it through the minmod and wet/dry decisions of 2000 limited steps.
* ``dam_break_ulp32``: the same from an initial depth perturbed by one unit in the
  last place of single precision (h (1 + 2^-23)): the oracle's response to a
  change of the size single-precision storage makes, which bounds how closely the
  FP32 tiers can follow it.
* ``dam_break_noise64`` and ``dam_break_store32``: the same run with the state
  changed after every step by rounding-level amounts, the way an implementation
  that rounds differently (or stores single precision) departs from the oracle at
  every step rather than once: each nodal value multiplied by (1 + d), d uniform in
  [-2^-52, 2^-52] (seeded), respectively rounded to single precision. These bound
  how closely the FP64 and the FP32 tiers can follow the oracle.
* ``tsunami``: the 500,000-triangle sloped-beach run (N = 4, 4 MRAB levels by the
  CFL rule, PP + TVB), 25 macro steps = 200 finest substeps. Summarised by the
  level assignment (counts and a SHA-256 of the per-element levels), dt_min, the
  element means of h, hu, hv and B on seeded samples (uniform, around the source,
  at the shore) and the global mass.

Run: ``python tests/golden/make_full_config_golden.py [dam_break] [dam_break_ulp] [dam_break_ulp32]
[dam_break_noise64] [dam_break_store32] [tsunami]`` (about 7 minutes for each dam-break run and
40 for the tsunami on 8 cores).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import problem  # noqa: E402
from workloads import scenarios as sc  # noqa: E402

OUT = os.path.join(HERE, "full_config_oracle.json")


def element_means(ref, q):
    """Element means of nodal fields (the mass-matrix weights over the reference area)."""
    return [q[c] @ ref.mean_w for c in range(q.shape[0])]


def samples(rng, idx, n):
    idx = np.asarray(idx)
    return np.sort(rng.choice(idx, size=min(n, idx.size), replace=False))


def run_dam_break(perturb=0.0, every_step=None):
    """every_step: None, "noise64" (each nodal value times (1 + d), d uniform in
    [-2^-52, 2^-52], seeded) or "store32" (each nodal value rounded to single
    precision), applied to the state after every step."""
    scn = sc.dam_break()
    if perturb:
        # the same run from an initial depth larger by a relative perturb (one unit in
        # the last place of double or of single precision): how far rounding-level
        # differences carry through 2000 limited steps
        init = scn.init

        def init_ulp(x, y, cx, cy, B):
            h, hu, hv = init(x, y, cx, cy, B)
            return np.asarray(h, np.float64) * (1.0 + perturb), hu, hv
        scn.init = init_ulp
    om, ref, model, integ = problem.build(scn)
    assert om.K == 20480 and integ.L == 1
    mass0 = float(om.area @ (integ.q_end[0] @ ref.mean_w))
    hmin = float(integ.q_end[0].min())
    t0 = time.time()
    rng_step = np.random.Generator(np.random.PCG64(23))
    for _ in range(scn.steps):
        integ.substep()
        if every_step == "noise64":
            integ.q_end = integ.q_end * (1.0 + rng_step.uniform(-2.0 ** -52, 2.0 ** -52, integ.q_end.shape))
        elif every_step == "store32":
            integ.q_end = integ.q_end.astype(np.float32).astype(np.float64)
        hmin = min(hmin, float(integ.q_end[0].min()))
    q = integ.q_end
    hb, hub, hvb = element_means(ref, q)
    col = np.floor(om.cx / 0.0625).astype(np.int64)
    assert col.min() == 0 and col.max() == 319
    w = np.bincount(col, weights=om.area, minlength=320)
    cols = {name: (np.bincount(col, weights=om.area * v, minlength=320) / w).tolist()
            for name, v in (("h", hb), ("hu", hub), ("hv", hvb))}
    rng = np.random.Generator(np.random.PCG64(21))
    el = samples(rng, np.arange(om.K), 512)
    return {
        "scenario": "workloads.scenarios.dam_break() (320 x 32 x 2 triangles, N = 3, PP + TVB M = 0, AB3)",
        "K": om.K, "N": scn.N, "steps": scn.steps, "dt": integ.dt_min, "time": integ.time,
        "mass0": mass0, "mass": float(om.area @ hb), "injected_mass": float(integ.injected),
        "hmin_over_steps": hmin,
        "columns": {"dx": 0.0625, **cols},
        "sample": {"elements": el.tolist(), "h": hb[el].tolist(), "hu": hub[el].tolist(), "hv": hvb[el].tolist()},
        "oracle_seconds": time.time() - t0,
    }


def run_tsunami(macro_steps=25):
    scn = sc.tsunami()
    om, ref, model, integ = problem.build(scn)
    assert om.K == 500_000 and integ.L == 4
    lev = np.asarray(integ.level, np.int8)
    t0 = time.time()
    integ.macro_step(macro_steps)
    q = integ.q_end
    hb, hub, hvb = element_means(ref, q)
    Bb = model.B @ ref.mean_w
    rng = np.random.Generator(np.random.PCG64(22))
    r2 = (om.cx - 200e3) ** 2 + (om.cy - 50e3) ** 2
    groups = {
        "uniform": samples(rng, np.arange(om.K), 1024),
        "source": samples(rng, np.nonzero(r2 < (40e3) ** 2)[0], 1024),
        "shore": samples(rng, np.nonzero(om.cx > 370e3)[0], 512),
    }
    sample = {}
    for name, el in groups.items():
        sample[name] = {"elements": el.tolist(), "h": hb[el].tolist(), "hu": hub[el].tolist(),
                        "hv": hvb[el].tolist(), "B": Bb[el].tolist()}
    return {
        "scenario": "workloads.scenarios.tsunami() (1000 x 250 x 2 triangles, N = 4, 4 levels, PP + TVB)",
        "K": om.K, "N": scn.N, "macro_steps": macro_steps, "substeps": macro_steps * 2 ** (integ.L - 1),
        "dt_min": integ.dt_min, "time": integ.time,
        "level_counts": np.bincount(lev, minlength=5)[1:].tolist(),
        "level_sha256": hashlib.sha256(lev.tobytes()).hexdigest(),
        "mass": float(om.area @ hb), "hmin": float(q[0].min()),
        "sample": sample,
        "oracle_seconds": time.time() - t0,
    }


def main(which):
    new = {}
    if "dam_break" in which:
        new["dam_break"] = run_dam_break()
        print("dam_break done", new["dam_break"]["oracle_seconds"], flush=True)
    if "dam_break_ulp" in which:
        new["dam_break_ulp"] = run_dam_break(perturb=2.0 ** -52)
        print("dam_break_ulp done", new["dam_break_ulp"]["oracle_seconds"], flush=True)
    if "dam_break_ulp32" in which:
        new["dam_break_ulp32"] = run_dam_break(perturb=2.0 ** -23)
        print("dam_break_ulp32 done", new["dam_break_ulp32"]["oracle_seconds"], flush=True)
    if "dam_break_noise64" in which:
        new["dam_break_noise64"] = run_dam_break(every_step="noise64")
        print("dam_break_noise64 done", new["dam_break_noise64"]["oracle_seconds"], flush=True)
    if "dam_break_store32" in which:
        new["dam_break_store32"] = run_dam_break(every_step="store32")
        print("dam_break_store32 done", new["dam_break_store32"]["oracle_seconds"], flush=True)
    if "tsunami" in which:
        new["tsunami"] = run_tsunami()
        print("tsunami done", new["tsunami"]["oracle_seconds"], flush=True)
    # merged into the file as it is now, so the two parts may run as separate processes
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_about"] = ("FP64 oracle results on the full-size benchmark configurations, written by "
                      "tests/golden/make_full_config_golden.py (oracle/ only).")
    data.update(new)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["dam_break", "dam_break_ulp", "dam_break_ulp32", "dam_break_noise64", "dam_break_store32",
                          "tsunami"])
