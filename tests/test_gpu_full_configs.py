"""GPU parity on benchmark configurations at their full sizes and full run
lengths, against FP64 oracle results stored in tests/golden/full_config_oracle.json
(written by tests/golden/make_full_config_golden.py, which calls only the oracle;
the oracle needs about 10 minutes for each dam-break run and 47 for the tsunami).

* Wet/dry dam break, 20,480 triangles, N = 3, positivity-preserving + TVB
  (M = 0) limiting every stage, 2000 AB3 steps, on every tier. The run is
  one-dimensional up to the triangulation: the 320 column averages of the element
  means and the means of a seeded sample of elements are compared where the
  oracle's wet/dry state is the same two columns to either side (a front moves by
  decisions taken in different precisions), and an L1 bound holds over all
  columns. Minmod and wet/dry decisions carry rounding-level differences through
  the run, so each tier is held to 10 times the oracle's own response to
  rounding-level changes of its state after every step, the way an implementation
  that rounds differently departs from it: each nodal value multiplied by
  (1 + d), d uniform in [-2^-52, 2^-52], for the FP64 tier; each rounded to single
  precision for the FP32 tiers (both oracle runs are stored beside its result). A
  single change of the initial depth moves the oracle less (stored too): about as
  far for a single-precision ulp as for a double-precision one, since near the
  fronts the limiter's decisions, not the size of the change, set the distance,
  but such decisions are taken anew at every step. Depth stays
  non-negative after every step. Mass: the FP64 books close (mass = initial mass +
  tallied dry-reset injection) to round-off; FP32 storage rounds every nodal value
  up to three times a step (commit, positivity rescale, TVB rebuild), each by at
  most 2^-24 relative, which bounds the FP32 books by
  3 T 2^-24 sum_k area_k sum_j |w_j| |h_kj| (w the element-mean weights), and the
  FP32 tiers' mass stays within 1e-6 of the oracle's.
* Sloped-beach tsunami, 500,000 triangles, N = 4, 4 multirate levels, PP + TVB,
  200 finest substeps (25 macro steps), built and launched as the benchmark does
  (levels from the library's CFL rule, graph-replayed macro steps, FP32
  tensor-core tier). The levels equal the oracle's bit for bit; element means of
  the free surface eta = h + B and of the momenta on seeded samples (uniform,
  around the source, at the shore) are compared in units of the 2 m wave: the
  tier's state bound 8e-5 times the amplitude A for eta and times A sqrt(g H),
  H = 4000 m, the momentum a linear wave of amplitude A carries, for hu and hv.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from workloads import scenarios as sc

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_config_oracle.json")

U32 = 2.0 ** -24
TSU_TOL_STATE = 8e-5      # the tensor-core tier's state bound
TSU_A, TSU_H = 2.0, 4000.0


@pytest.fixture(scope="module")
def golden():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()
    with open(GOLDEN) as f:
        return json.load(f)


def _geometry(scn):
    vx, vy, E = scn.build_mesh()
    x, y = vx[E], vy[E]
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    return (vx, vy, E), x.mean(axis=1), y.mean(axis=1), area


def _mean_weights(N):
    from oracle.refelem import RefElement
    return RefElement(N).mean_w


def _away_from_fronts(oh):
    """Columns two or more away from every wet/dry change of the columns ``oh``."""
    wet = oh > 1e-3
    fronts = np.nonzero(wet[1:] != wet[:-1])[0]
    away = np.ones(oh.size, bool)
    for c in fronts:
        away[max(0, c - 2):c + 4] = False
    return away, fronts


def _dam_errors(g, hb, hub, hvb, col, away):
    """Max differences of column averages and sampled element means, and L1 over
    columns, of element means (hb, hub, hvb) against the oracle summary ``g``."""
    area = g["_area"]
    wsum = np.bincount(col, weights=area, minlength=320)
    c = [np.bincount(col, weights=area * v, minlength=320) / wsum for v in (hb, hub, hvb)]
    o = [np.asarray(g["columns"][k]) for k in ("h", "hu", "hv")]
    e_h = np.abs(c[0] - o[0])[away].max()
    e_m = max(np.abs(c[1] - o[1])[away].max(), np.abs(c[2] - o[2])[away].max())
    l1 = np.abs(c[0] - o[0]).sum() / np.abs(o[0]).sum()
    el = np.asarray(g["sample"]["elements"])
    keep = away[col[el]] & ((hb[el] > 1e-3) == (np.asarray(g["sample"]["h"]) > 1e-3))
    s_h = np.abs(hb[el] - g["sample"]["h"])[keep].max()
    s_m = max(np.abs(hub[el] - g["sample"]["hu"])[keep].max(), np.abs(hvb[el] - g["sample"]["hv"])[keep].max())
    return e_h, e_m, l1, s_h, s_m, keep


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_dam_break_full_size_2000_steps(golden, precision):
    import paper_1403_1661_gb300 as P
    g = golden["dam_break"]
    scn = sc.dam_break()
    arrays, cx, cy, area = _geometry(scn)
    K = arrays[2].shape[0]
    assert K == g["K"] == 20480
    s = P.solver_from_scenario(scn, precision=precision, levels=np.ones(K, np.int32), dt_min=g["dt"],
                               mesh_arrays=arrays)
    st0 = s.stats()
    hmin = st0["hmin"]
    for _ in range(g["steps"]):
        s.substep(1)
        hmin = min(hmin, s.stats()["hmin"])
    st = s.stats()
    h, hu, hv, t = s.get_state()
    assert abs(t - g["time"]) <= 1e-12 * g["time"]
    assert not st["nonfinite"] and np.isfinite(h).all()

    w = _mean_weights(scn.N)
    col = np.floor(cx / g["columns"]["dx"]).astype(np.int64)
    away, fronts = _away_from_fronts(np.asarray(g["columns"]["h"]))
    g = dict(g, _area=area)
    e_h, e_m, l1, s_h, s_m, keep = _dam_errors(g, h @ w, hu @ w, hv @ w, col, away)
    mass_err = abs(st["mass"] - g["mass"]) / g["mass"]
    budget = abs(st["mass"] - (st0["mass"] + st["injected_mass"] - st0["injected_mass"])) / g["mass"]

    # the oracle's own response to rounding-level changes of its state after every
    # step: relative noise of one double-precision ulp (FP64 tier), rounding to
    # single precision (FP32 tiers)
    u = golden["dam_break_noise64" if precision == "fp64" else "dam_break_store32"]
    ub = np.asarray(u["sample"]["h"]), np.asarray(u["sample"]["hu"]), np.asarray(u["sample"]["hv"])
    uc = [np.asarray(u["columns"][k]) for k in ("h", "hu", "hv")]
    oc = [np.asarray(g["columns"][k]) for k in ("h", "hu", "hv")]
    os_ = [np.asarray(g["sample"][k]) for k in ("h", "hu", "hv")]
    r_h = max(np.abs(uc[0] - oc[0])[away].max(), np.abs(ub[0] - os_[0])[keep].max())
    r_m = max(np.abs(uc[1] - oc[1])[away].max(), np.abs(uc[2] - oc[2])[away].max(),
              np.abs(ub[1] - os_[1])[keep].max(), np.abs(ub[2] - os_[2])[keep].max())
    r_l1 = np.abs(uc[0] - oc[0]).sum() / np.abs(oc[0]).sum()
    r_mass = abs(u["mass"] - g["mass"]) / g["mass"]
    tol_h, tol_m, tol_l1 = (max(1e-9, 10 * r) for r in (r_h, r_m, r_l1))
    if precision == "fp64":
        tol_budget = 1e-11
        tol_mass = tol_budget + 10 * r_mass
    else:
        # FP32 storage rounds each nodal value up to three times a step (commit,
        # positivity rescale, TVB rebuild): the books close to that rounding bound, and
        # the drift from the oracle's mass is held to the 1e-6 of the tiers' mass bound
        tol_budget = 3 * g["steps"] * U32 * (area @ (np.abs(h) @ np.abs(w))) / g["mass"]
        tol_mass = 1e-6
    front_x = (fronts + 1) * g["columns"]["dx"]
    print(f"PARITY dam break full size {precision} 2000 steps: columns eh={e_h:.3e} em={e_m:.3e} "
          f"l1={l1:.3e}; sample eh={s_h:.3e} em={s_m:.3e} ({keep.sum()} of {keep.size}); mass {mass_err:.3e}, "
          f"budget {budget:.3e}; hmin over steps {hmin:.3e} (oracle {g['hmin_over_steps']:.3e}); "
          f"fronts at x = {front_x.tolist()}; bounds h {tol_h:.3e} m {tol_m:.3e} l1 {tol_l1:.3e} "
          f"mass {tol_mass:.3e} budget {tol_budget:.3e}; oracle one-ulp response h {r_h:.3e} m {r_m:.3e} "
          f"l1 {r_l1:.3e} mass {r_mass:.3e}", flush=True)
    assert hmin >= 0.0
    assert keep.sum() >= 0.8 * keep.size
    assert e_h < tol_h and s_h < tol_h
    assert e_m < tol_m and s_m < tol_m
    assert l1 < tol_l1
    assert budget < tol_budget and mass_err < tol_mass


def test_tsunami_full_size_200_substeps(golden):
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300.solver import scenario_inputs
    g = golden["tsunami"]
    scn = sc.tsunami()
    s = P.solver_from_scenario(scn, precision="fp32tc")      # as the benchmark builds it
    lev = np.asarray(s.level, np.int8)
    L, counts, dtm = s.level_info()
    assert lev.size == g["K"] == 500_000
    assert np.bincount(lev, minlength=5)[1:].tolist() == g["level_counts"]
    assert hashlib.sha256(lev.tobytes()).hexdigest() == g["level_sha256"]
    # the device takes each element's CFL step from its FP32 state, so dt_min (and
    # the time after n substeps) agrees with the oracle's to FP32 rounding
    assert abs(dtm - g["dt_min"]) <= 1e-6 * g["dt_min"]
    s.step(g["macro_steps"])
    st = s.stats()
    h, hu, hv, t = s.get_state()
    assert abs(t - g["time"]) <= 1e-6 * g["time"]
    assert not st["nonfinite"] and np.isfinite(h).all() and h.min() >= -1e-6

    w = _mean_weights(scn.N)
    B, _, _, _ = scenario_inputs(scn, s.mesh)
    B32 = B.astype(np.float32).astype(np.float64)             # the bed as the device holds it
    eta_scale = TSU_TOL_STATE * TSU_A
    mom_scale = TSU_TOL_STATE * TSU_A * np.sqrt(scn.g * TSU_H)
    worst = {}
    for name, grp in g["sample"].items():
        el = np.asarray(grp["elements"])
        eta_g = (h[el] + B32[el]) @ w
        eta_o = np.asarray(grp["h"]) + np.asarray(grp["B"])
        e_eta = np.abs(eta_g - eta_o).max()
        e_m = max(np.abs(hu[el] @ w - grp["hu"]).max(), np.abs(hv[el] @ w - grp["hv"]).max())
        # wet: mean depth above twice the dry-reset depth h0 (a dry element holds h0,
        # which the FP32 tiers return within a few ulp of the bed's height)
        wet_agree = ((h[el] @ w > 2 * scn.h0) == (np.asarray(grp["h"]) > 2 * scn.h0)).all()
        worst[name] = (e_eta, e_m, wet_agree)
    mass_err = abs(st["mass"] - g["mass"]) / g["mass"]
    print("PARITY tsunami full size fp32tc 200 substeps: "
          + "; ".join(f"{n} eta {e:.3e} m, hu/hv {m:.3e} m^2/s, wet/dry agree {a}" for n, (e, m, a) in worst.items())
          + f"; mass {mass_err:.3e}", flush=True)
    for name, (e_eta, e_m, wet_agree) in worst.items():
        assert wet_agree, name
        assert e_eta < eta_scale, (name, e_eta)
        assert e_m < mom_scale, (name, e_m)
    assert mass_err < 1e-6
