"""Single-precision tiers with the compensated state update
(swe_params.compensated = 1). The plain single-precision update rounds the state at
every commit and drifts in total mass by about 5e-9 of itself per step even in a
closed, fully wet basin; with the compensated sum the mass keeps to rounding and
the state stays far closer to FP64 (on the rarefaction wave at N = 3 the tier then
meets the same convergence bar as FP64). Checkpoints carry the compensation planes,
a regroup gathers them with the state, and a batch refuses such a solver."""
import math

import numpy as np
import pytest

from workloads import meshes, scenarios as sc

pytestmark = pytest.mark.gpu

# measured on GB300 (N = 2, 40 x 32 x 2 triangles, CFL 0.03, 7,181 steps to t = 8):
# 1.8e-9 (SIMT and tensor-core) against 3.5e-5 plain; bound = 10 x observed
COMP_DRIFT_MAX = 1.8e-8


def _hump(nx, N):
    """A closed basin (walls, flat bed), depth 1 with a Gaussian hump of 0.2: wet
    everywhere, the positivity limiter never triggers."""
    s = sc.Scenario(name=f"hump_{nx}", N=N, g=1.0, h0=1e-5, cfl=0.03, nlevels=1, limiter_mask=1, tvb_M=0.0,
                    mesh=lambda: meshes.structured_rect(0, 50, 0, 40, nx, nx * 4 // 5),
                    bathymetry=lambda x, y, cx=None, cy=None: 0.0 * x, init=None)
    s.init = lambda x, y, cx, cy, B: (1.0 + 0.2 * np.exp(-((x - 25) ** 2 + (y - 20) ** 2) / 20.0), 0 * x, 0 * x)
    return s


def _solver(scn, precision, comp, T=8.0):
    import paper_1403_1661_gb300 as P
    from oracle.mesh import Mesh, element_dt
    from oracle.refelem import RefElement
    vx, vy, E = scn.build_mesh()
    m = Mesh(vx, vy, E)
    ref = RefElement(scn.N)
    x, y = m.map_to_physical(ref.r, ref.s)
    h, hu, hv = scn.init(x, y, 0, 0, 0 * x)
    ns = int(math.ceil(T / element_dt(m, scn.N, h, hu, hv, scn.g, scn.cfl).min()))
    s = P.solver_from_scenario(scn, precision=precision, levels=np.ones(m.K, np.int32), dt_min=T / ns,
                               compensated=comp)
    return s, ns


def _unaccounted(st0, st):
    return abs((st["mass"] - st0["mass"]) - (st["injected_mass"] - st0["injected_mass"])) / st0["mass"]


@pytest.mark.parametrize("precision", ["fp32", "fp32tc"])
def test_compensated_update_keeps_mass_and_accuracy(precision):
    scn = _hump(40, 2)
    drift, state = {}, {}
    for comp in (False, True):
        s, ns = _solver(scn, precision, comp)
        st0 = s.stats()
        s.substep(ns)
        drift[comp] = _unaccounted(st0, s.stats())
        state[comp] = s.get_state()[0]
        s.close()
    ref, ns = _solver(scn, "fp64", False)
    ref.substep(ns)
    h64 = ref.get_state()[0]
    ref.close()
    err = {c: float(np.abs(state[c] - h64).max()) for c in (False, True)}
    print(f"PARITY compensated {precision} N=2 {ns} steps: unaccounted mass plain {drift[False]:.2e} "
          f"compensated {drift[True]:.2e}; max |h - h_fp64| plain {err[False]:.2e} compensated {err[True]:.2e}",
          flush=True)
    assert drift[True] < COMP_DRIFT_MAX
    assert drift[False] > 10 * drift[True]
    # the plain update's long-run error is its accumulated state rounding (1.9e-4
    # against FP64 here); the compensated one stays near FP32 round-off (2.2e-7 SIMT,
    # 4.9e-7 tensor-core)
    assert err[True] < 0.1 * err[False]


def test_compensated_checkpoint_resume_bit_identical():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    scn = _hump(24, 3)
    a, _ = _solver(scn, "fp32tc", True)
    a.step(40)
    b, _ = _solver(scn, "fp32tc", True)
    b.step(20)
    buf = b.full_state()
    c, _ = _solver(scn, "fp32tc", True)
    c.load_full_state(buf)
    c.step(20)
    for u, v in zip(a.get_state(), c.get_state()):
        assert np.array_equal(u, v)
    # a plain solver cannot load a compensated checkpoint (its sections differ)
    d, _ = _solver(scn, "fp32tc", False)
    with pytest.raises(nat.SWEError):
        d.load_full_state(buf)
    with pytest.raises(nat.SWEError) as ei:
        P.Batch([a])
    assert ei.value.code == nat.SWE_EUNSUPPORTED
    for s in (a, b, c, d):
        s.close()


def test_compensated_multirate_with_regroup():
    """The plane follows the state through a regroup (the elements are re-ordered)."""
    import paper_1403_1661_gb300 as P
    scn = sc.tsunami(nx=60, ny=15, N=3)
    s = P.solver_from_scenario(scn, precision="fp32tc", compensated=True)
    st0 = s.stats()
    s.step(4)
    s.regroup()
    s.step(4)
    st = s.stats()
    h = s.get_state()[0]
    print(f"PARITY compensated multirate regroup: unaccounted mass {_unaccounted(st0, st):.2e}", flush=True)
    assert np.isfinite(h).all() and not st["nonfinite"]
    assert _unaccounted(st0, st) < 1e-7
    s.close()


def test_compensated_rarefaction_n3_meets_the_fp64_bar():
    """Section 6.4's rarefaction wave at N = 3 (CFL 0.03, H = 1.25, 0.625, 0.3125): the
    plain single-precision tiers lose the local rate there (about 1e4 steps on the
    finest mesh); with the compensated update the tensor-core tier meets the bar the
    FP64 tier is held to (global >= 1.3, local >= 2.7; measured 1.35 and 3.16, FP64
    1.35 and 3.18)."""
    import paper_1403_1661_gb300 as P
    import test_gpu_verification as V
    orig = P.solver_from_scenario
    try:
        P.solver_from_scenario = lambda *a, **k: orig(*a, compensated=True, **k)
        res = V._wetdry_errors(lambda n: V._rare_scenario(n, 3, cfl=0.03), [40, 80, 160], V._rare_exact,
                               lambda m: (m.cx > 15) & (m.cx < 35), 2.0, 10.0, "fp32tc")
    finally:
        P.solver_from_scenario = orig
    g, l = V._rate([r[0] for r in res]), V._rate([r[1] for r in res])
    bg, bl, _ = V.RARE_BOUNDS[3]
    print(f"PARITY compensated rarefaction N=3 fp32tc global " + " ".join(f"{r[0]:.3e}" for r in res)
          + " local " + " ".join(f"{r[1]:.3e}" for r in res) + f" rates {g:.2f} {l:.2f}", flush=True)
    assert g >= bg and l >= bl
    assert max(r[2] for r in res) < 1e-6
