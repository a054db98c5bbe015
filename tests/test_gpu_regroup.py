"""Level regrouping without restart (Section 4's remark) through the C ABI, against
the oracle's MRAB.regroup.

* Graded tsunami beach, 4 levels, PP + TVB: three macro steps, a regroup to new
  levels (some finer, some coarser, the number of levels changing), two more macro
  steps: the state against the oracle doing the same, in every tier.
* The CFL rule (level=None): the same levels and margin as the oracle's rule.
* Regrouping to the same levels changes nothing (bit for bit).
* Argument checks leave the solver unchanged.
* Thacker's oscillation with 3 levels: without regrouping the shoreline floods cells
  whose coarse step no longer satisfies the CFL bound and the run blows up; with the
  CFL regroup after every macro step it stays within the single-rate accuracy.
"""
import math

import numpy as np
import pytest

from tests.gpu_helpers import both, state_errors
from tests.test_gpu_parity import TOL_STATE
from workloads import scenarios as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()


def _new_levels(level, seed=7):
    rng = np.random.default_rng(seed)
    new = level.copy()
    up = rng.random(level.size) < 0.3
    down = rng.random(level.size) < 0.3
    new[up] = np.minimum(level[up] + 1, 4)
    new[down & ~up] = np.maximum(level[down & ~up] - 1, 1)
    return new


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_regroup_matches_oracle(precision):
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    om, ref, model, integ, s = both(scn, precision)
    L = integ.L
    assert L == 4
    for _ in range(3 * 2 ** (L - 1)):
        integ.substep()
    s.step(3)
    new = _new_levels(integ.level)
    new[:5] = 4                                   # keep 4 levels in use
    integ.regroup(new)
    got, _ = s.regroup(new)
    assert np.array_equal(got, new)
    for _ in range(2 * 2 ** (integ.L - 1)):
        integ.substep()
    s.step(2)
    eh, em, (h, hu, hv, t) = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    print(f"PARITY regroup {precision} eh={eh / hmax:.3e} em={em / (hmax * np.sqrt(9.81 * hmax)):.3e}", flush=True)
    assert abs(t - integ.time) < 1e-12 * integ.time
    tol = TOL_STATE["tsunami"][precision]
    assert eh < tol * hmax and em < tol * hmax * np.sqrt(9.81 * hmax)


def test_regroup_cfl_rule_matches_oracle():
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    om, ref, model, integ, s = both(scn, "fp64")
    for _ in range(3 * 2 ** (integ.L - 1)):
        integ.substep()
    s.step(3)
    lev_o, margin_o = integ.cfl_levels(scn.cfl, scn.nlevels)
    lev_g, margin_g = s.regroup(None)
    assert np.array_equal(lev_g, lev_o)
    assert abs(margin_g - margin_o) < 1e-12 * margin_o


def test_regroup_to_same_levels_is_identity():
    import paper_1403_1661_gb300 as P
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    a = P.solver_from_scenario(scn, precision="fp32tc")
    b = P.solver_from_scenario(scn, precision="fp32tc")
    a.step(3)
    b.step(3)
    b.regroup(b.level.copy())
    a.step(2)
    b.step(2)
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        assert np.array_equal(x, y)


def test_regroup_argument_checks():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    scn = sc.tsunami(nx=24, ny=6, N=3, nlevels=3)
    s = P.solver_from_scenario(scn, precision="fp32")
    L = s.level_info()[0]
    assert L >= 2
    lev = s.level.copy()
    s.step(2)                                     # k = 2 * 2^(L-1) < 3 * 2^(L-1)
    with pytest.raises(nat.SWEError) as ei:
        s.regroup(lev)
    assert ei.value.code == nat.SWE_EINVAL
    s.step(1)
    s.substep(1)                                  # not level-synchronous
    with pytest.raises(nat.SWEError) as ei:
        s.regroup(lev)
    assert ei.value.code == nat.SWE_EINVAL
    s.substep(2 ** (L - 1) - 1)
    before = s.get_state()
    with pytest.raises(nat.SWEError) as ei:        # level out of 1..nlevels_max
        s.regroup(np.zeros_like(lev))
    assert ei.value.code == nat.SWE_EINVAL
    after = s.get_state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
    assert np.array_equal(s.level, lev)


def test_thacker_multirate_needs_regrouping():
    import paper_1403_1661_gb300 as P
    import tests.test_gpu_verification as tv
    scn = tv._thacker_scenario()
    scn.nlevels = 3
    T = 0.25 * 2 * math.pi / tv.TW
    res = {}
    for regroup in (False, True):
        s = P.solver_from_scenario(scn, precision="fp64")
        L0 = s.level_info()[0]
        t, k = 0.0, 0
        while t < T - 1e-12:
            L = s.level_info()[0]
            s.step(1)
            k += 2 ** (L - 1)
            h, _, _, t = s.get_state()
            if not np.isfinite(h).all():
                break
            if regroup and k >= 3 * 2 ** (L - 1):
                s.regroup(None)
        h, hu, hv, t = s.get_state()
        res[regroup] = (t, h)
    x, y = _thacker_nodes(scn)
    t1, h1 = res[True]
    he = tv._thacker(x, y, t1)[0]
    wet = he.min(axis=1) > 0.02
    l1 = np.abs(h1 - he)[wet].sum() / he[wet].sum()
    t0, h0 = res[False]
    print(f"PARITY thacker multirate L={L0}: without regroup finite={np.isfinite(h0).all()} at t={t0:.3f}; "
          f"with regroup t={t1:.3f} L1(wet) {l1:.3e} hmin {h1.min():.2e}", flush=True)
    assert not np.isfinite(h0).all()              # the limitation the regroup removes
    assert np.isfinite(h1).all() and l1 < 2.5e-2 and h1.min() >= 1e-3 - 1e-12


def _thacker_nodes(scn):
    from oracle.mesh import Mesh
    from oracle.refelem import RefElement
    vx, vy, E = scn.build_mesh()
    m, ref = Mesh(vx, vy, E), RefElement(scn.N)
    return m.map_to_physical(ref.r, ref.s)


def test_batch_refuses_stale_graph_after_regroup():
    """A batch captured before a solver's regroup would replay stale launches:
    swe_batch_step refuses until the batch is created again."""
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    from paper_1403_1661_gb300.batch import Batch
    scn = sc.tsunami(nx=24, ny=6, N=3, nlevels=3)
    a = P.solver_from_scenario(scn, precision="fp32")
    b = P.solver_from_scenario(scn, precision="fp32")
    batch = Batch([a, b])
    batch.step(3)
    a.regroup(a.level.copy())
    with pytest.raises(nat.SWEError) as ei:
        batch.step(1)
    assert ei.value.code == nat.SWE_EINVAL
    batch.close()
    again = Batch([a, b])
    again.step(1)
    again.close()
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        assert np.array_equal(x, y)


def test_checkpoint_after_regroup_resumes_bit_identically():
    import paper_1403_1661_gb300 as P
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    a = P.solver_from_scenario(scn, precision="fp32tc")
    a.step(3)
    a.regroup(_new_levels(a.level, seed=3))
    a.step(1)
    ck = a.full_state()
    a.step(2)
    ref = a.get_state()
    b = P.solver_from_scenario(scn, precision="fp32tc")
    b.load_full_state(ck)
    b.step(2)
    for x, y in zip(ref[:3], b.get_state()[:3]):
        assert np.array_equal(x, y)


def test_regroup_collocation_matches_oracle():
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    om, ref, model, integ, s = both(scn, "fp64", scheme="collocation")
    for _ in range(3 * 2 ** (integ.L - 1)):
        integ.substep()
    s.step(3)
    new = _new_levels(integ.level, seed=5)
    integ.regroup(new)
    s.regroup(new)
    for _ in range(2 * 2 ** (integ.L - 1)):
        integ.substep()
    s.step(2)
    eh, em, _ = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    print(f"PARITY regroup collocation fp64 eh={eh / hmax:.3e}", flush=True)
    assert eh < 1e-11 * hmax and em < 1e-11 * hmax * np.sqrt(9.81 * hmax)
