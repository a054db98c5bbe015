"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bounds: first derived from the arithmetic -- FP64 1e-11 relative per field; FP32 R
within 2e-5 of max|R| (single-precision rounding of the state, bed and operators,
amplified by the ~Np*Ncub-term contractions), states within 2e-5 max(h) (depth) and
2e-5 max(h) sqrt(g max h) (momentum); FP32 tensor cores (split-BF16 products,
relative error about 3 * 2^-16 each) R within 2e-4, states within 8e-5 -- then
tightened to about ten times the largest error observed on GB300 per tier,
configuration and order and frozen (the observed values are listed in the design
notes). Still water over any bed gives R = 0 exactly in the
FP32 tiers (the element reference split), so that bound is zero.
"""
import numpy as np
import pytest

from tests.gpu_helpers import both, state_errors
from workloads import meshes, scenarios as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()


def _report(name, **vals):
    print("PARITY", name, " ".join(f"{k}={v:.3e}" for k, v in vals.items()), flush=True)


def _rhs_case(N, precision, moving=True, bed="smooth", nx=9, ny=7, limiter_mask=0):
    """Hump on a jittered graded mesh over a bed; velocities from a smooth field."""
    scn = sc.Scenario(
        name=f"rhs_case_N{N}", N=N, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=limiter_mask,
        tvb_M=0.0,
        mesh=lambda: meshes.graded_jittered_rect(0.0, 1.0, 0.0, 1.0, nx, ny, ratio=2.0, jitter=0.2, seed=11),
        bathymetry=(sc.smooth_bump_bed(depth=1.0, amp=0.3) if bed == "smooth"
                    else sc.step_bed_by_centroid(0.5, -1.0, -0.8, 0.2)),
        init=None)

    def init(x, y, cx, cy, B):
        eta = 0.05 * np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / 0.05)
        h = eta - B
        if not moving:
            return h, 0 * h, 0 * h
        return h, h * 0.3 * np.sin(3 * x + y), h * (-0.2) * np.cos(2 * y - x)
    scn.init = init
    return scn


# R per field relative to max|R|, by tier and order N (observed x 10)
TOL_R = {"fp64": {1: 2e-13, 2: 4e-13, 3: 6e-13, 4: 5e-13, 5: 5e-13},
         "fp32": {1: 5e-6, 2: 6e-6, 3: 7e-6, 4: 6e-6, 5: 9e-6},
         "fp32tc": {1: 9e-5, 2: 1e-4, 3: 1.5e-4, 4: 8e-5, 5: 1e-4}}
# states: depth relative to max h, momentum relative to max h sqrt(g max h), by
# configuration and tier (observed x 10)
TOL_STATE = {"hump100": {"fp64": 3e-14, "fp32": 3e-8, "fp32tc": 5e-7},
             "tsunami": {"fp64": 1.5e-13, "fp32": 4e-7, "fp32tc": 4e-7},
             "one_element": {"fp64": 3e-14, "fp32": 1.3e-6, "fp32tc": 1.3e-6},
             "tsunami_n1": {"fp64": 1.5e-14, "fp32tc": 3e-7}}
TOL_R_ONE = {"fp64": 9e-13, "fp32": 5e-6, "fp32tc": 8e-5}
# still water at eta = 0.3, relative to g (max h)^2 max|r_x|; exactly zero in FP32
TOL_LAKE = {"fp64": 5e-15, "fp32": 0.0, "fp32tc": 0.0}
# small dam break (branchy): L1 over all elements; max norm over the elements away
# from the front; FP64 everywhere (observed x 10)
DAM_SMALL_L1 = {"fp32": 1e-6, "fp32tc": 8e-7}
DAM_SMALL_AWAY = {"fp32": 2.3e-5, "fp32tc": 3e-5}
DAM_SMALL_FP64 = 6e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_rhs_matches_oracle(N, precision):
    scn = _rhs_case(N, precision)
    om, ref, model, integ, s = both(scn, precision)
    q = integ.q_end
    R_o = model.rhs(q[0], q[1], q[2])
    R_g = s.rhs().cpu().numpy().astype(np.float64)
    errs = [np.abs(R_g[c] - R_o[c]).max() / np.abs(R_o[c]).max() for c in range(3)]
    _report(f"rhs N={N} {precision}", e_h=errs[0], e_hu=errs[1], e_hv=errs[2])
    assert max(errs) < TOL_R[precision][N]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
@pytest.mark.parametrize("bed", ["smooth", "discontinuous"])
def test_lake_at_rest(precision, bed):
    """Still water over a smooth or a face-discontinuous bed (Section 5.1): R = 0.
    At the datum eta = 0 the pre-balanced form is exact in any precision."""
    scn = _rhs_case(3, precision, moving=False, bed=bed)
    scn.init = lambda x, y, cx, cy, B: (0.0 - B, 0 * B, 0 * B)
    om, ref, model, integ, s = both(scn, precision)
    R = s.rhs().cpu().numpy()
    _report(f"lake eta=0 {bed} {precision}", maxR=float(np.abs(R).max()))
    assert np.abs(R).max() == 0.0
    # away from the datum: round-off of the still-water pressure only
    scn.init = lambda x, y, cx, cy, B: (0.3 - B, 0 * B, 0 * B)
    om, ref, model, integ, s = both(scn, precision)
    R = s.rhs().cpu().numpy()
    scale = 9.81 * 1.3 ** 2 * max(np.abs(om.rx).max(), np.abs(om.sy).max())
    _report(f"lake eta=0.3 {bed} {precision}", rel=float(np.abs(R).max() / scale))
    # FP32 tiers: the element reference split leaves nothing to round (exactly zero)
    assert np.abs(R).max() <= TOL_LAKE[precision] * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_hump_square_ab3_100_steps(precision):
    """The plain-method configuration at full size: 512 triangles, N = 2, AB3, 100 steps."""
    scn = sc.hump_square()
    om, ref, model, integ, s = both(scn, precision)
    for _ in range(scn.steps):
        integ.substep()
    s.substep(scn.steps)
    eh, em, (h, hu, hv, t) = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    _report(f"hump100 {precision}", eh=eh / hmax, em=em / (hmax * np.sqrt(9.81 * hmax)))
    assert abs(t - integ.time) < 1e-12 * integ.time
    tol = TOL_STATE["hump100"][precision]
    assert eh < tol * hmax and em < tol * hmax * np.sqrt(9.81 * hmax)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_mrab_tsunami_levels(precision):
    """Graded beach, 3-4 MRAB levels, positivity + TVB: two macro steps."""
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    om, ref, model, integ, s = both(scn, precision)
    nsub = 2 * 2 ** (integ.L - 1)
    for _ in range(nsub):
        integ.substep()
    s.substep(nsub)
    eh, em, _ = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    _report(f"tsunami L={integ.L} {precision}", eh=eh / hmax, em=em / (hmax * np.sqrt(9.81 * hmax)))
    tol = TOL_STATE["tsunami"][precision]
    assert eh < tol * hmax and em < tol * hmax * np.sqrt(9.81 * hmax)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_dam_break_small_pp_tvb(precision):
    """Wet/dry dam break with positivity + TVB (M = 0) every stage, 40 steps."""
    scn = sc.dam_break(nx=40, ny=4, N=3, steps=40)
    om, ref, model, integ, s = both(scn, precision)
    for _ in range(scn.steps):
        integ.substep()
    s.substep(scn.steps)
    h, hu, hv, t = s.get_state()
    q = integ.q_end
    eh = np.abs(h - q[0]).max()
    em = max(np.abs(hu - q[1]).max(), np.abs(hv - q[2]).max())
    l1 = np.abs(h - q[0]).sum() / np.abs(q[0]).sum()
    # max norm away from the front: elements whose wet/dry state agrees with the
    # oracle's, in columns of square cells more than two columns from any column where
    # the oracle's column-mean wet/dry state changes (a front moves by decisions taken
    # in different precisions)
    w = ref.mean_w
    cx = om.cx
    dx = 20.0 / 40
    col = np.floor(cx / dx).astype(np.int64)
    hb_o = q[0] @ w
    colh = np.bincount(col, weights=hb_o, minlength=40) / np.bincount(col, minlength=40)
    wetc = colh > 1e-3
    change = np.nonzero(wetc[1:] != wetc[:-1])[0]
    dist = np.full(40, 99)
    for c in change:
        dist = np.minimum(dist, np.minimum(np.abs(np.arange(40) - c), np.abs(np.arange(40) - (c + 1))))
    keep = (dist[col] > 2) & (((h @ w) > 1e-3) == (hb_o > 1e-3))
    hmax = q[0].max()
    ehk = np.abs(h - q[0])[keep].max() / hmax
    emk = max(np.abs(hu - q[1])[keep].max(), np.abs(hv - q[2])[keep].max()) / (hmax * np.sqrt(9.81 * hmax))
    _report(f"dambreak {precision}", eh=eh, em=em, l1=l1, hmin=h.min(), eh_away=ehk, em_away=emk,
            kept=float(keep.mean()))
    assert h.min() >= -1e-6
    assert keep.mean() > 0.5
    if precision == "fp64":
        assert eh < DAM_SMALL_FP64 and em < DAM_SMALL_FP64
    else:
        assert l1 < DAM_SMALL_L1[precision]
        assert ehk < DAM_SMALL_AWAY[precision] and emk < DAM_SMALL_AWAY[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp32tc"])
def test_graph_replay_equals_direct_launches(precision):
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    _, _, _, integ, a = both(scn, precision)
    import paper_1403_1661_gb300 as P
    b = P.solver_from_scenario(scn, precision=precision, levels=integ.level, dt_min=integ.dt_min)
    L = integ.L
    a.substep(3 * 2 ** (L - 1))
    b.step(3)
    ha = a.get_state()
    hb = b.get_state()
    for x, y in zip(ha[:3], hb[:3]):
        assert np.array_equal(x, y)
    assert a.stats()["dof_updates"] == b.stats()["dof_updates"]


def test_checkpoint_resume_bit_identical():
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    _, _, _, integ, a = both(scn, "fp32")
    L = integ.L
    a.step(1)
    ck = a.full_state()
    a.step(2)
    ref = a.get_state()
    import paper_1403_1661_gb300 as P
    b = P.solver_from_scenario(scn, precision="fp32")
    b.load_full_state(ck)
    b.step(2)
    got = b.get_state()
    for x, y in zip(ref, got):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_checkpoint_inside_a_macro_step_bit_identical():
    # three substeps into a macro step the levels are out of step with each other:
    # the restored history must reproduce every later substep exactly
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    import paper_1403_1661_gb300 as P
    a = P.solver_from_scenario(scn, precision="fp32")
    assert a.level_info()[0] >= 2
    a.step(1)
    a.substep(3)
    ck = a.full_state()
    a.substep(5)
    a.step(1)
    ref = a.get_state()
    b = P.solver_from_scenario(scn, precision="fp32")
    b.load_full_state(ck)
    b.substep(5)
    b.step(1)
    got = b.get_state()
    for x, y in zip(ref, got):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_corrupted_checkpoint_is_refused_and_the_state_kept():
    """A checkpoint whose header sizes, levels, dt_min, time or step count are
    invalid (or that is cut short) is refused with SWE_EINVAL before anything of the
    solver changes; the intact checkpoint then still resumes bit for bit. Offsets:
    the 112-byte header (magic, six int32, k and dof_updates int64, t0 and dt_min
    double, six uint64 section sizes), then K int32 levels."""
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    a = P.solver_from_scenario(scn, precision="fp32")
    a.step(1)
    ck = a.full_state()
    b = P.solver_from_scenario(scn, precision="fp32")
    b.step(2)
    before = b.get_state()

    def bad(offset, dtype, value):
        c = ck.copy()
        c[offset:offset + np.dtype(dtype).itemsize] = np.array([value], dtype).view(np.uint8)
        return c
    cases = {"magic": bad(0, np.uint8, 0), "k": bad(32, np.int64, -5), "t0": bad(48, np.float64, np.nan),
             "dt_min": bad(56, np.float64, -1.0), "bytes_q": bad(64, np.uint64, 1 << 40),
             "bytes_ring": bad(72, np.uint64, 8), "level 99": bad(112, np.int32, 99),
             "level 0": bad(112 + 4 * 5, np.int32, 0), "short": ck[:-1]}
    for name, c in cases.items():
        with pytest.raises(nat.SWEError) as ei:
            b.load_full_state(c)
        assert ei.value.code == nat.SWE_EINVAL, name
        for x, y in zip(before, b.get_state()):
            assert np.array_equal(np.asarray(x), np.asarray(y)), name
    for dtm in (np.inf, np.nan, 0.0):
        with pytest.raises(nat.SWEError) as ei:
            b.set_levels(np.ones(b.K, np.int32), dtm)
        assert ei.value.code == nat.SWE_EINVAL
    b.load_full_state(ck)
    a.step(1)
    b.step(1)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    a.close()
    b.close()


def test_mass_conservation_and_stats():
    scn = sc.hump_square(n=16, N=3)
    _, _, model, integ, s = both(scn, "fp64")
    m0 = s.stats()["mass"]
    assert abs(m0 - model.mass(integ.q_end[0])) < 1e-12 * m0
    s.substep(50)
    st = s.stats()
    _report("mass fp64", drift=abs(st["mass"] - m0) / m0)
    assert abs(st["mass"] - m0) < 1e-13 * m0 * 50
    assert st["dof_updates"] == 50 * integ.model.mesh.K * 10 * 3 and not st["nonfinite"]


def test_set_state_rejects_nonfinite_and_keeps_state():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    scn = sc.tsunami(nx=24, ny=6, N=3, nlevels=3)
    s = P.solver_from_scenario(scn, precision="fp32tc")
    s.step(1)
    before = s.get_state()
    h, hu, hv = (np.array(a) for a in before[:3])
    hu[3, 2] = np.nan
    with pytest.raises(nat.SWEError) as ei:
        s.set_state(h, hu, hv)
    assert ei.value.code == nat.SWE_EINVAL
    after = s.get_state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)
    # pinned output buffers give the same values
    import torch
    outs = tuple(torch.empty((s.K, s.Np), dtype=torch.float64, pin_memory=True).numpy() for _ in range(3))
    got = s.get_state(out=outs)
    for x, y in zip(before[:3], got[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_single_element_all_walls(precision):
    """Degenerate mesh: one triangle, every face a wall (one tile with 31 empty
    lanes on the tensor-core path): R and ten steps against the oracle."""
    scn = sc.Scenario(name="one", N=3, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=3, tvb_M=0.0,
                      mesh=lambda: (np.array([0.0, 1.0, 0.2]), np.array([0.0, 0.1, 0.9]),
                                    np.array([[0, 1, 2]], np.int32)),
                      bathymetry=lambda x, y, cx=None, cy=None: -1.0 + 0.1 * x, init=None)
    scn.init = lambda x, y, cx, cy, B: (0.05 * np.exp(-((x - 0.4) ** 2 + (y - 0.3) ** 2) / 0.05) - B,
                                        0.1 * x * (1.0 - B), 0 * x)
    om, ref, model, integ, s = both(scn, precision)
    assert om.K == 1
    q = integ.q_end
    R_o = model.rhs(q[0], q[1], q[2])
    R_g = s.rhs().cpu().numpy().astype(np.float64)
    e = max(np.abs(R_g[c] - R_o[c]).max() / np.abs(R_o[c]).max() for c in range(3))
    for _ in range(10):
        integ.substep()
    s.substep(10)
    eh, em, _ = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    _report(f"one element {precision}", eR=e, eh=eh / hmax, em=em / (hmax * np.sqrt(9.81 * hmax)))
    tol = TOL_STATE["one_element"][precision]
    assert e < TOL_R_ONE[precision]
    assert eh < tol * hmax and em < tol * hmax * np.sqrt(9.81 * hmax)


@pytest.mark.parametrize("precision", ["fp64", "fp32tc"])
def test_order_one_multirate_beach(precision):
    """N = 1 (linear elements, the paper's lowest order in Section 6): the graded beach
    with 4 levels and PP + TVB, two macro steps against the oracle."""
    scn = sc.tsunami(nx=40, ny=10, N=1, nlevels=4)
    om, ref, model, integ, s = both(scn, precision)
    nsub = 2 * 2 ** (integ.L - 1)
    for _ in range(nsub):
        integ.substep()
    s.substep(nsub)
    eh, em, _ = state_errors(s, integ)
    hmax = integ.q_end[0].max()
    _report(f"tsunami N=1 L={integ.L} {precision}", eh=eh / hmax, em=em / (hmax * np.sqrt(9.81 * hmax)))
    tol = TOL_STATE["tsunami_n1"][precision]
    assert eh < tol * hmax and em < tol * hmax * np.sqrt(9.81 * hmax)
