"""CPU tests of the native library: exports, host-side reference element, mesh
connectivity and level grouping against the oracle (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import mesh as omesh
from oracle import refelem as oref
from workloads import meshes, scenarios as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_1661_gb300 import build
    build.build()
    from paper_1403_1661_gb300 import _native
    return _native


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(swe_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(lib):
    L = C.CDLL(lib.LIB_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 30
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    # and the Python binding binds every one of them
    assert declared == set(lib.SIGNATURES), declared ^ set(lib.SIGNATURES)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_reference_element_matches_oracle(lib, N):
    import paper_1403_1661_gb300 as P
    Np, Ncub, Ng = P.ref_sizes(N)
    ref = oref.RefElement(N)
    assert (Np, Ncub, Ng) == (ref.Np, ref.Ncub, ref.Ng)
    r, s = P.ref_nodes(N)
    assert np.abs(r - ref.r).max() < 1e-13 and np.abs(s - ref.s).max() < 1e-13
    tol = 1e-11
    # the cubature ordering is the same tensor ordering on both sides
    for which, M in ((0, ref.Ic), (1, ref.Icr), (2, ref.Ics), (3, ref.Pr), (4, ref.Ps), (5, ref.P)):
        got = P.ref_operator(N, which)
        assert np.abs(got - M).max() < tol * max(1.0, np.abs(M).max()), which
    Lg = P.ref_operator(N, 6)
    want = np.concatenate(ref.Lg, axis=1)
    assert np.abs(Lg - want).max() < tol * np.abs(want).max()
    # face interpolation from the face nodes equals the full interpolation restricted to them
    I1 = P.ref_operator(N, 7)
    fn = [i for i in range(ref.Np) if abs(ref.s[i] + 1) < 1e-12]
    fn = sorted(fn, key=lambda i: ref.r[i])
    assert np.abs(I1 - ref.Ig[0][:, fn]).max() < 1e-12
    assert np.abs(P.ref_operator(N, 8) - ref.mean_w).max() < 1e-14
    assert np.abs(P.ref_operator(N, 9) - ref.Pi1[ref.vertex_nodes]).max() < 1e-12
    assert np.abs(P.ref_operator(N, 10) - ref.wc).max() < 1e-14
    assert np.abs(P.ref_operator(N, 11) - ref.wg).max() < 1e-14


@pytest.mark.parametrize("gen", [
    lambda: meshes.structured_rect(0, 1, 0, 1, 7, 5),
    lambda: meshes.graded_jittered_rect(0, 10, 0, 3, 9, 6, ratio=4, jitter=0.2, seed=7),
])
def test_connectivity_and_nodes_bit_exact(lib, gen):
    import paper_1403_1661_gb300 as P
    vx, vy, E = gen()
    E = E.copy()
    E[::4, 1], E[::4, 2] = E[::4, 2].copy(), E[::4, 1].copy()   # mixed orientation
    m = P.Mesh(vx, vy, E)
    om = omesh.Mesh(vx, vy, E)
    EToE, EToF = m.connectivity()
    assert np.array_equal(EToE, om.EToE) and np.array_equal(EToF, om.EToF)
    for N in (2, 4):
        x, y = m.node_coords(N)
        ref = oref.RefElement(N)
        ox, oy = om.map_to_physical(ref.r, ref.s)
        assert np.abs(x - ox).max() < 1e-12 and np.abs(y - oy).max() < 1e-12


def test_levels_bit_exact(lib):
    import paper_1403_1661_gb300 as P
    scn = sc.tsunami(nx=60, ny=15, N=3)
    vx, vy, E = scn.build_mesh()
    m = P.Mesh(vx, vy, E)
    om = omesh.Mesh(vx, vy, E)
    ref = oref.RefElement(scn.N)
    from oracle.problem import nodal_inputs
    B, h, hu, hv = nodal_inputs(scn, om, ref)
    lev, dtmin = m.levels(scn.N, h, hu, hv, scn.g, scn.cfl, scn.nlevels)
    olev, odtmin = omesh.assign_levels(omesh.element_dt(om, scn.N, h, hu, hv, scn.g, scn.cfl), scn.nlevels)
    assert np.array_equal(lev, olev)
    assert abs(dtmin - odtmin) <= 1e-15 * odtmin
    assert len(np.unique(lev)) >= 3


def test_levels_of_the_full_benchmark_mesh_equal_the_oracle(lib):
    """The level rule on the 500,000-triangle beach, evaluated at the library's own
    nodes, against the oracle's levels stored with its 200-substep run (SHA-256 of
    the per-element levels, counts, dt_min)."""
    import hashlib
    import json
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300.solver import scenario_inputs
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "full_config_oracle.json")))["tsunami"]
    scn = sc.tsunami()
    vx, vy, E = scn.build_mesh()
    m = P.Mesh(vx, vy, E)
    B, h, hu, hv = scenario_inputs(scn, m)
    lev, dtmin = m.levels(scn.N, h, hu, hv, scn.g, scn.cfl, scn.nlevels)
    lev = np.asarray(lev, np.int8)
    assert np.bincount(lev, minlength=5)[1:].tolist() == g["level_counts"]
    assert hashlib.sha256(lev.tobytes()).hexdigest() == g["level_sha256"]
    assert abs(dtmin - g["dt_min"]) <= 1e-15 * g["dt_min"]


def test_bad_meshes_are_rejected(lib):
    import paper_1403_1661_gb300 as P
    vx = np.array([0.0, 1.0, 0.0, 1.0, 0.5])
    vy = np.array([0.0, 0.0, 1.0, 1.0, -1.0])
    with pytest.raises(lib.SWEError) as ei:
        P.Mesh(vx, vy, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))   # face 0-1 shared 3 times
    assert ei.value.code == lib.SWE_EINVAL
    with pytest.raises(lib.SWEError):
        P.Mesh(vx, vy, np.array([[0, 1, 7]]))                           # bad index
    with pytest.raises(lib.SWEError):
        P.Mesh(vx, vy, np.zeros((0, 3), np.int32))                      # no elements
    with pytest.raises(lib.SWEError):
        P.Mesh(np.array([0.0, 1.0, 2.0]), np.array([0.0, 0.0, 0.0]), np.array([[0, 1, 2]]))  # degenerate


def test_regroup_rule_bit_exact(lib):
    """The library's CFL regroup rule against the oracle's, on random steps around
    the powers of two (including exact powers) and several substep counts."""
    import ctypes as C
    from oracle.mrab import cfl_regroup_levels
    rng = np.random.default_rng(9)
    K = 4000
    dt_min = 0.37
    for k, nl in ((24, 4), (8, 4), (12, 5), (7 * 16, 8), (3, 3)):
        ratio = np.exp2(rng.uniform(-1.5, 7.0, K))
        ratio[:40] = np.exp2(rng.integers(0, 7, 40))          # exact powers of two
        dt = np.ascontiguousarray(ratio * dt_min)
        old = np.ascontiguousarray(rng.integers(1, nl + 1, K).astype(np.int32))
        out = np.zeros(K, np.int32)
        margin = C.c_double()
        lib.check(lib.lib().swe_regroup_rule(lib.dptr(dt), lib.iptr(old), K, dt_min, k, nl, lib.iptr(out),
                                             C.byref(margin)), "swe_regroup_rule")
        olev, omargin = cfl_regroup_levels(dt, dt_min, old, k, nl)
        assert np.array_equal(out, olev)
        assert margin.value == omargin


def test_compensated_workspace_and_validation(lib):
    """swe_params.compensated: three more planes (eta, hu, hv) of Np x KS words on
    the single-precision tiers, nothing in FP64, anything but 0 or 1 refused."""
    import paper_1403_1661_gb300 as P
    vx, vy, E = meshes.structured_rect(0.0, 1.0, 0.0, 1.0, 9, 7)
    m = P.Mesh(vx, vy, E)
    K, N = m.K, 3
    Np, KS = (N + 1) * (N + 2) // 2, (K + 31) // 32 * 32

    def nbytes(precision, comp):
        prm = lib.swe_params(9.81, 1e-5, 0.0, 0.0, 1.5, 0.5, N, 1, precision, 1, 0, lib.SWE_SCHEME_CUBATURE, comp)
        out = C.c_size_t()
        rc = lib.lib().swe_workspace_bytes(m.handle, C.byref(prm), C.byref(out))
        return rc, out.value

    for prec in (lib.SWE_FP32, lib.SWE_FP32_TC):
        rc0, b0 = nbytes(prec, 0)
        rc1, b1 = nbytes(prec, 1)
        assert rc0 == rc1 == lib.SWE_OK
        planes = 3 * Np * KS * 4
        assert planes <= b1 - b0 < planes + 256        # the planes, 256-byte aligned
    rc0, b0 = nbytes(lib.SWE_FP64, 0)
    rc1, b1 = nbytes(lib.SWE_FP64, 1)
    assert rc0 == rc1 == lib.SWE_OK and b0 == b1
    rc, _ = nbytes(lib.SWE_FP32, 2)
    assert rc == lib.SWE_EINVAL


def test_binding_checks_array_shapes(lib):
    """The Python layer refuses arrays whose shapes do not match the mesh before
    the library reads them (the C calls take bare pointers and sizes)."""
    from paper_1403_1661_gb300.solver import Mesh
    vx, vy, E = meshes.structured_rect(0, 1, 0, 1, 3, 3)
    with pytest.raises(ValueError):
        Mesh(vx, vy[:-1], E)
    with pytest.raises(ValueError):
        Mesh(vx, vy, E[:, :2])
    with pytest.raises(ValueError):
        Mesh(vx, vy, E.reshape(-1))
    m = Mesh(vx, vy, E)
    h = np.ones((m.K, 10))                    # N = 3: 10 nodes per element
    lev, dtm = m.levels(3, h, 0 * h, 0 * h, 9.81, 0.3, 3)
    assert lev.shape == (m.K,) and dtm > 0
    with pytest.raises(ValueError):
        m.levels(3, h[:-1], 0 * h[:-1], 0 * h[:-1], 9.81, 0.3, 3)
    with pytest.raises(ValueError):
        m.levels(2, h, 0 * h, 0 * h, 9.81, 0.3, 3)  # N = 2 has 6 nodes per element
    m.close()


def test_level_rules_refuse_invalid_input(lib):
    """The CFL level rule and the regroup rule refuse what they cannot order: a
    non-finite state (a NaN would otherwise drop out of the wave-speed maximum), a
    state with no positive depth, non-finite or non-positive element steps and
    current levels outside 1..nlevels_max."""
    import ctypes as C
    from paper_1403_1661_gb300.solver import Mesh
    vx, vy, E = meshes.structured_rect(0, 1, 0, 1, 4, 4)
    m = Mesh(vx, vy, E)
    h = np.ones((m.K, 6))
    z = np.zeros_like(h)
    lev, dtm = m.levels(2, h, z, z, 9.81, 0.3, 3)
    assert (lev >= 1).all() and np.isfinite(dtm) and dtm > 0
    for bad in (np.nan, np.inf):
        for which in range(3):
            arrs = [h.copy(), z.copy(), z.copy()]
            arrs[which][3, 2] = bad
            with pytest.raises(lib.SWEError) as ei:
                m.levels(2, *arrs, 9.81, 0.3, 3)
            assert ei.value.code == lib.SWE_EINVAL
    with pytest.raises(lib.SWEError) as ei:
        m.levels(2, 0 * h, z, z, 9.81, 0.3, 3)           # dry everywhere
    assert ei.value.code == lib.SWE_EINVAL
    m.close()

    K = 16
    dt = np.full(K, 0.5)
    old = np.ones(K, np.int32)
    out = np.zeros(K, np.int32)
    margin = C.c_double()

    def rule(dt, old, dt_min=0.25, nl=3):
        return lib.lib().swe_regroup_rule(lib.dptr(dt), lib.iptr(old), K, dt_min, 8, nl, lib.iptr(out),
                                          C.byref(margin))
    assert rule(dt, old) == lib.SWE_OK and (out == 2).all()
    for v in (np.nan, np.inf, 0.0, -1.0):
        d = dt.copy()
        d[5] = v
        assert rule(d, old) == lib.SWE_EINVAL
    for v in (0, -1, 4):
        o = old.copy()
        o[7] = v
        assert rule(dt, o) == lib.SWE_EINVAL
    assert rule(dt, old, dt_min=np.inf) == lib.SWE_EINVAL
