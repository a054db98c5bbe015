"""Pins for the oracle's positivity-preserving limiter (Algorithm 3) and the TVB
limiter with its positivity modification (Section 5.3)."""
import numpy as np
import pytest

from oracle.limiters import _tvb_minmod, pp_limit, swe_eigenvectors, tvb_limit
from oracle.mesh import Mesh
from oracle.refelem import RefElement
from oracle.swe import SWEModel
from workloads import meshes

G = 9.81


def _model(N=3, nx=6, ny=5, B=None, h0=1e-3, jitter=0.2):
    vx, vy, E = meshes.graded_jittered_rect(0, 6, 0, 5, nx, ny, ratio=1.5, jitter=jitter, seed=5)
    m = Mesh(vx, vy, E)
    ref = RefElement(N)
    x, y = m.map_to_physical(ref.r, ref.s)
    Bn = np.zeros_like(x) if B is None else B(x, y)
    return SWEModel(m, ref, Bn, G, h0), x, y


def test_pp_identity_when_wet():
    model, x, y = _model()
    rng = np.random.default_rng(0)
    h = 1.0 + 0.3 * np.sin(x) * np.cos(y)
    hu, hv = rng.normal(size=(2,) + h.shape)
    h2, hu2, hv2, dry, inj = pp_limit(model, h, hu, hv)
    assert np.array_equal(h2, h) and np.array_equal(hu2, hu) and np.array_equal(hv2, hv)
    assert not dry.any() and inj == 0.0


def test_pp_partially_wet_positive_and_conservative():
    model, x, y = _model(N=4)
    ref = model.ref
    rng = np.random.default_rng(1)
    K = model.mesh.K
    h = 0.05 + 0.2 * rng.normal(size=(K, ref.Np))        # many negative nodes, most means > h0
    hu, hv = rng.normal(size=(2, K, ref.Np))
    h2, hu2, hv2, dry, inj = pp_limit(model, h, hu, hv)
    mw = ref.mean_w
    wet = ~dry
    hbar = h @ mw
    trig = h.min(axis=1) <= model.h0
    assert np.any(trig & wet)
    # means of all three fields are kept on wet/partially wet elements (Section 5.2)
    for a, b in ((h, h2), (hu, hu2), (hv, hv2)):
        assert np.abs((a @ mw - b @ mw)[wet]).max() < 1e-13
    # nodal depth >= h0 after limiting; limited elements are P1
    assert h2[wet].min() >= model.h0 - 1e-14
    lim = trig & wet
    assert np.abs(h2[lim] @ ref.Pi1.T - h2[lim]).max() < 1e-12
    # dry elements are reset and the injected mass is tallied
    assert np.all(h2[dry] == model.h0) and np.all(hu2[dry] == 0) and np.all(hv2[dry] == 0)
    area = model.mesh.area
    assert abs(inj - np.sum(area[dry] * (model.h0 - hbar[dry]))) < 1e-14
    assert abs((area * (h2 @ mw)).sum() - (area * hbar).sum() - inj) < 1e-12


def test_minmod():
    a = np.array([1.0, -1.0, 2.0, 0.5, 0.0, 3.0])
    b = np.array([2.0, -3.0, -1.0, 0.1, 1.0, 1.0])
    assert _tvb_minmod(a, b, 0.0).tolist() == [1.0, -1.0, 0.0, 0.1, 0.0, 1.0]
    assert _tvb_minmod(a, b, 2.5).tolist() == [1.0, -1.0, 2.0, 0.5, 0.0, 1.0]


def test_swe_eigenvectors():
    rng = np.random.default_rng(2)
    for _ in range(20):
        h, u, v = rng.uniform(0.1, 3), rng.normal(), rng.normal()
        th = rng.uniform(0, 2 * np.pi)
        nx, ny = np.cos(th), np.sin(th)
        c2 = G * h
        un = u * nx + v * ny
        # flux Jacobian n_x dF/dQ + n_y dG/dQ for Q = (h, hu, hv)
        A = np.array([[0.0, nx, ny],
                      [c2 * nx - u * un, un + u * nx, u * ny],
                      [c2 * ny - v * un, v * nx, un + v * ny]])
        R = swe_eigenvectors(np.array(h), np.array(u), np.array(v), nx, ny, G)
        lam = np.array([un - np.sqrt(c2), un, un + np.sqrt(c2)])
        assert np.abs(A @ R - R * lam[None, :]).max() < 1e-12


def test_tvb_constant_and_linear_states_unchanged():
    model, x, y = _model(N=3, jitter=0.25)
    m = model.mesh
    dry = np.zeros(m.K, bool)
    h = np.full_like(x, 1.3)
    out = tvb_limit(model, h, 0.2 + 0 * h, -0.1 + 0 * h, dry, M=0.0)
    assert not out[3].any()
    # a linear state: interior elements away from walls see consistent neighbour means
    h = 2.0 + 0.1 * x - 0.05 * y
    hu = 0.3 + 0.02 * y
    hv = -0.2 + 0.03 * x
    _, _, _, lim = tvb_limit(model, h, hu, hv, dry, M=0.0)
    nearwall = np.zeros(m.K, bool)
    for f in range(3):
        nb = m.EToE[:, f]
        nearwall |= nb < 0
    assert not lim[~nearwall].any()
    # with a large TVB constant nothing is limited at all
    _, _, _, lim = tvb_limit(model, h, hu, hv, dry, M=1e6)
    assert not lim.any()


def test_tvb_limits_jumps_keeps_means_and_positivity():
    model, x, y = _model(N=3, h0=1e-3)
    ref, m = model.ref, model.mesh
    mw = ref.mean_w
    rng = np.random.default_rng(4)
    cx = np.repeat(m.cx[:, None], ref.Np, 1)
    # a steep front plus noise, with a thin but wet layer on the right
    h = np.where(cx < 3.0, 1.0, 0.02) + 0.05 * rng.normal(size=x.shape) * (cx < 3.0) \
        + 0.015 * np.sin(7 * x) * (cx >= 3.0)
    hu = 0.3 * rng.normal(size=x.shape)
    hv = 0.3 * rng.normal(size=x.shape)
    dry = np.zeros(m.K, bool)
    h2, hu2, hv2, lim = tvb_limit(model, h, hu, hv, dry, M=0.0)
    assert lim.sum() > 5
    for a, b in ((h, h2), (hu, hu2), (hv, hv2)):
        assert np.abs((a @ mw) - (b @ mw)).max() < 1e-12
    # limited elements are P1 and their vertex depth is >= h0 (Eq. modified_TVB)
    assert np.abs(h2[lim] @ ref.Pi1.T - h2[lim]).max() < 1e-12
    assert h2[lim][:, ref.vertex_nodes].min() >= model.h0 - 1e-12
    # dry elements and their neighbours are skipped
    dry = np.zeros(m.K, bool)
    dry[np.nonzero(lim)[0][:3]] = True
    _, _, _, lim2 = tvb_limit(model, h, hu, hv, dry, M=0.0)
    skip = dry.copy()
    for f in range(3):
        nb = m.EToE[:, f]
        skip[nb >= 0] |= dry[nb[nb >= 0]]
    assert not lim2[skip].any()


def test_tvb_uses_free_surface_so_lake_at_rest_is_kept():
    """Reading: TVB acts on eta = h + B; still water over a curved bed is untouched."""
    bed = lambda X, Y: -2.0 + 0.5 * np.exp(-((X - 3) ** 2 + (Y - 2.5) ** 2))
    model, x, y = _model(N=3, B=bed)
    h = 0.3 - model.B
    dry = np.zeros(model.mesh.K, bool)
    h2, hu2, hv2, lim = tvb_limit(model, h, 0 * h, 0 * h, dry, M=0.0)
    assert np.abs(h2 - h).max() < 1e-12
