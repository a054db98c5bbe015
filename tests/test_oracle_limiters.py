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


# ---------------------------------------------------------------------------
# Two-sided pins of the two theta's: the limiters must be minimal (the lowest vertex
# lands exactly on h0), not merely positive, and must leave alone what needs no
# limiting. An over-limiting theta (theta = 0, or theta from the P^N minimum instead
# of the P1 vertex minimum) fails the equality pins; an under-limiting one fails the
# positivity pins above.


def _single_element_model(N, h0=1e-3):
    """One reference-shaped triangle (vertices (0,0), (1,0), (0,1)), flat bed."""
    vx = np.array([0.0, 1.0, 0.0])
    vy = np.array([0.0, 0.0, 1.0])
    m = Mesh(vx, vy, np.array([[0, 1, 2]]))
    ref = RefElement(N)
    x, y = m.map_to_physical(ref.r, ref.s)
    return SWEModel(m, ref, np.zeros_like(x), G, h0), x, y


def test_pp_theta_hand_computed_p1_element():
    """Algorithm 3 on one P1 element whose vertex values are chosen by hand:
    h = (-0.1, 0.5, 0.8), mean 0.4, h0 = 1e-3, so theta = (0.4 - 1e-3) / (0.4 + 0.1)
    = 0.798; the limited vertex values are theta (v - mean) + mean, the lowest equal
    to h0; the momenta (1, 2, 3) are scaled about their mean by the same theta."""
    model, x, y = _single_element_model(1)
    vn = model.ref.vertex_nodes
    h = np.zeros((1, 3))
    hu = np.zeros((1, 3))
    hv = np.zeros((1, 3))
    h[0, vn] = [-0.1, 0.5, 0.8]
    hu[0, vn] = [1.0, 2.0, 3.0]
    hv[0, vn] = [-3.0, 0.0, 0.0]
    h2, hu2, hv2, dry, inj = pp_limit(model, h, hu, hv)
    theta = 0.399 / 0.5
    assert not dry[0] and inj == 0.0
    assert np.allclose(h2[0, vn], [theta * -0.5 + 0.4, theta * 0.1 + 0.4, theta * 0.4 + 0.4], atol=1e-15)
    assert abs(h2[0, vn].min() - 1e-3) < 1e-15
    assert np.allclose(hu2[0, vn], [theta * -1.0 + 2.0, 2.0, theta * 1.0 + 2.0], atol=1e-15)
    assert np.allclose(hv2[0, vn], [theta * -2.0 - 1.0, theta * 1.0 - 1.0, theta * 1.0 - 1.0], atol=1e-15)


def test_pp_theta_uses_p1_vertex_minimum_not_nodal_minimum():
    """N = 2 element whose depth is quadratic: its nodal minimum (an edge-midpoint
    node) is below h0 and below the P1 vertex minimum. Algorithm 3 (reading: h1_min
    over the vertices of the P1 projection) gives theta from the P1 vertex values,
    computed here from an independent least-squares P1 fit."""
    model, x, y = _single_element_model(2)
    ref = model.ref
    # a linear depth minus a quadratic dip that vanishes on edges 1 and 2: its lowest
    # node (-0.1) is the midpoint of edge 0, its vertices are 0.3, 0.5, 0.4
    h = 0.3 + 0.2 * x + 0.1 * y - 2.0 * x * (1.0 - x - y)
    hu = 0.5 + x
    hv = 0.2 - y
    assert h.min() <= model.h0
    h2, hu2, hv2, dry, inj = pp_limit(model, h, hu, hv)
    # exact P1 projection of a polynomial through the reference-element L2 inner
    # product, evaluated by a cubature independent of the oracle's: degree-4 rule of
    # 6 points on the unit triangle (Strang-Fix), mapped from the monomials
    a, b = 0.445948490915965, 0.091576213509771
    w1, w2 = 0.223381589678011 / 2, 0.109951743655322 / 2
    P = np.array([[a, a], [1 - 2 * a, a], [a, 1 - 2 * a], [b, b], [1 - 2 * b, b], [b, 1 - 2 * b]])
    W = np.array([w1] * 3 + [w2] * 3)
    f = lambda X, Y: 0.3 + 0.2 * X + 0.1 * Y - 2.0 * X * (1.0 - X - Y)
    V = np.stack([np.ones(6), P[:, 0], P[:, 1]], axis=1)
    coef = np.linalg.solve(V.T @ (W[:, None] * V), V.T @ (W * f(P[:, 0], P[:, 1])))
    verts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    h1v = coef[0] + coef[1] * verts[:, 0] + coef[2] * verts[:, 1]
    hbar = W @ f(P[:, 0], P[:, 1]) / W.sum()
    theta = min(1.0, (hbar - model.h0) / (hbar - h1v.min()))
    vn = ref.vertex_nodes
    # vertex order of the oracle's element: (0,0), (1,0), (0,1)
    assert np.allclose(np.stack([x[0, vn], y[0, vn]], 1), verts, atol=1e-14)
    assert theta < 1.0 and not dry[0]
    assert np.allclose(h2[0, vn], theta * (h1v - hbar) + hbar, atol=1e-13)
    assert abs(h2[0].min() - model.h0) < 1e-13


def test_pp_minimal_on_random_elements():
    """On every limited element with theta < 1 the lowest vertex of the result is
    exactly h0; where theta = 1 (a nodal value triggered the limiter but the P1
    vertices are all at or above h0) the result is the P1 projection itself."""
    model, x, y = _model(N=4)
    ref = model.ref
    rng = np.random.default_rng(7)
    K = model.mesh.K
    h = 0.05 + 0.2 * rng.normal(size=(K, ref.Np))
    hu, hv = rng.normal(size=(2, K, ref.Np))
    h2, hu2, hv2, dry, inj = pp_limit(model, h, hu, hv)
    trig = h.min(axis=1) <= model.h0
    vn = ref.vertex_nodes
    p1 = [a @ ref.Pi1.T for a in (h, hu, hv)]
    hbar = h @ ref.mean_w
    v1min = p1[0][:, vn].min(axis=1)
    lim = trig & ~dry
    full = lim & (v1min >= model.h0)        # theta = 1: exactly the P1 projection
    part = lim & (v1min < model.h0)         # theta < 1: minimal limiting
    assert part.sum() > 5 and full.sum() > 0
    assert np.abs(h2[part][:, vn].min(axis=1) - model.h0).max() < 1e-13
    for a2, a1 in zip((h2, hu2, hv2), p1):
        assert np.abs(a2[full] - a1[full]).max() < 1e-13
    # the same theta for all fields: (q2 - qbar) = theta (q1 - qbar) for each field
    theta = (hbar[part] - model.h0) / (hbar[part] - v1min[part])
    for a, a2, a1 in zip((h, hu, hv), (h2, hu2, hv2), p1):
        qb = (a @ ref.mean_w)[part][:, None]
        assert np.abs((a2[part] - qb) - theta[:, None] * (a1[part] - qb)).max() < 1e-12
    # untriggered elements are untouched
    assert np.array_equal(h2[~trig], h[~trig])


def test_tvb_positivity_modification_hand_computed():
    """Eq. modified_TVB on hand-chosen deltas: hb = 0.1, deltas (0.05, -0.2, 0.1).
    Vertex offsets S = (d0 + d2 - d1, d1 + d0 - d2, d2 + d1 - d0) = (0.35, -0.25,
    -0.15); the lowest vertex 0.1 - 0.25 < h0 = 1e-3, so
    theta = (hb + dbar - h0) / (dbar - min S) with dbar = -0.05/3, and the modified
    lowest vertex is exactly h0. A second element already positive is left as is."""
    from oracle.limiters import positivity_modify
    h0 = 1e-3
    hb = np.array([0.1, 0.5])
    dh = np.array([[0.05, -0.2, 0.1], [0.05, -0.2, 0.1]])
    out = positivity_modify(hb, dh, h0)
    dbar = -0.05 / 3.0
    theta = (0.1 + dbar - h0) / (dbar + 0.25)
    assert abs(theta - 0.3528571428571429) < 1e-13
    assert np.allclose(out[0], dbar + theta * (dh[0] - dbar), atol=1e-15)
    S = np.array([out[0, 0] + out[0, 2] - out[0, 1], out[0, 1] + out[0, 0] - out[0, 2],
                  out[0, 2] + out[0, 1] - out[0, 0]])
    assert abs(hb[0] + S.min() - h0) < 1e-15
    assert abs(out[0].mean() - dbar) < 1e-16
    assert np.allclose(out[1], dh[1], atol=1e-16)


def test_tvb_positivity_modification_minimal():
    """On the TVB limiter as a whole: run it once with the modification disabled
    (h0 far below any depth) and once with h0 = 0.037, inside the range of the
    thin layer's vertex depths. Elements whose unmodified P1
    vertex minimum lies below h0 come out with that minimum exactly at h0 and the
    other vertices on the closed form m + theta (v - m), m the mean of the vertex
    values (Eq. modified_TVB), theta clipped to [0, 1]; every other limited element
    is unchanged."""
    model, x, y = _model(N=3, h0=1e-3)
    ref, m = model.ref, model.mesh
    rng = np.random.default_rng(4)
    cx = np.repeat(m.cx[:, None], ref.Np, 1)
    h = np.where(cx < 3.0, 1.0, 0.04) + 0.05 * rng.normal(size=x.shape) * (cx < 3.0) \
        + 0.03 * np.sin(7 * x) * (cx >= 3.0)
    hu = 0.3 * rng.normal(size=x.shape)
    hv = 0.3 * rng.normal(size=x.shape)
    dry = np.zeros(m.K, bool)
    vn = ref.vertex_nodes
    off = SWEModel(m, ref, model.B, G, -1e300)
    hp, _, _, limp = tvb_limit(off, h, hu, hv, dry, M=0.0)
    hmod = 0.037
    on = SWEModel(m, ref, model.B, G, hmod)
    h2, _, _, lim2 = tvb_limit(on, h, hu, hv, dry, M=0.0)
    assert np.array_equal(limp, lim2)
    Vp = hp[limp][:, vn]
    V2 = h2[limp][:, vn]
    fired = Vp.min(axis=1) < hmod
    assert fired.sum() >= 3 and (~fired).sum() >= 3
    mv = Vp[fired].mean(axis=1, keepdims=True)
    # a mean at or above h0: the lowest vertex lands on h0; below it theta clips to 0
    # and the element becomes flat at its mean
    up = mv[:, 0] >= hmod
    assert up.sum() >= 2 and (~up).sum() >= 1
    assert np.abs(V2[fired][up].min(axis=1) - hmod).max() < 1e-12
    assert np.abs(V2[fired][~up] - mv[~up]).max() < 1e-13
    span = mv - Vp[fired].min(axis=1, keepdims=True)
    # a flat element (span 0) is left flat whatever theta is; take theta = 0 there
    theta = np.clip(np.divide(mv - hmod, span, out=np.zeros_like(span), where=span > 0), 0.0, 1.0)
    assert np.abs(V2[fired] - (mv + theta * (Vp[fired] - mv))).max() < 1e-12
    assert np.abs(V2[~fired] - Vp[~fired]).max() < 1e-13
    # the element means are the unmodified ones
    assert np.abs((h2[limp] - hp[limp]) @ ref.mean_w).max() < 1e-13


def test_tvb_steepened_linear_element_closed_form():
    """A linear state L with one interior element's deviation doubled:
    q_e = L(b0) + 2 (L - L(b0)). Its neighbour-mean stencil reproduces L's midpoint
    deltas exactly (alpha, beta are the barycentric weights of m_i - b0), so per
    characteristic component minmod(2w, nu w) = nu w with nu = 1.5, the deltas
    already sum to zero, and the rebuilt element is L(b0) + 1.5 (L - L(b0)) at every
    node (the vertex <-> edge-midpoint map and the stencil both enter). Every other
    element is left as it was."""
    model, x, y = _model(N=3, jitter=0.2, h0=1e-3)
    m, ref = model.mesh, model.ref
    Lh = lambda X, Y: 2.0 + 0.10 * X - 0.05 * Y
    Lu = lambda X, Y: 0.3 + 0.04 * X + 0.02 * Y
    Lv = lambda X, Y: -0.2 - 0.03 * X + 0.05 * Y
    nearwall = np.zeros(m.K, bool)
    for f in range(3):
        nearwall |= m.EToE[:, f] < 0
    inner = np.nonzero(~nearwall)[0]
    # an element whose neighbours also have no boundary face
    e = next(k for k in inner if not any(nearwall[m.EToE[k, f]] for f in range(3)))
    fields = []
    for Lf in (Lh, Lu, Lv):
        q = Lf(x, y)
        c = Lf(m.cx[e], m.cy[e])
        q[e] = c + 2.0 * (q[e] - c)
        fields.append(q)
    dry = np.zeros(m.K, bool)
    h2, hu2, hv2, lim = tvb_limit(model, *fields, dry, M=0.0, nu=1.5)
    assert lim[e]
    for Lf, q2, q in zip((Lh, Lu, Lv), (h2, hu2, hv2), fields):
        c = Lf(m.cx[e], m.cy[e])
        assert np.abs(q2[e] - (c + 1.5 * (Lf(x[e], y[e]) - c))).max() < 1e-12
        others = np.arange(m.K) != e
        assert np.abs(q2[others & ~nearwall] - q[others & ~nearwall]).max() == 0.0
