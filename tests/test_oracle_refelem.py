"""Pins for the oracle's reference element (closed forms, brute force, invariants)."""
import math

import numpy as np
import pytest

from oracle import refelem as R
from tests.quadrature_helpers import duffy_rule, simplex_monomial_integral

ORDERS = [1, 2, 3, 4, 5]


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10])
def test_gauss_legendre_exact(n):
    x, w = R.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # and not exact one degree higher (the rule is Gaussian, not better)
    k = 2 * n
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-8


@pytest.mark.parametrize("n", [1, 3, 6, 8])
def test_gauss_jacobi_10_exact(n):
    x, w = R.gauss_jacobi(n, 1.0, 0.0)
    for k in range(2 * n):
        # int_{-1}^{1} (1-x) x^k dx
        ek = 0.0 if k % 2 else 2.0 / (k + 1)
        ek1 = 0.0 if (k + 1) % 2 else 2.0 / (k + 2)
        assert abs(np.sum(w * x ** k) - (ek - ek1)) < 1e-13


@pytest.mark.parametrize("deg", [1, 2, 5, 8, 11, 14])
def test_conical_cubature_monomials(deg):
    r, s, w = R.conical_cubature(deg)
    l0, l1, l2 = -(r + s) / 2, (1 + r) / 2, (1 + s) / 2
    assert abs(w.sum() - 2.0) < 1e-14
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                got = np.sum(w * l0 ** a * l1 ** b * l2 ** c)
                assert abs(got - simplex_monomial_integral(a, b, c)) < 1e-14


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_count_edges_and_symmetry(N):
    r, s = R.warp_blend_nodes(N)
    Np = (N + 1) * (N + 2) // 2
    assert r.size == Np
    # edge nodes are the Gauss-Lobatto-Legendre points (numpy's Legendre routine)
    if N >= 2:
        gll_in = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
    else:
        gll_in = np.array([])
    gll = np.concatenate([[-1.0], gll_in, [1.0]])
    e0 = np.sort(r[np.abs(s + 1) < 1e-12])
    assert np.allclose(e0, gll, atol=1e-13)
    e2 = np.sort(s[np.abs(r + 1) < 1e-12])
    assert np.allclose(e2, gll, atol=1e-13)
    e1 = np.sort(s[np.abs(r + s) < 1e-12])
    assert np.allclose(e1, gll, atol=1e-13)
    # symmetric under every permutation of the barycentric coordinates
    L = np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=1)
    key = lambda M: sorted(map(tuple, np.round(M, 10)))
    for p in [(1, 0, 2), (0, 2, 1), (2, 1, 0), (1, 2, 0), (2, 0, 1)]:
        assert key(L[:, p]) == key(L)
    if N <= 2:  # Warp & Blend with alpha = 0 and N <= 2 is the equidistant lattice
        assert np.allclose(np.sort(np.round(L * N, 12), axis=0), np.sort(np.round(L * N), axis=0))


def _into_triangle(r, s):
    """Nearest-ish point of the reference triangle (fold across r + s = 0, clamp at -1)."""
    d = np.maximum(r + s, 0.0) / 2
    return np.maximum(r - d, -1.0), np.maximum(s - d, -1.0)


def _lebesgue_constant(N, alpha, monkeypatch, M=150, keep=8, rounds=3):
    """max over the triangle of sum_i |l_i| for the Warp & Blend nodes with blend
    parameter alpha: a lattice of spacing 2/M (containing the centroid), then the
    `keep` largest lattice values refined by three nested 21x21 local searches."""
    table = list(R._ALPHA_OPT)
    table[N - 1] = alpha
    monkeypatch.setattr(R, "_ALPHA_OPT", table)
    rn, sn = R.warp_blend_nodes(N)
    Vi = np.linalg.inv(R.vandermonde(N, rn, sn))
    leb = lambda r, s: np.abs(R.vandermonde(N, r, s) @ Vi).sum(axis=1)
    i, j = np.meshgrid(np.arange(M + 1), np.arange(M + 1), indexing="ij")
    m = i + j <= M
    r, s = -1 + 2 * j[m] / M, -1 + 2 * i[m] / M
    v = leb(r, s)
    best = v.max()
    d = np.linspace(-1.0, 1.0, 21)
    for idx in np.argsort(v)[-keep:]:
        cr, cs, h = r[idx], s[idx], 2.0 / M
        for _ in range(rounds):
            pr, ps = _into_triangle(cr + h * d[:, None] + 0 * d[None, :], cs + h * d[None, :] + 0 * d[:, None])
            pv = leb(pr.ravel(), ps.ravel())
            k = int(np.argmax(pv))
            best = max(best, pv[k])
            cr, cs, h = pr.ravel()[k], ps.ravel()[k], h / 10
    return best


@pytest.mark.parametrize("N", [5, 6, 7])
def test_blend_parameter_minimises_lebesgue_constant(N, monkeypatch):
    """The blend parameters alpha_opt(N) were chosen (Warburton 2006) to minimise
    the Lebesgue constant of the node set. For N = 5..7 the tabulated value is that
    minimiser to within 0.002: a wrong digit in the first three decimals fails."""
    a0 = R._ALPHA_OPT[N - 1]
    lam0 = _lebesgue_constant(N, a0, monkeypatch)
    for da in (-0.002, 0.002):
        assert _lebesgue_constant(N, a0 + da, monkeypatch) > lam0 + 1e-5, da
    # and it is the global minimum over a coarse scan of alpha in [0, 2]
    scan = [_lebesgue_constant(N, a, monkeypatch) for a in np.arange(0.0, 2.01, 0.25)]
    assert lam0 < min(scan)


def test_blend_parameter_n4_on_the_flat_lebesgue_curve(monkeypatch):
    """For N = 4 the Lebesgue constant hardly depends on alpha (its maximum lies
    next to the alpha-independent edge nodes): the tabulated 0.1001 is within 1e-4
    (relative) of the minimum over alpha in [0, 2], which a misplaced digit
    (1.001, 0.01 is fine) breaks by far (1.001 gives +0.5 %)."""
    a0 = R._ALPHA_OPT[3]
    lam0 = _lebesgue_constant(4, a0, monkeypatch)
    scan = [_lebesgue_constant(4, a, monkeypatch) for a in np.arange(0.0, 2.01, 0.1)]
    assert lam0 <= min(scan) * (1 + 1e-4)
    assert _lebesgue_constant(4, 1.001, monkeypatch) > min(scan) * (1 + 2e-3)


@pytest.mark.parametrize("N", ORDERS)
def test_basis_orthonormal_bruteforce(N):
    r, s, w = duffy_rule(N + 3)
    V = R.vandermonde(N, r, s)
    G = V.T @ (w[:, None] * V)
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-12


@pytest.mark.parametrize("N", ORDERS)
def test_grad_basis_finite_difference(N):
    rng = np.random.default_rng(0)
    r0 = rng.uniform(-0.9, 0.2, 7)
    s0 = rng.uniform(-0.9, 0.0, 7)
    e = 1e-6
    gr, gs = R.grad_vandermonde(N, r0, s0)
    fdr = (R.vandermonde(N, r0 + e, s0) - R.vandermonde(N, r0 - e, s0)) / (2 * e)
    fds = (R.vandermonde(N, r0, s0 + e) - R.vandermonde(N, r0, s0 - e)) / (2 * e)
    assert np.abs(gr - fdr).max() < 1e-7 * max(1, np.abs(gr).max())
    assert np.abs(gs - fds).max() < 1e-7 * max(1, np.abs(gs).max())


def _poly(r, s, coef):
    return sum(c * r ** a * s ** b for (a, b), c in coef.items())


def _poly_dr(r, s, coef):
    return sum(c * a * r ** (a - 1) * s ** b for (a, b), c in coef.items() if a > 0)


def _poly_ds(r, s, coef):
    return sum(c * b * r ** a * s ** (b - 1) for (a, b), c in coef.items() if b > 0)


@pytest.mark.parametrize("N", ORDERS)
def test_interpolation_operators_exact_on_PN(N):
    ref = R.RefElement(N)
    rng = np.random.default_rng(N)
    coef = {(a, b): rng.normal() for a in range(N + 1) for b in range(N + 1 - a)}
    q = _poly(ref.r, ref.s, coef)
    assert np.abs(ref.Ic @ q - _poly(ref.rc, ref.sc, coef)).max() < 1e-12
    assert np.abs(ref.Icr @ q - _poly_dr(ref.rc, ref.sc, coef)).max() < 1e-11
    assert np.abs(ref.Ics @ q - _poly_ds(ref.rc, ref.sc, coef)).max() < 1e-11
    for f, (fr, fs) in enumerate(R.face_points(ref.tg)):
        assert np.abs(ref.Ig[f] @ q - _poly(fr, fs, coef)).max() < 1e-12
    # derivative rows annihilate constants
    assert np.abs(ref.Icr.sum(axis=1)).max() < 1e-12
    assert np.abs(ref.Ics.sum(axis=1)).max() < 1e-12


@pytest.mark.parametrize("N", ORDERS)
def test_projection_operators_are_weak_derivatives(N):
    """M Pr f = integral of (d l_i/dr) f for a polynomial f of degree 2N-1
    (brute force with an independent rule)."""
    ref = R.RefElement(N)
    rng = np.random.default_rng(10 + N)
    coef = {(a, b): rng.normal() for a in range(2 * N) for b in range(2 * N - a)}
    fc = _poly(ref.rc, ref.sc, coef)
    r, s, w = duffy_rule(3 * N + 2)
    f = _poly(r, s, coef)
    I = ref.interp_matrix(r, s)
    Vr, Vs = R.grad_vandermonde(N, r, s)
    Ir, Is = Vr @ ref.invV, Vs @ ref.invV
    assert np.abs(ref.M @ (ref.Pr @ fc) - Ir.T @ (w * f)).max() < 1e-11
    assert np.abs(ref.M @ (ref.Ps @ fc) - Is.T @ (w * f)).max() < 1e-11
    assert np.abs(ref.M @ (ref.P @ fc) - I.T @ (w * f)).max() < 1e-11


REF_NORMALS = [(0.0, -1.0), (1 / math.sqrt(2), 1 / math.sqrt(2)), (-1.0, 0.0)]
REF_SJ = [1.0, math.sqrt(2), 1.0]      # half the reference face lengths


@pytest.mark.parametrize("N", ORDERS)
def test_lift_bruteforce_and_discrete_divergence(N):
    ref = R.RefElement(N)
    rng = np.random.default_rng(20 + N)
    # lift: M Lg_f g = integral over face f of l_i g (t) dt for g of degree <= 2N
    tb, wb = np.polynomial.legendre.leggauss(40)
    for f, (fr, fs) in enumerate(R.face_points(tb)):
        c = rng.normal(size=2 * N + 1)
        g_b = np.polynomial.polynomial.polyval(tb, c)
        g_g = np.polynomial.polynomial.polyval(ref.tg, c)
        lhs = ref.M @ (ref.Lg[f] @ g_g)
        rhs = ref.interp_matrix(fr, fs).T @ (wb * g_b)
        assert np.abs(lhs - rhs).max() < 1e-12
    # constant flux (a, b): volume part + lifted normal flux = 0 (reference geometry)
    a, b = 0.7, -1.3
    vol = ref.Pr @ np.full(ref.Ncub, a) + ref.Ps @ np.full(ref.Ncub, b)
    srf = sum(REF_SJ[f] * ref.Lg[f] @ np.full(ref.Ng, a * REF_NORMALS[f][0] + b * REF_NORMALS[f][1])
              for f in range(3))
    assert np.abs(vol - srf).max() < 1e-12


@pytest.mark.parametrize("N", ORDERS)
def test_pi1_and_mean(N):
    ref = R.RefElement(N)
    rng = np.random.default_rng(30 + N)
    q = rng.normal(size=ref.Np)
    P1 = ref.Pi1
    assert np.abs(P1 @ P1 - P1).max() < 1e-12
    assert abs(ref.mean_w @ (P1 @ q) - ref.mean_w @ q) < 1e-13
    lin = 0.3 + 1.1 * ref.r - 0.4 * ref.s
    assert np.abs(P1 @ lin - lin).max() < 1e-12
    # Pi1 is the L2 projection: the residual is orthogonal to P1
    resid = q - P1 @ q
    for basis_fn in (np.ones_like(ref.r), ref.r, ref.s):
        assert abs(basis_fn @ ref.M @ resid) < 1e-12
    # mean of monomials against the Dirichlet integral
    l1 = (1 + ref.r) / 2
    l2 = (1 + ref.s) / 2
    if N >= 2:
        assert abs(ref.mean_w @ (l1 * l2) - simplex_monomial_integral(0, 1, 1) / 2) < 1e-14
    assert abs(ref.mean_w.sum() - 1.0) < 1e-14
    # vertices
    assert np.allclose(np.c_[ref.r, ref.s][ref.vertex_nodes], R.REF_VERTS)
