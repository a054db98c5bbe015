"""Pins for the oracle's right-hand side: well-balancing, brute force, flux
properties, conservation and convergence (Sections 2, 3, 5.1, 6)."""
import math

import numpy as np
import pytest

from oracle.mesh import Mesh
from oracle.mrab import MRAB
from oracle.refelem import RefElement
from oracle.swe import SWEModel, wb_lf_flux
from tests.quadrature_helpers import physical_triangle_rule
from workloads import meshes, scenarios as sc

G = 9.81


def _setup(N, gen, bed):
    vx, vy, E = gen()
    m = Mesh(vx, vy, E)
    ref = RefElement(N)
    x, y = m.map_to_physical(ref.r, ref.s)
    cx = np.repeat(m.cx[:, None], ref.Np, 1)
    cy = np.repeat(m.cy[:, None], ref.Np, 1)
    return m, ref, x, y, bed(x, y, cx, cy)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("bedname", ["smooth", "discontinuous"])
def test_lake_at_rest_is_exact(N, bedname):
    """Exact C-property (Section 5.1): still water over any bed gives R = 0."""
    bed = sc.smooth_bump_bed() if bedname == "smooth" else sc.step_bed_by_centroid(0.5, -2.0, -1.2, 0.3)
    gen = lambda: meshes.graded_jittered_rect(0, 1, 0, 1, 6, 5, ratio=2, jitter=0.2, seed=1)
    m, ref, x, y, B = _setup(N, gen, bed)
    h = 0.5 - B
    model = SWEModel(m, ref, B, G, 1e-5)
    R = model.rhs(h, 0 * h, 0 * h)
    scale = G * h.max() ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max(), np.abs(m.sx).max())
    assert np.abs(R).max() < 1e-13 * scale * ref.Np


def _ref_flux(hm, mum, mvm, Bm, hp, mup, mvp, Bp, nx, ny, g, h0):
    """Independent restatement of the well-balanced LLF normal flux (Eq. well_balance)."""
    out = np.zeros((3,) + np.shape(hm))
    for idx in np.ndindex(np.shape(hm)):
        a = [float(v[idx]) for v in (hm, mum, mvm, Bm, hp, mup, mvp, Bp, nx, ny)]
        hM, mxM, myM, BM, hP, mxP, myP, BP, n1, n2 = a
        uM, vM = (mxM / hM, myM / hM) if hM > h0 else (0.0, 0.0)
        uP, vP = (mxP / hP, myP / hP) if hP > h0 else (0.0, 0.0)
        bmax = max(BM, BP)
        sM = max(0.0, hM + BM - bmax)
        sP = max(0.0, hP + BP - bmax)

        def fn(s, u, v):
            un = u * n1 + v * n2
            return np.array([s * un, s * u * un + 0.5 * g * s * s * n1, s * v * un + 0.5 * g * s * s * n2])
        lam = max(abs(uM * n1 + vM * n2) + math.sqrt(g * sM), abs(uP * n1 + vP * n2) + math.sqrt(g * sP))
        f = 0.5 * (fn(sM, uM, vM) + fn(sP, uP, vP)) - 0.5 * lam * (
            np.array([sP, sP * uP, sP * vP]) - np.array([sM, sM * uM, sM * vM]))
        f[1] += 0.5 * g * (hM * hM - sM * sM) * n1
        f[2] += 0.5 * g * (hM * hM - sM * sM) * n2
        out[(slice(None),) + idx] = f
    return out


def test_flux_against_restatement_and_properties():
    rng = np.random.default_rng(3)
    n = 200
    hm, hp = rng.uniform(0, 2, n), rng.uniform(0, 2, n)
    hm[:20] = 0.0
    hp[20:40] = 1e-7
    mum, mvm, mup, mvp = rng.normal(size=(4, n))
    Bm, Bp = rng.normal(size=(2, n))
    th = rng.uniform(0, 2 * np.pi, n)
    nx, ny = np.cos(th), np.sin(th)
    got = np.array(wb_lf_flux(hm, mum, mvm, Bm, hp, mup, mvp, Bp, nx, ny, G, 1e-5))
    ref = _ref_flux(hm, mum, mvm, Bm, hp, mup, mvp, Bp, nx, ny, G, 1e-5)
    assert np.abs(got - ref).max() < 1e-12
    # consistency with the physical flux on a flat bed
    hw = rng.uniform(0.5, 2, n)
    f = np.array(wb_lf_flux(hw, mum, mvm, 0 * hw, hw, mum, mvm, 0 * hw, nx, ny, G, 1e-5))
    u, v = mum / hw, mvm / hw
    un = u * nx + v * ny
    exact = np.array([hw * un, mum * un + 0.5 * G * hw ** 2 * nx, mvm * un + 0.5 * G * hw ** 2 * ny])
    assert np.abs(f - exact).max() < 1e-12
    # conservation on a flat bed: F(a, b, n) = -F(b, a, -n)
    f1 = np.array(wb_lf_flux(hm, mum, mvm, 0 * hm, hp, mup, mvp, 0 * hm, nx, ny, G, 1e-5))
    f2 = np.array(wb_lf_flux(hp, mup, mvp, 0 * hm, hm, mum, mvm, 0 * hm, -nx, -ny, G, 1e-5))
    assert np.abs(f1 + f2).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3, 4])
def test_rhs_bruteforce_two_elements(N):
    """R from the oracle equals a brute-force evaluation of the weak form (Eq. weak_form)
    in a physical monomial basis with a 21x21-point rule: constant depth per element
    (polynomial fluxes), linear bed, different states on the two elements, walls."""
    vx = np.array([0.0, 1.3, 1.1, -0.1])
    vy = np.array([0.0, 0.1, 0.9, 1.2])
    E = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    m = Mesh(vx, vy, E)
    ref = RefElement(N)
    h0 = 1e-5
    x, y = m.map_to_physical(ref.r, ref.s)
    rng = np.random.default_rng(40 + N)
    bcoef = (-2.0, 0.3, -0.2)
    bed = lambda X, Y: bcoef[0] + bcoef[1] * X + bcoef[2] * Y
    mons = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    hconst = [1.7, 1.4]
    mcoef = [[{mn: 0.3 * rng.normal() for mn in mons} for _ in range(2)] for _ in range(2)]

    def state(k, X, Y):
        X0, Y0 = X - 0.5, Y - 0.5
        hu = sum(c * X0 ** a * Y0 ** b for (a, b), c in mcoef[k][0].items())
        hv = sum(c * X0 ** a * Y0 ** b for (a, b), c in mcoef[k][1].items())
        return np.full(np.shape(X), hconst[k]), hu, hv

    h = np.zeros((2, ref.Np)); hu = np.zeros_like(h); hv = np.zeros_like(h)
    for k in range(2):
        h[k], hu[k], hv[k] = state(k, x[k], y[k])
    B = bed(x, y)
    R = SWEModel(m, ref, B, G, h0).rhs(h, hu, hv)

    tg, wg = np.polynomial.legendre.leggauss(ref.Ng)
    for k in range(2):
        xv, yv = m.xv[k], m.yv[k]
        X, Y, W = physical_triangle_rule(xv, yv, 21)
        sc_ = 1.0
        phi = np.stack([((X - 0.5) / sc_) ** a * ((Y - 0.5) / sc_) ** b for (a, b) in mons])
        phix = np.stack([a * (X - 0.5) ** max(a - 1, 0) * (Y - 0.5) ** b if a else 0 * X for (a, b) in mons])
        phiy = np.stack([b * (X - 0.5) ** a * (Y - 0.5) ** max(b - 1, 0) if b else 0 * X for (a, b) in mons])
        hh, mx, my = state(k, X, Y)
        u, v = mx / hh, my / hh
        F = [mx, mx * u + 0.5 * G * hh ** 2, mx * v]
        Gf = [my, my * u, my * v + 0.5 * G * hh ** 2]
        S = [0 * X, -G * hh * bcoef[1], -G * hh * bcoef[2]]
        rhs = np.zeros((3, len(mons)))
        for c in range(3):
            rhs[c] = (phix * F[c] + phiy * Gf[c] + phi * S[c]) @ W
        # faces: same Gauss rule as the method, everything else recomputed here
        for f, (a_, b_) in enumerate(((0, 1), (1, 2), (2, 0))):
            dx, dy = xv[b_] - xv[a_], yv[b_] - yv[a_]
            L = math.hypot(dx, dy)
            nx, ny = dy / L, -dx / L
            Xg = xv[a_] + (1 + tg) / 2 * dx
            Yg = yv[a_] + (1 + tg) / 2 * dy
            hM, mM, nM = state(k, Xg, Yg)
            BM = bed(Xg, Yg)
            nb = m.EToE[k, f]
            if nb >= 0:
                hP, mP, nP = state(nb, Xg, Yg)
                BP = bed(Xg, Yg)
            else:
                mn = mM * nx + nM * ny
                hP, mP, nP, BP = hM, mM - 2 * mn * nx, nM - 2 * mn * ny, BM
            Fn = _ref_flux(hM, mM, nM, BM, hP, mP, nP, BP, np.full_like(Xg, nx), np.full_like(Xg, ny), G, h0)
            phig = np.stack([(Xg - 0.5) ** a * (Yg - 0.5) ** b for (a, b) in mons])
            for c in range(3):
                rhs[c] -= phig @ (wg * L / 2 * Fn[c])
        Gram = (phi * W) @ phi.T
        coef = np.linalg.solve(Gram, rhs.T).T
        phin = np.stack([(x[k] - 0.5) ** a * (y[k] - 0.5) ** b for (a, b) in mons])
        Rb = coef @ phin
        assert np.abs(Rb - R[:, k, :]).max() < 1e-10 * max(1.0, np.abs(Rb).max())


def test_mass_conserved_with_walls():
    s = sc.hump_square(n=8, N=3, steps=30)
    from oracle import problem
    mesh, ref, model, integ = problem.build(s)
    m0 = model.mass(integ.q_end[0])
    for _ in range(30):
        integ.substep()
        assert abs(model.mass(integ.q_end[0]) - m0) < 1e-14 * m0 * 10


def _vortex(beta=5.0, x0=0.0, y0=0.0):
    """Translating vortex of Section 6.2 (gamma = 2, g = 2)."""
    def exact(x, y, t):
        r2 = (x - t - x0) ** 2 + (y - y0) ** 2
        e = np.exp(1.0 - r2)
        h = 1.0 - beta ** 2 / (32.0 * np.pi ** 2) * e ** 2
        u = 1.0 - beta * e * (y - y0) / (2.0 * np.pi)
        v = beta * e * (x - t - x0) / (2.0 * np.pi)
        return h, h * u, h * v
    return exact


def _vortex_error(N, nx, ny, T, cfl):
    from oracle.mesh import element_dt
    exact = _vortex()
    vx, vy, E = meshes.structured_rect(-5, 10, -6, 6, nx, ny)
    m = Mesh(vx, vy, E)
    ref = RefElement(N)
    x, y = m.map_to_physical(ref.r, ref.s)
    h, hu, hv = exact(x, y, 0.0)
    model = SWEModel(m, ref, np.zeros_like(h), 2.0, 1e-8, dirichlet=exact)
    dt = element_dt(m, N, h, hu, hv, 2.0, cfl).min()
    nsteps = int(math.ceil(T / dt))
    dt = T / nsteps
    integ = MRAB(model, h, hu, hv, np.ones(m.K, int), dt)
    for _ in range(nsteps):
        integ.substep()
    he, _, _ = exact(x, y, T)
    err = integ.q_end[0] - he
    # L2 norm with the mass matrix
    e2 = np.einsum("ki,ij,kj->k", err, ref.M, err) * m.J
    return math.sqrt(e2.sum()), 15.0 / nx


@pytest.mark.parametrize("N", [2, 3, pytest.param(4, marks=pytest.mark.slow)])
def test_vortex_convergence(N):
    """Smooth translating vortex: least-squares EOC >= N + 0.3 on the two finest
    meshes (H = 0.75, 0.375); Section 6.2 reports O(H^{N+1/2})."""
    errs, hs = [], []
    for n in (20, 40):
        e, H = _vortex_error(N, n, int(n * 12 / 15 + 0.5), T=0.5, cfl=0.25)
        errs.append(e)
        hs.append(H)
    eoc = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert eoc >= N + 0.3, (errs, eoc)
