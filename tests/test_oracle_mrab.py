"""Pins for the oracle's multirate Adams-Bashforth integrator (Algorithms 1, 2)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import problem
from oracle.mesh import Mesh, element_dt
from oracle.mrab import MRAB, ab_coefficients, ab_partial_coefficients
from oracle.refelem import RefElement
from oracle.swe import SWEModel
from workloads import meshes, scenarios as sc

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_ab3_coefficients_match_paper_values():
    assert np.allclose(ab_coefficients(3), GOLD["ab3_alpha"]["value"], rtol=0, atol=1e-15)
    for d in (1, 2, 3):
        assert np.allclose(ab_partial_coefficients(d, 1.0), ab_coefficients(d), atol=1e-15)


@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75])
def test_partial_coefficients_integrate_interpolant_exactly(theta):
    # R(tau) = a + b tau + c tau^2 sampled at tau = 0, -1, -2; integral over [0, theta]
    a, b, c = 0.7, -1.1, 0.4
    Rs = [a + b * t + c * t * t for t in (0.0, -1.0, -2.0)]
    exact = a * theta + b * theta ** 2 / 2 + c * theta ** 3 / 3
    got = sum(w * r for w, r in zip(ab_partial_coefficients(3, theta), Rs))
    assert abs(got - exact) < 1e-14
    Rl = [a + b * t for t in (0.0, -1.0)]
    got2 = sum(w * r for w, r in zip(ab_partial_coefficients(2, theta), Rl))
    assert abs(got2 - (a * theta + b * theta ** 2 / 2)) < 1e-14


def test_single_level_is_plain_ab3():
    s = sc.hump_square(n=6, N=2)
    mesh, ref, model, integ = problem.build(s)
    q = integ.q_end.copy()
    dt = integ.dt_min
    hist = []
    for n in range(12):
        R = model.rhs(q[0], q[1], q[2])
        hist.insert(0, R)
        co = ab_coefficients(min(len(hist), 3))
        q = q + dt * sum(c * r for c, r in zip(co, hist))
        hist = hist[:3]
        integ.substep()
        assert np.array_equal(q, integ.q_end)


def _hump_run(dt, T, levels_fn=None, N=2):
    s = sc.hump_square(n=6, N=N)
    vx, vy, E = s.build_mesh()
    mesh = Mesh(vx, vy, E)
    lev = np.ones(mesh.K, int) if levels_fn is None else levels_fn(mesh)
    _, _, model, integ = problem.build(s, levels=lev, dt_min=dt, mesh_arrays=(vx, vy, E))
    n = int(round(T / dt))
    L = int(lev.max())
    assert n % (2 ** (L - 1)) == 0
    for _ in range(n):
        integ.substep()
    return integ.q_end, model


@pytest.mark.parametrize("two_level", [False, True])
def test_temporal_convergence_global(two_level):
    """Global error in a dt sweep. The start-up of each level (one Euler step, one
    AB2 step) limits the global order to 2; the multirate coupling must not make it
    worse, and the two-level error stays close to the single-rate one."""
    lf = (lambda m: np.where(m.cx < 0.5, 1, 2)) if two_level else None
    T = 0.03                      # the CFL step of this mesh is about 1.7e-3
    dts = [T / 48, T / 96, T / 192]
    ref_q, model = _hump_run(T / 1536, T, lf)
    errs = [np.abs(_hump_run(d, T, lf)[0] - ref_q).max() for d in dts]
    rates = np.diff(np.log(errs)) / np.diff(np.log(dts))
    assert rates.min() > 1.85, (errs, rates)
    if two_level:
        # half the domain steps with 2 dt: at second order its error is about 4x
        ref1, _ = _hump_run(T / 1536, T, None)
        e1 = [np.abs(_hump_run(d, T, None)[0] - ref1).max() for d in dts]
        assert max(e / f for e, f in zip(errs, e1)) < 5.0


def test_ab3_step_local_error_is_fourth_order():
    """Once the history is full, one step has local error O(dt^4) (third-order method):
    history and state taken from an RK4 reference trajectory written here."""
    s = sc.hump_square(n=6, N=2)
    mesh, ref, model, integ0 = problem.build(s)
    q0 = integ0.q_end.copy()

    def f(q):
        return model.rhs(q[0], q[1], q[2])

    def rk4(q, dt, n):
        out = [q.copy()]
        for _ in range(n):
            k1 = f(q); k2 = f(q + dt / 2 * k1); k3 = f(q + dt / 2 * k2); k4 = f(q + dt * k3)
            q = q + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            out.append(q.copy())
        return out

    errs = []
    dts = [0.8e-3, 0.4e-3, 0.2e-3]
    for dt in dts:
        sub = 16
        traj = rk4(q0, dt / sub, 3 * sub)
        Q = [traj[i * sub] for i in range(4)]
        integ = MRAB(model, Q[2][0], Q[2][1], Q[2][2], np.ones(mesh.K, int), dt)
        integ.hist[0] = f(Q[0])
        integ.hist[1] = f(Q[1])
        integ.count[:] = 2
        integ.k = 2
        integ.substep()
        errs.append(np.abs(integ.q_end - Q[3]).max())
    rates = np.diff(np.log(errs)) / np.diff(np.log(dts))
    assert rates.min() > 3.6, (errs, rates)   # AB2 would give 3


def test_two_level_vortex_close_to_single_rate():
    from tests.test_oracle_rhs import _vortex
    exact = _vortex()
    vx, vy, E = meshes.structured_rect(-5, 10, -6, 6, 20, 16)
    m = Mesh(vx, vy, E)
    ref = RefElement(2)
    x, y = m.map_to_physical(ref.r, ref.s)
    h, hu, hv = exact(x, y, 0.0)
    T = 0.5
    dt = element_dt(m, 2, h, hu, hv, 2.0, 0.2).min()
    n = 2 * int(math.ceil(T / dt / 2))
    dt = T / n
    errs = []
    for lev in (np.ones(m.K, int), np.where(m.cx > 2.5, 2, 1)):
        model = SWEModel(m, ref, np.zeros_like(h), 2.0, 1e-8, dirichlet=exact)
        integ = MRAB(model, h, hu, hv, lev, dt)
        for _ in range(n):
            integ.substep()
        he, _, _ = exact(x, y, T)
        errs.append(np.abs(integ.q_end[0] - he).max())
    assert errs[1] < 2.0 * errs[0], errs
