"""Pins of the oracle's level regrouping (Section 4's remark; reading in MRAB.regroup).

* The re-interpolated history is exact for an R history that is a quadratic in time
  (closed form), for moves one level coarser and one and two levels finer.
* Regrouping to the same levels changes nothing (bit for bit).
* A regroup keeps the scheme third order: against the run that keeps its levels,
  the difference falls like dt^3 (a restart with the Euler start-up falls like
  dt^2 and is far larger).
* The CFL regroup rule on hand-made steps.
"""
import numpy as np
import pytest

from oracle import problem
from oracle.mrab import MRAB, cfl_regroup_levels
from workloads import scenarios as sc


@pytest.fixture(scope="module")
def small():
    scn = sc.hump_square(n=8, N=2)
    om, ref, model, integ = problem.build(scn)
    rng = np.random.default_rng(1)
    levA = rng.integers(1, 3, om.K)
    levB = levA.copy()
    flip = rng.random(om.K) < 0.4
    levB[flip] = 3 - levA[flip]
    return model, integ.q_end.copy(), integ.dt_min, levA, levB


def test_regroup_history_exact_for_quadratic_in_time(small):
    model, q0, dt, levA, _ = small
    K = q0.shape[1]
    lev = np.where(np.arange(K) % 3 == 0, 3, levA)      # levels 1..3
    m = MRAB(model, q0[0], q0[1], q0[2], lev, dt)
    for _ in range(4 * 4):                              # k = 16 >= 3 * 2^(3-1)
        m.substep()
    k = m.k
    rng = np.random.default_rng(2)
    c = rng.standard_normal((3,) + q0.shape)           # R(t) = c0 + c1 t + c2 t^2 per value
    R = lambda t: c[0] + c[1] * t + c[2] * t * t
    for e in range(K):
        a, dl = k >> (lev[e] - 1), dt * 2 ** (lev[e] - 1)
        for s in (1, 2, 3):
            m.hist[(a - s) % 3, :, e] = R(m.time - s * dl)[:, e]
    new = lev.copy()
    new[lev == 1] = 2                                   # one level coarser
    new[(lev == 2) & (np.arange(K) % 2 == 0)] = 1       # one level finer
    new[lev == 3] = 1                                   # two levels finer
    m.regroup(new)
    assert m.L == 2 and np.array_equal(m.count, k >> (new - 1))
    for e in range(K):
        a, dl = k >> (new[e] - 1), dt * 2 ** (new[e] - 1)
        for s in (1, 2):
            np.testing.assert_allclose(m.hist[(a - s) % 3, :, e], R(m.time - s * dl)[:, e], rtol=1e-12, atol=1e-12)


def test_regroup_to_same_levels_is_identity(small):
    model, q0, dt, levA, _ = small
    a = MRAB(model, q0[0], q0[1], q0[2], levA, dt)
    b = MRAB(model, q0[0], q0[1], q0[2], levA, dt)
    for _ in range(8):
        a.substep()
        b.substep()
    b.regroup(levA)
    for _ in range(8):
        a.substep()
        b.substep()
    assert np.array_equal(a.q_end, b.q_end)


def test_regroup_keeps_third_order(small):
    model, q0, dt0, levA, levB = small

    def run(f, mode):
        m = MRAB(model, q0[0], q0[1], q0[2], levA, dt0 / f)
        for _ in range(16 * f):
            m.substep()
        if mode == "regroup":
            m.regroup(levB)
        elif mode == "restart":
            m = MRAB(model, m.q_end[0], m.q_end[1], m.q_end[2], levB, dt0 / f)
        for _ in range(16 * f):
            m.substep()
        return m.q_end

    d_reg = [np.abs(run(f, "regroup") - run(f, "none")).max() for f in (2, 4)]
    d_rst = np.abs(run(4, "restart") - run(4, "none")).max()
    assert d_reg[0] / d_reg[1] > 6.0          # third order (8); a restart gives 4
    assert d_reg[1] < d_rst / 20


def test_regroup_argument_checks(small):
    model, q0, dt, levA, levB = small
    m = MRAB(model, q0[0], q0[1], q0[2], levA, dt)
    for _ in range(4):
        m.substep()
    with pytest.raises(ValueError):
        m.regroup(levB)                        # k = 4 < 3 * 2^(2-1)
    m.substep()
    with pytest.raises(ValueError):
        m.regroup(levB)                        # not level-synchronous
    m.substep()
    with pytest.raises(ValueError):
        m.regroup(np.full_like(levB, 4))       # 2^3 does not divide k = 6


def test_cfl_regroup_rule():
    dt_min = 1.0
    dt = np.array([0.7, 1.0, 1.9, 2.0, 5.0, 9.0, 100.0, 3.0])
    level = np.array([1, 1, 1, 1, 1, 3, 1, 2])
    lev, margin = cfl_regroup_levels(dt, dt_min, level, k=12, nlevels=4)
    # CFL levels 1 1 1 2 3 4 4 2; at most one coarser: 1 1 1 2 2 4 2 2; k = 12 = 4 * 3 -> at most 3
    assert lev.tolist() == [1, 1, 1, 2, 2, 3, 2, 2]
    assert margin == pytest.approx(0.7)
    lev, _ = cfl_regroup_levels(dt, dt_min, level, k=8, nlevels=4)
    assert lev.tolist() == [1, 1, 1, 2, 2, 4, 2, 2]
