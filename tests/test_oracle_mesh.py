"""Pins for the oracle's connectivity, geometry and level grouping."""
import numpy as np
import pytest

from oracle.mesh import Mesh, assign_levels, element_dt
from oracle.refelem import RefElement
from workloads import meshes


def _bruteforce_connectivity(EToV):
    K = EToV.shape[0]
    fv = ((0, 1), (1, 2), (2, 0))
    E2E = -np.ones((K, 3), int)
    E2F = -np.ones((K, 3), int)
    for k in range(K):
        for f, (a, b) in enumerate(fv):
            s = {EToV[k, a], EToV[k, b]}
            for k2 in range(K):
                if k2 == k:
                    continue
                for f2, (a2, b2) in enumerate(fv):
                    if {EToV[k2, a2], EToV[k2, b2]} == s:
                        E2E[k, f], E2F[k, f] = k2, f2
    return E2E, E2F


@pytest.mark.parametrize("gen", [
    lambda: meshes.structured_rect(0, 1, 0, 1, 4, 3),
    lambda: meshes.graded_jittered_rect(0, 10, 0, 3, 6, 4, ratio=4, jitter=0.2, seed=7),
])
def test_connectivity_bruteforce(gen):
    vx, vy, E = gen()
    # scramble orientation of some triangles: the mesh must make them CCW
    E = E.copy()
    E[::3, 1], E[::3, 2] = E[::3, 2].copy(), E[::3, 1].copy()
    m = Mesh(vx, vy, E)
    E2E, E2F = _bruteforce_connectivity(m.EToV)
    assert np.array_equal(m.EToE, E2E)
    assert np.array_equal(m.EToF, E2F)
    inner = m.EToE >= 0
    k, f = np.nonzero(inner)
    assert np.array_equal(m.EToE[m.EToE[k, f], m.EToF[k, f]], k)
    assert np.all(m.J > 0)


def test_geometry():
    vx, vy, E = meshes.graded_jittered_rect(0, 10, 0, 3, 6, 4, ratio=4, jitter=0.2, seed=7)
    m = Mesh(vx, vy, E)
    assert abs(m.area.sum() - 30.0) < 1e-12
    # rx.. invert the affine map's Jacobian
    xr = (m.xv[:, 1] - m.xv[:, 0]) / 2
    xs = (m.xv[:, 2] - m.xv[:, 0]) / 2
    yr = (m.yv[:, 1] - m.yv[:, 0]) / 2
    ys = (m.yv[:, 2] - m.yv[:, 0]) / 2
    assert np.allclose(m.rx * xr + m.ry * yr, 1) and np.allclose(m.rx * xs + m.ry * ys, 0)
    assert np.allclose(m.sx * xr + m.sy * yr, 0) and np.allclose(m.sx * xs + m.sy * ys, 1)
    # unit outward normals; divergence theorem sum_f L_f n_f = 0
    assert np.allclose(np.hypot(m.nx, m.ny), 1)
    for f, (a, b) in enumerate(((0, 1), (1, 2), (2, 0))):
        mx = 0.5 * (m.xv[:, a] + m.xv[:, b]) - m.cx
        my = 0.5 * (m.yv[:, a] + m.yv[:, b]) - m.cy
        assert np.all(mx * m.nx[:, f] + my * m.ny[:, f] > 0)
    assert np.abs((m.L * m.nx).sum(1)).max() < 1e-12
    # neighbouring faces have opposite normals
    k, f = np.nonzero(m.EToE >= 0)
    assert np.allclose(m.nx[k, f], -m.nx[m.EToE[k, f], m.EToF[k, f]])


def test_face_point_map_matches_coordinates():
    vx, vy, E = meshes.graded_jittered_rect(0, 10, 0, 3, 5, 4, ratio=3, jitter=0.2, seed=2)
    m = Mesh(vx, vy, E)
    t, _ = np.polynomial.legendre.leggauss(5)
    perm, px, py = m.face_point_map(t)
    k, f = np.nonzero(m.EToE >= 0)
    k2, f2 = m.EToE[k, f], m.EToF[k, f]
    assert np.allclose(np.take_along_axis(px[k2, f2], perm[k, f], 1), px[k, f])
    assert np.allclose(np.take_along_axis(py[k2, f2], perm[k, f], 1), py[k, f])
    # with both faces counter-clockwise the match is the reversal g -> Ng-1-g
    assert np.all(perm[k, f] == np.arange(5)[::-1])


def test_assign_levels_closed_form():
    dt = np.array([1.0, 1.5, 1.999, 2.0, 3.9, 4.0, 7.0, 8.0, 100.0])
    lev, dtmin = assign_levels(dt, 4)
    assert dtmin == 1.0
    assert lev.tolist() == [1, 1, 1, 2, 2, 3, 3, 4, 4]
    lev2, _ = assign_levels(dt * 0.37, 2)
    assert lev2.tolist() == [1, 1, 1, 2, 2, 2, 2, 2, 2]


def test_element_dt_formula():
    vx, vy, E = meshes.structured_rect(0, 2, 0, 1, 2, 1)
    m = Mesh(vx, vy, E)
    ref = RefElement(2)
    h = np.full((m.K, ref.Np), 4.0)
    dt = element_dt(m, 2, h, 0 * h, 0 * h, g=1.0, cfl=0.9)
    # right isoceles triangles with legs 1: inradius = (2 - sqrt2)/2
    H = (2 - np.sqrt(2)) / 2
    assert np.allclose(dt, 0.9 / 9 * H / 2.0)
