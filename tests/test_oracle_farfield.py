"""Pins of the far-field boundary (a constant ghost state at every boundary face).

* Free stream: a uniform moving state over a flat bed, with the same state in the
  far field, has R = 0 to round-off (with walls instead it does not), and the TVB
  limiter leaves it unchanged.
* A state at rest over a bed with still water in the far field at the same level:
  R = 0 (well-balanced through the boundary faces).
"""
import numpy as np

from oracle.limiters import tvb_limit
from oracle.mesh import Mesh
from oracle.refelem import RefElement
from oracle.swe import SWEModel
from workloads import meshes


def _mesh():
    vx, vy, E = meshes.graded_jittered_rect(0.0, 1.0, 0.0, 1.0, 7, 5, ratio=2.0, jitter=0.2, seed=11)
    return Mesh(vx, vy, E)


def test_free_stream_is_preserved():
    m, ref = _mesh(), RefElement(3)
    h = np.full((m.K, ref.Np), 1.3)
    hu, hv = 0.4 * h, -0.25 * h
    B = np.full_like(h, -1.3)
    ff = SWEModel(m, ref, B, 9.81, 1e-5, farfield=(1.3, 0.4 * 1.3, -0.25 * 1.3))
    R = ff.rhs(h, hu, hv)
    scale = 9.81 * 1.3 ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max())
    assert np.abs(R).max() < 1e-13 * scale
    walls = SWEModel(m, ref, B, 9.81, 1e-5)
    assert np.abs(walls.rhs(h, hu, hv)).max() > 1e-3 * scale
    h2, hu2, hv2, lim = tvb_limit(ff, h, hu, hv, np.zeros(m.K, bool), M=0.0)
    assert np.array_equal(h2, h) and np.array_equal(hu2, hu) and np.array_equal(hv2, hv)


def test_still_water_through_far_field_faces():
    """Still water over a bump whose support lies inside the domain: the boundary
    faces see the flat bed, so the far field at the same level keeps R = 0."""
    m, ref = _mesh(), RefElement(3)
    x, y = m.map_to_physical(ref.r, ref.s)
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    B = -1.0 + 0.3 * np.maximum(0.0, 1.0 - r2 / 0.09) ** 2
    eta0 = 0.2
    h = eta0 - B
    ff = SWEModel(m, ref, B, 9.81, 1e-5, farfield=(eta0 + 1.0, 0.0, 0.0))
    R = ff.rhs(h, 0 * h, 0 * h)
    scale = 9.81 * 1.3 ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max())
    assert np.abs(R).max() < 1e-13 * scale
    # a far field at another level is not at rest
    ff2 = SWEModel(m, ref, B, 9.81, 1e-5, farfield=(eta0 + 1.1, 0.0, 0.0))
    assert np.abs(ff2.rhs(h, 0 * h, 0 * h)).max() > 1e-6 * scale


def test_mixed_faces_open_and_walls():
    """Open faces on the left and right sides, walls at the bottom and top: a stream
    along x with the same far field is at rest in R only if the walls are parallel
    to it (they are), and a stream along y is not (the walls reflect it)."""
    m, ref = _mesh(), RefElement(3)
    opn = np.zeros((m.K, 3), bool)
    for f in range(3):
        bnd = m.EToE[:, f] < 0
        opn[:, f] = bnd & (np.abs(m.nx[:, f]) > 0.5)      # faces on x = 0 and x = 1
    h = np.full((m.K, ref.Np), 1.3)
    B = np.full_like(h, -1.3)
    scale = 9.81 * 1.3 ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max())
    along_x = SWEModel(m, ref, B, 9.81, 1e-5, farfield=(1.3, 0.5 * 1.3, 0.0), farfield_faces=opn)
    assert np.abs(along_x.rhs(h, 0.5 * h, 0 * h)).max() < 1e-13 * scale
    along_y = SWEModel(m, ref, B, 9.81, 1e-5, farfield=(1.3, 0.0, 0.5 * 1.3), farfield_faces=opn)
    assert np.abs(along_y.rhs(h, 0 * h, 0.5 * h)).max() > 1e-3 * scale
    h2, hu2, hv2, _ = tvb_limit(along_x, h, 0.5 * h, 0 * h, np.zeros(m.K, bool), M=0.0)
    assert np.array_equal(hu2, 0.5 * h)
