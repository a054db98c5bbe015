"""Pins of the oracle's nodal-collocation variant (oracle/colloc.py).

* Still water over smooth and face-discontinuous beds: R = 0 (the pre-balanced
  pressure is linear in B at constant eta, so collocation loses nothing).
* Where every flux is a polynomial of degree <= N (velocity 0, linear eta and B,
  N >= 2) collocation is exact: R equals the cubature oracle's R, which integrates
  the same weak form exactly, and R_hu, R_hv equal the closed form -g h grad(eta).
* Face-node bookkeeping: the face nodes lie on their faces in order, and the lift of
  a constant unit flux on one face gives the face length's share of the mass
  (sum over nodes of M times the lift column = integral of the face basis).
"""
import numpy as np
import pytest

from oracle import problem
from oracle.colloc import CollocModel, face_node_indices
from oracle.refelem import RefElement
from workloads import meshes, scenarios as sc


def _case(N, bed, init):
    scn = sc.Scenario(name="c", N=N, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=0, tvb_M=0.0,
                      mesh=lambda: meshes.graded_jittered_rect(0.0, 1.0, 0.0, 1.0, 7, 5, ratio=2.0, jitter=0.2,
                                                               seed=11),
                      bathymetry=bed, init=init)
    om, ref, model, integ = problem.build(scn)
    return om, ref, model, CollocModel(om, ref, model.B, scn.g, scn.h0), integ.q_end


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("bed", ["smooth", "discontinuous"])
def test_colloc_lake_at_rest(N, bed):
    B = sc.smooth_bump_bed(depth=1.0, amp=0.3) if bed == "smooth" else sc.step_bed_by_centroid(0.5, -1.0, -0.8, 0.2)
    om, ref, model, cm, q = _case(N, B, lambda x, y, cx, cy, B: (0.3 - B, 0 * B, 0 * B))
    R = cm.rhs(q[0], q[1], q[2])
    assert np.abs(R).max() < 1e-12 * 9.81 * 1.3 ** 2 * np.abs(om.rx).max()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_colloc_exact_for_polynomial_fluxes(N):
    g = 9.81
    bed = lambda x, y, cx=None, cy=None: -1.0 + 0.2 * x - 0.1 * y
    eta = lambda x, y: 0.05 + 0.1 * x + 0.07 * y
    om, ref, model, cm, q = _case(N, bed, lambda x, y, cx, cy, B: (eta(x, y) - B, 0 * B, 0 * B))
    Rc = cm.rhs(q[0], q[1], q[2])
    Rq = model.rhs(q[0], q[1], q[2])
    # rounding scale: the pressure terms that cancel, g max(h)^2 max|grad r|
    scale = g * np.abs(q[0]).max() ** 2 * max(np.abs(om.rx).max(), np.abs(om.sy).max())
    assert np.abs(Rc - Rq).max() < 1e-12 * scale
    x, y = om.map_to_physical(ref.r, ref.s)
    h = eta(x, y) - bed(x, y)
    assert np.abs(Rc[0]).max() < 1e-12 * scale
    assert np.abs(Rc[1] - (-g * h * 0.1)).max() < 1e-12 * scale
    assert np.abs(Rc[2] - (-g * h * 0.07)).max() < 1e-12 * scale


@pytest.mark.parametrize("N", [2, 3, 5])
def test_colloc_face_nodes_and_lift(N):
    ref = RefElement(N)
    idx, ts = face_node_indices(ref)
    verts = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])
    for f in range(3):
        assert len(idx[f]) == N + 1
        a, b = verts[f], verts[(f + 1) % 3]
        # ordered from vertex f to vertex f+1
        assert np.allclose([ref.r[idx[f][0]], ref.s[idx[f][0]]], a)
        assert np.allclose([ref.r[idx[f][-1]], ref.s[idx[f][-1]]], b)
        assert np.all(np.diff(ts[f]) > 0)
    om, r2, model, cm, q = _case(N, sc.flat_bed(1.0), lambda x, y, cx, cy, B: (1.0 + 0 * x, 0 * x, 0 * x))
    # M * lift of a unit flux on face f, summed over nodes = integral over the face of
    # sum_i l_i = 2 (face parameter length)
    for f in range(3):
        tot = (ref.M @ cm.Lc[f] @ np.ones(N + 1)).sum()
        assert abs(tot - 2.0) < 1e-12
