"""Pins of the pre-balanced weak form (oracle/prebalanced.py).

* With the default rules (exact to degrees 3N - 1 and 3N) it equals the h form of
  oracle/swe.py on a moving state over a bed: the two forms differ by the static
  g B^2 / 2, which exact integration cancels against the source.
* With the rules of the integration order 2N (Fig. 2's caption: cubature of degree
  2N, N + 1 Gauss points) still water stays exactly at rest over smooth and
  discontinuous beds, where the h form with the same rules does not.
"""
import numpy as np
import pytest

from oracle import problem
from oracle.mesh import Mesh
from oracle.prebalanced import PreBalancedModel
from oracle.refelem import RefElement
from oracle.swe import SWEModel
from workloads import meshes, scenarios as sc


def _setup(N, bed, init, reduced):
    vx, vy, E = meshes.graded_jittered_rect(0.0, 1.0, 0.0, 1.0, 7, 5, ratio=2.0, jitter=0.2, seed=11)
    m = Mesh(vx, vy, E)
    ref = RefElement(N, cub_degree=2 * N, ng=N + 1) if reduced else RefElement(N)
    scn = sc.Scenario(name="p", N=N, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=0, tvb_M=0.0,
                      mesh=lambda: (vx, vy, E), bathymetry=bed, init=init)
    B, h, hu, hv = problem.nodal_inputs(scn, m, ref)
    return m, ref, B, h, hu, hv


def _moving(x, y, cx, cy, B):
    eta = 0.05 * np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / 0.05)
    h = eta - B
    return h, h * 0.3 * np.sin(3 * x + y), h * (-0.2) * np.cos(2 * y - x)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_prebalanced_equals_h_form_with_exact_rules(N):
    m, ref, B, h, hu, hv = _setup(N, sc.smooth_bump_bed(depth=1.0, amp=0.3), _moving, reduced=False)
    Rp = PreBalancedModel(m, ref, B, 9.81, 1e-5).rhs(h, hu, hv)
    Rh = SWEModel(m, ref, B, 9.81, 1e-5).rhs(h, hu, hv)
    scale = 9.81 * np.abs(h).max() ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max())
    assert np.abs(Rp - Rh).max() < 1e-12 * scale


@pytest.mark.parametrize("N", [2, 3, 4, 5])
@pytest.mark.parametrize("bed", ["smooth", "discontinuous"])
def test_reduced_rules_keep_still_water(N, bed):
    B = sc.smooth_bump_bed(depth=1.0, amp=0.3) if bed == "smooth" else sc.step_bed_by_centroid(0.5, -1.0, -0.8, 0.2)
    m, ref, Bn, h, hu, hv = _setup(N, B, lambda x, y, cx, cy, B: (0.3 - B, 0 * B, 0 * B), reduced=True)
    assert ref.Ncub == (N + 1) ** 2 and ref.Ng == N + 1
    scale = 9.81 * 1.3 ** 2 * max(np.abs(m.rx).max(), np.abs(m.sy).max())
    Rp = PreBalancedModel(m, ref, Bn, 9.81, 1e-5).rhs(h, hu, hv)
    assert np.abs(Rp).max() < 1e-12 * scale
    if bed == "smooth":       # the h form with the same rules is not balanced
        Rh = SWEModel(m, ref, Bn, 9.81, 1e-5).rhs(h, hu, hv)
        assert np.abs(Rh).max() > 1e-9 * scale
