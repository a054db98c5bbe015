"""Verification on the GPU against a closed-form solution: the stationary vortex.

Section 6.2's vortex without its translation is an exact steady solution of the
shallow-water equations for g = 2: h = 1 - beta^2/(32 pi^2) e^2, velocity
beta e/(2 pi) (-y, x), e = exp(1 - r^2), in cyclostrophic balance
g dh/dr = u_theta^2 / r. Its velocity is ~1e-14 at r = 6, so reflecting walls on
[-6, 6]^2 leave it unchanged. The test runs every tier through the C ABI to
T = 0.5 on three meshes and checks the L2 error of h at T against the exact
solution (order N + 1 expected), and the FP64 tier's error against the oracle's
on the same mesh and steps.
"""
import math

import numpy as np
import pytest

from workloads import meshes, scenarios as sc

pytestmark = pytest.mark.gpu

G = 2.0
T = 0.5
CFL = 0.25


def _exact(x, y, beta=5.0):
    r2 = x ** 2 + y ** 2
    e = np.exp(1.0 - r2)
    h = 1.0 - beta ** 2 / (32.0 * np.pi ** 2) * e ** 2
    return h, h * (-beta * e * y / (2 * np.pi)), h * (beta * e * x / (2 * np.pi))


def _scenario(N, n):
    scn = sc.Scenario(name=f"vortex_N{N}_{n}", N=N, g=G, h0=1e-8, cfl=CFL, nlevels=1, limiter_mask=0,
                      tvb_M=0.0, mesh=lambda: meshes.structured_rect(-6, 6, -6, 6, n, n),
                      bathymetry=lambda x, y, cx, cy: 0.0 * x, init=None)
    scn.init = lambda x, y, cx, cy, B: _exact(x, y)
    return scn


def _steps(N, n):
    from oracle.mesh import Mesh, element_dt
    from oracle.refelem import RefElement
    vx, vy, E = meshes.structured_rect(-6, 6, -6, 6, n, n)
    m, ref = Mesh(vx, vy, E), RefElement(N)
    x, y = m.map_to_physical(ref.r, ref.s)
    h, hu, hv = _exact(x, y)
    dt = element_dt(m, N, h, hu, hv, G, CFL).min()
    ns = int(math.ceil(T / dt))
    return m, ref, x, y, ns, T / ns


def _l2(m, ref, err):
    return math.sqrt((np.einsum("ki,ij,kj->k", err, ref.M, err) * m.J).sum())


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()


def _gpu_error(N, n, precision):
    import paper_1403_1661_gb300 as P
    m, ref, x, y, ns, dt = _steps(N, n)
    s = P.solver_from_scenario(_scenario(N, n), precision=precision, levels=np.ones(m.K, np.int32), dt_min=dt)
    s.substep(ns)
    h, hu, hv, t = s.get_state()
    assert abs(t - T) < 1e-12
    return _l2(m, ref, h - _exact(x, y)[0])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
@pytest.mark.parametrize("N", [2, 3])
def test_stationary_vortex_converges(N, precision):
    errs = [_gpu_error(N, n, precision) for n in (12, 24, 48)]
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print(f"PARITY vortex N={N} {precision} errors " + " ".join(f"{e:.3e}" for e in errs)
          + " EOC " + " ".join(f"{v:.2f}" for v in eoc), flush=True)
    assert eoc[0] >= N + 0.3 and eoc[1] >= N + 0.3


@pytest.mark.parametrize("N", [2, 3])
def test_stationary_vortex_error_equals_oracle(N):
    from oracle.mrab import MRAB
    from oracle.swe import SWEModel
    n = 24
    m, ref, x, y, ns, dt = _steps(N, n)
    h, hu, hv = _exact(x, y)
    integ = MRAB(SWEModel(m, ref, np.zeros_like(h), G, 1e-8), h, hu, hv, np.ones(m.K, int), dt)
    for _ in range(ns):
        integ.substep()
    e_oracle = _l2(m, ref, integ.q_end[0] - h)
    e_gpu = _gpu_error(N, n, "fp64")
    assert abs(e_gpu - e_oracle) < 1e-6 * e_oracle
