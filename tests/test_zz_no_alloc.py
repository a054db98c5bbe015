"""swe_mass_hmin_static against swe_stats and a host reduction.

swe_mass_hmin_static exists for callers that may not allocate device memory
themselves (their device memory is owned by a host application with a fixed
arena, or they run next to latency-critical work that a cudaMalloc could stall by
synchronising the device). It reduces nodal depths the caller already holds on
the device, using a fixed scratch array inside the library, and must agree with
the solver's own swe_stats within the FP64 tolerance of the other GPU tests
(1e-11 relative). Calls in a row check that the shared scratch carries no state
from one call into the next: the later calls reduce fewer elements, so they launch
fewer blocks than the first, and a final pass that read more partial slots than its
own call wrote would pick up the first call's leftovers. This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _areas(mesh):
    vx, vy, E = mesh.vx, mesh.vy, mesh.EToV
    x, y = vx[E], vy[E]
    return 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))


def _call(lib, nat, torch, N, K, dev_h, dev_area):
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.swe_mass_hmin_static(N, K, C.c_void_p(dev_h.data_ptr()), C.c_void_p(dev_area.data_ptr()),
                                  C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert rc == nat.SWE_OK, lib.swe_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("N", [1, 3])
def test_static_scratch_reduction_matches_stats_twice(N):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    from workloads import scenarios as sc

    scn = sc.dam_break(nx=96, ny=12, N=N)
    s = P.solver_from_scenario(scn, precision="fp64")
    area = _areas(s.mesh)
    dev_area = torch.tensor(area, dtype=torch.float64, device="cuda")
    lib = nat.lib()
    for call in range(2):
        s.substep(7 + 5 * call)
        st = s.stats()
        h, _, _, _ = s.get_state()
        dev_h = torch.tensor(h, dtype=torch.float64, device="cuda")
        mass, hmin = _call(lib, nat, torch, N, s.K, dev_h, dev_area)
        assert abs(mass - st["mass"]) <= 1e-11 * abs(st["mass"]), (call, mass, st["mass"])
        assert abs(hmin - st["hmin"]) <= 1e-11 * np.abs(h).max(), (call, hmin, st["hmin"])
    # fewer elements than the first call (fewer blocks: 2304 elements take 9 blocks of
    # 256, these take 1 and 3), checked against a host reduction of the same rows with
    # the library's own mean weights
    wts = np.zeros(s.Np)
    assert lib.swe_ref_operator(N, 8, wts.ctypes.data_as(C.POINTER(C.c_double)), s.Np) == nat.SWE_OK
    for Ks in (200, 700):
        mass, hmin = _call(lib, nat, torch, N, Ks, dev_h, dev_area)
        ref_mass = float(np.sum(area[:Ks] * (h[:Ks] @ wts)))
        assert abs(mass - ref_mass) <= 1e-11 * abs(ref_mass), (Ks, mass, ref_mass)
        assert hmin == h[:Ks].min(), (Ks, hmin, h[:Ks].min())
    # a NaN depth is not hidden by the minimum
    hn = h.copy()
    hn[5, 1] = np.nan
    dev_hn = torch.tensor(hn, dtype=torch.float64, device="cuda")
    mass, hmin = _call(lib, nat, torch, N, s.K, dev_hn, dev_area)
    assert np.isnan(mass) and np.isnan(hmin)
    # sizes beyond the limit are refused with a message
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lib.swe_mass_hmin_static(6, s.K, C.c_void_p(dev_h.data_ptr()), C.c_void_p(dev_area.data_ptr()),
                                  C.c_void_p(out.data_ptr()), None)
    assert rc == nat.SWE_EINVAL and b"N must be" in lib.swe_last_error()
