"""swe_mass_hmin_static against swe_stats.

swe_mass_hmin_static exists for callers that may not allocate device memory
themselves (their device memory is owned by a host application with a fixed
arena, or they run next to latency-critical work that a cudaMalloc could stall by
synchronising the device). It reduces nodal depths the caller already holds on
the device, using a fixed scratch array inside the library, and must agree with
the solver's own swe_stats within the FP64 tolerance of the other GPU tests
(1e-11 relative). Two calls in a row check that the shared scratch carries no
state from one call into the next. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_scratch_reduction_matches_stats_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    from workloads import scenarios as sc

    scn = sc.dam_break(nx=48, ny=6, N=3)
    s = P.solver_from_scenario(scn, precision="fp64")
    vx, vy, E = s.mesh.vx, s.mesh.vy, s.mesh.EToV
    x, y = vx[E], vy[E]
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    dev_area = torch.tensor(area, dtype=torch.float64, device="cuda")
    lib = nat.lib()
    for call in range(2):
        s.substep(7 + 5 * call)
        st = s.stats()
        h, _, _, _ = s.get_state()
        dev_h = torch.tensor(h, dtype=torch.float64, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        rc = lib.swe_mass_hmin_static(scn.N, s.K, C.c_void_p(dev_h.data_ptr()), C.c_void_p(dev_area.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == nat.SWE_OK, lib.swe_last_error()
        torch.cuda.synchronize()
        mass, hmin = out.cpu().numpy()
        assert abs(mass - st["mass"]) <= 1e-11 * abs(st["mass"]), (call, mass, st["mass"])
        assert abs(hmin - st["hmin"]) <= 1e-11 * np.abs(h).max(), (call, hmin, st["hmin"])
    # sizes beyond the limit are refused with a message
    rc = lib.swe_mass_hmin_static(6, s.K, C.c_void_p(dev_h.data_ptr()), C.c_void_p(dev_area.data_ptr()),
                                  C.c_void_p(out.data_ptr()), None)
    assert rc == nat.SWE_EINVAL and b"N must be" in lib.swe_last_error()
