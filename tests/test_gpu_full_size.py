"""Parity at the benchmark's full size: the 500,000-triangle N = 4 tsunami (4 MRAB
levels, positivity + TVB), FP32 tensor-core tier, built and launched exactly as
bench.py times it (solver_from_scenario, graph-replayed macro steps), against the
FP64 oracle on every element.

* R(Q) of the initial (limited) state, all 3 x 500,000 x 15 values, within the
  tensor-core tier's R tolerance relative to max|R| per field.
* The state after one macro step (8 finest substeps: every level, every
  multirate coupling, both limiters) within the tier's state tolerances. The
  free surface is also reported against the 2 m wave amplitude: the device keeps
  eta = h + B, so its error is the dynamics' and not the 4000 m depth's.

The oracle needs about a minute for the macro step; both sides are built once.
"""
import numpy as np
import pytest

from tests.gpu_helpers import both
from workloads import scenarios as sc

pytestmark = pytest.mark.gpu

# R per field relative to max|R| (the tier's derived bound; observed 4.3e-5 at this
# size and depth); one macro step: depth relative to max h, momentum relative to
# max h sqrt(g max h), free surface in metres (about ten times the observed errors)
TOL_R = 2e-4
TOL_STEP_H, TOL_STEP_M, TOL_STEP_ETA = 4e-7, 1.2e-10, 1e-5


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()
    scn = sc.tsunami()
    om, ref, model, integ, s = both(scn, "fp32tc")
    assert om.K == 500_000 and integ.L == 4
    integ.q_initial = integ.q_end.copy()     # the limited initial state, kept for later tests
    return scn, om, model, integ, s


def test_full_size_rhs_matches_oracle(full):
    scn, om, model, integ, s = full
    q = integ.q_end
    R_o = model.rhs(q[0], q[1], q[2])
    R_g = s.rhs().cpu().numpy().astype(np.float64)
    assert R_g.shape == R_o.shape == (3, 500_000, 15)
    errs = [np.abs(R_g[c] - R_o[c]).max() / np.abs(R_o[c]).max() for c in range(3)]
    print("PARITY full-size rhs fp32tc", " ".join(f"{e:.3e}" for e in errs), flush=True)
    assert np.isfinite(R_g).all()
    assert max(errs) < TOL_R


def test_full_size_macro_step_matches_oracle(full):
    scn, om, model, integ, s = full
    period = 2 ** (integ.L - 1)
    d_o, d_g = integ.dof_updates, s.stats()["dof_updates"]
    for _ in range(period):
        integ.substep()
    s.step(1)
    h, hu, hv, t = s.get_state()
    q = integ.q_end
    assert abs(t - integ.time) < 1e-12 * integ.time
    assert s.stats()["dof_updates"] - d_g == integ.dof_updates - d_o
    hmax = q[0].max()
    eh = np.abs(h - q[0]).max()
    em = max(np.abs(hu - q[1]).max(), np.abs(hv - q[2]).max())
    B32 = model.B.astype(np.float32).astype(np.float64)    # the bed as the device holds it
    deta = np.abs((h + B32) - (q[0] + model.B)).max()
    print(f"PARITY full-size macro step fp32tc eh={eh / hmax:.3e} em={em / (hmax * np.sqrt(9.81 * hmax)):.3e} "
          f"deta={deta:.3e} m (wave amplitude 2 m)", flush=True)
    assert np.isfinite(h).all() and h.min() >= -1e-6
    assert eh < TOL_STEP_H * hmax and em < TOL_STEP_M * hmax * np.sqrt(9.81 * hmax)
    assert deta < TOL_STEP_ETA


@pytest.mark.parametrize("scheme", ["collocation", "cubature_2n"])
def test_full_size_rhs_other_schemes(full, scheme):
    """R of the 500,000-triangle initial state with the collocation scheme and with
    the order-2N rules (tensor-core tier, as bench.py times them) against their oracles."""
    import paper_1403_1661_gb300 as P
    scn, om, model, integ, _ = full
    if scheme == "collocation":
        from oracle.colloc import CollocModel
        m2, ref2 = CollocModel(om, model.ref, model.B, scn.g, scn.h0), model.ref
    else:
        from oracle.prebalanced import PreBalancedModel
        from oracle.refelem import RefElement
        ref2 = RefElement(scn.N, cub_degree=2 * scn.N, ng=scn.N + 1)
        m2 = PreBalancedModel(om, ref2, model.B, scn.g, scn.h0)
    s = P.solver_from_scenario(scn, precision="fp32tc", levels=integ.level, dt_min=integ.dt_min, scheme=scheme)
    q = integ.q_initial                      # the limited initial state (the limiter is the same)
    R_o = m2.rhs(q[0], q[1], q[2])
    R_g = s.rhs().cpu().numpy().astype(np.float64)
    errs = [np.abs(R_g[c] - R_o[c]).max() / np.abs(R_o[c]).max() for c in range(3)]
    print(f"PARITY full-size rhs {scheme} fp32tc", " ".join(f"{e:.3e}" for e in errs), flush=True)
    assert np.isfinite(R_g).all()
    assert max(errs) < TOL_R
