"""The kernel-structure ablations of R(Q) (Section 7) through the C ABI.

* Every variant against the FP64 oracle on the graded, jittered bump case, N = 2..5,
  within the tolerance of the arithmetic it runs in (the SIMT variants of an
  SWE_FP32_TC solver run in plain FP32).
* The SIMT variants equal each other bit for bit (same arithmetic, operators in
  shared or global memory); the three-kernel split equals the fused SIMT kernel up
  to the order of the volume and surface sums.
* Argument checks: unknown variant, missing or small scratch, a state that is not
  level-synchronous.
"""
import numpy as np
import pytest

from tests.gpu_helpers import both
from tests.test_gpu_parity import TOL_R, _rhs_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()


def _rel(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(3))


@pytest.mark.parametrize("N", [2, 3, 4, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32tc"])
def test_variants_match_oracle(N, precision):
    from paper_1403_1661_gb300 import _native as nat
    scn = _rhs_case(N, precision, limiter_mask=1)
    om, ref, model, integ, s = both(scn, precision)
    q = integ.q_end
    R_o = model.rhs(q[0], q[1], q[2])
    R = {v: s.rhs_variant(v).cpu().numpy().astype(np.float64)
         for v in (nat.SWE_RHS_FUSED, nat.SWE_RHS_FUSED_SIMT, nat.SWE_RHS_GLOBAL_OPS, nat.SWE_RHS_SPLIT)}
    assert np.array_equal(R[nat.SWE_RHS_FUSED], s.rhs().cpu().numpy().astype(np.float64))
    simt_tol = TOL_R["fp32" if precision == "fp32tc" else precision][N]
    errs = {v: _rel(R[v], R_o) for v in R}
    print(f"PARITY ablation N={N} {precision} " + " ".join(f"v{v}={e:.3e}" for v, e in errs.items()), flush=True)
    assert errs[nat.SWE_RHS_FUSED] < TOL_R[precision][N]
    for v in (nat.SWE_RHS_FUSED_SIMT, nat.SWE_RHS_GLOBAL_OPS, nat.SWE_RHS_SPLIT):
        assert errs[v] < simt_tol
    assert np.array_equal(R[nat.SWE_RHS_FUSED_SIMT], R[nat.SWE_RHS_GLOBAL_OPS])
    # the split adds the same terms in another order: a few units of the last place
    # of the largest partial sums
    split_tol = 1e-13 if precision == "fp64" else 2e-6
    assert _rel(R[nat.SWE_RHS_SPLIT], R[nat.SWE_RHS_FUSED_SIMT]) < split_tol


def test_variant_argument_checks():
    import torch
    from paper_1403_1661_gb300 import _native as nat
    scn = _rhs_case(3, "fp32")
    _, _, _, integ, s = both(scn, "fp32")
    need = s.rhs_scratch_bytes(nat.SWE_RHS_SPLIT)
    assert need > 0 and s.rhs_scratch_bytes(nat.SWE_RHS_GLOBAL_OPS) == 0
    with pytest.raises(nat.SWEError) as ei:
        s.rhs_scratch_bytes(7)
    assert ei.value.code == nat.SWE_EINVAL
    small = torch.empty(need - 256, dtype=torch.uint8, device=s.device)
    with pytest.raises(nat.SWEError) as ei:
        s.rhs_variant(nat.SWE_RHS_SPLIT, small)
    assert ei.value.code == nat.SWE_ENOMEM
    # host memory never reaches the kernels
    with pytest.raises(ValueError):
        s.rhs_variant(nat.SWE_RHS_SPLIT, torch.empty(need, dtype=torch.uint8))
    # a caller-provided scratch gives the same R as one allocated per call
    scratch = torch.empty(need, dtype=torch.uint8, device=s.device)
    a = s.rhs_variant(nat.SWE_RHS_SPLIT, scratch).cpu().numpy()
    b = s.rhs_variant(nat.SWE_RHS_SPLIT).cpu().numpy()
    assert np.array_equal(a, b)


def test_variant_requires_synchronous_state():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    from workloads import scenarios as sc
    scn = sc.tsunami(nx=24, ny=6, N=3, nlevels=3)
    s = P.solver_from_scenario(scn, precision="fp32")
    assert s.level_info()[0] >= 2
    s.substep(1)
    with pytest.raises(nat.SWEError) as ei:
        s.rhs_variant(nat.SWE_RHS_SPLIT)
    assert ei.value.code == nat.SWE_EINVAL
    s.substep(2 ** (s.level_info()[0] - 1) - 1)
    assert np.array_equal(s.rhs_variant(nat.SWE_RHS_FUSED_SIMT).cpu().numpy(), s.rhs().cpu().numpy())
