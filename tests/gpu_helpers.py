"""Shared set-up for the GPU parity tests: the same seeded scenario built on the
oracle side and on the CUDA side (the CUDA side uses the oracle's level
assignment so both follow the same multirate schedule; level grouping itself is
compared bit-exactly in test_lib_host.py)."""
import numpy as np

from oracle import problem


def both(scn, precision, levels=None, dt_min=None, mesh_arrays=None, scheme="cubature"):
    import paper_1403_1661_gb300 as P
    arrays = scn.build_mesh() if mesh_arrays is None else mesh_arrays
    om, ref, model, integ = problem.build(scn, levels=levels, dt_min=dt_min, mesh_arrays=arrays)
    if scheme != "cubature":
        from oracle.mrab import MRAB
        if scheme == "collocation":
            from oracle.colloc import CollocModel
            model = CollocModel(om, ref, model.B, scn.g, scn.h0)
        else:   # rules of integration order 2N, pre-balanced form
            from oracle.prebalanced import PreBalancedModel
            from oracle.refelem import RefElement
            ref = RefElement(scn.N, cub_degree=2 * scn.N, ng=scn.N + 1)
            model = PreBalancedModel(om, ref, model.B, scn.g, scn.h0)
        B, h, hu, hv = problem.nodal_inputs(scn, om, ref)
        integ = MRAB(model, h, hu, hv, integ.level, integ.dt_min, limiter_mask=scn.limiter_mask,
                     tvb_M=scn.tvb_M, tvb_nu=scn.tvb_nu, dry_mode=scn.dry_mode)
    solver = P.solver_from_scenario(scn, precision=precision, levels=integ.level, dt_min=integ.dt_min,
                                    mesh_arrays=arrays, scheme=scheme)
    return om, ref, model, integ, solver


def state_errors(solver, integ):
    """max-norm differences of (h, hu, hv) and the scales they are measured against."""
    h, hu, hv, t = solver.get_state()
    q = integ.q_end
    eh = np.abs(h - q[0]).max()
    em = max(np.abs(hu - q[1]).max(), np.abs(hv - q[2]).max())
    return eh, em, (h, hu, hv, t)
