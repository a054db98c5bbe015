"""Assemble an oracle run from a scenario description (test infrastructure only)."""
from __future__ import annotations

import numpy as np

from .mesh import Mesh, assign_levels, element_dt
from .mrab import MRAB
from .refelem import RefElement
from .swe import SWEModel


def nodal_inputs(scn, mesh: Mesh, ref: RefElement):
    """Evaluate the scenario's bathymetry and initial state at the oracle's nodes."""
    x, y = mesh.map_to_physical(ref.r, ref.s)
    cx = np.repeat(mesh.cx[:, None], ref.Np, axis=1)
    cy = np.repeat(mesh.cy[:, None], ref.Np, axis=1)
    B = np.asarray(scn.bathymetry(x, y, cx, cy), np.float64)
    h, hu, hv = scn.init(x, y, cx, cy, B)
    return B, np.asarray(h, np.float64), np.asarray(hu, np.float64), np.asarray(hv, np.float64)


def build(scn, levels=None, dt_min=None, mesh_arrays=None):
    """Mesh, reference element, model and integrator for ``scn``.

    ``levels``/``dt_min`` override the CFL-based grouping (used by tests that force
    an assignment)."""
    vx, vy, EToV = scn.build_mesh() if mesh_arrays is None else mesh_arrays
    mesh = Mesh(vx, vy, EToV)
    ref = RefElement(scn.N)
    B, h, hu, hv = nodal_inputs(scn, mesh, ref)
    model = SWEModel(mesh, ref, B, scn.g, scn.h0)
    if levels is None:
        dt = element_dt(mesh, scn.N, h, hu, hv, scn.g, scn.cfl)
        levels, dtm = assign_levels(dt, scn.nlevels)
        if dt_min is None:
            dt_min = dtm
    integ = MRAB(model, h, hu, hv, levels, dt_min, limiter_mask=scn.limiter_mask,
                 tvb_M=scn.tvb_M, tvb_nu=scn.tvb_nu, dry_mode=scn.dry_mode)
    return mesh, ref, model, integ
