"""The weak form in the pre-balanced free-surface variables with any volume and face
rules (oracle, FP64; test infrastructure only).

eta = h + B; F = (hu, hu u + p, hu v), G = (hv, hv u, hv v + p) with
p = g/2 (eta^2 - 2 eta B); S = (0, -g eta B_x, -g eta B_y); the numerical flux is the
well-balanced LLF flux of Section 5.1 minus the own side's static (g/2) (B^-)^2 n.
In exact arithmetic this is Eq. swe_conservative (p differs from g h^2 / 2 by the
static g B^2 / 2, whose divergence the source's -g B grad B cancels), and with rules
exact to degrees 3N - 1 (volume) and 3N (faces) it equals SWEModel's h form to
rounding. With cheaper rules the two forms differ, and this one keeps still water
exactly at rest as long as the rules are exact to degree 2N - 1 (volume) and 2N
(faces): at constant eta, p is linear in B.

Used for the reduced-rule scheme: the integration order 2N that the caption of
Fig. 2 gives for its rules (volume cubature of degree 2N, N + 1 Gauss points per
face).
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh
from .refelem import RefElement
from .swe import SWEModel, velocity, wb_lf_flux


class PreBalancedModel(SWEModel):
    def __init__(self, mesh: Mesh, ref: RefElement, B, g: float, h0: float):
        super().__init__(mesh, ref, B, g, h0)

    def volume(self, h, hu, hv):
        ref, m, g = self.ref, self.mesh, self.g
        ec = (h + self.B) @ ref.Ic.T
        hc = h @ ref.Ic.T
        huc, hvc = hu @ ref.Ic.T, hv @ ref.Ic.T
        u, v = velocity(hc, huc, self.h0), velocity(hc, hvc, self.h0)
        p = 0.5 * g * (ec * ec - 2.0 * ec * self.Bc)
        F = (huc, huc * u + p, huc * v)
        G = (hvc, hvc * u, hvc * v + p)
        S = (np.zeros_like(hc), -g * ec * self.Bx, -g * ec * self.By)
        out = []
        for c in range(3):
            cF1 = m.rx[:, None] * F[c] + m.ry[:, None] * G[c]
            cF2 = m.sx[:, None] * F[c] + m.sy[:, None] * G[c]
            out.append(cF1 @ ref.Pr.T + cF2 @ ref.Ps.T + S[c] @ ref.P.T)
        return out

    def face_fluxes(self, own, nbr, t=0.0):
        Fn = super().face_fluxes(own, nbr, t)
        m = self.mesh
        ng = self.Bg.shape[2]
        nx = np.repeat(m.nx[:, :, None], ng, axis=2)
        ny = np.repeat(m.ny[:, :, None], ng, axis=2)
        stat = 0.5 * self.g * self.Bg * self.Bg
        return [Fn[0], Fn[1] - stat * nx, Fn[2] - stat * ny]
