"""Nodal-collocation variant of R(Q) (oracle, FP64; test infrastructure only).

The paper's method (Section 3) integrates the volume terms of the weak form with
a cubature rule and the face terms with Gauss rules. This variant evaluates
fluxes, source and numerical fluxes at the interpolation nodes instead and
integrates their degree-N interpolants exactly: roughly a third of the
arithmetic, at the price of aliasing. Readings (the paper does not define the
variant; these are the standard nodal choices, stated so the CUDA path can be
checked against them):

* Variables and fluxes in the pre-balanced free-surface form eta = h + B:
  F = (hu, hu u + p, hu v), G = (hv, hv u, hv v + p), p = g/2 (eta^2 - 2 eta B),
  S = (0, -g eta B_x, -g eta B_y), B_x and B_y the derivatives of the nodal
  interpolant of B. (Equal to Eq. swe_conservative in exact arithmetic; with
  collocation the choice matters, and this one keeps still water exactly at
  rest: p is then linear in B.)
* Volume: M^-1 Dr^T M (r_x F + r_y G) + M^-1 Ds^T M (s_x F + s_y G) + S, i.e.
  the weak-form volume integrals of the nodal interpolants, taken exactly.
* Faces: the numerical flux at the Nfp face nodes (traces are nodal values, the
  neighbour's at the coincident node), integrated exactly after interpolation
  along the face: -sum_f (sJ/J)_f M^-1 E_f F*_f with E_f the face mass matrix.
  F* is the well-balanced LLF flux of Section 5.1 minus the own side's static
  (g/2) (B^-)^2 n, the pre-balanced form's share of the pressure.
* Walls, velocities and the LLF speed as in the cubature oracle (oracle/swe.py).
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh
from .refelem import RefElement, face_points
from .swe import SWEModel, velocity, wb_lf_flux


def face_node_indices(ref: RefElement):
    """Node indices of each face ordered along the face (vertex f -> f+1) and their
    face parameters t in [-1, 1]."""
    idx, ts = [], []
    for f in range(3):
        if f == 0:
            on, t = np.isclose(ref.s, -1.0), ref.r
        elif f == 1:
            on, t = np.isclose(ref.r + ref.s, 0.0), ref.s
        else:
            on, t = np.isclose(ref.r, -1.0), -ref.s
        nodes = np.nonzero(on)[0]
        order = np.argsort(t[nodes])
        idx.append(nodes[order])
        ts.append(t[nodes][order])
    return idx, ts


class CollocModel(SWEModel):
    """SWEModel whose rhs() is the nodal-collocation variant (module docstring)."""

    def __init__(self, mesh: Mesh, ref: RefElement, B, g: float, h0: float):
        super().__init__(mesh, ref, B, g, h0)
        V, invV = ref.V, ref.invV
        from .refelem import grad_vandermonde
        Vr, Vs = grad_vandermonde(ref.N, ref.r, ref.s)
        self.Dr = Vr @ invV                     # nodal differentiation
        self.Ds = Vs @ invV
        self.Prc = ref.Minv @ self.Dr.T @ ref.M
        self.Psc = ref.Minv @ self.Ds.T @ ref.M
        self.fnodes, self.tnodes = face_node_indices(ref)
        # exact face lift: M^-1 E_f, E_f = integral over the face of l_i l_(f,m)
        self.Lc = [ref.Lg[f] @ ref.Ig[f][:, self.fnodes[f]] for f in range(3)]
        self.nperm, _, _ = mesh.face_point_map(self.tnodes[0])
        m = mesh
        self.Bxn = m.rx[:, None] * (self.B @ self.Dr.T) + m.sx[:, None] * (self.B @ self.Ds.T)
        self.Byn = m.ry[:, None] * (self.B @ self.Dr.T) + m.sy[:, None] * (self.B @ self.Ds.T)

    def volume(self, h, hu, hv):
        m, g = self.mesh, self.g
        eta = h + self.B
        u, v = velocity(h, hu, self.h0), velocity(h, hv, self.h0)
        p = 0.5 * g * (eta * eta - 2.0 * eta * self.B)
        F = (hu, hu * u + p, hu * v)
        G = (hv, hv * u, hv * v + p)
        S = (np.zeros_like(h), -g * eta * self.Bxn, -g * eta * self.Byn)
        out = []
        for c in range(3):
            cF1 = m.rx[:, None] * F[c] + m.ry[:, None] * G[c]
            cF2 = m.sx[:, None] * F[c] + m.sy[:, None] * G[c]
            out.append(cF1 @ self.Prc.T + cF2 @ self.Psc.T + S[c])
        return out

    def node_traces(self, h, hu, hv):
        return [np.stack([q[:, self.fnodes[f]] for f in range(3)], axis=1) for q in (h, hu, hv)]

    def rhs(self, h, hu, hv, nbr_state=None, t=0.0):
        m, g = self.mesh, self.g
        own = self.node_traces(h, hu, hv)
        nbr = own if nbr_state is None else self.node_traces(*nbr_state)
        Bm = np.stack([self.B[:, self.fnodes[f]] for f in range(3)], axis=1)
        hm, hum, hvm = own
        nfp = hm.shape[2]
        nx = np.repeat(m.nx[:, :, None], nfp, axis=2)
        ny = np.repeat(m.ny[:, :, None], nfp, axis=2)
        hp, hup, hvp, Bp = (np.empty_like(hm) for _ in range(4))
        inner = m.EToE >= 0
        kk, ff = np.nonzero(inner)
        k2, f2 = m.EToE[kk, ff], m.EToF[kk, ff]
        pm = self.nperm[kk, ff, :]
        for dst, src in ((hp, nbr[0]), (hup, nbr[1]), (hvp, nbr[2]), (Bp, Bm)):
            dst[kk, ff, :] = np.take_along_axis(src[k2, f2, :], pm, axis=1)
        kb, fb = np.nonzero(~inner)
        if kb.size:
            mn = hum[kb, fb] * nx[kb, fb] + hvm[kb, fb] * ny[kb, fb]
            hp[kb, fb] = hm[kb, fb]
            hup[kb, fb] = hum[kb, fb] - 2.0 * mn * nx[kb, fb]
            hvp[kb, fb] = hvm[kb, fb] - 2.0 * mn * ny[kb, fb]
            Bp[kb, fb] = Bm[kb, fb]
        Fn = wb_lf_flux(hm, hum, hvm, Bm, hp, hup, hvp, Bp, nx, ny, g, self.h0)
        stat = 0.5 * g * Bm * Bm
        Fn = [Fn[0], Fn[1] - stat * nx, Fn[2] - stat * ny]
        vol = self.volume(h, hu, hv)
        out = []
        for c in range(3):
            acc = 0.0
            for f in range(3):
                acc = acc + m.Fscale[:, f, None] * (Fn[c][:, f, :] @ self.Lc[f].T)
            out.append(vol[c] - acc)
        return np.stack(out)
