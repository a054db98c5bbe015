"""Right-hand side of the semi-discrete nodal DG shallow-water system (oracle, FP64).

Equations (Section 2, Eq. swe_conservative): Q = (h, hu, hv),
F = (hu, hu^2 + g h^2/2, huv), G = (hv, huv, hv^2 + g h^2/2), S = (0, -g h B_x, -g h B_y).

Weak form (Section 3, Eq. weak_form) with the numerical flux on the element
boundary, giving dQ/dt = N(Q) + S(Q^{g,+}, Q^{g,-}) (Eq. ode):
* volume term (Section 7.1): N = Pr cF1 + Ps cF2 + P cS with cF1 = r_x F + r_y G,
  cF2 = s_x F + s_y G and cS the source, all at cubature points;
* surface term (Section 7.2): S = -L^g F_n^*, with F_n^* the well-balanced local
  Lax-Friedrichs flux of Section 5.1 (Eq. well_balance) at Gauss points, scaled
  by the face's surface Jacobian over the volume Jacobian.

Readings where the paper is silent:
* "-" is the element's own trace, "+" the neighbour's (Section 5.1 wording).
* LLF speed lambda = max(|u^- . n| + sqrt(g h*^-), |u^+ . n| + sqrt(g h*^+)) per point.
* velocity u = hu/h where h > h0 (1 + 1e-6), else 0 (volume and surface alike).
* reflective wall: ghost h^+ = h^-, B^+ = B^-, m^+ = m^- - 2 (m^- . n) n.
* Dirichlet faces (the convergence pin) and far-field faces (a constant state):
  ghost = that state, bed continued.
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh
from .refelem import RefElement


def physical_flux(h, hu, hv, u, v, g):
    """F and G of Eq. swe_conservative given the velocities used for advection."""
    p = 0.5 * g * h * h
    F = (hu, hu * u + p, hu * v)
    G = (hv, hv * u, hv * v + p)
    return F, G


# The velocity threshold sits a relative 1e-6 above h0: the positivity limiter leaves
# depths exactly at h0 (the lowest vertex of a limited element), and those must take
# u = 0 whatever the rounding of a depth computed as eta - B.
VEL_MARGIN = 1e-6


def velocity(h, m, h0):
    hv = h0 * (1.0 + VEL_MARGIN)
    return np.where(h > hv, m / np.where(h > hv, h, 1.0), 0.0)


def wb_lf_flux(hm, hum, hvm, Bm, hp, hup, hvp, Bp, nx, ny, g, h0):
    """Well-balanced local Lax-Friedrichs normal flux seen by the "-" side (Eq. well_balance).

    h*^{+-} = max(0, h^{+-} + B^{+-} - max(B^+, B^-)), Q*^{+-} = h*^{+-} (1, u^{+-}, v^{+-});
    F* . n = F_LF(Q*^+, Q*^-) . n + (0, n_x, n_y) * (g/2) ((h^-)^2 - (h*^-)^2).
    """
    um, vm = velocity(hm, hum, h0), velocity(hm, hvm, h0)
    up, vp = velocity(hp, hup, h0), velocity(hp, hvp, h0)
    Bmax = np.maximum(Bm, Bp)
    hsm = np.maximum(0.0, hm + Bm - Bmax)
    hsp = np.maximum(0.0, hp + Bp - Bmax)
    qm = (hsm, hsm * um, hsm * vm)
    qp = (hsp, hsp * up, hsp * vp)
    Fm, Gm = physical_flux(qm[0], qm[1], qm[2], um, vm, g)
    Fp, Gp = physical_flux(qp[0], qp[1], qp[2], up, vp, g)
    lam = np.maximum(np.abs(um * nx + vm * ny) + np.sqrt(g * hsm),
                     np.abs(up * nx + vp * ny) + np.sqrt(g * hsp))
    out = []
    for c in range(3):
        out.append(0.5 * (Fm[c] * nx + Gm[c] * ny + Fp[c] * nx + Gp[c] * ny)
                   - 0.5 * lam * (qp[c] - qm[c]))
    corr = 0.5 * g * (hm * hm - hsm * hsm)
    out[1] = out[1] + corr * nx
    out[2] = out[2] + corr * ny
    return out


class SWEModel:
    """Mesh + reference element + bathymetry: evaluates R(Q) for all elements."""

    def __init__(self, mesh: Mesh, ref: RefElement, B, g: float, h0: float,
                 dirichlet=None, farfield=None, farfield_faces=None):
        self.mesh = mesh
        self.ref = ref
        self.B = np.asarray(B, np.float64)            # (K, Np) nodal bathymetry
        # far field: every boundary face sees the constant state (h, hu, hv), the bed
        # continued (B+ = B-); the TVB limiter's ghost mean is that state
        self.farfield = None if farfield is None else tuple(float(v) for v in farfield)
        # which boundary faces are open (K x 3 bool; None: all of them); the rest are walls
        self.farfield_faces = None if farfield_faces is None else np.asarray(farfield_faces, bool)
        if self.farfield is not None:
            hf, huf, hvf = self.farfield
            dirichlet = lambda x, y, t: (np.full(np.shape(x), hf), np.full(np.shape(x), huf),
                                         np.full(np.shape(x), hvf))
        self.g = float(g)
        self.h0 = float(h0)
        self.dirichlet = dirichlet                     # callable(x, y, t) -> (h, hu, hv) or None
        self.perm, self.gx, self.gy = mesh.face_point_map(ref.tg)
        # bathymetry and its gradient at cubature points are fixed in time
        self.Bc = self.B @ ref.Ic.T
        Br = self.B @ ref.Icr.T
        Bs = self.B @ ref.Ics.T
        m = mesh
        self.Bx = m.rx[:, None] * Br + m.sx[:, None] * Bs
        self.By = m.ry[:, None] * Br + m.sy[:, None] * Bs
        self.Bg = np.stack([self.B @ ref.Ig[f].T for f in range(3)], axis=1)   # (K, 3, Ng)
        xn, yn = mesh.map_to_physical(ref.r, ref.s)
        self.xn, self.yn = xn, yn

    # -- volume term, Section 7.1 ---------------------------------------------
    def volume(self, h, hu, hv):
        ref, m, g = self.ref, self.mesh, self.g
        hc, huc, hvc = h @ ref.Ic.T, hu @ ref.Ic.T, hv @ ref.Ic.T
        u, v = velocity(hc, huc, self.h0), velocity(hc, hvc, self.h0)
        F, G = physical_flux(hc, huc, hvc, u, v, g)
        S = (np.zeros_like(hc), -g * hc * self.Bx, -g * hc * self.By)
        out = []
        for c in range(3):
            cF1 = m.rx[:, None] * F[c] + m.ry[:, None] * G[c]
            cF2 = m.sx[:, None] * F[c] + m.sy[:, None] * G[c]
            out.append(cF1 @ ref.Pr.T + cF2 @ ref.Ps.T + S[c] @ ref.P.T)
        return out

    # -- traces at Gauss points -------------------------------------------------
    def traces(self, h, hu, hv):
        ref = self.ref
        return [np.stack([q @ ref.Ig[f].T for f in range(3)], axis=1) for q in (h, hu, hv)]

    def face_fluxes(self, own, nbr, t=0.0):
        """F_n^* at every (k, f, g) given own traces and neighbour traces (K,3,Ng)."""
        m = self.mesh
        hm, hum, hvm = own
        Bm = self.Bg
        K, _, ng = hm.shape
        nx = np.repeat(m.nx[:, :, None], ng, axis=2)
        ny = np.repeat(m.ny[:, :, None], ng, axis=2)
        hp = np.empty_like(hm)
        hup = np.empty_like(hm)
        hvp = np.empty_like(hm)
        Bp = np.empty_like(hm)
        inner = m.EToE >= 0
        kk, ff = np.nonzero(inner)
        k2 = m.EToE[kk, ff]
        f2 = m.EToF[kk, ff]
        p = self.perm[kk, ff, :]
        hp[kk, ff, :] = np.take_along_axis(nbr[0][k2, f2, :], p, axis=1)
        hup[kk, ff, :] = np.take_along_axis(nbr[1][k2, f2, :], p, axis=1)
        hvp[kk, ff, :] = np.take_along_axis(nbr[2][k2, f2, :], p, axis=1)
        Bp[kk, ff, :] = np.take_along_axis(self.Bg[k2, f2, :], p, axis=1)
        # boundary faces
        kb, fb = np.nonzero(~inner)
        if kb.size:
            if self.dirichlet is None:
                opn = np.zeros(kb.size, bool)
            elif self.farfield_faces is None:
                opn = np.ones(kb.size, bool)
            else:
                opn = self.farfield_faces[kb, fb]
            kw, fw = kb[~opn], fb[~opn]
            mn = hum[kw, fw] * nx[kw, fw] + hvm[kw, fw] * ny[kw, fw]
            hp[kw, fw] = hm[kw, fw]
            hup[kw, fw] = hum[kw, fw] - 2.0 * mn * nx[kw, fw]
            hvp[kw, fw] = hvm[kw, fw] - 2.0 * mn * ny[kw, fw]
            Bp[kw, fw] = Bm[kw, fw]
            ko, fo = kb[opn], fb[opn]
            if ko.size:
                eh, ehu, ehv = self.dirichlet(self.gx[ko, fo], self.gy[ko, fo], t)
                hp[ko, fo], hup[ko, fo], hvp[ko, fo] = eh, ehu, ehv
                Bp[ko, fo] = Bm[ko, fo]
        return wb_lf_flux(hm, hum, hvm, Bm, hp, hup, hvp, Bp, nx, ny, self.g, self.h0)

    # -- surface term, Section 7.2 --------------------------------------------
    def surface(self, Fn):
        ref, m = self.ref, self.mesh
        out = []
        for c in range(3):
            acc = 0.0
            for f in range(3):
                acc = acc + m.Fscale[:, f, None] * (Fn[c][:, f, :] @ ref.Lg[f].T)
            out.append(-acc)
        return out

    def rhs(self, h, hu, hv, nbr_state=None, t=0.0):
        """R(Q) = N(Q) + S(Q^{g,+}, Q^{g,-}) for all elements.

        ``nbr_state`` (h, hu, hv) is the state whose traces the neighbours show
        (the multirate integrator passes reconstructed values for neighbours
        that are between steps); by default it is the state itself.
        """
        own = self.traces(h, hu, hv)
        nbr = own if nbr_state is None else self.traces(*nbr_state)
        vol = self.volume(h, hu, hv)
        Fn = self.face_fluxes(own, nbr, t)
        srf = self.surface(Fn)
        return np.stack([vol[c] + srf[c] for c in range(3)])

    def element_means(self, q):
        return q @ self.ref.mean_w

    def mass(self, h):
        return float(np.sum(self.mesh.area * self.element_means(h)))
