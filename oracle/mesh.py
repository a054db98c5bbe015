"""Mesh connectivity, affine geometry, face-point matching and the local time
step / level grouping, for the oracle (FP64, numpy).

Section 3: conforming triangles D^k; affine map from the reference triangle.
Section 4 (Eq. cfl and the level rule): per-element dt_k = C H^k / a, elements
with 2^{l-1} dt_min <= dt_k < 2^l dt_min form level l, stepped with
2^{l-1} dt_min.

Conventions: face f of element k joins its vertices f and f+1 (mod 3); the
element is made counter-clockwise (vertices 1 and 2 swapped when its signed area
is negative). Boundary faces have EToE = EToF = -1.
"""
from __future__ import annotations

import math

import numpy as np

from .refelem import FACE_VERTS, face_points


class Mesh:
    def __init__(self, vx, vy, EToV):
        self.vx = np.asarray(vx, np.float64)
        self.vy = np.asarray(vy, np.float64)
        E = np.array(EToV, dtype=np.int64, copy=True)
        x = self.vx[E]
        y = self.vy[E]
        area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
        if np.any(area2 == 0.0):
            raise ValueError("degenerate triangle")
        flip = area2 < 0
        E[flip, 1], E[flip, 2] = E[flip, 2].copy(), E[flip, 1].copy()
        self.EToV = E
        self.K = E.shape[0]
        self._connect()
        self._geometry()

    # -- connectivity: match faces by their (sorted) vertex pair ----------------
    def _connect(self):
        K = self.K
        faces = {}
        EToE = -np.ones((K, 3), np.int64)
        EToF = -np.ones((K, 3), np.int64)
        for k in range(K):
            for f, (a, b) in enumerate(FACE_VERTS):
                va, vb = int(self.EToV[k, a]), int(self.EToV[k, b])
                key = (min(va, vb), max(va, vb))
                faces.setdefault(key, []).append((k, f))
        for key, lst in faces.items():
            if len(lst) > 2:
                raise ValueError(f"non-manifold face {key}")
            if len(lst) == 2:
                (k1, f1), (k2, f2) = lst
                EToE[k1, f1], EToF[k1, f1] = k2, f2
                EToE[k2, f2], EToF[k2, f2] = k1, f1
        self.EToE = EToE
        self.EToF = EToF

    # -- affine geometry -------------------------------------------------------
    def _geometry(self):
        x = self.vx[self.EToV]
        y = self.vy[self.EToV]
        self.xv, self.yv = x, y
        xr = (x[:, 1] - x[:, 0]) / 2.0
        xs = (x[:, 2] - x[:, 0]) / 2.0
        yr = (y[:, 1] - y[:, 0]) / 2.0
        ys = (y[:, 2] - y[:, 0]) / 2.0
        J = xr * ys - xs * yr
        self.J = J
        self.rx = ys / J
        self.ry = -xs / J
        self.sx = -yr / J
        self.sy = xr / J
        self.area = 2.0 * J
        L = np.zeros((self.K, 3))
        nx = np.zeros((self.K, 3))
        ny = np.zeros((self.K, 3))
        for f, (a, b) in enumerate(FACE_VERTS):
            dx = x[:, b] - x[:, a]
            dy = y[:, b] - y[:, a]
            L[:, f] = np.hypot(dx, dy)
            nx[:, f] = dy / L[:, f]
            ny[:, f] = -dx / L[:, f]
        self.L = L                       # face lengths
        self.nx, self.ny = nx, ny        # outward unit normals
        self.sJ = L / 2.0                # surface Jacobian of t in [-1, 1]
        self.Fscale = self.sJ / J[:, None]
        self.cx = x.mean(axis=1)
        self.cy = y.mean(axis=1)

    def map_to_physical(self, r, s):
        """Physical coordinates of reference points, shape (K, npts)."""
        r = np.asarray(r)[None, :]
        s = np.asarray(s)[None, :]
        x = -(r + s) / 2 * self.xv[:, :1] + (1 + r) / 2 * self.xv[:, 1:2] + (1 + s) / 2 * self.xv[:, 2:3]
        y = -(r + s) / 2 * self.yv[:, :1] + (1 + r) / 2 * self.yv[:, 1:2] + (1 + s) / 2 * self.yv[:, 2:3]
        return x, y

    def face_point_map(self, t):
        """For every (k, f, g): the index g' of the physically coincident point on
        the neighbour face (found by nearest distance), or -1 on the boundary."""
        K = self.K
        n = len(t)
        px = np.zeros((K, 3, n))
        py = np.zeros((K, 3, n))
        for f, (fr, fs) in enumerate(face_points(t)):
            px[:, f, :], py[:, f, :] = self.map_to_physical(fr, fs)
        perm = -np.ones((K, 3, n), np.int64)
        inner = self.EToE >= 0
        kk, ff = np.nonzero(inner)
        k2 = self.EToE[kk, ff]
        f2 = self.EToF[kk, ff]
        d = ((px[kk, ff, :, None] - px[k2, f2, None, :]) ** 2
             + (py[kk, ff, :, None] - py[k2, f2, None, :]) ** 2)
        perm[kk, ff, :] = np.argmin(d, axis=2)
        scale = np.maximum(self.L[kk, ff], 1e-300)
        if d.size and np.sqrt(np.min(d, axis=2)).max() / scale.min() > 1e-9:
            raise ValueError("face points do not match")
        return perm, px, py


# ----------------------------------------------------------------------------
# CFL step (Eq. cfl) and level grouping (Section 4)


def element_dt(mesh: Mesh, N: int, h, hu, hv, g: float, cfl: float):
    """dt_k = C H^k / a_k with H^k = the inradius, C = cfl / (N+1)^2 and
    a_k = max over the element's nodes of |(u,v)| + sqrt(g max(h, h_ref)),
    h_ref = 1e-2 * max(h) so that dry elements keep a finite step."""
    perim = mesh.L.sum(axis=1)
    H = 2.0 * mesh.area / perim          # inradius = area / semi-perimeter
    hmax = float(np.max(h))
    href = 1e-2 * hmax
    hh = np.maximum(h, href)
    u = np.where(h > href, hu / np.where(h > href, h, 1.0), 0.0)
    v = np.where(h > href, hv / np.where(h > href, h, 1.0), 0.0)
    a = np.max(np.hypot(u, v) + np.sqrt(g * hh), axis=1)
    C = cfl / (N + 1) ** 2
    return C * H / a


def assign_levels(dt, nlevels: int):
    """Level l (1-based) with 2^{l-1} dt_min <= dt < 2^l dt_min, capped at nlevels."""
    dt = np.asarray(dt, np.float64)
    dtmin = float(dt.min())
    lev = np.empty(dt.shape, np.int64)
    for k, d in enumerate(dt):
        _, e = math.frexp(d / dtmin)     # d/dtmin = m 2^e, m in [0.5, 1)
        lev[k] = min(max(e, 1), nlevels)
    return lev, dtmin
