"""Reference triangle for the oracle (FP64, numpy/scipy).

Section 3 of the paper: Lagrange basis on Warp & Blend nodes, cubature rules for
the volume integrals, Gauss-Legendre rules for the surface integrals, and the
projection matrices "premultiplied with cubature integration weights"
(Section 7.1: N(Q) = Pr cF1 + Ps cF2 + P cS) and the lift operator L^g
(Section 7.2: S = -L^g F_n^*).

Reference triangle: vertices v0 = (-1,-1), v1 = (1,-1), v2 = (-1,1) in (r, s);
area 2. Face f joins v_f to v_{f+1 mod 3} (counter-clockwise).

Choices where the paper is silent (readings):
* cubature: Stroud conical product of q-point Gauss-Legendre (collapsed
  direction a) and q-point Gauss-Jacobi(alpha=1, beta=0) (direction b), exact to
  degree 2q-1; default degree 3N-1 so the lake-at-rest balance is exact.
* Gauss rule on faces: Ng = ceil((3N+1)/2) points (exact to degree 3N).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

# Warburton (2006) optimised blend parameters for the Warp & Blend node family,
# as tabulated by Hesthaven & Warburton (2008) for N = 1..15.
_ALPHA_OPT = [0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
              1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258]


# ----------------------------------------------------------------------------
# 1D orthogonal polynomials and rules


def jacobi_normalized(x, alpha: float, beta: float, n: int):
    """Jacobi polynomial P_n^(alpha,beta)(x) scaled to unit norm under the weight
    (1-x)^alpha (1+x)^beta on [-1, 1]."""
    x = np.asarray(x, dtype=np.float64)
    p = special.eval_jacobi(n, alpha, beta, x)
    lg = ((alpha + beta + 1) * math.log(2.0) - math.log(2 * n + alpha + beta + 1)
          + special.gammaln(n + alpha + 1) + special.gammaln(n + beta + 1)
          - special.gammaln(n + alpha + beta + 1) - special.gammaln(n + 1))
    return p / math.exp(0.5 * lg)


def jacobi_normalized_deriv(x, alpha: float, beta: float, n: int):
    """d/dx of :func:`jacobi_normalized` (uses dP_n/dx ~ P_{n-1}^(alpha+1,beta+1))."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return math.sqrt(n * (n + alpha + beta + 1)) * jacobi_normalized(x, alpha + 1, beta + 1, n - 1)


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (exact to degree 2n-1)."""
    x, w = special.roots_legendre(n)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


def gauss_jacobi(n: int, alpha: float, beta: float):
    """n-point Gauss-Jacobi rule for the weight (1-x)^alpha (1+x)^beta."""
    x, w = special.roots_jacobi(n, alpha, beta)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


def gauss_lobatto_nodes(N: int):
    """N+1 Gauss-Lobatto-Legendre points: +-1 and the roots of P_N'."""
    if N == 1:
        return np.array([-1.0, 1.0])
    xi, _ = special.roots_jacobi(N - 1, 1.0, 1.0)
    return np.concatenate([[-1.0], np.sort(xi), [1.0]])


# ----------------------------------------------------------------------------
# Warp & Blend nodes (Warburton 2006)


def _warp_factor(N: int, rout):
    """1D warp (GLL minus equidistant) interpolated to rout, divided by the edge
    blend 1 - r^2 so that blend * warp reproduces the 1D warp on each edge."""
    rout = np.asarray(rout, dtype=np.float64)
    req = np.linspace(-1.0, 1.0, N + 1)
    d = gauss_lobatto_nodes(N) - req
    # Lagrange interpolation of d from the equidistant points (product formula)
    warp = np.zeros_like(rout)
    for i in range(N + 1):
        li = np.ones_like(rout)
        for j in range(N + 1):
            if j != i:
                li = li * (rout - req[j]) / (req[i] - req[j])
        warp = warp + d[i] * li
    inside = np.abs(rout) < 1.0 - 1e-10
    out = np.zeros_like(rout)
    out[inside] = warp[inside] / (1.0 - rout[inside] ** 2)
    return out


def warp_blend_nodes(N: int):
    """Warp & Blend nodes on the reference triangle, in lattice order.

    Order: for i = 0..N (barycentric weight of v2 = i/N), j = 0..N-i (weight of
    v1 = j/N). The first N+1 nodes lie on face 0 from v0 to v1.
    """
    alpha = _ALPHA_OPT[N - 1] if N <= len(_ALPHA_OPT) else 5.0 / 3.0
    L1, L3 = [], []
    for i in range(N + 1):
        for j in range(N + 1 - i):
            L1.append(i / N)
            L3.append(j / N)
    L1 = np.array(L1)
    L3 = np.array(L3)
    L2 = 1.0 - L1 - L3
    # equilateral triangle: v0 = (-1,-1/sqrt3), v1 = (1,-1/sqrt3), v2 = (0, 2/sqrt3)
    x = -L2 + L3
    y = (-L2 - L3 + 2.0 * L1) / math.sqrt(3.0)
    b1 = 4.0 * L2 * L3
    b2 = 4.0 * L1 * L3
    b3 = 4.0 * L1 * L2
    w1 = b1 * _warp_factor(N, L3 - L2) * (1.0 + (alpha * L1) ** 2)
    w2 = b2 * _warp_factor(N, L1 - L3) * (1.0 + (alpha * L2) ** 2)
    w3 = b3 * _warp_factor(N, L2 - L1) * (1.0 + (alpha * L3) ** 2)
    c2, s2 = math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)
    c3, s3 = math.cos(4 * math.pi / 3), math.sin(4 * math.pi / 3)
    x = x + w1 + c2 * w2 + c3 * w3
    y = y + s2 * w2 + s3 * w3
    # back to the reference right triangle through barycentric coordinates
    l1 = (math.sqrt(3.0) * y + 1.0) / 3.0
    l2 = (-3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    l3 = (3.0 * x - math.sqrt(3.0) * y + 2.0) / 6.0
    r = -l2 + l3 - l1
    s = -l2 - l3 + l1
    return r, s


# ----------------------------------------------------------------------------
# orthonormal (PKDO / Dubiner) basis on the reference triangle


def mode_list(N: int):
    """(i, j) mode indices, i + j <= N, i outer."""
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def _collapse(r, s):
    r = np.asarray(r, np.float64)
    s = np.asarray(s, np.float64)
    a = np.where(np.abs(1.0 - s) > 1e-14, 2.0 * (1.0 + r) / np.where(np.abs(1.0 - s) > 1e-14, 1.0 - s, 1.0) - 1.0, -1.0)
    return a, s


def basis(r, s, i: int, j: int):
    """psi_ij(r,s) = sqrt2 P_i(a) P_j^(2i+1,0)(b) (1-b)^i, orthonormal on the triangle."""
    a, b = _collapse(r, s)
    return (math.sqrt(2.0) * jacobi_normalized(a, 0, 0, i)
            * jacobi_normalized(b, 2 * i + 1, 0, j) * (1.0 - b) ** i)


def grad_basis(r, s, i: int, j: int):
    """(d psi_ij / dr, d psi_ij / ds) by the chain rule through (a, b)."""
    a, b = _collapse(r, s)
    fa = jacobi_normalized(a, 0, 0, i)
    dfa = jacobi_normalized_deriv(a, 0, 0, i)
    gb = jacobi_normalized(b, 2 * i + 1, 0, j)
    dgb = jacobi_normalized_deriv(b, 2 * i + 1, 0, j)
    if i == 0:
        dr = np.zeros_like(a)
        ds = fa * dgb
    else:
        pm = (1.0 - b) ** (i - 1)
        dr = 2.0 * dfa * gb * pm
        ds = dfa * gb * (1.0 + a) * pm + fa * (dgb * (1.0 - b) ** i - i * gb * pm)
    return math.sqrt(2.0) * dr, math.sqrt(2.0) * ds


def vandermonde(N: int, r, s):
    return np.stack([basis(r, s, i, j) for (i, j) in mode_list(N)], axis=-1)


def grad_vandermonde(N: int, r, s):
    gr, gs = zip(*[grad_basis(r, s, i, j) for (i, j) in mode_list(N)])
    return np.stack(gr, axis=-1), np.stack(gs, axis=-1)


# ----------------------------------------------------------------------------
# volume cubature (conical product)


def conical_cubature(degree: int):
    """Stroud conical-product rule on the reference triangle exact to ``degree``.

    r = (1+a)(1-b)/2 - 1, s = b, dr ds = (1-b)/2 da db; Gauss-Legendre in a,
    Gauss-Jacobi(1,0) in b, q = ceil((degree+1)/2) points each.
    """
    q = max(1, int(math.ceil((degree + 1) / 2.0)))
    xa, wa = gauss_legendre(q)
    xb, wb = gauss_jacobi(q, 1.0, 0.0)
    A, Bv = np.meshgrid(xa, xb, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    r = (1.0 + A) * (1.0 - Bv) / 2.0 - 1.0
    s = Bv
    w = WA * WB / 2.0
    return r.ravel(), s.ravel(), w.ravel()


# ----------------------------------------------------------------------------
# the reference element


FACE_VERTS = ((0, 1), (1, 2), (2, 0))
REF_VERTS = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])


def face_points(t):
    """Reference (r, s) of parameter t in [-1,1] on each face, traversed v_f -> v_{f+1}."""
    t = np.asarray(t, np.float64)
    return [
        (t, -np.ones_like(t)),          # face 0: v0 -> v1
        (-t, t),                          # face 1: v1 -> v2
        (-np.ones_like(t), -t),           # face 2: v2 -> v0
    ]


class RefElement:
    """All reference operators of Sections 3 and 7 for polynomial order N."""

    def __init__(self, N: int, cub_degree: int | None = None, ng: int | None = None):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.Np = (N + 1) * (N + 2) // 2
        self.Nfp = N + 1
        self.cub_degree = 3 * N - 1 if cub_degree is None else cub_degree
        self.Ng = int(math.ceil((3 * N + 1) / 2.0)) if ng is None else ng
        self.modes = mode_list(N)
        self.r, self.s = warp_blend_nodes(N)
        self.V = vandermonde(N, self.r, self.s)
        self.invV = np.linalg.inv(self.V)
        self.M = np.linalg.inv(self.V @ self.V.T)          # mass matrix of the Lagrange basis
        self.Minv = self.V @ self.V.T
        # cubature and the interpolation / projection operators (Section 7.1)
        self.rc, self.sc, self.wc = conical_cubature(self.cub_degree)
        self.Ncub = self.rc.size
        Vc = vandermonde(N, self.rc, self.sc)
        Vcr, Vcs = grad_vandermonde(N, self.rc, self.sc)
        self.Ic = Vc @ self.invV           # nodal -> values at cubature points
        self.Icr = Vcr @ self.invV         # nodal -> d/dr at cubature points
        self.Ics = Vcs @ self.invV         # nodal -> d/ds at cubature points
        W = np.diag(self.wc)
        self.Pr = self.Minv @ self.Icr.T @ W
        self.Ps = self.Minv @ self.Ics.T @ W
        self.P = self.Minv @ self.Ic.T @ W
        # faces: Gauss-Legendre points, interpolation and lift (Section 7.2)
        self.tg, self.wg = gauss_legendre(self.Ng)
        self.Ig = []
        self.Lg = []
        for (fr, fs) in face_points(self.tg):
            Ig = vandermonde(N, fr, fs) @ self.invV
            self.Ig.append(Ig)
            self.Lg.append(self.Minv @ Ig.T @ np.diag(self.wg))
        # projection onto P1 (Algorithm 3): keep the modes of total degree <= 1
        keep = np.array([1.0 if (i + j) <= 1 else 0.0 for (i, j) in self.modes])
        self.Pi1 = self.V @ np.diag(keep) @ self.invV
        # element mean: (1/|T|) * integral = (1/2) * column sums of M
        self.mean_w = self.M.sum(axis=0) / 2.0
        # vertex nodes
        self.vertex_nodes = np.array([
            int(np.argmin((self.r - vr) ** 2 + (self.s - vs) ** 2)) for (vr, vs) in REF_VERTS])

    def interp_matrix(self, r, s):
        """Nodal values -> values at arbitrary reference points."""
        return vandermonde(self.N, r, s) @ self.invV
