"""Brute-force quadrature used only by the tests to pin the oracle.

A dense Gauss-Legendre tensor rule pulled back to the triangle through the
collapsed (Duffy) map, with the Jacobian (1-b)/2 written explicitly; it uses
numpy's Legendre routine and nothing from the oracle.
"""
import math

import numpy as np


def duffy_rule(n):
    """n*n-point rule on the reference triangle (-1,-1),(1,-1),(-1,1); exact for
    polynomials of total degree <= 2n-2."""
    x, w = np.polynomial.legendre.leggauss(n)
    A, B = np.meshgrid(x, x, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    r = (1 + A) * (1 - B) / 2 - 1
    s = B
    return r.ravel(), s.ravel(), (WA * WB * (1 - B) / 2).ravel()


def simplex_monomial_integral(a, b, c):
    """Integral over the reference triangle (area 2) of l0^a l1^b l2^c where
    l0 = -(r+s)/2, l1 = (1+r)/2, l2 = (1+s)/2 (Dirichlet integral)."""
    return 2.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) * 2 / math.factorial(a + b + c + 2)


def physical_triangle_rule(xv, yv, n):
    """Brute-force rule on a physical triangle with vertices (xv[i], yv[i])."""
    r, s, w = duffy_rule(n)
    x = -(r + s) / 2 * xv[0] + (1 + r) / 2 * xv[1] + (1 + s) / 2 * xv[2]
    y = -(r + s) / 2 * yv[0] + (1 + r) / 2 * yv[1] + (1 + s) / 2 * yv[2]
    J = ((xv[1] - xv[0]) * (yv[2] - yv[0]) - (xv[2] - xv[0]) * (yv[1] - yv[0])) / 4
    return x, y, w * abs(J)
