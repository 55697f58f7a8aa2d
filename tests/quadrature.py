"""Brute-force numerical integration of Gaussian integrals, independent of the oracle's
closed forms (used only to pin the oracle).

Primitive Cartesian Gaussians g(r) = (x-A_x)^l (y-A_y)^m (z-A_z)^n exp(-alpha |r-A|^2).
  * overlap:  tensor Gauss-Hermite quadrature of the product (exact for these polynomials).
  * kinetic:  1/2 <grad a | grad b> (the integrated-by-parts form), Gauss-Hermite.
  * 1/r:      1/|r| = (2/sqrt(pi)) int_0^inf exp(-u^2 r^2) du, u = sqrt(c) tan(theta),
              Gauss-Legendre in theta; each fixed-u integrand is a separable Gaussian whose
              1-D (or 2-D) factors are done exactly by Gauss-Hermite after completing the square.
"""
from __future__ import annotations

import math

import numpy as np

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(12)
_GL_X, _GL_W = np.polynomial.legendre.leggauss(160)


def _prod_1d(alpha, A, beta, B):
    p = alpha + beta
    P = (alpha * A + beta * B) / p
    K = math.exp(-alpha * beta / p * (A - B) ** 2)
    return p, P, K


def overlap_1d(la, A, alpha, lb, B, beta):
    """int (x-A)^la (x-B)^lb exp(-alpha (x-A)^2 - beta (x-B)^2) dx."""
    p, P, K = _prod_1d(alpha, A, beta, B)
    x = P + _GH_X / math.sqrt(p)
    f = (x - A) ** la * (x - B) ** lb
    return K * float(np.sum(_GH_W * f)) / math.sqrt(p)


def _deriv_terms(l, alpha):
    """d/dx [x^l e^{-alpha x^2}] as [(coefficient, power)]."""
    out = []
    if l > 0:
        out.append((float(l), l - 1))
    out.append((-2.0 * alpha, l + 1))
    return out


def overlap(a, b):
    """a, b = (alpha, centre[3], (l, m, n))."""
    (al, A, la), (be, B, lb) = a, b
    return math.prod(overlap_1d(la[k], A[k], al, lb[k], B[k], be) for k in range(3))


def kinetic(a, b):
    (al, A, la), (be, B, lb) = a, b
    total = 0.0
    for k in range(3):
        s = 0.0
        for ca, pa in _deriv_terms(la[k], al):
            for cb, pb in _deriv_terms(lb[k], be):
                s += ca * cb * overlap_1d(pa, A[k], al, pb, B[k], be)
        others = math.prod(overlap_1d(la[j], A[j], al, lb[j], B[j], be) for j in range(3) if j != k)
        total += 0.5 * s * others
    return total


def _theta_nodes(c):
    """Nodes/weights for int_0^inf h(u) du with u = sqrt(c) tan(theta), theta in [0, pi/2)."""
    th = 0.25 * math.pi * (_GL_X + 1.0)
    w = 0.25 * math.pi * _GL_W
    u = math.sqrt(c) * np.tan(th)
    du = math.sqrt(c) / np.cos(th) ** 2
    return u, w * du


def nuclear(a, b, C):
    """int g_a g_b / |r - C| dr (one unit charge; the attraction is minus Z times this)."""
    (al, A, la), (be, B, lb) = a, b
    p = al + be
    us, ws = _theta_nodes(p)
    total = 0.0
    for u, w in zip(us, ws):
        val = 1.0
        for k in range(3):
            pk, Pk, Kk = _prod_1d(al, A[k], be, B[k])
            # exp(-p (x-P)^2 - u^2 (x-C)^2) = exp(-s (x-M)^2) exp(-p u^2/s (P-C)^2)
            s = pk + u * u
            M = (pk * Pk + u * u * C[k]) / s
            pref = Kk * math.exp(-pk * u * u / s * (Pk - C[k]) ** 2)
            x = M + _GH_X / math.sqrt(s)
            f = (x - A[k]) ** la[k] * (x - B[k]) ** lb[k]
            val *= pref * float(np.sum(_GH_W * f)) / math.sqrt(s)
        total += w * val
    return 2.0 / math.sqrt(math.pi) * total


def eri(a, b, c, d):
    """(ab|cd) = int int g_a(1) g_b(1) g_c(2) g_d(2) / r12, brute force."""
    (al, A, la), (be, B, lb) = a, b
    (ga, Cc, lc), (de, D, ld) = c, d
    p, q = al + be, ga + de
    rho = p * q / (p + q)
    us, ws = _theta_nodes(rho)
    X1, X2 = np.meshgrid(_GH_X, _GH_X, indexing="ij")
    W2 = np.outer(_GH_W, _GH_W)
    total = 0.0
    for u, w in zip(us, ws):
        val = 1.0
        for k in range(3):
            pk, Pk, Kab = _prod_1d(al, A[k], be, B[k])
            qk, Qk, Kcd = _prod_1d(ga, Cc[k], de, D[k])
            u2 = u * u
            Mm = np.array([[pk + u2, -u2], [-u2, qk + u2]])
            rhs = np.array([pk * Pk, qk * Qk])
            v0 = np.linalg.solve(Mm, rhs)
            E0 = pk * (v0[0] - Pk) ** 2 + qk * (v0[1] - Qk) ** 2 + u2 * (v0[0] - v0[1]) ** 2
            Lc = np.linalg.cholesky(Mm)
            LinvT = np.linalg.inv(Lc).T
            x1 = v0[0] + LinvT[0, 0] * X1 + LinvT[0, 1] * X2
            x2 = v0[1] + LinvT[1, 0] * X1 + LinvT[1, 1] * X2
            f = ((x1 - A[k]) ** la[k] * (x1 - B[k]) ** lb[k]
                 * (x2 - Cc[k]) ** lc[k] * (x2 - D[k]) ** ld[k])
            val *= Kab * Kcd * math.exp(-E0) / float(np.prod(np.diag(Lc))) * float(np.sum(W2 * f))
        total += w * val
    return 2.0 / math.sqrt(math.pi) * total
