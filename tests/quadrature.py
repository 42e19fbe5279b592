"""Brute-force numerical quadrature of Coulomb integrals over Cartesian
Gaussians, independent of the Boys function and of any recursion.

Uses 1/r12 = (2/sqrt(pi)) int_0^inf exp(-t^2 r12^2) dt.  For fixed t the
6-dimensional integrand factorises into three 2-dimensional integrals
I_d(t) = int int poly(x1, x2) exp(-Q(x1, x2; t)) dx1 dx2 with Q quadratic; after
the change of variables that diagonalises Q each is integrated exactly by a
tensor Gauss-Hermite rule (polynomial degree <= 6 needs 4 points; 10 are used).
The t integral maps t = s/(1-s) onto [0, 1) and uses Gauss-Legendre.
Test-only helper.
"""

import math

import numpy as np

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(10)


def _gauss_legendre_01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def prim_coulomb(a, A, pa, b, B, pb, g, C, pc, nt=400):
    """(g_a g_b | g_c) for unnormalised primitives x_A^pa e^{-a r_A^2} etc.
    b = 0 with pb = (0,0,0) gives the 2-centre integral (g_a | g_c)."""
    s, ws = _gauss_legendre_01(nt)
    t = s / (1.0 - s)
    dt = ws / (1.0 - s) ** 2
    t2 = t * t
    total = np.ones_like(t)
    for d in range(3):
        # exponent: -(a+b+t2) x1^2 + 2 t2 x1 x2 - (t2+g) x2^2 + 2(aA+bB) x1 + 2 g C x2 - s0
        m11 = a + b + t2
        m22 = t2 + g
        m12 = -t2
        b1 = a * A[d] + b * B[d]
        b2 = g * C[d]
        s0 = a * A[d] ** 2 + b * B[d] ** 2 + g * C[d] ** 2
        det = m11 * m22 - m12 * m12
        # mean m = M^-1 b
        mu1 = (m22 * b1 - m12 * b2) / det
        mu2 = (-m12 * b1 + m11 * b2) / det
        c0 = b1 * mu1 + b2 * mu2 - s0
        # Cholesky M = L L^T, L = [[l11,0],[l21,l22]]; z = mu + L^-T y
        l11 = np.sqrt(m11)
        l21 = m12 / l11
        l22 = np.sqrt(m22 - l21 * l21)
        # L^-T = [[1/l11, -l21/(l11 l22)], [0, 1/l22]]
        y1 = _GH_X[:, None, None]
        y2 = _GH_X[None, :, None]
        x1 = mu1 + y1 / l11 - y2 * l21 / (l11 * l22)
        x2 = mu2 + y2 / l22
        poly = (x1 - A[d]) ** pa[d] * (x1 - B[d]) ** pb[d] * (x2 - C[d]) ** pc[d]
        w2 = _GH_W[:, None, None] * _GH_W[None, :, None]
        integ = np.sum(w2 * poly, axis=(0, 1)) / (l11 * l22) * np.exp(c0)
        total = total * integ
    return 2.0 / math.sqrt(math.pi) * np.sum(total * dt)


def _dfact(n):
    r = 1.0
    for k in range(2 * n - 1, 1, -2):
        r *= k
    return r


def _prim_norm(a, pw):
    l = sum(pw)
    return (2 * a / math.pi) ** 0.75 * (4 * a) ** (0.5 * l) / math.sqrt(
        _dfact(pw[0]) * _dfact(pw[1]) * _dfact(pw[2])
    )


def _overlap_prim_same_center(a, b, pw):
    """<x^pw e^{-a r^2} | x^pw e^{-b r^2}> at one centre (closed form)."""
    p = a + b
    v = 1.0
    for k in pw:
        v *= _dfact(k) / (2 * p) ** k * math.sqrt(math.pi / p)
    return v


def contracted_norm(exps, coefs, pw):
    s = 0.0
    for a, ca in zip(exps, coefs):
        for b, cb in zip(exps, coefs):
            s += ca * cb * _prim_norm(a, pw) * _prim_norm(b, pw) * _overlap_prim_same_center(a, b, pw)
    return 1.0 / math.sqrt(s)


def contracted_3c(sa, A, pa, sb, B, pb, sc, C, pc, nt=400):
    """(chi_a chi_b | chi_c) for normalised contracted components."""
    na = contracted_norm(sa.exps, sa.coefs, pa)
    nb = contracted_norm(sb.exps, sb.coefs, pb)
    nc = contracted_norm(sc.exps, sc.coefs, pc)
    v = 0.0
    for a, ca in zip(sa.exps, sa.coefs):
        for b, cb in zip(sb.exps, sb.coefs):
            for g, cg in zip(sc.exps, sc.coefs):
                v += (
                    ca * _prim_norm(a, pa) * cb * _prim_norm(b, pb) * cg * _prim_norm(g, pc)
                    * prim_coulomb(a, A, pa, b, B, pb, g, C, pc, nt)
                )
    return v * na * nb * nc


def contracted_2c(sp, A, pp, sq, C, pq, nt=400):
    npn = contracted_norm(sp.exps, sp.coefs, pp)
    nq = contracted_norm(sq.exps, sq.coefs, pq)
    v = 0.0
    for a, ca in zip(sp.exps, sp.coefs):
        for g, cg in zip(sq.exps, sq.coefs):
            v += (
                ca * _prim_norm(a, pp) * cg * _prim_norm(g, pq)
                * prim_coulomb(a, A, pp, 0.0, A, (0, 0, 0), g, C, pq, nt)
            )
    return v * npn * nq
