"""Coefficients of the link-phase polynomials in ahs_device.cuh (link_sincos).

After the reduction th = k pi + r, |r| <= pi/2, the kernel evaluates
    sin r = r + r^3 S(r^2),   S of degree 3 (sin of degree 9),
    cos r = 1 + r^2 C(r^2),   C of degree 4 (cos of degree 10).
S is fitted to (sin r - r)/r^3 weighted so that the error of sin r is relative;
C to (cos r - 1)/r^2 weighted so that the error of cos r is absolute.  Both are
near-minimax fits by Lawson's algorithm (C. L. Lawson, 1961: iteratively
reweighted least squares, the weights multiplied by the current error each pass)
on 20001 Chebyshev-spaced points of (0, pi/2].  The coefficients are rounded to
float32 once.

    python paper_2005_14454_gb300/csrc/gen_link_sincos.py
prints them in the order the kernel uses (lowest power first).
"""
import numpy as np


def lawson(f, powers, weight, x, iters=400):
    A = np.stack([x ** p for p in powers], 1)
    u = np.full(x.size, 1.0 / x.size)
    for _ in range(iters):
        w = np.sqrt(u) * weight
        c = np.linalg.lstsq(A * w[:, None], f * w, rcond=None)[0]
        e = np.abs((A @ c - f) * weight)
        u *= e
        u /= u.sum()
    return c, float(np.max(np.abs((A @ c - f) * weight)))


def nodes(n=20001):
    x = (np.cos(np.linspace(0.0, np.pi, n)) * 0.5 + 0.5) * (np.pi / 2) * 1.0001
    return x[x > 1e-6]


def coefficients():
    x = nodes()
    s, es = lawson((np.sin(x) - x) / x ** 3, [0, 2, 4, 6], x ** 3 / np.sin(x), x)
    c, ec = lawson((np.cos(x) - 1.0) / x ** 2, [0, 2, 4, 6, 8], x ** 2, x)
    return [float(np.float32(v)) for v in s], [float(np.float32(v)) for v in c], es, ec


if __name__ == "__main__":
    S, C, es, ec = coefficients()
    print("// sin: relative error of the fit %.2e" % es)
    print("S = " + ", ".join(repr(v) + "f" for v in S))
    print("// cos: absolute error of the fit %.2e" % ec)
    print("C = " + ", ".join(repr(v) + "f" for v in C))
