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

    python paper_2005_14454_gb300/csrc/gen_link_sincos.py [--double]
prints them in the order the kernel uses (lowest power first).

FP64 precision mode (`--double`): sin r = r + r^3 S(r^2) with S of degree 7 (sin of
degree 17) and cos r = 1 + r^2 C(r^2) with C of degree 7 (cos of degree 16), fitted
the same way in 40-digit arithmetic (mpmath) on 400 Chebyshev nodes with 60 Lawson
passes; error of the fit 2.8e-19 relative (sin) and 4.2e-18 absolute (cos), the
coefficients rounded to FP64 once.
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


def coefficients64(nodes_n=400, iters=60):
    import mpmath as mp
    mp.mp.dps = 40

    def fit(fun, weight, powers, nodes):
        A = [[x ** p for p in powers] for x in nodes]
        f = [fun(x) for x in nodes]
        w = [weight(x) for x in nodes]
        u = [mp.mpf(1) / len(nodes)] * len(nodes)
        m = len(powers)
        for _ in range(iters):
            M, b = mp.matrix(m, m), mp.matrix(m, 1)
            for i in range(len(nodes)):
                wi = u[i] * w[i] ** 2
                for j in range(m):
                    b[j] += wi * A[i][j] * f[i]
                    for k in range(m):
                        M[j, k] += wi * A[i][j] * A[i][k]
            c = mp.lu_solve(M, b)
            e = [abs((sum(c[j] * A[i][j] for j in range(m)) - f[i]) * w[i]) for i in range(len(nodes))]
            tot = sum(u[i] * e[i] for i in range(len(nodes)))
            u = [u[i] * e[i] / tot for i in range(len(nodes))]
        return [float(c[j]) for j in range(m)], float(max(e))

    nodes = [(mp.cos(mp.pi * (i + mp.mpf(0.5)) / nodes_n) + 1) / 2 * mp.pi / 2 for i in range(nodes_n)]
    S, es = fit(lambda x: (mp.sin(x) - x) / x ** 3, lambda x: x ** 3 / mp.sin(x), list(range(0, 16, 2)), nodes)
    C, ec = fit(lambda x: (mp.cos(x) - 1) / x ** 2, lambda x: x ** 2, list(range(0, 16, 2)), nodes)
    return S, C, es, ec


if __name__ == "__main__":
    import sys
    if "--double" in sys.argv:
        S, C, es, ec = coefficients64()
        print("// sin: relative error of the fit %.2e" % es)
        print("S = " + ", ".join(repr(v) for v in S))
        print("// cos: absolute error of the fit %.2e" % ec)
        print("C = " + ", ".join(repr(v) for v in C))
        sys.exit(0)
    S, C, es, ec = coefficients()
    print("// sin: relative error of the fit %.2e" % es)
    print("S = " + ", ".join(repr(v) + "f" for v in S))
    print("// cos: absolute error of the fit %.2e" % ec)
    print("C = " + ", ".join(repr(v) + "f" for v in C))
