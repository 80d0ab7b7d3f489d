"""Exact (rational) integration of polynomials over physical simplices, for pinning
the oracle independently of any quadrature rule.

A polynomial f(x) over the simplex with vertices X0..Xd is integrated by the affine
map x = X0 + J xi: int_T f = |det J| int_ref f(X0 + J xi) dxi, and each monomial
xi^a eta^b zeta^c of the reference simplex integrates to a! b! c! / (a+b+c+d)!.
"""
from fractions import Fraction
from math import factorial

import sympy as sp


def symbols(d):
    return sp.symbols("x0:%d" % d)


def integrate_simplex(f, X, xs):
    """Exact integral of the sympy polynomial f(xs) over the simplex with rational vertices X."""
    d = len(xs)
    X = [[sp.Rational(v) for v in row] for row in X]
    J = sp.Matrix(d, d, lambda r, c: X[c + 1][r] - X[0][r])
    det = J.det()
    xi = sp.symbols("xi0:%d" % d)
    sub = {xs[r]: X[0][r] + sum(J[r, c] * xi[c] for c in range(d)) for r in range(d)}
    g = sp.Poly(sp.expand(f.subs(sub, simultaneous=True)), *xi)
    total = sp.Rational(0)
    for mon, coeff in g.terms():
        num = 1
        for e in mon:
            num *= factorial(e)
        total += coeff * sp.Rational(num, factorial(sum(mon) + d))
    return abs(det) * total


def lattice(d, k):
    out = []
    cmax = k if d == 3 else 0
    for c in range(cmax + 1):
        for b in range(k - c + 1):
            for a in range(k - b - c + 1):
                out.append((a, b, c)[:d])
    return out


def physical_nodes(X, k):
    """Degree-k Lagrange nodes of the simplex X (rational), in the library's node order."""
    d = len(X) - 1
    X = [[sp.Rational(v) for v in row] for row in X]
    nodes = []
    for idx in lattice(d, k):
        lam = [sp.Rational(i, k) for i in idx]
        p = [X[0][r] + sum(lam[c] * (X[c + 1][r] - X[0][r]) for c in range(d)) for r in range(d)]
        nodes.append(p)
    return nodes


def random_poly(xs, k, rng):
    """A polynomial of total degree <= k with small random rational coefficients."""
    d = len(xs)
    f = sp.Rational(0)
    for mon in lattice(d, k):
        c = sp.Rational(int(rng.integers(-8, 9)), int(rng.integers(1, 5)))
        term = c
        for r, e in enumerate(mon):
            term *= xs[r] ** e
        f += term
    return sp.expand(f)


def evaluate(f, xs, pts):
    return [f.subs(dict(zip(xs, p)), simultaneous=True) for p in pts]


def to_float_matrix(X):
    return [[float(Fraction(str(v))) for v in row] for row in X]
