"""Pins of the oracle's vector Burgers assembly on prisms (section 5.2 runs Burgers on the
third element shape too).

The rule ((3k+3)//2 Gauss-Legendre points per direction, Duffy-collapsed triangle factor) is
checked against exact monomial integrals; on sheared right prisms (affine map) it integrates
the residual's trilinear integrand exactly, so the residual is compared with the exact
sympy integral of the weak form for vector polynomials u, v; the Jacobian is the residual's
derivative (R is quadratic in u, so central differences are exact) on twisted prisms; at u = 0
it is nu times the vector Laplacian, i.e. nu (HELMHOLTZ - MASS) of the scalar prism assembly
(already pinned) on every diagonal block; constant fields have zero residual.
"""
from math import factorial

import numpy as np
import pytest
import sympy as sp

import oracle
from tests import exact
from tests.test_oracle_prism_pins import (prism_nodes_ref, prism_map, rational_prism, sym_map,
                                          integrate_ref_prism)

MASS, HELMHOLTZ = oracle.MASS, oracle.HELMHOLTZ


def one_prism(X, n):
    """coords, c2v, c2d of a single prism whose n nodes are its own coefficient nodes."""
    return (np.asarray(X, dtype=np.float64), np.arange(6, dtype=np.int32)[None],
            np.arange(n, dtype=np.int32)[None])


def twisted(seed):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]], dtype=np.float64)
    return X + rng.uniform(-0.15, 0.15, X.shape)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_burgers_rule_integrates_monomials_exactly(k):
    pts, w = oracle.prism_burgers_rule(k)
    n = (3 * k + 3) // 2
    assert np.all(w > 0) and len(w) == n ** 3
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            for c in range(2 * n):
                val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                ex = factorial(a) * factorial(b) / factorial(a + b + 2) / (c + 1)
                assert abs(val - ex) <= 4e-15 * ex + 1e-17, (a, b, c, val, ex)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_affine_prism_burgers_residual_exact(k):
    """sum V.R(u) = int (u.grad u).v + nu grad u : grad v on a sheared right prism, for vector
    polynomials u, v of degree k (the prism space holds them exactly, the rule integrates the
    degree 3k-1 integrand exactly)."""
    rng = np.random.default_rng(400 + k)
    Xs = rational_prism(rng, twisted=False)
    xs = exact.symbols(3)
    u = [exact.random_poly(xs, k, rng) for _ in range(3)]
    v = [exact.random_poly(xs, k, rng) for _ in range(3)]
    xi = sp.symbols("s t z")
    phys = sym_map(Xs, xi)
    J = sp.Matrix(3, 3, lambda r, c: sp.diff(phys[r], xi[c]))
    det = sp.simplify(J.det())
    assert det.is_number  # affine
    nu = sp.Rational(1, 100)
    conv = sum(sum(u[m] * sp.diff(u[c], xs[m]) for m in range(3)) * v[c] for c in range(3))
    visc = sum(sum(sp.diff(u[c], xs[m]) * sp.diff(v[c], xs[m]) for m in range(3)) for c in range(3))
    sub = dict(zip(xs, phys))
    ex = float(integrate_ref_prism(sp.expand((conv + nu * visc).subs(sub, simultaneous=True)) * abs(det), xi))
    X = np.array([[float(c) for c in row] for row in Xs])
    nodes = prism_map(X, prism_nodes_ref(k))
    U = np.array([[float(ui.subs(dict(zip(xs, p)))) for ui in u] for p in nodes])  # [n, 3]
    V = np.array([[float(vi.subs(dict(zip(xs, p)))) for vi in v] for p in nodes])
    R = oracle.prism_burgers(k, *one_prism(X, len(nodes))[:2], U, one_prism(X, len(nodes))[2], nu=0.01,
                             residual=True)[0]
    Vb = V.T.ravel()  # blocked by component, like R
    scale = np.abs(Vb) @ np.abs(R) + abs(ex)
    assert abs(Vb @ R - ex) < 1e-13 * scale


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_burgers_jacobian_equals_central_difference_of_residual(k):
    """Twisted (non-affine) prism: column (cj, j) of the Jacobian is (R(u + h e) - R(u - h e)) / 2h
    exactly, R being quadratic in u."""
    X = twisted(500 + k)
    n = oracle.prism_ndof(k)
    coords, c2v, c2d = one_prism(X, n)
    u = np.random.default_rng(k).standard_normal((n, 3))
    A = oracle.prism_burgers(k, coords, c2v, u, c2d)[0]
    assert A.shape == (3 * n, 3 * n)
    rng = np.random.default_rng(600 + k)
    cols = [(cj, j) for cj in range(3) for j in range(n)]
    for cj, j in [cols[i] for i in rng.choice(len(cols), size=min(len(cols), 24), replace=False)]:
        up, um = u.copy(), u.copy()
        up[j, cj] += 1.0
        um[j, cj] -= 1.0
        Rp = oracle.prism_burgers(k, coords, c2v, up, c2d, residual=True)[0]
        Rm = oracle.prism_burgers(k, coords, c2v, um, c2d, residual=True)[0]
        assert np.abs((Rp - Rm) / 2.0 - A[:, cj * n + j]).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_burgers_at_zero_velocity_is_nu_times_the_laplacian(k):
    """u = 0 leaves nu grad du : grad v: every diagonal block is nu (HELMHOLTZ - MASS) of the scalar
    prism assembly, the off-diagonal blocks vanish (affine prism: both rules exact)."""
    rng = np.random.default_rng(700 + k)
    X = np.array([[float(c) for c in row] for row in rational_prism(rng, twisted=False)])
    n = oracle.prism_ndof(k)
    coords, c2v, c2d = one_prism(X, n)
    A = oracle.prism_burgers(k, coords, c2v, np.zeros((n, 3)), c2d, nu=0.25)[0]
    S = oracle.prism_assemble(HELMHOLTZ, k, coords, c2v)[0] - oracle.prism_assemble(MASS, k, coords, c2v)[0]
    for ci in range(3):
        for cj in range(3):
            blk = A[ci * n:(ci + 1) * n, cj * n:(cj + 1) * n]
            want = 0.25 * S if ci == cj else np.zeros_like(S)
            assert np.abs(blk - want).max() < 1e-13 * np.abs(S).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_twisted_prism_constant_velocity_has_zero_residual_and_jacobian_rows_of_its_advection(k):
    """For constant u (grad u = 0 at every point) R(u) = 0, and J(u) w = J(0) w + the advection
    term int (u.grad w).v, linear in u: J(u) - J(0) is linear in u (tested for u and 2u)."""
    X = twisted(800 + k)
    n = oracle.prism_ndof(k)
    coords, c2v, c2d = one_prism(X, n)
    c = np.array([0.3, -1.2, 0.7])
    U = np.tile(c, (n, 1))
    R = oracle.prism_burgers(k, coords, c2v, U, c2d, residual=True)[0]
    A0 = oracle.prism_burgers(k, coords, c2v, np.zeros((n, 3)), c2d)[0]
    A1 = oracle.prism_burgers(k, coords, c2v, U, c2d)[0]
    A2 = oracle.prism_burgers(k, coords, c2v, 2 * U, c2d)[0]
    assert np.abs(R).max() < 1e-13 * (np.abs(A1).max() * np.abs(c).max())
    assert np.abs((A2 - A0) - 2 * (A1 - A0)).max() < 1e-13 * np.abs(A2).max()
