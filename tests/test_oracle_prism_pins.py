"""Pins of the oracle's prism assembly (the paper's third element shape, section 5.2).

Prisms are not affine: the Jacobian varies over the cell, so the element matrix is the
quadrature sum of a fixed rule rather than an exact integral. The pins therefore check the
rule against exact monomial integrals, the basis against its defining properties, right
(affine) prisms against exact rational integration of polynomial bilinear forms (the rule is
exact there), and twisted prisms against what holds for any quadrature of this rule: the
mass integrand is polynomial (its sum is the exact volume), stiffness annihilates constants,
and for linear functions the stiffness form is pointwise constant.
"""
from math import factorial

import numpy as np
import pytest
import sympy as sp

import oracle
from tests import exact

MASS, HELMHOLTZ = oracle.MASS, oracle.HELMHOLTZ


def tri_lattice(k):
    return [(a, b) for b in range(k + 1) for a in range(k + 1 - b)]


def prism_nodes_ref(k):
    """Reference nodes (a/k, b/k, c/k): zeta level c slowest, triangle lattice order inside."""
    return np.array([(a / k, b / k, c / k) for c in range(k + 1) for (a, b) in tri_lattice(k)])


def prism_map(X, xi):
    """Physical point of the prism with vertices X [6, 3] at reference points xi [n, 3]."""
    s, t, z = xi[:, 0:1], xi[:, 1:2], xi[:, 2:3]
    lam = [1 - s - t, s, t]
    return sum(lam[v] * ((1 - z) * X[v] + z * X[v + 3]) for v in range(3))


def one_prism(X):
    return np.asarray(X, dtype=np.float64), np.arange(6, dtype=np.int32)[None]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_rule_integrates_monomials_exactly(k):
    pts, w = oracle.prism_rule(k)
    assert np.all(w > 0) and len(w) == (k + 2) ** 3
    for a in range(2 * k + 3):
        for b in range(2 * k + 3 - a):
            for c in range(2 * k + 4):
                val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                ex = factorial(a) * factorial(b) / factorial(a + b + 2) / (c + 1)
                assert abs(val - ex) <= 2e-15 * ex + 1e-17, (a, b, c, val, ex)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_basis_nodal_partition_and_linear_reproduction(k):
    nodes = prism_nodes_ref(k)
    phi, dphi = oracle.prism_basis(k, nodes)
    np.testing.assert_allclose(phi, np.eye(len(nodes)), atol=1e-12)
    rng = np.random.default_rng(k)
    x = rng.random((20, 3))
    x[:, :2] *= 0.5  # inside the triangle
    phi, dphi = oracle.prism_basis(k, x)
    np.testing.assert_allclose(phi.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(dphi.sum(axis=1), 0.0, atol=1e-10)
    np.testing.assert_allclose(phi @ nodes, x, atol=1e-12)  # linear functions are reproduced
    for a in range(3):
        np.testing.assert_allclose(np.einsum("pi,pi->p", dphi[:, :, a], np.tile(nodes[:, a], (20, 1))),
                                   1.0, atol=1e-10)


def test_p1_reference_prism_mass_is_triangle_mass_times_interval_mass():
    X, c2v = one_prism([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]])
    M = oracle.prism_assemble(MASS, 1, X, c2v)[0]
    Mt = (1.0 / 24.0) * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])  # |T| = 1/2
    Ml = (1.0 / 6.0) * np.array([[2, 1], [1, 2]])
    np.testing.assert_allclose(M, np.kron(Ml, Mt), rtol=0, atol=1e-15)  # zeta level slowest


def rational_prism(rng, twisted):
    """Vertices with small rational coordinates: a sheared right prism (affine) or a twisted one."""
    frac = lambda: sp.Rational(int(rng.integers(-3, 4)), 8)
    base = [[sp.Rational(0), sp.Rational(0), sp.Rational(0)],
            [sp.Rational(1) + frac(), frac(), frac() / 2],
            [frac(), sp.Rational(1) + frac(), frac() / 2]]
    shift = [frac(), frac(), sp.Rational(1) + frac()]
    top = [[base[v][r] + shift[r] + (frac() / 2 if twisted else 0) for r in range(3)] for v in range(3)]
    return base + top


def sym_map(Xs, xi):
    s, t, z = xi
    lam = [1 - s - t, s, t]
    return [sum(lam[v] * ((1 - z) * Xs[v][r] + z * Xs[v + 3][r]) for v in range(3)) for r in range(3)]


def integrate_ref_prism(f, xi):
    """Exact integral over the reference prism of a polynomial f(s, t, z)."""
    s, t, z = xi
    return sp.integrate(sp.integrate(sp.integrate(f, (s, 0, 1 - t)), (t, 0, 1)), (z, 0, 1))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_affine_prism_bilinear_identity_exact(k):
    """On a sheared right prism the map is affine and the rule exact: Q^T A P = int grad p.grad q + pq."""
    rng = np.random.default_rng(50 + k)
    Xs = rational_prism(rng, twisted=False)
    xs = exact.symbols(3)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    xi = sp.symbols("s t z")
    phys = sym_map(Xs, xi)
    J = sp.Matrix(3, 3, lambda r, c: sp.diff(phys[r], xi[c]))
    det = sp.simplify(J.det())
    assert det.is_number  # affine
    sub = dict(zip(xs, phys))
    integrand = sum(sp.diff(p, x) * sp.diff(q, x) for x in xs) + p * q
    ex = float(integrate_ref_prism(sp.expand(integrand.subs(sub, simultaneous=True)) * abs(det), xi))
    X = np.array([[float(v) for v in row] for row in Xs])
    nodes = prism_map(X, prism_nodes_ref(k))
    P = np.array([float(p.subs(dict(zip(xs, n)))) for n in nodes])
    Q = np.array([float(q.subs(dict(zip(xs, n)))) for n in nodes])
    A = oracle.prism_assemble(HELMHOLTZ, k, *one_prism(X))[0]
    scale = np.abs(Q) @ np.abs(A) @ np.abs(P)
    assert abs(Q @ A @ P - ex) < 1e-12 * scale
    assert abs(P @ A @ Q - ex) < 1e-12 * scale


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_twisted_prism_volume_rowsums_and_linear_stiffness(k):
    rng = np.random.default_rng(70 + k)
    Xs = rational_prism(rng, twisted=True)
    xi = sp.symbols("s t z")
    phys = sym_map(Xs, xi)
    J = sp.Matrix(3, 3, lambda r, c: sp.diff(phys[r], xi[c]))
    det = sp.expand(J.det())
    assert not det.is_number  # not affine
    vol = float(integrate_ref_prism(det, xi))  # det > 0 throughout for these small twists
    X = np.array([[float(v) for v in row] for row in Xs])
    c = one_prism(X)
    M = oracle.prism_assemble(MASS, k, *c)[0]
    H = oracle.prism_assemble(HELMHOLTZ, k, *c)[0]
    K = H - M
    assert abs(M.sum() - vol) < 1e-13 * vol
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(M, M.T, atol=1e-15 * np.abs(M).max())
    np.testing.assert_allclose(K, K.T, atol=1e-14 * np.abs(K).max())
    assert np.linalg.eigvalsh(M).min() > 0
    # linear p, q lie in the space (isoparametric): grad p . grad q is constant at every point
    nodes = prism_map(X, prism_nodes_ref(k))
    a, b = rng.standard_normal(3), rng.standard_normal(3)
    P, Q = nodes @ a + 0.3, nodes @ b - 0.7
    assert abs(Q @ K @ P - vol * (a @ b)) < 1e-12 * (np.abs(Q) @ np.abs(K) @ np.abs(P))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prism_mesh_global_mass_is_the_unit_cube_and_numbering_conforms(k):
    """The perturbed prism mesh tiles the unit cube (boundary fixed): the assembled global mass
    matrix sums to 1, the global stiffness annihilates constants, and every cell places a shared
    node at the same physical point."""
    from paper_1407_0904_gb300 import meshgen
    m = meshgen.prism_mesh(3, 2, perturb=0.15, seed=6)
    c2d, nn = meshgen.cell2dof(m, k)
    X = m.coords[m.cell2vert]  # [ncells, 6, 3]
    ref = prism_nodes_ref(k)
    pts = np.stack([prism_map(X[e], ref) for e in range(m.ncells)])
    where = np.full((nn, 3), np.nan)
    where[c2d.ravel()] = pts.reshape(-1, 3)
    assert np.max(np.abs(where[c2d.ravel()] - pts.reshape(-1, 3))) < 1e-14
    rp, ci = oracle.csr_pattern(c2d, nn)
    M = oracle.csr_assemble(oracle.prism_assemble(MASS, k, m.coords, m.cell2vert), c2d, rp, ci)
    H = oracle.csr_assemble(oracle.prism_assemble(HELMHOLTZ, k, m.coords, m.cell2vert), c2d, rp, ci)
    assert abs(M.sum() - 1.0) < 1e-13
    rows = np.repeat(np.arange(nn), np.diff(rp))
    np.testing.assert_allclose(np.bincount(rows, weights=H - M, minlength=nn), 0.0, atol=1e-12 * np.abs(H).max())


ADVDIFF = oracle.ADVDIFF


def vertex_coef(rng, X):
    """(eps, b) rows per prism vertex: eps = a0 + a.x and b = B x + c, linear in the position."""
    a0, a = 1.0 + 0.2 * rng.random(), 0.3 * rng.standard_normal(3)
    Bm, cvec = 0.5 * rng.standard_normal((3, 3)), rng.standard_normal(3)
    eps = a0 + X @ a
    b = X @ Bm.T + cvec
    return np.concatenate([eps[:, None], b], axis=1), (a0, a, Bm, cvec)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_twisted_prism_advdiff_annihilates_constants_linear_and_reduces_to_stiffness(k):
    rng = np.random.default_rng(90 + k)
    X = np.array([[float(v) for v in row] for row in rational_prism(rng, twisted=True)])
    c2v = np.arange(6, dtype=np.int32)[None]
    c2d = c2v.copy()
    coef1, _ = vertex_coef(rng, X)
    coef2, _ = vertex_coef(rng, X)
    A1 = oracle.prism_assemble(ADVDIFF, k, X, c2v, coef1.ravel(), c2d)[0]
    A2 = oracle.prism_assemble(ADVDIFF, k, X, c2v, coef2.ravel(), c2d)[0]
    A12 = oracle.prism_assemble(ADVDIFF, k, X, c2v, (0.3 * coef1 - 1.7 * coef2).ravel(), c2d)[0]
    np.testing.assert_allclose(A1.sum(axis=1), 0.0, atol=1e-12 * np.abs(A1).max())  # A 1 = 0
    np.testing.assert_allclose(A12, 0.3 * A1 - 1.7 * A2, atol=1e-13 * np.abs(A12).max())
    unit = np.zeros((6, 4))
    unit[:, 0] = 1.0  # eps = 1, b = 0: the stiffness part of Helmholtz
    S = oracle.prism_assemble(ADVDIFF, k, X, c2v, unit.ravel(), c2d)[0]
    H = oracle.prism_assemble(HELMHOLTZ, k, X, c2v)[0] - oracle.prism_assemble(MASS, k, X, c2v)[0]
    np.testing.assert_allclose(S, H, atol=1e-13 * np.abs(H).max())


@pytest.mark.parametrize("k", [1, 2])
def test_affine_prism_advdiff_bilinear_identity_exact(k):
    """Sheared right prism, eps and b linear in x: Q^T A P = int eps grad p.grad q + q (b.grad p)."""
    rng = np.random.default_rng(110 + k)
    Xs = rational_prism(rng, twisted=False)
    X = np.array([[float(v) for v in row] for row in Xs])
    coef, (a0, a, Bm, cvec) = vertex_coef(rng, X)
    xs = exact.symbols(3)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    eps = a0 + sum(float(a[r]) * xs[r] for r in range(3))
    b = [sum(float(Bm[c, r]) * xs[r] for r in range(3)) + float(cvec[c]) for c in range(3)]
    xi = sp.symbols("s t z")
    phys = sym_map(Xs, xi)
    J = sp.Matrix(3, 3, lambda r, c: sp.diff(phys[r], xi[c]))
    det = sp.simplify(J.det())
    gp = [sp.diff(p, x) for x in xs]
    gq = [sp.diff(q, x) for x in xs]
    integrand = eps * sum(u * v for u, v in zip(gp, gq)) + q * sum(bb * g for bb, g in zip(b, gp))
    ex = float(integrate_ref_prism(sp.expand(integrand.subs(dict(zip(xs, phys)), simultaneous=True)) * abs(det), xi))
    nodes = prism_map(X, prism_nodes_ref(k))
    P = np.array([float(p.subs(dict(zip(xs, n)))) for n in nodes])
    Q = np.array([float(q.subs(dict(zip(xs, n)))) for n in nodes])
    A = oracle.prism_assemble(ADVDIFF, k, X, np.arange(6, dtype=np.int32)[None], coef.ravel(),
                              np.arange(6, dtype=np.int32)[None])[0]
    assert abs(Q @ A @ P - ex) < 1e-11 * (np.abs(Q) @ np.abs(A) @ np.abs(P))
