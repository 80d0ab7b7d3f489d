"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
monomial integrals, textbook P1 matrices (golden fixtures), the element sizes the
paper prints, exact rational integration of polynomial bilinear forms (sympy),
finite differences that are exact for the polynomial dependence on coefficients,
and invariants (symmetry, zero row sums, partition of unity, measure).
"""
import itertools
import os
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_1407_0904_gb300 import meshgen
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CELLS = [oracle.TRIANGLE, oracle.TETRAHEDRON]
NAME = {"triangle": oracle.TRIANGLE, "tetrahedron": oracle.TETRAHEDRON}
FORMS = {"mass": oracle.MASS, "helmholtz": oracle.HELMHOLTZ, "advdiff": oracle.ADVDIFF,
         "burgers_jac": oracle.BURGERS_JAC}


def ref_cell(cell):
    d = oracle.dim(cell)
    return np.vstack([np.zeros(d), np.eye(d)])


def one_cell(X):
    return np.asarray(X, dtype=np.float64), np.arange(len(X), dtype=np.int32)[None, :]


def scaled_err(A, B):
    return float(np.max(np.abs(A - B)) / np.max(np.abs(B)))


# --- quadrature -------------------------------------------------------------------
@pytest.mark.parametrize("cell", CELLS)
@pytest.mark.parametrize("p", range(0, 13))
def test_quadrature_integrates_monomials_exactly(cell, p):
    d = oracle.dim(cell)
    pts, w = oracle.quadrature(cell, p)
    assert np.all(w > 0)
    for e in itertools.product(range(p + 1), repeat=d):
        if sum(e) > p:
            continue
        val = np.sum(w * np.prod(pts ** np.array(e), axis=1))
        ex = np.prod([factorial(x) for x in e]) / factorial(sum(e) + d)
        assert abs(val - ex) <= 1e-14 * ex, (e, val, ex)


# --- basis ------------------------------------------------------------------------
@pytest.mark.parametrize("cell", CELLS)
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_basis_nodality_partition_and_linear_reproduction(cell, k):
    X = oracle.nodes(cell, k)
    phi, _ = oracle.basis(cell, k, X)
    assert np.abs(phi - np.eye(len(X))).max() < 1e-13
    x = np.random.default_rng(k).random((40, X.shape[1])) / X.shape[1]
    phi, dphi = oracle.basis(cell, k, x)
    assert np.abs(phi.sum(axis=1) - 1).max() < 1e-13
    assert np.abs(dphi.sum(axis=1)).max() < 1e-12
    assert np.abs(phi @ X - x).max() < 1e-13  # sum_i X_i phi_i(x) = x
    grad_x = np.einsum("pia,ib->pab", dphi, X)  # d/dxi_a of sum_i X_i[b] phi_i = delta_ab
    assert np.abs(grad_x - np.eye(X.shape[1])).max() < 1e-12


def test_node_order_lattice_c_slowest():
    X = oracle.nodes(oracle.TETRAHEDRON, 2)
    assert np.allclose(X[:4], [[0, 0, 0], [0.5, 0, 0], [1, 0, 0], [0, 0.5, 0]])
    assert np.allclose(oracle.nodes(oracle.TRIANGLE, 1), [[0, 0], [1, 0], [0, 1]])


# --- golden fixtures ----------------------------------------------------------------
def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_golden_element_sizes_printed_in_paper():
    rows = read_golden("element_sizes.txt")
    assert len(rows) >= 4
    for r in rows:
        if r[1] == "prism":
            assert r[0] == "helmholtz" and oracle.prism_ndof(int(r[2])) == int(r[3])
            continue
        form, cell, k, n = FORMS[r[0]], NAME[r[1]], int(r[2]), int(r[3])
        assert oracle.ndof(form, k, cell) == n


def test_golden_p1_reference_matrices():
    rows = read_golden("p1_reference_matrices.txt")
    assert len(rows) == 4
    for r in rows:
        cell, n = NAME[r[1]], int(r[2])
        M = np.array([float(Fraction(v)) for v in r[3:3 + n * n]]).reshape(n, n)
        X, c2v = one_cell(ref_cell(cell))
        mass = oracle.assemble(oracle.MASS, 1, cell, X, c2v)[0]
        helm = oracle.assemble(oracle.HELMHOLTZ, 1, cell, X, c2v)[0]
        got = mass if r[0] == "mass" else helm - mass
        assert np.abs(got - M).max() < 1e-15


# --- closed forms on physical cells --------------------------------------------------
def random_cells(cell, n, seed):
    d = oracle.dim(cell)
    rng = np.random.default_rng(seed)
    X = ref_cell(cell)[None] + rng.uniform(-0.25, 0.25, size=(n, d + 1, d))
    X = X * rng.uniform(0.5, 2.0, size=(n, 1, 1)) + rng.uniform(-3, 3, size=(n, 1, d))
    return X


def measure(X):
    d = X.shape[-1]
    J = np.swapaxes(X[:, 1:] - X[:, :1], 1, 2)
    return np.abs(np.linalg.det(J)) / factorial(d)


def barycentric_gradients(X):
    """grad lambda_v via the inverse of [[1, x_v]] (row v), independent of J/K."""
    n, nv, d = X.shape
    M = np.concatenate([np.ones((n, nv, 1)), X], axis=2)  # lambda = M^{-T} [1, x]
    Minv = np.linalg.inv(M)  # columns: coefficients of lambda_v
    return np.swapaxes(Minv[:, 1:, :], 1, 2)  # [n, v, d]


@pytest.mark.parametrize("cell", CELLS)
def test_p1_mass_and_stiffness_closed_forms(cell):
    X = random_cells(cell, 20, seed=7)
    nv = X.shape[1]
    c2v = np.arange(20 * nv, dtype=np.int32).reshape(20, nv)
    coords = X.reshape(-1, X.shape[2])
    mass = oracle.assemble(oracle.MASS, 1, cell, coords, c2v)
    helm = oracle.assemble(oracle.HELMHOLTZ, 1, cell, coords, c2v)
    vol = measure(X)
    base = np.ones((nv, nv)) + np.eye(nv)
    expect_mass = vol[:, None, None] * base / (12.0 if cell == oracle.TRIANGLE else 20.0)
    assert scaled_err(mass, expect_mass) < 1e-13
    G = barycentric_gradients(X)
    expect_stiff = vol[:, None, None] * np.einsum("nvd,nwd->nvw", G, G)
    assert scaled_err(helm - mass, expect_stiff) < 1e-12


@pytest.mark.parametrize("cell", CELLS)
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_mass_sum_symmetry_and_stiffness_row_sums(cell, k):
    X = random_cells(cell, 6, seed=10 + k)
    nv = X.shape[1]
    c2v = np.arange(6 * nv, dtype=np.int32).reshape(6, nv)
    coords = X.reshape(-1, X.shape[2])
    mass = oracle.assemble(oracle.MASS, k, cell, coords, c2v)
    helm = oracle.assemble(oracle.HELMHOLTZ, k, cell, coords, c2v)
    stiff = helm - mass
    vol = measure(X)
    assert np.allclose(mass.sum(axis=(1, 2)), vol, rtol=1e-13, atol=0)
    assert np.abs(mass - np.swapaxes(mass, 1, 2)).max() < 1e-15 * np.abs(mass).max() * 10
    assert np.abs(stiff - np.swapaxes(stiff, 1, 2)).max() < 1e-13 * np.abs(stiff).max()
    assert np.abs(stiff.sum(axis=2)).max() < 1e-12 * np.abs(stiff).max()
    # positive semi-definite stiffness, positive definite mass
    assert np.linalg.eigvalsh(mass).min() > 0
    assert np.linalg.eigvalsh(stiff).min() > -1e-12 * np.abs(stiff).max()


def test_mesh_mass_sums_to_domain_measure():
    m = meshgen.tri_mesh(16, perturb=0.2, seed=1)
    assert abs(oracle.assemble(oracle.MASS, 2, oracle.TRIANGLE, m.coords, m.cell2vert).sum() - 1) < 1e-13
    t = meshgen.tet_mesh(4, perturb=0.15, seed=2)
    assert abs(oracle.assemble(oracle.MASS, 3, oracle.TETRAHEDRON, t.coords, t.cell2vert).sum() - 1) < 1e-13


@pytest.mark.parametrize("cell", CELLS)
def test_translation_invariance_and_scaling(cell):
    d = oracle.dim(cell)
    X = random_cells(cell, 1, seed=3)[0]
    for form, power in [(oracle.MASS, d), (oracle.HELMHOLTZ, None)]:
        coords, c2v = one_cell(X)
        A = oracle.assemble(form, 3, cell, coords, c2v)[0]
        B = oracle.assemble(form, 3, cell, coords + np.array([5.5, -2.25, 1.0][:d]), c2v)[0]
        assert scaled_err(B, A) < 1e-12
    coords, c2v = one_cell(X)
    s = 0.375
    M1 = oracle.assemble(oracle.MASS, 2, cell, coords, c2v)[0]
    M2 = oracle.assemble(oracle.MASS, 2, cell, coords * s, c2v)[0]
    assert scaled_err(M2, M1 * s ** d) < 1e-13
    S1 = oracle.assemble(oracle.HELMHOLTZ, 2, cell, coords, c2v)[0] - M1
    S2 = oracle.assemble(oracle.HELMHOLTZ, 2, cell, coords * s, c2v)[0] - M2
    assert scaled_err(S2, S1 * s ** (d - 2)) < 1e-12


# --- exact bilinear identities (sympy) -----------------------------------------------
SIMPLEX = {
    oracle.TRIANGLE: [[sp.Rational(1, 8), sp.Rational(-1, 4)], [sp.Rational(9, 8), sp.Rational(1, 8)],
                      [sp.Rational(-1, 4), sp.Rational(5, 4)]],
    oracle.TETRAHEDRON: [[0, sp.Rational(1, 8), 0], [sp.Rational(5, 4), 0, sp.Rational(1, 4)],
                         [sp.Rational(1, 4), sp.Rational(9, 8), 0],
                         [sp.Rational(-1, 8), sp.Rational(1, 4), sp.Rational(3, 2)]],
}


def _grad(f, xs):
    return [sp.diff(f, x) for x in xs]


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3), (1, 4)])
def test_helmholtz_bilinear_identity_exact(cell, k):
    """Q^T A P = int grad p . grad q + p q for polynomials p, q of degree <= k."""
    d = oracle.dim(cell)
    X = SIMPLEX[cell]
    xs = exact.symbols(d)
    rng = np.random.default_rng(100 + 10 * cell + k)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    nodes = exact.physical_nodes(X, k)
    P = np.array([float(v) for v in exact.evaluate(p, xs, nodes)])
    Q = np.array([float(v) for v in exact.evaluate(q, xs, nodes)])
    coords, c2v = one_cell(exact.to_float_matrix(X))
    A = oracle.assemble(oracle.HELMHOLTZ, k, cell, coords, c2v)[0]
    M = oracle.assemble(oracle.MASS, k, cell, coords, c2v)[0]
    ex_h = float(exact.integrate_simplex(_dot(_grad(p, xs), _grad(q, xs)) + p * q, X, xs))
    ex_m = float(exact.integrate_simplex(p * q, X, xs))
    scale_h = np.abs(Q) @ np.abs(A) @ np.abs(P)
    scale_m = np.abs(Q) @ np.abs(M) @ np.abs(P)
    assert abs(Q @ A @ P - ex_h) < 1e-13 * scale_h
    assert abs(Q @ M @ P - ex_m) < 1e-13 * scale_m
    # the test-function index is the row: a non-symmetric check uses Q on the left only
    assert abs(P @ A @ Q - ex_h) < 1e-13 * scale_h


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3)])
def test_advdiff_bilinear_identity_exact(cell, k):
    """Q^T A P = int eps grad p . grad q + q (b . grad p) with P1 fields eps, b."""
    d = oracle.dim(cell)
    X = SIMPLEX[cell]
    xs = exact.symbols(d)
    rng = np.random.default_rng(200 + 10 * cell + k)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    eps = exact.random_poly(xs, 1, rng)
    b = [exact.random_poly(xs, 1, rng) for _ in range(d)]
    verts = [[sp.Rational(v) for v in row] for row in X]
    eps_v = np.array([float(v) for v in exact.evaluate(eps, xs, verts)])
    b_v = np.array([[float(bb.subs(dict(zip(xs, v)))) for bb in b] for v in verts])
    coef = np.concatenate([eps_v[:, None], b_v], axis=1).ravel()
    c2d = np.arange(d + 1, dtype=np.int32)[None]
    nodes = exact.physical_nodes(X, k)
    P = np.array([float(v) for v in exact.evaluate(p, xs, nodes)])
    Q = np.array([float(v) for v in exact.evaluate(q, xs, nodes)])
    coords, c2v = one_cell(exact.to_float_matrix(X))
    A = oracle.assemble(oracle.ADVDIFF, k, cell, coords, c2v, coef, c2d)[0]
    gp, gq = _grad(p, xs), _grad(q, xs)
    ex = float(exact.integrate_simplex(eps * _dot(gp, gq) + q * _dot(b, gp), X, xs))
    assert abs(Q @ A @ P - ex) < 1e-13 * (np.abs(Q) @ np.abs(A) @ np.abs(P))


def _burgers_cell(cell, k, seed):
    d = oracle.dim(cell)
    X = SIMPLEX[cell]
    xs = exact.symbols(d)
    rng = np.random.default_rng(seed)
    u = [exact.random_poly(xs, k, rng) for _ in range(d)]
    v = [exact.random_poly(xs, k, rng) for _ in range(d)]
    nodes = exact.physical_nodes(X, k)
    U = np.array([[float(ui.subs(dict(zip(xs, n)))) for ui in u] for n in nodes])  # [ns, d]
    V = np.array([[float(vi.subs(dict(zip(xs, n)))) for vi in v] for n in nodes])
    return X, xs, u, v, U, V


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_burgers_residual_exact(cell, k):
    """sum V.R(u) = int (u.grad u).v + nu grad u : grad v for vector polynomials u, v."""
    d = oracle.dim(cell)
    X, xs, u, v, U, V = _burgers_cell(cell, k, 300 + 10 * cell + k)
    nu = sp.Rational(1, 100)
    ns = U.shape[0]
    coords, c2v = one_cell(exact.to_float_matrix(X))
    c2d = np.arange(ns, dtype=np.int32)[None]
    R = oracle.burgers_residual(k, cell, coords, c2v, U, c2d, nu=0.01)[0]  # [(c, i)]
    Vb = V.T.ravel()  # blocked by component
    conv = sum(sum(u[m] * sp.diff(u[c], xs[m]) for m in range(d)) * v[c] for c in range(d))
    visc = sum(_dot(_grad(u[c], xs), _grad(v[c], xs)) for c in range(d))
    ex = float(exact.integrate_simplex(sp.expand(conv + nu * visc), X, xs))
    scale = np.abs(Vb) @ np.abs(R) + abs(ex)
    assert abs(Vb @ R - ex) < 1e-13 * scale


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3), (1, 4)])
def test_burgers_jacobian_equals_central_difference_of_residual(cell, k):
    """R is quadratic in u, so (R(u+h e_J) - R(u-h e_J)) / 2h is column J exactly, any h."""
    m = meshgen.tet_mesh(1, seed=5) if cell == oracle.TETRAHEDRON else meshgen.tri_mesh(1, seed=5)
    c2v = m.cell2vert[:1]
    c2d, nn = meshgen.cell2dof(m, k)
    c2d = c2d[:1]
    u = np.random.default_rng(k).standard_normal((nn, m.dim))
    A = oracle.assemble(oracle.BURGERS_JAC, k, cell, m.coords, c2v, u, c2d)[0]
    ns = c2d.shape[1]
    d = m.dim
    h = 1.0
    for cj in range(d):
        for j in range(ns):
            up, um = u.copy(), u.copy()
            up[c2d[0, j], cj] += h
            um[c2d[0, j], cj] -= h
            Rp = oracle.burgers_residual(k, cell, m.coords, c2v, up, c2d)[0]
            Rm = oracle.burgers_residual(k, cell, m.coords, c2v, um, c2d)[0]
            col = (Rp - Rm) / (2 * h)
            assert np.abs(col - A[:, cj * ns + j]).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("cell", CELLS)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_advdiff_constant_trial_and_linearity(cell, k):
    m = meshgen.tet_mesh(2, seed=6) if cell == oracle.TETRAHEDRON else meshgen.tri_mesh(3, seed=6)
    coef, c2d, nn = meshgen.advdiff_coefficients(m, seed=6)
    A = oracle.assemble(oracle.ADVDIFF, k, cell, m.coords, m.cell2vert, coef, c2d)
    assert np.abs(A.sum(axis=2)).max() < 1e-12 * np.abs(A).max()  # A 1 = 0
    c2 = np.random.default_rng(1).uniform(-1, 1, size=coef.shape)
    A2 = oracle.assemble(oracle.ADVDIFF, k, cell, m.coords, m.cell2vert, c2, c2d)
    A3 = oracle.assemble(oracle.ADVDIFF, k, cell, m.coords, m.cell2vert, 2 * coef - 3 * c2, c2d)
    assert scaled_err(A3, 2 * A - 3 * A2) < 1e-13
    # eps = 1, b = 0 reduces to the stiffness part of Helmholtz
    ones = np.concatenate([np.ones((nn, 1)), np.zeros((nn, m.dim))], axis=1).ravel()
    S = oracle.assemble(oracle.ADVDIFF, k, cell, m.coords, m.cell2vert, ones, c2d)
    H = oracle.assemble(oracle.HELMHOLTZ, k, cell, m.coords, m.cell2vert)
    M = oracle.assemble(oracle.MASS, k, cell, m.coords, m.cell2vert)
    assert scaled_err(S, H - M) < 1e-12


# --- backward ------------------------------------------------------------------------
def _local_loss(form, k, cell, coords, c2v, dout, coef, c2d, cells):
    A = oracle.assemble_cells(form, k, cell, coords, c2v, cells, coef, c2d)
    return float(np.sum(A * dout[cells]))


@pytest.mark.parametrize("form,cell,k", [(oracle.HELMHOLTZ, 1, 2), (oracle.ADVDIFF, 1, 2),
                                         (oracle.MASS, 0, 3), (oracle.HELMHOLTZ, 0, 2),
                                         (oracle.ADVDIFF, 0, 1), (oracle.BURGERS_JAC, 1, 1)])
def test_backward_matches_central_differences(form, cell, k):
    m = meshgen.tet_mesh(2, seed=9) if cell == oracle.TETRAHEDRON else meshgen.tri_mesh(3, seed=9)
    coef = c2d = None
    if form == oracle.ADVDIFF:
        coef, c2d, _ = meshgen.advdiff_coefficients(m, seed=9)
    elif form == oracle.BURGERS_JAC:
        coef, c2d, _ = meshgen.burgers_coefficients(m, k, seed=9)
    n = oracle.ndof(form, k, cell)
    rng = np.random.default_rng(11)
    dout = rng.standard_normal((m.ncells, n, n))
    gx, gc = oracle.assemble_backward(form, k, cell, m.coords, m.cell2vert, dout, coef, c2d)
    d = m.dim
    hx = 1e-6
    for vtx in rng.choice(m.nverts, size=4, replace=False):
        cells = np.nonzero((m.cell2vert == vtx).any(axis=1))[0]
        for r in range(d):
            cp, cm = m.coords.copy(), m.coords.copy()
            cp[vtx, r] += hx
            cm[vtx, r] -= hx
            fd = (_local_loss(form, k, cell, cp, m.cell2vert, dout, coef, c2d, cells)
                  - _local_loss(form, k, cell, cm, m.cell2vert, dout, coef, c2d, cells)) / (2 * hx)
            assert abs(fd - gx[vtx, r]) <= 1e-6 * max(abs(gx).max(), 1e-30), (vtx, r, fd, gx[vtx, r])
    if coef is not None:
        flat = coef.ravel()
        nn = c2d.max() + 1
        for idx in rng.choice(flat.size, size=6, replace=False):
            node = idx % nn if (form == oracle.ADVDIFF and idx < nn) else None
            cp, cm = flat.copy(), flat.copy()
            h = 1.0 if form == oracle.ADVDIFF else 1e-6  # advdiff is linear in its coefficients
            cp[idx] += h
            cm[idx] -= h
            cells = np.arange(m.ncells)
            fd = (_local_loss(form, k, cell, m.coords, m.cell2vert, dout, cp.reshape(coef.shape), c2d, cells)
                  - _local_loss(form, k, cell, m.coords, m.cell2vert, dout, cm.reshape(coef.shape), c2d, cells)) / (2 * h)
            g = gc.ravel()[idx]
            assert abs(fd - g) <= 1e-6 * max(abs(gc).max(), 1e-30), (idx, fd, g)
            del node


def test_mass_backward_closed_form():
    """For MASS, A_e = |det J| Mhat, so dL/dx = sum_e <dout_e, Mhat> d|det J|/dx."""
    m = meshgen.tet_mesh(2, seed=12)
    rng = np.random.default_rng(12)
    dout = rng.standard_normal((m.ncells, 4, 4))
    gx, _ = oracle.assemble_backward(oracle.MASS, 1, oracle.TETRAHEDRON, m.coords, m.cell2vert, dout)
    Mhat = (np.ones((4, 4)) + np.eye(4)) / 120.0  # reference P1 tet mass
    X = m.coords[m.cell2vert]
    J = np.swapaxes(X[:, 1:] - X[:, :1], 1, 2)
    det = np.linalg.det(J)
    dD_dJ = np.abs(det)[:, None, None] * np.swapaxes(np.linalg.inv(J), 1, 2)  # d|det|/dJ = |det| J^-T
    s = np.einsum("eij,ij->e", dout, Mhat)
    gJ = s[:, None, None] * dD_dJ  # [e, r, c], J[r][c] = x_{c+1}[r] - x_0[r]
    expect = np.zeros_like(m.coords)
    for c in range(3):
        np.add.at(expect, m.cell2vert[:, c + 1], gJ[:, :, c])
        np.add.at(expect, m.cell2vert[:, 0], -gJ[:, :, c])
    assert np.abs(gx - expect).max() < 1e-12 * np.abs(expect).max()
