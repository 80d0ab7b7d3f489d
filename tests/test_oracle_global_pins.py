"""Pins of the oracle's global assembly (the consumer of local assembly: element
matrices added into a global sparse matrix through the local-to-global dof map).

The global matrix is checked against facts that do not come from the oracle:
  * its sparsity against brute-force sets of dof pairs;
  * the domain identities of a conforming degree-k space on a mesh of the unit square /
    cube whose boundary is fixed: for polynomials p, q of degree <= k, the nodal vectors
    P, Q satisfy Q^T A P = integral over the box of the bilinear form, computed exactly
    (sympy) from monomial integrals over [0, 1]^d -- this fixes every scatter index and
    every summation;
  * the quadratic dependence of the Burgers residual on u: the assembled global
    Jacobian times a direction equals the central difference of the assembled residual.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from paper_1407_0904_gb300 import meshgen
from tests import exact


def small_mesh(cell, seed=11):
    if cell == oracle.TRIANGLE:
        return meshgen.tri_mesh(4, perturb=0.2, seed=seed)
    return meshgen.tet_mesh(2, perturb=0.15, seed=seed)


def node_coordinates(mesh, k, c2d, nnodes):
    """Physical position of every global degree-k node; asserts that all cells sharing a
    node place it at the same point (the numbering is conforming)."""
    d = mesh.dim
    L = np.array(exact.lattice(d, k), dtype=np.float64) / k  # [ns, d]
    X = mesh.coords[mesh.cell2vert]  # [ncells, d+1, d]
    pts = X[:, :1, :] + np.einsum("na,cad->cnd", L, X[:, 1:, :] - X[:, :1, :])
    out = np.full((nnodes, d), np.nan)
    flat_ids, flat_pts = c2d.ravel(), pts.reshape(-1, d)
    out[flat_ids] = flat_pts
    assert np.max(np.abs(out[flat_ids] - flat_pts)) < 1e-14
    return out


def box_integral(f, xs):
    """Exact integral of a sympy polynomial over [0, 1]^d."""
    g = sp.Poly(sp.expand(f), *xs)
    total = sp.Rational(0)
    for mon, coeff in g.terms():
        term = coeff
        for e in mon:
            term *= sp.Rational(1, e + 1)
        total += term
    return total


def grad(f, xs):
    return [sp.diff(f, x) for x in xs]


def dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def at_nodes(f, xs, pts):
    fn = sp.lambdify(xs, f, "numpy")
    v = fn(*[pts[:, r] for r in range(pts.shape[1])])
    return np.broadcast_to(np.asarray(v, dtype=np.float64), (pts.shape[0],)).copy()


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_pattern_is_the_set_of_cell_dof_pairs(cell, k):
    m = small_mesh(cell)
    c2d, nn = meshgen.cell2dof(m, k, permute_seed=5)
    rowptr, colidx = oracle.csr_pattern(c2d, nn)
    pairs = set()
    for row in c2d:
        for a in row:
            for b in row:
                pairs.add((int(a), int(b)))
    got = set()
    for r in range(nn):
        cols = colidx[rowptr[r]:rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
        got.update((r, int(c)) for c in cols)
    assert got == pairs
    assert rowptr[-1] == len(pairs)


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3)])
def test_global_helmholtz_and_mass_domain_identity(cell, k):
    """Q^T A P = int_[0,1]^d grad p . grad q + p q, and 1^T M 1 = 1 (the box's measure)."""
    m = small_mesh(cell)
    d = m.dim
    c2d, nn = meshgen.cell2dof(m, k)
    xs = exact.symbols(d)
    rng = np.random.default_rng(40 + 10 * cell + k)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    pts = node_coordinates(m, k, c2d, nn)
    P, Q = at_nodes(p, xs, pts), at_nodes(q, xs, pts)
    rowptr, colidx = oracle.csr_pattern(c2d, nn)
    A_e = oracle.assemble(oracle.HELMHOLTZ, k, m.cell, m.coords, m.cell2vert)
    M_e = oracle.assemble(oracle.MASS, k, m.cell, m.coords, m.cell2vert)
    A = oracle.csr_dense(rowptr, colidx, oracle.csr_assemble(A_e, c2d, rowptr, colidx))
    M = oracle.csr_dense(rowptr, colidx, oracle.csr_assemble(M_e, c2d, rowptr, colidx))
    ex = float(box_integral(dot(grad(p, xs), grad(q, xs)) + p * q, xs))
    scale = np.abs(Q) @ np.abs(A) @ np.abs(P)
    assert abs(Q @ A @ P - ex) < 1e-12 * scale
    assert abs(P @ A @ Q - ex) < 1e-12 * scale
    assert abs(M.sum() - 1.0) < 1e-13
    # stiffness annihilates constants; the matrix is symmetric
    np.testing.assert_allclose((A - M).sum(axis=1), 0.0, atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(A, A.T, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_global_advdiff_domain_identity(cell, k):
    """Q^T A P = int eps grad p . grad q + q (b . grad p) with eps, b linear over the box."""
    m = small_mesh(cell)
    d = m.dim
    c2d, nn = meshgen.cell2dof(m, k)
    c1, n1 = meshgen.cell2dof(m, 1)
    xs = exact.symbols(d)
    rng = np.random.default_rng(70 + 10 * cell + k)
    p, q = exact.random_poly(xs, k, rng), exact.random_poly(xs, k, rng)
    eps = exact.random_poly(xs, 1, rng)
    b = [exact.random_poly(xs, 1, rng) for _ in range(d)]
    vpts = node_coordinates(m, 1, c1, n1)
    coef = np.concatenate([at_nodes(eps, xs, vpts)[:, None]] + [at_nodes(bb, xs, vpts)[:, None] for bb in b],
                          axis=1).ravel()
    pts = node_coordinates(m, k, c2d, nn)
    P, Q = at_nodes(p, xs, pts), at_nodes(q, xs, pts)
    rowptr, colidx = oracle.csr_pattern(c2d, nn)
    A_e = oracle.assemble(oracle.ADVDIFF, k, m.cell, m.coords, m.cell2vert, coef, c1)
    A = oracle.csr_dense(rowptr, colidx, oracle.csr_assemble(A_e, c2d, rowptr, colidx))
    gp, gq = grad(p, xs), grad(q, xs)
    ex = float(box_integral(eps * dot(gp, gq) + q * dot(b, gp), xs))
    assert abs(Q @ A @ P - ex) < 1e-12 * (np.abs(Q) @ np.abs(A) @ np.abs(P))


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_global_burgers_jacobian_is_difference_of_global_residual(cell, k):
    m = small_mesh(cell)
    d = m.dim
    c2d, nn = meshgen.cell2dof(m, k)
    rng = np.random.default_rng(90 + 10 * cell + k)
    u = rng.standard_normal((nn, d))
    l2g = np.concatenate([c2d.astype(np.int64) + c * nn for c in range(d)], axis=1)  # component-blocked
    rowptr, colidx = oracle.csr_pattern(l2g, d * nn)
    J_e = oracle.assemble(oracle.BURGERS_JAC, k, m.cell, m.coords, m.cell2vert, u.ravel(), c2d)
    J = oracle.csr_dense(rowptr, colidx, oracle.csr_assemble(J_e, l2g, rowptr, colidx))

    def residual(uu):
        R_e = oracle.burgers_residual(k, m.cell, m.coords, m.cell2vert, uu, c2d)
        return np.bincount(l2g.ravel(), weights=R_e.ravel(), minlength=d * nn)

    du = rng.standard_normal((nn, d))
    h = 0.37  # any step: R is quadratic in u
    fd = (residual(u + h * du) - residual(u - h * du)) / (2 * h)
    Jdu = J @ du.T.ravel()  # global vectors are blocked by component
    assert np.max(np.abs(Jdu - fd)) < 1e-12 * np.max(np.abs(J)) * np.abs(du).sum() / du.shape[0]
