"""The seeded input recipe: mesh sizes of the benchmark configurations, perturbation bounds,
no inverted or degenerate cells, conforming degree-k numbering, coefficient ranges and the
Zipf split of the mixed batch. These are properties of the inputs both the CUDA path and the
oracle consume; none of them involves the assembly arithmetic."""
import numpy as np
import pytest

from paper_1407_0904_gb300 import meshgen


def det_and_volume(mesh):
    X = mesh.coords[mesh.cell2vert]                       # [ncells, d+1, d]
    J = (X[:, 1:] - X[:, :1]).transpose(0, 2, 1)          # columns x_{c+1} - x_0
    det = np.linalg.det(J)
    fact = 2.0 if mesh.dim == 2 else 6.0
    return det, np.abs(det) / fact


def test_configuration_sizes():
    assert meshgen.tri_mesh(64, seed=1).ncells == 8192
    assert meshgen.tri_mesh(512, seed=4).ncells == 2 ** 19
    m = meshgen.tet_mesh(64, 64, 43, seed=3, ncells=2 ** 20)
    assert m.ncells == 2 ** 20 and m.cell2vert.max() < m.nverts
    assert meshgen.tet_mesh(64, 64, 22, seed=5, ncells=2 ** 19).ncells == 2 ** 19
    assert meshgen.prism_mesh(48, 48, seed=6).ncells == 221184


@pytest.mark.parametrize("make,p", [(lambda: meshgen.tri_mesh(64, perturb=0.2, seed=1), 0.2),
                                    (lambda: meshgen.tet_mesh(24, perturb=0.15, seed=2), 0.15)])
def test_perturbation_bounds_and_no_inverted_cells(make, p):
    m = make()
    n = np.asarray(m.shape)
    grid_pts = np.zeros_like(m.coords)
    grid_pts[m.cell2vert.ravel()] = m.grid.reshape(-1, m.dim)
    disp = (m.coords - grid_pts / n) * n                  # in units of h
    interior = np.all((grid_pts > 0) & (grid_pts < n), axis=1)
    assert np.abs(disp[interior]).max() <= p and np.abs(disp[interior]).max() > 0.9 * p
    assert np.abs(disp[~interior]).max() < 1e-12          # boundary fixed: the box is tiled exactly
    det, vol = det_and_volume(m)
    h = 1.0 / n[0]
    # the unperturbed cells have |det| = h^d; the bounded moves keep every cell well away from 0
    assert np.abs(det).min() > 0.05 * h ** m.dim
    assert abs(vol.sum() - 1.0) < 1e-12


def test_kuhn_orientations_alternate_and_cover_the_cube():
    m = meshgen.tet_mesh(4, perturb=0.0, seed=2)
    det, vol = det_and_volume(m)
    assert np.allclose(np.abs(det), (1 / 4) ** 3)
    assert (det > 0).sum() == (det < 0).sum() == m.ncells // 2
    assert abs(vol.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 3), (1, 2), (1, 4), (2, 2)])
def test_numbering_is_conforming_and_seeded(cell, k):
    m = {0: lambda: meshgen.tri_mesh(6, seed=1), 1: lambda: meshgen.tet_mesh(3, seed=2),
         2: lambda: meshgen.prism_mesh(3, 2, seed=6)}[cell]()
    c2d, nn = meshgen.cell2dof(m, k)
    # every lattice point of the refined grid is used, and one point has one id everywhere
    assert c2d.min() == 0 and c2d.max() == nn - 1 and len(np.unique(c2d)) == nn
    # a node at a cell's vertex carries that vertex's id on the refined grid, so neighbours agree
    per_cell = len(meshgen.lattice(cell if cell != 2 else 0, k)) * (k + 1 if cell == 2 else 1)
    assert c2d.shape == (m.ncells, per_cell)
    dims = np.array([k * s + 1 for s in m.shape])
    pts = _lattice_points(cell, k)
    for v, corner in enumerate(_corners(cell, k)):
        col = pts.index(corner)
        expect = np.zeros(m.ncells, dtype=np.int64)
        mult = 1
        for a in range(m.dim):
            expect += k * m.grid[:, v, a] * mult
            mult *= dims[a]
        assert np.array_equal(c2d[:, col], expect), (v, corner)
    # the permuted variant is a relabelling by a seeded permutation
    p1, _ = meshgen.cell2dof(m, k, permute_seed=5)
    p2, _ = meshgen.cell2dof(m, k, permute_seed=5)
    assert np.array_equal(p1, p2) and not np.array_equal(p1, c2d)
    perm = np.full(nn, -1)
    perm[c2d.ravel()] = p1.ravel()
    assert (perm >= 0).all() and len(np.unique(perm)) == nn


def _lattice_points(cell, k):
    if cell == 2:
        return [(a, b, c) for c in range(k + 1) for (a, b) in map(tuple, meshgen.lattice(0, k))]
    return list(map(tuple, meshgen.lattice(cell, k)))


def _corners(cell, k):
    """Lattice point of each vertex of the cell, in vertex order."""
    if cell == 0:
        return [(0, 0), (k, 0), (0, k)]
    if cell == 1:
        return [(0, 0, 0), (k, 0, 0), (0, k, 0), (0, 0, k)]
    return [(0, 0, 0), (k, 0, 0), (0, k, 0), (0, 0, k), (k, 0, k), (0, k, k)]


def test_coefficient_ranges_and_seeding():
    m = meshgen.tet_mesh(6, seed=3)
    coef, c2d, nn = meshgen.advdiff_coefficients(m, seed=3)
    rows = coef.reshape(nn, 4)
    assert rows[:, 0].min() >= 0.5 and rows[:, 0].max() <= 1.5
    assert np.abs(rows[:, 1:]).max() <= 1.0
    assert np.array_equal(c2d, m.cell2vert)              # P1 nodes are the vertices
    u, c2, nn2 = meshgen.burgers_coefficients(m, 2, seed=3)
    assert u.shape == (nn2, 3) and abs(u.mean()) < 0.05 and abs(u.std() - 1.0) < 0.05
    u2, _, _ = meshgen.burgers_coefficients(m, 2, seed=3)
    assert np.array_equal(u, u2)


def test_zipf_split_of_the_mixed_batch():
    counts = meshgen.zipf_counts(12, 2 ** 19, s=1.0, seed=4)
    assert counts.sum() == 2 ** 19 and (counts > 0).all()
    ranks = np.random.default_rng(4).permutation(12) + 1
    order = np.argsort(ranks)
    assert np.all(np.diff(counts[order]) <= 0)            # larger rank, fewer cells
    tri, tet = meshgen.tri_mesh(32, seed=4), meshgen.tet_mesh(8, seed=5)
    groups = meshgen.batch_groups(tri, tet, seed=4)
    assert len(groups) == 21
    for cell, mesh in ((0, tri), (1, tet)):
        gs = [g for g in groups if g["cell"] == cell]
        assert sum(g["count"] for g in gs) == mesh.ncells
        assert gs[0]["start"] == 0
        assert all(a["start"] + a["count"] == b["start"] for a, b in zip(gs, gs[1:]))
