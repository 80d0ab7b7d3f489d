"""Seeded synthetic inputs: perturbed structured simplex meshes and coefficient fields.

These generators stand in for the "real unstructured meshes" the paper runs its
benchmarks on (section 5.2), which are not available. They hold no part of the
assembly arithmetic: only mesh topology, vertex positions, degree-k node numbering
and random coefficient values. Both the CUDA path and the FP64 oracle consume
exactly the arrays produced here.

Conventions:
  * vertices of an n^d grid are numbered lexicographically, x fastest; h = 1/n;
  * triangles: each square (i,j) is cut along (i,j)-(i+1,j+1) into
    [v00, v10, v11] and [v00, v11, v01];
  * tetrahedra: each cube is cut into the 6 Kuhn tetrahedra, one per permutation
    of the axes, [v0, v0+e_s0, v0+e_s0+e_s1, v0+(1,1,1)] (half are negatively
    oriented, which the |det J| measure accepts);
  * interior vertices move by U[-p*h, p*h] independently per coordinate; boundary
    vertices stay fixed, so the mesh still tiles the unit square/cube exactly;
  * a degree-k node of a cell with grid vertices V0..Vd and lattice index (a,b,c)
    is the integer point k*V0 + a(V1-V0) + b(V2-V0) + c(V3-V0) of the (k*n+1)^d
    lattice, which makes the numbering conforming across cells;
  * prisms: the triangle mesh of the unit square extruded through nz layers of the unit
    cube; a prism's vertices are its bottom triangle, then the three vertices above it;
    its degree-k node (a,b) at level c is the integer point k*V0 + a(V1-V0) + b(V2-V0)
    + c*(V3-V0) (with V3 above V0), zeta level slowest.
"""
import itertools
import numpy as np

TRIANGLE, TETRAHEDRON, PRISM = 0, 1, 2

_PERMS3 = list(itertools.permutations(range(3)))


class Mesh:
    """A simplex mesh: coords [nverts,d] float64, cell2vert [ncells,d+1] int32,
    grid [ncells,d+1,d] int64 (unperturbed integer vertex positions), n (grid size per axis)."""

    def __init__(self, cell, coords, cell2vert, grid, shape):
        self.cell = cell
        self.coords = coords
        self.cell2vert = cell2vert
        self.grid = grid
        self.shape = shape  # cells per axis

    @property
    def dim(self):
        return 2 if self.cell == TRIANGLE else 3

    @property
    def nvc(self):
        """vertices per cell"""
        return {TRIANGLE: 3, TETRAHEDRON: 4, PRISM: 6}[self.cell]

    @property
    def ncells(self):
        return self.cell2vert.shape[0]

    @property
    def nverts(self):
        return self.coords.shape[0]


def _perturb(pts_int, shape, perturb, rng):
    """Grid points scaled to the unit box; interior ones moved by U[-p h, p h]."""
    shape = np.asarray(shape)
    h = 1.0 / shape
    x = pts_int * h
    interior = np.all((pts_int > 0) & (pts_int < shape), axis=1)
    noise = rng.uniform(-perturb, perturb, size=x.shape) * h
    x[interior] += noise[interior]
    return x


def tri_mesh(n, perturb=0.2, seed=1):
    """Unit square, n x n squares, 2 triangles each (2 n^2 cells)."""
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    pts = np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.int64)
    coords = _perturb(pts.astype(np.float64), (n, n), perturb, rng)
    vid = lambda i, j: j * (n + 1) + i
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00, v10, v11, v01 = vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)
    c2v = np.empty((n * n, 2, 3), dtype=np.int64)
    c2v[:, 0] = np.stack([v00, v10, v11], axis=1)
    c2v[:, 1] = np.stack([v00, v11, v01], axis=1)
    c2v = c2v.reshape(-1, 3)
    grid = pts[c2v]
    return Mesh(TRIANGLE, np.ascontiguousarray(coords), c2v.astype(np.int32), grid, (n, n))


def tet_mesh(nx, ny=None, nz=None, perturb=0.15, seed=2, ncells=None):
    """Unit cube, nx*ny*nz cubes, 6 Kuhn tets each; optionally keep the first ncells."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    pts = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int64)
    coords = _perturb(pts.astype(np.float64), (nx, ny, nz), perturb, rng)
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)  # cube origins, x fastest
    eye = np.eye(3, dtype=np.int64)
    corners = np.empty((base.shape[0], 6, 4, 3), dtype=np.int64)
    for p, s in enumerate(_PERMS3):
        corners[:, p, 0] = base
        corners[:, p, 1] = base + eye[s[0]]
        corners[:, p, 2] = base + eye[s[0]] + eye[s[1]]
        corners[:, p, 3] = base + 1
    grid = corners.reshape(-1, 4, 3)
    if ncells is not None:
        grid = grid[:ncells]
    c2v = grid[..., 0] + (nx + 1) * (grid[..., 1] + (ny + 1) * grid[..., 2])
    return Mesh(TETRAHEDRON, np.ascontiguousarray(coords), c2v.astype(np.int32), grid, (nx, ny, nz))


def prism_mesh(n, nz=None, perturb=0.15, seed=6):
    """Unit cube: the n x n two-triangle mesh of the square extruded through nz layers
    (2 n^2 nz prisms); interior vertices perturbed, so the quadrilateral faces are not
    planar and the prisms are not affine."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    pts = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int64)
    coords = _perturb(pts.astype(np.float64), (n, n, nz), perturb, rng)
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    b00 = np.stack([ci, cj, ck], axis=1)
    ex, ey, ez = np.array([1, 0, 0]), np.array([0, 1, 0]), np.array([0, 0, 1])
    corners = np.empty((b00.shape[0], 2, 6, 3), dtype=np.int64)
    for half, tri in enumerate(((0 * ex, ex, ex + ey), (0 * ex, ex + ey, ey))):
        for v in range(3):
            corners[:, half, v] = b00 + tri[v]
            corners[:, half, v + 3] = b00 + tri[v] + ez
    grid = corners.reshape(-1, 6, 3)
    c2v = grid[..., 0] + (n + 1) * (grid[..., 1] + (n + 1) * grid[..., 2])
    return Mesh(PRISM, np.ascontiguousarray(coords), c2v.astype(np.int32), grid, (n, n, nz))


def lattice(cell, k):
    """Lattice multi-indices (a,b[,c]), a+b+c <= k, c slowest then b then a."""
    out = []
    cmax = k if cell == TETRAHEDRON else 0
    for c in range(cmax + 1):
        for b in range(k - c + 1):
            for a in range(k - b - c + 1):
                out.append((a, b, c) if cell == TETRAHEDRON else (a, b))
    return np.array(out, dtype=np.int64)


def cell2dof(mesh, k, permute_seed=None):
    """Conforming degree-k node numbering: (cell2dof [ncells, ns] int32, nnodes).

    With permute_seed the global node ids are shuffled by a seeded permutation
    (a gather-locality stress case)."""
    g = mesh.grid  # [ncells, nvc, d]
    V0 = g[:, 0]
    if mesh.cell == PRISM:
        T = lattice(TRIANGLE, k)
        L = np.array([(a, b, c) for c in range(k + 1) for (a, b) in T], dtype=np.int64)
        E = np.stack([g[:, 1] - V0, g[:, 2] - V0, g[:, 3] - V0], axis=1)  # V3 is above V0
    else:
        L = lattice(mesh.cell, k)  # [ns, d]
        E = g[:, 1:] - V0[:, None, :]  # [ncells, d, d] rows = V_{a+1}-V0
    pts = k * V0[:, None, :] + np.einsum("na,cad->cnd", L, E)  # [ncells, ns, d]
    dims = [k * s + 1 for s in mesh.shape]
    ids = np.zeros(pts.shape[:2], dtype=np.int64)
    mult = 1
    for a in range(mesh.dim):
        ids += pts[..., a] * mult
        mult *= dims[a]
    nnodes = mult
    if permute_seed is not None:
        perm = np.random.default_rng(permute_seed).permutation(nnodes)
        ids = perm[ids]
    return ids.astype(np.int32), int(nnodes)


def advdiff_coefficients(mesh, seed, permute_seed=None):
    """eps ~ U[0.5,1.5] and b ~ U[-1,1]^d per P1 node: (coef [nnodes*(1+d)] with rows
    (eps, b_0, .., b_{d-1}), cell2dof, nnodes)."""
    c2d, nn = cell2dof(mesh, 1, permute_seed)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.5, 1.5, size=nn)
    b = rng.uniform(-1.0, 1.0, size=(nn, mesh.dim))
    return np.concatenate([eps[:, None], b], axis=1).ravel(), c2d, nn


def burgers_coefficients(mesh, k, seed, permute_seed=None):
    """u ~ N(0,1) per component of every degree-k node: (u [nnodes,d], cell2dof, nnodes)."""
    c2d, nn = cell2dof(mesh, k, permute_seed)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(size=(nn, mesh.dim))
    return u, c2d, nn


def zipf_counts(ngroups, total, s=1.0, seed=4):
    """Seeded Zipf split of `total` cells over `ngroups` groups: counts[group]."""
    rng = np.random.default_rng(seed)
    ranks = rng.permutation(ngroups) + 1  # group -> rank
    H = np.sum(1.0 / np.arange(1, ngroups + 1) ** s)
    counts = np.floor(total * ranks.astype(np.float64) ** (-s) / H).astype(np.int64)
    counts[np.argmin(ranks)] += total - counts.sum()
    return counts


def sliver_tet(rng=None, flat=1e-3):
    """A near-degenerate tetrahedron (height `flat` relative to its base)."""
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.3, 0.3, flat]])
    if rng is not None:
        X = X + rng.uniform(-1e-3, 1e-3, size=X.shape) * flat
    return X


BATCH_FORMS = (0, 1, 2)  # mass, Helmholtz, advection-diffusion


def batch_groups(tri_mesh_, tet_mesh_, tri_degrees=(1, 2, 3, 4), tet_degrees=(1, 2, 3), seed=4):
    """Mixed-batch groups: every (form, degree) on both meshes, each group a contiguous
    range of cells whose size follows a seeded Zipf(s=1) split of the mesh's cells.

    Returns a list of dicts {form, degree, cell, start, count}."""
    out = []
    for mesh, degrees, sd in ((tri_mesh_, tri_degrees, seed), (tet_mesh_, tet_degrees, seed + 1)):
        kinds = [(f, k) for k in degrees for f in BATCH_FORMS]
        counts = zipf_counts(len(kinds), mesh.ncells, s=1.0, seed=sd)
        start = 0
        for (f, k), n in zip(kinds, counts):
            out.append({"form": f, "degree": k, "cell": mesh.cell, "start": int(start), "count": int(n)})
            start += n
    return out
