"""FP64 CPU oracle for finite-element local assembly (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``oracle.cpp`` (plain C++, FP64,
its own quadrature and Lagrange tabulation) through ctypes. It shares no code with
the CUDA library and the library never imports it.

Every function returns NumPy arrays and follows the paper's local-assembly kernel
structure (section 2 and Listings 1-2): Jacobian, tabulated basis at quadrature
points, then the quadrature loop nest over test and trial functions.
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC = 0, 1, 2, 3
TRIANGLE, TETRAHEDRON, PRISM = 0, 1, 2


def build(force=False):
    """Compile oracle.cpp into liboracle.so (g++, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I, L, D = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_ndof.argtypes = [I, I, I]
        lib.oracle_quadrature.argtypes = [I, I, P, P]
        lib.oracle_nodes.argtypes = [I, I, P]
        lib.oracle_basis.argtypes = [I, I, I, P, P, P]
        lib.oracle_assemble.argtypes = [I, I, I, D, P, P, P, P, L, L, P, I]
        lib.oracle_assemble_cells.argtypes = [I, I, I, D, P, P, P, P, L, P, L, P, I]
        lib.oracle_burgers_residual.argtypes = [I, I, D, P, P, P, P, L, L, P]
        lib.oracle_assemble_backward.argtypes = [I, I, I, D, P, P, P, P, L, L, P, P, P, I]
        lib.oracle_prism_ndof.argtypes = [I]
        lib.oracle_prism_rule.argtypes = [I, P, P]
        lib.oracle_prism_basis.argtypes = [I, I, P, P, P]
        lib.oracle_prism_assemble.argtypes = [I, I, P, P, P, P, L, P, I]
        lib.oracle_prism_burgers_rule.argtypes = [I, P, P]
        lib.oracle_prism_burgers.argtypes = [I, I, ctypes.c_double, P, P, P, P, L, P, I]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def dim(cell):
    return 2 if cell == TRIANGLE else 3


def threads_available():
    return int(_load().oracle_threads_available())


def ndof(form, degree, cell):
    n = _load().oracle_ndof(form, degree, cell)
    if n < 0:
        raise ValueError("unsupported (form, degree, cell)")
    return n


def quadrature(cell, degree):
    """Collapsed Gauss-Legendre rule exact to `degree`: (points [nq,d], weights [nq])."""
    lib = _load()
    nq = lib.oracle_quadrature(cell, degree, None, None)
    pts = np.zeros((nq, dim(cell)))
    wts = np.zeros(nq)
    lib.oracle_quadrature(cell, degree, _p(pts), _p(wts))
    return pts, wts


def nodes(cell, k):
    lib = _load()
    n = lib.oracle_nodes(cell, k, None)
    X = np.zeros((n, dim(cell)))
    lib.oracle_nodes(cell, k, _p(X))
    return X


def basis(cell, k, x):
    """Lagrange basis (Vandermonde inversion) at points x: (phi [np,n], dphi [np,n,d])."""
    x = _f64(np.atleast_2d(x))
    n = nodes(cell, k).shape[0]
    phi = np.zeros((x.shape[0], n))
    dphi = np.zeros((x.shape[0], n, dim(cell)))
    _load().oracle_basis(cell, k, x.shape[0], _p(x), _p(phi), _p(dphi))
    return phi, dphi


def _ncoefnodes(form, coef, cell):
    if coef is None:
        return 0
    d = dim(cell)
    if form == ADVDIFF:
        return coef.size // (1 + d)
    if form == BURGERS_JAC:
        return coef.size // d
    return 0


def assemble(form, degree, cell, coords, c2v, coef=None, c2d=None, nu=0.01, threads=0):
    """Element matrices [ncells, ndof, ndof] float64 for every cell of c2v."""
    coords, c2v, coef, c2d = _f64(coords), _i32(c2v), _f64(coef), _i32(c2d)
    ncells = c2v.shape[0]
    n = ndof(form, degree, cell)
    out = np.zeros((ncells, n, n))
    rc = _load().oracle_assemble(form, degree, cell, nu, _p(coords), _p(c2v), _p(coef), _p(c2d),
                                 _ncoefnodes(form, coef, cell), ncells, _p(out), threads)
    if rc != 0:
        raise ValueError("oracle_assemble failed")
    return out


def assemble_cells(form, degree, cell, coords, c2v, sel, coef=None, c2d=None, nu=0.01, threads=0):
    """Element matrices of the selected cells only: [len(sel), ndof, ndof]."""
    coords, c2v, coef, c2d = _f64(coords), _i32(c2v), _f64(coef), _i32(c2d)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    n = ndof(form, degree, cell)
    out = np.zeros((sel.shape[0], n, n))
    rc = _load().oracle_assemble_cells(form, degree, cell, nu, _p(coords), _p(c2v), _p(coef),
                                       _p(c2d), _ncoefnodes(form, coef, cell), _p(sel),
                                       sel.shape[0], _p(out), threads)
    if rc != 0:
        raise ValueError("oracle_assemble_cells failed")
    return out


def burgers_residual(degree, cell, coords, c2v, u, c2d, nu=0.01):
    """Burgers element residuals [ncells, d*ns] of int (u.grad u).v + nu grad u : grad v."""
    coords, c2v, u, c2d = _f64(coords), _i32(c2v), _f64(u), _i32(c2d)
    ncells = c2v.shape[0]
    n = ndof(BURGERS_JAC, degree, cell)
    out = np.zeros((ncells, n))
    rc = _load().oracle_burgers_residual(degree, cell, nu, _p(coords), _p(c2v), _p(u), _p(c2d),
                                         u.size // dim(cell), ncells, _p(out))
    if rc != 0:
        raise ValueError("oracle_burgers_residual failed")
    return out


def assemble_backward(form, degree, cell, coords, c2v, dout, coef=None, c2d=None, nu=0.01,
                      threads=0):
    """(dL/dcoords [nverts,d], dL/dcoef (coef layout) or None) for the loss gradient dout."""
    coords, c2v, coef, c2d = _f64(coords), _i32(c2v), _f64(coef), _i32(c2d)
    dout = _f64(dout)
    ncells = c2v.shape[0]
    d_coords = np.zeros_like(coords)
    d_coef = np.zeros_like(coef) if coef is not None else None
    rc = _load().oracle_assemble_backward(form, degree, cell, nu, _p(coords), _p(c2v), _p(coef),
                                          _p(c2d), _ncoefnodes(form, coef, cell), ncells,
                                          _p(dout), _p(d_coords), _p(d_coef), threads)
    if rc != 0:
        raise ValueError("oracle_assemble_backward failed")
    return d_coords, d_coef


# ---------------------------------------------------------------- global assembly
# Local assembly yields each cell's contribution to the global system (section 2); the
# framework that runs the kernels over the mesh adds the element matrices into a global
# sparse matrix through the local-to-global dof map (section 4). The oracle states that
# step by its definition, in NumPy and FP64: A[l2g[e,i], l2g[e,j]] += A_e[i,j].

def csr_pattern(l2g, nrows):
    """CSR sparsity (rowptr int64 [nrows+1], colidx int32 [nnz]): (r, c) is stored iff some
    cell has r = l2g[e,i] and c = l2g[e,j]; columns ascend within a row."""
    l2g = np.asarray(l2g, dtype=np.int64)
    n = l2g.shape[1]
    rows = np.repeat(l2g, n, axis=1).ravel()
    cols = np.tile(l2g, (1, n)).ravel()
    key = np.unique(rows * nrows + cols)
    r, c = key // nrows, key % nrows
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(r, minlength=nrows))
    return rowptr, c.astype(np.int32)


def csr_assemble(A_e, l2g, rowptr, colidx):
    """Global matrix values [nnz] (FP64): the sum over cells e and entries (i, j) of A_e[e,i,j]
    at the CSR position of (l2g[e,i], l2g[e,j]), contributions summed in cell order."""
    l2g = np.asarray(l2g, dtype=np.int64)
    n = l2g.shape[1]
    nrows = rowptr.shape[0] - 1
    rows = np.repeat(l2g, n, axis=1).ravel()
    cols = np.tile(l2g, (1, n)).ravel()
    row_of = np.repeat(np.arange(nrows, dtype=np.int64), np.diff(rowptr))
    keys = row_of * nrows + colidx.astype(np.int64)  # ascending, one per stored entry
    pos = np.searchsorted(keys, rows * nrows + cols)
    if np.any(keys[np.minimum(pos, keys.size - 1)] != rows * nrows + cols):
        raise ValueError("an element entry is outside the pattern")
    return np.bincount(pos, weights=np.asarray(A_e, dtype=np.float64).ravel(), minlength=keys.size)


def csr_dense(rowptr, colidx, vals):
    """Dense [nrows, nrows] copy of a CSR matrix (small cases only)."""
    nrows = rowptr.shape[0] - 1
    A = np.zeros((nrows, nrows))
    r = np.repeat(np.arange(nrows), np.diff(rowptr))
    A[r, colidx] = vals
    return A


# ---------------------------------------------------------------- prisms
# The paper's third element shape (section 5.2): triangle x interval, degree-k tensor-product
# Lagrange space, geometry by the degree-1 prism functions (not affine), quadrature fixed as
# n = k+2 Gauss-Legendre points per direction, the triangle factor collapsed by the Duffy map.

def prism_ndof(k):
    return _load().oracle_prism_ndof(k)


def prism_rule(k):
    """(pts [nq, 3], wts [nq]) of the prism quadrature rule."""
    L = _load()
    nq = L.oracle_prism_rule(k, None, None)
    pts, wts = np.zeros((nq, 3)), np.zeros(nq)
    L.oracle_prism_rule(k, _p(pts), _p(wts))
    return pts, wts


def prism_basis(k, x):
    """(phi [npts, n], dphi [npts, n, 3]) of the degree-k prism basis at reference points x [npts, 3]."""
    x = _f64(np.atleast_2d(x))
    n = prism_ndof(k)
    phi, dphi = np.zeros((x.shape[0], n)), np.zeros((x.shape[0], n, 3))
    if _load().oracle_prism_basis(k, x.shape[0], _p(x), _p(phi), _p(dphi)) != 0:
        raise ValueError("oracle_prism_basis failed")
    return phi, dphi


def prism_assemble(form, k, coords, c2v, coef=None, c2d=None, threads=0):
    """Element matrices [ncells, n, n] of MASS, HELMHOLTZ or ADVDIFF on prisms (c2v [ncells, 6];
    ADVDIFF: coef rows (eps, b0, b1, b2) per node, c2d [ncells, 6])."""
    coords, c2v, coef, c2d = _f64(coords), _i32(c2v), _f64(coef), _i32(c2d)
    n = prism_ndof(k)
    out = np.zeros((c2v.shape[0], n, n))
    if _load().oracle_prism_assemble(form, k, _p(coords), _p(c2v), _p(coef), _p(c2d), c2v.shape[0], _p(out),
                                     threads) != 0:
        raise ValueError("oracle_prism_assemble failed")
    return out


def prism_burgers_rule(k):
    """(pts [nq, 3], wts [nq]) of the Burgers prism rule: (3k+3)//2 points per direction."""
    L = _load()
    nq = L.oracle_prism_burgers_rule(k, None, None)
    pts, wts = np.zeros((nq, 3)), np.zeros(nq)
    L.oracle_prism_burgers_rule(k, _p(pts), _p(wts))
    return pts, wts


def prism_burgers(k, coords, c2v, u, c2d, nu=0.01, residual=False, threads=0):
    """Vector Burgers on prisms (section 5.2's third shape): the Jacobians [ncells, 3n, 3n] of
    R[(c,i)] = int (u.grad u_c) phi_i + nu grad u_c . grad phi_i, or with residual=True the
    residual vectors [ncells, 3n]; u [ncoefnodes, 3] nodal values, c2d [ncells, n]."""
    coords, c2v, u, c2d = _f64(coords), _i32(c2v), _f64(u), _i32(c2d)
    N = 3 * prism_ndof(k)
    out = np.zeros((c2v.shape[0], N) if residual else (c2v.shape[0], N, N))
    if _load().oracle_prism_burgers(k, 1 if residual else 0, nu, _p(coords), _p(c2v), _p(u), _p(c2d),
                                    c2v.shape[0], _p(out), threads) != 0:
        raise ValueError("oracle_prism_burgers failed")
    return out
