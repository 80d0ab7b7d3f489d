"""CPU checks of the C-ABI library: it loads, exports every declared symbol, rejects bad
arguments on the host, and its host-side tabulation agrees with the oracle's own."""
import ctypes
import itertools
import os
import re
import subprocess
from math import factorial

import numpy as np
import pytest

import oracle
import paper_1407_0904_gb300 as coffee

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(coffee_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = coffee.lib()
    names = declared_symbols()
    assert {"coffee_tabulate", "coffee_assemble", "coffee_assemble_ex",
            "coffee_assemble_backward", "coffee_check_errors"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", coffee.binding.LIB_PATH],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (coffee_\w+)", out))
    missing = names - exported
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_host_argument_errors_before_any_launch():
    lib = coffee.lib()
    a = coffee.binding.AssembleArgs()
    a.form, a.degree, a.cell, a.precision, a.ncells = 9, 1, 0, 0, 10
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    a.form, a.degree = 1, 7
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    a.degree, a.precision = 2, 11
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    a.precision, a.ncells = 0, -1
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    assert b"ncells" in lib.coffee_last_error()
    a.ncells = 5  # NULL pointers
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    a.ncells = 0  # empty input is a no-op that never touches the GPU
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == 0
    a.form, a.ncells = coffee.ADVDIFF, 3
    a.coords = a.cell2vert = a.out = 16  # non-NULL, never dereferenced on the host
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1  # advdiff without coefficients
    assert lib.coffee_tabulate(5, 1, 2, None, None, None, None, None, None) == -1
    # weighted batch plans reject missing or non-positive tile costs before touching a device
    plan = ctypes.c_void_p()
    P = ctypes.c_void_p
    lib.coffee_batch_plan_costs.argtypes = [ctypes.POINTER(coffee.binding.AssembleArgs), ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(P)]
    one = (coffee.binding.AssembleArgs * 1)(a)
    assert lib.coffee_batch_plan_costs(one, 1, 0, None, ctypes.byref(plan)) == -1
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        assert lib.coffee_batch_plan_costs(one, 1, 0, (ctypes.c_double * 1)(bad), ctypes.byref(plan)) == -1
        assert b"tile_cost" in lib.coffee_last_error()
    assert lib.coffee_ndof(0, 9, 0) == -1


@pytest.mark.parametrize("cell", [0, 1])
def test_ndof(cell):
    for k in range(1, 5):
        ns = (k + 1) * (k + 2) // 2 if cell == 0 else (k + 1) * (k + 2) * (k + 3) // 6
        assert coffee.ndof(coffee.HELMHOLTZ, k, cell) == ns == oracle.ndof(oracle.HELMHOLTZ, k, cell)
        assert coffee.ndof(coffee.BURGERS_JAC, k, cell) == (2 + cell) * ns


@pytest.mark.parametrize("cell", [0, 1])
@pytest.mark.parametrize("p", range(0, 15))
def test_tabulate_rule_exact_on_monomials(cell, p):
    d = 2 + cell
    pts, w, _, _ = coffee.tabulate(cell, 1, p)
    assert np.all(w > 0)
    for e in itertools.product(range(p + 1), repeat=d):
        if sum(e) > p:
            continue
        val = np.sum(w * np.prod(pts ** np.array(e), axis=1))
        ex = np.prod([factorial(x) for x in e]) / factorial(sum(e) + d)
        assert abs(val - ex) <= 2e-14 * ex


@pytest.mark.parametrize("cell", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_tabulate_basis_matches_oracle(cell, k):
    pts, w, phi, grd = coffee.tabulate(cell, k, 2 * k)
    ophi, ogrd = oracle.basis(cell, k, pts)
    assert np.abs(phi - ophi).max() < 1e-13
    assert np.abs(grd - ogrd).max() < 1e-12


@pytest.mark.parametrize("form", [coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF])
@pytest.mark.parametrize("cell", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_reference_tensor_on_reference_cell_matches_oracle(form, cell, k):
    """On the reference cell J = I, |det| = 1, so G is known without geometry code:
    MASS G=[1]; HELMHOLTZ G=[1, delta_ab]; ADVDIFF G=[eps_v delta_ab | b_v,a]."""
    d = 2 + cell
    T = coffee.reference_tensor(form, k, cell)
    ns = oracle.ndof(form, k, cell)
    X = np.vstack([np.zeros(d), np.eye(d)])
    c2v = np.arange(d + 1, dtype=np.int32)[None]
    pairs = [(a, b) for a in range(d) for b in range(a, d)]
    coef = c2d = None
    if form == coffee.MASS:
        G = np.array([1.0])
    elif form == coffee.HELMHOLTZ:
        G = np.array([1.0] + [1.0 if a == b else 0.0 for a, b in pairs])
    else:
        rng = np.random.default_rng(k)
        eps = rng.uniform(0.5, 1.5, d + 1)
        b = rng.uniform(-1, 1, (d + 1, d))
        coef = np.concatenate([eps[:, None], b], axis=1).ravel()
        c2d = c2v.copy()
        G = np.concatenate([[eps[v] * (1.0 if a == bb else 0.0) for v in range(d + 1) for a, bb in pairs],
                            b.ravel()])
    A = (G @ T).reshape(ns, ns)
    R = oracle.assemble(form, k, cell, X, c2v, coef, c2d)[0]
    assert np.abs(A - R).max() < 1e-13 * np.abs(R).max()


@pytest.mark.parametrize("cell,k", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_burgers_reference_tensor_on_reference_cell_matches_oracle(cell, k):
    """Reference cell, u given: block (ci,cj) = sum_{r,a} u[r,ci] delta_{a,cj} T1 +
    [ci==cj] (sum_{r,a} u[r,a] T2 + nu sum_p delta_p T3)."""
    d = 2 + cell
    T = coffee.reference_tensor(coffee.BURGERS_JAC, k, cell)
    ns = oracle.ndof(oracle.MASS, k, cell)
    X = np.vstack([np.zeros(d), np.eye(d)])
    c2v = np.arange(d + 1, dtype=np.int32)[None]
    u = np.random.default_rng(3).standard_normal((ns, d))
    c2d = np.arange(ns, dtype=np.int32)[None]
    T1, T2, T3 = T[:ns * d], T[ns * d:2 * ns * d], T[2 * ns * d:]
    pairs = [(a, b) for a in range(d) for b in range(a, d)]
    A = np.zeros((d * ns, d * ns))
    for ci in range(d):
        for cj in range(d):
            G1 = np.array([u[r, ci] * (1.0 if a == cj else 0.0) for r in range(ns) for a in range(d)])
            blk = G1 @ T1
            if ci == cj:
                blk = blk + u.ravel() @ T2 + 0.01 * np.array([1.0 if a == b else 0.0 for a, b in pairs]) @ T3
            A[ci * ns:(ci + 1) * ns, cj * ns:(cj + 1) * ns] = blk.reshape(ns, ns)
    R = oracle.assemble(oracle.BURGERS_JAC, k, cell, X, c2v, u, c2d)[0]
    assert np.abs(A - R).max() < 1e-13 * np.abs(R).max()


def test_support_queries_cover_prisms():
    """Host-only queries: prisms take MASS, HELMHOLTZ and ADVDIFF (FP64 and tensor cores P1-P4),
    locally and fused into CSR; the Burgers Jacobian (locally and into CSR) and residual in FP64."""
    P = coffee.PRISM
    for form in (coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF):
        for k in range(1, 5):
            assert coffee.supported(form, k, P, coffee.FP64)
            assert coffee.csr_supported(form, k, P, coffee.FP64)
            for prec in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16):
                assert coffee.supported(form, k, P, prec)
                assert coffee.csr_supported(form, k, P, prec)
    for form in (coffee.BURGERS_JAC, coffee.BURGERS_RESIDUAL):
        for k in range(1, 5):
            assert coffee.supported(form, k, P, coffee.FP64)
            assert bool(coffee.csr_supported(form, k, P, coffee.FP64)) == (form == coffee.BURGERS_JAC)
            for prec in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16):
                assert not coffee.supported(form, k, P, prec)
                assert not coffee.csr_supported(form, k, P, prec)


def test_assemble_path_query():
    """Host-only: which kernel family runs. Small element matrices (MASS, HELMHOLTZ, ADVDIFF on
    P1 simplices and P2 triangles, the Burgers Jacobian and residual on P1 simplices) default to the FP32
    CUDA-core kernel, the rest of the tensor-core precisions to the tensor cores; the flags force
    either where both exist; FP64 is the FP64 kernel; unsupported combinations raise."""
    T, R, P = coffee.TETRAHEDRON, coffee.TRIANGLE, coffee.PRISM
    for form in (coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF):
        for cell, k, default in ((T, 1, 2), (R, 1, 2), (R, 2, 2), (T, 2, 1), (R, 3, 1), (T, 3, 1), (R, 4, 1)):
            for prec in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16):
                assert coffee.assemble_path(form, k, cell, prec) == default
                assert coffee.assemble_path(form, k, cell, prec, coffee.FLAG_TENSOR_CORES) == 1
                forced = 2 if (cell == T and k <= 2) or (cell == R and k <= 3) else 1
                assert coffee.assemble_path(form, k, cell, prec, coffee.FLAG_CUDA_CORES) == forced
            assert coffee.assemble_path(form, k, cell, coffee.FP64) == 0
        assert coffee.assemble_path(form, 2, P, coffee.TF32X3, coffee.FLAG_CUDA_CORES) == 1
    # the Burgers forms: P1 and triangles P2 on the CUDA cores, the rest on the tensor cores
    for form in (coffee.BURGERS_JAC, coffee.BURGERS_RESIDUAL):
        for cell, k in ((T, 1), (R, 1), (R, 2)):
            assert coffee.assemble_path(form, k, cell, coffee.TF32X3) == 2
            assert coffee.assemble_path(form, k, cell, coffee.TF32X3, coffee.FLAG_TENSOR_CORES) == 1
        assert coffee.assemble_path(form, 2, T, coffee.TF32X3, coffee.FLAG_CUDA_CORES) == 1
        assert coffee.assemble_path(form, 3, R, coffee.TF32X3) == 1
    with pytest.raises(coffee.CoffeeError):
        coffee.assemble_path(coffee.BURGERS_JAC, 1, P, coffee.TF32X3)


def test_reference_tensor_queries_for_residual_and_prisms():
    """Host-only: the residual contracts the Jacobian's reference tensors; prisms, whose
    Jacobian varies over the cell, have none and are rejected."""
    for cell, k in ((0, 2), (1, 1), (1, 2)):
        R = coffee.reference_tensor(coffee.BURGERS_RESIDUAL, k, cell)
        J = coffee.reference_tensor(coffee.BURGERS_JAC, k, cell)
        assert R.shape == J.shape and R.shape[0] > 0
        assert np.array_equal(R, J)
    with pytest.raises(coffee.CoffeeError):
        coffee.reference_tensor(coffee.HELMHOLTZ, 2, coffee.PRISM)


def test_binding_checks_input_extents_before_any_pointer_is_passed():
    """The C ABI sees bare pointers; the binding checks the extents it can see (CPU tensors
    suffice: check_shapes looks at shapes only)."""
    import torch
    from paper_1407_0904_gb300 import meshgen
    from paper_1407_0904_gb300.binding import check_shapes
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    for cell, mesh in ((0, meshgen.tri_mesh(4, seed=1)), (1, meshgen.tet_mesh(3, seed=1)),
                       (2, meshgen.prism_mesh(3, 2, seed=1))):
        x, c2v = t(mesh.coords), t(mesh.cell2vert)
        coef, c2d, _ = meshgen.advdiff_coefficients(mesh, 3)
        check_shapes(coffee.ADVDIFF, 2, cell, x, c2v, t(coef), t(c2d))
        with pytest.raises(ValueError):  # fewer cell2dof rows than cells
            check_shapes(coffee.ADVDIFF, 2, cell, x, c2v, t(coef), t(c2d[:-1]))
        with pytest.raises(ValueError):  # a column short
            check_shapes(coffee.ADVDIFF, 2, cell, x, c2v, t(coef), t(c2d[:, :-1]))
        with pytest.raises(ValueError):  # coef rows are (eps, b_0 .. b_{d-1})
            check_shapes(coffee.ADVDIFF, 2, cell, x, c2v, t(coef.ravel()[:-1]), t(c2d))
        with pytest.raises(ValueError):
            check_shapes(coffee.HELMHOLTZ, 2, cell, x[:, :1], c2v)
        with pytest.raises(ValueError):
            check_shapes(coffee.HELMHOLTZ, 2, cell, x, c2v[:, :-1])
        if cell == 2:
            continue
        for k in (1, 2, 3):
            u, c2d, _ = meshgen.burgers_coefficients(mesh, k, 3)
            for form in (coffee.BURGERS_JAC, coffee.BURGERS_RESIDUAL):
                check_shapes(form, k, cell, x, c2v, t(u.ravel()), t(c2d))
                with pytest.raises(ValueError):  # the map of another degree
                    check_shapes(form, k + 1, cell, x, c2v, t(u.ravel()), t(c2d))


def test_host_buffer_entry_point_rejects_bad_arguments_before_any_cuda_call():
    """coffee_assemble_host: argument checks come before the first CUDA call (no device here)."""
    lib = coffee.lib()
    A = coffee.binding.AssembleArgs
    lib.coffee_assemble_host.argtypes = [ctypes.POINTER(A), ctypes.c_int, ctypes.c_void_p]
    assert lib.coffee_assemble_host(None, 4, None) == -1
    a = A()
    a.form, a.degree, a.cell, a.precision, a.ncells = coffee.HELMHOLTZ, 3, coffee.TETRAHEDRON, coffee.TF32X3, 0
    assert lib.coffee_assemble_host(ctypes.byref(a), 0, None) == -1
    assert b"chunks" in lib.coffee_last_error()
    assert lib.coffee_assemble_host(ctypes.byref(a), 4, None) == 0  # empty: nothing to copy
    a.ncells = 10
    assert lib.coffee_assemble_host(ctypes.byref(a), 4, None) == -1  # NULL host pointers
    a.coords = a.cell2vert = a.out = 16  # non-NULL, never dereferenced before the size checks
    assert lib.coffee_assemble_host(ctypes.byref(a), 4, None) == -1
    assert b"nverts" in lib.coffee_last_error()
    a.form, a.nverts = coffee.ADVDIFF, 20
    assert lib.coffee_assemble_host(ctypes.byref(a), 4, None) == -1
    assert b"coef" in lib.coffee_last_error()
    a.form, a.degree, a.cell = coffee.BURGERS_JAC, 4, coffee.TETRAHEDRON
    a.coef = a.cell2dof = 16
    a.ncoefnodes = 20
    a.precision = coffee.BF16X3  # the Burgers Jacobian on tet P4 has no BF16X3 kernel
    assert lib.coffee_assemble_host(ctypes.byref(a), 4, None) == -2


def test_size_limits_are_rejected_on_the_host():
    """The largest inputs the kernels index: more than 2^31 * 128 cells, nnz of 2^32 or more and an
    unaligned entry map are refused before any CUDA call."""
    lib = coffee.lib()
    A = coffee.binding.AssembleArgs
    a = A()
    a.form, a.degree, a.cell, a.precision = coffee.HELMHOLTZ, 2, coffee.TETRAHEDRON, coffee.TF32X3
    a.coords = a.cell2vert = a.out = 16
    a.nverts = 10
    a.ncells = (2 ** 31 - 1) * 128 + 1
    assert lib.coffee_assemble_ex(ctypes.byref(a), None) == -1
    assert b"ncells" in lib.coffee_last_error()
    lib.coffee_assemble_csr.argtypes = [ctypes.POINTER(A), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p]
    a.ncells = 10
    assert lib.coffee_assemble_csr(ctypes.byref(a), 256, 256, 2 ** 32, None) == -1
    assert b"nnz" in lib.coffee_last_error()
    assert lib.coffee_assemble_csr(ctypes.byref(a), 260, 256, 100, None) == -1
    assert b"aligned" in lib.coffee_last_error()
    lib.coffee_sparsity.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    nnz = ctypes.c_int64()
    assert lib.coffee_sparsity(16, 2 ** 31, 4, 10, 16, None, ctypes.byref(nnz), None) == -1
    assert lib.coffee_sparsity(16, 10, 129, 10, 16, None, ctypes.byref(nnz), None) == -1
