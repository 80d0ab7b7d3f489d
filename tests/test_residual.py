"""Parity of the Burgers residual (element vectors, form BURGERS_RESIDUAL) with the oracle.

The residual R(u) = int (u.grad u).v + nu grad u : grad v is quadratic in u; the oracle
evaluates it by quadrature (pinned in test_oracle_pins against exact rational integrals).
Error metrics, both bounded by the element-matrix tolerances (tests.helpers.TOL):
  per cell: max_i |R_e - R_oracle,e| / max_i (|J_e| |u_e|)_i, where J_e is the oracle's Burgers
    Jacobian of the cell and u_e its component-blocked dofs. R = (J_c / 2 + J_nu) u is a sum of
    products that cancel (with u ~ N(0,1) single entries, even whole cells, of R can be nearly
    zero), so the un-cancelled magnitude |J_e| |u_e| of the same products is the cell's scale;
    a cell whose error is large against its own terms fails, wherever |R| itself is small.
  global: max |R - R_oracle| over all entries divided by max |R_oracle| over the mesh.
The plain per-cell ratio max_i |dR| / max_i |R_oracle| is printed (maximum and median) and, for
FP64 and the split precisions, bounded as well.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, BURGERS_JAC, TOL, to_device

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RES = coffee.BURGERS_RESIDUAL


def ragged_mesh(cell, seed):
    if cell == TRI:
        return meshgen.tri_mesh(23, perturb=0.2, seed=seed)        # 1058 cells = 8 tiles + 34
    return meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=1000)  # 7 tiles + 104


def errors(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape)
    glob = float(np.abs(got - ref).max() / np.abs(ref).max())
    per = np.abs(got - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)
    return glob, float(np.median(per)), float(per.max())


def cell_errors(got, ref, k, cell, coords, c2v, u, c2d):
    """Per cell: max_i |dR_i| / max_i (|J| |u|)_i with the oracle's Jacobian J of the cell."""
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape)
    J = oracle.assemble(BURGERS_JAC, k, cell, coords, c2v, u.ravel(), c2d, threads=0)
    ub = np.transpose(u[c2d], (0, 2, 1)).reshape(len(c2v), -1)  # component-blocked
    scale = np.einsum("eij,ej->ei", np.abs(J), np.abs(ub)).max(axis=1)
    return float((np.abs(got - ref).max(axis=1) / np.maximum(scale, 1e-300)).max())


CASES = [(c, k, p) for c in (TRI, TET) for k in (1, 2, 3, 4)
         for p in (coffee.FP64, coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16)]


@pytest.mark.parametrize("cell,k,prec", CASES)
def test_residual_matches_oracle(cell, k, prec):
    if not coffee.supported(RES, k, cell, prec):
        pytest.skip("no kernel for this combination")
    mesh = ragged_mesh(cell, seed=60 + k)
    u, c2d, _ = meshgen.burgers_coefficients(mesh, k, seed=8)
    ref = oracle.burgers_residual(k, cell, mesh.coords, mesh.cell2vert, u, c2d)
    x, c2v, cf, cd = to_device(mesh, u.ravel(), c2d, DEV)
    out = coffee.assemble(RES, k, cell, x, c2v, cf, cd, precision=prec, validate=True)
    coffee.check_errors()
    n = coffee.ndof(RES, k, cell)
    assert tuple(out.shape) == (mesh.ncells, n)
    got = out.cpu().numpy()
    glob, med, worst = errors(got, ref)
    per = cell_errors(got, ref, k, cell, mesh.coords, mesh.cell2vert, u, c2d)
    print("residual %s P%d %s: per cell %.3e, global %.3e (max_i|dR|/max_i|R| per cell: median %.3e, max %.3e)"
          % ("tri" if cell == TRI else "tet", k, coffee.PRECISION_NAMES[prec], per, glob, med, worst))
    assert per < TOL[prec] and glob < TOL[prec]
    if prec in (coffee.FP64, coffee.TF32X3, coffee.BF16X3):
        assert worst < TOL[prec]  # the split precisions meet the bound against max|R| of each cell too


@pytest.mark.parametrize("cell", [TRI, TET])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3])
def test_residual_p1_both_kernel_families(cell, prec):
    """P1 runs on the CUDA cores by default; the tensor-core kernel, forced, meets the same bounds
    (per cell against the un-cancelled magnitude and globally)."""
    mesh = ragged_mesh(cell, seed=64)
    u, c2d, _ = meshgen.burgers_coefficients(mesh, 1, seed=9)
    ref = oracle.burgers_residual(1, cell, mesh.coords, mesh.cell2vert, u, c2d)
    x, c2v, cf, cd = to_device(mesh, u.ravel(), c2d, DEV)
    assert coffee.assemble_path(RES, 1, cell, prec) == 2
    for tune in (0, coffee.FLAG_TENSOR_CORES):
        out = coffee.assemble(RES, 1, cell, x, c2v, cf, cd, precision=prec, validate=True, tune=tune)
        coffee.check_errors()
        got = out.cpu().numpy()
        glob, _, worst = errors(got, ref)
        per = cell_errors(got, ref, 1, cell, mesh.coords, mesh.cell2vert, u, c2d)
        assert per < TOL[prec] and glob < TOL[prec] and worst < TOL[prec]


def test_residual_is_the_jacobian_applied_to_u_minus_the_convective_half():
    """R(u) = J_c(u) u / 2 + J_nu u for the quadratic residual, where J_c is the convective part of
    the Jacobian: so J(u) u - R(u) = N(u, u) (the convective term once more); checked on the GPU
    with the FP64 kernels of both forms against the oracle's residual."""
    mesh = ragged_mesh(TET, seed=5)
    k = 2
    u, c2d, _ = meshgen.burgers_coefficients(mesh, k, seed=9)
    x, c2v, cf, cd = to_device(mesh, u.ravel(), c2d, DEV)
    J = coffee.assemble(coffee.BURGERS_JAC, k, TET, x, c2v, cf, cd, precision=coffee.FP64).cpu().numpy()
    R = coffee.assemble(RES, k, TET, x, c2v, cf, cd, precision=coffee.FP64).cpu().numpy()
    ue = u[c2d]  # [ncells, ns, d]
    ub = np.transpose(ue, (0, 2, 1)).reshape(mesh.ncells, -1)  # component-blocked
    Ju = np.einsum("eij,ej->ei", J, ub)
    # viscous part is linear: (J u - R) is the convective residual; 2 R - J u is the viscous one
    nu0 = oracle.burgers_residual(k, TET, mesh.coords, mesh.cell2vert, u, c2d, nu=0.0)
    np.testing.assert_allclose(Ju - R, nu0, rtol=0, atol=1e-11 * np.abs(nu0).max())


def test_residual_errors_and_empty():
    mesh = ragged_mesh(TRI, seed=3)
    u, c2d, _ = meshgen.burgers_coefficients(mesh, 2, seed=8)
    x, c2v, cf, cd = to_device(mesh, u.ravel(), c2d, DEV)
    out = coffee.assemble(RES, 2, TRI, x, c2v[:0].contiguous(), cf, cd[:0].contiguous(), precision=coffee.TF32X3)
    assert out.shape[0] == 0
    with pytest.raises(coffee.CoffeeError):  # a residual is not a matrix
        M = coffee.CsrMatrix(coffee.vector_l2g(cd, u.shape[0], 2), 2 * u.shape[0])
        M.assemble(RES, 2, TRI, x, c2v, cf, cd, precision=coffee.FP64)
    with pytest.raises(coffee.CoffeeError):  # no adjoint for the Burgers forms
        coffee.assemble_backward(RES, 2, TRI, x, c2v, torch.zeros((mesh.ncells, 12), dtype=torch.float64,
                                                                  device=DEV), cf, cd)


def test_config3_residual_2pow20_sampled():
    """2^20 Kuhn tets (64x64x43 truncated), P2, u ~ N(0,1): 2048 sampled cells vs the oracle."""
    mesh = meshgen.tet_mesh(64, 64, 43, perturb=0.15, seed=3, ncells=2 ** 20)
    u, c2d, _ = meshgen.burgers_coefficients(mesh, 2, seed=3)
    x, c2v, cf, cd = to_device(mesh, u.ravel(), c2d, DEV)
    out = coffee.assemble(RES, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3)
    coffee.check_errors()
    sel = np.sort(np.random.default_rng(3).choice(mesh.ncells, 2048, replace=False))
    ref = oracle.burgers_residual(2, TET, mesh.coords, mesh.cell2vert[sel], u, c2d[sel])
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy()
    glob, _, _ = errors(got, ref)
    per = cell_errors(got, ref, 2, TET, mesh.coords, mesh.cell2vert[sel], u, c2d[sel])
    assert per < TOL[coffee.TF32X3] and glob < TOL[coffee.TF32X3]
