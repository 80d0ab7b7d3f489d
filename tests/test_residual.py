"""Parity of the Burgers residual (element vectors, form BURGERS_RESIDUAL) with the oracle.

The residual R(u) = int (u.grad u).v + nu grad u : grad v is quadratic in u; the oracle
evaluates it by quadrature (pinned in test_oracle_pins against exact rational integrals).
Error metric: max |R - R_oracle| over all entries divided by max |R_oracle| over the mesh
(entries of single cells can cancel to nearly zero, so a per-cell ratio is reported, not
bounded). Tolerances follow the element-matrix tests: the tensor-core path forms
C[i][s] (one contraction against the Jacobian's T2|T3 tensors, error eps_prec relative to
sum_k |G_k T_k|) and then R = C u in FP32 with ns-term sums: FP64 1e-12, TF32X3 1e-5,
BF16X3 1e-4, TF32 1e-2, BF16 2e-2.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, to_device

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RES = coffee.BURGERS_RESIDUAL
TOL = {coffee.FP64: 1e-12, coffee.TF32X3: 1e-5, coffee.BF16X3: 1e-4, coffee.TF32: 1e-2, coffee.BF16: 2e-2}


def ragged_mesh(cell, seed):
    if cell == TRI:
        return meshgen.tri_mesh(23, perturb=0.2, seed=seed)        # 1058 cells = 8 tiles + 34
    return meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=1000)  # 7 tiles + 104


def errors(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape)
    glob = float(np.abs(got - ref).max() / np.abs(ref).max())
    per = np.abs(got - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)
    return glob, float(np.median(per))


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
    glob, med = errors(out.cpu().numpy(), ref)
    print("residual %s P%d %s: %.3e (median per cell %.3e)" % ("tri" if cell == TRI else "tet", k,
                                                                coffee.PRECISION_NAMES[prec], glob, med))
    assert glob < TOL[prec]


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
    glob, _ = errors(got, ref)
    assert glob < TOL[coffee.TF32X3]
