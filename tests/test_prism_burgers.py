"""Parity of the FP64 vector Burgers kernel on prisms with the oracle (section 5.2 runs Burgers on
the third element shape too).

Both sides evaluate the same fixed rule ((3k+3)//2 Gauss-Legendre points per direction, the
triangle factor Duffy-collapsed), each from its own implementation, on twisted (non-affine)
prisms with u drawn per node through a shuffled cell-to-node map: Jacobians and residuals agree
to rounding, held to 1e-12 of each cell's largest entry like the other FP64 kernels.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import rel_err_per_cell

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PRISM = coffee.PRISM
SIZES = {1: (6, 4), 2: (5, 3), 3: (3, 3), 4: (3, 1)}  # prism_mesh(n, nz): 2 n^2 nz cells


def problem(k, seed):
    n_, nz = SIZES[k]
    mesh = meshgen.prism_mesh(n_, nz, perturb=0.15, seed=seed)
    n = coffee.nnodes(PRISM, k)
    rng = np.random.default_rng(seed)
    nnodes = mesh.ncells * n + 5  # a few coefficient nodes no cell uses
    c2d = rng.permutation(nnodes)[:mesh.ncells * n].reshape(mesh.ncells, n).astype(np.int32)
    u = rng.standard_normal((nnodes, 3))
    return mesh, u, c2d


def on_device(mesh, u, c2d):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t(mesh.coords), t(mesh.cell2vert), t(u), t(c2d)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("residual", [False, True])
def test_prism_burgers_fp64_matches_oracle(k, residual):
    mesh, u, c2d = problem(k, 30 + k)
    form = coffee.BURGERS_RESIDUAL if residual else coffee.BURGERS_JAC
    ref = oracle.prism_burgers(k, mesh.coords, mesh.cell2vert, u, c2d, nu=0.05, residual=residual)
    x, c2v, ud, cd = on_device(mesh, u, c2d)
    out = coffee.assemble(form, k, PRISM, x, c2v, ud, cd, precision=coffee.FP64, nu=0.05, validate=True)
    coffee.check_errors()
    assert out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism Burgers %s P%d: %.3e" % ("residual" if residual else "Jacobian", k, err))
    assert err < 1e-12


def test_prism_burgers_checks_and_edges():
    mesh, u, c2d = problem(1, 40)
    x, c2v, ud, cd = on_device(mesh, u, c2d)
    assert coffee.supported(coffee.BURGERS_JAC, 2, PRISM, coffee.FP64)
    assert not coffee.supported(coffee.BURGERS_JAC, 2, PRISM, coffee.TF32X3)
    with pytest.raises(coffee.CoffeeError):  # no tensor-core kernel for Burgers on prisms
        coffee.assemble(coffee.BURGERS_JAC, 1, PRISM, x, c2v, ud, cd, precision=coffee.TF32X3)
    with pytest.raises(coffee.CoffeeError):  # u is required
        coffee.assemble(coffee.BURGERS_JAC, 1, PRISM, x, c2v, precision=coffee.FP64)
    bad = cd.clone()
    bad[3, 2] = u.shape[0] + 1
    coffee.assemble(coffee.BURGERS_JAC, 1, PRISM, x, c2v, ud, bad, precision=coffee.FP64, validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    badv = c2v.clone()
    badv[1, 4] = -3
    coffee.assemble(coffee.BURGERS_RESIDUAL, 1, PRISM, x, badv, ud, cd, precision=coffee.FP64, validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    empty = coffee.assemble(coffee.BURGERS_JAC, 2, PRISM, x, c2v[:0].contiguous(), ud,
                            torch.empty((0, 18), dtype=torch.int32, device=DEV), precision=coffee.FP64)
    assert empty.shape == (0, 54, 54)
    # a ragged count of cells (odd, not a multiple of the warps per block) matches the oracle
    sl = slice(0, 7)
    ref = oracle.prism_burgers(1, mesh.coords, mesh.cell2vert[sl], u, c2d[sl])
    out = coffee.assemble(coffee.BURGERS_JAC, 1, PRISM, x, c2v[sl].contiguous(), ud, cd[sl].contiguous(),
                          precision=coffee.FP64)
    coffee.check_errors()
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_prism_burgers_global_assembly_fp64(k):
    """The Jacobian added straight into CSR values over a conforming vector dof numbering
    (component-blocked: global row c * nnodes + node), against the oracle's element matrices
    scattered by the oracle's own CSR assembly."""
    mesh = meshgen.prism_mesh(4, 3, perturb=0.15, seed=60 + k)
    u, c2d, nn = meshgen.burgers_coefficients(mesh, k, seed=61 + k)
    l2g = np.concatenate([c2d.astype(np.int64) + c * nn for c in range(3)], axis=1).astype(np.int32)
    A_e = oracle.prism_burgers(k, mesh.coords, mesh.cell2vert, u, c2d)
    x, c2v, ud, cd = on_device(mesh, u, c2d)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), 3 * nn)
    vals = M.assemble(coffee.BURGERS_JAC, k, PRISM, x, c2v, ud, cd, precision=coffee.FP64, validate=True)
    coffee.check_errors()
    rp, ci = M.rowptr.cpu().numpy(), M.colidx.cpu().numpy()
    ref = oracle.csr_assemble(A_e, l2g, rp, ci)
    np.testing.assert_allclose(vals.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
