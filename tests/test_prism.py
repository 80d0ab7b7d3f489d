"""Parity of the FP64 prism kernel (the paper's third element shape) with the oracle.

Both sides evaluate the same fixed quadrature rule (n = k+2 Gauss-Legendre points per
direction, Duffy-collapsed triangle factor), each from its own implementation, on
non-affine (twisted) prisms: the results agree to rounding, held to 1e-12 of each cell's
max |A_e| like the FP64 simplex kernel.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import MASS, HELMHOLTZ, rel_err_per_cell

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PRISM = coffee.PRISM


def to_dev(mesh):
    return (torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.cell2vert).to(DEV))


@pytest.mark.parametrize("form", [MASS, HELMHOLTZ])
@pytest.mark.parametrize("k,n,nz", [(1, 9, 6), (2, 9, 6), (3, 6, 4), (4, 4, 3)])
def test_prism_fp64_matches_oracle(form, k, n, nz):
    mesh = meshgen.prism_mesh(n, nz, perturb=0.15, seed=10 + k)
    ref = oracle.prism_assemble(form, k, mesh.coords, mesh.cell2vert)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(form, k, PRISM, x, c2v, precision=coffee.FP64, validate=True)
    coffee.check_errors()
    assert out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism %s P%d: %.3e" % (coffee.FORM_NAMES[form], k, err))
    assert err < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_prism_global_assembly_fp64(k):
    mesh = meshgen.prism_mesh(6, 4, perturb=0.15, seed=20 + k)
    c2d, nn = meshgen.cell2dof(mesh, k)
    x, c2v = to_dev(mesh)
    M = coffee.CsrMatrix(torch.from_numpy(c2d).to(DEV), nn)
    mass = M.assemble(MASS, k, PRISM, x, c2v, precision=coffee.FP64)
    helm = M.assemble(HELMHOLTZ, k, PRISM, x, c2v, precision=coffee.FP64)
    coffee.check_errors()
    assert abs(mass.sum().item() - 1.0) < 1e-12  # the mesh tiles the unit cube
    rp, ci = M.rowptr.cpu().numpy(), M.colidx.cpu().numpy()
    ref = oracle.csr_assemble(oracle.prism_assemble(HELMHOLTZ, k, mesh.coords, mesh.cell2vert), c2d, rp, ci)
    np.testing.assert_allclose(helm.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_prism_errors():
    mesh = meshgen.prism_mesh(3, 2, seed=1)
    x, c2v = to_dev(mesh)
    with pytest.raises(coffee.CoffeeError):  # tensor-core prisms stop at P2
        coffee.assemble(HELMHOLTZ, 3, PRISM, x, c2v, precision=coffee.TF32X3)
    with pytest.raises(coffee.CoffeeError):  # prisms cover MASS and HELMHOLTZ
        coffee.assemble(coffee.ADVDIFF, 1, PRISM, x, c2v, torch.zeros(64, dtype=torch.float64, device=DEV),
                        c2v[:, :4].contiguous(), precision=coffee.FP64)
    bad = c2v.clone()
    bad[5, 3] = mesh.nverts + 7
    coffee.assemble(MASS, 1, PRISM, x, bad, precision=coffee.FP64, validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    empty = coffee.assemble(MASS, 2, PRISM, x, c2v[:0].contiguous(), precision=coffee.FP64)
    assert empty.shape == (0, 18, 18)


TC_TOL = {coffee.TF32X3: 1e-5, coffee.BF16X3: 1e-4, coffee.TF32: 1e-2, coffee.BF16: 2e-2}


@pytest.mark.parametrize("form", [MASS, HELMHOLTZ])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_prism_tensor_cores_match_oracle(form, k, prec):
    """K-chunked streamed contraction on the tensor cores (972 cells: 7 tiles + a ragged one)."""
    mesh = meshgen.prism_mesh(9, 6, perturb=0.15, seed=30 + k)
    ref = oracle.prism_assemble(form, k, mesh.coords, mesh.cell2vert)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(form, k, PRISM, x, c2v, precision=prec, validate=True)
    coffee.check_errors()
    assert out.dtype == torch.float32 and out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism TC %s P%d %s: %.3e" % (coffee.FORM_NAMES[form], k, coffee.PRECISION_NAMES[prec], err))
    assert err < TC_TOL[prec]


def test_prism_tc_full_size_sampled():
    """The benchmark's 221,184 twisted P2 prisms (48 x 48 x 2 x 48, seed 6), TF32X3: 512 sampled
    cells against the oracle."""
    mesh = meshgen.prism_mesh(48, 48, perturb=0.15, seed=6)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(HELMHOLTZ, 2, PRISM, x, c2v, precision=coffee.TF32X3)
    coffee.check_errors()
    sel = np.sort(np.random.default_rng(6).choice(mesh.ncells, 512, replace=False))
    ref = oracle.prism_assemble(HELMHOLTZ, 2, mesh.coords, mesh.cell2vert[sel])
    err = rel_err_per_cell(out[torch.from_numpy(sel).to(DEV)].cpu().numpy(), ref)
    print("prism TC full size: %.3e" % err)
    assert err < TC_TOL[coffee.TF32X3]
