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
from tests.helpers import MASS, HELMHOLTZ, ADVDIFF, TOL, rel_err_per_cell

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
    with pytest.raises(coffee.CoffeeError):  # Burgers on prisms runs in FP64 only
        coffee.assemble(coffee.BURGERS_JAC, 1, PRISM, x, c2v, torch.zeros(64 * 3, dtype=torch.float64, device=DEV),
                        c2v, precision=coffee.TF32X3)
    with pytest.raises(coffee.CoffeeError):  # advection-diffusion needs its coefficients
        coffee.assemble(ADVDIFF, 1, PRISM, x, c2v, precision=coffee.FP64)
    coef, c2d, _ = meshgen.advdiff_coefficients(mesh, 1)
    badd = torch.from_numpy(c2d).to(DEV)
    badd[2, 4] = -1
    coffee.assemble(ADVDIFF, 1, PRISM, x, c2v, torch.from_numpy(coef).to(DEV), badd, precision=coffee.FP64,
                    validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    coffee.assemble(ADVDIFF, 1, PRISM, x, c2v, torch.from_numpy(coef).to(DEV), badd, precision=coffee.TF32X3,
                    validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    bad = c2v.clone()
    bad[5, 3] = mesh.nverts + 7
    coffee.assemble(MASS, 1, PRISM, x, bad, precision=coffee.FP64, validate=True)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    empty = coffee.assemble(MASS, 2, PRISM, x, c2v[:0].contiguous(), precision=coffee.FP64)
    assert empty.shape == (0, 18, 18)


TC_TOL = TOL


def prism_tol(prec, form, k):
    """The simplex bounds (tests.helpers.TOL) hold for prisms as well: no allowance is added for
    the long K = (k+2)^3 KQ of the quadrature-point contraction."""
    return TOL[prec]


@pytest.mark.parametrize("form", [MASS, HELMHOLTZ])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_prism_tensor_cores_match_oracle(form, k, prec):
    """K-chunked streamed contraction on the tensor cores (972 cells: 7 tiles + a ragged one;
    P3's 13 and P4's 44 output slices run in groups of at most three)."""
    mesh = meshgen.prism_mesh(9, 6, perturb=0.15, seed=30 + k)
    ref = oracle.prism_assemble(form, k, mesh.coords, mesh.cell2vert)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(form, k, PRISM, x, c2v, precision=prec, validate=True)
    coffee.check_errors()
    assert out.dtype == torch.float32 and out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism TC %s P%d %s: %.3e" % (coffee.FORM_NAMES[form], k, coffee.PRECISION_NAMES[prec], err))
    assert err < prism_tol(prec, form, k)


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


def advdiff_case(n, nz, seed):
    mesh = meshgen.prism_mesh(n, nz, perturb=0.15, seed=seed)
    coef, c2d, _ = meshgen.advdiff_coefficients(mesh, seed)
    return mesh, coef, c2d, torch.from_numpy(coef).to(DEV), torch.from_numpy(c2d).to(DEV)


@pytest.mark.parametrize("k,n,nz", [(1, 9, 6), (2, 9, 6), (3, 6, 4), (4, 4, 3)])
def test_prism_advdiff_fp64_matches_oracle(k, n, nz):
    """Advection-diffusion with P1 eps and b (random per vertex) on twisted prisms."""
    mesh, coef, c2d, cf, cd = advdiff_case(n, nz, 40 + k)
    ref = oracle.prism_assemble(ADVDIFF, k, mesh.coords, mesh.cell2vert, coef, c2d)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(ADVDIFF, k, PRISM, x, c2v, cf, cd, precision=coffee.FP64, validate=True)
    coffee.check_errors()
    assert out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism ADVDIFF P%d: %.3e" % (k, err))
    assert err < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_prism_advdiff_tensor_cores_match_oracle(k, prec):
    """K = 9 Q factors per cell (six diffusion pairs, three advection factors): 972 cells."""
    mesh, coef, c2d, cf, cd = advdiff_case(9, 6, 50 + k)
    ref = oracle.prism_assemble(ADVDIFF, k, mesh.coords, mesh.cell2vert, coef, c2d)
    x, c2v = to_dev(mesh)
    out = coffee.assemble(ADVDIFF, k, PRISM, x, c2v, cf, cd, precision=prec, validate=True)
    coffee.check_errors()
    assert out.dtype == torch.float32 and out.shape == ref.shape
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("prism TC ADVDIFF P%d %s: %.3e" % (k, coffee.PRECISION_NAMES[prec], err))
    assert err < prism_tol(prec, ADVDIFF, k)


def test_prism_advdiff_global_assembly():
    """Fused CSR assembly of the P2 advection-diffusion operator on prisms, FP64 and TF32X3."""
    mesh, coef, c2d1, cf, cd = advdiff_case(6, 4, 60)
    c2d, nn = meshgen.cell2dof(mesh, 2)
    x, c2v = to_dev(mesh)
    M = coffee.CsrMatrix(torch.from_numpy(c2d).to(DEV), nn)
    ref_local = oracle.prism_assemble(ADVDIFF, 2, mesh.coords, mesh.cell2vert, coef, c2d1)
    rp, ci = M.rowptr.cpu().numpy(), M.colidx.cpu().numpy()
    ref = oracle.csr_assemble(ref_local, c2d, rp, ci)
    for prec, tol in [(coffee.FP64, 1e-12), (coffee.TF32X3, 1e-5)]:
        vals = M.assemble(ADVDIFF, 2, PRISM, x, c2v, cf, cd, precision=prec)
        coffee.check_errors()
        np.testing.assert_allclose(vals.cpu().numpy(), ref, rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("form", [MASS, HELMHOLTZ, ADVDIFF])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prism_global_assembly_tensor_cores(form, k):
    """The tensor-core prism kernel adding its entries straight into the CSR values (972 cells,
    a ragged last tile), against the oracle's element matrices scattered on the host."""
    mesh, coef, c2d1, cf, cd = advdiff_case(9, 6, 70 + k)
    c2d, nn = meshgen.cell2dof(mesh, k)
    x, c2v = to_dev(mesh)
    M = coffee.CsrMatrix(torch.from_numpy(c2d).to(DEV), nn)
    extra = (coef, c2d1) if form == ADVDIFF else ()
    ref = oracle.csr_assemble(oracle.prism_assemble(form, k, mesh.coords, mesh.cell2vert, *extra), c2d,
                              M.rowptr.cpu().numpy(), M.colidx.cpu().numpy())
    dev_extra = (cf, cd) if form == ADVDIFF else ()
    vals = M.assemble(form, k, PRISM, x, c2v, *dev_extra, precision=coffee.TF32X3, validate=True)
    coffee.check_errors()
    assert vals.dtype == torch.float32
    np.testing.assert_allclose(vals.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    # an entry of the map past nnz is skipped and reported
    bad = M.map.clone()
    bad[5] = M.nnz + 3
    coffee.assemble_csr(form, k, PRISM, x, c2v, bad, torch.zeros_like(vals), *dev_extra,
                        precision=coffee.TF32X3)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
