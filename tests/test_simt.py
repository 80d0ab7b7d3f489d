"""Parity of the FP32 CUDA-core kernel for small element matrices (k_simt.cu: MASS, HELMHOLTZ,
ADVDIFF on triangles P1-P3 and tetrahedra P1-P2) with the FP64 oracle, and of the tensor-core
kernel on the same cases when it is forced (the library's default for P1 and for triangles P2
is the CUDA-core kernel). Error metric and bounds as in test_parity_tc: per cell max_ij |A - A_oracle| /
max_ij |A_oracle|; the CUDA-core kernel computes in FP32 whatever tensor-core precision is asked
for, so it is held to the split precisions' 1e-5 for every precision.
Sizes span several 32-cell warp tiles with a ragged last one; the output tail past the last
cell must stay untouched; a misaligned output takes the scalar store path."""
import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import (TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, TOL, coefficients,
                           rel_err_per_cell, to_device, oracle_ref)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SIMT = coffee.FLAG_CUDA_CORES
TC = coffee.FLAG_TENSOR_CORES

CASES = [(f, c, k) for f in (MASS, HELMHOLTZ, ADVDIFF) for c, ks in ((TRI, (1, 2, 3)), (TET, (1, 2))) for k in ks]


def mesh_of(cell, seed, ncells=None):
    if cell == TRI:
        m = meshgen.tri_mesh(23, perturb=0.2, seed=seed)  # 1058 cells = 33 warp tiles + 2
        return m if ncells is None else meshgen.Mesh(TRI, m.coords, m.cell2vert[:ncells].copy(), None, m.shape)
    return meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=ncells or 1001)  # 31 warp tiles + 9


@pytest.mark.parametrize("form,cell,k", CASES)
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16])
def test_cuda_core_kernel_matches_oracle(form, cell, k, prec):
    mesh = mesh_of(cell, seed=40 + k)
    coef, c2d = coefficients(form, mesh, k, seed=41)
    ref = oracle_ref(form, k, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True, tune=SIMT)
    coffee.check_errors()
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("simt %s %s P%d: %.3e" % (coffee.FORM_NAMES[form], "tri" if cell == TRI else "tet", k, err))
    assert err < 1e-5


@pytest.mark.parametrize("cell", [TRI, TET])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16, coffee.BF16X3])
def test_burgers_p1_on_the_cuda_cores(cell, prec):
    """The Burgers Jacobian on P1 simplices (the default path): factored blocks in FP32 against
    the oracle, within the split precisions' bound whatever precision is asked for; with the
    float coefficient copy bit for bit the same; a ragged last warp tile."""
    mesh = mesh_of(cell, seed=70)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 1, seed=71)
    ref = oracle_ref(BURGERS_JAC, 1, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    assert coffee.assemble_path(BURGERS_JAC, 1, cell, prec) == 2
    out = coffee.assemble(BURGERS_JAC, 1, cell, x, c2v, cf, cd, precision=prec, validate=True)
    coffee.check_errors()
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("simt burgers %s P1: %.3e" % ("tri" if cell == TRI else "tet", err))
    assert err < 1e-5
    out2 = coffee.assemble(BURGERS_JAC, 1, cell, x, c2v, cf, cd, precision=prec, coef_f32=coffee.round_coef(cf))
    assert torch.equal(out, out2)


@pytest.mark.parametrize("form", [BURGERS_JAC, coffee.BURGERS_RESIDUAL])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16])
def test_burgers_triangles_p2_on_the_cuda_cores(form, prec):
    """Triangles P2 (the default path there): Jacobian and residual within the split
    precisions' bound of the oracle."""
    mesh = mesh_of(TRI, seed=74)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, seed=75)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    assert coffee.assemble_path(form, 2, TRI, prec, coffee.FLAG_CUDA_CORES) == 2
    out = coffee.assemble(form, 2, TRI, x, c2v, cf, cd, precision=prec, validate=True, tune=coffee.FLAG_CUDA_CORES)
    coffee.check_errors()
    if form == BURGERS_JAC:
        ref = oracle_ref(BURGERS_JAC, 2, TRI, mesh, coef, c2d)
        assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5
    else:
        import oracle
        ref = oracle.burgers_residual(2, TRI, mesh.coords, mesh.cell2vert, coef.reshape(-1, 2), c2d)
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


def test_burgers_p1_flags_a_bad_index():
    mesh = mesh_of(TET, seed=72)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 1, seed=73)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    bad = cd.clone()
    bad[5, 2] = mesh.nverts * 10
    out = coffee.assemble(BURGERS_JAC, 1, TET, x, c2v, cf, bad, precision=coffee.TF32X3, validate=True)
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4
    assert torch.count_nonzero(out[5]) == 0


@pytest.mark.parametrize("form,cell", [(f, c) for f in (MASS, HELMHOLTZ, ADVDIFF) for c in (TRI, TET)])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_tensor_core_kernel_p1_when_forced(form, cell, prec):
    mesh = mesh_of(cell, seed=50)
    coef, c2d = coefficients(form, mesh, 1, seed=51)
    ref = oracle_ref(form, 1, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(form, 1, cell, x, c2v, cf, cd, precision=prec, validate=True, tune=TC)
    coffee.check_errors()
    assert rel_err_per_cell(out.cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("ncells", [1, 31, 32, 33, 95, 257])
@pytest.mark.parametrize("cell,k", [(TET, 1), (TET, 2), (TRI, 3)])
def test_ragged_tails_and_untouched_tail(ncells, cell, k):
    mesh = mesh_of(cell, seed=60, ncells=ncells)
    ref = oracle_ref(HELMHOLTZ, k, cell, mesh, None, None)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    n = coffee.ndof(HELMHOLTZ, k, cell)
    buf = torch.full((ncells + 2, n, n), 7.0, dtype=torch.float32, device=DEV)
    coffee.assemble(HELMHOLTZ, k, cell, x, c2v, precision=coffee.TF32X3, out=buf[:ncells], tune=SIMT)
    torch.cuda.synchronize()
    assert rel_err_per_cell(buf[:ncells].cpu().numpy(), ref) < 1e-5
    assert torch.all(buf[ncells:] == 7.0)


def test_misaligned_output_takes_scalar_stores():
    mesh = mesh_of(TET, seed=61)
    coef, c2d = coefficients(ADVDIFF, mesh, 1, seed=62)
    ref = oracle_ref(ADVDIFF, 1, TET, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    flat = torch.full((mesh.ncells * 16 + 2,), 7.0, dtype=torch.float32, device=DEV)
    out = flat[1:1 + mesh.ncells * 16].view(mesh.ncells, 4, 4)
    coffee.assemble(ADVDIFF, 1, TET, x, c2v, cf, cd, precision=coffee.TF32X3, out=out, tune=SIMT)
    torch.cuda.synchronize()
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5
    assert flat[0].item() == 7.0 and flat[-1].item() == 7.0


def test_sliver_cells_take_fp64_geometry():
    """Badly conditioned cells take the FP64 geometry: same bound as regular cells."""
    rng = np.random.default_rng(5)
    X = np.concatenate([meshgen.sliver_tet(rng, flat) for flat in (1e-1, 1e-2, 1e-3, 1e-4)])
    c2v = np.arange(16, dtype=np.int32).reshape(4, 4)
    mesh = meshgen.Mesh(TET, X, c2v, None, (1, 1, 1))
    for k in (1, 2):
        ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None)
        x, cv, _, _ = to_device(mesh, None, None, DEV)
        out = coffee.assemble(HELMHOLTZ, k, TET, x, cv, precision=coffee.TF32X3, tune=SIMT)
        assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


def test_coordinates_outside_the_integer_split_take_fp64_geometry():
    """Coordinates of magnitude below 2^-70 but not zero (here the zeros of the boundary
    replaced by +-1e-30) are outside what the integer (hi, lo) split covers: those cells take
    the FP64 geometry, and every cell still meets the bound."""
    mesh = meshgen.tet_mesh(5, perturb=0.15, seed=65)
    X = mesh.coords.copy()
    zeros = X == 0.0
    assert zeros.any()
    X[zeros] = np.where(np.random.default_rng(66).random(zeros.sum()) < 0.5, -1e-30, 1e-30)
    mesh = meshgen.Mesh(TET, X, mesh.cell2vert, None, mesh.shape)
    for k in (1, 2):
        ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None)
        x, c2v, _, _ = to_device(mesh, None, None, DEV)
        out = coffee.assemble(HELMHOLTZ, k, TET, x, c2v, precision=coffee.TF32X3, tune=SIMT)
        assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


def test_zero_and_negative_coordinates():
    """A mesh around the origin (coordinates of both signs and exact zeros) against the oracle."""
    mesh = meshgen.tet_mesh(5, perturb=0.15, seed=63)
    mesh = meshgen.Mesh(TET, mesh.coords - mesh.coords[37], mesh.cell2vert, None, mesh.shape)
    assert (mesh.coords == 0.0).any() and (mesh.coords < 0).any()
    ref = oracle_ref(HELMHOLTZ, 2, TET, mesh, None, None)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 2, TET, x, c2v, precision=coffee.TF32X3, tune=SIMT)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


def test_cuda_core_kernel_flags_a_bad_index():
    mesh = meshgen.tet_mesh(3, seed=4)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    bad = c2v.clone()
    bad[17, 1] = -3
    out = coffee.assemble(HELMHOLTZ, 1, TET, x, bad, precision=coffee.TF32X3, validate=True, tune=SIMT)
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4
    assert torch.count_nonzero(out[17]) == 0


@pytest.mark.parametrize("cell,k,path", [(TRI, 1, SIMT), (TET, 1, SIMT), (TRI, 2, SIMT), (TET, 2, TC), (TRI, 3, TC)])
def test_default_path(cell, k, path):
    """Without a flag, P1 (both cells) and triangles P2 take the CUDA-core kernel, tets P2 and
    triangles P3 the tensor cores: bit for bit the result with that path forced."""
    mesh = mesh_of(cell, seed=64)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    a = coffee.assemble(HELMHOLTZ, k, cell, x, c2v, precision=coffee.TF32X3, tune=0)
    b = coffee.assemble(HELMHOLTZ, k, cell, x, c2v, precision=coffee.TF32X3, tune=path)
    assert torch.equal(a, b)


@pytest.mark.parametrize("k", [1, 2])
def test_full_size_tets_sampled(k):
    """1,572,864 Kuhn tets (64^3 x 6), Helmholtz Pk on the CUDA cores, in the launch configuration
    the benchmark times: 2000 sampled cells and both ends against the oracle."""
    mesh = meshgen.tet_mesh(64, perturb=0.15, seed=2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, k, TET, x, c2v, precision=coffee.TF32X3, tune=SIMT)
    sel = np.concatenate([np.random.default_rng(70 + k).choice(mesh.ncells, size=2000, replace=False),
                          [0, mesh.ncells - 1]])
    ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None, sel=sel)
    assert rel_err_per_cell(out[torch.from_numpy(sel).to(DEV)].cpu().numpy(), ref) < 1e-5
