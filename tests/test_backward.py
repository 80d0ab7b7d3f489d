"""Adjoint kernel (coffee_assemble_backward / AssembleFn) against the FP64 oracle's
dual-number gradient and against central finite differences of cell-local losses."""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import (TRI, TET, MASS, HELMHOLTZ, ADVDIFF, small_mesh, coefficients, to_device)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = [(f, c, k) for f in (MASS, HELMHOLTZ, ADVDIFF) for c in (TRI, TET) for k in (1, 2, 3, 4)]


@pytest.mark.parametrize("form,cell,k", CASES)
@pytest.mark.parametrize("deterministic", [False, True])
def test_backward_matches_oracle(form, cell, k, deterministic):
    mesh = small_mesh(cell, seed=30 + k)
    coef, c2d = coefficients(form, mesh, k, seed=31)
    n = coffee.ndof(form, k, cell)
    dout = np.random.default_rng(k).standard_normal((mesh.ncells, n, n))
    gx, gc = oracle.assemble_backward(form, k, cell, mesh.coords, mesh.cell2vert, dout, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    dx, dc = coffee.assemble_backward(form, k, cell, x, c2v, torch.from_numpy(dout).to(DEV), cf, cd,
                                      deterministic=deterministic, validate=True)
    coffee.check_errors()
    assert rel(dx.cpu().numpy(), gx) < 1e-10
    if form == ADVDIFF:
        assert rel(dc.cpu().numpy(), gc) < 1e-10


def test_deterministic_mode_is_bitwise_repeatable_and_matches_atomics():
    mesh = meshgen.tet_mesh(8, seed=5)
    coef, c2d = coefficients(ADVDIFF, mesh, 2, seed=5)
    dout = torch.randn((mesh.ncells, 10, 10), dtype=torch.float64, device=DEV)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    runs = [coffee.assemble_backward(ADVDIFF, 2, TET, x, c2v, dout, cf, cd, deterministic=True)
            for _ in range(2)]
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    at = coffee.assemble_backward(ADVDIFF, 2, TET, x, c2v, dout, cf, cd, deterministic=False)
    assert rel(at[0].cpu().numpy(), runs[0][0].cpu().numpy()) < 1e-12
    assert rel(at[1].cpu().numpy(), runs[0][1].cpu().numpy()) < 1e-12


@pytest.mark.parametrize("form", [HELMHOLTZ, ADVDIFF])
def test_autograd_function_central_differences(form):
    """loss = sum(W * A(coords, coef)); gradient through AssembleFn vs central differences
    (h = 1e-6) of the GPU forward on the cells touching each perturbed vertex."""
    mesh = meshgen.tet_mesh(3, seed=8)
    coef, c2d = coefficients(form, mesh, 2, seed=8)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    x = x.clone().requires_grad_(True)
    if cf is not None:
        cf = cf.clone().requires_grad_(True)
    W = torch.randn((mesh.ncells, 10, 10), dtype=torch.float64, device=DEV)
    A = coffee.AssembleFn.apply(x, cf, c2v, cd, form, 2, TET, coffee.FP64, False)
    (A * W).sum().backward()
    gx = x.grad.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(0)
    xs = mesh.coords.copy()
    for v in rng.choice(mesh.nverts, size=6, replace=False):
        cells = torch.from_numpy(np.nonzero((mesh.cell2vert == v).any(axis=1))[0]).to(DEV)
        for r in range(3):
            def loss(shift):
                xp = xs.copy()
                xp[v, r] += shift
                Ap = coffee.assemble(form, 2, TET, torch.from_numpy(xp).to(DEV), c2v, cf.detach() if cf is not None else None, cd)
                return float((Ap[cells] * W[cells]).sum())
            fd = (loss(h) - loss(-h)) / (2 * h)
            assert abs(fd - gx[v, r]) <= 1e-6 * np.abs(gx).max(), (v, r, fd, gx[v, r])
    if form == ADVDIFF:
        gc = cf.grad.cpu().numpy()
        flat = coef.copy()
        for idx in rng.choice(flat.size, size=8, replace=False):
            def lossc(shift):
                cp = flat.copy()
                cp[idx] += shift
                Ap = coffee.assemble(form, 2, TET, x.detach(), c2v, torch.from_numpy(cp).to(DEV), cd)
                return float((Ap * W).sum())
            fd = (lossc(1.0) - lossc(-1.0)) / 2.0  # A is linear in the coefficients
            assert abs(fd - gc[idx]) <= 1e-9 * np.abs(gc).max()


@pytest.mark.parametrize("form", [HELMHOLTZ, ADVDIFF])
def test_fp32_dout_path(form):
    """TF32X3 forward + float32 dL/dA: the adjoint runs in FP32 (vertex differences in FP64),
    so the gradient matches the FP64 oracle (fed the same float32 dL/dA) to FP32 accuracy:
    K x N-term contractions and the chain rule, held to 1e-5 of max|grad| (measured ~4e-7)."""
    mesh = meshgen.tet_mesh(4, seed=9)
    coef, c2d = coefficients(form, mesh, 2, seed=9)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    dout32 = torch.randn((mesh.ncells, 10, 10), dtype=torch.float32, device=DEV)
    gx, gc = oracle.assemble_backward(form, 2, TET, mesh.coords, mesh.cell2vert,
                                      dout32.double().cpu().numpy(), coef, c2d)
    dx, dc = coffee.assemble_backward(form, 2, TET, x, c2v, dout32, cf, cd, precision=coffee.TF32X3)
    ex = rel(dx.cpu().numpy(), gx)
    print("fp32 adjoint %s: coords %.2e" % (coffee.FORM_NAMES[form], ex))
    assert ex < 1e-5
    if form == ADVDIFF:
        ec = rel(dc.cpu().numpy(), gc)
        print("fp32 adjoint coef %.2e" % ec)
        assert ec < 1e-5


@pytest.mark.parametrize("form", [HELMHOLTZ, ADVDIFF])
def test_config5_full_size_sampled_vertices(form):
    """2^19 P2 tets (Kuhn 64x64x22 truncated), dL/dA ~ N(0,1): gradients at sampled vertices
    vs the oracle's adjoint over exactly the cells incident to them."""
    mesh = meshgen.tet_mesh(64, 64, 22, perturb=0.15, seed=5, ncells=2 ** 19)
    coef, c2d = coefficients(form, mesh, 2, seed=5)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    g = torch.Generator(device=DEV).manual_seed(5)
    dout = torch.randn((mesh.ncells, 10, 10), dtype=torch.float64, device=DEV, generator=g)
    dx, dc = coffee.assemble_backward(form, 2, TET, x, c2v, dout, cf, cd, deterministic=True)
    rng = np.random.default_rng(5)
    verts = rng.choice(np.unique(mesh.cell2vert), size=40, replace=False)
    cells = np.nonzero(np.isin(mesh.cell2vert, verts).any(axis=1))[0]
    sub_dout = dout[torch.from_numpy(cells).to(DEV)].cpu().numpy()
    gx, gc = oracle.assemble_backward(form, 2, TET, mesh.coords, mesh.cell2vert[cells], sub_dout, coef,
                                      None if c2d is None else c2d[cells])
    got = dx.cpu().numpy()[verts]
    assert rel(got, gx[verts]) < 1e-10
    if form == ADVDIFF:
        # P1 coefficient nodes are the vertices here (cell2dof numbers the vertex lattice)
        nodes = np.unique(c2d[cells][np.isin(mesh.cell2vert[cells], verts)])
        assert rel(dc.cpu().numpy().reshape(-1, 4)[nodes], gc.reshape(-1, 4)[nodes]) < 1e-10
