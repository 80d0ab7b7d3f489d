"""The host-buffer pipeline (assemble_host): host inputs copied in, the cell range assembled in
chunks, element matrices or vectors copied back on a second stream while the next chunk
computes. Each chunk is an ordinary launch over a slice of the cells, so the result must be
bitwise equal to one device-side launch over all cells, and within the kernels' tolerance of
the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, TOL, coefficients, rel_err_per_cell

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RES = coffee.BURGERS_RESIDUAL


def host_inputs(form, cell, k, seed):
    mesh = (meshgen.tri_mesh(23, perturb=0.2, seed=seed) if cell == TRI          # 1058 cells
            else meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=1000))
    coef, c2d = coefficients(BURGERS_JAC if form == RES else form, mesh, k, seed=seed + 1)
    pin = lambda a, dt: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    return mesh, coef, c2d, (pin(mesh.coords, torch.float64), pin(mesh.cell2vert, torch.int32),
                             pin(coef, torch.float64), pin(c2d, torch.int32))


@pytest.mark.parametrize("form,cell,k,prec,chunks", [
    (HELMHOLTZ, TET, 3, coffee.TF32X3, 4), (MASS, TRI, 2, coffee.FP64, 3), (ADVDIFF, TET, 2, coffee.TF32X3, 5),
    (BURGERS_JAC, TRI, 2, coffee.BF16X3, 2), (RES, TET, 2, coffee.TF32X3, 3), (HELMHOLTZ, TRI, 1, coffee.TF32X3, 7)])
def test_host_pipeline_equals_one_device_launch_and_matches_oracle(form, cell, k, prec, chunks):
    mesh, coef, c2d, (x, c2v, cf, cd) = host_inputs(form, cell, k, seed=11)
    got = coffee.assemble_host(form, k, cell, x, c2v, cf, cd, precision=prec, chunks=chunks)
    torch.cuda.synchronize()
    assert not got.is_cuda and got.is_pinned()
    dev = lambda t: None if t is None else t.to(DEV)
    ref_dev = coffee.assemble(form, k, cell, dev(x), dev(c2v), dev(cf), dev(cd), precision=prec)
    coffee.check_errors()
    assert torch.equal(got, ref_dev.cpu())
    if form == RES:
        ref = oracle.burgers_residual(k, cell, mesh.coords, mesh.cell2vert, coef.reshape(-1, 2 + cell), c2d, 0.01)
        err = float(np.abs(got.numpy() - ref).max() / np.abs(ref).max())
    else:
        ref = oracle.assemble(form, k, cell, mesh.coords, mesh.cell2vert, coef, c2d)
        err = rel_err_per_cell(got.numpy(), ref)
    assert err < TOL[prec], err


def test_host_pipeline_empty_and_more_chunks_than_cells():
    mesh, _, _, (x, c2v, _, _) = host_inputs(MASS, TRI, 1, seed=3)
    empty = coffee.assemble_host(MASS, 1, TRI, x, c2v[:0], chunks=4)
    torch.cuda.synchronize()
    assert empty.shape == (0, 3, 3)
    few = c2v[:5].clone().pin_memory()
    got = coffee.assemble_host(HELMHOLTZ, 2, TRI, x, few, precision=coffee.TF32X3, chunks=16)
    torch.cuda.synchronize()
    ref = oracle.assemble(HELMHOLTZ, 2, TRI, mesh.coords, mesh.cell2vert[:5], None, None)
    assert rel_err_per_cell(got.numpy(), ref) < 1e-5


def test_host_pipeline_with_pageable_memory_and_validation():
    """Pageable host tensors take the same path (copies no longer overlap); validate=True
    reports a bad vertex id found in any chunk."""
    mesh, coef, c2d, _ = host_inputs(ADVDIFF, TET, 2, seed=5)
    x, c2v = torch.from_numpy(mesh.coords), torch.from_numpy(mesh.cell2vert)
    cf, cd = torch.from_numpy(coef), torch.from_numpy(c2d)
    out = torch.empty((mesh.ncells, 10, 10), dtype=torch.float32)  # pageable
    got = coffee.assemble_host(ADVDIFF, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3, out=out, chunks=3,
                               validate=True)
    torch.cuda.synchronize()
    coffee.check_errors()
    ref = oracle.assemble(ADVDIFF, 2, TET, mesh.coords, mesh.cell2vert, coef, c2d)
    assert got.data_ptr() == out.data_ptr() and rel_err_per_cell(got.numpy(), ref) < 1e-5
    bad = c2v.clone()
    bad[mesh.ncells - 2, 3] = mesh.nverts + 1  # last chunk
    coffee.assemble_host(ADVDIFF, 2, TET, x, bad, cf, cd, precision=coffee.TF32X3, out=out, chunks=3,
                         validate=True)
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4


@pytest.mark.parametrize("form", [BURGERS_JAC, RES])
def test_host_pipeline_prism_burgers(form):
    """Vector Burgers on prisms (FP64) through the host pipeline: u per conforming P2 prism node,
    288 cells in three chunks; bitwise the device launch, and the oracle's values."""
    mesh = meshgen.prism_mesh(6, 4, perturb=0.15, seed=12)
    u, c2d, _ = meshgen.burgers_coefficients(mesh, 2, seed=13)
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    x, c2v, cf, cd = (pin(mesh.coords, torch.float64), pin(mesh.cell2vert, torch.int32), pin(u, torch.float64),
                      pin(c2d, torch.int32))
    got = coffee.assemble_host(form, 2, coffee.PRISM, x, c2v, cf, cd, precision=coffee.FP64, chunks=3)
    torch.cuda.synchronize()
    ref_dev = coffee.assemble(form, 2, coffee.PRISM, x.to(DEV), c2v.to(DEV), cf.to(DEV), cd.to(DEV),
                              precision=coffee.FP64)
    coffee.check_errors()
    assert torch.equal(got, ref_dev.cpu())
    ref = oracle.prism_burgers(2, mesh.coords, mesh.cell2vert, u, c2d, residual=form == RES)
    assert rel_err_per_cell(got.numpy(), ref) < 1e-12
