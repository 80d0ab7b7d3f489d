"""Parity of the plain FP64 GPU kernel (coffee_assemble / precision FP64) with the
FP64 oracle: element by element, 1e-12 relative to max|A_e| per cell."""
import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import (TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, small_mesh,
                           coefficients, rel_err_per_cell, to_device, oracle_ref)

pytestmark = pytest.mark.gpu
TOL = 1e-12
DEV = "cuda:0"

CASES = [(f, c, k) for f in (MASS, HELMHOLTZ, ADVDIFF) for c in (TRI, TET) for k in (1, 2, 3, 4)]
CASES += [(BURGERS_JAC, c, k) for c in (TRI, TET) for k in (1, 2, 3, 4)]


@pytest.mark.parametrize("form,cell,k", CASES)
def test_fp64_matches_oracle_small(form, cell, k):
    mesh = small_mesh(cell, seed=11 + k)
    coef, c2d = coefficients(form, mesh, k, seed=5)
    ref = oracle_ref(form, k, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=coffee.FP64, validate=True)
    coffee.check_errors()
    assert out.dtype == torch.float64 and out.shape == ref.shape
    assert rel_err_per_cell(out.cpu().numpy(), ref) < TOL


def test_plain_signature_equals_ex():
    mesh = small_mesh(TET, seed=3)
    coef, c2d = coefficients(ADVDIFF, mesh, 2)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    a = coffee.assemble(ADVDIFF, 2, TET, x, c2v, cf, cd)
    b = coffee.assemble_plain(ADVDIFF, 2, TET, x, c2v, cf, cd)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_permuted_coefficient_numbering():
    mesh = small_mesh(TET, seed=4)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, permute_seed=99)
    ref = oracle_ref(BURGERS_JAC, 2, TET, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(BURGERS_JAC, 2, TET, x, c2v, cf, cd)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < TOL


def test_empty_and_single_cell():
    mesh = small_mesh(TRI, n=2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 2, TRI, x, c2v[:0])
    assert out.shape == (0, 6, 6)
    out = coffee.assemble(HELMHOLTZ, 2, TRI, x, c2v[:1].contiguous())
    ref = oracle_ref(HELMHOLTZ, 2, TRI, mesh, None, None)[:1]
    assert rel_err_per_cell(out.cpu().numpy(), ref) < TOL


def test_sliver_cells():
    rng = np.random.default_rng(5)
    X = np.concatenate([meshgen.sliver_tet(rng, flat) for flat in (1e-2, 1e-4, 1e-6)])
    c2v = np.arange(12, dtype=np.int32).reshape(3, 4)
    mesh = meshgen.Mesh(TET, X, c2v, None, (1, 1, 1))
    ref = oracle_ref(HELMHOLTZ, 3, TET, mesh, None, None)
    x, cv, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 3, TET, x, cv)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-9  # conditioning ~1/flat


def test_validation_flags_out_of_range_index():
    mesh = small_mesh(TET)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    bad = c2v.clone()
    bad[5, 2] = mesh.nverts + 7
    coffee.assemble(MASS, 1, TET, x, bad, validate=True)
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4
    coffee.check_errors()  # the word was cleared


def test_full_size_config1_triangles():
    """8192 perturbed triangles, P1 mass and Helmholtz, every cell."""
    mesh = meshgen.tri_mesh(64, perturb=0.2, seed=1)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    for form in (MASS, HELMHOLTZ):
        ref = oracle_ref(form, 1, TRI, mesh, None, None)
        out = coffee.assemble(form, 1, TRI, x, c2v)
        assert rel_err_per_cell(out.cpu().numpy(), ref) < TOL
    m = coffee.assemble(MASS, 1, TRI, x, c2v)
    assert abs(m.sum().item() - 1.0) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_full_size_config2_sampled(k):
    """1,572,864 Kuhn tets (64^3 x 6), Helmholtz Pk: sampled cells vs oracle, and the
    mass of the whole mesh equals the cube's volume."""
    mesh = meshgen.tet_mesh(64, perturb=0.15, seed=2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, k, TET, x, c2v)
    sel = np.random.default_rng(k).choice(mesh.ncells, size=3000, replace=False)
    sel = np.concatenate([sel, [0, mesh.ncells - 1]])
    ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None, sel=sel)
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy()
    assert rel_err_per_cell(got, ref) < TOL
    del out
    if k <= 2:
        m = coffee.assemble(MASS, k, TET, x, c2v)
        assert abs(m.sum().item() - 1.0) < 1e-10
