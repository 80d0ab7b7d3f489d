"""Parity of GPU global assembly (CSR sparsity, entry map, fused assembly) with the oracle.

Integer results (rowptr, colidx, the entry map) must be bit-identical. Values: the
fused kernels add element-matrix entries with floating-point atomics, so the bound is
derived per global row r from the element-level tolerance eps of the precision (the
bound of the element-matrix parity tests, relative to each cell's max |A_e|) and the
rounding of the summation:
    |vals - oracle| <= (eps + n_r * u) * S_r,
with n_r the number of cells that contain row r's dof, S_r the sum of max |A_e| over
those cells and u the unit roundoff of the value type (2^-24 float, 2^-53 double):
every partial sum is bounded by S_r and each of the n_r additions rounds once.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, TOL, coefficients, to_device

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = TOL


def ragged_mesh(cell, seed):
    if cell == TRI:
        return meshgen.tri_mesh(23, perturb=0.2, seed=seed)        # 1058 cells = 8 tiles + 34
    return meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=1000)  # 7 tiles + 104


def global_map(form, mesh, k, permute_seed=None):
    """(l2g [ncells, nloc] int32, nrows): the element matrix's rows to global dofs."""
    c2d, nn = meshgen.cell2dof(mesh, k, permute_seed=permute_seed)
    if form == BURGERS_JAC:
        d = mesh.dim
        l2g = np.concatenate([c2d.astype(np.int64) + c * nn for c in range(d)], axis=1)
        return l2g.astype(np.int32), d * nn
    return c2d, nn


def row_bound(A_e, l2g, nrows, eps, unit):
    nloc = l2g.shape[1]
    scale = np.abs(A_e).reshape(A_e.shape[0], -1).max(axis=1)
    S = np.bincount(l2g.ravel(), weights=np.repeat(scale, nloc), minlength=nrows)
    n = np.bincount(l2g.ravel(), minlength=nrows)
    return (eps + n * unit) * S


def check_values(vals, ref, rowptr, bound):
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    err = np.abs(np.asarray(vals, dtype=np.float64) - ref)
    worst = float(np.max(err / np.maximum(bound[rows], 1e-300)))
    assert worst <= 1.0, worst
    return float(np.max(err) / np.max(np.abs(ref)))


@pytest.mark.parametrize("form,cell,k,perm", [
    (HELMHOLTZ, TRI, 1, None), (HELMHOLTZ, TRI, 2, None), (HELMHOLTZ, TRI, 3, 9), (HELMHOLTZ, TRI, 4, None),
    (HELMHOLTZ, TET, 1, None), (HELMHOLTZ, TET, 2, 9), (HELMHOLTZ, TET, 3, None), (HELMHOLTZ, TET, 4, None),
    (BURGERS_JAC, TRI, 2, None), (BURGERS_JAC, TET, 2, 9)])
def test_sparsity_and_map_bit_exact(form, cell, k, perm):
    mesh = ragged_mesh(cell, seed=30 + k)
    l2g, nrows = global_map(form, mesh, k, perm)
    rp_ref, ci_ref = oracle.csr_pattern(l2g, nrows)
    g = torch.from_numpy(l2g).to(DEV)
    rowptr, colidx = coffee.sparsity(g, nrows)
    np.testing.assert_array_equal(rowptr.cpu().numpy(), rp_ref)
    np.testing.assert_array_equal(colidx.cpu().numpy(), ci_ref)
    m = coffee.csr_map(g, rowptr, colidx)
    coffee.check_errors()
    # expected positions from the oracle's pattern
    n = l2g.shape[1]
    rows = np.repeat(l2g.astype(np.int64), n, axis=1).ravel()
    cols = np.tile(l2g.astype(np.int64), (1, n)).ravel()
    row_of = np.repeat(np.arange(nrows, dtype=np.int64), np.diff(rp_ref))
    keys = row_of * nrows + ci_ref
    pos = np.searchsorted(keys, rows * nrows + cols)
    mm = coffee.csr_map_unblock(m, l2g.shape[0], n)
    np.testing.assert_array_equal(mm.ravel().astype(np.int64), pos)
    flat = m.cpu().numpy().view(np.uint32)
    assert flat.size == coffee.csr_map_len(l2g.shape[0], n)
    assert np.sum(flat != 0xFFFFFFFF) == pos.size  # everything else is padding


def test_sparsity_edge_cases():
    # no cells: empty rows
    g0 = torch.zeros((0, 3), dtype=torch.int32, device=DEV)
    rp, ci = coffee.sparsity(g0, 5)
    assert rp.cpu().tolist() == [0] * 6 and ci.numel() == 0
    # dofs that no cell references give empty rows; one-cell mesh is a dense block
    g = torch.tensor([[4, 1, 7]], dtype=torch.int32, device=DEV)
    rp, ci = coffee.sparsity(g, 9)
    assert rp.cpu().tolist() == [0, 0, 3, 3, 3, 6, 6, 6, 9, 9]
    assert ci.cpu().tolist() == [1, 4, 7] * 3
    # an index outside [0, nrows) is rejected
    with pytest.raises(coffee.CoffeeError):
        coffee.sparsity(g, 7)
    # a row gathering more than 4096 entries is rejected (1100 cells around dof 0)
    star = np.stack([np.zeros(1100, np.int64), 1 + 3 * np.arange(1100), 2 + 3 * np.arange(1100),
                     3 + 3 * np.arange(1100)], axis=1).astype(np.int32)
    with pytest.raises(coffee.CoffeeError):
        coffee.sparsity(torch.from_numpy(star).to(DEV), 3301)


def test_map_of_a_pattern_that_misses_entries_flags_an_error():
    mesh = ragged_mesh(TRI, seed=3)
    l2g, nrows = global_map(HELMHOLTZ, mesh, 2)
    g = torch.from_numpy(l2g).to(DEV)
    rowptr, colidx = coffee.sparsity(g[:10].contiguous(), nrows)  # pattern of the first 10 cells only
    m = coffee.csr_map(g, rowptr, colidx)
    with pytest.raises(coffee.CoffeeError):
        coffee.check_errors()
    mm = coffee.csr_map_unblock(m, l2g.shape[0], l2g.shape[1])
    assert np.all(mm[:10] < colidx.numel()) and np.any(mm[10:] == 0xFFFFFFFF)


FP64_CASES = [(f, c, k) for f in (MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC) for c in (TRI, TET) for k in (1, 2, 3)]


@pytest.mark.parametrize("form,cell,k", FP64_CASES)
def test_fp64_global_assembly(form, cell, k):
    mesh = ragged_mesh(cell, seed=40 + k)
    coef, c2d = coefficients(form, mesh, k, seed=5)
    l2g, nrows = global_map(form, mesh, k)
    A_e = oracle.assemble(form, k, cell, mesh.coords, mesh.cell2vert, coef, c2d)
    rp, ci = oracle.csr_pattern(l2g, nrows)
    ref = oracle.csr_assemble(A_e, l2g, rp, ci)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), nrows)
    vals = M.assemble(form, k, cell, x, c2v, cf, cd, precision=coffee.FP64, validate=True)
    coffee.check_errors()
    err = check_values(vals.cpu().numpy(), ref, rp, row_bound(A_e, l2g, nrows, EPS[coffee.FP64], 2.0 ** -53))
    print("FP64 %s %s P%d: %.3e" % (coffee.FORM_NAMES[form], "tri" if cell == TRI else "tet", k, err))


TC_CASES = [(f, c, k, p) for f in (MASS, HELMHOLTZ, ADVDIFF) for c in (TRI, TET) for k in (1, 2, 3, 4)
            for p in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16)]


@pytest.mark.parametrize("form,cell,k,prec", TC_CASES)
def test_tc_fused_global_assembly(form, cell, k, prec):
    if not coffee.csr_supported(form, k, cell, prec):
        pytest.skip("no fused kernel (operands exceed shared memory)")
    mesh = ragged_mesh(cell, seed=50 + k)
    coef, c2d = coefficients(form, mesh, k, seed=6)
    l2g, nrows = global_map(form, mesh, k)
    A_e = oracle.assemble(form, k, cell, mesh.coords, mesh.cell2vert, coef, c2d)
    rp, ci = oracle.csr_pattern(l2g, nrows)
    ref = oracle.csr_assemble(A_e, l2g, rp, ci)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), nrows)
    vals = M.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True)
    coffee.check_errors()
    assert vals.dtype == torch.float32
    err = check_values(vals.cpu().numpy(), ref, rp, row_bound(A_e, l2g, nrows, EPS[prec], 2.0 ** -24))
    print("%s %s %s P%d: %.3e" % (coffee.PRECISION_NAMES[prec], coffee.FORM_NAMES[form],
                                  "tri" if cell == TRI else "tet", k, err))


@pytest.mark.parametrize("tune", [0, coffee.FLAG_SUBTILE_32, coffee.FLAG_SUBTILE_64 | coffee.FLAG_TWO_STAGES])
def test_fused_assembly_adds_into_vals_and_knobs_agree(tune):
    mesh = ragged_mesh(TET, seed=8)
    l2g, nrows = global_map(HELMHOLTZ, mesh, 2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), nrows)
    once = M.assemble(HELMHOLTZ, 2, TET, x, c2v, precision=coffee.TF32X3, tune=tune)
    twice = M.assemble(HELMHOLTZ, 2, TET, x, c2v, precision=coffee.TF32X3, vals=once.clone(), tune=tune)
    coffee.check_errors()
    torch.testing.assert_close(twice, 2 * once, rtol=1e-6, atol=1e-6 * once.abs().max().item())
    # the scattered element matrices sum to the same global matrix as the plain kernel's output
    A = coffee.assemble(HELMHOLTZ, 2, TET, x, c2v, precision=coffee.TF32X3).double().cpu().numpy()
    rp, ci = M.rowptr.cpu().numpy(), M.colidx.cpu().numpy()
    ref = oracle.csr_assemble(A, l2g, rp, ci)
    np.testing.assert_allclose(once.double().cpu().numpy(), ref, rtol=0, atol=1e-6 * np.abs(ref).max())


def test_fused_assembly_rejects_burgers_on_tensor_cores_and_bad_dtypes():
    mesh = ragged_mesh(TRI, seed=9)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, seed=6)
    l2g, nrows = global_map(BURGERS_JAC, mesh, 2)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), nrows)
    with pytest.raises(coffee.CoffeeError):
        M.assemble(BURGERS_JAC, 2, TRI, x, c2v, cf, cd, precision=coffee.TF32X3)
    with pytest.raises(TypeError):
        M.assemble(BURGERS_JAC, 2, TRI, x, c2v, cf, cd, precision=coffee.FP64,
                   vals=torch.zeros(M.nnz, dtype=torch.float32, device=DEV))


def test_full_size_helmholtz_p3_sampled_rows():
    """64^3 x 6 Kuhn tets, P3, TF32X3 (the benchmark's global-assembly workload): 64 sampled
    rows against the oracle's sum over the incident cells; the mass matrix sums to the
    measure of the unit cube."""
    mesh = meshgen.tet_mesh(64, perturb=0.15, seed=2)
    k = 3
    l2g, nrows = global_map(HELMHOLTZ, mesh, k)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    M = coffee.CsrMatrix(torch.from_numpy(l2g).to(DEV), nrows)
    vals = M.assemble(HELMHOLTZ, k, TET, x, c2v, precision=coffee.TF32X3)
    mass = M.assemble(MASS, k, TET, x, c2v, precision=coffee.TF32X3)
    coffee.check_errors()
    assert abs(mass.double().sum().item() - 1.0) < 1e-5
    rp, ci = M.rowptr.cpu().numpy(), M.colidx.cpu().numpy()
    v = vals.cpu().numpy()
    rng = np.random.default_rng(12)
    rows = rng.choice(nrows, 64, replace=False)
    flat = l2g.ravel()
    order = np.argsort(flat, kind="stable")
    starts = np.searchsorted(flat[order], rows)
    ends = np.searchsorted(flat[order], rows, side="right")
    for r, a, b in zip(rows, starts, ends):
        hits = order[a:b]
        cells, local = hits // l2g.shape[1], hits % l2g.shape[1]
        A_e = oracle.assemble_cells(HELMHOLTZ, k, TET, mesh.coords, mesh.cell2vert, cells)
        row = {}
        for A, e, i in zip(A_e, cells, local):
            for j in range(l2g.shape[1]):
                row[int(l2g[e, j])] = row.get(int(l2g[e, j]), 0.0) + A[i, j]
        cols = ci[rp[r]:rp[r + 1]]
        assert sorted(row) == cols.tolist()
        ref = np.array([row[c] for c in cols.tolist()])
        S = np.abs(A_e).reshape(len(cells), -1).max(axis=1).sum()
        bound = (EPS[coffee.TF32X3] + len(cells) * 2.0 ** -24) * S
        assert np.max(np.abs(v[rp[r]:rp[r + 1]] - ref)) <= bound
