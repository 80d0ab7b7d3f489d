"""Parity of the tcgen05 tensor-core kernel with the FP64 oracle.

Error metric: per cell, max_ij |A - A_oracle| / max_ij |A_oracle|, maximised over cells.
Tolerances (tests.helpers.TOL): TF32X3 and BF16X3 1e-5, single-pass TF32 and BF16 1e-2.
TF32X3 keeps the three products of order <= 1 of two-part operands (2^-22 each); BF16X3 the
six products of order <= 2 of three-part operands (2^-24 each); BF16 holds T in two parts so
that only the factors' single rounding (2^-8) remains, and the stiffness factors are the
edge factors c_ij = |det J| grad(lambda_i).grad(lambda_j), whose sum_k |G_k T_k| / max|A_e|
stays near 1-2 instead of 4-6 for the reference-direction pairs.
Sizes span several 128-cell tiles with a ragged last tile.
"""
import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import (TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, TOL, coefficients,
                           rel_err_per_cell, to_device, oracle_ref)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def ragged_mesh(cell, seed):
    if cell == TRI:
        return meshgen.tri_mesh(23, perturb=0.2, seed=seed)        # 1058 cells = 8 tiles + 34
    return meshgen.tet_mesh(6, perturb=0.15, seed=seed, ncells=1000)  # 7 tiles + 104


CASES = [(f, c, k, p) for f in (MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC) for c in (TRI, TET)
         for k in (1, 2, 3, 4) for p in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16)]


@pytest.mark.parametrize("form,cell,k,prec", CASES)
def test_tc_matches_oracle(form, cell, k, prec):
    if not coffee.supported(form, k, cell, prec):
        pytest.skip("combination not built (operands exceed shared memory)")
    mesh = ragged_mesh(cell, seed=20 + k)
    coef, c2d = coefficients(form, mesh, k, seed=7)
    ref = oracle_ref(form, k, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True)
    coffee.check_errors()
    assert out.dtype == torch.float32
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("%s %s P%d %s: %.3e" % (coffee.FORM_NAMES[form], "tri" if cell == TRI else "tet", k,
                                  coffee.PRECISION_NAMES[prec], err))
    assert err < TOL[prec]


BURGERS_FORMS = [(c, k, p) for c, ks in ((TRI, (1, 2, 3)), (TET, (1, 2))) for k in ks
                 for p in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16)]


@pytest.mark.parametrize("cell,k,prec", BURGERS_FORMS)
def test_burgers_block_form_when_forced(cell, k, prec):
    """Component blocks of at most 128 entries have two forms: the block form (every block
    contracted over [T1 | T2 | T3]) and the factored form (T1 against u, P applied in the
    epilogue); each forced by its flag meets the bounds against the oracle."""
    mesh = ragged_mesh(cell, seed=60 + k)
    coef, c2d = coefficients(BURGERS_JAC, mesh, k, seed=61)
    ref = oracle_ref(BURGERS_JAC, k, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    tc = coffee.FLAG_TENSOR_CORES  # P1 would otherwise take the CUDA-core kernel
    blocks = coffee.assemble(BURGERS_JAC, k, cell, x, c2v, cf, cd, precision=prec, validate=True,
                             tune=tc | coffee.FLAG_BURGERS_BLOCKS)
    fact = coffee.assemble(BURGERS_JAC, k, cell, x, c2v, cf, cd, precision=prec, validate=True,
                           tune=tc | coffee.FLAG_BURGERS_FACTORED)
    coffee.check_errors()
    eb = rel_err_per_cell(blocks.cpu().numpy(), ref)
    ef = rel_err_per_cell(fact.cpu().numpy(), ref)
    print("burgers %s P%d %s: blocks %.3e factored %.3e" % ("tri" if cell == TRI else "tet", k,
                                                           coffee.PRECISION_NAMES[prec], eb, ef))
    assert eb < TOL[prec] and ef < TOL[prec]


@pytest.mark.parametrize("ncells", [1, 63, 64, 65, 127, 128, 129, 191, 257])
def test_burgers_factored_tile_edges(ncells):
    """64-cell tiles in pairs: single tiles, odd tile counts and ragged last tiles; nothing
    written past the last cell."""
    mesh = meshgen.tet_mesh(4, perturb=0.15, seed=62, ncells=ncells)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, seed=63)
    ref = oracle_ref(BURGERS_JAC, 2, TET, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = torch.full((ncells + 2, 30, 30), 7.0, dtype=torch.float32, device=DEV)
    coffee.assemble(BURGERS_JAC, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3, out=out[:ncells])
    torch.cuda.synchronize()
    coffee.check_errors()
    assert rel_err_per_cell(out[:ncells].cpu().numpy(), ref) < 1e-5
    assert torch.all(out[ncells:] == 7.0)


@pytest.mark.parametrize("ncells", [1, 127, 128, 129, 255, 257])
def test_tile_edges(ncells):
    mesh = meshgen.tet_mesh(4, perturb=0.15, seed=3, ncells=ncells)
    ref = oracle_ref(HELMHOLTZ, 3, TET, mesh, None, None)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = torch.full((ncells + 3, 20, 20), 7.0, dtype=torch.float32, device=DEV)
    coffee.assemble(HELMHOLTZ, 3, TET, x, c2v, precision=coffee.TF32X3, out=out[:ncells])
    torch.cuda.synchronize()
    assert rel_err_per_cell(out[:ncells].cpu().numpy(), ref) < 1e-5
    assert torch.all(out[ncells:] == 7.0)  # nothing written past the last cell


def test_empty_input_is_noop():
    mesh = meshgen.tet_mesh(2, seed=3)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 2, TET, x, c2v[:0], precision=coffee.TF32X3)
    assert out.shape == (0, 10, 10)


def test_sliver_cells_take_fp64_geometry():
    rng = np.random.default_rng(5)
    X = np.concatenate([meshgen.sliver_tet(rng, flat) for flat in (1e-1, 1e-2, 1e-3, 1e-4)])
    c2v = np.arange(16, dtype=np.int32).reshape(4, 4)
    mesh = meshgen.Mesh(TET, X, c2v, None, (1, 1, 1))
    ref = oracle_ref(HELMHOLTZ, 2, TET, mesh, None, None)
    x, cv, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 2, TET, x, cv, precision=coffee.TF32X3)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


def test_validation_flags_bad_index_tc():
    mesh = meshgen.tet_mesh(3, seed=4)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    bad = c2v.clone()
    bad[17, 1] = -3
    coffee.assemble(MASS, 2, TET, x, bad, precision=coffee.TF32X3, validate=True)
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4


def test_permuted_coefficient_numbering_tc():
    mesh = ragged_mesh(TET, seed=8)
    coef, c2d = coefficients(ADVDIFF, mesh, 2, seed=8, permute_seed=77)
    ref = oracle_ref(ADVDIFF, 2, TET, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(ADVDIFF, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3)
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_full_size_config2_tc_sampled(k):
    """1,572,864 Kuhn tets, Helmholtz Pk in TF32X3, in the launch configuration the
    benchmark times: sampled cells vs the oracle, plus the mesh's total mass."""
    mesh = meshgen.tet_mesh(64, perturb=0.15, seed=2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, k, TET, x, c2v, precision=coffee.TF32X3)
    sel = np.random.default_rng(k).choice(mesh.ncells, size=2000, replace=False)
    sel = np.concatenate([sel, [0, mesh.ncells - 1]])
    ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None, sel=sel)
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy()
    assert rel_err_per_cell(got, ref) < 1e-5
    del out
    m = coffee.assemble(MASS, k, TET, x, c2v, precision=coffee.TF32X3)
    assert abs(m.double().sum().item() - 1.0) < 1e-5


def test_config3_advdiff_p2_2pow20_sampled():
    mesh = meshgen.tet_mesh(64, 64, 43, perturb=0.15, seed=3, ncells=2 ** 20)
    coef, c2d = coefficients(ADVDIFF, mesh, 2, seed=3)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(ADVDIFF, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3)
    sel = np.random.default_rng(3).choice(mesh.ncells, size=3000, replace=False)
    ref = oracle_ref(ADVDIFF, 2, TET, mesh, coef, c2d, sel=sel)
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy()
    assert rel_err_per_cell(got, ref) < 1e-5
    # A 1 = 0 on every cell (both terms vanish on constants)
    rows = out.double().sum(dim=2).abs().amax(dim=1) / out.double().abs().amax(dim=(1, 2))
    assert rows.max().item() < 1e-5


def test_config3_burgers_p2_2pow20_sampled():
    """2^20 Kuhn tets, vector P2 Burgers Jacobian (nu = 0.01, u ~ N(0,1)) in TF32X3:
    sampled cells vs the oracle."""
    mesh = meshgen.tet_mesh(64, 64, 43, perturb=0.15, seed=3, ncells=2 ** 20)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, seed=3)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(BURGERS_JAC, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3)
    assert out.shape == (2 ** 20, 30, 30)
    sel = np.random.default_rng(4).choice(mesh.ncells, size=2000, replace=False)
    sel = np.concatenate([sel, [mesh.ncells - 1]])
    ref = oracle_ref(BURGERS_JAC, 2, TET, mesh, coef, c2d, sel=sel)
    got = out[torch.from_numpy(sel).to(DEV)].cpu().numpy()
    assert rel_err_per_cell(got, ref) < 1e-5


def test_burgers_permuted_numbering_tc():
    mesh = ragged_mesh(TET, seed=9)
    coef, c2d = coefficients(BURGERS_JAC, mesh, 2, seed=9, permute_seed=5)
    ref = oracle_ref(BURGERS_JAC, 2, TET, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    out = coffee.assemble(BURGERS_JAC, 2, TET, x, c2v, cf, cd, precision=coffee.TF32X3, validate=True)
    coffee.check_errors()
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("form,cell,k", [(HELMHOLTZ, TET, 3), (HELMHOLTZ, TET, 1), (ADVDIFF, TET, 2),
                                         (MASS, TRI, 2), (HELMHOLTZ, TET, 4), (BURGERS_JAC, TET, 2)])
def test_tuning_knobs_give_identical_results(form, cell, k):
    """The autotuner's knobs (cells or outputs on the TMEM lanes, operand stages) change
    only speed: every setting writes bit-identical element matrices."""
    mesh = ragged_mesh(cell, seed=60 + k)
    coef, c2d = coefficients(form, mesh, k, seed=61)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    outs = [coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=coffee.TF32X3, tune=t)
            for t in (0, coffee.FLAG_OUTPUT_LANES, coffee.FLAG_TWO_STAGES,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_TWO_STAGES,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_SUBTILE_64,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_SUBTILE_32,
                      coffee.FLAG_SUBTILE_128, coffee.FLAG_CELL_LANES,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_STAGED_STORE,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_STAGED_STORE | coffee.FLAG_SUBTILE_32,
                      coffee.FLAG_OUTPUT_LANES | coffee.FLAG_STAGED_STORE | coffee.FLAG_TWO_STAGES)]
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("k,ncells", [(4, 1), (4, 3), (4, 5), (4, 127), (4, 130), (4, 1000), (2, 131), (2, 1000),
                                      (3, 133)])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3])
def test_staged_rows_ragged_tails(k, ncells, prec):
    """Staged epilogue (rows of 8 or 32 consecutive cells gathered in shared memory, whole groups
    of four rows written by one bulk copy, the ragged last rows by plain stores): equal to the
    direct warp stores bit for bit, within the bound of the oracle, and nothing written past the
    last cell, for cell counts that end mid-group, mid-tile and mid-sub-tile."""
    mesh = meshgen.tet_mesh(6, perturb=0.15, seed=70 + k, ncells=ncells)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    n = coffee.ndof(HELMHOLTZ, k, TET)
    outs = []
    for t in (coffee.FLAG_OUTPUT_LANES, coffee.FLAG_OUTPUT_LANES | coffee.FLAG_STAGED_STORE):
        buf = torch.full((ncells + 5, n, n), 7.0, dtype=torch.float32, device=DEV)
        coffee.assemble(HELMHOLTZ, k, TET, x, c2v, precision=prec, out=buf[:ncells], tune=t)
        torch.cuda.synchronize()
        assert torch.all(buf[ncells:] == 7.0)
        outs.append(buf[:ncells])
    assert torch.equal(outs[0], outs[1])
    ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None)
    assert rel_err_per_cell(outs[1].cpu().numpy(), ref) < TOL[prec]


def test_split_coords_are_hi_lo_float_pairs():
    """coffee_split_coords: for 2^-70 <= |x| < 2^100, hi is x with the 29 fraction bits below a
    float's 24 significant bits cleared and lo the float rounding of x - hi (exact in FP64);
    outside that range hi = (float)x, lo = (float)(x - hi); either way hi + lo holds x to 2^-48
    of |x| where lo stays a normal float (2^-100 <= |x| < 2^127)."""
    mesh = meshgen.tet_mesh(5, perturb=0.15, seed=80)
    rng = np.random.default_rng(81)
    extra = np.concatenate([
        [0.0, -0.0, 1.0, -1.0, 2.0 ** -70, -(2.0 ** -70), 2.0 ** 100 * (1 - 2.0 ** -53), 2.0 ** 100, -(2.0 ** 100),
         2.0 ** -71, 1e-30, -1e-35, 1e35, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -25, 1.0 - 2.0 ** -53],
        rng.standard_normal(64) * 10.0 ** rng.integers(-25, 28, 64)])
    x64 = np.concatenate([mesh.coords.ravel(), extra])
    x = torch.from_numpy(x64).to(DEV)
    s = coffee.split_coords(x).double().cpu().numpy().reshape(-1, 2)
    assert s.shape == (x64.size, 2)
    inr = (np.abs(x64) >= 2.0 ** -70) & (np.abs(x64) < 2.0 ** 100)
    hi_t = (x64.view(np.uint64) & ~np.uint64((1 << 29) - 1)).view(np.float64)
    hi = np.where(inr, hi_t, x64.astype(np.float32).astype(np.float64))
    hi[x64 == 0] = 0.0
    np.testing.assert_array_equal(s[:, 0], hi)
    np.testing.assert_array_equal(s[:, 1], (x64 - hi).astype(np.float32).astype(np.float64))
    normal = (np.abs(x64) >= 2.0 ** -100) & (np.abs(x64) < 2.0 ** 127)
    assert (normal | (x64 == 0)).sum() > x64.size - 8
    err = np.abs((s[:, 0] - x64) + s[:, 1])  # s0 - x is exact: no rounding in the check itself
    assert np.all(err[normal] <= 2.0 ** -48 * np.abs(x64[normal]))
    # odd counts and pointers off the 16-byte boundary take the one-value-per-thread path
    s1 = coffee.split_coords(x[1:]).double().cpu().numpy().reshape(-1, 2)
    np.testing.assert_array_equal(s1, s[1:])
    buf = torch.empty(2 * x64.size + 2, dtype=torch.float32, device=DEV)
    coffee.split_coords(x, out=buf[2:])
    np.testing.assert_array_equal(buf[2:].double().cpu().numpy().reshape(-1, 2), s)
    with pytest.raises(RuntimeError):
        coffee.split_coords(x, out=buf[1:-1])  # 4-byte offset: not a float pair boundary


SPLIT_CASES = [(f, c, k, p) for f in (MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC) for c in (TRI, TET)
               for k in (1, 2, 4) for p in (coffee.TF32X3, coffee.BF16X3, coffee.BF16)]


@pytest.mark.parametrize("form,cell,k,prec", SPLIT_CASES)
def test_split_coordinates_match_oracle(form, cell, k, prec):
    """The Jacobian's vertex differences taken in FP32 from the (hi, lo) float pairs of the
    coordinates: same bounds against the oracle as the FP64 differences."""
    if not coffee.supported(form, k, cell, prec):
        pytest.skip("combination not built")
    mesh = ragged_mesh(cell, seed=90 + k)
    coef, c2d = coefficients(form, mesh, k, seed=9)
    ref = oracle_ref(form, k, cell, mesh, coef, c2d)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    xs = coffee.split_coords(x)
    out = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True, coords_split=xs)
    coffee.check_errors()
    err = rel_err_per_cell(out.cpu().numpy(), ref)
    print("split coords %s %s P%d %s: %.3e" % (coffee.FORM_NAMES[form], "tri" if cell == TRI else "tet", k,
                                               coffee.PRECISION_NAMES[prec], err))
    assert err < TOL[prec]


def test_round_coef_is_the_float_rounding():
    """coffee_round_coef: every coefficient as (float)coef, bit for bit (ties to even, carries into
    the exponent, overflow to infinity, results below the normal range, zeros, infinities, NaN),
    also for odd lengths and a start that is not 16-byte aligned (the scalar loop)."""
    rng = np.random.default_rng(81)
    u = 2.0 ** -24
    fmax = float(np.finfo(np.float32).max)
    edge = np.array([1 + u, 1 + 3 * u, 1 + u + 2.0 ** -52, 1 + u - 2.0 ** -52, 2 - u, 2 - u / 2, 2 - 2 * u,
                     fmax, fmax * (1 + u / 2), fmax * (1 + u / 2) * (1 - 2.0 ** -52), fmax * (1 + u),
                     2.0 ** 127 * (2 - 2.0 ** -30), 2.0 ** 128, 1e39, 2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -30),
                     2.0 ** -127, 1e-40, 1e-45, 1e-50, 2.0 ** -1074, 0.0, np.inf, np.nan, 0.1, 1 / 3])
    edge = np.concatenate([edge, -edge])
    c = torch.from_numpy(np.concatenate([rng.standard_normal(100001) * 10.0 ** rng.integers(-30, 30, 100001),
                                         edge])).to(DEV)
    for v in (c, c[1:], c[2:]):
        r = coffee.round_coef(v)
        assert torch.equal(r.view(torch.int32), v.float().view(torch.int32))


COEF_CASES = ([(f, c, k, p) for f in (ADVDIFF, BURGERS_JAC, coffee.BURGERS_RESIDUAL) for c in (TRI, TET)
               for k in (1, 2, 3, 4) for p in (coffee.TF32X3, coffee.BF16)]
              + [(ADVDIFF, coffee.PRISM, k, coffee.TF32X3) for k in (1, 2, 4)])


@pytest.mark.parametrize("form,cell,k,prec", COEF_CASES)
def test_float_coefficients_give_the_same_bits(form, cell, k, prec):
    """The coefficients read from their float copy (round_coef) instead of converted in the kernel:
    every kernel that reads coefficients (advection-diffusion factors, the Burgers Jacobian in its
    resident and streamed kernels, the residual, prisms) gives the same bits."""
    if not coffee.supported(form, k, cell, prec):
        pytest.skip("combination not built")
    if cell == coffee.PRISM:
        mesh = meshgen.prism_mesh(6, 4, perturb=0.15, seed=82)
        coef, c2d, _ = meshgen.advdiff_coefficients(mesh, 84)
    else:
        mesh = ragged_mesh(cell, seed=83 + k)
        coef, c2d = coefficients(BURGERS_JAC if form == coffee.BURGERS_RESIDUAL else form, mesh, k, seed=84)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    a = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True)
    b = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, validate=True,
                        coef_f32=coffee.round_coef(cf))
    coffee.check_errors()
    assert torch.equal(a, b)


def test_split_coordinates_sliver_cells_and_full_size():
    """Badly conditioned cells fall back to FP64 from the FP64 coordinates with the split given too;
    the 1,572,864-tet Helmholtz P1 and P2 meshes with split coordinates, sampled against the oracle."""
    rng = np.random.default_rng(5)
    X = np.concatenate([meshgen.sliver_tet(rng, flat) for flat in (1e-1, 1e-2, 1e-3, 1e-4)])
    c2v = np.arange(16, dtype=np.int32).reshape(4, 4)
    sl = meshgen.Mesh(TET, X, c2v, None, (1, 1, 1))
    ref = oracle_ref(HELMHOLTZ, 2, TET, sl, None, None)
    x, cv, _, _ = to_device(sl, None, None, DEV)
    out = coffee.assemble(HELMHOLTZ, 2, TET, x, cv, precision=coffee.TF32X3, coords_split=coffee.split_coords(x))
    assert rel_err_per_cell(out.cpu().numpy(), ref) < 1e-5
    mesh = meshgen.tet_mesh(64, perturb=0.15, seed=2)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    xs = coffee.split_coords(x)
    sel = np.concatenate([np.random.default_rng(11).choice(mesh.ncells, size=1000, replace=False),
                          [0, mesh.ncells - 1]])
    for k in (1, 2):
        out = coffee.assemble(HELMHOLTZ, k, TET, x, c2v, precision=coffee.TF32X3, coords_split=xs)
        ref = oracle_ref(HELMHOLTZ, k, TET, mesh, None, None, sel=sel)
        assert rel_err_per_cell(out[torch.from_numpy(sel).to(DEV)].cpu().numpy(), ref) < 1e-5
