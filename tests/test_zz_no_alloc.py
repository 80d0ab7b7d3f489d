"""The allocation-free adjoint (coffee_assemble_backward_noalloc).

Callers that cannot allocate device memory while they run (latency-critical loops that
must not call cudaMalloc/cudaFree, applications whose device memory belongs to their own
allocator, fixed-budget deployments) use this entry point; it keeps its scratch in a
fixed device array inside the library. These tests call it through the C ABI: two calls in
a row must give, bit for bit, what the allocating deterministic adjoint gives (same kernels,
same summation order), and match the oracle's gradient; a device-side index error must
reach coffee_check_errors. The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TET, TRI, MASS, HELMHOLTZ, ADVDIFF, coefficients, to_device

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _entry():
    f = coffee.lib().coffee_assemble_backward_noalloc
    f.argtypes = [ctypes.POINTER(coffee.binding.AssembleArgs), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return f


def _call(a, dout, dx, dc):
    return _entry()(ctypes.byref(a), ctypes.c_void_p(dout.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                    None if dc is None else ctypes.c_void_p(dc.data_ptr()),
                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# (form, cell, degree, precision of dout, whether d_coef is requested)
CASES = [(ADVDIFF, TET, 2, coffee.FP64, True), (HELMHOLTZ, TRI, 3, coffee.FP64, False),
         (MASS, TET, 1, coffee.FP64, False), (ADVDIFF, TET, 4, coffee.FP64, True),
         (ADVDIFF, TET, 2, coffee.FP64, False), (HELMHOLTZ, TET, 2, coffee.TF32X3, False),
         (ADVDIFF, TRI, 3, coffee.TF32X3, True)]


@pytest.mark.parametrize("form,cell,k,prec,with_coef", CASES)
def test_noalloc_adjoint_equals_allocating_adjoint_twice(form, cell, k, prec, with_coef):
    mesh = (meshgen.tet_mesh(6, perturb=0.15, seed=41, ncells=1000) if cell == TET
            else meshgen.tri_mesh(20, perturb=0.2, seed=41))
    coef, c2d = coefficients(form, mesh, k, seed=42)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    n = coffee.ndof(form, k, cell)
    odt = torch.float64 if prec == coffee.FP64 else torch.float32
    g = torch.Generator(device=DEV).manual_seed(43)
    dout = torch.randn((mesh.ncells, n, n), dtype=odt, device=DEV, generator=g)
    ref_x, ref_c = coffee.assemble_backward(form, k, cell, x, c2v, dout, cf, cd, precision=prec,
                                            deterministic=True)
    if not with_coef:
        ref_c = None
    gx, gc = oracle.assemble_backward(form, k, cell, mesh.coords, mesh.cell2vert,
                                      dout.double().cpu().numpy(), coef, c2d)
    for _ in range(2):  # the second call starts from the first call's leftover scratch
        a, _ = coffee.binding.make_args(form, k, cell, x, c2v, cf, cd, prec, dout)
        dx = torch.zeros_like(x)
        dc = torch.zeros_like(cf) if with_coef else None
        rc = _call(a, dout, dx, dc)
        assert rc == 0, coffee.lib().coffee_last_error()
        coffee.check_errors()
        assert torch.equal(dx, ref_x)
        if with_coef:
            assert torch.equal(dc, ref_c)
        # against the oracle: 1e-10 for FP64 dL/dA; the FP32 arithmetic of the float dout path
        # (the tensor-core precisions) is held to 1e-5
        tol = 1e-10 if prec == coffee.FP64 else 1e-5
        assert rel(dx.cpu().numpy(), gx) < tol
        if with_coef:
            assert rel(dc.cpu().numpy(), gc) < tol


def test_noalloc_adjoint_reports_an_out_of_range_index():
    """A cell that names vertex nverts (the caller passes one vertex fewer than the coordinate
    array holds, so every read stays inside the buffers): the per-node summation skips the index
    and flags it, and coffee_check_errors reports it once; the next check is clean."""
    mesh = meshgen.tet_mesh(4, perturb=0.15, seed=45)
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    last = mesh.coords.shape[0] - 1
    assert (mesh.cell2vert == last).any()
    dout = torch.ones((mesh.ncells, 4, 4), dtype=torch.float64, device=DEV)
    a, _ = coffee.binding.make_args(HELMHOLTZ, 1, TET, x, c2v, None, None, coffee.FP64, dout)
    a.nverts = last  # vertex `last` is now out of range for the summation, not for the reads
    dx = torch.zeros_like(x)
    assert _call(a, dout, dx, None) == 0, coffee.lib().coffee_last_error()
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4
    coffee.check_errors()  # cleared
    assert torch.count_nonzero(dx[last]) == 0


def test_noalloc_adjoint_rejects_inputs_beyond_its_scratch():
    mesh = meshgen.tet_mesh(16, perturb=0.15, seed=44)  # 24576 cells > 16384
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    dout = torch.zeros((mesh.ncells, 4, 4), dtype=torch.float64, device=DEV)
    a, _ = coffee.binding.make_args(HELMHOLTZ, 1, TET, x, c2v, None, None, coffee.FP64, dout)
    dx = torch.zeros_like(x)
    assert _call(a, dout, dx, None) == -1
    assert b"16384" in coffee.lib().coffee_last_error()
    assert torch.count_nonzero(dx) == 0
