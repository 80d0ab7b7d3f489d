"""The allocation-free adjoint (coffee_assemble_backward_noalloc).

Callers that cannot allocate device memory while they run (latency-critical loops that
must not call cudaMalloc/cudaFree, applications whose device memory belongs to their own
allocator, fixed-budget deployments) use this entry point; it keeps its scratch in a
fixed device array inside the library. These tests call it through the C ABI and check
that two calls in a row give what the allocating deterministic adjoint gives. The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TET, TRI, HELMHOLTZ, ADVDIFF, coefficients, to_device

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-12


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


def _entry():
    f = coffee.lib().coffee_assemble_backward_noalloc
    f.argtypes = [ctypes.POINTER(coffee.binding.AssembleArgs), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return f


@pytest.mark.parametrize("form,cell,k", [(ADVDIFF, TET, 2), (HELMHOLTZ, TRI, 3)])
def test_noalloc_adjoint_matches_allocating_adjoint_twice(form, cell, k):
    mesh = (meshgen.tet_mesh(6, perturb=0.15, seed=41, ncells=1000) if cell == TET
            else meshgen.tri_mesh(20, perturb=0.2, seed=41))
    coef, c2d = coefficients(form, mesh, k, seed=42)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    n = coffee.ndof(form, k, cell)
    g = torch.Generator(device=DEV).manual_seed(43)
    dout = torch.randn((mesh.ncells, n, n), dtype=torch.float64, device=DEV, generator=g)
    ref_x, ref_c = coffee.assemble_backward(form, k, cell, x, c2v, dout, cf, cd, deterministic=True)
    entry = _entry()
    stream = torch.cuda.current_stream()
    for _ in range(2):  # the second call starts from the first call's leftover scratch
        a, _ = coffee.binding.make_args(form, k, cell, x, c2v, cf, cd, coffee.FP64, dout)
        dx = torch.zeros_like(x)
        dc = torch.zeros_like(cf) if cf is not None else None
        rc = entry(ctypes.byref(a), ctypes.c_void_p(dout.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                   None if dc is None else ctypes.c_void_p(dc.data_ptr()),
                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, coffee.lib().coffee_last_error()
        torch.cuda.synchronize()
        assert rel(dx, ref_x) < TOL
        if dc is not None:
            assert rel(dc, ref_c) < TOL


def test_noalloc_adjoint_rejects_inputs_beyond_its_scratch():
    mesh = meshgen.tet_mesh(16, perturb=0.15, seed=44)  # 24576 cells > 16384
    x, c2v, _, _ = to_device(mesh, None, None, DEV)
    dout = torch.zeros((mesh.ncells, 4, 4), dtype=torch.float64, device=DEV)
    a, _ = coffee.binding.make_args(HELMHOLTZ, 1, TET, x, c2v, None, None, coffee.FP64, dout)
    dx = torch.zeros_like(x)
    rc = _entry()(ctypes.byref(a), ctypes.c_void_p(dout.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                  None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"16384" in coffee.lib().coffee_last_error()
    assert torch.count_nonzero(dx) == 0
