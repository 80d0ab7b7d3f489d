"""Padded output rows (coffee_assemble_args.out_stride): every element matrix starts out_stride
entries after the previous one, the padding is left untouched, and the entries are bit for bit
those of the contiguous layout (the same kernel writes them; only the row addresses differ).
Covers the tensor-core kernel in both epilogue orientations, the CUDA-core kernel and the FP64
kernel, a stride that is a multiple of 32 entries (128-byte rows) and an odd one (no vector
stores), ragged last tiles. The argument checks run without a GPU."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, coefficients, to_device

DEV = "cuda:0"
CASES = [(HELMHOLTZ, TET, 4, coffee.TF32X3, 0), (HELMHOLTZ, TET, 2, coffee.TF32X3, 0),
         (HELMHOLTZ, TET, 2, coffee.TF32X3, coffee.FLAG_CELL_LANES), (ADVDIFF, TET, 3, coffee.TF32X3, 0),
         (MASS, TRI, 4, coffee.BF16X3, 0), (HELMHOLTZ, TET, 1, coffee.TF32X3, coffee.FLAG_TENSOR_CORES),
         (HELMHOLTZ, TET, 1, coffee.TF32X3, coffee.FLAG_CUDA_CORES), (ADVDIFF, TRI, 2, coffee.TF32X3, 0),
         (HELMHOLTZ, TET, 3, coffee.FP64, 0), (ADVDIFF, TRI, 1, coffee.FP64, 0)]


@pytest.mark.gpu
@pytest.mark.parametrize("form,cell,k,prec,tune", CASES)
@pytest.mark.parametrize("pad", ["line", "odd"])
def test_padded_rows_equal_contiguous_rows(form, cell, k, prec, tune, pad):
    mesh = (meshgen.tet_mesh(6, perturb=0.15, seed=90, ncells=1001) if cell == TET
            else meshgen.tri_mesh(23, perturb=0.2, seed=90))
    coef, c2d = coefficients(form, mesh, k, seed=91)
    x, c2v, cf, cd = to_device(mesh, coef, c2d, DEV)
    n = coffee.ndof(form, k, cell)
    N = n * n
    stride = (N + 31) // 32 * 32 if pad == "line" else N + 3
    if stride == N:
        stride += 32
    ref = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, tune=tune)
    odt = torch.float64 if prec == coffee.FP64 else torch.float32
    buf = torch.full((mesh.ncells, stride), 7.0, dtype=odt, device=DEV)
    got = coffee.assemble(form, k, cell, x, c2v, cf, cd, precision=prec, tune=tune, out=buf, out_stride=stride)
    torch.cuda.synchronize()
    coffee.check_errors()
    assert got.shape == ref.shape and torch.equal(got, ref)
    assert torch.all(buf[:, N:] == 7.0)  # padding untouched


def _args(form, degree, cell, stride, prec=coffee.TF32X3):
    a = coffee.binding.AssembleArgs()
    a.form, a.degree, a.cell, a.precision, a.nu = form, degree, cell, prec, 0.01
    # non-NULL placeholders: the checks reject the call before any pointer is used
    a.coords = a.cell2vert = a.out = a.coef = a.cell2dof = 0x1000
    a.nverts, a.ncells, a.ncoefnodes = 10, 4, 10
    a.out_stride = stride
    return a


@pytest.mark.parametrize("form,degree,cell,stride", [
    (HELMHOLTZ, 2, TET, 99),                     # below ndof^2 = 100
    (BURGERS_JAC, 2, TET, 1024),                 # padded rows only for MASS/HELMHOLTZ/ADVDIFF
    (coffee.BURGERS_RESIDUAL, 2, TET, 64),
    (HELMHOLTZ, 2, coffee.PRISM, 400)])
def test_out_stride_argument_checks(form, degree, cell, stride):
    a = _args(form, degree, cell, stride)
    assert coffee.lib().coffee_assemble_ex(ctypes.byref(a), None) == -1
    assert b"out_stride" in coffee.lib().coffee_last_error()


def test_out_stride_equal_to_the_matrix_size_is_the_contiguous_layout():
    # accepted by the checks (then stopped by the NULL out pointer before any launch)
    a = _args(BURGERS_JAC, 2, TET, 900)
    a.out = None
    assert coffee.lib().coffee_assemble_ex(ctypes.byref(a), None) == -1
    assert b"out_stride" not in coffee.lib().coffee_last_error()


def test_host_path_rejects_out_stride():
    a = _args(HELMHOLTZ, 2, TET, 128)
    f = coffee.lib().coffee_assemble_host
    f.argtypes = [ctypes.POINTER(coffee.binding.AssembleArgs), ctypes.c_int, ctypes.c_void_p]
    assert f(ctypes.byref(a), 1, None) == -1
    assert b"out_stride" in coffee.lib().coffee_last_error()
