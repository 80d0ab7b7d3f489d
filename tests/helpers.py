"""Shared helpers for the parity tests: seeded inputs, device transfer, error metric."""
import numpy as np

import oracle
from paper_1407_0904_gb300 import meshgen

TRI, TET = 0, 1
MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC = 0, 1, 2, 3
FP64, TF32, TF32X3, BF16, BF16X3 = 0, 1, 2, 3, 4

# Parity bounds of every precision, per cell: max_ij |A - A_oracle| / max_ij |A_oracle|.
# FP64 1e-12; the split precisions TF32X3 and BF16X3 1e-5; single-pass TF32 and BF16 1e-2.
TOL = {FP64: 1e-12, TF32X3: 1e-5, BF16X3: 1e-5, TF32: 1e-2, BF16: 1e-2}


def small_mesh(cell, n=None, seed=1):
    if cell == TRI:
        return meshgen.tri_mesh(n or 7, perturb=0.2, seed=seed)
    return meshgen.tet_mesh(n or 3, perturb=0.15, seed=seed)


def coefficients(form, mesh, degree, seed=3, permute_seed=None):
    if form == ADVDIFF:
        coef, c2d, _ = meshgen.advdiff_coefficients(mesh, seed, permute_seed)
        return coef, c2d
    if form == BURGERS_JAC:
        u, c2d, _ = meshgen.burgers_coefficients(mesh, degree, seed, permute_seed)
        return u.ravel(), c2d
    return None, None


def rel_err_per_cell(got, ref):
    """max over cells of max_ij |got - ref| / max_ij |ref| (the benchmark's error metric)."""
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    scale = np.abs(ref).max(axis=1)
    scale[scale == 0] = 1.0
    return float(np.max(np.abs(got - ref).max(axis=1) / scale))


def to_device(mesh, coef, c2d, dev):
    import torch
    t = lambda a, dt: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
    return (t(mesh.coords, torch.float64), t(mesh.cell2vert, torch.int32),
            t(coef, torch.float64), t(c2d, torch.int32))


def oracle_ref(form, degree, cell, mesh, coef, c2d, sel=None):
    if sel is None:
        return oracle.assemble(form, degree, cell, mesh.coords, mesh.cell2vert, coef, c2d, threads=0)
    return oracle.assemble_cells(form, degree, cell, mesh.coords, mesh.cell2vert, sel, coef, c2d, threads=0)
