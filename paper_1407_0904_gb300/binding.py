"""Python binding of libcoffee.so (ctypes): argument marshalling only.

Every step of local assembly runs inside the library's CUDA kernels; this module
checks tensor dtypes/devices, passes raw device pointers and the current CUDA stream
through the C ABI declared in include/coffee.h, and turns status codes into
exceptions. There is no CPU fallback: if the library is missing the calls raise.
"""
import ctypes
import os

import numpy as np
import torch

MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC = 0, 1, 2, 3
BURGERS_RESIDUAL = 4  # element vectors [ncells, d*ns] of the residual whose Jacobian is BURGERS_JAC
TRIANGLE, TETRAHEDRON, PRISM = 0, 1, 2
FP64, TF32, TF32X3, BF16, BF16X3 = 0, 1, 2, 3, 4
FLAG_VALIDATE = 1
FLAG_OUTPUT_LANES = 2   # tuning knob: element-matrix entries on the TMEM lanes
FLAG_TWO_STAGES = 4     # tuning knob: at most two operand stages
FLAG_SUBTILE_64 = 8     # tuning knob: 64 cells per TMEM accumulator
FLAG_SUBTILE_32 = 16    # tuning knob: 32 cells per TMEM accumulator
FLAG_SUBTILE_128 = 32   # tuning knob: 128 cells per TMEM accumulator
FLAG_CELL_LANES = 64    # tuning knob: cells on the TMEM lanes (element matrices <= 128 entries)
FLAG_STAGED_STORE = 256  # tuning knob: rows staged in shared memory, written by bulk copies
FLAG_TENSOR_CORES = 512  # small element matrices: force the tcgen05 kernel
FLAG_CUDA_CORES = 1024   # small element matrices: force the FP32 CUDA-core kernel
FLAG_BURGERS_BLOCKS = 2048    # Burgers Jacobian: the block form (every block over [T1|T2|T3])
FLAG_BURGERS_FACTORED = 4096  # Burgers Jacobian: the factored form (T1 against u, P in the epilogue)

FORM_NAMES = {MASS: "mass", HELMHOLTZ: "helmholtz", ADVDIFF: "advdiff", BURGERS_JAC: "burgers_jac",
              BURGERS_RESIDUAL: "burgers_residual"}
PRECISION_NAMES = {FP64: "fp64", TF32: "tf32", TF32X3: "tf32x3", BF16: "bf16", BF16X3: "bf16x3"}

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcoffee.so")
_lib = None


class CoffeeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("coffee status %d: %s" % (status, msg))
        self.status = status


class AssembleArgs(ctypes.Structure):
    _fields_ = [
        ("form", ctypes.c_int), ("degree", ctypes.c_int), ("cell", ctypes.c_int),
        ("precision", ctypes.c_int), ("nu", ctypes.c_double),
        ("coords", ctypes.c_void_p), ("nverts", ctypes.c_int64),
        ("cell2vert", ctypes.c_void_p),
        ("coef", ctypes.c_void_p), ("ncoefnodes", ctypes.c_int64),
        ("cell2dof", ctypes.c_void_p),
        ("out", ctypes.c_void_p), ("ncells", ctypes.c_int64),
        ("flags", ctypes.c_uint),
        ("coords_split", ctypes.c_void_p),
        ("coef_f32", ctypes.c_void_p),
        ("out_stride", ctypes.c_int64),
    ]


def lib():
    """Load libcoffee.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcoffee.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, L64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.coffee_ndof.argtypes = [I, I, I]
        L.coffee_tabulate.argtypes = [I, I, I, P, P, P, P, P, P]
        L.coffee_reference_tensor.argtypes = [I, I, I, P, P, P]
        L.coffee_assemble.argtypes = [I, I, I, P, P, P, P, P, L64, P]
        L.coffee_assemble_ex.argtypes = [ctypes.POINTER(AssembleArgs), P]
        L.coffee_assemble_backward.argtypes = [ctypes.POINTER(AssembleArgs), P, P, P, I, P]
        L.coffee_check_errors.argtypes = [P]
        L.coffee_supported.argtypes = [I, I, I, I]
        L.coffee_split_coords.argtypes = [P, L64, P, P]
        L.coffee_round_coef.argtypes = [P, L64, P, P]
        L.coffee_assemble_path.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint]
        L.coffee_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise CoffeeError(rc, lib().coffee_last_error().decode())
    return rc


def dim(cell):
    return 2 if cell == TRIANGLE else 3


def verts_per_cell(cell):
    return {TRIANGLE: 3, TETRAHEDRON: 4, PRISM: 6}[cell]


def ndof(form, degree, cell):
    n = lib().coffee_ndof(form, degree, cell)
    if n < 0:
        _check(n)
    return n


def supported(form, degree, cell, precision):
    """True if the library has a kernel for this (form, degree, cell, precision)."""
    return bool(lib().coffee_supported(form, degree, cell, precision))


def csr_supported(form, degree, cell, precision):
    """True if the fused global assembly has a kernel for this combination."""
    L = lib()
    L.coffee_csr_supported.argtypes = [ctypes.c_int] * 4
    return bool(L.coffee_csr_supported(form, degree, cell, precision))


def tc_available(form, degree, cell, precision):
    return precision != FP64 and supported(form, degree, cell, precision)


def nnodes(cell, degree):
    return ndof(MASS, degree, cell)


def tabulate(cell, degree, quad_degree):
    """Quadrature rule and Lagrange basis on the reference cell (host, FP64).

    Returns (points [nq,d], weights [nq], basis [nq,ndof], grads [nq,ndof,d])."""
    L = lib()
    nq, nd = ctypes.c_int(), ctypes.c_int()
    _check(L.coffee_tabulate(cell, degree, quad_degree, ctypes.byref(nq), ctypes.byref(nd),
                             None, None, None, None))
    d = dim(cell)
    pts = np.zeros((nq.value, d))
    wts = np.zeros(nq.value)
    phi = np.zeros((nq.value, nd.value))
    grd = np.zeros((nq.value, nd.value, d))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(L.coffee_tabulate(cell, degree, quad_degree, None, None, p(pts), p(wts), p(phi), p(grd)))
    return pts, wts, phi, grd


def reference_tensor(form, degree, cell):
    """Reference tensors T [K, ns*ns] (host, FP64)."""
    L = lib()
    K, N = ctypes.c_int(), ctypes.c_int()
    _check(L.coffee_reference_tensor(form, degree, cell, ctypes.byref(K), ctypes.byref(N), None))
    T = np.zeros((K.value, N.value))
    _check(L.coffee_reference_tensor(form, degree, cell, None, None, T.ctypes.data_as(ctypes.c_void_p)))
    return T


def diag_wait_timeout(stream=None):
    """Enqueue the diagnostic wait that runs out (coffee_diag_wait_timeout); the next
    check_errors() raises CoffeeError with COFFEE_ERR_TIMEOUT."""
    L = lib()
    L.coffee_diag_wait_timeout.argtypes = [ctypes.c_void_p]
    _check(L.coffee_diag_wait_timeout(_stream_handle(stream)))


def peak_fp64():
    """Measured FP64 FMA rate of the current GPU in TFLOP/s (coffee_peak_fp64)."""
    L = lib()
    L.coffee_peak_fp64.argtypes = [ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    _check(L.coffee_peak_fp64(ctypes.byref(v)))
    return v.value


def peak_mma(precision=TF32, n=256):
    """Measured tcgen05 MMA rate (M=128, N=n, one 32-byte K-step per instruction) in TFLOP/s
    for precision TF32 (kind::tf32) or BF16 (kind::f16) (coffee_peak_mma)."""
    L = lib()
    L.coffee_peak_mma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    _check(L.coffee_peak_mma(int(precision), int(n), ctypes.byref(v)))
    return v.value


def _dev(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def coef_width(form, degree, cell):
    """Columns of cell2dof for a form: the cell's vertices for ADVDIFF (P1 eps and b), the
    scalar Pk nodes for the Burgers forms (u), 0 for forms without a coefficient."""
    if form == ADVDIFF:
        return verts_per_cell(cell)
    if form in (BURGERS_JAC, BURGERS_RESIDUAL):
        return nnodes(cell, degree)
    return 0


def check_shapes(form, degree, cell, coords, cell2vert, coef=None, cell2dof=None):
    """Shape checks of the inputs against the layouts of include/coffee.h, made before any
    pointer is passed: the library receives bare pointers and cannot check extents."""
    d = dim(cell)
    nv = verts_per_cell(cell)
    if cell2vert.dim() != 2 or cell2vert.shape[1] != nv:
        raise ValueError("cell2vert must be [ncells, %d]" % nv)
    if coords.dim() != 2 or coords.shape[1] != d:
        raise ValueError("coords must be [nverts, %d]" % d)
    w = coef_width(form, degree, cell)
    if w == 0:
        return
    if coef is None or cell2dof is None:
        return  # the library rejects the missing pointers itself
    if cell2dof.dim() != 2 or cell2dof.shape[0] != cell2vert.shape[0] or cell2dof.shape[1] != w:
        raise ValueError("cell2dof must be [ncells, %d] = [%d, %d], got %s"
                         % (w, cell2vert.shape[0], w, list(cell2dof.shape)))
    row = 1 + d if form == ADVDIFF else d
    if coef.numel() % row != 0:
        raise ValueError("coef must be [ncoefnodes, %d]" % row)


def split_coords(coords, out=None, stream=None):
    """coffee_split_coords: every coordinate as a float pair (hi, lo) with hi + lo = x to 2^-48 |x|
    (hi: x truncated to 24 significant bits, lo: the rest rounded to a float; for |x| outside
    [2^-70, 2^100) hi = (float)x, lo = (float)(x - hi)), a float32 tensor [nverts, d, 2] on the
    device: the coords_split input of assemble, with which the kernels take the Jacobian's vertex
    differences in FP32 without splitting each vertex again for every cell that uses it."""
    coords = _dev(coords, torch.float64, "coords")
    if out is None:
        out = torch.empty(tuple(coords.shape) + (2,), dtype=torch.float32, device=coords.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != 2 * coords.numel():
            raise ValueError("out must hold 2 floats per coordinate")
    _check(lib().coffee_split_coords(_ptr(coords), ctypes.c_int64(coords.numel()), _ptr(out),
                                     _stream_handle(stream)))
    return out


PATH_NAMES = {0: "fp64", 1: "tensor cores", 2: "cuda cores fp32"}


def assemble_path(form, degree, cell, precision, flags=0):
    """coffee_assemble_path: 0 the FP64 kernel, 1 the tensor cores, 2 the FP32 CUDA-core kernel."""
    r = lib().coffee_assemble_path(form, degree, cell, precision, int(flags))
    if r < 0:
        _check(r)
    return r


def round_coef(coef, out=None, stream=None):
    """coffee_round_coef: every coefficient rounded to the nearest float, a float32 tensor of coef's
    shape on the device: the coef_f32 input of assemble, read by the tensor-core kernels instead
    of converting each coefficient once per cell that uses it (same results bit for bit)."""
    coef = _dev(coef, torch.float64, "coef")
    if out is None:
        out = torch.empty(tuple(coef.shape), dtype=torch.float32, device=coef.device)
    else:
        _dev(out, torch.float32, "out")
        if out.numel() != coef.numel():
            raise ValueError("out must hold one float per coefficient")
    _check(lib().coffee_round_coef(_ptr(coef), ctypes.c_int64(coef.numel()), _ptr(out),
                                   _stream_handle(stream)))
    return out


def make_args(form, degree, cell, coords, cell2vert, coef=None, cell2dof=None, precision=FP64,
              out=None, nu=0.01, validate=False, ncoefnodes=None, tune=0, alloc_out=True, coords_split=None,
              coef_f32=None, out_stride=0):
    coords = _dev(coords, torch.float64, "coords")
    cell2vert = _dev(cell2vert, torch.int32, "cell2vert")
    coef = _dev(coef, torch.float64, "coef")
    cell2dof = _dev(cell2dof, torch.int32, "cell2dof")
    check_shapes(form, degree, cell, coords, cell2vert, coef, cell2dof)
    d = dim(cell)
    ncells = cell2vert.shape[0]
    n = ndof(form, degree, cell)
    odt = torch.float64 if precision == FP64 else torch.float32
    shape = (ncells, n) if form == BURGERS_RESIDUAL else (ncells, n, n)  # element vectors or matrices
    if out_stride:
        # padded rows: out is the flat buffer [ncells, out_stride] (see assemble)
        if out is None:
            if alloc_out:
                out = torch.empty((ncells, out_stride), dtype=odt, device=coords.device)
        else:
            _dev(out, odt, "out")
            if ncells and out.numel() < (ncells - 1) * out_stride + int(np.prod(shape[1:])):
                raise ValueError("out must hold (ncells - 1) * out_stride + %d elements" % int(np.prod(shape[1:])))
    elif out is None:
        if alloc_out:
            out = torch.empty(shape, dtype=odt, device=coords.device)
    else:
        _dev(out, odt, "out")
        if out.numel() != int(np.prod(shape)):
            raise ValueError("out must hold %s elements" % "x".join(map(str, shape)))
    if ncoefnodes is None and coef is not None:
        ncoefnodes = coef.numel() // (1 + d) if form == ADVDIFF else coef.numel() // d
    a = AssembleArgs()
    a.form, a.degree, a.cell, a.precision, a.nu = form, degree, cell, precision, nu
    a.coords, a.nverts = _ptr(coords), coords.shape[0]
    a.cell2vert = _ptr(cell2vert)
    a.coef, a.ncoefnodes = _ptr(coef), int(ncoefnodes or 0)
    a.cell2dof = _ptr(cell2dof)
    a.out, a.ncells = _ptr(out), ncells
    a.flags = (FLAG_VALIDATE if validate else 0) | int(tune)
    if coords_split is not None:
        _dev(coords_split, torch.float32, "coords_split")
        if coords_split.numel() != 2 * coords.numel():
            raise ValueError("coords_split must hold 2 floats per coordinate (split_coords)")
    a.coords_split = _ptr(coords_split)
    if coef_f32 is not None:
        _dev(coef_f32, torch.float32, "coef_f32")
        if coef is None or coef_f32.numel() != coef.numel():
            raise ValueError("coef_f32 must hold one float per coefficient of coef (round_coef)")
    a.coef_f32 = _ptr(coef_f32)
    a.out_stride = int(out_stride or 0)
    return a, out


def assemble(form, degree, cell, coords, cell2vert, coef=None, cell2dof=None, precision=FP64,
             out=None, nu=0.01, validate=False, stream=None, tune=None, coords_split=None, coef_f32=None,
             out_stride=None):
    """Element matrices [ncells, ndof, ndof] (float64 for FP64, float32 otherwise) on the device.

    tune: FLAG_OUTPUT_LANES / FLAG_TWO_STAGES knobs; None uses the autotuner's choice for
    this (form, degree, cell, precision) when one is cached, else the library default.
    coords_split: the (hi, lo) float pairs of coords (split_coords), optional.
    coef_f32: coef rounded to floats (round_coef), optional.
    out_stride: entries between consecutive element matrices (padded rows, e.g. a multiple of 32
    so that every matrix starts on a 128-byte line); out is then the flat buffer of ncells rows of
    out_stride entries (allocated when None), and the result is the strided view
    [ncells, ndof, ndof] of it. The padding is not written."""
    if tune is None:
        tune = _tuned_flags(form, degree, cell, precision)
    a, out = make_args(form, degree, cell, coords, cell2vert, coef, cell2dof, precision, out, nu,
                       validate, tune=tune, coords_split=coords_split, coef_f32=coef_f32,
                       out_stride=out_stride or 0)
    _check(lib().coffee_assemble_ex(ctypes.byref(a), _stream_handle(stream)))
    if out_stride:
        n = ndof(form, degree, cell)
        return out.as_strided((cell2vert.shape[0], n, n), (int(out_stride), n, 1))
    return out


_tune_cache = None


def _tuned_flags(form, degree, cell, precision):
    """Knobs chosen by the autotuner (paper_1407_0904_gb300.tune) for this GPU; without a tuned
    entry, the tuner's cost model chooses them from the element-matrix shape."""
    global _tune_cache
    if precision == FP64 or form in (BURGERS_JAC, BURGERS_RESIDUAL):
        return 0
    from . import tune as _tune
    if _tune_cache is None:
        try:
            _tune_cache = _tune.load_cache()
        except (OSError, ValueError):
            _tune_cache = {}
    ent = _tune_cache.get("%d/%d/%d/%d" % (form, degree, cell, precision))
    if ent is not None:
        return int(ent.get("flags", 0))
    return _tune.model_flags(ndof(form, degree, cell) ** 2,
                             assemble_path(form, degree, cell, precision, FLAG_CUDA_CORES) == 2)


def assemble_plain(form, degree, cell, coords, cell2vert, coef=None, cell2dof=None, out=None,
                   stream=None):
    """coffee_assemble, the plain-argument FP64 entry point (nu = 0.01)."""
    coords = _dev(coords, torch.float64, "coords")
    cell2vert = _dev(cell2vert, torch.int32, "cell2vert")
    coef = _dev(coef, torch.float64, "coef")
    cell2dof = _dev(cell2dof, torch.int32, "cell2dof")
    n = ndof(form, degree, cell)
    ncells = cell2vert.shape[0]
    if out is None:
        out = torch.empty((ncells, n, n), dtype=torch.float64, device=coords.device)
    _check(lib().coffee_assemble(form, degree, cell, _ptr(coords), _ptr(cell2vert), _ptr(coef),
                                 _ptr(cell2dof), _ptr(out), ncells, _stream_handle(stream)))
    return out


def check_errors(stream=None):
    """Synchronise the stream and raise if a kernel flagged an error."""
    _check(lib().coffee_check_errors(_stream_handle(stream)))


def _host(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def assemble_host(form, degree, cell, coords, cell2vert, coef=None, cell2dof=None, precision=FP64,
                  out=None, nu=0.01, chunks=4, device=None, validate=False, tune=None):
    """Local assembly from HOST tensors into a host tensor (coffee_assemble_host).

    The library copies the coordinates and coefficients to the device once, assembles the
    cells in `chunks` launches and copies each chunk's results back on its own stream while
    the next chunk computes (page-locked tensors let the copies overlap). Returns the host
    tensor `out` (allocated page-locked if None); it is complete once the current CUDA stream
    of `device` has reached this point."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    coords = _host(coords, torch.float64, "coords")
    cell2vert = _host(cell2vert, torch.int32, "cell2vert")
    coef = _host(coef, torch.float64, "coef")
    cell2dof = _host(cell2dof, torch.int32, "cell2dof")
    check_shapes(form, degree, cell, coords, cell2vert, coef, cell2dof)
    ncells = cell2vert.shape[0]
    n = ndof(form, degree, cell)
    odt = torch.float64 if precision == FP64 else torch.float32
    shape = (ncells, n) if form == BURGERS_RESIDUAL else (ncells, n, n)
    if out is None:
        out = torch.empty(shape, dtype=odt, pin_memory=True)
    else:
        _host(out, odt, "out")
        if out.numel() != int(np.prod(shape)):
            raise ValueError("out must hold %s elements" % "x".join(map(str, shape)))
    if tune is None:
        tune = _tuned_flags(form, degree, cell, precision)
    d = dim(cell)
    a = AssembleArgs()
    a.form, a.degree, a.cell, a.precision, a.nu = form, degree, cell, precision, nu
    a.coords, a.nverts = _ptr(coords), coords.shape[0]
    a.cell2vert = _ptr(cell2vert)
    a.coef = _ptr(coef)
    a.ncoefnodes = 0 if coef is None else coef.numel() // ((1 + d) if form == ADVDIFF else d)
    a.cell2dof = _ptr(cell2dof)
    a.out, a.ncells = _ptr(out), ncells
    a.flags = (FLAG_VALIDATE if validate else 0) | int(tune)
    L = lib()
    L.coffee_assemble_host.argtypes = [ctypes.POINTER(AssembleArgs), ctypes.c_int, ctypes.c_void_p]
    with torch.cuda.device(dev):
        _check(L.coffee_assemble_host(ctypes.byref(a), int(chunks), _stream_handle(None)))
    return out


def host_pool_trim():
    """Release the device staging memory kept by assemble_host's pool (coffee_host_pool_trim)."""
    _check(lib().coffee_host_pool_trim())


def assemble_backward(form, degree, cell, coords, cell2vert, dout, coef=None, cell2dof=None,
                      precision=FP64, d_coords=None, d_coef=None, deterministic=False,
                      validate=False, nu=0.01, stream=None):
    """Adjoint of assemble: accumulates dL/dcoords (and dL/dcoef) for dout = dL/dA.

    dout is float64 for precision FP64 and float32 otherwise. Returns (d_coords, d_coef);
    tensors passed in are accumulated into (+=), missing ones start at zero."""
    odt = torch.float64 if precision == FP64 else torch.float32
    a, _ = make_args(form, degree, cell, coords, cell2vert, coef, cell2dof, precision,
                     _dev(dout, odt, "dout"), nu, validate)
    if d_coords is None:
        d_coords = torch.zeros_like(coords)
    _dev(d_coords, torch.float64, "d_coords")
    if coef is not None and form == ADVDIFF:
        if d_coef is None:
            d_coef = torch.zeros_like(coef)
        _dev(d_coef, torch.float64, "d_coef")
    else:
        d_coef = None
    _check(lib().coffee_assemble_backward(ctypes.byref(a), _ptr(dout), _ptr(d_coords), _ptr(d_coef),
                                          1 if deterministic else 0, _stream_handle(stream)))
    return d_coords, d_coef


class AssembleFn(torch.autograd.Function):
    """Element matrices as a differentiable function of vertex coordinates and coefficients.

    AssembleFn.apply(coords, coef, cell2vert, cell2dof, form, degree, cell, precision,
    deterministic) -> [ncells, ndof, ndof]; backward gives dL/dcoords and dL/dcoef through
    the library's adjoint kernel (geometry recomputed, not stored)."""

    @staticmethod
    def forward(ctx, coords, coef, cell2vert, cell2dof, form, degree, cell, precision=FP64,
                deterministic=False):
        out = assemble(form, degree, cell, coords, cell2vert, coef, cell2dof, precision=precision)
        ctx.save_for_backward(coords, coef, cell2vert, cell2dof)
        ctx.meta = (form, degree, cell, precision, deterministic)
        return out

    @staticmethod
    def backward(ctx, dout):
        coords, coef, c2v, c2d = ctx.saved_tensors
        form, degree, cell, precision, deterministic = ctx.meta
        dc, dk = assemble_backward(form, degree, cell, coords, c2v, dout.contiguous(), coef, c2d,
                                   precision=precision, deterministic=deterministic)
        return dc, dk, None, None, None, None, None, None, None


def assemble_backward_noalloc(form, degree, cell, coords, cell2vert, dout, coef=None, cell2dof=None,
                              precision=FP64, d_coords=None, d_coef=None, stream=None):
    """The allocation-free adjoint (coffee_assemble_backward_noalloc): the same result as
    assemble_backward(..., deterministic=True) without any device allocation inside the
    library; at most 16384 cells and 16384 vertices / coefficient nodes."""
    L = lib()
    L.coffee_assemble_backward_noalloc.argtypes = [ctypes.POINTER(AssembleArgs), ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    odt = torch.float64 if precision == FP64 else torch.float32
    a, _ = make_args(form, degree, cell, coords, cell2vert, coef, cell2dof, precision,
                     _dev(dout, odt, "dout"), 0.01, False)
    if d_coords is None:
        d_coords = torch.zeros_like(coords)
    if coef is not None and form == ADVDIFF and d_coef is None:
        d_coef = torch.zeros_like(coef)
    _check(L.coffee_assemble_backward_noalloc(ctypes.byref(a), _ptr(dout), _ptr(d_coords),
                                              _ptr(d_coef if form == ADVDIFF else None),
                                              _stream_handle(stream)))
    return d_coords, (d_coef if form == ADVDIFF else None)


def batch_split(costs, grid):
    """The CTA split of a mixed batch (coffee_batch_split, host-only): ranges [grid+1] int64,
    CTA b taking work items [ranges[b], ranges[b+1]) of about equal total cost."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    r = np.zeros(int(grid) + 1, dtype=np.int64) if int(grid) >= 1 else np.zeros(1, dtype=np.int64)
    L = lib()
    L.coffee_batch_split.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    _check(L.coffee_batch_split(c.ctypes.data_as(ctypes.c_void_p), c.size, int(grid),
                                r.ctypes.data_as(ctypes.c_void_p)))
    return r


class BatchPlan:
    """Several (form, degree, cell) groups assembled by one persistent tensor-core launch, plus
    one CUDA-core launch for the groups of small element matrices that run there by default
    (P1 simplices, P2 triangles), unless all_tensor_cores.

    groups: list of dicts with keys form, degree, cell, coords, cell2vert and optionally
    coef, cell2dof, out, coords_split (split_coords of coords), coef_f32 (round_coef of coef).
    All groups use `precision`
    (a tensor-core precision).
    launch() only enqueues the plan's kernels (`launches` of them) on the current stream
    (CUDA-graph capturable).

    Work is split over the CTAs by cost. costs="measured" (default) takes each group's time
    per 128-cell tile from the autotuner's cache for this GPU (coffee_batch_plan_costs) and
    falls back to the byte model (bytes written + item_overhead per 128-output slice,
    coffee_batch_plan) when a group is not in the cache; costs="bytes" forces the byte
    model; a list gives one tile cost per group."""

    def __init__(self, groups, precision=TF32X3, grid=0, item_overhead=-1.0, validate=False,
                 costs="measured", all_tensor_cores=False):
        L = lib()
        L.coffee_batch_plan.argtypes = [ctypes.POINTER(AssembleArgs), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]
        L.coffee_batch_plan_costs.argtypes = [ctypes.POINTER(AssembleArgs), ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)]
        L.coffee_batch_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.coffee_batch_free.argtypes = [ctypes.c_void_p]
        self._keep = []
        self.outputs = []
        arr = (AssembleArgs * len(groups))()
        for i, g in enumerate(groups):
            a, out = make_args(g["form"], g["degree"], g["cell"], g["coords"], g["cell2vert"],
                               g.get("coef"), g.get("cell2dof"), precision, g.get("out"),
                               g.get("nu", 0.01), validate, coords_split=g.get("coords_split"),
                               coef_f32=g.get("coef_f32"),
                               tune=FLAG_TENSOR_CORES if (all_tensor_cores and i == 0) else 0)
            arr[i] = a
            self.outputs.append(out)
            self._keep.append((g["coords"], g["cell2vert"], g.get("coef"), g.get("cell2dof"), out,
                               g.get("coords_split"), g.get("coef_f32")))
        if item_overhead is None or item_overhead < 0:
            try:
                from . import tune as _tune
                item_overhead = float(_tune.load_batch().get("item_overhead", -1.0))
            except Exception:
                item_overhead = -1.0
        simt = [not all_tensor_cores and assemble_path(g["form"], g["degree"], g["cell"], precision) == 2
                for g in groups]
        self.launches = int(any(simt)) + int(not all(simt))
        if isinstance(costs, str):
            costs = self.measured_costs(groups, precision) if costs == "measured" else None
        self.costs = costs
        self._plan = ctypes.c_void_p()
        if costs is not None:
            c = (ctypes.c_double * len(groups))(*[float(x) for x in costs])
            _check(L.coffee_batch_plan_costs(arr, len(groups), grid, c, ctypes.byref(self._plan)))
        else:
            _check(L.coffee_batch_plan(arr, len(groups), grid, item_overhead, ctypes.byref(self._plan)))

    @staticmethod
    def measured_costs(groups, precision):
        """Per-group cost of a 128-cell tile from the autotuner's cache for this GPU: the batch
        kernel's own time per tile for that group shape (tune --batch-tiles) when every group has
        one, else the group's tuned single-group kernel time per tile; None if neither covers
        every group."""
        try:
            from . import tune as _tune
            entries = _tune.load_cache() or {}
            tiles = _tune.load_batch().get("tile_ms", {}) if entries else {}
        except Exception:
            return None
        keys = ["%d/%d/%d/%d" % (g["form"], g["degree"], g["cell"], precision) for g in groups]
        if all(tiles.get(k, 0) > 0 for k in keys):
            return [float(tiles[k]) for k in keys]
        out = []
        for k in keys:
            ent = entries.get(k)
            if not ent or not ent.get("ms") or not ent.get("ncells"):
                return None
            out.append(float(ent["ms"]) * 128.0 / float(ent["ncells"]))
        return out

    def launch(self, stream=None):
        _check(lib().coffee_batch_launch(self._plan, _stream_handle(stream)))
        return self.outputs

    def free(self):
        if self._plan:
            lib().coffee_batch_free(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- global assembly
def vector_l2g(cell2dof, nnodes, d):
    """Component-blocked local-to-global map of a d-vector field on the nodes of cell2dof:
    [ncells, d*ns] with entry (e, c*ns + i) = c*nnodes + cell2dof[e, i]."""
    return torch.cat([cell2dof + c * nnodes for c in range(d)], dim=1).contiguous()


def csr_map_len(ncells, nloc):
    """Length of the blocked entry map: cells padded to 32, entries padded to a multiple of 4."""
    return (ncells + 31) // 32 * 32 * ((nloc * nloc + 3) // 4 * 4)


def csr_map_unblock(m, ncells, nloc):
    """[ncells, nloc*nloc] uint32 NumPy view of a blocked entry map (host copy; for inspection):
    block (cb, ob) = [32 cells][width] at 32*(cb*npad + 32*ob), width = min(32, npad - 32*ob)."""
    m = (m.cpu().numpy() if isinstance(m, torch.Tensor) else np.asarray(m)).view(np.uint32)
    n2 = nloc * nloc
    npad = (n2 + 3) // 4 * 4
    e = np.arange(ncells)[:, None]
    idx = np.arange(n2)[None, :]
    ob = idx // 32
    bw = np.minimum(32, npad - ob * 32)
    return m[32 * ((e // 32) * npad + 32 * ob) + (e % 32) * bw + idx % 32]


def sparsity(l2g, nrows, stream=None):
    """CSR sparsity of the global matrix of the map l2g [ncells, nloc] (int32, CUDA):
    (rowptr int64 [nrows+1], colidx int32 [nnz]), columns ascending in each row."""
    l2g = _dev(l2g, torch.int32, "l2g")
    if l2g.dim() != 2:
        raise ValueError("l2g must be [ncells, nloc]")
    L = lib()
    L.coffee_sparsity.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    ncells, nloc = l2g.shape
    rowptr = torch.empty(nrows + 1, dtype=torch.int64, device=l2g.device)
    nnz = ctypes.c_int64(0)
    st = _stream_handle(stream)
    _check(L.coffee_sparsity(_ptr(l2g), ncells, nloc, nrows, _ptr(rowptr), None, ctypes.byref(nnz), st))
    colidx = torch.empty(nnz.value, dtype=torch.int32, device=l2g.device)
    if nnz.value:
        _check(L.coffee_sparsity(_ptr(l2g), ncells, nloc, nrows, _ptr(rowptr), _ptr(colidx), None, st))
    return rowptr, colidx


def csr_map(l2g, rowptr, colidx, stream=None):
    """Position in colidx of every element-matrix entry, blocked as the fused kernels read it
    (see csr_map_len / csr_map_unblock): uint32 values held in a flat int32 tensor (reinterpret;
    entries >= 2^31 read as negative); padding entries are 0xffffffff."""
    l2g = _dev(l2g, torch.int32, "l2g")
    rowptr = _dev(rowptr, torch.int64, "rowptr")
    colidx = _dev(colidx, torch.int32, "colidx")
    L = lib()
    L.coffee_csr_map.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    ncells, nloc = l2g.shape
    m = torch.empty(csr_map_len(ncells, nloc), dtype=torch.int32, device=l2g.device)
    _check(L.coffee_csr_map(_ptr(l2g), ncells, nloc, _ptr(rowptr), _ptr(colidx), rowptr.numel() - 1, _ptr(m),
                            _stream_handle(stream)))
    return m


def assemble_csr(form, degree, cell, coords, cell2vert, csr_map_, vals, coef=None, cell2dof=None,
                 precision=FP64, nu=0.01, validate=False, stream=None, tune=0):
    """Fused global assembly: vals[map[e, o]] += A_e[o] over all cells (vals float64 for FP64,
    float32 otherwise; zero it first for a new matrix). Returns vals."""
    odt = torch.float64 if precision == FP64 else torch.float32
    vals = _dev(vals, odt, "vals")
    csr_map_ = _dev(csr_map_, torch.int32, "map")
    n = ndof(form, degree, cell)
    if csr_map_.numel() != csr_map_len(cell2vert.shape[0], n):
        raise ValueError("map must hold csr_map_len(ncells, ndof) entries")
    a, _ = make_args(form, degree, cell, coords, cell2vert, coef, cell2dof, precision, None, nu, validate,
                     tune=tune, alloc_out=False)
    L = lib()
    L.coffee_assemble_csr.argtypes = [ctypes.POINTER(AssembleArgs), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p]
    _check(L.coffee_assemble_csr(ctypes.byref(a), _ptr(csr_map_), _ptr(vals), vals.numel(),
                                 _stream_handle(stream)))
    return vals


class CsrMatrix:
    """Global sparse matrix of one local-to-global map: pattern and entry map built once
    (setup), then assembled any number of times by the fused kernels."""

    def __init__(self, l2g, nrows, stream=None):
        self.l2g = _dev(l2g, torch.int32, "l2g")
        self.nrows = int(nrows)
        self.rowptr, self.colidx = sparsity(self.l2g, self.nrows, stream)
        self.map = csr_map(self.l2g, self.rowptr, self.colidx, stream)

    @property
    def nnz(self):
        return self.colidx.numel()

    def assemble(self, form, degree, cell, coords, cell2vert, coef=None, cell2dof=None, precision=FP64,
                 vals=None, nu=0.01, validate=False, stream=None, tune=0):
        """Values [nnz] of the assembled global matrix (vals, if given, is added into)."""
        if vals is None:
            vals = torch.zeros(self.nnz, dtype=torch.float64 if precision == FP64 else torch.float32,
                               device=self.l2g.device)
        return assemble_csr(form, degree, cell, coords, cell2vert, self.map, vals, coef, cell2dof, precision,
                            nu, validate, stream, tune)

    def to_torch(self, vals):
        """torch sparse CSR tensor of the values (shares the pattern)."""
        return torch.sparse_csr_tensor(self.rowptr, self.colidx, vals, size=(self.nrows, self.nrows))
