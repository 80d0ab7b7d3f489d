#!/usr/bin/env python3
"""Benchmark of GB300 local assembly. Default workload: Helmholtz P3 element matrices on
the 64^3 x 6 = 1,572,864-cell perturbed Kuhn mesh, tensor-core form (TF32X3).

One step = one pass of the whole local-assembly path (gather -> geometry ->
contraction -> store) over the whole mesh: one launch of the library's assembly kernel
through the C ABI. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32x3|fp64|...]
                  [--workload helmholtz-p3-tet|advdiff-p2-tet|burgers-p2-tet|...]
  python bench.py --impl reference ...   # the FP64 CPU oracle on bounded samples

Multi-GPU (torchrun): the forward path has no exchange step, so every rank runs an
independent replica of the workload (weak scaling); the time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE = "helmholtz-p3-tet"
METRIC = "Helmholtz P3-tet element matrices/s: TC form vs FP64 kernel, % roofline"
UNIT = "element matrices/s"
L2_BYTES = 129 * 2 ** 20

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# tensor-core kernel on the headline workload, keyed by the sha256 prefix of the kernel
# source it was measured on; reported as null once the source has changed.
# DRAM bytes per launch of the headline kernel (ncu, one launch, full size), by kernel source hash
TRAFFIC = {"64f9c5da8e0a5bb9": 2.4903e9,   # 31.86 MB read + 2.4584 GB written
           "3996a5005b13b753": 2.4902e9}   # 31.86 MB read + 2.4583 GB written

MASS, HELMHOLTZ, ADVDIFF, BURGERS_JAC, BURGERS_RESIDUAL = 0, 1, 2, 3, 4
TRIANGLE, TETRAHEDRON, PRISM = 0, 1, 2
_DEVICE_PEAKS = {}


def device_peaks(coffee):
    """FP64 FMA and tcgen05 MMA rates of this GPU, measured by the library's own loops
    (coffee_peak_fp64 / coffee_peak_mma): the FP64 and tensor-core roofline denominators,
    which the measured-peaks file (copy bandwidth, cuBLAS bf16) does not give."""
    if not _DEVICE_PEAKS:
        _DEVICE_PEAKS.update({
            "fp64_tflops": coffee.peak_fp64(),
            "tf32_tflops": coffee.peak_mma(coffee.TF32, 256),
            "tf32_n128_tflops": coffee.peak_mma(coffee.TF32, 128),
            "bf16_tflops": coffee.peak_mma(coffee.BF16, 256),
            "source": "coffee_peak_fp64 / coffee_peak_mma (M=128, N=256 and 128, one CTA per SM)"})
    return _DEVICE_PEAKS


class Workload:
    """A named benchmark case: form, degree, cell and the seeded synthetic mesh."""

    def __init__(self, name, form, degree, cell, mesh_desc, make):
        self.name, self.form, self.degree, self.cell = name, form, degree, cell
        self.mesh_desc, self._make = mesh_desc, make

    def build(self, nx=None):
        from paper_1407_0904_gb300 import meshgen
        mesh = self._make(meshgen, nx)
        coef = c2d = None
        if self.form == ADVDIFF:
            coef, c2d, _ = meshgen.advdiff_coefficients(mesh, seed=3)
        elif self.form in (BURGERS_JAC, BURGERS_RESIDUAL):
            u, c2d, _ = meshgen.burgers_coefficients(mesh, self.degree, seed=3)
            coef = u.ravel()
        return mesh, coef, c2d


def _kuhn64(mg, nx):
    return mg.tet_mesh(nx or 64, perturb=0.15, seed=2)


def _kuhn2pow20(mg, nx):
    if nx:
        return mg.tet_mesh(nx, perturb=0.15, seed=3)
    return mg.tet_mesh(64, 64, 43, perturb=0.15, seed=3, ncells=2 ** 20)


def _kuhn32(mg, nx):
    return mg.tet_mesh(nx or 32, perturb=0.15, seed=3)


def _prism48(mg, nx):
    return mg.prism_mesh(nx or 48, nx or 48, perturb=0.15, seed=6)


def _prism24(mg, nx):
    return mg.prism_mesh(nx or 24, nx or 24, perturb=0.15, seed=6)


def _tri64(mg, nx):
    return mg.tri_mesh(nx or 64, perturb=0.2, seed=1)


def _tri1024(mg, nx):
    return mg.tri_mesh(nx or 1024, perturb=0.2, seed=1)


WORKLOADS = {}
for _k in (1, 2, 3, 4):
    WORKLOADS["helmholtz-p%d-tet" % _k] = Workload(
        "helmholtz-p%d-tet" % _k, HELMHOLTZ, _k, TETRAHEDRON,
        "64^3x6 Kuhn tets perturbed 0.15h (seed 2)", _kuhn64)
WORKLOADS["advdiff-p2-tet"] = Workload("advdiff-p2-tet", ADVDIFF, 2, TETRAHEDRON,
                                       "Kuhn 64x64x43 truncated to 2^20 tets, perturbed 0.15h (seed 3), "
                                       "eps~U[0.5,1.5], b~U[-1,1]^3 per vertex", _kuhn2pow20)
WORKLOADS["burgers-p1-tet"] = Workload("burgers-p1-tet", BURGERS_JAC, 1, TETRAHEDRON,
                                       "Kuhn 64x64x43 truncated to 2^20 tets, perturbed 0.15h (seed 3), "
                                       "vector P1 u~N(0,1), nu=0.01", _kuhn2pow20)
WORKLOADS["burgers-p2-tet"] = Workload("burgers-p2-tet", BURGERS_JAC, 2, TETRAHEDRON,
                                       "Kuhn 64x64x43 truncated to 2^20 tets, perturbed 0.15h (seed 3), "
                                       "vector P2 u~N(0,1), nu=0.01", _kuhn2pow20)
for _k in (3, 4):
    WORKLOADS["burgers-p%d-tet" % _k] = Workload(
        "burgers-p%d-tet" % _k, BURGERS_JAC, _k, TETRAHEDRON,
        "32^3x6 = 196,608 Kuhn tets perturbed 0.15h (seed 3), vector P%d u~N(0,1), nu=0.01" % _k, _kuhn32)
WORKLOADS["burgers-residual-p2-tet"] = Workload("burgers-residual-p2-tet", BURGERS_RESIDUAL, 2, TETRAHEDRON,
                                                "Kuhn 64x64x43 truncated to 2^20 tets, perturbed 0.15h (seed 3), "
                                                "vector P2 u~N(0,1), nu=0.01; element vectors", _kuhn2pow20)
WORKLOADS["helmholtz-p2-prism"] = Workload("helmholtz-p2-prism", HELMHOLTZ, 2, PRISM,
                                           "unit cube, 48x48 two-triangle columns x 48 layers = 221,184 "
                                           "twisted prisms perturbed 0.15h (seed 6); FP64", _prism48)
WORKLOADS["helmholtz-p3-prism"] = Workload("helmholtz-p3-prism", HELMHOLTZ, 3, PRISM,
                                           "unit cube, 48x48 two-triangle columns x 48 layers = 221,184 "
                                           "twisted prisms perturbed 0.15h (seed 6)", _prism48)
WORKLOADS["helmholtz-p4-prism"] = Workload("helmholtz-p4-prism", HELMHOLTZ, 4, PRISM,
                                           "unit cube, 24x24 two-triangle columns x 24 layers = 27,648 "
                                           "twisted prisms perturbed 0.15h (seed 6)", _prism24)
WORKLOADS["advdiff-p2-prism"] = Workload("advdiff-p2-prism", ADVDIFF, 2, PRISM,
                                         "unit cube, 48x48 two-triangle columns x 48 layers = 221,184 "
                                         "twisted prisms perturbed 0.15h (seed 6), eps~U[0.5,1.5], "
                                         "b~U[-1,1]^3 per vertex", _prism48)
WORKLOADS["burgers-p2-prism"] = Workload("burgers-p2-prism", BURGERS_JAC, 2, PRISM,
                                         "unit cube, 24x24 two-triangle columns x 24 layers = 27,648 "
                                         "twisted prisms perturbed 0.15h (seed 6), vector P2 u~N(0,1) per "
                                         "conforming node, nu=0.01; FP64 only (--precision fp64)", _prism24)
WORKLOADS["burgers-residual-p2-prism"] = Workload("burgers-residual-p2-prism", BURGERS_RESIDUAL, 2, PRISM,
                                                  "unit cube, 24x24 two-triangle columns x 24 layers = 27,648 "
                                                  "twisted prisms perturbed 0.15h (seed 6), vector P2 u~N(0,1) per "
                                                  "conforming node, nu=0.01; element vectors; FP64 only", _prism24)
WORKLOADS["helmholtz-p1-tri"] = Workload("helmholtz-p1-tri", HELMHOLTZ, 1, TRIANGLE,
                                         "unit square 64x64x2 triangles perturbed 0.2h (seed 1)", _tri64)
# the same problem at a size where HBM, not the launch, sets the time (its roofline fraction)
WORKLOADS["helmholtz-p1-tri-1024"] = Workload("helmholtz-p1-tri-1024", HELMHOLTZ, 1, TRIANGLE,
                                              "unit square 1024x1024x2 triangles perturbed 0.2h (seed 1)", _tri1024)


# workloads with their own step (not a single-group forward launch)
SPECIAL = {
    "batch-mixed": "21 (form, degree) groups, Zipf(s=1) counts (seed 4): 2^19 triangles "
                   "(512^2 x 2, P1-P4) + 2^19 Kuhn tets (64x64x22 truncated, P1-P3); mass, "
                   "Helmholtz, advection-diffusion; one persistent launch per step",
    "global-helmholtz-p3-tet": "fused global assembly (CSR) of Helmholtz P3 on 64^3 x 6 = 1,572,864 Kuhn "
                               "tets (seed 2): one step zeroes the CSR values and adds every element matrix "
                               "into them from the tensor-core accumulators; pattern and entry map are set-up",
    "adjoint-helmholtz-p2-tet": "backward of Helmholtz P2 on 2^19 Kuhn tets (64x64x22 truncated, "
                                "seed 5), dL/dA ~ N(0,1), atomic accumulation",
    "adjoint-advdiff-p2-tet": "backward of advection-diffusion P2 on 2^19 Kuhn tets (64x64x22 "
                              "truncated, seed 5), dL/dA ~ N(0,1), atomic accumulation",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS) + sorted(SPECIAL))
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-kernel comparison")
    ap.add_argument("--out-stride", type=int, default=0,
                    help="entries between consecutive element matrices (padded rows; 0 = contiguous). "
                         "-1: the matrix size rounded up to 32 entries (128-byte rows)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tensor-cores", "cuda-cores"],
                    help="small element matrices: force the tcgen05 or the FP32 CUDA-core kernel "
                         "(auto: the library's choice)")
    ap.add_argument("--no-coef-f32", action="store_true",
                    help="tensor-core kernels convert the FP64 coefficients per cell instead of reading the "
                         "float copy that each step rounds once per node")
    ap.add_argument("--coords-split", default="auto", choices=["auto", "on", "off"],
                    help="split the coordinates into float (hi, lo) pairs once per vertex in each step "
                         "(coffee_split_coords, timed with the assembly) and pass them to the kernel; "
                         "auto: on for degree 1 and the residual (many cells per vertex, little work per cell; "
                         "measured faster there, even on P1 triangles, slower on the tensor-core P2 matrices)")
    ap.add_argument("--graph", default="auto", choices=["auto", "on", "off"],
                    help="replay each timed step as a CUDA graph captured once (auto: when a step launches "
                         "more than one kernel, so that host time between the launches is not timed)")
    ap.add_argument("--nx", type=int, default=None, help="smaller mesh (cells per axis) for profiling")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_over_ranks(x, world, op, device=None):
    """Max or sum of a float over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def out_entries(wl, ndof):
    """Entries written per cell: the element vector (residual) or the element matrix."""
    return ndof if wl.form == BURGERS_RESIDUAL else ndof * ndof


def alg_bytes_per_cell(wl, mesh, c2d, coef, ndof, out_bytes):
    """Algorithmic HBM bytes per cell: every input once, plus the element matrix (or vector)."""
    d = 2 if wl.cell == TRIANGLE else 3
    b = 4 * mesh.nvc + 8 * d * mesh.nverts / mesh.ncells + out_bytes * out_entries(wl, ndof)
    if c2d is not None:
        b += 4 * c2d.shape[1] + 8 * coef.size / mesh.ncells
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "power_w_max": float(max(pw)) if pw else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def kernel_source_sha():
    h = hashlib.sha256()
    for name in ("k_tc.cu", "k_tc_kernel.cuh", "tc_common.cuh"):
        with open(os.path.join(ROOT, "paper_1407_0904_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def oracle_cells(wl, mesh, coef, c2d, sel, threads=0):
    import oracle
    if wl.cell == PRISM and wl.form in (BURGERS_JAC, BURGERS_RESIDUAL):
        return oracle.prism_burgers(wl.degree, mesh.coords, mesh.cell2vert[sel], coef.reshape(-1, 3), c2d[sel],
                                    residual=wl.form == BURGERS_RESIDUAL, threads=threads)
    if wl.cell == PRISM:
        extra = (coef, c2d[sel]) if wl.form == ADVDIFF else ()
        return oracle.prism_assemble(wl.form, wl.degree, mesh.coords, mesh.cell2vert[sel], *extra, threads=threads)
    if wl.form == BURGERS_RESIDUAL:
        d = 2 if wl.cell == TRIANGLE else 3
        return oracle.burgers_residual(wl.degree, wl.cell, mesh.coords, mesh.cell2vert[sel], coef.reshape(-1, d),
                                       c2d[sel])
    return oracle.assemble_cells(wl.form, wl.degree, wl.cell, mesh.coords, mesh.cell2vert, sel,
                                 coef, c2d, threads=threads)


def cpu_baseline(wl, mesh, coef, c2d, target_seconds):
    """The FP64 oracle, as it stands, on a bounded prefix of the same workload."""
    import oracle
    threads = oracle.threads_available()
    pilot = np.arange(min(2048, mesh.ncells), dtype=np.int64)
    t0 = time.perf_counter()
    oracle_cells(wl, mesh, coef, c2d, pilot, threads)
    per = (time.perf_counter() - t0) / len(pilot)
    n = int(min(mesh.ncells, max(len(pilot), target_seconds / max(per, 1e-9))))
    sel = np.arange(n, dtype=np.int64)
    t0 = time.perf_counter()
    oracle_cells(wl, mesh, coef, c2d, sel, threads)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first %d of %d cells of the same mesh (FP64 oracle, OpenMP over cells, %.1f s)"
                      % (n, mesh.ncells, dt)}


def metric_of(wl):
    if wl.name == HEADLINE:
        return METRIC
    if wl.form == BURGERS_RESIDUAL:
        return "Burgers residual P%d-%s element vectors/s" % (wl.degree, "tri" if wl.cell == TRIANGLE else "tet")
    return "%s P%d-%s element matrices/s" % (["Mass", "Helmholtz", "Advection-diffusion", "Burgers Jacobian"][wl.form],
                                             wl.degree, ["tri", "tet", "prism"][wl.cell])


def mesh_desc_of(wl, nx, mesh):
    if nx is None:
        return wl.mesh_desc
    return "%d cells (reduced mesh, %d per axis)" % (mesh.ncells, nx)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = WORKLOADS[args.workload]
    mesh, coef, c2d = wl.build(args.nx)
    threads = oracle.threads_available()
    pilot = np.arange(min(2048, mesh.ncells), dtype=np.int64)
    t0 = time.perf_counter()
    oracle_cells(wl, mesh, coef, c2d, pilot, threads)
    per_cell = (time.perf_counter() - t0) / len(pilot)
    # every step is a bounded sample so that warm-up + steps take about two minutes
    budget = min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup))
    n = int(min(mesh.ncells, max(256, budget / max(per_cell, 1e-9))))
    total_cells, total_s = 0, 0.0
    for i in range(args.warmup + args.steps):
        lo = (i * n) % max(1, mesh.ncells - n)
        sel = np.arange(lo, lo + n, dtype=np.int64)
        t0 = time.perf_counter()
        oracle_cells(wl, mesh, coef, c2d, sel, threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            total_cells += n
            total_s += dt
    value = total_cells / total_s
    cpu = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "%d steps of %d consecutive cells of the benchmark mesh (FP64 oracle, OpenMP over "
                     "cells, %.2f s timed)" % (args.steps, n, total_s)}
    line = {"impl": "reference", "metric": metric_of(wl), "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s, %s" % (wl.name, mesh_desc_of(wl, args.nx, mesh)),
                       "ncells": mesh.ncells, "degree": wl.degree},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_1407_0904_gb300 as coffee

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {v: k for k, v in coffee.PRECISION_NAMES.items()}[args.precision]
    wl = WORKLOADS[args.workload]
    form, cell, degree = wl.form, wl.cell, wl.degree
    if not coffee.supported(form, degree, cell, prec):
        raise SystemExit("no kernel for %s in %s" % (wl.name, args.precision))

    # the kernel family the library runs for this workload (the FP32 CUDA-core kernel for small
    # element matrices, where it is faster than the tensor cores)
    force = {"auto": 0, "tensor-cores": coffee.FLAG_TENSOR_CORES, "cuda-cores": coffee.FLAG_CUDA_CORES}[args.kernel]
    tune = None
    if force:
        tune = force | (coffee.binding._tuned_flags(form, degree, cell, prec)
                        & ~(coffee.FLAG_TENSOR_CORES | coffee.FLAG_CUDA_CORES))
    path = coffee.assemble_path(form, degree, cell, prec,
                                tune if tune is not None else coffee.binding._tuned_flags(form, degree, cell, prec))
    mesh, coef_np, c2d_np = wl.build(args.nx)
    ndof = coffee.ndof(form, degree, cell)
    coords = torch.from_numpy(mesh.coords).to(dev)
    c2v = torch.from_numpy(mesh.cell2vert).to(dev)
    coef = None if coef_np is None else torch.from_numpy(coef_np).to(dev)
    c2d = None if c2d_np is None else torch.from_numpy(c2d_np).to(dev)
    ncells = mesh.ncells
    out_bytes = 8 if prec == coffee.FP64 else 4
    odt = torch.float64 if prec == coffee.FP64 else torch.float32
    oshape = (ncells, ndof) if form == BURGERS_RESIDUAL else (ncells, ndof, ndof)
    ostride = args.out_stride if args.out_stride >= 0 else (ndof * ndof + 31) // 32 * 32
    if ostride:
        out = torch.empty((ncells, ostride), dtype=odt, device=dev)  # padded rows
    else:
        out = torch.empty(oshape, dtype=odt, device=dev)
    stream = torch.cuda.current_stream()

    # forms with coefficients: each step rounds them to floats once per node (coffee_round_coef,
    # inside the timed step), and the tensor-core kernel reads that copy
    cf32 = (torch.empty(coef.shape, dtype=torch.float32, device=dev)
            if coef is not None and prec != coffee.FP64 and not args.no_coef_f32 else None)

    # small element matrices: each step also splits every coordinate once per vertex into float
    # (hi, lo) pairs (coffee_split_coords, inside the timed step), from which the kernel takes the
    # Jacobian's vertex differences, instead of splitting each vertex once per cell that uses it
    xsplit = None
    if (prec != coffee.FP64 and cell != PRISM
            and (args.coords_split == "on"
                 or (args.coords_split == "auto" and (degree == 1 or form == BURGERS_RESIDUAL)))):
        xsplit = torch.empty(tuple(coords.shape) + (2,), dtype=torch.float32, device=dev)
    launches_per_step = 1 + (cf32 is not None) + (xsplit is not None)

    def step(precision, o):
        fast = precision != coffee.FP64
        if xsplit is not None and fast:
            coffee.split_coords(coords, out=xsplit)
        if cf32 is not None and fast:
            coffee.round_coef(coef, out=cf32)
        coffee.assemble(form, degree, cell, coords, c2v, coef, c2d, precision=precision, out=o,
                        coef_f32=cf32 if fast else None, out_stride=ostride or None,
                        coords_split=xsplit if fast else None, tune=tune if fast else None)

    # one checked launch before timing (parity against the oracle is the test suite's job)
    step(prec, out)
    coffee.check_errors()

    def capture(fn):
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                fn()
        stream.wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        return g

    # a step of several launches (coordinate split, coefficient rounding, assembly) replays as one
    # CUDA graph: launched one by one from Python, the host time between them is in the step
    run = lambda: step(prec, out)
    step_graph = None
    if args.graph == "on" or (args.graph == "auto" and launches_per_step > 1):
        step_graph = capture(run)
        run = step_graph.replay

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), float(np.mean([a.elapsed_time(b) for a, b in evs]))

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)  # let nvidia-smi start sampling before the timed region
    total_ms, launch_ms = timed(run, args.steps, args.warmup)
    clocks = sampler.stop()
    coffee.check_errors()
    total_ms = reduce_over_ranks(total_ms, world, "max", dev)
    ms_per_step = total_ms / args.steps
    value = reduce_over_ranks(ncells * args.steps, world, "sum", dev) / (total_ms / 1e3)

    # launch-bound sizes (output under 64 MB): the kernel's own rate, from a CUDA graph of 100
    # launches replayed 10 times, so host launch overhead is out of the measurement
    graph = None
    if ncells * out_entries(wl, ndof) * out_bytes < (64 << 20):
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                step(prec, out)
        stream.wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(100):
                step(prec, out)
        g.replay()
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        for _ in range(10):
            g.replay()
        gb.record(stream)
        torch.cuda.synchronize()
        gms = ga.elapsed_time(gb)
        graph = {"launches": 1000, "value": ncells * 1000 / (gms / 1e3), "unit": UNIT,
                 "us_per_launch": gms, "note": "CUDA-graph replay; the step loop above includes host launch cost"}
        del g
        coffee.check_errors()

    # roofline of the dominant (only) kernel: algorithmic bytes per launch / launch time
    per_cell = alg_bytes_per_cell(wl, mesh, c2d_np, coef_np, ndof, out_bytes)
    achieved = per_cell * ncells / (launch_ms / 1e3) / 1e9
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    peak = float(peaks.get("hbm_gbs", 6800.0))
    sha = kernel_source_sha()
    traffic = TRAFFIC.get(sha) if (prec != coffee.FP64 and wl.name == HEADLINE and args.nx is None) else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "alg_bytes_per_cell": per_cell, "kernel_ms": launch_ms}
    if launches_per_step > 1:
        roof["kernel_ms_spans"] = " and ".join(
            ["coffee_split_coords"] * (xsplit is not None) + ["coffee_round_coef"] * (cf32 is not None)
            + ["the assembly kernel (one step)"])
    if prec == coffee.FP64:
        roof["note"] = ("FP64 kernel: bound by the FP64 ALU (%.2f TFLOP/s measured by coffee_peak_fp64); "
                        "HBM fraction for context" % device_peaks(coffee)["fp64_tflops"])
    if cell == PRISM and form in (BURGERS_JAC, BURGERS_RESIDUAL):
        # vector Burgers, evaluated point by point: per point the factors (u, grad u, K: about 12
        # FMAs per node and component set) and, per scalar pair (i, j), 9 FMAs for the component
        # blocks and 12 for the diagonal terms (residual: 12 per node)
        Q = ((3 * degree + 3) // 2) ** 3
        n = ndof // 3
        fma = Q * (12 * n + 60 + (12 * n if form == BURGERS_RESIDUAL else 21 * n * n))
        tf = 2.0 * fma * ncells / (launch_ms / 1e3) / 1e12
        p64 = device_peaks(coffee)["fp64_tflops"]
        roof = {"bound": "alu", "achieved": tf, "peak": p64, "unit": "TFLOP/s", "frac": tf / p64, "traffic": None,
                "peak_source": "FP64 FMA loop measured on this GPU (coffee_peak_fp64)",
                "flops_per_cell": 2.0 * fma, "kernel_ms": launch_ms, "hbm_gbs": achieved}
    elif cell == PRISM:
        # non-affine cells: the contraction over all quadrature points (K = KQ Q) dominates
        Q = (degree + 2) ** 3
        K = Q * {HELMHOLTZ: 7, ADVDIFF: 9}.get(form, 1)
        flops = 2.0 * K * ndof * ndof + 250.0 * Q  # algorithmic, per cell
        if prec == coffee.FP64:
            tf = flops * ncells / (launch_ms / 1e3) / 1e12
            p64 = device_peaks(coffee)["fp64_tflops"]
            roof = {"bound": "alu", "achieved": tf, "peak": p64, "unit": "TFLOP/s",
                    "frac": tf / p64, "traffic": None,
                    "peak_source": "FP64 FMA loop measured on this GPU (coffee_peak_fp64)", "flops_per_cell": flops,
                    "kernel_ms": launch_ms, "hbm_gbs": achieved}
        else:
            # tensor pipe: executed MMA flops (K padded to the 64-byte chunk plus the centre
            # chunk, outputs to 128-row slices, one pass per product of operand parts the
            # precision keeps) against the tf32/bf16 dense peak
            tf32 = prec in (coffee.TF32, coffee.TF32X3)
            kc = 16 if tf32 else 32
            kpad = -(-K // kc) * kc + kc
            npad = -(-(ndof * ndof) // 128) * 128
            passes = {coffee.TF32: 1, coffee.TF32X3: 3, coffee.BF16: 2, coffee.BF16X3: 6}[prec]
            executed = 2.0 * kpad * npad * passes
            if tf32:
                peak_t = device_peaks(coffee)["tf32_tflops"]
                src = "tcgen05 kind::tf32 loop measured on this GPU (coffee_peak_mma, N=256)"
            else:
                peak_t = float(peaks.get("bf16_tflops", 1990.0))
                src = "measured bf16 (cuBLAS)"
            tf = executed * ncells / (launch_ms / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": tf, "peak": peak_t, "unit": "TFLOP/s", "frac": tf / peak_t,
                    "traffic": None, "peak_source": src,
                    "executed_flops_per_cell": executed, "algorithmic_flops_per_cell": flops,
                    "kernel_ms": launch_ms, "hbm_gbs": achieved}

    fp64 = None
    if prec != coffee.FP64 and not args.no_fp64:
        out64 = torch.empty(tuple(out.shape), dtype=torch.float64, device=dev)  # same row layout
        fsteps = max(3, min(args.steps // 20, 100))
        tms, lms = timed(lambda: step(coffee.FP64, out64), fsteps, 3)
        fp64 = {"value": ncells * fsteps / (tms / 1e3), "kernel_ms": lms, "steps": fsteps}
        del out64

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_coords = torch.from_numpy(mesh.coords).pin_memory()
        h_c2v = torch.from_numpy(mesh.cell2vert).pin_memory()
        h_coef = None if coef_np is None else torch.from_numpy(coef_np).pin_memory()
        h_c2d = None if c2d_np is None else torch.from_numpy(c2d_np).pin_memory()
        h_out = torch.empty(oshape, dtype=odt).pin_memory()
        e_steps = max(3, min(args.steps // 20, 50))
        call = lambda: coffee.assemble_host(form, degree, cell, h_coords, h_c2v, h_coef, h_c2d,
                                            precision=prec, out=h_out)
        for _ in range(2):
            call()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e_steps):
            call()
        b.record(stream)
        torch.cuda.synchronize()
        ems = reduce_over_ranks(a.elapsed_time(b), world, "max", dev)
        h2d = h_coords.numel() * 8 + h_c2v.numel() * 4
        if h_coef is not None:
            h2d += h_coef.numel() * 8 + h_c2d.numel() * 4
        e2e = {"value": reduce_over_ranks(ncells * e_steps, world, "sum", dev) / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size())}
        # the host link on this machine: one device-to-host copy of the step's output bytes into the
        # same page-locked buffer, the bound of the end-to-end step
        src = out.reshape(-1)[:h_out.numel()]
        dst = h_out.reshape(-1)
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        cms = a.elapsed_time(b) / 3
        e2e["link"] = {"d2h_gbs": e2e["d2h_bytes_per_step"] / (cms / 1e3) / 1e9, "output_copy_ms": cms,
                       "step_ms": ems / e_steps, "step_over_copy": (ems / e_steps) / cms,
                       "note": "one device-to-host copy of the output bytes, page-locked, CUDA events"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.nx is None:
        cpu = cpu_baseline(wl, mesh, coef_np, c2d_np, args.cpu_seconds)

    if rank == 0:
        line = {"metric": metric_of(wl), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if path == 2 else {"fp64": "f64"}.get(args.precision, args.precision),
                "data": "synthetic",
                "config": {"workload": "%s, %s" % (wl.name, mesh_desc_of(wl, args.nx, mesh)),
                           "ncells": ncells, "degree": degree, "ndof": ndof,
                           "precision": args.precision, "out_dtype": str(odt).replace("torch.", ""),
                           "l2": l2_note(ncells * out_entries(wl, ndof) * out_bytes),
                           "parallelism": "replicas" if world > 1 else "single",
                           "out_layout": ("[ncells][ndof][ndof] contiguous" if not ostride else
                                          "rows padded to %d entries (the padding is not written; the "
                                          "roofline counts the ndof^2 entries only)" % ostride),
                           "kernel": coffee.PATH_NAMES[path] + (" (the faster kernel for this element matrix; "
                                                                 "%s requested)" % args.precision if path == 2 else ""),
                           "coefficients": (None if coef is None else
                                            "rounded to float once per node each step (coffee_round_coef, "
                                            "timed with the assembly)" if cf32 is not None else
                                            "FP64, converted per cell in the kernel"),
                           "launch": ("each step replays a CUDA graph of its %d kernels" % launches_per_step
                                      if step_graph is not None else "each step launched from Python"),
                           "coordinates": ("split into float (hi, lo) pairs once per vertex each step "
                                           "(coffee_split_coords, timed with the assembly)" if xsplit is not None
                                           else "FP64, split per cell in the kernel")},
                "roofline": roof, "fp64_kernel": fp64,
                "tc_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
                "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": args.steps * launches_per_step,
                "clocks": clocks, "kernel_sha": sha, "device_peaks": device_peaks(coffee),
                "graph_replay": graph}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def l2_note(out_bytes):
    if out_bytes > L2_BYTES:
        return "no flush: each step writes %.2f GB of element matrices (> 129 MB L2)" % (out_bytes / 1e9)
    return "output %.2f MB fits in L2: no flush, a latency-bound small case" % (out_bytes / 1e6)


def timed_steps(step, steps, warmup, world, stream):
    """CUDA-event time of `steps` calls of step() after `warmup` untimed ones (ms total, ms per call)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        step()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), float(np.mean([a.elapsed_time(b) for a, b in evs]))


def run_special(args):
    """Config-4 mixed batch and config-5 adjoint workloads."""
    import torch
    import paper_1407_0904_gb300 as coffee
    from paper_1407_0904_gb300 import meshgen
    rank, world, local = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prec = {v: k for k, v in coffee.PRECISION_NAMES.items()}[args.precision]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    global_kernel_ms = None
    if args.workload == "batch-mixed":
        tri = meshgen.tri_mesh(512, perturb=0.2, seed=4)
        tet = meshgen.tet_mesh(64, 64, 22, perturb=0.15, seed=4, ncells=2 ** 19)
        if args.nx:
            tri = meshgen.tri_mesh(args.nx * 4, perturb=0.2, seed=4)
            tet = meshgen.tet_mesh(args.nx, perturb=0.15, seed=4)
        meshes = {}
        for m in (tri, tet):
            coef, c2d, _ = meshgen.advdiff_coefficients(m, seed=4)
            meshes[m.cell] = (m, torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.cell2vert).to(dev),
                              coef, c2d, torch.from_numpy(coef).to(dev), torch.from_numpy(c2d).to(dev))
        groups, specs, per_bytes = [], [], 0.0
        for spec in meshgen.batch_groups(tri, tet, seed=4):
            m, x, c2v, coef, c2d, cf, cd = meshes[spec["cell"]]
            sl = slice(spec["start"], spec["start"] + spec["count"])
            g = dict(form=spec["form"], degree=spec["degree"], cell=spec["cell"], coords=x,
                     cell2vert=c2v[sl].contiguous())
            d = m.dim
            nd = coffee.ndof(spec["form"], spec["degree"], spec["cell"])
            per_bytes += spec["count"] * (4 * (d + 1) + 4 * nd * nd)
            if spec["form"] == ADVDIFF:
                g["coef"], g["cell2dof"] = cf, cd[sl].contiguous()
                per_bytes += spec["count"] * 4 * (d + 1)
            groups.append(g)
            specs.append(spec)
        per_bytes += sum(8 * meshes[c][0].coords.size for c in meshes)
        plan = coffee.BatchPlan(groups, precision=prec)
        ncells = sum(s["count"] for s in specs)
        plan.launch()
        coffee.check_errors()
        step = plan.launch
        kernel = "k_batch_tc + k_simt_batch (small element matrices)" if plan.launches == 2 else "k_batch_tc"
        launches_per_step = plan.launches
        note = None
    elif args.workload == "global-helmholtz-p3-tet":
        k = 3
        mesh = meshgen.tet_mesh(args.nx or 64, perturb=0.15, seed=2)
        c2d, nn = meshgen.cell2dof(mesh, k)
        x = torch.from_numpy(mesh.coords).to(dev)
        c2v = torch.from_numpy(mesh.cell2vert).to(dev)
        M = coffee.CsrMatrix(torch.from_numpy(c2d).to(dev), nn)
        ncells = mesh.ncells
        odt = torch.float64 if prec == coffee.FP64 else torch.float32
        vals = torch.zeros(M.nnz, dtype=odt, device=dev)

        def assemble_only():
            M.assemble(HELMHOLTZ, k, TETRAHEDRON, x, c2v, precision=prec, vals=vals)

        def step():
            vals.zero_()
            assemble_only()

        step()
        coffee.check_errors()
        # the fused kernel alone (accumulating), for the roofline
        _, kernel_ms_alone = timed_steps(assemble_only, 20, 3, world, stream)
        N = c2d.shape[1] ** 2
        per_bytes = ncells * (4 * 4 + 4 * N) + 8 * mesh.coords.size + 2 * M.nnz * vals.element_size()
        kernel = "k_assemble_tc<HELMHOLTZ,tet,%s,CSR>" % args.precision
        launches_per_step = 1
        note = ("roofline of the fused kernel alone (%.4f ms): cell2vert + coords + the uint32 entry map "
                "read once + every CSR value read and written once (nnz = %d); the step adds the zeroing "
                "of the values" % (kernel_ms_alone, M.nnz))
        global_kernel_ms = kernel_ms_alone
    else:
        form = HELMHOLTZ if "helmholtz" in args.workload else ADVDIFF
        mesh = meshgen.tet_mesh(64, 64, 22, perturb=0.15, seed=5, ncells=2 ** 19) if not args.nx else \
            meshgen.tet_mesh(args.nx, perturb=0.15, seed=5)
        coef = c2d = None
        if form == ADVDIFF:
            coef, c2d, _ = meshgen.advdiff_coefficients(mesh, seed=5)
        x = torch.from_numpy(mesh.coords).to(dev)
        c2v = torch.from_numpy(mesh.cell2vert).to(dev)
        cf = None if coef is None else torch.from_numpy(coef).to(dev)
        cd = None if c2d is None else torch.from_numpy(c2d).to(dev)
        ncells = mesh.ncells
        odt = torch.float64 if prec == coffee.FP64 else torch.float32
        g = torch.Generator(device=dev).manual_seed(5)
        dout = torch.randn((ncells, 10, 10), dtype=odt, device=dev, generator=g)
        dx = torch.zeros_like(x)
        dc = None if cf is None else torch.zeros_like(cf)
        step = lambda: coffee.assemble_backward(form, 2, TETRAHEDRON, x, c2v, dout, cf, cd, precision=prec,
                                                d_coords=dx, d_coef=dc)
        per_bytes = ncells * (16 + dout.element_size() * 100) + 8 * mesh.coords.size * 2
        if cf is not None:
            per_bytes += ncells * 16 + 8 * coef.size * 2
        kernel = "k_backward"
        launches_per_step = 1
        note = "adjoint: bound by the FP64 ALU (per cell K*N FP64 FMAs); HBM fraction for context"
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    total_ms, launch_ms = timed_steps(step, args.steps, args.warmup, world, stream)
    clocks = sampler.stop()
    if args.workload == "global-helmholtz-p3-tet":
        launch_ms = global_kernel_ms
    coffee.check_errors()
    total_ms = reduce_over_ranks(total_ms, world, "max", dev)
    value = reduce_over_ranks(ncells * args.steps, world, "sum", dev) / (total_ms / 1e3)
    achieved = per_bytes / (launch_ms / 1e3) / 1e9
    if rank == 0:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_step": per_bytes, "kernel_ms": launch_ms, "kernel": kernel}
        if note:
            roof["note"] = note
        line = {"metric": SPECIAL[args.workload].split(",")[0] + " cells/s", "value": value, "unit": "cells/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64"}.get(args.precision, args.precision), "data": "synthetic",
                "config": {"workload": "%s: %s" % (args.workload, SPECIAL[args.workload]), "ncells": ncells,
                           "precision": args.precision, "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roof, "e2e": None, "cpu_baseline": None,
                "gpu_launches": args.steps * launches_per_step, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload in SPECIAL:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the CPU reference arm covers the "
                              "single-group workloads"}))
            return 0
        return run_special(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
