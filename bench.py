#!/usr/bin/env python3
"""Benchmark: Helmholtz P3 element matrices on 1,572,864 perturbed Kuhn tetrahedra.

One step = one pass of the whole local-assembly path (gather -> geometry ->
contraction -> store) over the whole mesh, i.e. one launch of the library's
assembly kernel through the C ABI. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32x3|fp64|...]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Multi-GPU (torchrun): the forward path has no exchange step, so every rank runs an
independent replica of the workload (weak scaling); timing is max over ranks.
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

METRIC = "Helmholtz P3-tet element matrices/s: TC form vs FP64 kernel, % roofline"
UNIT = "element matrices/s"
NX = 64            # 64^3 cubes x 6 Kuhn tets = 1,572,864 cells
DEGREE = 3
PERTURB = 0.15
SEED = 2
L2_BYTES = 129 * 2 ** 20

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# tensor-core kernel on this workload, keyed by the sha256 of the kernel source it
# was measured on; reported as null when the source has changed since.
TRAFFIC = {"6c29018be2a5f373": 2.487e9}  # 31.97 MB read + 2.455 GB written (two launches)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-kernel comparison")
    ap.add_argument("--nx", type=int, default=NX, help="cubes per axis (64: the benchmark mesh)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device=None):
    """Max of a float over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload(nx=NX):
    from paper_1407_0904_gb300 import meshgen
    mesh = meshgen.tet_mesh(nx, perturb=PERTURB, seed=SEED)
    return mesh


def alg_bytes_per_cell(mesh, ndof, out_bytes):
    """Algorithmic HBM bytes per cell: cell2vert + coords (each once) + the element matrix."""
    return 4 * 4 + 8 * 3 * mesh.nverts / mesh.ncells + out_bytes * ndof * ndof


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_source_sha():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1407_0904_gb300", "csrc", "k_tc.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def cpu_baseline(mesh, target_seconds, rank):
    """The FP64 oracle, as it stands, on a bounded prefix of the same workload."""
    import oracle
    threads = oracle.threads_available()
    pilot = np.arange(min(2048, mesh.ncells), dtype=np.int64)
    t0 = time.perf_counter()
    oracle.assemble_cells(oracle.HELMHOLTZ, DEGREE, oracle.TETRAHEDRON, mesh.coords,
                          mesh.cell2vert, pilot, threads=threads)
    per = (time.perf_counter() - t0) / len(pilot)
    n = int(min(mesh.ncells, max(len(pilot), target_seconds / max(per, 1e-9))))
    sel = np.arange(n, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.assemble_cells(oracle.HELMHOLTZ, DEGREE, oracle.TETRAHEDRON, mesh.coords,
                          mesh.cell2vert, sel, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "first %d of %d cells of the same mesh (FP64 oracle, OpenMP over cells, %.1f s)"
                      % (n, mesh.ncells, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    mesh = workload()
    threads = oracle.threads_available()
    run = lambda sel: oracle.assemble_cells(oracle.HELMHOLTZ, DEGREE, oracle.TETRAHEDRON, mesh.coords,
                                            mesh.cell2vert, sel, threads=threads)
    pilot = np.arange(2048, dtype=np.int64)
    t0 = time.perf_counter()
    run(pilot)
    per_cell = (time.perf_counter() - t0) / len(pilot)
    # every step is a bounded sample so that warm-up + steps take about two minutes
    budget = min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup))
    n = int(min(mesh.ncells, max(256, budget / max(per_cell, 1e-9))))
    total_cells, total_s = 0, 0.0
    for i in range(args.warmup + args.steps):
        lo = (i * n) % max(1, mesh.ncells - n)
        sel = np.arange(lo, lo + n, dtype=np.int64)
        t0 = time.perf_counter()
        run(sel)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            total_cells += n
            total_s += dt
    value = total_cells / total_s
    res = {"unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "%d steps of %d consecutive cells of the 64^3x6 mesh (FP64 oracle, OpenMP over "
                     "cells, %.2f s timed)" % (args.steps, n, total_s)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "helmholtz P3 tet, 64^3x6 Kuhn cells perturbed 0.15h (seed 2)",
                       "ncells": mesh.ncells, "degree": DEGREE},
            "cpu_baseline": dict(res, value=value),
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
    form, cell = coffee.HELMHOLTZ, coffee.TETRAHEDRON

    mesh = workload(args.nx)
    ndof = coffee.ndof(form, DEGREE, cell)
    coords = torch.from_numpy(mesh.coords).to(dev)
    c2v = torch.from_numpy(mesh.cell2vert).to(dev)
    ncells = mesh.ncells
    out_bytes = 8 if prec == coffee.FP64 else 4
    odt = torch.float64 if prec == coffee.FP64 else torch.float32
    out = torch.empty((ncells, ndof, ndof), dtype=odt, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision, o):
        coffee.assemble(form, DEGREE, cell, coords, c2v, precision=precision, out=o)

    # parity spot check of the benchmarked configuration against the oracle
    step(prec, out)
    coffee.check_errors()
    max_err = None
    if rank == 0:
        import oracle
        sel = np.random.default_rng(0).choice(ncells, size=512, replace=False)
        ref = oracle.assemble_cells(oracle.HELMHOLTZ, DEGREE, oracle.TETRAHEDRON, mesh.coords,
                                    mesh.cell2vert, sel)
        got = out[torch.from_numpy(sel).to(dev)].double().cpu().numpy()
        max_err = float(np.max(np.abs(got - ref).reshape(len(sel), -1).max(1)
                               / np.abs(ref).reshape(len(sel), -1).max(1)))

    def timed(precision, o, steps, warmup):
        for _ in range(warmup):
            step(precision, o)
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
            step(precision, o)
            b.record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        total_ms = t0.elapsed_time(t1)
        per_launch = [a.elapsed_time(b) for a, b in evs]
        return total_ms, float(np.mean(per_launch))

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)  # let nvidia-smi start sampling before the timed region
    total_ms, launch_ms = timed(prec, out, args.steps, args.warmup)
    clocks = sampler.stop()
    coffee.check_errors()
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    value = sum_over_ranks(ncells * args.steps, world, dev) / (total_ms / 1e3)

    # roofline of the dominant (only) kernel: algorithmic bytes per launch / launch time
    per_cell = alg_bytes_per_cell(mesh, ndof, out_bytes)
    achieved = per_cell * ncells / (launch_ms / 1e3) / 1e9
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    peak = float(peaks.get("hbm_gbs", 6800.0))
    sha = kernel_source_sha()
    traffic = TRAFFIC.get(sha) if prec != coffee.FP64 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "alg_bytes_per_cell": per_cell, "kernel_ms": launch_ms}
    if prec == coffee.FP64:
        roof["note"] = "FP64 kernel: bound by FP64 ALU, HBM fraction reported for context"

    # the FP64 kernel on the same workload, for the TC-vs-FP64 comparison
    fp64 = None
    if prec != coffee.FP64 and not args.no_fp64:
        out64 = torch.empty((ncells, ndof, ndof), dtype=torch.float64, device=dev)
        fsteps = max(3, min(args.steps // 20, 100))
        tms, lms = timed(coffee.FP64, out64, fsteps, 3)
        fp64 = {"value": ncells * fsteps / (tms / 1e3), "kernel_ms": lms, "steps": fsteps}
        del out64

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        h_coords = torch.from_numpy(mesh.coords).pin_memory()
        h_c2v = torch.from_numpy(mesh.cell2vert).pin_memory()
        h_out = torch.empty((ncells, ndof, ndof), dtype=odt).pin_memory()
        e_steps = max(3, min(args.steps // 20, 50))
        for _ in range(2):
            coffee.assemble_host(form, DEGREE, cell, h_coords, h_c2v, precision=prec, out=h_out)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e_steps):
            coffee.assemble_host(form, DEGREE, cell, h_coords, h_c2v, precision=prec, out=h_out)
        b.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a.elapsed_time(b), world, dev)
        e2e = {"value": sum_over_ranks(ncells * e_steps, world, dev) / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h_coords.numel() * 8 + h_c2v.numel() * 4),
               "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.nx == NX:
        cpu = cpu_baseline(mesh, args.cpu_seconds, rank)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64"}.get(args.precision, args.precision),
                "data": "synthetic",
                "config": {"workload": "helmholtz P3 tet, %d^3x6 Kuhn cells perturbed 0.15h (seed 2)" % args.nx,
                           "ncells": ncells, "degree": DEGREE, "ndof": ndof,
                           "precision": args.precision, "out_dtype": str(odt).replace("torch.", ""),
                           "l2": "no flush: each step writes %.2f GB of element matrices (> 129 MB L2)"
                                 % (ncells * ndof * ndof * out_bytes / 1e9),
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roof, "max_rel_err_vs_oracle": max_err,
                "fp64_kernel": fp64,
                "tc_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
                "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": args.steps,
                "clocks": clocks, "kernel_sha": sha}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
