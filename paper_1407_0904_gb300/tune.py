"""Autotuner of the tensor-core kernels.

The paper chooses its transformation parameters (split factor, unroll-and-jam factor, loop
permutation) with a cost model rather than by autotuning, because autotuning every
generated kernel at JIT time is too slow (section 4). Here the kernels are fixed and few,
so they are tuned once per GPU: for every (form, degree, cell, precision) the tuner times
each combination of the kernels' knobs on a seeded synthetic mesh and records the fastest
in a JSON cache that `assemble` consults. For the mixed batch it tunes the plan's per-item
cost overhead (how work is balanced over the CTAs).

Knobs (all give bit-identical results; only speed changes):
  FLAG_OUTPUT_LANES   element-matrix entries on the TMEM lanes even for tiny matrices
  FLAG_CELL_LANES     cells on the TMEM lanes for matrices of up to 128 entries
  FLAG_SUBTILE_128/64/32  cells per TMEM accumulator with outputs on the lanes (MMA N)
  FLAG_TWO_STAGES     at most two operand stages
  FLAG_STAGED_STORE   rows of consecutive cells gathered in shared memory, one bulk copy each
                      (tried where rows do not start on 32-byte sectors)
  FLAG_CUDA_CORES / FLAG_TENSOR_CORES  the FP32 CUDA-core kernel or the tensor cores, where a
                      small element matrix has both

  python -m paper_1407_0904_gb300.tune [--ncells N] [--out PATH]
  python -m paper_1407_0904_gb300.tune --study    # cost model vs the tuned choices (no GPU)

The study mirrors the paper's trade-off between a cost model and autotuning: `model_flags`
chooses the knobs from the element-matrix shape alone (no timing), and `study` measures, on
the timings the tuner recorded for every candidate, how much slower the model's choice and
the library's built-in default are than the tuned best.
"""
import argparse
import json
import os
import sys

import numpy as np

CACHE_VERSION = 1


def cache_path():
    return os.environ.get("COFFEE_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json"))


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else ""


def load_cache(path=None, gpu=None):
    """Entries tuned on this GPU model ({} when there is no cache for it)."""
    p = path or cache_path()
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        data = json.load(f)
    if data.get("version") != CACHE_VERSION:
        return {}
    name = gpu if gpu is not None else _gpu_name()
    if data.get("gpu") and name and data["gpu"] != name:
        return {}
    return data.get("entries", {})


def load_batch(path=None, gpu=None):
    """Tuned mixed-batch settings for this GPU model ({} when none)."""
    p = path or cache_path()
    if not os.path.exists(p) or not load_cache(p, gpu):
        return {}
    with open(p) as f:
        return json.load(f).get("batch", {})


def candidates(coffee, n_outputs, cuda_cores=False):
    """Knob combinations to time. Where the element matrix also has the FP32 CUDA-core kernel
    (cuda_cores), the tensor-core combinations are forced onto the tensor cores and the
    CUDA-core kernel is one more candidate; 0 (the library's default path) stays in the list."""
    F = coffee
    c = [0, F.FLAG_TWO_STAGES, F.FLAG_SUBTILE_128, F.FLAG_SUBTILE_64, F.FLAG_SUBTILE_32,
         F.FLAG_SUBTILE_64 | F.FLAG_TWO_STAGES]
    if n_outputs <= 128:
        c += [F.FLAG_OUTPUT_LANES, F.FLAG_CELL_LANES, F.FLAG_CELL_LANES | F.FLAG_TWO_STAGES]
    if (n_outputs * 4) % 32:  # rows not on 32-byte sectors: rows staged for bulk copies
        c += [F.FLAG_OUTPUT_LANES | F.FLAG_STAGED_STORE, F.FLAG_OUTPUT_LANES | F.FLAG_STAGED_STORE | F.FLAG_TWO_STAGES]
    if cuda_cores:
        c = [0, F.FLAG_CUDA_CORES] + [t | F.FLAG_TENSOR_CORES for t in c]
    return sorted(set(c))


def _mesh(cell, ncells, seed=7):
    from . import meshgen
    if cell == 0:
        n = 1
        while 2 * n * n < ncells:
            n += 1
        return meshgen.tri_mesh(n, perturb=0.2, seed=seed)
    n = 1
    while 6 * n ** 3 < ncells:
        n += 1
    return meshgen.tet_mesh(n, perturb=0.15, seed=seed, ncells=ncells)


def time_case(coffee, form, degree, cell, precision, mesh, tune, reps=20, warmup=3):
    import torch
    from . import meshgen
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(mesh.coords).to(dev)
    c2v = torch.from_numpy(mesh.cell2vert).to(dev)
    cf = cd = None
    if form == coffee.ADVDIFF:
        coef, c2d, _ = meshgen.advdiff_coefficients(mesh, seed=3)
        cf, cd = torch.from_numpy(coef).to(dev), torch.from_numpy(c2d).to(dev)
    elif form == coffee.BURGERS_JAC:
        u, c2d, _ = meshgen.burgers_coefficients(mesh, degree, seed=3)
        cf, cd = torch.from_numpy(u.ravel()).to(dev), torch.from_numpy(c2d).to(dev)
    n = coffee.ndof(form, degree, cell)
    out = torch.empty((mesh.ncells, n, n), dtype=torch.float32, device=dev)
    run = lambda: coffee.assemble(form, degree, cell, x, c2v, cf, cd, precision=precision, out=out, tune=tune)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        run()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_all(forms=None, cells=(0, 1), degrees=(1, 2, 3, 4), precisions=None, ncells=2 ** 19, reps=20,
             log=print):
    from . import binding as coffee
    forms = forms or (coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF)
    precisions = precisions or (coffee.TF32X3,)
    entries = {}
    meshes = {c: _mesh(c, ncells) for c in cells}
    for form in forms:
        for cell in cells:
            for k in degrees:
                for prec in precisions:
                    if not coffee.supported(form, k, cell, prec):
                        continue
                    n = coffee.ndof(form, k, cell) ** 2
                    times = {}
                    simt = coffee.assemble_path(form, k, cell, prec, coffee.FLAG_CUDA_CORES) == 2
                    for t in candidates(coffee, n, simt):
                        times[t] = time_case(coffee, form, k, cell, prec, meshes[cell], t, reps=reps)
                    best = min(times, key=times.get)
                    key = "%d/%d/%d/%d" % (form, k, cell, prec)
                    entries[key] = {"flags": int(best), "ms": times[best], "ncells": meshes[cell].ncells,
                                    "candidates": {str(t): round(v, 5) for t, v in times.items()}}
                    log("%s %s P%d %s: best flags %d (%.4f ms; default %.4f ms)" % (
                        coffee.FORM_NAMES[form], "tri" if cell == 0 else "tet", k,
                        coffee.PRECISION_NAMES[prec], best, times[best], times[0]))
    return entries


def tune_batch_tiles(ncells=2 ** 17, precisions=None, reps=20, log=print):
    """Time per 128-cell tile (ms, on one SM) of every group shape inside the batch kernel:
    each (form, degree, cell) runs alone as a one-group batch of `ncells` cells. These are the
    per-group costs BatchPlan splits the work by (costs="measured")."""
    import torch
    from . import binding as coffee
    from . import meshgen
    dev = torch.device("cuda", torch.cuda.current_device())
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    precisions = precisions or (coffee.TF32X3,)
    out = {}
    for cell in (0, 1):
        m = _mesh(cell, ncells)
        x, c2v = torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.cell2vert).to(dev)
        coef, c2d, _ = meshgen.advdiff_coefficients(m, seed=4)
        cf, cd = torch.from_numpy(coef).to(dev), torch.from_numpy(c2d).to(dev)
        for form in (coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF):
            for k in (1, 2, 3, 4):
                for prec in precisions:
                    g = dict(form=form, degree=k, cell=cell, coords=x, cell2vert=c2v)
                    if form == coffee.ADVDIFF:
                        g["coef"], g["cell2dof"] = cf, cd
                    try:
                        plan = coffee.BatchPlan([g], precision=prec, costs="bytes")
                    except coffee.CoffeeError:
                        continue  # shape not covered by the batch kernel
                    for _ in range(3):
                        plan.launch()
                    torch.cuda.synchronize()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    for _ in range(reps):
                        plan.launch()
                    b.record()
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b) / reps
                    plan.free()
                    tiles = (m.ncells + 127) // 128
                    key = "%d/%d/%d/%d" % (form, k, cell, prec)
                    out[key] = ms * min(tiles, nsm) / tiles
                    log("batch tile %s: %.3f us per tile (%.4f ms for %d cells)" % (key, out[key] * 1e3, ms, m.ncells))
    return out


def tune_batch(ncells_per_mesh=2 ** 17, log=print):
    """Per-item overhead of the batch plan's cost model, timed on a mixed batch."""
    import torch
    from . import binding as coffee
    from . import meshgen
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 1
    while 2 * n * n < ncells_per_mesh:
        n += 1
    tri = meshgen.tri_mesh(n, perturb=0.2, seed=4)
    tet = meshgen.tet_mesh(48, perturb=0.15, seed=4, ncells=ncells_per_mesh)
    groups = []
    for m in (tri, tet):
        coef, c2d, _ = meshgen.advdiff_coefficients(m, seed=4)
        x, c2v = torch.from_numpy(m.coords).to(dev), torch.from_numpy(m.cell2vert).to(dev)
        cf, cd = torch.from_numpy(coef).to(dev), torch.from_numpy(c2d).to(dev)
        for spec in meshgen.batch_groups(tri, tet, seed=4):
            if spec["cell"] != m.cell:
                continue
            sl = slice(spec["start"], spec["start"] + spec["count"])
            g = dict(form=spec["form"], degree=spec["degree"], cell=spec["cell"], coords=x,
                     cell2vert=c2v[sl].contiguous())
            if spec["form"] == coffee.ADVDIFF:
                g["coef"], g["cell2dof"] = cf, cd[sl].contiguous()
            groups.append(g)
    times = {}
    for ovh in (0.0, 4096.0, 16384.0, 65536.0, 262144.0):
        plan = coffee.BatchPlan(groups, item_overhead=ovh, costs="bytes")
        for _ in range(3):
            plan.launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            plan.launch()
        b.record()
        torch.cuda.synchronize()
        times[ovh] = a.elapsed_time(b) / 20
        plan.free()
    best = min(times, key=times.get)
    log("batch: best item overhead %g (%.4f ms)" % (best, times[best]))
    return {"item_overhead": best, "ms": times[best], "candidates": {str(k): round(v, 5) for k, v in times.items()}}


def model_flags(n_outputs, cuda_cores=False):
    """Knobs chosen without timing, from the number of entries N of the element matrix.

    - Where the element matrix also has the FP32 CUDA-core kernel (cuda_cores): that kernel
      when N <= 36 (its K-term sums for N entries cost N K FMAs per cell against the
      tensor-core kernel's fixed hand-offs per 128-cell tile), else the tensor cores with the
      knobs below.
    - Cells on the TMEM lanes when N <= 64: one thread then writes its cell's whole row
      (<= 256 bytes, at most two 128-byte lines) with 16-byte stores, so rows are completed
      by one thread in order; above that a thread holds too many accumulator columns.
    - With outputs on the lanes and exactly two 128-output slices (64 < N <= 256), 64 cells
      per accumulator: twice the accumulators in flight, so the stores of the second, partly
      filled slice overlap the next sub-tile's MMAs.
    - Otherwise the library default (128 cells per accumulator up to four slices).
    """
    from . import binding as coffee
    if cuda_cores:
        if n_outputs <= 36:
            return coffee.FLAG_CUDA_CORES
        return model_flags(n_outputs) | coffee.FLAG_TENSOR_CORES
    mtiles = (n_outputs + 127) // 128
    if n_outputs <= 64:
        return coffee.FLAG_CELL_LANES
    if mtiles == 2:
        return coffee.FLAG_SUBTILE_64
    return 0


def study(entries=None, log=print):
    """Regret (time / tuned best - 1) of the cost model and of the built-in default for every
    tuned (form, degree, cell, precision), from the candidates' recorded times."""
    from . import binding as coffee
    entries = entries if entries is not None else load_cache(gpu="")
    rows = []
    for key, ent in sorted(entries.items()):
        form, k, cell, prec = map(int, key.split("/"))
        n = coffee.ndof(form, k, cell) ** 2
        cands = {int(float(c)): t for c, t in ent["candidates"].items()}
        best = min(cands.values())
        mf = model_flags(n, coffee.assemble_path(form, k, cell, prec, coffee.FLAG_CUDA_CORES) == 2)
        model_t = cands.get(mf)
        rows.append({"key": key, "form": coffee.FORM_NAMES[form], "degree": k, "cell": "tri" if cell == 0 else "tet",
                     "N": n, "best_flags": int(ent["flags"]), "best_ms": best, "model_flags": mf,
                     "model_regret": None if model_t is None else model_t / best - 1.0,
                     "default_regret": cands.get(0, float("nan")) / best - 1.0})
    for r in rows:
        log("%-10s P%d %s N=%4d  tuned %-3d %.4f ms  model %-3d regret %s  default regret %.1f%%" % (
            r["form"], r["degree"], r["cell"], r["N"], r["best_flags"], r["best_ms"], r["model_flags"],
            "n/a" if r["model_regret"] is None else "%.1f%%" % (100 * r["model_regret"]), 100 * r["default_regret"]))
    mr = [r["model_regret"] for r in rows if r["model_regret"] is not None]
    dr = [r["default_regret"] for r in rows]
    if mr:
        log("model:   mean regret %.2f%%, max %.2f%%, best choice in %d of %d" % (
            100 * np.mean(mr), 100 * max(mr), sum(x <= 1e-9 for x in mr), len(mr)))
    log("default: mean regret %.2f%%, max %.2f%%, best choice in %d of %d" % (
        100 * np.mean(dr), 100 * max(dr), sum(x <= 1e-9 for x in dr), len(dr)))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncells", type=int, default=2 ** 19)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default=None)
    ap.add_argument("--study", action="store_true", help="cost model vs the cached tuned choices (no GPU)")
    ap.add_argument("--batch-tiles", action="store_true",
                    help="only (re)measure the batch kernel's per-group tile costs into the existing cache")
    args = ap.parse_args(argv)
    if args.study:
        study()
        return 0
    if args.batch_tiles:
        with open(cache_path()) as f:
            data = json.load(f)
        data.setdefault("batch", {})["tile_ms"] = tune_batch_tiles()
        out = args.out or cache_path()
        with open(out, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        print("wrote", out)
        return 0
    entries = tune_all(ncells=args.ncells, reps=args.reps)
    batch = tune_batch()
    batch["tile_ms"] = tune_batch_tiles()
    data = {"version": CACHE_VERSION, "gpu": _gpu_name(), "entries": entries, "batch": batch}
    out = args.out or cache_path()
    with open(out, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print("wrote", out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
