"""Mixed batch: all (form, degree) groups of triangles and tetrahedra in one persistent
launch (coffee_batch_plan / coffee_batch_launch), checked against the single-group
kernel (same arithmetic, so bitwise equal) and the FP64 oracle, plus CUDA-graph replay."""
import numpy as np
import pytest
import torch

import paper_1407_0904_gb300 as coffee
from paper_1407_0904_gb300 import meshgen
from tests.helpers import TRI, TET, ADVDIFF, rel_err_per_cell, oracle_ref

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def make_batch(tri, tet, seed=4, split=False):
    dev = {}
    for m in (tri, tet):
        coef, c2d, _ = meshgen.advdiff_coefficients(m, seed=seed)
        dev[m.cell] = dict(mesh=m, coords=torch.from_numpy(m.coords).to(DEV),
                           c2v=torch.from_numpy(m.cell2vert).to(DEV), coef_np=coef, c2d_np=c2d,
                           coef=torch.from_numpy(coef).to(DEV), c2d=torch.from_numpy(c2d).to(DEV))
        dev[m.cell]["xs"] = coffee.split_coords(dev[m.cell]["coords"]) if split else None
    groups = []
    for spec in meshgen.batch_groups(tri, tet, seed=seed):
        d = dev[spec["cell"]]
        sl = slice(spec["start"], spec["start"] + spec["count"])
        g = dict(form=spec["form"], degree=spec["degree"], cell=spec["cell"], coords=d["coords"],
                 cell2vert=d["c2v"][sl].contiguous(), spec=spec, coords_split=d["xs"])
        if spec["form"] == ADVDIFF:
            g["coef"] = d["coef"]
            g["cell2dof"] = d["c2d"][sl].contiguous()
        groups.append(g)
    return dev, groups


def check_groups(dev, groups, outs, prec, tol, sample=None):
    for g, out in zip(groups, outs):
        spec = g["spec"]
        if spec["count"] == 0:
            continue
        # the batch runs each group on its default kernel family (the CUDA cores for small
        # element matrices, the tensor cores otherwise): the single-group launch on the same
        simt = coffee.assemble_path(g["form"], g["degree"], g["cell"], prec) == 2
        single = coffee.assemble(g["form"], g["degree"], g["cell"], g["coords"], g["cell2vert"],
                                 g.get("coef"), g.get("cell2dof"), precision=prec,
                                 coords_split=g.get("coords_split"),
                                 tune=coffee.FLAG_CUDA_CORES if simt else coffee.FLAG_TENSOR_CORES)
        assert torch.equal(out, single), spec
        d = dev[g["cell"]]
        m = d["mesh"]
        rows = np.arange(spec["start"], spec["start"] + spec["count"])
        if sample is not None and len(rows) > sample:
            idx = np.random.default_rng(spec["start"]).choice(len(rows), size=sample, replace=False)
        else:
            idx = np.arange(len(rows))
        coef = d["coef_np"] if g["form"] == ADVDIFF else None
        c2d = d["c2d_np"] if g["form"] == ADVDIFF else None
        ref = oracle_ref(g["form"], g["degree"], g["cell"], m, coef, c2d, sel=rows[idx])
        got = out[torch.from_numpy(idx).to(DEV)].cpu().numpy()
        assert rel_err_per_cell(got, ref) < tol, spec


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("prec,tol", [(coffee.TF32X3, 1e-5), (coffee.BF16X3, 1e-5)])
def test_small_mixed_batch(prec, tol, split):
    """Every group equal bit for bit to its single-group launch and within the bound of the oracle,
    with FP64 coordinates or with their (hi, lo) float pairs."""
    tri = meshgen.tri_mesh(40, perturb=0.2, seed=4)
    tet = meshgen.tet_mesh(8, perturb=0.15, seed=5)
    dev, groups = make_batch(tri, tet, split=split)
    plan = coffee.BatchPlan(groups, precision=prec, validate=True)
    outs = plan.launch()
    coffee.check_errors()
    check_groups(dev, groups, outs, prec, tol)


def test_batch_all_on_the_tensor_cores():
    """all_tensor_cores keeps the small-matrix groups in the tensor-core launch: every group then
    equals its single-group tensor-core launch bit for bit and meets the bound."""
    tri = meshgen.tri_mesh(24, perturb=0.2, seed=12)
    tet = meshgen.tet_mesh(6, perturb=0.15, seed=13)
    dev, groups = make_batch(tri, tet, seed=12)
    plan = coffee.BatchPlan(groups, precision=coffee.TF32X3, all_tensor_cores=True)
    assert plan.launches == 1
    outs = plan.launch()
    coffee.check_errors()
    for g, out in zip(groups, outs):
        if g["spec"]["count"] == 0:
            continue
        single = coffee.assemble(g["form"], g["degree"], g["cell"], g["coords"], g["cell2vert"],
                                 g.get("coef"), g.get("cell2dof"), precision=coffee.TF32X3,
                                 tune=coffee.FLAG_TENSOR_CORES)
        assert torch.equal(out, single), g["spec"]
    assert coffee.BatchPlan(groups, precision=coffee.TF32X3).launches == 2


def test_batch_plan_options_do_not_change_results():
    tri = meshgen.tri_mesh(24, perturb=0.2, seed=6)
    tet = meshgen.tet_mesh(6, perturb=0.15, seed=7)
    dev, groups = make_batch(tri, tet, seed=6)
    a = [o.clone() for o in coffee.BatchPlan(groups).launch()]
    for grid, ovh in [(7, 0.0), (1, 1e6), (300, -1.0)]:
        b = coffee.BatchPlan(groups, grid=grid, item_overhead=ovh, costs="bytes").launch()
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    # measured tile costs (coffee_batch_plan_costs): other splits, the same matrices
    rng = np.random.default_rng(1)
    for grid, costs in [(0, "measured"), (5, list(rng.uniform(0.1, 10.0, len(groups)))), (0, [1.0] * len(groups))]:
        b = coffee.BatchPlan(groups, grid=grid, costs=costs).launch()
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)


def test_batch_cuda_graph_replay():
    tri = meshgen.tri_mesh(32, perturb=0.2, seed=8)
    tet = meshgen.tet_mesh(6, perturb=0.15, seed=9)
    dev, groups = make_batch(tri, tet, seed=8)
    plan = coffee.BatchPlan(groups)
    ref = [o.clone() for o in plan.launch()]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.launch()  # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            plan.launch()
    for o in plan.outputs:
        o.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for x, y in zip(ref, plan.outputs):
        assert torch.equal(x, y)


def test_config4_full_size_sampled():
    """2^19 triangles (512^2 x 2) and 2^19 tets (Kuhn 64x64x22 truncated), 21 groups with
    Zipf counts, one launch; every group sampled against the oracle."""
    tri = meshgen.tri_mesh(512, perturb=0.2, seed=4)
    tet = meshgen.tet_mesh(64, 64, 22, perturb=0.15, seed=4, ncells=2 ** 19)
    dev, groups = make_batch(tri, tet)
    assert len(groups) == 21 and sum(g["spec"]["count"] for g in groups) == 2 ** 20
    plan = coffee.BatchPlan(groups)
    outs = plan.launch()
    coffee.check_errors()
    check_groups(dev, groups, outs, coffee.TF32X3, 1e-5, sample=200)


def test_batch_validation_reports_a_bad_index_and_leaves_the_rest_intact():
    """validate=True: an out-of-range vertex id in one group is reported through check_errors,
    that cell's matrix is zero and every other cell of every group is unchanged."""
    tri = meshgen.tri_mesh(24, perturb=0.2, seed=6)
    tet = meshgen.tet_mesh(6, perturb=0.15, seed=7)
    dev, groups = make_batch(tri, tet, seed=6)
    clean = [o.clone() for o in coffee.BatchPlan(groups, validate=True).launch()]
    coffee.check_errors()
    gi = max(range(len(groups)), key=lambda i: groups[i]["spec"]["count"])
    bad = groups[gi]["cell2vert"].clone()
    bad[3, 1] = dev[groups[gi]["cell"]]["mesh"].nverts + 5
    groups[gi] = dict(groups[gi], cell2vert=bad)
    outs = coffee.BatchPlan(groups, validate=True).launch()
    with pytest.raises(coffee.CoffeeError) as ei:
        coffee.check_errors()
    assert ei.value.status == -4
    for i, (a, b) in enumerate(zip(clean, outs)):
        if i != gi:
            assert torch.equal(a, b)
    assert torch.count_nonzero(outs[gi][3]) == 0
    keep = torch.ones(outs[gi].shape[0], dtype=torch.bool, device=DEV)
    keep[3] = False
    assert torch.equal(outs[gi][keep], clean[gi][keep])

