"""The benchmark's reference arm (the FP64 oracle on the host cores) on a reduced mesh: one JSON
line with the keys of the benchmark contract, rank 0 only under a multi-rank launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "6",
        "--steps", "3", "--warmup", "3", "--cpu-seconds", "0.2"]


def run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run(ARGS, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert len(lines) == 1
    d = lines[0]
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    assert run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_algorithmic_bytes_per_cell_of_the_headline_and_burgers_workloads():
    """Roofline numerators: every input read once plus the output written once. Helmholtz P3 on the
    64^3 x 6 Kuhn mesh: 16 B of cell2vert, 24 nverts/ncells B of coordinates and 1600 B of element
    matrix = 1620.2 B per cell; Burgers P2 on 2^20 tets adds cell2dof (40 B) and u."""
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.WORKLOADS[bench.HEADLINE]
    mesh, coef, c2d = wl.build(None)
    b = bench.alg_bytes_per_cell(wl, mesh, c2d, coef, 20, 4)
    assert abs(b - (16 + 24 * 65 ** 3 / (64 ** 3 * 6) + 1600)) < 1e-9 and abs(b - 1620.2) < 0.05
    wl = bench.WORKLOADS["burgers-p2-tet"]
    mesh, coef, c2d = wl.build(None)
    nn = coef.size // 3
    b = bench.alg_bytes_per_cell(wl, mesh, c2d, coef, 30, 4)
    want = 16 + 24 * mesh.nverts / mesh.ncells + 3600 + 40 + 24 * nn / mesh.ncells
    assert abs(b - want) < 1e-9 and abs(b - 3693) < 1.0
