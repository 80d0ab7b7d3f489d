"""The oracle and the CUDA path share no code and neither imports the other; the benchmark
reaches the oracle only in its CPU-baseline and reference legs. Checked on the sources."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1407_0904_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def sources(top, exts):
    for dirpath, _, files in os.walk(top):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_package_never_imports_or_includes_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"].*oracle)", re.M)
    bad = [p for p in sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")) if pat.search(open(p).read())]
    assert not bad, bad


def test_oracle_never_imports_the_package_or_its_headers():
    pat = re.compile(r"paper_1407_0904_gb300|#\s*include\s*[<\"][^>\"]*(coffee|tc_common|k_tc)", re.M)
    bad = [p for p in sources(ORACLE, (".py", ".cpp", ".c", ".h")) if pat.search(open(p).read())]
    assert not bad, bad


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"oracle_cells", "cpu_baseline", "run_reference"}
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for n in ast.walk(fn):
            if isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names):
                assert fn.name in allowed, fn.name
            if isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id == "oracle_cells":
                assert fn.name in {"cpu_baseline", "run_reference"}, fn.name
    top_imports = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(getattr(n, "module", None) == "oracle" or any(a.name == "oracle" for a in n.names)
                   for n in top_imports)


def test_missing_library_fails_loudly_without_a_fallback(tmp_path):
    """With libcoffee.so absent every call raises; nothing falls back to another implementation."""
    import subprocess
    import sys
    code = ("import paper_1407_0904_gb300.binding as b\n"
            "b.LIB_PATH = %r\n"
            "for call in (lambda: b.ndof(1, 2, 1), lambda: b.supported(1, 3, 1, 2),\n"
            "             lambda: b.reference_tensor(0, 1, 0)):\n"
            "    try:\n"
            "        call()\n"
            "    except RuntimeError as e:\n"
            "        assert 'not built' in str(e)\n"
            "    else:\n"
            "        raise SystemExit('no error')\n"
            "print('raised')\n" % str(tmp_path / "libcoffee.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "raised", r.stdout + r.stderr


def test_only_tests_smoke_build_and_the_benchmark_cpu_legs_import_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)", re.M)
    users = set()
    # the product: the package and the scripts at the repository root
    product = list(sources(PKG, (".py",))) + [os.path.join(ROOT, f) for f in os.listdir(ROOT) if f.endswith(".py")]
    for p in product:
        rel = os.path.relpath(p, ROOT)
        if pat.search(open(p).read()):
            users.add(rel)
    assert users <= {"__graft_entry__.py", "bench.py"}, users
    tree = ast.parse(open(os.path.join(ROOT, "__graft_entry__.py")).read())
    for fn in [n for n in tree.body if isinstance(n, ast.FunctionDef)]:
        imports = [a.name for n in ast.walk(fn) if isinstance(n, ast.Import) for a in n.names]
        if "oracle" in imports:
            assert fn.name in {"build", "smoke"}, fn.name
