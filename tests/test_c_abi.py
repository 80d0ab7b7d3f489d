"""The boundary as a C program sees it: tests/c/abi_check.c includes the three public headers
as plain C11, takes the address of every entry point, links libcoffee.so and runs the host-only
calls (no CUDA device needed)."""
import os
import shutil
import subprocess

import pytest

import paper_1407_0904_gb300 as coffee

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_program_compiles_links_and_runs_against_the_headers(tmp_path):
    lib = coffee.binding.LIB_PATH
    coffee.lib()  # raises if the library is not built
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_check.c"),
           "-o", exe, "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + os.path.dirname(lib), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
