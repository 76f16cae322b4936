"""The C ABI from C: tests/c/abi_smoke.c, compiled as C99 against
include/pie.h and linked with libpie.so, runs the calls that need no GPU
(mesh construction, counts, edge table, argument errors)."""
import os
import shutil
import subprocess

import pytest

from tests._lib import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_caller(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    ensure_built()
    libdir = os.path.join(ROOT, "paper_1806_04164_gb300")
    exe = tmp_path / "abi_smoke"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                         os.path.join(ROOT, "tests", "c", "abi_smoke.c"), "-L", libdir, "-lpie",
                         f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    lines = run.stdout.split("\n")
    assert lines[0] == "mesh 6 8 12" and "ok" in lines
    assert lines[2].startswith("defaults 7 0.08 8 3 1")
