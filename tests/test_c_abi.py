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


@pytest.mark.gpu
def test_c99_caller_runs_the_path(tmp_path):
    """tests/c/abi_apply.c drives mesh, problem, product and solve through
    the C ABI alone; its product equals the Python binding's bit for bit
    (same library, same arithmetic) and its solve converges."""
    import numpy as np
    import torch

    import paper_1806_04164_gb300 as pg
    import pie_inputs as pi
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    ensure_built()
    libdir = os.path.join(ROOT, "paper_1806_04164_gb300")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "abi_apply"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
                         os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c", "abi_apply.c"), "-L", libdir,
                         "-lpie", "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
                         f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    xyz, tri = pi.icosphere(3)
    k0, L = 0.01, 3
    mesh = pg.Mesh(xyz, tri)
    x = pi.complex_normal(mesh.nt + mesh.ne, 5)
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.int64(len(xyz)).tobytes() + np.int64(len(tri)).tobytes())
        f.write(np.ascontiguousarray(xyz, np.float64).tobytes() + np.ascontiguousarray(tri, np.int32).tobytes())
        f.write(np.float64(k0).tobytes() + np.int32(L).tobytes() + np.ascontiguousarray(x).tobytes())
    out = tmp_path / "out.bin"
    run = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    raw = open(out, "rb").read()
    n = mesh.nt + mesh.ne
    y_c = np.frombuffer(raw[:16 * n], np.complex128)
    its = np.frombuffer(raw[16 * n:16 * n + 4], np.int32)[0]
    res = np.frombuffer(raw[16 * n + 4:16 * n + 12], np.float64)[0]
    pr = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_MIXED)
    y_py = pr.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y_c, y_py)
    assert its > 0 and res <= 1e-6
