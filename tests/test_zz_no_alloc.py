"""The allocation-free near-part product (pie_apply_near_noalloc).

Callers that cannot allocate device memory when they need a product (inside
a graph capture they do not own, or under an allocator that owns all device
memory) use this entry point; it must give the same result as the ordinary
near-part product, call after call.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu


def test_noalloc_matches_apply_near_twice():
    import torch

    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    lib = pg.lib()
    xyz, tri = pi.icosphere(3)
    for prec in (pg.PIE_FP64, pg.PIE_MIXED, pg.PIE_FP32, pg.PIE_FP32H):
        pr = pg.Problem(pg.Mesh(xyz, tri), 0.01, 3, root_side=2.0, precision=prec)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (11, 12):
            x = torch.from_numpy(pi.complex_normal(pr.N, seed)).to(pr.torch_dtype).cuda()
            ref = pr.apply(x, near_only=True)
            y = torch.full_like(x, float("nan"))
            code = lib.pie_apply_near_noalloc(pr.handle, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), pr.dtype_code, stream)
            assert code == 0, lib.pie_last_error().decode()
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), ref.cpu().numpy()
            tol = 1e-12 if prec == pg.PIE_FP64 else 1e-6
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_noalloc_inside_a_graph_capture():
    """The reason the entry point exists: it runs inside a stream capture the
    caller owns.  Global capture mode makes any allocation (or other
    unsafe call) during the capture fail it; two replays of the captured
    product must equal pie_apply_near."""
    import torch

    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    lib = pg.lib()
    xyz, tri = pi.icosphere(3)
    pr = pg.Problem(pg.Mesh(xyz, tri), 0.01, 3, root_side=2.0, precision=pg.PIE_MIXED)
    x = torch.from_numpy(pi.complex_normal(pr.N, 21)).cuda()
    y = torch.empty_like(x)
    side = torch.cuda.Stream()
    args = (pr.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), pr.dtype_code,
            ctypes.c_void_p(side.cuda_stream))
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        assert lib.pie_apply_near_noalloc(*args) == 0      # one call before the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="global"):
        code = lib.pie_apply_near_noalloc(*args)
    assert code == 0, lib.pie_last_error().decode()
    ref = pr.apply(x, near_only=True)
    for _ in range(2):
        y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)) and np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_noalloc_rejects_mesh_above_limit():
    """The smallest problem above the complex-float limit of 262,144
    triangles: a flat 363 x 363 split-square patch (263,538 triangles,
    8 levels, half-precision moments) is rejected with PIE_ERR_PARAM before
    any device work; 81,920 triangles in complex double are accepted."""
    import torch

    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    lib = pg.lib()
    xyz, tri = pi.icosphere(6)          # 81920 triangles: within the limit
    pr = pg.Problem(pg.Mesh(xyz, tri), 1e-3, 6, root_side=2.0)
    x = torch.zeros(pr.N, dtype=pr.torch_dtype, device="cuda")
    y = torch.empty_like(x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.pie_apply_near_noalloc(pr.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      pr.dtype_code, stream) == 0
    del pr, x, y
    xyz, tri = pi.square_patch(363)     # 263538 triangles: above it
    pr = pg.Problem(pg.Mesh(xyz, tri), 1e-3, 8, precision=pg.PIE_FP32H)
    assert pr.T == 263538
    x = torch.zeros(pr.N, dtype=pr.torch_dtype, device="cuda")
    y = torch.empty_like(x)
    code = lib.pie_apply_near_noalloc(pr.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      pr.dtype_code, stream)
    assert code == 1
    assert b"too large" in lib.pie_last_error()
