"""Python binding of libpie (include/pie.h): argument marshalling only.

Every step of the operator runs in the CUDA library; this module converts
numpy / torch arguments into the C ABI's plain pointers and sizes.  Device
buffers are torch tensors on a CUDA device (complex128 for PIE_FP64 and
PIE_MIXED problems, complex64 for PIE_FP32); streams default to torch's
current stream.  Importing works without a GPU; creating a problem needs one
and raises if the library has not been built.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libpie.so")

PIE_FP64, PIE_FP32, PIE_MIXED, PIE_FP32H = 0, 1, 2, 3
PIE_C128, PIE_C64 = 0, 1
STATUS = {0: "PIE_OK", 1: "PIE_ERR_PARAM", 2: "PIE_ERR_NONMANIFOLD", 3: "PIE_ERR_DEGENERATE",
          4: "PIE_ERR_ORIENTATION", 5: "PIE_ERR_OOM", 6: "PIE_ERR_CUDA", 7: "PIE_ERR_LEAF",
          8: "PIE_ERR_NOCONV", 9: "PIE_ERR_BREAKDOWN", 10: "PIE_ERR_NAN"}

# Parameters found by the Eq. (4)-(5) error search (truncation tau, kappa*a, N_theta).
DEFAULT_TAU, DEFAULT_KAPPA_A, DEFAULT_NTHETA = 7, 0.08, 8


class PieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("root_side", ctypes.c_double), ("tau", ctypes.c_int),
                ("kappa_a", ctypes.c_double), ("ntheta", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_nrhs", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("E", ctypes.c_int64), ("T", ctypes.c_int64), ("L", ctypes.c_int32),
                ("P", ctypes.c_int32), ("boxes", ctypes.c_int64 * 24), ("near_pairs", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("leaf_size", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("overlap", ctypes.c_int32), ("near_ctas_per_sm", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32),
                ("near_rhs_block", ctypes.c_int32), ("far_rows", ctypes.c_int32), ("near_kernel", ctypes.c_int32)]

    def as_dict(self):
        return dict(overlap=self.overlap, near_ctas_per_sm=self.near_ctas_per_sm, rhs_chunk=self.rhs_chunk,
                    near_rhs_block=self.near_rhs_block, far_rows=self.far_rows, near_kernel=self.near_kernel)


class NestedParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("inner_restart", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("outer_restart", ctypes.c_int32), ("max_outer", ctypes.c_int32)]


class NestedStats(ctypes.Structure):
    _fields_ = [("inner_iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("outer_products", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("inner_product_seconds", ctypes.c_double), ("outer_product_seconds", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("reorthogonalizations", ctypes.c_int32), ("product_seconds", ctypes.c_double)]


_lib = None
EXPORTS = ["pie_last_error", "pie_params_default", "pie_mesh_create", "pie_mesh_destroy", "pie_mesh_info",
           "pie_mesh_edges", "pie_problem_create", "pie_problem_destroy", "pie_problem_info", "pie_problem_perm",
           "pie_problem_level", "pie_problem_near", "pie_apply", "pie_apply_near", "pie_problem_stage", "pie_rhs_planewave",
           "pie_farfield", "pie_solve", "pie_profile_begin", "pie_profile_end", "pie_apply_near_noalloc", "pie_apply_t",
           "pie_farfield_adjoint", "pie_apply_single_layer", "pie_solve_single_layer", "pie_rhs_potential",
           "pie_nearfield", "pie_problem_get_tuning", "pie_problem_set_tuning", "pie_problem_autotune",
           "pie_tune_levels", "pie_group_create", "pie_group_apply", "pie_group_info", "pie_group_destroy",
           "pie_apply_levels", "pie_problem_quadrature", "pie_rhs_potentials", "pie_solve_guess",
           "pie_solve_nested", "pie_measure_peaks"]
STAGES = ["coef", "near", "aggregation", "interpolation", "translation", "anterpolation", "disaggregation",
          "assembly"]


def lib():
    """Load libpie.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"libpie.so not built ({LIBPATH}); run paper_1806_04164_gb300/build.py")
        L = ctypes.CDLL(LIBPATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P64 = ctypes.POINTER(ctypes.c_int64)
        P32 = ctypes.POINTER(ctypes.c_int32)
        PD = ctypes.POINTER(ctypes.c_double)
        L.pie_last_error.restype = ctypes.c_char_p
        L.pie_params_default.argtypes = [ctypes.POINTER(Params)]
        L.pie_mesh_create.argtypes = [PD, i64, P32, i64, ctypes.POINTER(vp)]
        L.pie_mesh_destroy.argtypes = [vp]
        L.pie_mesh_info.argtypes = [vp, P64, P64, P64]
        L.pie_mesh_edges.argtypes = [vp, P32, P32, P32]
        L.pie_problem_create.argtypes = [vp, dbl, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
        L.pie_problem_destroy.argtypes = [vp]
        L.pie_problem_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.pie_problem_perm.argtypes = [vp, P64]
        L.pie_problem_level.argtypes = [vp, i32, P64, P64, P64, P64, P64, P32]
        L.pie_problem_near.argtypes = [vp, P64, P64, P64]
        L.pie_apply.argtypes = [vp, vp, vp, i32, i32, vp]
        L.pie_apply_near.argtypes = [vp, vp, vp, i32, i32, vp]
        L.pie_apply_near_noalloc.argtypes = [vp, vp, vp, i32, vp]
        L.pie_apply_t.argtypes = [vp, vp, vp, i32, i32, i32, vp]
        L.pie_farfield_adjoint.argtypes = [vp, PD, i64, vp, vp, vp]
        L.pie_apply_single_layer.argtypes = [vp, vp, vp, vp]
        L.pie_solve_single_layer.argtypes = [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(SolveStats), vp]
        L.pie_rhs_potential.argtypes = [vp, PD, PD, dbl, vp, vp]
        L.pie_nearfield.argtypes = [vp, vp, vp, PD, i64, vp, vp]
        L.pie_problem_stage.argtypes = [vp, i32, i32, PD, vp]
        L.pie_rhs_planewave.argtypes = [vp, PD, PD, dbl, vp, i32, vp]
        L.pie_farfield.argtypes = [vp, vp, PD, i64, vp, i32, vp]
        L.pie_problem_quadrature.argtypes = [vp, PD, PD]
        L.pie_rhs_potentials.argtypes = [vp, vp, vp, vp, i32, vp]
        L.pie_profile_begin.argtypes = [vp, i32]
        L.pie_profile_end.argtypes = [vp, PD, P32]
        L.pie_solve.argtypes = [vp, vp, vp, i32, dbl, i32, i32, ctypes.POINTER(SolveStats), vp]
        L.pie_solve_guess.argtypes = [vp, vp, vp, i32, dbl, i32, i32, ctypes.POINTER(SolveStats), vp]
        L.pie_apply_levels.argtypes = [vp, vp, vp, ctypes.c_uint32, i32, i32, vp]
        L.pie_measure_peaks.argtypes = [PD, PD, PD, PD, vp]
        L.pie_solve_nested.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(NestedParams),
                                       ctypes.POINTER(NestedStats), vp]
        PT = ctypes.POINTER(Tuning)
        L.pie_problem_get_tuning.argtypes = [vp, PT]
        L.pie_problem_set_tuning.argtypes = [vp, PT]
        L.pie_problem_autotune.argtypes = [vp, i32, i32, PT, PD, vp]
        L.pie_tune_levels.argtypes = [vp, dbl, ctypes.POINTER(Params), i32, i32, i32, vp, P32, PD]
        L.pie_group_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
        L.pie_group_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp]
        L.pie_group_info.argtypes = [vp, P64, P64]
        L.pie_group_destroy.argtypes = [vp]
        _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise PieError(code, lib().pie_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dense(t):
    """Materialise lazy conjugate / negative views: the C ABI reads raw memory."""
    return t.resolve_conj().resolve_neg().contiguous()


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Mesh:
    """Triangulated surface (pie_mesh_create)."""

    def __init__(self, xyz, tri):
        self.xyz = np.ascontiguousarray(xyz, np.float64)
        self.tri = np.ascontiguousarray(tri, np.int32)
        h = ctypes.c_void_p()
        _check(lib().pie_mesh_create(_ptr(self.xyz, ctypes.c_double), self.xyz.shape[0],
                                     _ptr(self.tri, ctypes.c_int32), self.tri.shape[0], ctypes.byref(h)))
        self.handle = h
        nv, nt, ne = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pie_mesh_info(h, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(ne)))
        self.nv, self.nt, self.ne = nv.value, nt.value, ne.value

    def edges(self):
        e = np.zeros((self.ne, 2), np.int32)
        et = np.zeros((self.ne, 2), np.int32)
        ef = np.zeros((self.ne, 2), np.int32)
        _check(lib().pie_mesh_edges(self.handle, _ptr(e, ctypes.c_int32), _ptr(et, ctypes.c_int32),
                                    _ptr(ef, ctypes.c_int32)))
        return e, et, ef

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pie_mesh_destroy(self.handle)
            self.handle = None


class Problem:
    """PIE operator for one mesh and wavenumber (pie_problem_create)."""

    def __init__(self, mesh, k0, levels, root_side=0.0, tau=DEFAULT_TAU, kappa_a=DEFAULT_KAPPA_A,
                 ntheta=DEFAULT_NTHETA, precision=PIE_FP64, max_nrhs=1, stream=None):
        self.mesh = mesh
        self.k0 = float(k0)
        self.precision = precision
        p = Params(levels, root_side, tau, kappa_a, ntheta, precision, max_nrhs)
        h = ctypes.c_void_p()
        _check(lib().pie_problem_create(mesh.handle, self.k0, ctypes.byref(p), _stream(stream), ctypes.byref(h)))
        self.handle = h
        info = Info()
        _check(lib().pie_problem_info(h, ctypes.byref(info)))
        self.N, self.E, self.T, self.L, self.P = info.N, info.E, info.T, info.L, info.P
        self.boxes = [info.boxes[l] for l in range(self.L + 1)]
        self.near_pairs = info.near_pairs
        self.device_bytes = info.device_bytes
        self.leaf_size = info.leaf_size
        self.dtype_code = PIE_C64 if precision in (PIE_FP32, PIE_FP32H) else PIE_C128

    @property
    def torch_dtype(self):
        import torch
        return torch.complex64 if self.dtype_code == PIE_C64 else torch.complex128

    def perm(self):
        out = np.zeros(self.T, np.int64)
        _check(lib().pie_problem_perm(self.handle, _ptr(out, ctypes.c_int64)))
        return out

    def level(self, l):
        nb, nl = ctypes.c_int64(), ctypes.c_int64()
        null64 = ctypes.POINTER(ctypes.c_int64)()
        _check(lib().pie_problem_level(self.handle, l, ctypes.byref(nb), ctypes.byref(nl), null64, null64,
                                       null64, ctypes.POINTER(ctypes.c_int32)()))
        keys = np.zeros(nb.value, np.int64)
        ptr = np.zeros(nb.value + 1, np.int64)
        idx = np.zeros(nl.value, np.int64)
        off = np.zeros(nl.value, np.int32)
        _check(lib().pie_problem_level(self.handle, l, ctypes.byref(nb), ctypes.byref(nl),
                                       _ptr(keys, ctypes.c_int64), _ptr(ptr, ctypes.c_int64),
                                       _ptr(idx, ctypes.c_int64), _ptr(off, ctypes.c_int32)))
        return keys, ptr, idx, off

    def near(self):
        nl = ctypes.c_int64()
        null64 = ctypes.POINTER(ctypes.c_int64)()
        _check(lib().pie_problem_near(self.handle, ctypes.byref(nl), null64, null64))
        ptr = np.zeros(self.boxes[self.L] + 1, np.int64)
        idx = np.zeros(nl.value, np.int64)
        _check(lib().pie_problem_near(self.handle, ctypes.byref(nl), _ptr(ptr, ctypes.c_int64),
                                      _ptr(idx, ctypes.c_int64)))
        return ptr, idx

    def apply(self, x, y=None, stream=None, near_only=False):
        """y = Z x for device tensors of shape [N] or [nrhs, N] (row j = right-hand
        side j); near_only=True applies the near part Z_near alone."""
        import torch
        x = _dense(x)
        assert x.is_cuda and x.dtype == self.torch_dtype
        if y is None:
            y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        assert x.shape[-1] == self.N and y.shape == x.shape and y.is_contiguous()
        fn = lib().pie_apply_near if near_only else lib().pie_apply
        _check(fn(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), nrhs,
                  self.dtype_code, _stream(stream)))
        return y

    def apply_levels(self, x, levels, near=False, y=None, stream=None):
        """y = [Z_near x] + sum over `levels` of Z_l x (pie_apply_levels): the
        part of the product translated at the given tree levels."""
        import torch
        x = _dense(x)
        assert x.is_cuda and x.dtype == self.torch_dtype and x.dim() == 1 and x.shape[0] == self.N
        if y is None:
            y = torch.empty_like(x)
        mask = 0
        for l in levels:
            mask |= 1 << int(l)
        _check(lib().pie_apply_levels(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      mask, 1 if near else 0, self.dtype_code, _stream(stream)))
        return y

    def profile_begin(self, max_applies):
        _check(lib().pie_profile_begin(self.handle, max_applies))

    def profile_end(self):
        """Summed milliseconds per stage of the products recorded since profile_begin."""
        ms = np.zeros(len(STAGES), np.float64)
        n = ctypes.c_int32()
        _check(lib().pie_profile_end(self.handle, _ptr(ms, ctypes.c_double), ctypes.byref(n)))
        return dict(zip(STAGES, ms.tolist())), n.value

    def apply_t(self, x, conj=False, y=None, stream=None):
        """y = Z^T x, or Z^H x with conj=True (pie_apply_t)."""
        import torch
        x = _dense(x)
        assert x.is_cuda and x.dtype == self.torch_dtype
        if y is None:
            y = torch.empty_like(x)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        _check(lib().pie_apply_t(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), nrhs,
                                 self.dtype_code, 1 if conj else 0, _stream(stream)))
        return y

    def farfield_adjoint(self, E, rhat, stream=None):
        """u = F^H E (pie_farfield_adjoint)."""
        import torch
        rh = np.ascontiguousarray(rhat, np.float64)
        E = _dense(E)
        u = torch.empty(self.N, dtype=self.torch_dtype, device="cuda")
        _check(lib().pie_farfield_adjoint(self.handle, _ptr(rh, ctypes.c_double), rh.shape[0],
                                          ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                          _stream(stream)))
        return u

    def apply_single_layer(self, q, stream=None):
        """y = S q, S_tu = <p_t, g, p_u> (the operator of Eq. (3))."""
        import torch
        q = _dense(q)
        y = torch.empty_like(q)
        _check(lib().pie_apply_single_layer(self.handle, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                            _stream(stream)))
        return y

    def solve_single_layer(self, b, tol=1e-6, maxit=2000, restart=300, stream=None):
        """GMRES on S q = b (Eq. (3))."""
        import torch
        b = _dense(b)
        x = torch.zeros_like(b)
        st = SolveStats()
        code = lib().pie_solve_single_layer(self.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                            tol, maxit, restart, ctypes.byref(st), _stream(stream))
        if code not in (0, 8):
            _check(code)
        return x, dict(iterations=st.iterations, rel_residual=st.rel_residual, seconds=st.seconds,
                       converged=code == 0, reorthogonalizations=st.reorthogonalizations,
                       product_seconds=st.product_seconds)

    def rhs_potential(self, khat, pol, E0=1.0, stream=None):
        """b_t = <p_t, Phi^inc> for the plane wave (right-hand side of Eq. (3))."""
        import torch
        b = torch.empty(self.T, dtype=torch.complex128, device="cuda")
        kh = np.ascontiguousarray(khat, np.float64)
        po = np.ascontiguousarray(pol, np.float64)
        _check(lib().pie_rhs_potential(self.handle, _ptr(kh, ctypes.c_double), _ptr(po, ctypes.c_double), E0,
                                       ctypes.c_void_p(b.data_ptr()), _stream(stream)))
        return b

    def nearfield(self, x, rho, pts, stream=None):
        """Scattered E at points off the surface from the solution x and the
        charge-density pulse coefficients rho."""
        import torch
        x = _dense(x)
        rho = _dense(rho)
        p = np.ascontiguousarray(pts, np.float64)
        E = torch.empty((p.shape[0], 3), dtype=torch.complex128, device="cuda")
        _check(lib().pie_nearfield(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                   _ptr(p, ctypes.c_double), p.shape[0], ctypes.c_void_p(E.data_ptr()),
                                   _stream(stream)))
        return E

    def stage(self, which, level=0, stream=None):
        if which in (0, 1):
            n = self.boxes[level] * 5 * self.P
            shape = (self.boxes[level], 5, self.P)
        elif which == 4:
            n = 8 * self.near_pairs
            shape = (8, self.near_pairs)
        elif which == 5:
            n = self.T * self.P // 2
            shape = (self.T, self.P // 2)
        elif which == 6:
            n = self.T * 3 * self.P // 2
            shape = (self.T, 3, self.P // 2)
        else:
            n = self.T * 6
            shape = (self.T, 6)
        out = np.zeros(2 * n, np.float64)
        _check(lib().pie_problem_stage(self.handle, which, level, _ptr(out, ctypes.c_double), _stream(stream)))
        return (out[0::2] + 1j * out[1::2]).reshape(shape)

    def rhs_planewave(self, khat, pol, E0=1.0, stream=None):
        import torch
        b = torch.empty(self.N, dtype=self.torch_dtype, device="cuda")
        kh = np.ascontiguousarray(khat, np.float64)
        po = np.ascontiguousarray(pol, np.float64)
        _check(lib().pie_rhs_planewave(self.handle, _ptr(kh, ctypes.c_double), _ptr(po, ctypes.c_double), E0,
                                       ctypes.c_void_p(b.data_ptr()), self.dtype_code, _stream(stream)))
        return b

    def quadrature(self):
        """Quadrature points [T, 7, 3] and weights [T, 7] of every triangle
        (mesh order; pie_problem_quadrature)."""
        pts = np.zeros((self.T, 7, 3), np.float64)
        wts = np.zeros((self.T, 7), np.float64)
        _check(lib().pie_problem_quadrature(self.handle, _ptr(pts, ctypes.c_double), _ptr(wts, ctypes.c_double)))
        return pts, wts

    def rhs_potentials(self, A_q, Phi_q, stream=None):
        """Right-hand side for incident potentials given at the quadrature
        points: A_q [T, 7, 3], Phi_q [T, 7] complex128 device tensors
        (pie_rhs_potentials)."""
        import torch
        A_q, Phi_q = _dense(A_q), _dense(Phi_q)
        assert A_q.is_cuda and Phi_q.is_cuda and A_q.dtype == torch.complex128 and Phi_q.dtype == torch.complex128
        assert A_q.shape == (self.T, 7, 3) and Phi_q.shape == (self.T, 7)
        b = torch.empty(self.N, dtype=self.torch_dtype, device="cuda")
        _check(lib().pie_rhs_potentials(self.handle, ctypes.c_void_p(A_q.data_ptr()), ctypes.c_void_p(Phi_q.data_ptr()),
                                        ctypes.c_void_p(b.data_ptr()), self.dtype_code, _stream(stream)))
        return b

    def farfield(self, x, rhat, stream=None):
        """E [ndir, 3] for x [N], or [nrhs, ndir, 3] for x [nrhs, N] (pie_farfield)."""
        import torch
        rh = np.ascontiguousarray(rhat, np.float64)
        x = _dense(x)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        shape = (rh.shape[0], 3) if x.dim() == 1 else (nrhs, rh.shape[0], 3)
        E = torch.empty(shape, dtype=torch.complex128, device="cuda")
        if nrhs == 0:
            return E
        _check(lib().pie_farfield(self.handle, ctypes.c_void_p(x.data_ptr()), _ptr(rh, ctypes.c_double),
                                  rh.shape[0], ctypes.c_void_p(E.data_ptr()), nrhs, _stream(stream)))
        return E

    def solve(self, b, tol=1e-6, maxit=1000, restart=100, stream=None, x0=None):
        """Restarted GMRES on Z x = b (pie_solve; pie_solve_guess from the
        initial guess x0 when given).  b [N] gives (x, stats); b [nrhs, N]
        gives (x [nrhs, N], [stats per column])."""
        import torch
        b = _dense(b)
        x = torch.zeros_like(b) if x0 is None else _dense(x0).clone()
        assert x.shape == b.shape and x.dtype == b.dtype
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        st = (SolveStats * max(nrhs, 1))()
        if nrhs == 0:
            return x, []
        fn = lib().pie_solve if x0 is None else lib().pie_solve_guess
        code = fn(self.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs, tol, maxit, restart,
                  st, _stream(stream))
        if code not in (0, 8):
            _check(code)
        stats = [dict(iterations=s.iterations, rel_residual=s.rel_residual, seconds=s.seconds,
                      converged=s.rel_residual <= tol, reorthogonalizations=s.reorthogonalizations,
                      product_seconds=s.product_seconds) for s in st[:nrhs]]
        return (x, stats[0]) if b.dim() == 1 else (x, stats)

    def solve_nested(self, b, inner, tol=1e-6, maxit=30000, inner_restart=20, inner_tol=0.05, outer_restart=80,
                     max_outer=1000, stream=None):
        """Nested mixed-precision solve (pie_solve_nested): flexible GMRES on
        this problem's operator, each outer step preconditioned by one GMRES
        cycle on `inner` (a Problem on the same mesh and k0, typically
        PIE_FP32 at a cheap (tau, kappa_a, ntheta)).  b [N] gives (x, stats);
        b [nrhs, N] gives (x [nrhs, N], [stats per column])."""
        import torch
        b = _dense(b)
        x = torch.zeros_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        st = (NestedStats * max(nrhs, 1))()
        if nrhs == 0:
            return x, []
        p = NestedParams(tol, maxit, inner_restart, inner_tol, outer_restart, max_outer)
        code = lib().pie_solve_nested(self.handle, inner.handle, ctypes.c_void_p(b.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), nrhs, ctypes.byref(p), st, _stream(stream))
        if code not in (0, 8):
            _check(code)
        stats = [dict(inner_iterations=s.inner_iterations, outer_iterations=s.outer_iterations,
                      outer_products=s.outer_products, rel_residual=s.rel_residual, seconds=s.seconds,
                      inner_product_seconds=s.inner_product_seconds, outer_product_seconds=s.outer_product_seconds,
                      converged=s.rel_residual <= tol) for s in st[:nrhs]]
        return (x, stats[0]) if b.dim() == 1 else (x, stats)

    @property
    def tuning(self):
        """Launch settings of the product (pie_problem_get_tuning), as a dict."""
        t = Tuning()
        _check(lib().pie_problem_get_tuning(self.handle, ctypes.byref(t)))
        return t.as_dict()

    @tuning.setter
    def tuning(self, d):
        t = Tuning(**{**self.tuning, **d})
        _check(lib().pie_problem_set_tuning(self.handle, ctypes.byref(t)))

    def autotune(self, nrhs=1, reps=5, stream=None):
        """Time the launch settings and keep the fastest (pie_problem_autotune);
        returns (settings dict, milliseconds per right-hand side)."""
        t = Tuning()
        ms = ctypes.c_double()
        _check(lib().pie_problem_autotune(self.handle, nrhs, reps, ctypes.byref(t), ctypes.byref(ms),
                                          _stream(stream)))
        return t.as_dict(), ms.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pie_problem_destroy(self.handle)
            self.handle = None


def tune_levels(mesh, k0, lmin, lmax, nrhs=1, root_side=0.0, tau=DEFAULT_TAU, kappa_a=DEFAULT_KAPPA_A,
                ntheta=DEFAULT_NTHETA, precision=PIE_FP64, max_nrhs=1, stream=None):
    """Level count with the fastest autotuned product for this mesh
    (pie_tune_levels); returns (L, {L: ms per right-hand side})."""
    p = Params(lmin, root_side, tau, kappa_a, ntheta, precision, max_nrhs)
    best = ctypes.c_int32()
    ms = np.zeros(lmax - lmin + 1, np.float64)
    _check(lib().pie_tune_levels(mesh.handle, float(k0), ctypes.byref(p), lmin, lmax, nrhs, _stream(stream),
                                 ctypes.byref(best), _ptr(ms, ctypes.c_double)))
    return best.value, {lmin + i: float(v) for i, v in enumerate(ms) if v > 0}


def measure_peaks(stream=None):
    """FP64 and FP32 fused multiply-add throughput of the current device
    (pie_measure_peaks): dict with TFLOP/s and the SM clock (MHz) each probe
    ran at."""
    f64, f32, m64, m32 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pie_measure_peaks(ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(m64), ctypes.byref(m32),
                                   _stream(stream)))
    return dict(fp64_tflops=f64.value, fp32_tflops=f32.value, fp64_mhz=m64.value, fp32_mhz=m32.value)


class Group:
    """Several problems applied in one CUDA-graph launch (pie_group_*)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p.handle for p in self.problems])
        h = ctypes.c_void_p()
        _check(lib().pie_group_create(arr, len(self.problems), ctypes.byref(h)))
        self.handle = h

    def apply(self, xs, ys, stream=None):
        """ys[i] = Z_i xs[i] for all members at once; xs[i], ys[i]: device
        tensors [nrhs, N_i] (the same nrhs for all).  Keep ys (and xs) alive
        and reuse them: the captured graph is tied to their addresses."""
        xs = [_dense(x) for x in xs]
        nrhs = xs[0].shape[0] if xs[0].dim() == 2 else 1
        for p, x, y in zip(self.problems, xs, ys):
            assert x.is_cuda and y.is_cuda and x.dtype == p.torch_dtype and y.dtype == p.torch_dtype
            assert x.numel() == nrhs * p.N and y.numel() == nrhs * p.N and y.is_contiguous()
        xa = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        _check(lib().pie_group_apply(self.handle, xa, ya, nrhs, _stream(stream)))
        return ys

    def info(self):
        g, n = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pie_group_info(self.handle, ctypes.byref(g), ctypes.byref(n)))
        return dict(graphs=g.value, launches=n.value)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.pie_group_destroy(self.handle)
            self.handle = None
