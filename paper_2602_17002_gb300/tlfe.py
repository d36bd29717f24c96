"""Python binding of libtlfe (ctypes): argument marshalling only.

Every computation happens in the CUDA library; this module checks tensor
shapes/dtypes/devices, passes raw device pointers and the current CUDA stream,
and turns non-zero status codes into exceptions. The function names mirror the
C ABI in include/tlfe.h.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# TLFE_LIB may name another build of the library, e.g. the bounds-checked
# _build/libtlfe_checked.so (build_lib.build(checked=True))
LIB_PATH = os.environ.get("TLFE_LIB") or os.path.join(HERE, "_build", "libtlfe.so")

T4, T10, H8, Q27 = 0, 1, 2, 3
SVK, NEOHOOKE, MOONEY_RIVLIN = 0, 1, 2
FP64, FP32 = 0, 1
SCATTER_ATOMIC, SCATTER_COLOR, SCATTER_SORTED = 0, 1, 2
PATH_AUTO, PATH_SLAB, PATH_AFFINE = 0, 1, 2
LAUNCH_AUTO, LAUNCH_PER_PASS, LAUNCH_FUSED = 0, 1, 2
PATCH_BANKED, PATCH_SORTED = 0, 1
NPE = {T4: 4, T10: 10, H8: 8, Q27: 27}

STATUS = {0: "TLFE_OK", 1: "TLFE_E_INVALID", 2: "TLFE_E_OOM", 3: "TLFE_E_CUDA", 4: "TLFE_E_INVERTED",
          5: "TLFE_E_NOT_CONVERGED", 6: "TLFE_E_TIMEOUT", 7: "TLFE_E_UNSUPPORTED", 8: "TLFE_E_NONFINITE"}


class TLFEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class tlfe_block(C.Structure):
    _fields_ = [("type", C.c_int32), ("n_elem", C.c_int32), ("n_qp", C.c_int32),
                ("conn", C.c_void_p), ("body", C.c_void_p)]


class tlfe_material(C.Structure):
    _fields_ = [("model", C.c_int32), ("mu", C.c_double), ("lambda_", C.c_double),
                ("mu_v", C.c_double), ("lambda_v", C.c_double), ("rho", C.c_double), ("mu01", C.c_double)]


class tlfe_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("X_ref", C.c_void_p), ("n_blocks", C.c_int32),
                ("blocks", C.c_void_p), ("n_bodies", C.c_int32), ("body_mat", C.c_void_p),
                ("elem_mu_lambda", C.c_void_p), ("precision", C.c_int32), ("scatter", C.c_int32),
                ("color_seed", C.c_uint64), ("element_path", C.c_int32), ("patch_layout", C.c_int32)]


class tlfe_mesh_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_elem", C.c_int32), ("n_blocks", C.c_int32),
                ("n_colors", C.c_int32), ("precision", C.c_int32), ("scatter", C.c_int32),
                ("n_qp", C.c_int64), ("stream_bytes_force", C.c_int64),
                ("stream_bytes_matvec", C.c_int64), ("stream_bytes_vjp", C.c_int64),
                ("device_bytes", C.c_int64), ("n_affine_blocks", C.c_int32), ("n_passes", C.c_int32),
                ("n_fused_passes", C.c_int32), ("n_fused_items", C.c_int32), ("launches_force", C.c_int32),
                ("launches_matvec", C.c_int32), ("patch_layout", C.c_int32), ("patch_passes", C.c_double),
                ("force_matvec_fused", C.c_int32), ("stream_bytes_force_matvec", C.c_int64)]


class tlfe_step_params(C.Structure):
    _fields_ = [("h", C.c_double), ("gravity", C.c_double * 3), ("newton_rtol", C.c_double),
                ("cg_rtol", C.c_double), ("max_newton", C.c_int32), ("max_cg", C.c_int32),
                ("fixed_dev", C.c_void_p), ("use_graph", C.c_int32), ("f_ext_dev", C.c_void_p),
                ("n_cons", C.c_int32), ("cons_dev", C.c_void_p), ("rho", C.c_double), ("alm_tol", C.c_double),
                ("max_outer", C.c_int32), ("lambda_dev", C.c_void_p)]


class tlfe_step_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("cg_iters", C.c_int32), ("status", C.c_int32),
                ("n_bodies_converged", C.c_int32), ("rel_residual", C.c_double), ("outer_iters", C.c_int32),
                ("c_norm", C.c_double)]


class tlfe_host_step(C.Structure):
    _fields_ = [("u_host", C.c_void_p), ("udot_host", C.c_void_p), ("v_host", C.c_void_p),
                ("cot_host", C.c_void_p), ("a_M", C.c_double), ("a_K", C.c_double), ("a_C", C.c_double),
                ("f_host", C.c_void_p), ("y_host", C.c_void_p), ("g_u_host", C.c_void_p),
                ("g_udot_host", C.c_void_p), ("g_mu_lambda_host", C.c_void_p)]


# bilateral constraint records (tlfe_constraint): points P, Q[, R, T] as (global
# element, parent coordinates); element < 0 = ground point at world coordinates
CON_CD, CON_DIST, CON_DP1, CON_DP2 = 0, 1, 2, 3
CON_DTYPE = np.dtype([("type", np.int32), ("elem", np.int32, (4,)), ("xi", np.float64, (4, 3)),
                      ("d", np.float64, (3,)), ("f", np.float64)], align=True)



class tlfe_split_cg(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_rows", C.c_int32), ("fixed", C.c_void_p), ("own", C.c_void_p),
                ("x", C.c_void_p), ("r", C.c_void_p), ("p", C.c_void_p), ("q", C.c_void_p),
                ("dinv", C.c_void_p), ("work", C.c_void_p), ("dots", C.c_void_p)]


_lib = None

EXPORTS = ["tlfe_create_mesh", "tlfe_destroy_mesh", "tlfe_get_mesh_info", "tlfe_get_colors",
           "tlfe_get_scatter_targets", "tlfe_set_launch_mode", "tlfe_force_matvec", "tlfe_step_host",
           "tlfe_step_host_wait", "tlfe_peak_probe", "tlfe_gather_nodes",
           "tlfe_scatter_nodes", "tlfe_sync",
           "tlfe_internal_force", "tlfe_internal_force_host", "tlfe_tangent_matvec", "tlfe_jacobi_diag",
           "tlfe_vjp", "tlfe_set_elem_mu_lambda", "tlfe_autotune", "tlfe_point_loads", "tlfe_surface_traction",
           "tlfe_constraint_eval", "tlfe_constraint_jt", "tlfe_constraint_j", "tlfe_newton_step", "tlfe_body_norms", "tlfe_norm_noalloc", "tlfe_selftest_wait_timeout", "tlfe_last_error",
           "tlfe_version", "tlfe_newton_operator", "tlfe_split_work_doubles", "tlfe_split_prep",
           "tlfe_split_residual", "tlfe_split_velocity", "tlfe_split_dot", "tlfe_split_cg_dinv",
           "tlfe_split_cg_start", "tlfe_split_cg_pq", "tlfe_split_cg_update", "tlfe_split_cg_direction"]


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libtlfe.so. Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtlfe.so not built at {path}; run __graft_entry__.build() "
                          "(the TL-FEA path has no CPU fallback)")
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "tlfe_create_mesh": [C.POINTER(tlfe_mesh_desc), P, C.POINTER(P)],
        "tlfe_destroy_mesh": [P],
        "tlfe_get_mesh_info": [P, C.POINTER(tlfe_mesh_info)],
        "tlfe_get_colors": [P, P],
        "tlfe_get_scatter_targets": [P, P, P],
        "tlfe_set_launch_mode": [P, I],
        "tlfe_step_host": [P, C.POINTER(tlfe_host_step), P],
        "tlfe_step_host_wait": [P],
        "tlfe_peak_probe": [I, I, C.c_int64, P, C.POINTER(C.c_double), P],
        "tlfe_gather_nodes": [I, P, P, I, P, P, I, P],
        "tlfe_scatter_nodes": [I, P, P, P, I, P, P],
        "tlfe_force_matvec": [P, P, P, P, D, D, D, P, P, P],
        "tlfe_sync": [P, P, C.POINTER(C.c_int64)],
        "tlfe_internal_force": [P, P, P, P, P],
        "tlfe_internal_force_host": [P, P, P, P, P],
        "tlfe_tangent_matvec": [P, P, P, P, D, D, D, P, P],
        "tlfe_jacobi_diag": [P, P, P, D, D, D, P, P],
        "tlfe_vjp": [P, P, P, P, P, P, P, P],
        "tlfe_newton_step": [P, P, P, C.POINTER(tlfe_step_params), P, C.POINTER(tlfe_step_report), P],
        "tlfe_body_norms": [P, P, P, P],
        "tlfe_set_elem_mu_lambda": [P, P, P],
        "tlfe_autotune": [P, P, P, P, P],
        "tlfe_point_loads": [P, I, P, P, P, P, P],
        "tlfe_surface_traction": [P, I, P, P, P, P, P],
        "tlfe_constraint_eval": [P, I, P, P, P, P],
        "tlfe_constraint_jt": [P, I, P, P, P, P, P],
        "tlfe_constraint_j": [P, I, P, P, P, P, P],
        "tlfe_norm_noalloc": [P, C.c_int64, P, P],
        "tlfe_selftest_wait_timeout": [P, C.c_int64, P],
        "tlfe_newton_operator": [P, P, P, P, D, D, D, P, P],
        "tlfe_split_prep": [C.POINTER(tlfe_split_cg), D, P, P, P, P, P, P, P, P],
        "tlfe_split_residual": [C.POINTER(tlfe_split_cg), P, P, P, P],
        "tlfe_split_velocity": [C.POINTER(tlfe_split_cg), P, I, P, P],
        "tlfe_split_dot": [C.POINTER(tlfe_split_cg), P, P, P],
        "tlfe_split_cg_dinv": [C.POINTER(tlfe_split_cg), P, P],
        "tlfe_split_cg_start": [C.POINTER(tlfe_split_cg), P, P],
        "tlfe_split_cg_pq": [C.POINTER(tlfe_split_cg), P],
        "tlfe_split_cg_update": [C.POINTER(tlfe_split_cg), D, P],
        "tlfe_split_cg_direction": [C.POINTER(tlfe_split_cg), D, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.tlfe_last_error.restype = C.c_char_p
    L.tlfe_last_error.argtypes = []
    L.tlfe_version.restype = C.c_char_p
    L.tlfe_version.argtypes = []
    L.tlfe_split_work_doubles.restype = C.c_int64
    L.tlfe_split_work_doubles.argtypes = [C.c_int64]
    _lib = L
    return L


def _check(code: int):
    if code != 0:
        raise TLFEError(code, load().tlfe_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


class Mesh:
    """Owner of a tlfe_mesh handle (see include/tlfe.h for the operations)."""

    def __init__(self, X: np.ndarray, blocks: Sequence[tuple], materials: Sequence[tuple],
                 elem_mu_lambda: Optional[np.ndarray] = None, precision: int = FP32,
                 scatter: int = SCATTER_ATOMIC, color_seed: int = 0, stream=None, element_path: int = PATH_AUTO,
                 patch_layout: int = PATCH_BANKED):
        """X: (n_nodes, 3) float64 reference coordinates.
        blocks: (etype, n_qp, conn (n_elem, npe) int32, body (n_elem,) int32 or None).
        materials: per body (model, mu, lam, mu_v, lam_v, rho[, mu01]).
        element_path: PATH_AUTO, PATH_SLAB or PATH_AFFINE; patch_layout: PATCH_BANKED or
        PATCH_SORTED (see include/tlfe.h)."""
        L = load()
        self._keep = []
        X = np.ascontiguousarray(X, dtype=np.float64)
        assert X.ndim == 2 and X.shape[1] == 3
        cb = (tlfe_block * len(blocks))()
        for k, (et, nq, conn, body) in enumerate(blocks):
            conn = np.ascontiguousarray(conn, dtype=np.int32)
            body = None if body is None else np.ascontiguousarray(body, dtype=np.int32)
            self._keep += [conn, body]
            cb[k] = tlfe_block(int(et), int(conn.shape[0]), int(nq), conn.ctypes.data,
                               None if body is None else body.ctypes.data)
        cm = (tlfe_material * len(materials))()
        for k, mt in enumerate(materials):
            vals = [float(x) for x in mt[1:7]] + [0.0] * (7 - len(mt))
            cm[k] = tlfe_material(int(mt[0]), *vals)
        eml = None
        if elem_mu_lambda is not None:
            eml = np.ascontiguousarray(elem_mu_lambda, dtype=np.float64)
            self._keep.append(eml)
        desc = tlfe_mesh_desc(X.shape[0], X.ctypes.data, len(blocks), C.addressof(cb), len(materials),
                              C.addressof(cm), None if eml is None else eml.ctypes.data,
                              int(precision), int(scatter), C.c_uint64(color_seed), int(element_path),
                              int(patch_layout))
        h = C.c_void_p()
        _check(L.tlfe_create_mesh(C.byref(desc), _stream(stream), C.byref(h)))
        self._h = h
        self.precision = precision
        self.n_nodes = X.shape[0]
        self._n_bodies = len(materials)
        self.block_sizes = [tuple(int(x) for x in np.asarray(b[2]).reshape(-1, NPE[int(b[0])]).shape) for b in blocks]
        self.info = self.get_info()
        self._keep = None

    @classmethod
    def from_workload(cls, wl, precision=FP32, scatter=SCATTER_ATOMIC, color_seed=0, stream=None,
                      element_path=PATH_AUTO, patch_layout=PATCH_BANKED):
        blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
        mats = [(int(wl.model[k]), *wl.params[k]) for k in range(wl.n_bodies)]
        return cls(wl.X, blocks, mats, wl.elem_mu_lambda, precision, scatter, color_seed, stream, element_path,
                   patch_layout)

    @property
    def handle(self):
        return self._h

    @property
    def torch_dtype(self):
        import torch
        return torch.float32 if self.precision == FP32 else torch.float64

    def get_info(self) -> dict:
        info = tlfe_mesh_info()
        _check(load().tlfe_get_mesh_info(self._h, C.byref(info)))
        return {k: getattr(info, k) for k, _ in tlfe_mesh_info._fields_}

    def colors(self) -> np.ndarray:
        out = np.zeros(self.info["n_elem"], np.int32)
        _check(load().tlfe_get_colors(self._h, out.ctypes.data))
        return out

    def scatter_targets(self):
        """(gather, scatter): per block, (n_elem, nodes) int32 arrays of the
        node each (element, local node) is gathered from and scattered to by
        the element kernels' device tables (tlfe_get_scatter_targets)."""
        sizes = self.block_sizes
        total = sum(n * npe for n, npe in sizes)
        g = np.full(total, -2, np.int32)
        s = np.full(total, -2, np.int32)
        _check(load().tlfe_get_scatter_targets(self._h, g.ctypes.data, s.ctypes.data))
        out_g, out_s, off = [], [], 0
        for n, npe in sizes:
            out_g.append(g[off:off + n * npe].reshape(n, npe))
            out_s.append(s[off:off + n * npe].reshape(n, npe))
            off += n * npe
        return out_g, out_s

    def set_launch_mode(self, mode):
        """LAUNCH_AUTO, LAUNCH_PER_PASS or LAUNCH_FUSED (tlfe_set_launch_mode)."""
        _check(load().tlfe_set_launch_mode(self._h, int(mode)))
        self.info = self.get_info()

    def force_matvec(self, u, udot, v, a_M=0.0, a_K=1.0, a_C=0.0, f=None, y=None, stream=None):
        """f = f_int(u, udot) and y = a_M M v + a_K K_t v + a_C C v in one call,
        replayed from a CUDA graph the mesh keeps (tlfe_force_matvec); one pass
        per element block and law where info["force_matvec_fused"] is 1."""
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        self._node_array(v, "v")
        f = self._new() if f is None else self._node_array(f, "f")
        y = self._new() if y is None else self._node_array(y, "y")
        _check(load().tlfe_force_matvec(self._h, _ptr(u), _ptr(udot), _ptr(v), float(a_M), float(a_K), float(a_C),
                                        _ptr(f), _ptr(y), _stream(stream)))
        return f, y

    def step_host(self, u, udot=None, v=None, cot=None, f=None, y=None, g_u=None, g_udot=None,
                  g_mu_lambda=None, a_M=0.0, a_K=1.0, a_C=0.0, stream=None):
        """Host-buffer element operations (tlfe_step_host): every array is a
        contiguous CPU torch tensor or numpy array (pinned memory lets the
        copies overlap); u float64 (n_nodes, 3), the other node arrays in the
        mesh dtype, g_mu_lambda float64 (n_elem, 2). Asynchronous: the outputs
        are complete after step_host_wait()."""
        import torch
        dt = np.float32 if self.precision == FP32 else np.float64

        def ptr(a, dtype, shape, name):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                ok = (not a.is_cuda and a.is_contiguous() and tuple(a.shape) == shape
                      and a.dtype == (torch.float32 if dtype == np.float32 else torch.float64))
                p = a.data_ptr()
            else:
                ok = a.dtype == dtype and a.flags.c_contiguous and a.shape == shape
                p = a.ctypes.data
            if not ok:
                raise TLFEError(1, f"{name} must be a contiguous host array {shape} of {np.dtype(dtype).name}")
            return p
        n3 = (self.n_nodes, 3)
        args = tlfe_host_step(ptr(u, np.float64, n3, "u"), ptr(udot, dt, n3, "udot"), ptr(v, dt, n3, "v"),
                              ptr(cot, dt, n3, "cot"), float(a_M), float(a_K), float(a_C),
                              ptr(f, dt, n3, "f"), ptr(y, dt, n3, "y"), ptr(g_u, dt, n3, "g_u"),
                              ptr(g_udot, dt, n3, "g_udot"),
                              ptr(g_mu_lambda, np.float64, (self.info["n_elem"], 2), "g_mu_lambda"))
        _check(load().tlfe_step_host(self._h, C.byref(args), _stream(stream)))

    def step_host_wait(self):
        _check(load().tlfe_step_host_wait(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().tlfe_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- checks
    def _node_array(self, t, name, dtype=None):
        import torch
        if t is None:
            return None
        dt = dtype or self.torch_dtype
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()
                and tuple(t.shape) == (self.n_nodes, 3)):
            raise TLFEError(1, f"{name} must be a contiguous CUDA {dt} tensor of shape ({self.n_nodes}, 3)")
        return t

    def _new(self, dtype=None):
        import torch
        return torch.empty((self.n_nodes, 3), dtype=dtype or self.torch_dtype, device="cuda")

    # ---- operations (outputs are allocated when not given)
    def sync(self, stream=None) -> int:
        n = C.c_int64(0)
        _check(load().tlfe_sync(self._h, _stream(stream), C.byref(n)))
        return n.value

    def selftest_wait_timeout(self, spin_limit=4096, stream=None):
        """Run a bounded device wait that cannot complete
        (tlfe_selftest_wait_timeout); the next sync() raises TLFEError with
        TLFE_E_TIMEOUT (6) and the mesh stays usable."""
        _check(load().tlfe_selftest_wait_timeout(self._h, int(spin_limit), _stream(stream)))

    def internal_force(self, u, udot=None, out=None, stream=None):
        """u: (n_nodes, 3) float64 displacement (FP64 in both precisions); udot
        and the returned force are in the mesh dtype."""
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        out = self._new() if out is None else self._node_array(out, "out")
        _check(load().tlfe_internal_force(self._h, _ptr(u), _ptr(udot), _ptr(out), _stream(stream)))
        return out

    def internal_force_host(self, u: np.ndarray, udot: Optional[np.ndarray], out: np.ndarray, stream=None):
        """Host-buffer call: u (float64), udot and out (mesh dtype) are contiguous
        numpy arrays of shape (n_nodes, 3)."""
        dt = np.float32 if self.precision == FP32 else np.float64
        if u.dtype != np.float64 or not u.flags.c_contiguous or u.shape != (self.n_nodes, 3):
            raise TLFEError(1, "u must be a contiguous float64 (n_nodes, 3) array")
        for a in (udot, out):
            if a is not None and (a.dtype != dt or not a.flags.c_contiguous or a.shape != (self.n_nodes, 3)):
                raise TLFEError(1, "host arrays must be contiguous (n_nodes, 3) of the mesh dtype")
        _check(load().tlfe_internal_force_host(self._h, u.ctypes.data, None if udot is None else udot.ctypes.data,
                                               out.ctypes.data, _stream(stream)))
        return out

    def internal_force_host_ptr(self, u_ptr: int, udot_ptr: Optional[int], out_ptr: int, stream=None):
        _check(load().tlfe_internal_force_host(self._h, C.c_void_p(u_ptr),
                                               None if udot_ptr is None else C.c_void_p(udot_ptr),
                                               C.c_void_p(out_ptr), _stream(stream)))

    def tangent_matvec(self, u, udot, v, a_M=0.0, a_K=1.0, a_C=0.0, out=None, stream=None):
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        self._node_array(v, "v")
        out = self._new() if out is None else self._node_array(out, "out")
        _check(load().tlfe_tangent_matvec(self._h, _ptr(u), _ptr(udot), _ptr(v), float(a_M), float(a_K),
                                          float(a_C), _ptr(out), _stream(stream)))
        return out

    def newton_operator(self, u, udot, v, a_M=0.0, a_K=1.0, a_C=0.0, out=None, stream=None):
        """y = a_M M v + a_K K^e v + a_C C v, the symmetric CG operator of the
        Newton step (tlfe_newton_operator)."""
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        self._node_array(v, "v")
        out = self._new() if out is None else self._node_array(out, "out")
        _check(load().tlfe_newton_operator(self._h, _ptr(u), _ptr(udot), _ptr(v), float(a_M), float(a_K),
                                           float(a_C), _ptr(out), _stream(stream)))
        return out

    def jacobi_diag(self, u, udot=None, a_M=0.0, a_K=1.0, a_C=0.0, out=None, stream=None):
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        out = self._new() if out is None else self._node_array(out, "out")
        _check(load().tlfe_jacobi_diag(self._h, _ptr(u), _ptr(udot), float(a_M), float(a_K), float(a_C),
                                       _ptr(out), _stream(stream)))
        return out

    def autotune(self, u, udot=None, v=None, stream=None):
        """Pick launch schedules by measurement (tlfe_autotune); u float64 (n_nodes, 3),
        udot / v in the mesh dtype or None."""
        import torch
        self._node_array(u, "u", torch.float64)
        if udot is not None:
            self._node_array(udot, "udot")
        if v is not None:
            self._node_array(v, "v")
        _check(load().tlfe_autotune(self._h, _ptr(u), _ptr(udot), _ptr(v), _stream(stream)))
        self.info = self.get_info()   # the tuner may switch between fused and per-pass launches

    def set_elem_mu_lambda(self, theta, stream=None):
        """theta: contiguous CUDA float64 tensor (n_elem, 2) of per-element (mu, lambda)."""
        import torch
        if not (theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()
                and tuple(theta.shape) == (self.info["n_elem"], 2)):
            raise TLFEError(1, f"theta must be a contiguous CUDA float64 tensor ({self.info['n_elem']}, 2)")
        _check(load().tlfe_set_elem_mu_lambda(self._h, _ptr(theta), _stream(stream)))

    def vjp(self, u, udot, cot, want_u=True, want_udot=True, want_theta=True, stream=None):
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(udot, "udot")
        self._node_array(cot, "cot")
        gu = self._new() if want_u else None
        gud = self._new() if want_udot else None
        gth = torch.empty((self.info["n_elem"], 2), dtype=torch.float64, device="cuda") if want_theta else None
        _check(load().tlfe_vjp(self._h, _ptr(u), _ptr(udot), _ptr(cot), _ptr(gu), _ptr(gud), _ptr(gth),
                               _stream(stream)))
        return gu, gud, gth

    def body_norms(self, x, out=None, stream=None):
        """Per-body 2-norms of a (n_nodes, 3) float64 CUDA tensor."""
        import torch
        self._node_array(x, "x", torch.float64)
        out = torch.empty(self._n_bodies, dtype=torch.float64, device="cuda") if out is None else out
        _check(load().tlfe_body_norms(self._h, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def point_loads(self, elem, xi, force, out=None, stream=None):
        """Add s_i(xi_k) force_k (Sec. 4, pointwise loads) into out (float64
        (n_nodes, 3), zeros when None): elem (k,) int32 global element ids,
        xi (k, 3) parent coordinates, force (k, 3), CUDA float64."""
        import torch
        out = self._new(torch.float64).zero_() if out is None else out
        self._node_array(out, "out", torch.float64)
        n = int(elem.numel())
        _check(load().tlfe_point_loads(self._h, n, _ptr(elem), _ptr(xi), _ptr(force), _ptr(out), _stream(stream)))
        return out

    def surface_traction(self, elem, face, t0, out=None, stream=None):
        """Add int s_i t0 dA0 (Sec. 4, surface tractions) into out: face k is
        local face face[k] of global element elem[k] (both int32), t0 (k, 3)
        nominal traction, CUDA float64."""
        import torch
        out = self._new(torch.float64).zero_() if out is None else out
        self._node_array(out, "out", torch.float64)
        n = int(elem.numel())
        _check(load().tlfe_surface_traction(self._h, n, _ptr(elem), _ptr(face), _ptr(t0), _ptr(out),
                                            _stream(stream)))
        return out

    def _cons(self, cons):
        """(device bytes tensor, count) of a CON_DTYPE array (numpy, host)."""
        import torch
        arr = np.ascontiguousarray(cons, dtype=CON_DTYPE)
        return torch.from_numpy(arr.view(np.uint8).copy()).cuda(), int(arr.shape[0])

    def constraint_eval(self, cons, u, stream=None):
        """c_k(X + u) of the constraint records (Sec. 3 primitives), float64 CUDA (n,)."""
        import torch
        self._node_array(u, "u", torch.float64)
        dc, n = self._cons(cons)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(load().tlfe_constraint_eval(self._h, n, _ptr(dc), _ptr(u), _ptr(out), _stream(stream)))
        return out

    def constraint_jt(self, cons, u, w, out=None, stream=None):
        """out += C_q^T w (float64 (n_nodes, 3); zeros when None)."""
        import torch
        self._node_array(u, "u", torch.float64)
        out = self._new(torch.float64).zero_() if out is None else out
        dc, n = self._cons(cons)
        _check(load().tlfe_constraint_jt(self._h, n, _ptr(dc), _ptr(u), _ptr(w), _ptr(out), _stream(stream)))
        return out

    def constraint_j(self, cons, u, v, stream=None):
        """C_q v, float64 CUDA (n,)."""
        import torch
        self._node_array(u, "u", torch.float64)
        self._node_array(v, "v", torch.float64)
        dc, n = self._cons(cons)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(load().tlfe_constraint_j(self._h, n, _ptr(dc), _ptr(u), _ptr(v), _ptr(out), _stream(stream)))
        return out

    def newton_step(self, u_n, v_n, h, gravity=(0.0, 0.0, -9.81), fixed=None, newton_rtol=1e-8, cg_rtol=1e-4,
                    max_newton=20, max_cg=1000, use_graph=True, v_out=None, stream=None, f_ext=None,
                    constraints=None, rho=1.0, alm_tol=1e-10, max_outer=20, lam=None):
        """Backward-Euler step (tlfe_newton_step). With constraints (a CON_DTYPE
        array) it is the augmented-Lagrangian step; lam (float64 CUDA (n,),
        zeros when None) carries the multipliers in and out."""
        import torch
        self._node_array(u_n, "u_n", torch.float64)
        self._node_array(v_n, "v_n", torch.float64)
        if f_ext is not None:
            self._node_array(f_ext, "f_ext", torch.float64)
        v_out = self._new(torch.float64) if v_out is None else v_out
        if fixed is not None and not (fixed.is_cuda and fixed.dtype == torch.uint8 and fixed.numel() == self.n_nodes):
            raise TLFEError(1, "fixed must be a CUDA uint8 tensor with one entry per node")
        dc, n_cons = (None, 0) if constraints is None else self._cons(constraints)
        if n_cons and lam is None:
            lam = torch.zeros(n_cons, dtype=torch.float64, device="cuda")
        p = tlfe_step_params(float(h), (C.c_double * 3)(*[float(g) for g in gravity]), float(newton_rtol),
                             float(cg_rtol), int(max_newton), int(max_cg), _ptr(fixed), int(bool(use_graph)),
                             _ptr(f_ext), n_cons, _ptr(dc), float(rho), float(alm_tol), int(max_outer),
                             _ptr(lam if n_cons else None))
        rep = tlfe_step_report()
        code = load().tlfe_newton_step(self._h, _ptr(u_n), _ptr(v_n), C.byref(p), _ptr(v_out), C.byref(rep),
                                       _stream(stream))
        report = {k: getattr(rep, k) for k, _ in tlfe_step_report._fields_}
        if n_cons:
            report["lam"] = lam
        if code not in (0, 5):
            _check(code)
        report["code"] = code
        return v_out, report


# ---- C-ABI-named module functions -------------------------------------------

def tlfe_create_mesh(*args, **kw) -> Mesh:
    return Mesh(*args, **kw)


def tlfe_destroy_mesh(mesh: Mesh):
    mesh.close()


def tlfe_internal_force(mesh: Mesh, u, udot, f, stream=None):
    return mesh.internal_force(u, udot, out=f, stream=stream)


def tlfe_internal_force_host(mesh: Mesh, u, udot, f, stream=None):
    return mesh.internal_force_host(u, udot, f, stream=stream)


def tlfe_tangent_matvec(mesh: Mesh, u, udot, v, a_M, a_K, a_C, y, stream=None):
    return mesh.tangent_matvec(u, udot, v, a_M, a_K, a_C, out=y, stream=stream)


def tlfe_jacobi_diag(mesh: Mesh, u, udot, a_M, a_K, a_C, d, stream=None):
    return mesh.jacobi_diag(u, udot, a_M, a_K, a_C, out=d, stream=stream)


def tlfe_vjp(mesh: Mesh, u, udot, cot, stream=None):
    return mesh.vjp(u, udot, cot, stream=stream)


def tlfe_autotune(mesh: Mesh, u, udot=None, v=None, stream=None):
    return mesh.autotune(u, udot, v, stream)


def tlfe_point_loads(mesh: Mesh, elem, xi, force, f, stream=None):
    return mesh.point_loads(elem, xi, force, f, stream)


def tlfe_surface_traction(mesh: Mesh, elem, face, t0, f, stream=None):
    return mesh.surface_traction(elem, face, t0, f, stream)


def tlfe_constraint_eval(mesh: Mesh, cons, u, stream=None):
    return mesh.constraint_eval(cons, u, stream)


def tlfe_constraint_jt(mesh: Mesh, cons, u, w, f, stream=None):
    return mesh.constraint_jt(cons, u, w, f, stream)


def tlfe_constraint_j(mesh: Mesh, cons, u, v, stream=None):
    return mesh.constraint_j(cons, u, v, stream)


def tlfe_set_elem_mu_lambda(mesh: Mesh, theta, stream=None):
    return mesh.set_elem_mu_lambda(theta, stream=stream)


def tlfe_newton_step(mesh: Mesh, u_n, v_n, h, **kw):
    return mesh.newton_step(u_n, v_n, h, **kw)


def tlfe_body_norms(mesh: Mesh, x, out=None, stream=None):
    return mesh.body_norms(x, out=out, stream=stream)


def peak_probe(precision=FP32, ctas_per_sm=4, iters=1 << 16, repeats=5, stream=None):
    """FMA peak of this GPU in TFLOP/s (tlfe_peak_probe, timed with CUDA events
    on the launching stream; best of `repeats` launches after one warm-up)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    out = torch.zeros(2, dtype=torch.float32 if precision == FP32 else torch.float64, device="cuda")
    flop = C.c_double(0.0)
    L = load()
    _check(L.tlfe_peak_probe(int(precision), int(ctas_per_sm), C.c_int64(iters), _ptr(out), C.byref(flop),
                             _stream(s)))
    best = None
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(L.tlfe_peak_probe(int(precision), int(ctas_per_sm), C.c_int64(iters), _ptr(out), C.byref(flop),
                                 _stream(s)))
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return flop.value / (best * 1e-3) / 1e12, best


def _rows_prec(*ts):
    import torch
    prec = {torch.float32: FP32, torch.float64: FP64}.get(ts[0].dtype)
    if prec is None or not all(t.is_cuda and t.dtype == ts[0].dtype and t.is_contiguous() and t.dim() == 2
                               and t.shape[1] == 3 for t in ts):
        raise TLFEError(1, "node rows: contiguous CUDA (n, 3) float32 / float64 arrays of one dtype")
    return prec


def _idx(i, n):
    import torch
    if i is None:
        return None
    if not (i.is_cuda and i.dtype == torch.int32 and i.is_contiguous() and i.numel() == n):
        raise TLFEError(1, "node rows: index arrays are contiguous CUDA int32 of one length")
    return i


def gather_nodes(x, idx, out, out_idx=None, clear=False, stream=None):
    """out[out_idx[k]] = x[idx[k]] (out[k] without out_idx), after zeroing out
    when clear (tlfe_gather_nodes)."""
    prec = _rows_prec(x, out)
    n = int(idx.numel())
    _check(load().tlfe_gather_nodes(prec, _ptr(x), _ptr(_idx(idx, n)), n, _ptr(out), _ptr(_idx(out_idx, n)),
                                    int(out.shape[0]) if clear else 0, _stream(stream)))
    return out


def scatter_nodes(buf, idx, x, buf_idx=None, stream=None):
    """x[idx[k]] = buf[buf_idx[k]] (buf[k] without buf_idx) (tlfe_scatter_nodes)."""
    prec = _rows_prec(x, buf)
    n = int(idx.numel())
    _check(load().tlfe_scatter_nodes(prec, _ptr(buf), _ptr(_idx(buf_idx, n)), _ptr(_idx(idx, n)), n, _ptr(x),
                                     _stream(stream)))
    return x


class SplitCG:
    """Device vectors of one share of a body split across GPUs and the
    marshalling of the tlfe_split_* calls on them (the per-rank vector work of
    the split backward-Euler step). x, r, p, q, dinv are (n_rows, 3) CUDA
    tensors in the operator mesh's precision; dots is the float64 CUDA [2]
    tensor that receives each call's partial sums over the owned rows (the
    calls that sum return it; the caller all-reduces it before the next call
    overwrites it). fixed / own: uint8 CUDA [n_rows] or None."""

    def __init__(self, n_rows, precision, fixed=None, own=None, device="cuda"):
        import torch
        dt = torch.float32 if precision == FP32 else torch.float64
        for m, name in ((fixed, "fixed"), (own, "own")):
            if m is not None and not (m.is_cuda and m.dtype == torch.uint8 and m.is_contiguous()
                                      and m.numel() == n_rows):
                raise TLFEError(1, f"{name} must be a contiguous CUDA uint8 tensor of {n_rows} rows")
        self.n_rows, self.precision, self.dtype = int(n_rows), precision, dt
        self.fixed, self.own = fixed, own
        self.x, self.r, self.p, self.q, self.dinv = (torch.zeros((n_rows, 3), dtype=dt, device=device)
                                                     for _ in range(5))
        self.work = torch.zeros(int(load().tlfe_split_work_doubles(C.c_int64(n_rows))), dtype=torch.float64,
                                device=device)
        self.dots = torch.zeros(2, dtype=torch.float64, device=device)
        self.c = tlfe_split_cg(int(precision), self.n_rows, _ptr(fixed), _ptr(own), _ptr(self.x), _ptr(self.r),
                               _ptr(self.p), _ptr(self.q), _ptr(self.dinv), _ptr(self.work), _ptr(self.dots))

    def _rows(self, t, name, dtype=None):
        import torch
        dt = dtype or torch.float64
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()
                and tuple(t.shape) == (self.n_rows, 3)):
            raise TLFEError(1, f"{name} must be a contiguous CUDA {dt} tensor of shape ({self.n_rows}, 3)")
        return t

    def prep(self, h, gravity, u_n, v_n, v, u_out, w_out, v_op_out=None, stream=None):
        for t, n in ((u_n, "u_n"), (v_n, "v_n"), (v, "v"), (u_out, "u_out"), (w_out, "w_out")):
            self._rows(t, n)
        if v_op_out is not None:
            self._rows(v_op_out, "v_op_out", self.dtype)
        g = (C.c_double * 3)(*[float(x) for x in gravity])
        _check(load().tlfe_split_prep(C.byref(self.c), float(h), g, _ptr(u_n), _ptr(v_n), _ptr(v), _ptr(u_out),
                                      _ptr(w_out), _ptr(v_op_out), _stream(stream)))

    def residual(self, f, y, g, stream=None):
        for t, n in ((f, "f"), (y, "y"), (g, "g")):
            self._rows(t, n)
        _check(load().tlfe_split_residual(C.byref(self.c), _ptr(f), _ptr(y), _ptr(g), _stream(stream)))
        return g

    def velocity(self, v_base, add_x, v_out, stream=None):
        self._rows(v_base, "v_base")
        self._rows(v_out, "v_out")
        _check(load().tlfe_split_velocity(C.byref(self.c), _ptr(v_base), int(bool(add_x)), _ptr(v_out),
                                          _stream(stream)))
        return v_out

    def dot(self, a, b, stream=None):
        self._rows(a, "a")
        self._rows(b, "b")
        _check(load().tlfe_split_dot(C.byref(self.c), _ptr(a), _ptr(b), _stream(stream)))
        return self.dots[:1]

    def cg_dinv(self, D, stream=None):
        self._rows(D, "D", self.dtype)
        _check(load().tlfe_split_cg_dinv(C.byref(self.c), _ptr(D), _stream(stream)))

    def cg_start(self, g, stream=None):
        self._rows(g, "g")
        _check(load().tlfe_split_cg_start(C.byref(self.c), _ptr(g), _stream(stream)))
        return self.dots

    def cg_pq(self, stream=None):
        _check(load().tlfe_split_cg_pq(C.byref(self.c), _stream(stream)))
        return self.dots[:1]

    def cg_update(self, alpha, stream=None):
        _check(load().tlfe_split_cg_update(C.byref(self.c), float(alpha), _stream(stream)))
        return self.dots

    def cg_direction(self, beta, stream=None):
        _check(load().tlfe_split_cg_direction(C.byref(self.c), float(beta), _stream(stream)))


def tlfe_norm_noalloc(x, out, stream=None):
    """2-norm of the contiguous float64 CUDA tensor x into out (float64, 1 value);
    allocates nothing on the device."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TLFEError(1, "x must be a contiguous CUDA float64 tensor")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise TLFEError(1, "out must be a CUDA float64 tensor with at least one element")
    _check(load().tlfe_norm_noalloc(_ptr(x), C.c_int64(x.numel()), _ptr(out), _stream(stream)))
    return out


def tlfe_sync(mesh: Mesh, stream=None):
    return mesh.sync(stream)


def tlfe_version() -> str:
    return load().tlfe_version().decode()


# ---------------------------------------------------------------------------
# checkpoint / resume of a time-stepping run
# ---------------------------------------------------------------------------

def save_checkpoint(path, u, v, step, lam=None, **meta):
    """Write the state of a backward-Euler run to an .npz file: displacement
    u and velocity v (float64 (n_nodes, 3)), the step index, the constraint
    multipliers lam when the run has constraints, and any scalar metadata
    (step size, seeds, ...). The arrays are copied bit for bit, so a run
    resumed with load_checkpoint on a mesh built the same way repeats the
    original steps exactly where the step itself is deterministic (colour
    scatter: no atomic accumulation)."""
    import numpy as np
    arrs = {"u": u.detach().cpu().numpy(), "v": v.detach().cpu().numpy(), "step": np.int64(step)}
    if lam is not None:
        arrs["lam"] = lam.detach().cpu().numpy()
    for k, x in meta.items():
        arrs["meta_" + k] = np.asarray(x)
    np.savez(path, **arrs)


def load_checkpoint(path, device="cuda"):
    """Read a save_checkpoint file: returns a dict with u, v (float64 tensors
    on `device`), step (int), lam (tensor or None) and meta (dict)."""
    import numpy as np
    import torch
    with np.load(path) as z:
        out = {"u": torch.from_numpy(z["u"].copy()).to(device), "v": torch.from_numpy(z["v"].copy()).to(device),
               "step": int(z["step"]), "lam": torch.from_numpy(z["lam"].copy()).to(device) if "lam" in z else None,
               "meta": {k[5:]: z[k].item() if z[k].ndim == 0 else z[k] for k in z.files if k.startswith("meta_")}}
    return out
