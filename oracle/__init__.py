"""CPU FP64 oracle for the TL-FEA hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. It wraps
``oracle.c`` (plain C, FP64, ``-ffp-contract=off``) through ctypes and shares
no code with the CUDA library. Each wrapper names the paper equation its C
routine restates.

Parity unpinned: none. Every routine is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, finite differences,
exact integration, brute force).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MAT_DTYPE = np.dtype([("model", np.int32), ("mu", np.float64), ("lam", np.float64),
                      ("mu_v", np.float64), ("lam_v", np.float64), ("rho", np.float64),
                      ("mu01", np.float64)], align=True)
NPE = {0: 4, 1: 10, 2: 8, 3: 27}


class Report(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("cg_iters", C.c_int32), ("status", C.c_int32),
                ("rel_residual", C.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, no CUDA)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
               "-Wall", "-o", tmp, src, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            i32, f64 = C.c_int, C.c_double
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_splitmix64.argtypes = [C.c_uint64]
            for name, args in {
                "orc_nodes_per_elem": [i32],
                "orc_shape": [i32, P, P],
                "orc_shape_grad": [i32, P, P],
                "orc_quad_rule": [i32, i32, P, P],
                "orc_exact_rule": [i32, i32, P, P],
                "orc_precompute": [i32, i32, i32, P, P, P, P, P],
                "orc_stress": [P, P, P, P],
                "orc_strain_energy": [P, P, P],
                "orc_internal_force": [i32, i32, i32, P, i32, P, P, P, P, i32, P],
                "orc_operator_apply": [i32, i32, i32, P, i32, P, P, P, P, f64, f64, f64, i32,
                                       i32, P, P],
                "orc_element_matrices": [i32, i32, P, P, P, P, P, P, P, P],
                "orc_element_matrices_sym": [i32, i32, P, P, P, P, P, P, P, P],
                "orc_vjp": [i32, i32, i32, P, i32, P, P, P, P, P, P, P, P],
                "orc_lumped_row_sums": [i32, i32, P, i32, P, P, P],
                "orc_gravity": [i32, i32, P, i32, P, P, P, P],
                "orc_newton_step": [i32, i32, i32, P, i32, P, P, P, P, f64, P, P, f64, f64,
                                    i32, i32, P, P],
                "orc_color_greedy": [i32, i32, P, i32, C.c_uint64, P],
                "orc_point_loads": [i32, i32, P, P, P, P, P],
                "orc_surface_traction": [i32, i32, P, P, P, P, P, P],
                "orc_constraint_eval": [i32, i32, P, P, P, P, P],
                "orc_constraint_jt": [i32, i32, P, P, P, P, P, P],
                "orc_constraint_j": [i32, i32, P, P, P, P, P, P],
                "orc_newton_step_alm": [i32, i32, i32, P, i32, P, P, P, P, f64, P, P, f64, f64, i32, i32,
                                        i32, P, f64, f64, i32, i32, P, P, P, P, P],
                "orc_constraint_row_weights": [i32, i32, P, P, P, P],
            }.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")
    return rc


# --------------------------------------------------------------------------
# element-level primitives
# --------------------------------------------------------------------------

def shape(etype, xi):
    s = np.zeros(NPE[etype])
    _check(lib().orc_shape(etype, _p(_f64(xi)), _p(s)), "shape")
    return s


def shape_grad(etype, xi):
    g = np.zeros((NPE[etype], 3))
    _check(lib().orc_shape_grad(etype, _p(_f64(xi)), _p(g)), "shape_grad")
    return g


def quad_rule(etype, nq):
    pts = np.zeros((nq, 3))
    w = np.zeros(nq)
    _check(lib().orc_quad_rule(etype, nq, _p(pts), _p(w)), "quad_rule")
    return pts, w


def exact_rule(etype, order):
    pts = np.zeros((order ** 3, 3))
    w = np.zeros(order ** 3)
    _check(lib().orc_exact_rule(etype, order, _p(pts), _p(w)), "exact_rule")
    return pts, w


def precompute(etype, nq, conn, X):
    """H[e, q, i, :] = h_i and wJ[e, q] = w_q J_p (Section 6)."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    ne = conn.shape[0]
    H = np.zeros((ne, nq, NPE[etype], 3))
    wJ = np.zeros((ne, nq))
    jmin = np.zeros(1)
    bad = _check(lib().orc_precompute(etype, nq, ne, _p(conn), _p(_f64(X)), _p(H), _p(wJ),
                                      _p(jmin)), "precompute")
    return H, wJ, bad


def material(model, mu, lam, mu_v=0.0, lam_v=0.0, rho=1000.0, mu01=0.0):
    """Material record: model 0 SVK, 1 neo-Hookean, 2 Mooney-Rivlin (mu10 = mu/2 - mu01)."""
    m = np.zeros(1, MAT_DTYPE)
    m["model"], m["mu"], m["lam"], m["mu_v"], m["lam_v"], m["rho"] = model, mu, lam, mu_v, lam_v, rho
    m["mu01"] = mu01
    return m


def stress(mat, F, Fdot=None):
    """P(F, Fdot) of Section 3 (SVK / neo-Hookean + Kelvin-Voigt)."""
    P = np.zeros((3, 3))
    st = lib().orc_stress(_p(mat), _p(_f64(F)), _p(_f64(Fdot)), _p(P))
    _check(st, "stress")
    return P, st


def strain_energy(mat, F):
    psi = np.zeros(1)
    _check(lib().orc_strain_energy(_p(mat), _p(_f64(F)), _p(psi)), "strain_energy")
    return float(psi[0])


def element_matrices(etype, nq, conn_e, X, u, udot, mat):
    n3 = 3 * NPE[etype]
    Ke, Ce, Me = (np.zeros((n3, n3)) for _ in range(3))
    conn_e = np.ascontiguousarray(conn_e, dtype=np.int32)
    _check(lib().orc_element_matrices(etype, nq, _p(conn_e), _p(_f64(X)), _p(_f64(u)),
                                      _p(_f64(udot)), _p(mat), _p(Ke), _p(Ce), _p(Me)),
           "element_matrices")
    return Ke, Ce, Me


def jacobi_diag(wl, a_M=0.0, a_K=1.0, a_C=0.0, u=None, udot="state"):
    """diag(a_M M + a_K K^e + a_C C) from the closed-form element matrices
    (K^e: elastic part, the viscous stiffness left out)."""
    u = _f64(wl.u if u is None else u)
    udot = _f64(wl.udot if isinstance(udot, str) else udot)
    X = _f64(wl.X)
    d = np.zeros_like(X)
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi)
        n3 = 3 * NPE[blk.etype]
        Ke, Ce, Me = (np.zeros((n3, n3)) for _ in range(3))
        for e in range(blk.n_elem):
            ce = np.ascontiguousarray(blk.conn[e], dtype=np.int32)
            _check(lib().orc_element_matrices_sym(blk.etype, blk.nq, _p(ce), _p(X), _p(u), _p(udot),
                                                  _p(m[e:e + 1]), _p(Ke), _p(Ce), _p(Me)), "element_matrices")
            dg = a_M * np.diag(Me) + a_K * np.diag(Ke) + a_C * np.diag(Ce)
            np.add.at(d, ce, dg.reshape(-1, 3))
    return d


def splitmix64(x):
    return int(lib().orc_splitmix64(C.c_uint64(x)))


# --------------------------------------------------------------------------
# workload-level calls (sum over the element blocks of a synth.Workload)
# --------------------------------------------------------------------------

def block_materials(wl, bi):
    """Per-element material records of block bi (per-body parameters, with
    the optional per-element (mu, lam) override applied)."""
    blk = wl.blocks[bi]
    off = sum(b.n_elem for b in wl.blocks[:bi])
    m = np.zeros(blk.n_elem, MAT_DTYPE)
    pb = wl.params[blk.body]
    m["model"] = wl.model[blk.body]
    m["mu"], m["lam"], m["mu_v"], m["lam_v"], m["rho"] = pb.T[:5]
    if pb.shape[1] > 5:                      # optional sixth column: Mooney-Rivlin mu01
        m["mu01"] = pb[:, 5]
    if wl.elem_mu_lambda is not None:
        m["mu"] = wl.elem_mu_lambda[off:off + blk.n_elem, 0]
        m["lam"] = wl.elem_mu_lambda[off:off + blk.n_elem, 1]
    return m


def internal_force(wl, u=None, udot="state", kin_form=2, mats=None):
    """Assembled f_int (Eq. internal_force_universal); returns (f, n_inverted)."""
    u = _f64(wl.u if u is None else u)
    udot = _f64(wl.udot if isinstance(udot, str) else udot)
    X = _f64(wl.X)
    f = np.zeros_like(X)
    bad = 0
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi) if mats is None else mats[bi]
        bad += _check(lib().orc_internal_force(blk.etype, blk.nq, blk.n_elem, _p(blk.conn),
                                               wl.n_nodes, _p(X), _p(u), _p(udot), _p(m),
                                               kin_form, _p(f)), "internal_force")
    return f, bad


def operator_apply(wl, v, a_M=0.0, a_K=1.0, a_C=0.0, transpose=False, sym_only=False,
                   u=None, udot="state"):
    """y = a_M M v + a_K K_t v + a_C C v from the closed-form element blocks."""
    u = _f64(wl.u if u is None else u)
    udot = _f64(wl.udot if isinstance(udot, str) else udot)
    X = _f64(wl.X)
    v = _f64(v)
    y = np.zeros_like(X)
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi)
        _check(lib().orc_operator_apply(blk.etype, blk.nq, blk.n_elem, _p(blk.conn), wl.n_nodes,
                                        _p(X), _p(u), _p(udot), _p(m), a_M, a_K, a_C,
                                        int(transpose), int(sym_only), _p(v), _p(y)),
               "operator_apply")
    return y


def vjp(wl, r, u=None, udot="state"):
    """(g_u, g_udot, g_theta) = (K_t^T r, C^T r, d(r.f)/d(mu_e, lam_e))."""
    u = _f64(wl.u if u is None else u)
    udot = _f64(wl.udot if isinstance(udot, str) else udot)
    X = _f64(wl.X)
    r = _f64(r)
    g_u = np.zeros_like(X)
    g_ud = np.zeros_like(X)
    g_th = np.zeros((wl.n_elem, 2))
    off = 0
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi)
        gt = np.zeros((blk.n_elem, 2))
        _check(lib().orc_vjp(blk.etype, blk.nq, blk.n_elem, _p(blk.conn), wl.n_nodes, _p(X),
                             _p(u), _p(udot), _p(m), _p(r), _p(g_u), _p(g_ud), _p(gt)), "vjp")
        g_th[off:off + blk.n_elem] = gt
        off += blk.n_elem
    return g_u, g_ud, g_th


def gravity_load(wl, g):
    X = _f64(wl.X)
    f = np.zeros_like(X)
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi)
        _check(lib().orc_gravity(blk.etype, blk.n_elem, _p(blk.conn), wl.n_nodes, _p(X), _p(m),
                                 _p(_f64(g)), _p(f)), "gravity")
    return f


def mass_row_sums(wl):
    X = _f64(wl.X)
    m_row = np.zeros(wl.n_nodes)
    for bi, blk in enumerate(wl.blocks):
        m = block_materials(wl, bi)
        _check(lib().orc_lumped_row_sums(blk.etype, blk.n_elem, _p(blk.conn), wl.n_nodes, _p(X),
                                         _p(m), _p(m_row)), "mass")
    return m_row


def newton_step(wl, u_n, v_n, h, gravity, fixed=None, newton_rtol=1e-8, cg_rtol=1e-4,
                max_newton=20, max_cg=2000):
    """Backward-Euler step (Section 7, no constraints): returns (v, report)."""
    assert len(wl.blocks) == 1, "oracle Newton step takes one element block"
    blk = wl.blocks[0]
    m = block_materials(wl, 0)
    X = _f64(wl.X)
    v = np.zeros_like(X)
    rep = Report()
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
    _check(lib().orc_newton_step(blk.etype, blk.nq, blk.n_elem, _p(blk.conn), wl.n_nodes, _p(X),
                                 _p(m), _p(_f64(u_n)), _p(_f64(v_n)), float(h),
                                 _p(_f64(gravity)), _p(fx), newton_rtol, cg_rtol,
                                 int(max_newton), int(max_cg), _p(v), C.byref(rep)),
           "newton_step")
    return v, {"newton_iters": rep.newton_iters, "cg_iters": rep.cg_iters,
               "status": rep.status, "rel_residual": rep.rel_residual}


def color_greedy(conn, n_nodes, seed):
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    col = np.zeros(conn.shape[0], np.int32)
    nc = _check(lib().orc_color_greedy(conn.shape[0], conn.shape[1], _p(conn), int(n_nodes),
                                       C.c_uint64(seed), _p(col)), "color")
    return col, nc


def point_loads(wl, block, elem, xi, force):
    """Assembled f_iP = s_i(xi_P) f_P (Sec. 4, pointwise loads) of loads at
    parent points xi (k, 3) of block-local elements elem (k,)."""
    blk = wl.blocks[block]
    f = np.zeros((wl.n_nodes, 3))
    _check(lib().orc_point_loads(blk.etype, len(elem), _p(blk.conn), _p(np.ascontiguousarray(elem, np.int32)),
                                 _p(_f64(xi)), _p(_f64(force)), _p(f)), "point_loads")
    return f


def surface_traction(wl, block, elem, face, t0):
    """Assembled f_i = int s_i t0 dA0 (Sec. 4, surface tractions) over faces
    `face` of block-local elements `elem` with nominal tractions t0 (k, 3)."""
    blk = wl.blocks[block]
    f = np.zeros((wl.n_nodes, 3))
    _check(lib().orc_surface_traction(blk.etype, len(elem), _p(blk.conn), _p(_f64(wl.X)),
                                      _p(np.ascontiguousarray(elem, np.int32)),
                                      _p(np.ascontiguousarray(face, np.int32)), _p(_f64(t0)), _p(f)),
           "surface_traction")
    return f


CON_DTYPE = np.dtype([("type", np.int32), ("elem", np.int32, (4,)), ("xi", np.float64, (4, 3)),
                      ("d", np.float64, (3,)), ("f", np.float64)], align=True)
CD, DIST, DP1, DP2 = 0, 1, 2, 3


def constraints(items):
    """Constraint records from dicts {type, elem: [..], xi: [[..], ..], d, f}
    (points P, Q[, R, T]; elem < 0 marks a ground point at world coordinates xi)."""
    c = np.zeros(len(items), CON_DTYPE)
    for k, it in enumerate(items):
        c[k]["type"] = it["type"]
        el = list(it["elem"]) + [-1] * (4 - len(it["elem"]))
        c[k]["elem"] = el
        xi = np.zeros((4, 3))
        xi[:len(it["xi"])] = it["xi"]
        c[k]["xi"] = xi
        c[k]["d"] = it.get("d", (0.0, 0.0, 0.0))
        c[k]["f"] = it.get("f", 0.0)
    return c


def constraint_eval(wl, cons, u=None):
    """c(q) of the constraint primitives (CD, DIST, DP1, DP2) at q = X + u."""
    blk = wl.blocks[0]
    out = np.zeros(len(cons))
    _check(lib().orc_constraint_eval(blk.etype, len(cons), _p(cons), _p(blk.conn), _p(_f64(wl.X)),
                                     _p(_f64(wl.u if u is None else u)), _p(out)), "constraint_eval")
    return out


def constraint_jt(wl, cons, w, u=None):
    """C_q^T w as an (n_nodes, 3) array."""
    blk = wl.blocks[0]
    f = np.zeros((wl.n_nodes, 3))
    _check(lib().orc_constraint_jt(blk.etype, len(cons), _p(cons), _p(blk.conn), _p(_f64(wl.X)),
                                   _p(_f64(wl.u if u is None else u)), _p(_f64(w)), _p(f)), "constraint_jt")
    return f


def constraint_j(wl, cons, v, u=None):
    """C_q v as an (n_cons,) array."""
    blk = wl.blocks[0]
    out = np.zeros(len(cons))
    _check(lib().orc_constraint_j(blk.etype, len(cons), _p(cons), _p(blk.conn), _p(_f64(wl.X)),
                                  _p(_f64(wl.u if u is None else u)), _p(_f64(v)), _p(out)), "constraint_j")
    return out


def constraint_row_weights(wl, cons):
    """Row weights of Eq. row_weights (DP1 rows 1/sqrt(|a0|^2 + |b0|^2) at the
    reference configuration, all other rows 1)."""
    blk = wl.blocks[0]
    w = np.zeros(len(cons))
    _check(lib().orc_constraint_row_weights(blk.etype, len(cons), _p(cons), _p(blk.conn), _p(_f64(wl.X)), _p(w)),
           "constraint_row_weights")
    return w


def newton_step_alm(wl, u_n, v_n, h, gravity, cons, rho, lam=None, fixed=None, newton_rtol=1e-8, cg_rtol=1e-4,
                    max_newton=20, max_cg=2000, alm_tol=1e-10, max_outer=50, row_norm=True):
    """Augmented-Lagrangian backward-Euler step (Sec. 7) on the row-normalised
    constraints (Eqs. row_weights, rev_normalized; row_norm=False: raw rows):
    returns (v, lam, report), lam the multipliers of the rows used."""
    assert len(wl.blocks) == 1
    blk = wl.blocks[0]
    m = block_materials(wl, 0)
    v = np.zeros_like(_f64(wl.X))
    lam = np.zeros(len(cons)) if lam is None else np.array(lam, dtype=np.float64)
    rep = Report()
    outer = C.c_int(0)
    cn = C.c_double(0.0)
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
    _check(lib().orc_newton_step_alm(blk.etype, blk.nq, blk.n_elem, _p(blk.conn), wl.n_nodes, _p(_f64(wl.X)),
                                     _p(m), _p(_f64(u_n)), _p(_f64(v_n)), C.c_double(h), _p(_f64(gravity)), _p(fx),
                                     C.c_double(newton_rtol), C.c_double(cg_rtol), int(max_newton), int(max_cg),
                                     len(cons), _p(cons), C.c_double(rho), C.c_double(alm_tol), int(max_outer),
                                     int(bool(row_norm)), _p(lam), _p(v), C.byref(rep), C.byref(outer), C.byref(cn)),
           "newton_step_alm")
    return v, lam, {"newton_iters": rep.newton_iters, "cg_iters": rep.cg_iters, "status": rep.status,
                    "rel_residual": rep.rel_residual, "outer_iters": outer.value, "c_norm": cn.value}
