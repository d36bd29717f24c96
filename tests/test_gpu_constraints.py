"""Constraint primitives of Sec. 3 (tlfe_constraint_eval / _j / _jt) and the
augmented-Lagrangian Newton step of Sec. 7 on the GPU, against the FP64 oracle."""

import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU, LAM = 3.8e6, 5.8e6
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def _records(items, dtype):
    c = np.zeros(len(items), dtype)
    for k, it in enumerate(items):
        c[k]["type"] = it["type"]
        c[k]["elem"] = list(it["elem"]) + [-1] * (4 - len(it["elem"]))
        xi = np.zeros((4, 3))
        xi[:len(it["xi"])] = it["xi"]
        c[k]["xi"] = xi
        c[k]["d"] = it.get("d", (0.0, 0.0, 0.0))
        c[k]["f"] = it.get("f", 0.0)
    return c


def _two_beams():
    m1 = synth.box_mesh(synth.T10, (4, 1, 1), (0.2, 0.05, 0.05))
    m2 = synth.box_mesh(synth.T10, (4, 1, 1), (0.2, 0.05, 0.05), origin=(0.0, 0.1, 0.0))
    m = synth.concat_meshes([m1, m2])
    rng = np.random.default_rng(41)
    u = 0.002 * rng.standard_normal(m.X.shape)
    return Workload("two", m.X, [Block(synth.T10, 5, m.conn, m.body)], np.array([1, 1], np.int32),
                    np.array([[MU, LAM, 0.0, 0.0, 1000.0]] * 2), u=u, udot=None)


def _items(wl, rng):
    ne = wl.blocks[0].n_elem
    half = ne // 2

    def pt(body):
        return int(rng.integers(0, half)) + (half if body else 0), rng.dirichlet(np.ones(4))[1:]
    items = []
    for t, bodies in ((0, [0, 1]), (1, [0, 1]), (2, [0, 0, 1, 1]), (3, [0, 0, 0, 1])):
        pts = [pt(b) for b in bodies]
        items.append({"type": t, "elem": [p[0] for p in pts], "xi": [p[1] for p in pts], "d": (0.0, 1.0, 0.0),
                      "f": 0.03})
    e, xi = pt(0)
    items.append({"type": 0, "elem": [e, -1], "xi": [xi, [0.05, 0.02, 0.01]], "d": (1.0, 0.0, 0.0)})
    return items


@pytest.mark.parametrize("prec", [0, 1])
def test_constraint_values_and_jacobian_actions_match_oracle(prec):
    tl = T()
    wl = _two_beams()
    rng = np.random.default_rng(42)
    items = _items(wl, rng)
    oc = _records(items, oracle.CON_DTYPE)
    gc = _records(items, tl.CON_DTYPE)
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    u = torch.from_numpy(wl.u).cuda()
    v = rng.standard_normal(wl.X.shape)
    w = rng.standard_normal(len(items))
    c = mesh.constraint_eval(gc, u).cpu().numpy()
    jv = mesh.constraint_j(gc, u, torch.from_numpy(v).cuda()).cpu().numpy()
    jtw = mesh.constraint_jt(gc, u, torch.from_numpy(w).cuda()).cpu().numpy()
    c_ref = oracle.constraint_eval(wl, oc)
    assert np.abs(c - c_ref).max() <= 1e-13 * max(1.0, np.abs(c_ref).max())
    assert np.abs(jv - oracle.constraint_j(wl, oc, v)).max() <= 1e-12 * np.abs(jv).max()
    ref = oracle.constraint_jt(wl, oc, w)
    assert np.abs(jtw - ref).max() <= 1e-12 * np.abs(ref).max()


def test_bad_constraint_element_is_rejected():
    tl = T()
    wl = _two_beams()
    gc = _records([{"type": 0, "elem": [10 ** 6, 0], "xi": [[0.1, 0.1, 0.1], [0.1, 0.1, 0.1]], "d": (1, 0, 0)}],
                  tl.CON_DTYPE)
    mesh = tl.Mesh.from_workload(wl, precision=0)
    with pytest.raises(tl.TLFEError) as ei:
        mesh.constraint_eval(gc, torch.from_numpy(wl.u).cuda())
    assert ei.value.code == 1


def _clamp_problem():
    m = synth.box_mesh(synth.T10, (4, 1, 1), (0.2, 0.05, 0.05))
    wl = Workload("b", m.X, [Block(synth.T10, 5, m.conn, np.zeros(m.n_elem, np.int32))], np.array([1], np.int32),
                  np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=np.zeros_like(m.X))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    rows = [ln.split() for ln in open(os.path.join(GOLD, "t10_parent_nodes.txt")) if ln.strip() and ln[0] != "#"]
    nxi = np.array([[float(x) for x in r[5:8]] for r in rows])
    items = []
    for node in np.nonzero(fixed)[0]:
        e, i = [(e, i) for e in range(m.n_elem) for i in range(10) if m.conn[e, i] == node][0]
        for d in range(3):
            dv = [0.0, 0.0, 0.0]
            dv[d] = 1.0
            items.append({"type": 0, "elem": [e, -1], "xi": [nxi[i], m.X[node]], "d": dv, "f": 0.0})
    return wl, fixed, items


@pytest.mark.parametrize("prec,use_graph", [(0, True), (1, True), (1, False)])
def test_alm_step_matches_oracle_and_the_projected_clamp(prec, use_graph):
    """A face clamped by coordinate-difference constraints to ground points
    (Sec. 3 CD, Sec. 7 ALM): the GPU step agrees with the oracle's ALM step and
    with the projected clamp."""
    tl = T()
    wl, fixed, items = _clamp_problem()
    g = np.array([0.0, 0.0, -9.81])
    z = np.zeros_like(wl.X)
    kw = dict(newton_rtol=1e-10, cg_rtol=1e-10)
    v_proj, _ = oracle.newton_step(wl, z, z, 1e-3, g, fixed=fixed, **kw)
    v_ref, lam_ref, r_ref = oracle.newton_step_alm(wl, z, z, 1e-3, g, _records(items, oracle.CON_DTYPE), rho=1e10,
                                                   alm_tol=1e-12, max_outer=20, **kw)
    assert r_ref["status"] == 0
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    zt = torch.zeros(wl.X.shape, dtype=torch.float64, device="cuda")
    v, rep = mesh.newton_step(zt, zt, 1e-3, gravity=g, max_newton=20, max_cg=4000, use_graph=use_graph,
                              constraints=_records(items, tl.CON_DTYPE), rho=1e10, alm_tol=1e-12, max_outer=20, **kw)
    assert rep["status"] == 0 and rep["c_norm"] <= 1e-12, rep
    v = v.cpu().numpy()
    assert np.abs(v - v_ref).max() <= 1e-6 * np.abs(v_ref).max()
    assert np.abs(v - v_proj).max() <= 1e-6 * np.abs(v_proj).max()
    lam = rep["lam"].cpu().numpy()
    assert np.abs(lam - lam_ref).max() <= 1e-4 * np.abs(lam_ref).max()


@pytest.mark.parametrize("prec,use_graph", [(0, True), (1, True), (1, False)])
def test_alm_revolute_joint_with_row_normalisation_matches_oracle(prec, use_graph):
    """A revolute-type joint (three CD rows, two DP1 rows on 2 cm fibres)
    between a clamped and a hanging beam: the step works on the row-normalised
    constraints (Eqs. row_weights, rev_normalized) and agrees with the
    oracle's normalised step in velocities and multipliers."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_pins import _revolute_problem
    tl = T()
    wl, fixed, cons = _revolute_problem(0.02)
    g = np.array([0.0, 0.0, -9.81])
    z = np.zeros_like(wl.X)
    kw = dict(newton_rtol=1e-10, cg_rtol=1e-10)
    v_ref, lam_ref, r_ref = oracle.newton_step_alm(wl, z, z, 1e-3, g, cons, rho=1e9, fixed=fixed, alm_tol=1e-10,
                                                   max_outer=40, max_newton=30, max_cg=5000, **kw)
    assert r_ref["status"] == 0
    gc = np.zeros(len(cons), tl.CON_DTYPE)
    for name in tl.CON_DTYPE.names:
        gc[name] = cons[name]
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    zt = torch.zeros(wl.X.shape, dtype=torch.float64, device="cuda")
    v, rep = mesh.newton_step(zt, zt, 1e-3, gravity=g, fixed=torch.from_numpy(fixed).cuda(), max_newton=30,
                              max_cg=5000, use_graph=use_graph, constraints=gc, rho=1e9, alm_tol=1e-10, max_outer=40,
                              **kw)
    assert rep["status"] == 0 and rep["c_norm"] <= 1e-10, rep
    v = v.cpu().numpy()
    # both stop at ||c^|| <= 1e-10: velocities agree to about alm_tol / h
    assert np.abs(v - v_ref).max() <= 2e-10 / 1e-3
    lam = rep["lam"].cpu().numpy()
    assert np.abs(lam - lam_ref).max() <= 1e-4 * np.abs(lam_ref).max()
