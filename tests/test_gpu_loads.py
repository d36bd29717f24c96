"""External loads of Sec. 4 on the GPU (tlfe_point_loads,
tlfe_surface_traction) against the FP64 oracle, and the applied load in the
backward-Euler residual."""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def _curved(wl, amp, seed):
    X = wl.X.copy()
    rng = np.random.default_rng(seed)
    for blk in wl.blocks:
        if blk.etype == synth.T10:
            mids = np.unique(blk.conn[:, 4:])
            X[mids] += rng.uniform(-amp, amp, (mids.size, 3))
    return Workload(wl.name + "_curved", X, wl.blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v)


def _cuda(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("curved", [False, True])
def test_point_loads_and_tractions_match_oracle(curved):
    wl = synth.batch_bodies(n_bodies=6, seed=11, ne_range=(60, 300))
    if curved:
        wl = _curved(wl, 0.004, 3)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    rng = np.random.default_rng(5)
    f_ref_p = np.zeros((wl.n_nodes, 3))
    f_ref_t = np.zeros((wl.n_nodes, 3))
    E, XI, FP, TE, TF, T0 = [], [], [], [], [], []
    base = 0
    for bi, blk in enumerate(wl.blocks):
        k = 9
        el = rng.integers(0, blk.n_elem, k).astype(np.int32)
        xi = rng.uniform(-1, 1, (k, 3)) if blk.etype == synth.H8 else rng.dirichlet(np.ones(4), k)[:, 1:]
        fp = rng.standard_normal((k, 3))
        f_ref_p += oracle.point_loads(wl, bi, el, xi, fp)
        E.append(el + base), XI.append(xi), FP.append(fp)
        fe, ff = synth.boundary_faces(blk.etype, blk.conn)
        t0 = rng.standard_normal((fe.size, 3)) * 1e4
        f_ref_t += oracle.surface_traction(wl, bi, fe, ff, t0)
        TE.append(fe + base), TF.append(ff), T0.append(t0)
        base += blk.n_elem
    f_p = mesh.point_loads(_cuda(np.concatenate(E), torch.int32), _cuda(np.concatenate(XI), torch.float64),
                           _cuda(np.concatenate(FP), torch.float64))
    f_t = mesh.surface_traction(_cuda(np.concatenate(TE), torch.int32), _cuda(np.concatenate(TF), torch.int32),
                                _cuda(np.concatenate(T0), torch.float64))
    mesh.sync()
    for got, ref in ((f_p, f_ref_p), (f_t, f_ref_t)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_bad_face_is_reported_and_skipped():
    wl = synth.small_beam(cells=(3, 1, 1))
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP64)
    f = mesh.surface_traction(_cuda(np.array([0, 1], np.int32), torch.int32), _cuda(np.array([7, 0], np.int32), torch.int32),
                              _cuda(np.ones((2, 3)), torch.float64))
    with pytest.raises(tl.TLFEError) as ei:
        mesh.sync()
    assert ei.value.code == 8
    ref = oracle.surface_traction(wl, 0, np.array([1], np.int32), np.array([0], np.int32), np.ones((1, 3)))
    assert np.abs(f.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_applied_load_enters_the_step_residual(prec):
    """Gravity given as the applied load f_ext = M g (with zero body force)
    gives the same step as the body force itself; a tip traction load then
    converges to the residual tolerance."""
    m = synth.box_mesh(synth.T10, (8, 2, 2), (0.4, 0.1, 0.1))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    wl = Workload("beam", m.X, [Block(synth.T10, 5, m.conn, np.zeros(m.n_elem, np.int32))],
                  np.array([1], np.int32), np.array([[3.8e6, 5.8e6, 0.0, 0.0, 1000.0]]), u=np.zeros_like(m.X))
    g = np.array([0.0, 0.0, -9.81])
    f_grav = oracle.gravity_load(wl, g)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = _cuda(fixed, torch.uint8)
    kw = dict(fixed=fx, newton_rtol=1e-10, cg_rtol=1e-6, max_newton=20, max_cg=2000)
    v1, r1 = mesh.newton_step(z, z, 1e-3, gravity=g, **kw)
    v2, r2 = mesh.newton_step(z, z, 1e-3, gravity=(0.0, 0.0, 0.0), f_ext=_cuda(f_grav, torch.float64), **kw)
    assert r1["status"] == 0 and r2["status"] == 0
    v1, v2 = v1.cpu().numpy(), v2.cpu().numpy()
    assert np.abs(v1 - v2).max() <= 1e-8 * np.abs(v1).max()
    # tip traction on the x = 0.4 face
    fe, ff = synth.boundary_faces(synth.T10, m.conn)
    cen = np.array([m.X[m.conn[e, synth.face_corners(synth.T10, f)]].mean(axis=0) for e, f in zip(fe, ff)])
    tip = np.abs(cen[:, 0] - 0.4) < 1e-9
    t0 = np.tile([0.0, 2e4, -5e4], (int(tip.sum()), 1))
    f_tip = mesh.surface_traction(_cuda(fe[tip], torch.int32), _cuda(ff[tip], torch.int32), _cuda(t0, torch.float64))
    v3, r3 = mesh.newton_step(z, z, 1e-3, gravity=(0.0, 0.0, 0.0), f_ext=f_tip, **kw)
    assert r3["status"] == 0 and r3["rel_residual"] <= 1e-10
    assert np.abs(v3.cpu().numpy()).max() > 0
