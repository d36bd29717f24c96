"""The batch of uneven bodies (mixed T4 / T10 / H8, several laws) in one
persistent launch per operation, and the graph-replayed force + K v call
(tlfe_force_matvec), against the FP64 oracle (Sec. 4.3, Eq.
internal_force_universal; App. C tangents)."""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def dev(a, dt):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def relerr(got, ref):
    got = got.double().cpu().numpy() if hasattr(got, "cpu") else got
    den = np.abs(ref).max()
    return np.abs(got - ref).max() / (den if den > 0 else 1.0)


def _mixed(n_bodies=14, seed=11, damped=True, mr=True):
    """Mixed element types and laws (SVK, neo-Hookean, Mooney-Rivlin), some
    bodies damped, with a velocity field."""
    wl = synth.batch_bodies(n_bodies=n_bodies, seed=seed, ne_range=(40, 400))
    model = np.asarray(wl.model).copy()
    if mr:
        model[::5] = 2
    params = np.concatenate([wl.params, 0.15 * wl.params[:, :1]], axis=1)
    if damped:
        params[1::3, 2] = 1e3
    wl.model, wl.params = model, params
    wl.udot = 0.01 * np.random.default_rng(seed + 20).standard_normal(wl.X.shape)
    return wl


@pytest.mark.parametrize("scatter", [0, 2])
def test_fused_launch_matches_oracle_and_per_pass_launches(scatter):
    """Every pass of every block in one launch per operation: force and the
    full operator product match the oracle at the FP32 bar and the per-pass
    launches to rounding; the sorted scatter repeats bit for bit."""
    tl = T()
    wl = _mixed()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=scatter)
    info = mesh.info
    assert info["n_fused_passes"] == info["n_passes"] >= 4
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, torch.float32), dev(wl.v, torch.float32)
    res = {}
    for mode in (tl.LAUNCH_FUSED, tl.LAUNCH_PER_PASS):
        mesh.set_launch_mode(mode)
        exp = 1 + (1 if scatter == 2 else 0) if mode == tl.LAUNCH_FUSED else info["n_passes"] + (scatter == 2)
        assert mesh.info["launches_force"] == exp and mesh.info["launches_matvec"] == exp
        f = mesh.internal_force(u, ud)
        y = mesh.tangent_matvec(u, ud, v, 1.0 / 1e-3, 1e-3, 1.0)
        mesh.sync()
        res[mode] = (f.cpu().numpy(), y.cpu().numpy())
    f_ref, _ = oracle.internal_force(wl)
    y_ref = oracle.operator_apply(wl, wl.v, a_M=1.0 / 1e-3, a_K=1e-3, a_C=1.0)
    for mode in res:
        assert relerr(res[mode][0], f_ref) <= TOL32
        assert relerr(res[mode][1], y_ref) <= TOL32
    assert relerr(res[tl.LAUNCH_FUSED][0], res[tl.LAUNCH_PER_PASS][0]) <= 1e-6
    assert relerr(res[tl.LAUNCH_FUSED][1], res[tl.LAUNCH_PER_PASS][1]) <= 1e-6
    if scatter == 2:
        mesh.set_launch_mode(tl.LAUNCH_FUSED)
        f2 = mesh.internal_force(u, ud).cpu().numpy()
        assert np.array_equal(f2.view(np.uint32), res[tl.LAUNCH_FUSED][0].view(np.uint32))
    mesh.close()


def test_fused_launch_covers_affine_passes_and_leaves_the_rest():
    """Curved (slab-path) and warp-per-element Q27 blocks keep their own
    launches beside the fused one; results still match the oracle."""
    tl = T()
    base = synth.batch_bodies(n_bodies=6, seed=9, ne_range=(60, 300))
    X = base.X.copy()
    rng = np.random.default_rng(3)
    t10 = [b for b in base.blocks if b.etype == synth.T10]
    if t10:
        mids = np.unique(t10[0].conn[:, 4:])
        X[mids] += rng.uniform(-0.004, 0.004, (mids.size, 3))   # curved T10: slab path
    q = synth.q27_beam(cells=(3, 2, 2))
    off = X.shape[0]
    blocks = list(base.blocks) + [Block(synth.Q27, 27, q.blocks[0].conn + off,
                                        np.full(q.blocks[0].n_elem, base.n_bodies, np.int32))]
    wl = Workload("mix", np.concatenate([X, q.X]), blocks, np.append(base.model, 1),
                  np.concatenate([base.params, [[3.8e6, 5.8e6, 0.0, 0.0, 1000.0]]]),
                  u=np.concatenate([base.u, q.u]), udot=None, v=np.concatenate([base.v, q.v]))
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    mesh.set_launch_mode(tl.LAUNCH_FUSED)
    info = mesh.info
    assert 2 <= info["n_fused_passes"] < info["n_passes"]
    u, v = dev(wl.u, torch.float64), dev(wl.v, torch.float32)
    f = mesh.internal_force(u, None)
    y = mesh.tangent_matvec(u, None, v, 0.0, 1.0, 0.0)
    mesh.sync()
    assert relerr(f, oracle.internal_force(wl)[0]) <= TOL32
    assert relerr(y, oracle.operator_apply(wl, wl.v)) <= TOL32
    mesh.close()


@pytest.mark.parametrize("scatter", [0, 2])
def test_force_matvec_graph_replays_and_recaptures(scatter):
    """tlfe_force_matvec: the first call evaluates and captures; replays with
    the same pointers read the arrays' current contents; new pointers or
    coefficients capture again; autotuning invalidates the graph."""
    tl = T()
    wl = _mixed(seed=5)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=scatter)
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, torch.float32), dev(wl.v, torch.float32)
    f, y = torch.empty_like(v), torch.empty_like(v)
    f_ref, _ = oracle.internal_force(wl)
    for _ in range(3):
        f.fill_(7.0)
        y.fill_(7.0)
        mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0, f=f, y=y)
        mesh.sync()
        assert relerr(f, f_ref) <= TOL32
        assert relerr(y, oracle.operator_apply(wl, wl.v, a_K=1.0, a_C=1.0)) <= TOL32
    # same pointers, new contents: the replay reads them
    v2 = np.random.default_rng(77).standard_normal(wl.X.shape)
    v.copy_(dev(v2, torch.float32))
    mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0, f=f, y=y)
    mesh.sync()
    assert relerr(y, oracle.operator_apply(wl, v2, a_K=1.0, a_C=1.0)) <= TOL32
    # new coefficients and new output arrays: a new capture
    f3, y3 = torch.empty_like(v), torch.empty_like(v)
    mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0, f=f3, y=y3)
    mesh.sync()
    assert relerr(y3, oracle.operator_apply(wl, v2, a_K=1.0, u=wl.u, udot=None)) <= TOL32
    # after autotuning the graph is captured again with the tuned schedules
    mesh.autotune(u, ud, v)
    mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0, f=f, y=y)
    mesh.sync()
    assert relerr(f, f_ref) <= TOL32
    if scatter == 2:
        a = f.cpu().numpy().copy()
        mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0, f=f, y=y)
        mesh.sync()
        assert np.array_equal(a.view(np.uint32), f.cpu().numpy().view(np.uint32))
    mesh.close()


def _body_samples(wl, per_body, rng):
    """Per body: its first node (a corner of the box, where the stretch's
    traction makes the force large) and per_body - 1 random nodes."""
    lo = np.full(wl.n_bodies, np.iinfo(np.int64).max)
    hi = np.full(wl.n_bodies, -1)
    for blk in wl.blocks:                      # every body owns one contiguous node range
        np.minimum.at(lo, blk.body, blk.conn.min(axis=1))
        np.maximum.at(hi, blk.body, blk.conn.max(axis=1))
    ks, owner = [], []
    for b in range(wl.n_bodies):
        pick = [lo[b]] + list(lo[b] + rng.choice(hi[b] - lo[b] + 1, per_body - 1, replace=False))
        ks += pick
        owner += [b] * len(pick)
    return np.array(ks), np.array(owner)


def _sub(wl, ks):
    blocks = []
    for blk in wl.blocks:
        sel = np.isin(blk.conn, ks).any(axis=1)
        blocks.append(Block(blk.etype, blk.nq, blk.conn[sel], blk.body[sel]))
    return Workload("sub", wl.X, blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v)


def test_batch_512_full_size_graph_replay():
    """The 512-body batch the benchmark times (19.6 M elements, mixed T4 /
    T10 / H8, SVK and neo-Hookean), in its launch configuration: autotuned,
    one persistent launch per operation, force + K v replayed from the
    library's graph. Force and K v at six sampled nodes of every body
    (a node's value depends only on the elements holding it) against the
    oracle, each body normalised by its own largest sampled value."""
    tl = T()
    wl = synth.batch_bodies(512)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    info = mesh.info
    assert info["n_fused_passes"] == info["n_passes"] == 6
    u, v = dev(wl.u, torch.float64), dev(wl.v, torch.float32)
    mesh.autotune(u, None, v)
    mesh.set_launch_mode(tl.LAUNCH_FUSED)
    f, y = torch.empty_like(v), torch.empty_like(v)
    for _ in range(3):                   # capture, then replays
        mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0, f=f, y=y)
    mesh.sync()
    assert mesh.info["launches_force"] == 1 and mesh.info["launches_matvec"] == 1
    ks, owner = _body_samples(wl, 6, np.random.default_rng(12))
    sub = _sub(wl, ks)
    f_ref, bad = oracle.internal_force(sub)
    assert bad == 0
    y_ref = oracle.operator_apply(sub, wl.v, a_K=1.0)
    fg, yg = f.double().cpu().numpy()[ks], y.double().cpu().numpy()[ks]
    for got, ref in ((fg, f_ref[ks]), (yg, y_ref[ks])):
        err = np.abs(got - ref).max(axis=1)
        den = np.zeros(wl.n_bodies)
        np.maximum.at(den, owner, np.abs(ref).max(axis=1))
        assert (err / den[owner]).max() <= TOL32
    mesh.close()
