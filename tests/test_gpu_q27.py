"""The Q27 triquadratic brick (App. A) on the GPU against the FP64 oracle:
internal force, tangent/mass/damping operator, adjoint and Jacobi diagonal on
the affine and slab paths, curved (non-affine) bricks, Mooney-Rivlin, ragged
tiles, external loads, constraints on Q27 hosts, and the Newton step.

Tolerances as in the other parity tests: FP64 1e-12, FP32 2e-5 (max-norm,
relative to the oracle's max |value|)."""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

from test_gpu_parity import run_all, check_all

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q27 = synth.Q27


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def _cuda(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_q27_beam_full_operator(prec, path):
    wl = synth.q27_beam(cells=(8, 3, 2))
    h = 1e-3
    mesh, out = run_all(wl, prec, aM=1.0 / h, aK=h, aC=1.0, path=path)
    assert mesh.info["n_affine_blocks"] == (1 if path == 0 else 0)
    check_all(wl, out, prec, aM=1.0 / h, aK=h, aC=1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_q27_curved_bricks_take_the_slab_path(prec):
    wl = synth.q27_beam(cells=(6, 2, 2), curve=0.04)
    mesh, out = run_all(wl, prec, aK=1.0, aC=2.0, path=0)
    assert mesh.info["n_affine_blocks"] == 0
    check_all(wl, out, prec, aK=1.0, aC=2.0)
    tl = T()
    with pytest.raises(tl.TLFEError):
        tl.Mesh.from_workload(wl, precision=prec, element_path=tl.PATH_AFFINE)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_q27_mooney_rivlin(prec, path):
    wl = synth.q27_beam(cells=(5, 2, 2), model=2, damping=0.0, mu01=0.3 * 3.8e6 / 2)
    _, out = run_all(wl, prec, path=path)
    check_all(wl, out, prec)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n_elem", [1, 31, 33])
def test_q27_ragged_tiles(n_elem, path):
    base = synth.q27_beam(cells=(12, 2, 2))
    blk = base.blocks[0]
    wl = Workload("ragged", base.X, [Block(Q27, 27, blk.conn[:n_elem], blk.body[:n_elem])],
                  base.model, base.params, u=base.u, udot=base.udot, v=base.v)
    for prec in (0, 1):
        _, out = run_all(wl, prec, path=path)
        check_all(wl, out, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_q27_beside_t10_and_h8_blocks(prec):
    """A Q27 body in one mesh with a T10/T4/H8 batch: one block per type."""
    a = synth.batch_bodies(n_bodies=5, seed=7, ne_range=(40, 200))
    b = synth.q27_beam(cells=(4, 2, 2))
    off = a.n_nodes
    blocks = list(a.blocks) + [Block(Q27, 27, b.blocks[0].conn + off, b.blocks[0].body + a.n_bodies)]
    wl = Workload("mixed_q27", np.concatenate([a.X, b.X + [0.0, 2.0, 0.0]]), blocks,
                  np.concatenate([a.model, b.model]), np.concatenate([a.params, b.params]),
                  u=np.concatenate([a.u, b.u]),
                  v=np.random.default_rng(3).standard_normal((a.n_nodes + b.n_nodes, 3)))
    _, out = run_all(wl, prec)
    check_all(wl, out, prec)


def test_q27_loads_match_oracle():
    wl = synth.q27_beam(cells=(4, 2, 3), curve=0.03)
    blk = wl.blocks[0]
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    rng = np.random.default_rng(8)
    el = rng.integers(0, blk.n_elem, 11).astype(np.int32)
    xi = rng.uniform(-1, 1, (11, 3))
    fp = rng.standard_normal((11, 3))
    fe, ff = synth.boundary_faces(Q27, blk.conn)
    t0 = rng.standard_normal((fe.size, 3)) * 1e4
    f_p = mesh.point_loads(_cuda(el, torch.int32), _cuda(xi, torch.float64), _cuda(fp, torch.float64))
    f_t = mesh.surface_traction(_cuda(fe, torch.int32), _cuda(ff, torch.int32), _cuda(t0, torch.float64))
    mesh.sync()
    for got, ref in ((f_p, oracle.point_loads(wl, 0, el, xi, fp)), (f_t, oracle.surface_traction(wl, 0, fe, ff, t0))):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_q27_constraints_match_oracle(prec):
    wl = synth.q27_beam(cells=(4, 2, 2))
    tl = T()
    rng = np.random.default_rng(4)
    items = []
    for t in range(4):
        npts = 4 if t >= 2 else 2
        items.append({"type": t, "elem": [int(x) for x in rng.integers(0, wl.n_elem, npts)],
                      "xi": rng.uniform(-1, 1, (npts, 3)).tolist(),
                      "d": rng.standard_normal(3).tolist(), "f": float(rng.uniform(0.01, 0.1))})
    cons = oracle.constraints(items)
    gc = np.zeros(len(items), tl.CON_DTYPE)
    for name in tl.CON_DTYPE.names:
        gc[name] = cons[name]
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    u = _cuda(wl.u, torch.float64)
    v = rng.standard_normal(wl.X.shape)
    w = rng.standard_normal(len(items))
    c = mesh.constraint_eval(gc, u).cpu().numpy()
    jv = mesh.constraint_j(gc, u, _cuda(v, torch.float64)).cpu().numpy()
    jtw = mesh.constraint_jt(gc, u, _cuda(w, torch.float64)).cpu().numpy()
    c_ref = oracle.constraint_eval(wl, cons)
    assert np.abs(c - c_ref).max() <= 1e-13 * max(1.0, np.abs(c_ref).max())
    ref = oracle.constraint_j(wl, cons, v)
    assert np.abs(jv - ref).max() <= 1e-12 * np.abs(ref).max()
    ref = oracle.constraint_jt(wl, cons, w)
    assert np.abs(jtw - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_q27_clamped_newton_step_matches_oracle(prec):
    m = synth.box_mesh(Q27, (4, 1, 1), (0.2, 0.05, 0.05))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    wl = Workload("q27_clamped", m.X, [Block(Q27, 27, m.conn, m.body)],
                  np.array([1], np.int32), np.array([[3.8e6, 5.8e6, 0.0, 0.0, 1000.0]]),
                  u=np.zeros_like(m.X), udot=np.zeros_like(m.X), fixed=fixed)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    G = np.array([0.0, 0.0, -9.81])
    h = 1e-3
    # FP64: both steps solved with CG to 1e-8, which lands the last Newton
    # iteration on the rounding floor of the residual: equal to 1e-10. FP32:
    # the operator's rounding bounds the step at 1e-6
    rtol, cg_rtol, bar = (1e-10, 1e-8, 1e-10) if prec == 0 else (1e-10, 1e-6, 1e-6)
    v, rep = mesh.newton_step(z, z.clone(), h, gravity=G, fixed=torch.from_numpy(fixed).cuda(), newton_rtol=rtol,
                              cg_rtol=cg_rtol, max_newton=20, max_cg=2000, use_graph=True)
    torch.cuda.synchronize()
    v = v.cpu().numpy()
    assert rep["status"] == 0 and rep["rel_residual"] <= rtol
    v_ref, rep_ref = oracle.newton_step(wl, np.zeros_like(wl.X), np.zeros_like(wl.X), h, G, fixed=fixed,
                                        newton_rtol=1e-10, cg_rtol=1e-8)
    assert rep_ref["status"] == 0 and rep_ref["rel_residual"] <= 1e-10
    assert np.abs(v - v_ref).max() <= bar * np.abs(v_ref).max()
    assert np.abs(v[fixed == 1]).max() == 0.0


def _q27_variants(kind):
    """The Q27 beam with per-element (mu, lambda) or with several bodies of
    different laws in one block (per-element material index)."""
    wl = synth.q27_beam(cells=(6, 2, 2))
    rng = np.random.default_rng(17)
    if kind == "elam":
        theta = np.stack([3.8e6 * np.exp(0.3 * rng.standard_normal(wl.n_elem)),
                          5.8e6 * np.exp(0.3 * rng.standard_normal(wl.n_elem))], axis=1)
        return Workload("q27_elam", wl.X, wl.blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v,
                        elem_mu_lambda=theta)
    blk = wl.blocks[0]
    body = (np.arange(blk.n_elem) % 3).astype(np.int32)
    params = np.array([[3.8e6, 5.8e6, 1e3, 0.0, 1000.0], [2.0e6, 4.0e6, 0.0, 0.0, 1200.0],
                       [5.0e6, 7.0e6, 2e3, 1e3, 800.0]])
    return Workload("q27_mats", wl.X, [Block(Q27, 27, blk.conn, body)], np.array([1, 0, 1], np.int32), params,
                    u=wl.u, udot=wl.udot, v=wl.v)


@pytest.mark.parametrize("kind", ["elam", "mats"])
@pytest.mark.parametrize("prec", [0, 1])
def test_q27_per_element_parameters_and_materials(prec, kind):
    """Warp-per-element kernels with per-element (mu, lambda), and with the
    law and damping read per element (several bodies in one block)."""
    wl = _q27_variants(kind)
    h = 1e-3
    _, out = run_all(wl, prec, aM=1.0 / h, aK=h, aC=1.0)
    check_all(wl, out, prec, aM=1.0 / h, aK=h, aC=1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_q27_sorted_scatter(prec):
    """Sorted scatter on the warp-per-element path (27 partials per element)
    beside tile-kernel blocks: parity with the oracle and bit-exact repeats."""
    wl = _q27_variants("mats")
    tl = T()
    h = 1e-3
    mesh, out = run_all(wl, prec, scatter=tl.SCATTER_SORTED, aM=1.0 / h, aK=h, aC=1.0)
    check_all(wl, out, prec, aM=1.0 / h, aK=h, aC=1.0)
    dt = mesh.torch_dtype
    u, ud, v = _cuda(wl.u, torch.float64), _cuda(wl.udot, dt), _cuda(wl.v, dt)
    assert torch.equal(mesh.internal_force(u, ud), out["f"])
    assert torch.equal(mesh.tangent_matvec(u, ud, v, 1.0 / h, h, 1.0), out["y"])


def test_q27_colour_scatter_and_mass_only():
    """Colour passes (plain read-add-write scatter) on the warp-per-element
    path, and the operator product with a_K = a_C = 0 (mass only)."""
    wl = synth.q27_beam(cells=(6, 3, 2))
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=tl.SCATTER_COLOR, color_seed=7)
    assert mesh.info["n_colors"] >= 8 and mesh.info["n_affine_blocks"] == 1
    dt = mesh.torch_dtype
    u, ud, v = _cuda(wl.u, torch.float64), _cuda(wl.udot, dt), _cuda(wl.v, dt)
    f1 = mesh.internal_force(u, ud).cpu().numpy()
    f2 = mesh.internal_force(u, ud).cpu().numpy()
    assert np.array_equal(f1.view(np.uint32), f2.view(np.uint32))
    f_ref, _ = oracle.internal_force(wl)
    assert np.abs(f1 - f_ref).max() <= 2e-5 * np.abs(f_ref).max()
    y = mesh.tangent_matvec(u, ud, v, 1.0, 0.0, 0.0).cpu().numpy()
    y_ref = oracle.operator_apply(wl, wl.v, a_M=1.0, a_K=0.0, a_C=0.0)
    assert np.abs(y - y_ref).max() <= 2e-5 * np.abs(y_ref).max()
    mesh.sync()


def test_q27_full_size_bench_configuration():
    """The 80k-brick Q27 beam the benchmark times, with its schedules
    autotuned as the benchmark does: force, K v + C v and the adjoint at
    sampled nodes (a node's value depends only on the bricks holding it),
    on the warp-per-element path (FP32, FP64) and the slab path (FP32)."""
    from test_gpu_parity import _subset, relerr
    wl = synth.q27_beam(cells=(200, 20, 20))
    rng = np.random.default_rng(9)
    ks = rng.choice(wl.n_nodes, 120, replace=False)
    sub = _subset(wl, np.isin(wl.blocks[0].conn, ks).any(axis=1))
    f_ref, bad = oracle.internal_force(sub)
    assert bad == 0
    y_ref = oracle.operator_apply(sub, wl.v, a_K=1.0, a_C=1.0)
    g_ref, gd_ref, _ = oracle.vjp(sub, wl.v)
    tl = T()
    for prec, tol, path in ((1, 2e-5, 0), (1, 2e-5, 1), (0, 1e-12, 0)):
        mesh = tl.Mesh.from_workload(wl, precision=prec, element_path=path)
        dt = mesh.torch_dtype
        u, ud, v = _cuda(wl.u, torch.float64), _cuda(wl.udot, dt), _cuda(wl.v, dt)
        mesh.autotune(u, ud, v)
        f = mesh.internal_force(u, ud)
        y = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)
        gu, gud, _ = mesh.vjp(u, ud, v)
        mesh.sync()
        for got, ref in ((f, f_ref), (y, y_ref), (gu, g_ref), (gud, gd_ref)):
            assert relerr(got.double().cpu().numpy()[ks], ref[ks]) <= tol
        mesh.close()
