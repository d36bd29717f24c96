"""Batched backward-Euler Newton/CG step on the GPU against closed forms and the
FP64 oracle (Section 7 without constraints)."""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = np.array([0.0, 0.0, -9.81])
H = 1e-3


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def beams(n_bodies, sizes, clamp=True, damping=0.0):
    """n_bodies small clamped beams (one body each) concatenated."""
    ms = [synth.box_mesh(synth.T10, (c, 1, 1), (0.05 * c, 0.05, 0.05)) for c in sizes[:n_bodies]]
    big = synth.concat_meshes(ms)
    fixed = (np.abs(big.X[:, 0]) < 1e-12).astype(np.uint8) if clamp else None
    params = np.tile(np.array([[3.8e6, 5.8e6, damping, 0.0, 1000.0]]), (n_bodies, 1))
    wl = Workload("beams", big.X, [Block(synth.T10, 5, big.conn, big.body)],
                  np.full(n_bodies, synth.workloads.NEOHOOKE, np.int32), params,
                  u=np.zeros_like(big.X), udot=np.zeros_like(big.X), fixed=fixed)
    return wl


def step(wl, prec, use_graph=True, rtol=1e-8, cg_rtol=1e-4):
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = None if wl.fixed is None else torch.from_numpy(wl.fixed).cuda()
    v, rep = mesh.newton_step(z, z.clone(), H, gravity=G, fixed=fx, newton_rtol=rtol, cg_rtol=cg_rtol,
                              max_newton=20, max_cg=2000, use_graph=use_graph)
    torch.cuda.synchronize()
    return v.cpu().numpy(), rep, mesh


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_free_fall_is_exact(prec, use_graph):
    wl = beams(2, [3, 4], clamp=False)
    v, rep, _ = step(wl, prec, use_graph, rtol=1e-10)
    assert rep["code"] == 0 and rep["status"] == 0
    assert np.abs(v - H * G).max() < 1e-9 * 9.81 * H


# (Newton tolerance, CG tolerance, velocity bar) per mesh precision. One FP64
# step equals the oracle's step to 1e-10: with CG solved to 1e-8 the last
# Newton iteration lands on the FP64 rounding floor of the residual (about
# 1e-11 relative on these beams), and two such solves agree in velocity to
# about 1e-12 (at h = 1e-3 the Newton matrix is close to M / h, so the
# velocity error is of the order of the residual). The FP32 operator's
# rounding (about 1e-7 of |f|) bounds the FP32 step at 1e-6.
NEWTON_BAR = {0: (1e-10, 1e-8, 1e-10), 1: (1e-10, 1e-6, 1e-6)}


@pytest.mark.parametrize("prec", [0, 1])
def test_clamped_beam_matches_oracle(prec):
    rtol, cg_rtol, bar = NEWTON_BAR[prec]
    wl = beams(1, [6], clamp=True)
    v, rep, _ = step(wl, prec, True, rtol=rtol, cg_rtol=cg_rtol)
    assert rep["status"] == 0 and rep["rel_residual"] <= rtol
    v_ref, rep_ref = oracle.newton_step(wl, np.zeros_like(wl.X), np.zeros_like(wl.X), H, G, fixed=wl.fixed,
                                        newton_rtol=1e-10, cg_rtol=1e-8)
    assert rep_ref["status"] == 0 and rep_ref["rel_residual"] <= 1e-10
    assert np.abs(v - v_ref).max() <= bar * np.abs(v_ref).max()
    assert np.abs(v[wl.fixed == 1]).max() == 0.0


def test_batched_bodies_equal_single_body_solves_and_graph_equals_host_loop():
    sizes = [3, 5, 8]
    wl = beams(3, sizes, clamp=True)
    vb, rep, _ = step(wl, 1, True)
    assert rep["status"] == 0 and rep["n_bodies_converged"] == 3
    vh, reph, _ = step(wl, 1, False)
    assert np.array_equal(vb, vh)
    assert rep["cg_iters"] == reph["cg_iters"]
    off = 0
    for k, c in enumerate(sizes):
        one = beams(1, [c], clamp=True)
        v1, r1, _ = step(one, 1, True)
        n = one.n_nodes
        assert r1["status"] == 0
        # same problem, same iterates up to the order of the FP32 operator sums
        assert np.abs(vb[off:off + n] - v1).max() <= 1e-6 * np.abs(v1).max()
        off += n


def test_step_is_replayable_and_reports_iterations():
    wl = beams(2, [4, 6], clamp=True)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = torch.from_numpy(wl.fixed).cuda()
    v1, r1 = mesh.newton_step(z, z.clone(), H, gravity=G, fixed=fx)
    v2, r2 = mesh.newton_step(z, z.clone(), H, gravity=G, fixed=fx)
    assert torch.equal(v1, v2) and r1 == r2
    assert r1["newton_iters"] >= 1 and r1["cg_iters"] >= 1


def test_not_converged_is_reported():
    wl = beams(1, [6], clamp=True)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = torch.from_numpy(wl.fixed).cuda()
    v, rep = mesh.newton_step(z, z.clone(), H, gravity=G, fixed=fx, newton_rtol=1e-14, max_newton=1, max_cg=1)
    assert rep["code"] == 5 and rep["status"] == 5


def test_body_norms_match_numpy():
    wl = beams(3, [3, 5, 4], clamp=False)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(wl.X.shape)
    out = mesh.body_norms(torch.from_numpy(x).cuda()).cpu().numpy()
    body = np.zeros(wl.n_nodes, int)
    for blk in wl.blocks:
        for e in range(blk.n_elem):
            body[blk.conn[e]] = blk.body[e]
    ref = np.array([np.linalg.norm(x[body == b]) for b in range(3)])
    assert np.abs(out - ref).max() <= 1e-12 * ref.max()


def test_newton_full_size_bench_configuration():
    """The 64-beam, 6.75 M-element implicit step the benchmark times, in its
    configuration (FP32 operator, FP64 residual, graph, Newton to 1e-8 with
    CG tolerance 1e-4): every body converges, and the smallest body's
    velocities match the oracle's step of that body alone (bodies do not
    interact), solved to 1e-10. At h = 1e-3 the Newton matrix is dominated by
    M / h, so a 1e-8 relative residual bounds the velocity error far below
    the 1e-6 tolerance used here."""
    tl = T()
    wl = synth.newton_beams(64)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = torch.from_numpy(wl.fixed).cuda()
    v, rep = mesh.newton_step(z, z.clone(), H, gravity=G, fixed=fx, newton_rtol=1e-8, cg_rtol=1e-4,
                              max_newton=20, max_cg=4000, use_graph=True)
    torch.cuda.synchronize()
    assert rep["status"] == 0 and rep["n_bodies_converged"] == 64 and rep["rel_residual"] <= 1e-8
    bodies = synth.split_bodies(wl)
    k = int(np.argmin([b.n_elem for b in bodies]))
    b = bodies[k]
    lo = int(wl.blocks[0].conn[wl.blocks[0].body == k].min())
    vb = v.cpu().numpy()[lo:lo + b.n_nodes]
    zb = np.zeros_like(b.X)
    v_ref, rep_ref = oracle.newton_step(b, zb, zb, H, G, fixed=b.fixed, newton_rtol=1e-10, cg_rtol=1e-8,
                                        max_newton=20, max_cg=20000)
    assert rep_ref["status"] == 0
    assert np.abs(vb - v_ref).max() <= 1e-6 * np.abs(v_ref).max()
    assert np.abs(vb[b.fixed == 1]).max() == 0.0


def _run(mesh, wl, u, v, steps):
    """steps backward-Euler steps from (u, v): v_{k+1} = step(u_k, v_k), u_{k+1} = u_k + h v_{k+1}."""
    fx = torch.from_numpy(wl.fixed).cuda()
    for _ in range(steps):
        v_new, rep = mesh.newton_step(u, v, H, gravity=G, fixed=fx, newton_rtol=1e-10, cg_rtol=1e-6,
                                      max_newton=20, max_cg=2000, use_graph=True)
        assert rep["status"] == 0
        u = u + H * v_new
        v = v_new.clone()
    return u, v


@pytest.mark.parametrize("mode", ["colour", "sorted"])
def test_checkpoint_restart_is_bit_exact_in_colour_mode(tmp_path, mode):
    """Run 4 steps, checkpointing after 2 (save_checkpoint); a fresh mesh that
    resumes from the file (load_checkpoint) reproduces steps 3 and 4 bit for
    bit in both deterministic scatter modes: colour passes scatter without
    atomics, the sorted mode sums each node's tile partials in a fixed order,
    and the CG reductions are fixed-order."""
    tl = T()
    scatter = tl.SCATTER_COLOR if mode == "colour" else tl.SCATTER_SORTED
    wl = beams(2, [4, 6], clamp=True, damping=1e3)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=scatter)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    u2, v2 = _run(mesh, wl, z, z.clone(), 2)
    path = str(tmp_path / "state.npz")
    tl.save_checkpoint(path, u2, v2, step=2, h=H, seed=5)
    u4, v4 = _run(mesh, wl, u2, v2, 2)
    mesh.close()
    ck = tl.load_checkpoint(path)
    assert ck["step"] == 2 and ck["meta"]["h"] == H and ck["meta"]["seed"] == 5 and ck["lam"] is None
    assert torch.equal(ck["u"], u2) and torch.equal(ck["v"], v2)
    fresh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=scatter)
    u4b, v4b = _run(fresh, wl, ck["u"], ck["v"], 2)
    assert torch.equal(u4b, u4) and torch.equal(v4b, v4)
    assert float(v4.abs().max()) > 0.0
