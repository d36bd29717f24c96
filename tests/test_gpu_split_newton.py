"""Backward-Euler step of one body split across GPUs (Sec. 7), run on one GPU:
the shares of a clamped beam's slabs are meshes of their own, stepped by
shard.split_newton_step through the library (tlfe_split_* vector kernels,
tlfe_internal_force, tlfe_tangent_matvec, tlfe_jacobi_diag and
tlfe_newton_operator on each share), with the interface rows summed through
the library's compact-buffer kernels (LocalGroup: what the all-reduce does
across GPUs). No kernel waits on another share. The velocity equals the
unsplit FP64 oracle step's, and the symmetric Newton operator equals the
oracle's K^v-free operator."""

import numpy as np
import pytest

import oracle
import synth
from paper_2602_17002_gb300 import shard
from test_split_newton_cpu import G, H, clamped_beam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _shares(wl, n, prec):
    from paper_2602_17002_gb300 import tlfe
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    masks = shard.slab_partition(wl.X, blocks, n)
    nodes = [shard.local_blocks(blocks, m)[0] for m in masks]
    ifs = shard.interfaces(nodes)
    parts = []
    for m, nd, itf in zip(masks, nodes, ifs):
        sw, _ = shard.sub_workload(wl, m)
        res = tlfe.Mesh.from_workload(sw, precision=tlfe.FP64)
        op = res if prec == tlfe.FP64 else tlfe.Mesh.from_workload(sw, precision=prec)
        z = torch.zeros((sw.n_nodes, 3), dtype=torch.float64, device="cuda")
        own = torch.from_numpy(shard.owned_rows(nd.size, itf).astype(np.uint8)).cuda()
        parts.append(shard.SplitShare(res, op, z, z.clone(), G, fixed=torch.from_numpy(sw.fixed).cuda(), own=own))
    return parts, nodes, ifs


# (mesh precision of the CG operator, Newton tolerance, CG tolerance, velocity bar): the FP64 step
# equals the oracle's to 1e-10 (both solved to the FP64 rounding floor of the residual); the FP32
# operator's rounding (about 1e-7 of |f|) bounds the FP32 CG solves, the FP64 residual the step
BARS = [(0, 1e-10, 1e-8, 1e-10), (1, 1e-10, 1e-6, 1e-6)]


@pytest.mark.parametrize("prec,rtol,cg_rtol,bar", BARS)
@pytest.mark.parametrize("n_shares,damping", [(2, 0.0), (3, 1e3)])
def test_split_step_matches_the_unsplit_oracle(prec, rtol, cg_rtol, bar, n_shares, damping):
    wl = clamped_beam(cells=9, damping=damping)
    parts, nodes, ifs = _shares(wl, n_shares, prec)
    group = shard.LocalGroup(ifs, "cuda")
    rep = shard.split_newton_step(parts, group, H, newton_rtol=rtol, cg_rtol=cg_rtol)
    torch.cuda.synchronize()
    assert rep["status"] == 0 and rep["rel_residual"] <= rtol and rep["newton_iters"] >= 1
    v_ref, rep_ref = oracle.newton_step(wl, np.zeros_like(wl.X), np.zeros_like(wl.X), H, G, fixed=wl.fixed,
                                        newton_rtol=1e-10, cg_rtol=1e-8)
    assert rep_ref["status"] == 0
    for s, nd in zip(parts, nodes):
        v = s.v.cpu().numpy()
        assert np.abs(v - v_ref[nd]).max() <= bar * np.abs(v_ref).max()
        assert np.abs(v[wl.fixed[nd] == 1]).max(initial=0.0) == 0.0
    for s in parts:
        assert s.res.sync() == 0 and s.op.sync() == 0


def test_split_step_repeats_bit_for_bit_in_sorted_scatter_mode():
    from paper_2602_17002_gb300 import tlfe
    wl = clamped_beam(cells=8)
    outs = []
    for _ in range(2):
        blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
        masks = shard.slab_partition(wl.X, blocks, 2)
        nodes = [shard.local_blocks(blocks, m)[0] for m in masks]
        ifs = shard.interfaces(nodes)
        parts = []
        for m, nd, itf in zip(masks, nodes, ifs):
            sw, _ = shard.sub_workload(wl, m)
            mesh = tlfe.Mesh.from_workload(sw, precision=tlfe.FP64, scatter=tlfe.SCATTER_SORTED)
            z = torch.zeros((sw.n_nodes, 3), dtype=torch.float64, device="cuda")
            own = torch.from_numpy(shard.owned_rows(nd.size, itf).astype(np.uint8)).cuda()
            parts.append(shard.SplitShare(mesh, mesh, z, z.clone(), G, fixed=torch.from_numpy(sw.fixed).cuda(),
                                          own=own))
        rep = shard.split_newton_step(parts, shard.LocalGroup(ifs, "cuda"), H)
        outs.append(([s.v.cpu().numpy() for s in parts], rep))
    assert outs[0][1] == outs[1][1]
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)


def test_newton_operator_is_the_viscous_stiffness_free_operator():
    from paper_2602_17002_gb300 import tlfe
    wl = synth.small_beam(cells=(6, 2, 2))          # neo-Hookean + Kelvin-Voigt, deformed and moving
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP64)
    u = torch.from_numpy(wl.u).cuda()
    ud = torch.from_numpy(wl.udot).cuda()
    v = torch.from_numpy(wl.v).cuda()
    y = mesh.newton_operator(u, ud, v, 1.0 / H, H, 1.0).cpu().numpy()
    ref = oracle.operator_apply(wl, wl.v, a_M=1.0 / H, a_K=H, a_C=1.0, sym_only=True)
    full = oracle.operator_apply(wl, wl.v, a_M=1.0 / H, a_K=H, a_C=1.0)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(full - ref).max() > 1e-9 * np.abs(ref).max()   # K^v matters on this state


def test_split_vector_kernels_against_numpy():
    from paper_2602_17002_gb300 import tlfe
    rng = np.random.default_rng(9)
    n = 3000                                             # 9000 values: three chunks, the last ragged
    fixed = (rng.random(n) < 0.1).astype(np.uint8)
    own = (rng.random(n) < 0.8).astype(np.uint8)
    cg = tlfe.SplitCG(n, tlfe.FP64, fixed=torch.from_numpy(fixed).cuda(), own=torch.from_numpy(own).cuda())
    g, D, q = (rng.standard_normal((n, 3)) for _ in range(3))
    D = np.abs(D) + 0.5
    D[5] = 0.0
    fx, ow = fixed.astype(bool)[:, None], own.astype(bool)
    cg.cg_dinv(torch.from_numpy(D).cuda())
    with np.errstate(divide="ignore"):
        dinv = np.where(fx | (D == 0.0), 0.0, 1.0 / D)
    assert np.abs(cg.dinv.cpu().numpy() - dinv).max() <= 1e-15
    d = cg.cg_start(torch.from_numpy(g).cuda()).cpu().numpy()
    r = np.where(fx, 0.0, -g)
    z = dinv * r
    assert np.allclose(d, [(r * z)[ow].sum(), (r * r)[ow].sum()], rtol=1e-13, atol=0)
    assert np.array_equal(cg.p.cpu().numpy(), cg.dinv.cpu().numpy() * cg.r.cpu().numpy())
    cg.q.copy_(torch.from_numpy(q))
    pq = cg.cg_pq().cpu().numpy()[0]
    qp = np.where(fx, 0.0, q)
    assert np.array_equal(cg.q.cpu().numpy(), qp)
    terms = (z * qp)[ow]
    assert abs(pq - terms.sum()) <= 1e-13 * np.abs(terms).sum()
    d = cg.cg_update(0.7).cpu().numpy()
    x, r = 0.7 * z, r - 0.7 * qp
    assert np.abs(cg.x.cpu().numpy() - x).max() <= 1e-15 * np.abs(x).max() + 1e-300
    assert np.allclose(d, [(r * dinv * r)[ow].sum(), (r * r)[ow].sum()], rtol=1e-13, atol=0)
    cg.cg_direction(0.3)
    pe = dinv * r + 0.3 * z
    assert np.abs(cg.p.cpu().numpy() - pe).max() <= 1e-14 * np.abs(pe).max()
    # the empty share writes zero sums
    e = tlfe.SplitCG(0, tlfe.FP32)
    assert e.cg_pq().cpu().numpy()[0] == 0.0
