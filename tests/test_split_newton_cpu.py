"""Backward-Euler step of one body split across ranks (Sec. 7), host logic
on CPU: paper_2602_17002_gb300.shard.split_newton_step drives the inexact
Newton / Jacobi-PCG iteration over slabs of a clamped beam whose interface
nodes are duplicated; per operator application the ranks sum the interface
rows, per CG iteration they all-reduce p.q, then r.z and r.r in FP64.

Each share here is a CPU stand-in with the methods of shard.SplitShare: the
element operators are the FP64 oracle's on the share's own mesh, the vector
work is plain numpy. Two gloo ranks (DistGroup), and one process holding both
shares (LocalGroup, the exchange the single-GPU test uses), reproduce the
unsplit oracle step's velocity to 1e-10 of its maximum."""

import os
import socket

import numpy as np
import pytest

import synth
from paper_2602_17002_gb300 import shard
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

H = 1e-3
G = np.array([0.0, 0.0, -9.81])


def clamped_beam(cells=8, damping=0.0):
    """A 5:1:1-style T10 beam of `cells` cells (0.05 m), x = 0 face clamped,
    neo-Hookean mu = 3.8e6, lambda = 5.8e6, rho = 1000, at rest."""
    m = synth.box_mesh(synth.T10, (cells, 1, 1), (0.05 * cells, 0.05, 0.05))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    params = np.array([[3.8e6, 5.8e6, damping, 0.0, 1000.0]])
    return Workload("clamped_beam", m.X, [Block(synth.T10, 5, m.conn, m.body)],
                    np.array([synth.workloads.NEOHOOKE], np.int32), params,
                    u=np.zeros_like(m.X), udot=np.zeros_like(m.X), fixed=fixed)


class OracleShare:
    """CPU stand-in of shard.SplitShare: the oracle's force, mass and Newton
    operator products and Jacobi diagonal on the share's mesh, numpy vector
    work; the arrays it returns are torch views of its own numpy storage, so
    that the group's in-place interface sums reach it. With op_dtype float32
    the CG vectors, the diagonal and the operator products are held in FP32
    (the oracle's FP64 values rounded), as an FP32 operator mesh holds them,
    while the residual and the velocity stay FP64."""

    def __init__(self, wl, own, gravity, op_dtype=np.float64):
        import oracle
        self.o = oracle
        self.wl = wl
        self.dt = np.dtype(op_dtype)
        n = wl.n_nodes
        self.fx = wl.fixed.astype(bool) if wl.fixed is not None else np.zeros(n, bool)
        self.own = np.asarray(own, bool)
        self.b0 = np.asarray(gravity, np.float64)
        self.u_n = np.zeros((n, 3))
        self.v_n = np.zeros((n, 3))
        self.g = np.zeros((n, 3))
        self.D = np.zeros((n, 3), self.dt)
        self.q = np.zeros((n, 3), self.dt)

    def _dots(self, *pairs):
        return torch.tensor([float((a[self.own].astype(np.float64) * b[self.own].astype(np.float64)).sum())
                             for a, b in pairs], dtype=torch.float64)

    def start(self):
        self.v = np.where(self.fx[:, None], 0.0, self.v_n)

    def residual(self, h):
        self.u = self.u_n + h * self.v
        w = (self.v - self.v_n) - h * self.b0
        f, _ = self.o.internal_force(self.wl, u=self.u, udot=self.v)
        y = self.o.operator_apply(self.wl, w, a_M=1.0 / h, a_K=0.0, a_C=0.0, u=self.u, udot=self.v)
        self.g[:] = np.where(self.fx[:, None], 0.0, f + y)
        return torch.from_numpy(self.g)

    def dot_g(self):
        return self._dots((self.g, self.g))

    def diag(self, h):
        self.D[:] = self.o.jacobi_diag(self.wl, a_M=1.0 / h, a_K=h, a_C=1.0, u=self.u, udot=self.v)
        return torch.from_numpy(self.D)

    def cg_start(self):
        with np.errstate(divide="ignore"):
            self.dinv = np.where(self.fx[:, None] | (self.D == 0), self.dt.type(0), 1 / self.D).astype(self.dt)
        self.r = np.where(self.fx[:, None], 0.0, -self.g).astype(self.dt)
        self.x = np.zeros_like(self.r)
        self.p = self.dinv * self.r
        return self._dots((self.r, self.dinv * self.r), (self.r, self.r))

    def apply(self, h):
        self.q[:] = self.o.operator_apply(self.wl, self.p.astype(np.float64), a_M=1.0 / h, a_K=h, a_C=1.0,
                                          sym_only=True, u=self.u, udot=self.v)
        return torch.from_numpy(self.q)

    def cg_pq(self):
        self.q[self.fx] = 0
        return self._dots((self.p, self.q))

    def cg_update(self, alpha):
        a = self.dt.type(alpha)
        self.x += a * self.p
        self.r -= a * self.q
        return self._dots((self.r, self.dinv * self.r), (self.r, self.r))

    def cg_direction(self, beta):
        self.p = self.dinv * self.r + self.dt.type(beta) * self.p

    def newton_update(self):
        self.v = np.where(self.fx[:, None], 0.0, self.v + self.x.astype(np.float64))


def _np_pack(x, idx, buf, pos):
    buf.zero_()
    buf[pos.long()] = x[idx.long()]


def _np_unpack(buf, pos, x, idx):
    x[idx.long()] = buf[pos.long()]


def _split(wl, n):
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    masks = shard.slab_partition(wl.X, blocks, n)
    nodes = [shard.local_blocks(blocks, m)[0] for m in masks]
    return masks, nodes, shard.interfaces(nodes)


def _reference(wl):
    import oracle
    v, rep = oracle.newton_step(wl, np.zeros_like(wl.X), np.zeros_like(wl.X), H, G, fixed=wl.fixed,
                                newton_rtol=1e-10, cg_rtol=1e-8)
    assert rep["status"] == 0
    return v, rep


@pytest.mark.parametrize("n_shares,damping,op_dtype", [(2, 0.0, np.float64), (3, 1e3, np.float64),
                                                     (2, 1e3, np.float32)])
def test_one_process_holding_every_share_matches_the_unsplit_oracle_step(n_shares, damping, op_dtype):
    wl = clamped_beam(cells=9, damping=damping)
    masks, nodes, ifs = _split(wl, n_shares)
    parts = [OracleShare(shard.sub_workload(wl, m)[0], shard.owned_rows(nd.size, itf), G, op_dtype)
             for m, nd, itf in zip(masks, nodes, ifs)]
    group = shard.LocalGroup(ifs, "cpu", pack=_np_pack, unpack=_np_unpack)
    fp32 = op_dtype == np.float32
    rep = shard.split_newton_step(parts, group, H, newton_rtol=1e-10, cg_rtol=1e-6 if fp32 else 1e-8)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10 and rep["newton_iters"] >= 1
    v_ref, rep_ref = _reference(wl)
    seen = np.zeros(wl.n_nodes, int)
    for s, nd in zip(parts, nodes):
        assert np.abs(s.v - v_ref[nd]).max() <= (1e-6 if fp32 else 1e-10) * np.abs(v_ref).max()
        seen[nd] += 1
    assert seen.min() == 1 and seen.max() == 2
    # the interface sums went through one compact buffer per dtype of the rows summed
    assert set(group.sums) == ({torch.float64, torch.float32} if fp32 else {torch.float64})
    if not fp32:   # the CG iterations follow the oracle's up to rounding order
        assert abs(rep["cg_iters"] - rep_ref["cg_iters"]) <= 2 * rep["newton_iters"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_split_newton_cpu as t
    from paper_2602_17002_gb300 import shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = t.clamped_beam(cells=9, damping=1e3)
        masks, nodes, ifs = t._split(wl, world)
        share, _ = sh.sub_workload(wl, masks[rank])
        part = t.OracleShare(share, sh.owned_rows(nodes[rank].size, ifs[rank]), t.G)
        grp = sh.DistGroup(ifs[rank], "cpu", pack=t._np_pack, unpack=t._np_unpack)
        rep = sh.split_newton_step([part], grp, t.H, newton_rtol=1e-10, cg_rtol=1e-8)
        q.put((rank, nodes[rank], part.v, rep))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_step_one_split_body_like_the_unsplit_oracle():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, nodes, v, rep = q.get(timeout=300)
        got[r] = (nodes, v, rep)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = clamped_beam(cells=9, damping=1e3)
    v_ref, _ = _reference(wl)
    reps = [got[r][2] for r in range(world)]
    assert reps[0] == reps[1]                      # every rank took the same decisions
    assert reps[0]["status"] == 0 and reps[0]["rel_residual"] <= 1e-10
    for r in range(world):
        nodes, v, _ = got[r]
        assert np.abs(v - v_ref[nodes]).max() <= 1e-10 * np.abs(v_ref).max()
        assert np.abs(v[wl.fixed[nodes] == 1]).max(initial=0.0) == 0.0


def test_edge_cases_one_share_and_a_body_already_at_rest_in_equilibrium():
    """One share (no interface nodes) is the unsplit step; a body at rest
    with no load has g(v_n) = 0 and takes no Newton iteration."""
    wl = clamped_beam(cells=6)
    masks, nodes, ifs = _split(wl, 1)
    assert ifs[0].n == 0 and nodes[0].size == wl.n_nodes
    part = OracleShare(shard.sub_workload(wl, masks[0])[0], shard.owned_rows(nodes[0].size, ifs[0]), G)
    rep = shard.split_newton_step([part], shard.LocalGroup(ifs, "cpu", pack=_np_pack, unpack=_np_unpack), H,
                                  newton_rtol=1e-10, cg_rtol=1e-8)
    v_ref, _ = _reference(wl)
    assert rep["status"] == 0 and np.abs(part.v - v_ref[nodes[0]]).max() <= 1e-10 * np.abs(v_ref).max()
    rest = OracleShare(shard.sub_workload(wl, masks[0])[0], np.ones(wl.n_nodes, bool), np.zeros(3))
    rep0 = shard.split_newton_step([rest], shard.LocalGroup(ifs, "cpu", pack=_np_pack, unpack=_np_unpack), H)
    assert rep0 == {"newton_iters": 0, "cg_iters": 0, "status": 0, "rel_residual": 0.0}
    assert np.array_equal(rest.v, np.zeros_like(rest.v))
