"""Multi-GPU work split (paper_2602_17002_gb300.shard), host logic on CPU.

A body split into slabs sums the partial forces of its duplicated interface
nodes over the ranks; independent bodies are bin-packed and need no
exchange. Two gloo ranks compute their shares with the FP64 oracle and
exchange through the package's InterfaceSum protocol (compact buffer,
all-reduce), with pack / unpack written here on CPU tensors; the assembled
force, operator product and adjoint equal the unpartitioned oracle to 1e-12.
"""

import os
import socket

import numpy as np
import pytest

import synth
from paper_2602_17002_gb300 import shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _blocks(wl):
    return [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]


def test_pack_bodies_is_a_balanced_partition():
    rng = np.random.default_rng(1)
    costs = np.exp(rng.uniform(np.log(1e3), np.log(2e5), 512))
    for n in (1, 2, 3, 8):
        parts = shard.pack_bodies(costs, n)
        allb = np.concatenate(parts)
        assert np.array_equal(np.sort(allb), np.arange(512))
        loads = np.array([costs[p].sum() for p in parts])
        # greedy largest-first: no rank exceeds the mean by more than the largest body
        assert loads.max() <= costs.sum() / n + costs.max() + 1e-9


def test_body_costs_follow_the_element_mix():
    wl = synth.batch_bodies(n_bodies=9, seed=7, ne_range=(40, 400))
    c = shard.body_costs(_blocks(wl), wl.n_bodies)
    ref = np.zeros(wl.n_bodies)
    for b in wl.blocks:
        for e in range(b.n_elem):
            ref[b.body[e]] += b.nq * {0: 4, 1: 10, 2: 8}[b.etype]
    assert np.array_equal(c, ref)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_slab_partition_covers_every_element_once_and_interfaces_agree(n):
    wl = synth.small_beam(cells=(10, 2, 2))
    masks = shard.slab_partition(wl.X, _blocks(wl), n)
    cnt = sum(m[0].astype(int) for m in masks)
    assert np.all(cnt == 1)
    sizes = [int(m[0].sum()) for m in masks]
    assert max(sizes) - min(sizes) <= 1
    nodes = [shard.local_blocks(_blocks(wl), m)[0] for m in masks]
    ifs = shard.interfaces(nodes)
    for nd, itf in zip(nodes, ifs):
        assert itf.local.size == itf.pos.size and itf.n == ifs[0].n
        # positions name the same global node on every rank
        assert np.all(np.diff(itf.pos) > 0)
    glob = {}
    for nd, itf in zip(nodes, ifs):
        for l, p in zip(itf.local, itf.pos):
            glob.setdefault(int(p), set()).add(int(nd[l]))
    assert all(len(v) == 1 for v in glob.values()) and len(glob) == ifs[0].n
    # every node is owned by exactly one rank
    own = np.zeros(wl.n_nodes, int)
    for nd, itf in zip(nodes, ifs):
        own[nd[shard.owned_rows(nd.size, itf)]] += 1
    assert np.all(own == 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _np_pack(x, idx, buf, pos):
    buf.zero_()
    buf[pos.long()] = x[idx.long()]


def _np_unpack(buf, pos, x, idx):
    x[idx.long()] = buf[pos.long()]


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import synth as sy
    from paper_2602_17002_gb300 import shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        # one body in slabs along the beam axis: force, K v + C v, adjoint
        wl = sy.small_beam(cells=(8, 2, 2))
        blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
        masks = sh.slab_partition(wl.X, blocks, world)
        nodes_all = [sh.local_blocks(blocks, m)[0] for m in masks]
        itf = sh.interfaces(nodes_all)[rank]
        share, nodes = sh.sub_workload(wl, masks[rank])
        xs = sh.InterfaceSum(itf, torch.float64, "cpu", pack=_np_pack, unpack=_np_unpack)
        f, _ = oracle.internal_force(share)
        y = oracle.operator_apply(share, share.v, a_K=1.0, a_C=1.0)
        gu, gud, gth = oracle.vjp(share, share.v)
        res = {}
        for name, a in (("f", f), ("y", y), ("gu", gu), ("gud", gud)):
            t = torch.from_numpy(a.copy())
            xs(t)
            res[name] = t.numpy()
        # a sum over nodes counts every node once: the loss-like square sum
        keep = sh.owned_rows(nodes.size, itf)
        s = torch.tensor([float((res["f"][keep] ** 2).sum())], dtype=torch.float64)
        dist.all_reduce(s)
        out["beam"] = (nodes, res, gth, sh.sub_workload(wl, masks[rank])[0].n_elem, float(s[0]))
        # independent bodies, bin-packed: no exchange
        bw = sy.batch_bodies(n_bodies=7, seed=21, ne_range=(30, 300))
        bblocks = [(b.etype, b.nq, b.conn, b.body) for b in bw.blocks]
        parts = sh.pack_bodies(sh.body_costs(bblocks, bw.n_bodies), world)
        bm = sh.body_masks(bblocks, parts[rank])
        bshare, bnodes = sh.sub_workload(bw, bm, bodies=parts[rank])
        bf, _ = oracle.internal_force(bshare)
        by = oracle.operator_apply(bshare, bshare.v)
        out["batch"] = (bnodes, bf, by, parts[rank])
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_interfaces_and_match_the_unpartitioned_oracle():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the beam, assembled from both ranks (interface rows agree after the sum)
    wl = synth.small_beam(cells=(8, 2, 2))
    f_ref, _ = oracle.internal_force(wl)
    y_ref = oracle.operator_apply(wl, wl.v, a_K=1.0, a_C=1.0)
    gu_ref, gud_ref, gth_ref = oracle.vjp(wl, wl.v)
    refs = {"f": f_ref, "y": y_ref, "gu": gu_ref, "gud": gud_ref}
    seen = np.zeros(wl.n_nodes, int)
    ne = [got[r]["beam"][3] for r in range(world)]
    assert sum(ne) == wl.n_elem and min(ne) > 0
    for r in range(world):
        nodes, res, gth, _, sq = got[r]["beam"]
        seen[nodes] += 1
        for name, ref in refs.items():
            assert np.abs(res[name] - ref[nodes]).max() <= 1e-12 * np.abs(ref).max(), (r, name)
        assert abs(sq - float((f_ref ** 2).sum())) <= 1e-12 * float((f_ref ** 2).sum())
    assert seen.min() >= 1 and seen.max() == 2          # interface nodes are duplicated
    # the per-element parameter gradients, in slab order, are the oracle's
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    masks = shard.slab_partition(wl.X, blocks, world)
    for r in range(world):
        assert np.abs(got[r]["beam"][2] - gth_ref[masks[r][0]]).max() <= 1e-12 * np.abs(gth_ref).max()
    # the batch: every body on exactly one rank, values equal to the whole batch's
    bw = synth.batch_bodies(n_bodies=7, seed=21, ne_range=(30, 300))
    bf_ref, _ = oracle.internal_force(bw)
    by_ref = oracle.operator_apply(bw, bw.v)
    bodies = np.concatenate([got[r]["batch"][3] for r in range(world)])
    assert np.array_equal(np.sort(bodies), np.arange(bw.n_bodies))
    for r in range(world):
        nodes, bf, by, _ = got[r]["batch"]
        assert np.abs(bf - bf_ref[nodes]).max() <= 1e-12 * np.abs(bf_ref).max()
        assert np.abs(by - by_ref[nodes]).max() <= 1e-12 * np.abs(by_ref).max()
