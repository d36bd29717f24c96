"""The split-body exchange on the GPU, in one process: two shares of the beam
evaluated by the library, their interface rows packed into the compact
buffer by tlfe_gather_nodes, the two buffers added (what the all-reduce does
across GPUs), the sums written back by tlfe_scatter_nodes; the assembled
force, operator product and adjoint equal the whole mesh's and the oracle's.
No kernel waits on another rank."""

import numpy as np
import pytest

import oracle
import synth
from paper_2602_17002_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def relerr(got, ref):
    return float(np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("prec", [0, 1])
def test_two_shares_with_interface_sums_equal_the_whole_mesh(prec):
    from paper_2602_17002_gb300 import tlfe
    wl = synth.small_beam(cells=(12, 3, 3))
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    world = 2
    masks = shard.slab_partition(wl.X, blocks, world)
    nodes_all = [shard.local_blocks(blocks, m)[0] for m in masks]
    ifs = shard.interfaces(nodes_all)
    dt = torch.float32 if prec == 1 else torch.float64
    outs, bufs = [], []
    for r in range(world):
        share, nodes = shard.sub_workload(wl, masks[r])
        assert np.array_equal(nodes, nodes_all[r])
        mesh = tlfe.Mesh.from_workload(share, precision=prec)
        u = torch.from_numpy(share.u).cuda()
        ud, v = (torch.from_numpy(a).to("cuda", dt) for a in (share.udot, share.v))
        res = {"f": mesh.internal_force(u, ud), "y": mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)}
        res["gu"], res["gud"], _ = mesh.vjp(u, ud, v)
        idx = torch.from_numpy(ifs[r].local).cuda()
        pos = torch.from_numpy(ifs[r].pos).cuda()
        b = {}
        for k, x in res.items():
            buf = torch.full((ifs[r].n, 3), 7.0, dtype=dt, device="cuda")   # cleared by the gather
            tlfe.gather_nodes(x, idx, buf, out_idx=pos, clear=True)
            b[k] = buf
        outs.append((nodes, res, idx, pos))
        bufs.append(b)
        mesh.sync()
    total = {k: bufs[0][k] + bufs[1][k] for k in bufs[0]}   # the all-reduce of the GPUs
    full = tlfe.Mesh.from_workload(wl, precision=prec)
    u = torch.from_numpy(wl.u).cuda()
    ud, v = (torch.from_numpy(a).to("cuda", dt) for a in (wl.udot, wl.v))
    ref_gpu = {"f": full.internal_force(u, ud), "y": full.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)}
    ref_gpu["gu"], ref_gpu["gud"], _ = full.vjp(u, ud, v)
    f_ref, _ = oracle.internal_force(wl)
    gu_ref, gud_ref, _ = oracle.vjp(wl, wl.v)
    ref_orc = {"f": f_ref, "y": oracle.operator_apply(wl, wl.v, a_K=1.0, a_C=1.0), "gu": gu_ref, "gud": gud_ref}
    tol = 1e-12 if prec == 0 else 2e-5
    for nodes, res, idx, pos in outs:
        for k, x in res.items():
            tlfe.scatter_nodes(total[k], idx, x, buf_idx=pos)
            got = x.double().cpu().numpy()
            assert relerr(got, ref_orc[k][nodes]) <= tol, k
            assert relerr(got, ref_gpu[k].double().cpu().numpy()[nodes]) <= (1e-13 if prec == 0 else 1e-6), k
