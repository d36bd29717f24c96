"""Work split of the element hot path over several GPUs (one process per GPU).

Two splits, both host logic on index arrays (no element arithmetic):

* Independent bodies (the batch of uneven bodies, the Newton step of many
  bodies; Sec. 7 is a per-body step): ``pack_bodies`` gives every rank a
  disjoint set of bodies by a cost model (quadrature points x element nodes
  per element, summed over the body), largest first onto the least-loaded
  rank. The ranks then need no exchange at all.

* One body (the beam, the differentiation block): ``slab_partition`` cuts
  the elements into equal-count slabs along an axis (by element centroid);
  each rank holds its slab's elements and every node they touch, so the
  nodes on a slab interface are duplicated. The assembled force (Sec. 4.3)
  at an interface node is the sum of its ranks' partial forces:
  ``InterfaceSum`` adds them after each operator application through one
  compact buffer holding the interface nodes only (gathered and scattered by
  the library's tlfe_gather_nodes / tlfe_scatter_nodes, summed by an
  all-reduce of torch.distributed; peers' data is copied into local memory
  by the collective, never read in place).

* The backward-Euler step of one split body (Sec. 7): ``split_newton_step``
  runs the inexact Newton / Jacobi-PCG iteration of tlfe_newton_step from
  the host over the rank's shares, with the interface sum after every
  operator application and an FP64 all-reduce of the CG scalars (p.q, then
  r.z and r.r) per iteration; ``SplitShare`` does a share's work in the
  library, ``DistGroup`` / ``LocalGroup`` make the exchanges across
  processes or within one.

``local_blocks`` renumbers a rank's share into a self-contained mesh.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

NPE = {0: 4, 1: 10, 2: 8, 3: 27}


def element_cost(etype: int, nq: int) -> int:
    """Work per element in the cost model: quadrature points x element nodes."""
    return nq * NPE[etype]


def body_costs(blocks: Sequence[Tuple[int, int, np.ndarray, np.ndarray]], n_bodies: int) -> np.ndarray:
    """Cost of every body: blocks are (etype, nq, conn, body)."""
    c = np.zeros(n_bodies, np.float64)
    for et, nq, conn, body in blocks:
        np.add.at(c, np.asarray(body), float(element_cost(et, nq)))
    return c


def pack_bodies(costs: np.ndarray, n_ranks: int) -> List[np.ndarray]:
    """Longest-processing-time bin packing: bodies by decreasing cost, each onto
    the rank with the least cost so far (ties: the lower rank). Returns the
    sorted body ids of every rank; every body goes to exactly one rank."""
    order = np.argsort(-np.asarray(costs, np.float64), kind="stable")
    load = np.zeros(n_ranks)
    out = [[] for _ in range(n_ranks)]
    for b in order:
        r = int(np.argmin(load))
        out[r].append(int(b))
        load[r] += costs[b]
    return [np.array(sorted(o), np.int64) for o in out]


def body_masks(blocks, bodies: np.ndarray) -> List[np.ndarray]:
    """Per block, the elements that belong to the given bodies."""
    return [np.isin(np.asarray(body), bodies) for _, _, _, body in blocks]


def slab_partition(X: np.ndarray, blocks, n_ranks: int, axis: int = 0) -> List[List[np.ndarray]]:
    """Per rank, per block, the elements of its slab: all elements ordered by
    the centroid coordinate along `axis` (ties by global element index) and
    cut into n_ranks runs of equal count."""
    cents, owners = [], []
    for bi, (et, nq, conn, body) in enumerate(blocks):
        conn = np.asarray(conn)
        if conn.shape[0] == 0:
            continue
        cents.append(X[conn, axis].mean(axis=1))
        owners.append(np.stack([np.full(conn.shape[0], bi), np.arange(conn.shape[0])], axis=1))
    cent = np.concatenate(cents)
    own = np.concatenate(owners)
    order = np.lexsort((np.arange(cent.size), cent))
    cuts = [cent.size * r // n_ranks for r in range(n_ranks + 1)]
    masks = [[np.zeros(np.asarray(b[2]).shape[0], bool) for b in blocks] for _ in range(n_ranks)]
    for r in range(n_ranks):
        sel = own[order[cuts[r]:cuts[r + 1]]]
        for bi in np.unique(sel[:, 0]):
            masks[r][bi][sel[sel[:, 0] == bi, 1]] = True
    return masks


def local_blocks(blocks, masks: Sequence[np.ndarray]):
    """A rank's share as a self-contained mesh: the global ids of its nodes
    (sorted) and its blocks with connectivity renumbered to them."""
    used = [np.asarray(conn)[m].ravel() for (_, _, conn, _), m in zip(blocks, masks)]
    nodes = np.unique(np.concatenate(used)) if used else np.zeros(0, np.int64)
    out = []
    for (et, nq, conn, body), m in zip(blocks, masks):
        c = np.asarray(conn)[m]
        out.append((et, nq, np.searchsorted(nodes, c).astype(np.int32), np.asarray(body)[m]))
    return nodes, out


def sub_workload(wl, masks: Sequence[np.ndarray], bodies: np.ndarray = None):
    """A rank's share of a workload object (X, blocks of (etype, nq, conn,
    body), model, params and optional u, udot, v, fixed, elem_mu_lambda, as
    the seeded generators build them) as a new object of the same type:
    elements masks[b] of every block, the nodes they touch (renumbered), and,
    with `bodies`, only those bodies' materials with body ids renumbered in
    ascending order. Returns (share, global node ids)."""
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    nodes, loc = local_blocks(blocks, masks)
    Blk = type(wl.blocks[0])
    new_blocks = []
    for et, nq, conn, body in loc:
        body = np.asarray(body)
        if bodies is not None:
            body = np.searchsorted(bodies, body).astype(np.int32)
        new_blocks.append(Blk(et, nq, conn, body.astype(np.int32)))
    pick = lambda a: None if a is None else np.ascontiguousarray(a[nodes])  # noqa: E731
    model, params = wl.model, wl.params
    if bodies is not None:
        model, params = np.asarray(model)[bodies], np.asarray(params)[bodies]
    eml = None
    if wl.elem_mu_lambda is not None:
        off, parts = 0, []
        for b, m in zip(wl.blocks, masks):
            parts.append(wl.elem_mu_lambda[off:off + b.n_elem][m])
            off += b.n_elem
        eml = np.concatenate(parts)
    share = type(wl)(name=f"{wl.name}_share", X=np.ascontiguousarray(wl.X[nodes]), blocks=new_blocks,
                     model=model, params=params, u=pick(wl.u), udot=pick(wl.udot), v=pick(wl.v),
                     elem_mu_lambda=eml, fixed=pick(wl.fixed))
    return share, nodes


@dataclass
class Interface:
    """The duplicated nodes of one rank: local row ids, their positions in the
    global interface list, and that list's length (the same on every rank)."""
    local: np.ndarray   # int32 [k] rows of the rank's node arrays
    pos: np.ndarray     # int32 [k] positions in the compact buffer
    n: int              # interface nodes over all ranks
    owner: np.ndarray   # bool [k]: this rank owns the node (the lowest rank holding it)


def interfaces(rank_nodes: Sequence[np.ndarray]) -> List[Interface]:
    """Nodes held by two or more ranks, numbered in ascending global id, and
    each rank's view of them."""
    allnodes = np.concatenate(rank_nodes)
    ids, counts = np.unique(allnodes, return_counts=True)
    shared = ids[counts > 1]
    out, seen = [], np.zeros(0, np.int64)
    for nodes in rank_nodes:
        is_sh = np.isin(nodes, shared)
        loc = np.flatnonzero(is_sh).astype(np.int32)
        glob = nodes[is_sh]
        pos = np.searchsorted(shared, glob).astype(np.int32)
        owner = ~np.isin(glob, seen)
        seen = np.union1d(seen, glob)
        out.append(Interface(loc, pos, int(shared.size), owner))
    return out


def owned_rows(n_local: int, iface: Interface) -> np.ndarray:
    """Rows a rank counts in a sum over nodes (a norm, a loss): all but the
    interface nodes some lower rank holds."""
    keep = np.ones(n_local, bool)
    keep[iface.local[~iface.owner]] = False
    return keep


class InterfaceSum:
    """Sums the partial rows of the interface nodes over all ranks, in place:
    the rank's interface rows go to their positions of a zeroed compact buffer
    (tlfe_gather_nodes), the buffer is all-reduced (SUM) over the process
    group, and the sums go back to the rows (tlfe_scatter_nodes). `pack` /
    `unpack` may be replaced (the CPU tests pass their own); the defaults are
    the library's kernels and take CUDA arrays only."""

    def __init__(self, iface: Interface, dtype, device, group=None, pack=None, unpack=None):
        import torch
        self.iface = iface
        self.group = group
        self.idx = torch.as_tensor(iface.local, dtype=torch.int32, device=device)
        self.pos = torch.as_tensor(iface.pos, dtype=torch.int32, device=device)
        self.buf = torch.zeros((max(1, iface.n), 3), dtype=dtype, device=device)
        self.pack = pack or self._pack
        self.unpack = unpack or self._unpack

    @staticmethod
    def _pack(x, idx, buf, pos):
        from . import tlfe
        tlfe.gather_nodes(x, idx, buf, out_idx=pos, clear=True)

    @staticmethod
    def _unpack(buf, pos, x, idx):
        from . import tlfe
        tlfe.scatter_nodes(buf, idx, x, buf_idx=pos)

    def __call__(self, x):
        import torch.distributed as dist
        self.pack(x, self.idx, self.buf, self.pos)
        dist.all_reduce(self.buf, op=dist.ReduceOp.SUM, group=self.group)
        self.unpack(self.buf, self.pos, x, self.idx)
        return x


# ---------------------------------------------------------------------------
# Backward-Euler step of one body split across ranks (Sec. 7)
# ---------------------------------------------------------------------------

class DistGroup:
    """The exchanges of a split step when every rank is its own process (one
    share per process): interface rows by an InterfaceSum (one compact buffer
    per dtype of the rows summed: the FP64 residual, the operator mesh's
    diagonal and CG products), scalars by an FP64 all-reduce of
    torch.distributed. `pack` / `unpack` as for InterfaceSum."""

    def __init__(self, iface: Interface, device, group=None, pack=None, unpack=None):
        self.iface, self.device, self.group = iface, device, group
        self.pack, self.unpack = pack, unpack
        self.sums = {}

    def sum_rows(self, xs):
        (x,) = xs
        if x.dtype not in self.sums:
            self.sums[x.dtype] = InterfaceSum(self.iface, x.dtype, self.device, group=self.group,
                                              pack=self.pack, unpack=self.unpack)
        self.sums[x.dtype](x)

    def sum_scalars(self, ds) -> np.ndarray:
        import torch.distributed as dist
        (d,) = ds
        dist.all_reduce(d, op=dist.ReduceOp.SUM, group=self.group)
        return d.cpu().numpy().astype(np.float64)


class LocalGroup:
    """The same exchanges when one process holds every share of the body (the
    shares run one after another on one device): the interface rows of all
    shares are added in share order through one compact buffer per share and
    dtype, and the scalars are added in share order on the host. `pack` /
    `unpack` are those of InterfaceSum (the library's row kernels by default)."""

    def __init__(self, ifaces: Sequence[Interface], device, pack=None, unpack=None):
        self.ifaces, self.device = list(ifaces), device
        self.pack, self.unpack = pack, unpack
        self.sums = {}

    def sum_rows(self, xs):
        import torch
        dt = xs[0].dtype
        if dt not in self.sums:
            sums = [InterfaceSum(itf, dt, self.device, pack=self.pack, unpack=self.unpack) for itf in self.ifaces]
            self.sums[dt] = (sums, torch.zeros_like(sums[0].buf))
        sums, total = self.sums[dt]
        total.zero_()
        for s, x in zip(sums, xs):
            s.pack(x, s.idx, s.buf, s.pos)
            total += s.buf          # stands in for the all-reduce of the buffers
        for s, x in zip(sums, xs):
            s.unpack(total, s.pos, x, s.idx)

    def sum_scalars(self, ds) -> np.ndarray:
        tot = None
        for d in ds:
            a = d.cpu().numpy().astype(np.float64)
            tot = a if tot is None else tot + a
        return tot


def split_newton_step(parts, group, h, newton_rtol=1e-8, cg_rtol=1e-4, max_newton=20, max_cg=2000):
    """Inexact Newton / Jacobi-PCG step of Sec. 7 on one body split into the
    shares `parts` (this process's shares; the group adds the other ranks'):
    g(v) = M/h (v - v_n) + f_int(q_n + h v, v) - f_ff (Eq. residual), each
    Newton iteration solving (M/h + h K^e + C) dv = -g (the symmetric part of
    dg/dv, as tlfe_newton_step) by Jacobi-PCG, then v += dv, until
    ||g|| <= newton_rtol ||g(v_n)||. Per operator application the ranks sum
    the interface rows (group.sum_rows); per CG iteration they all-reduce
    p.q, then r.z and r.r (group.sum_scalars: three FP64 scalars). Each share
    (SplitShare below, or a stand-in with the same methods) does its own
    vector and element work. Returns a report; every share holds its v."""
    for s in parts:
        s.start()
    def residual_norm():
        group.sum_rows([s.residual(h) for s in parts])
        return float(np.sqrt(max(group.sum_scalars([s.dot_g() for s in parts])[0], 0.0)))
    g0 = residual_norm()
    gn, it, cg_total = g0, 0, 0
    while g0 > 0.0 and gn > newton_rtol * g0 and it < max_newton:
        group.sum_rows([s.diag(h) for s in parts])
        rz, rr = group.sum_scalars([s.cg_start() for s in parts])[:2]
        r0 = np.sqrt(max(rr, 0.0))
        k = 0
        while np.sqrt(max(rr, 0.0)) > cg_rtol * r0 and k < max_cg:
            group.sum_rows([s.apply(h) for s in parts])
            pq = group.sum_scalars([s.cg_pq() for s in parts])[0]
            alpha = rz / pq
            rz1, rr = group.sum_scalars([s.cg_update(alpha) for s in parts])[:2]
            beta = rz1 / rz
            rz = rz1
            for s in parts:
                s.cg_direction(beta)
            k += 1
        cg_total += k
        for s in parts:
            s.newton_update()
        gn = residual_norm()
        it += 1
    conv = not (g0 > 0.0 and gn > newton_rtol * g0)
    return {"newton_iters": it, "cg_iters": cg_total, "status": 0 if conv else 5,
            "rel_residual": gn / g0 if g0 > 0.0 else 0.0}


class SplitShare:
    """One share of a split body on the GPU for split_newton_step: its FP64
    mesh for the residual, its operator mesh (FP64 or FP32) for the CG
    products and the Jacobi diagonal, and the library's split-step vector
    kernels (tlfe.SplitCG); every computation runs in libtlfe. u_n, v_n:
    float64 CUDA (n_rows, 3) of the share's nodes; fixed: uint8 CUDA [n_rows]
    or None; own: uint8 CUDA [n_rows] (owned_rows) or None; gravity: b0."""

    def __init__(self, res_mesh, op_mesh, u_n, v_n, gravity, fixed=None, own=None):
        import torch
        from . import tlfe
        self.res, self.op = res_mesh, op_mesh
        n = res_mesh.n_nodes
        self.u_n, self.v_n = u_n, v_n
        self.grav = [float(g) for g in gravity]
        self.cg = tlfe.SplitCG(n, op_mesh.precision, fixed=fixed, own=own)
        z = lambda: torch.zeros((n, 3), dtype=torch.float64, device=u_n.device)  # noqa: E731
        self.v, self.u, self.w, self.f, self.y, self.g = z(), z(), z(), z(), z(), z()
        self.v_op = None if op_mesh.precision == tlfe.FP64 else \
            torch.zeros((n, 3), dtype=op_mesh.torch_dtype, device=u_n.device)
        self.D = torch.zeros((n, 3), dtype=op_mesh.torch_dtype, device=u_n.device)

    def _ud(self):
        return self.v if self.v_op is None else self.v_op

    def start(self):
        self.cg.velocity(self.v_n, False, self.v)

    def residual(self, h):
        self.cg.prep(h, self.grav, self.u_n, self.v_n, self.v, self.u, self.w,
                     None if self.v_op is None else self.v_op)
        self.res.internal_force(self.u, self.v, out=self.f)
        self.res.tangent_matvec(self.u, self.v, self.w, 1.0 / h, 0.0, 0.0, out=self.y)
        self.cg.residual(self.f, self.y, self.g)
        return self.g

    def dot_g(self):
        return self.cg.dot(self.g, self.g)

    def diag(self, h):
        return self.op.jacobi_diag(self.u, self._ud(), 1.0 / h, h, 1.0, out=self.D)

    def cg_start(self):
        self.cg.cg_dinv(self.D)
        return self.cg.cg_start(self.g)

    def apply(self, h):
        return self.op.newton_operator(self.u, self._ud(), self.cg.p, 1.0 / h, h, 1.0, out=self.cg.q)

    def cg_pq(self):
        return self.cg.cg_pq()

    def cg_update(self, alpha):
        return self.cg.cg_update(alpha)

    def cg_direction(self, beta):
        self.cg.cg_direction(beta)

    def newton_update(self):
        self.cg.velocity(self.v, True, self.v)
