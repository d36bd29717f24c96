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
