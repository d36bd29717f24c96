"""Structured mesh topology: boxes of hexahedral cells, kept as H8 bricks or
split into six Kuhn tetrahedra per cell (T4 corners only, T10 with mid-edge
nodes).

Node ordering conventions follow the paper's element tables:

* T10 (Appendix A.1 node table): corners 1-4 are the vertices with parent
  coordinates (0,0,0), (1,0,0), (0,1,0), (0,0,1); nodes 5-10 sit on the edges
  (1,2), (2,3), (1,3), (1,4), (2,4), (3,4).
* T4: the four corners in the same order.
* Q27 (Appendix, 27-node hexahedron table): node i + 3 j + 9 k at parent
  coordinates (i - 1, j - 1, k - 1), on the half-step grid.
* H8: tensor-product ordering with the first index fastest, as in the Q27
  table of Appendix A.2, on the vertex grid {-1, 1}^3.

Every tetrahedron is oriented so that det[c2-c1, c3-c1, c4-c1] > 0, i.e. the
parent-to-reference Jacobian determinant is positive (Section 6).
"""

from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

T4, T10, H8, Q27 = 0, 1, 2, 3
NODES_PER_ELEM = {T4: 4, T10: 10, H8: 8, Q27: 27}
TYPE_NAME = {T4: "T4", T10: "T10", H8: "H8", Q27: "Q27"}


@dataclass
class Mesh:
    """One element block over a node set.

    X     : (n_nodes, 3) float64 reference coordinates.
    conn  : (n_elem, nodes_per_elem) int32, 0-based node ids.
    etype : T4 / T10 / H8.
    body  : (n_elem,) int32 body id of each element.
    """

    X: np.ndarray
    conn: np.ndarray
    etype: int
    body: np.ndarray = field(default=None)

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.conn = np.ascontiguousarray(self.conn, dtype=np.int32)
        if self.body is None:
            self.body = np.zeros(self.conn.shape[0], dtype=np.int32)
        self.body = np.ascontiguousarray(self.body, dtype=np.int32)

    @property
    def n_nodes(self) -> int:
        return self.X.shape[0]

    @property
    def n_elem(self) -> int:
        return self.conn.shape[0]


def _kuhn_paths():
    """The six monotone vertex paths (0,0,0) -> (1,1,1) of a unit cube.

    Each path steps once along every axis; the permutation of axes picks one
    of the six tetrahedra sharing the main diagonal. All cells use the same
    diagonal, so the split is conforming across cell faces.
    """
    paths = []
    for perm in permutations(range(3)):
        v = np.zeros(3, dtype=np.int64)
        verts = [v.copy()]
        for ax in perm:
            v[ax] += 1
            verts.append(v.copy())
        paths.append(np.array(verts))
    return paths


def _grid_index(ix, iy, iz, nx1, ny1):
    return ix + nx1 * (iy + ny1 * iz)


def box_mesh(etype: int, cells, size, origin=(0.0, 0.0, 0.0)) -> Mesh:
    """Box [origin, origin+size] with cells = (nx, ny, nz) hexahedral cells.

    T4 / H8 use the vertex grid ((nx+1)(ny+1)(nz+1) nodes). T10 uses the
    half-step grid ((2nx+1)(2ny+1)(2nz+1) nodes); every half-grid point is a
    corner or a mid-edge node of the Kuhn split.
    """
    nx, ny, nz = (int(c) for c in cells)
    lx, ly, lz = (float(s) for s in size)
    step = 2 if etype in (T10, Q27) else 1
    gx, gy, gz = step * nx + 1, step * ny + 1, step * nz + 1
    xs = origin[0] + np.linspace(0.0, lx, gx)
    ys = origin[1] + np.linspace(0.0, ly, gy)
    zs = origin[2] + np.linspace(0.0, lz, gz)
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    X = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1)

    # cells ordered with x fastest
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cell = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)  # (n_cells, 3)

    if etype == Q27:
        # half-step grid; node i + 3 j + 9 k of a cell sits at 2 cell + (i, j, k)
        conn = np.empty((cell.shape[0], 27), dtype=np.int64)
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    p = 2 * cell + np.array([i, j, k])
                    conn[:, i + 3 * j + 9 * k] = _grid_index(p[:, 0], p[:, 1], p[:, 2], gx, gy)
        return Mesh(X, conn.astype(np.int32), Q27)

    if etype == H8:
        conn = np.empty((cell.shape[0], 8), dtype=np.int64)
        for k in range(2):
            for j in range(2):
                for i in range(2):
                    p = cell + np.array([i, j, k])
                    conn[:, i + 2 * j + 4 * k] = _grid_index(p[:, 0], p[:, 1], p[:, 2], gx, gy)
        return Mesh(X, conn.astype(np.int32), H8)

    conns = []
    for path in _kuhn_paths():
        corners = path.copy()  # (4, 3) offsets in {0,1}
        e1, e2, e3 = corners[1] - corners[0], corners[2] - corners[0], corners[3] - corners[0]
        if np.linalg.det(np.stack([e1, e2, e3], axis=1).astype(float)) < 0:
            corners[[2, 3]] = corners[[3, 2]]
        if etype == T4:
            cols = []
            for c in corners:
                p = cell + c
                cols.append(_grid_index(p[:, 0], p[:, 1], p[:, 2], gx, gy))
            conns.append(np.stack(cols, axis=1))
        else:
            # corners live at even half-grid indices; the midpoint of edge
            # (a, b) is the half-grid point 2*cell + a + b
            pts = [2 * c for c in corners]
            edges = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
            pts += [corners[a] + corners[b] for a, b in edges]
            cols = []
            for p0 in pts:
                p = 2 * cell + p0
                cols.append(_grid_index(p[:, 0], p[:, 1], p[:, 2], gx, gy))
            conns.append(np.stack(cols, axis=1))
    # interleave: the six tets of a cell are consecutive
    conn = np.stack(conns, axis=1).reshape(-1, conns[0].shape[1])
    return Mesh(X, conn.astype(np.int32), etype)


def concat_meshes(meshes):
    """Disjoint union of several single-type meshes: node ids are offset and
    every element keeps the body id of its source mesh index."""
    X = []
    conn = []
    body = []
    off = 0
    for b, m in enumerate(meshes):
        X.append(m.X)
        conn.append(m.conn.astype(np.int64) + off)
        body.append(np.full(m.n_elem, b, dtype=np.int32))
        off += m.n_nodes
    etype = meshes[0].etype
    assert all(m.etype == etype for m in meshes)
    return Mesh(np.concatenate(X), np.concatenate(conn).astype(np.int32), etype,
                np.concatenate(body))


def face_corners(etype: int, face: int):
    """Local corner nodes of a parent face: tetrahedra, face k is opposite
    vertex k (the other three corners in increasing order); bricks, face
    2 d + s holds the corners whose bit d equals s (Q27: the corner nodes
    with tensor index 0 or 2 along d)."""
    if etype in (T4, T10):
        return [j for j in range(4) if j != face]
    d, s = divmod(face, 2)
    if etype == Q27:
        out = []
        for n in range(27):
            idx = (n % 3, (n // 3) % 3, n // 9)
            if all(t in (0, 2) for t in idx) and idx[d] == 2 * s:
                out.append(n)
        return out
    return [n for n in range(8) if ((n >> d) & 1) == s]


def boundary_faces(etype: int, conn: np.ndarray):
    """(element, local face) of every face that belongs to exactly one element."""
    nf = 4 if etype in (T4, T10) else 6   # bricks (H8, Q27): 6 faces
    seen = {}
    for e in range(conn.shape[0]):
        for f in range(nf):
            key = tuple(sorted(int(conn[e, c]) for c in face_corners(etype, f)))
            seen.setdefault(key, []).append((e, f))
    faces = [v[0] for v in seen.values() if len(v) == 1]
    faces.sort()
    return np.array([e for e, _ in faces], np.int32), np.array([f for _, f in faces], np.int32)
