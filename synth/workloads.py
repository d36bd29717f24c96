"""Seeded workloads shaped like the five benchmark configurations.

Each builder returns a :class:`Workload`: one global node array, one or more
type-homogeneous element blocks, per-body materials, and the state (nodal
displacement u = x - X, nodal velocity) the hot path is evaluated at. Random
numbers come from ``numpy.random.default_rng(seed)`` (PCG64) so that the
oracle and the CUDA path see the same inputs.

Material parameters are Lame constants (mu, lam) plus the Kelvin-Voigt
viscous constants (mu_v, lam_v) and a density rho. Material model codes:
0 = St. Venant-Kirchhoff, 1 = compressible neo-Hookean.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .mesh import T4, T10, H8, Q27, NODES_PER_ELEM, box_mesh

SVK, NEOHOOKE = 0, 1
DEFAULT_NQ = {T4: 1, T10: 5, H8: 8, Q27: 27}


def lame_from_young(E: float, nu: float):
    """(mu, lam) of an isotropic solid from Young's modulus and Poisson ratio."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


@dataclass
class Block:
    etype: int
    nq: int
    conn: np.ndarray      # (n_elem, nodes_per_elem) int32, global node ids
    body: np.ndarray      # (n_elem,) int32 global body ids

    @property
    def n_elem(self):
        return self.conn.shape[0]


@dataclass
class Workload:
    name: str
    X: np.ndarray                     # (n_nodes, 3) float64
    blocks: List[Block]
    model: np.ndarray                 # (n_bodies,) int32
    params: np.ndarray                # (n_bodies, 5) float64: mu, lam, mu_v, lam_v, rho
    u: np.ndarray                     # (n_nodes, 3) float64 displacement
    udot: Optional[np.ndarray] = None  # (n_nodes, 3) float64 velocity
    v: Optional[np.ndarray] = None     # (n_nodes, 3) probe vector for K v
    elem_mu_lambda: Optional[np.ndarray] = None  # (n_elem_total, 2) override
    fixed: Optional[np.ndarray] = None  # (n_nodes,) uint8, 1 = clamped
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return self.X.shape[0]

    @property
    def n_elem(self):
        return sum(b.n_elem for b in self.blocks)

    @property
    def n_qp(self):
        return sum(b.n_elem * b.nq for b in self.blocks)

    @property
    def n_bodies(self):
        return self.model.shape[0]


def _uniform_noise(rng, shape, amp):
    return rng.uniform(-amp, amp, size=shape)


def block_t10_svk(cells: int = 4, seed: int = 1, vseed: int = 11, nq: int = 4) -> Workload:
    """1 m cube, cells^3 hex cells x 6 Kuhn T10, SVK E=1e7 Pa nu=0.3, nodal
    positions = reference + U(+-1 % of the cell edge), K v probe v ~ N(0, 1)."""
    m = box_mesh(T10, (cells, cells, cells), (1.0, 1.0, 1.0))
    h = 1.0 / cells
    rng = np.random.default_rng(seed)
    u = _uniform_noise(rng, m.X.shape, 0.01 * h)
    v = np.random.default_rng(vseed).standard_normal(m.X.shape)
    mu, lam = lame_from_young(1e7, 0.3)
    return Workload(
        name=f"block{cells}^3_T10_Q{nq}_SVK", X=m.X,
        blocks=[Block(T10, nq, m.conn, m.body)],
        model=np.array([SVK], np.int32),
        params=np.array([[mu, lam, 0.0, 0.0, 1000.0]]), u=u, udot=None, v=v)


def _bending_field(X, length, tip, rng, noise_amp):
    """Euler-Bernoulli-like cantilever bending about y with tip deflection
    `tip`: w(x) = tip x^2 (3L - x) / (2 L^3); sections stay plane and normal."""
    x, z = X[:, 0], X[:, 2]
    L = length
    w = tip * x * x * (3.0 * L - x) / (2.0 * L ** 3)
    dw = tip * 3.0 * x * (2.0 * L - x) / (2.0 * L ** 3)
    zc = 0.5 * (X[:, 2].max() + X[:, 2].min())
    u = np.zeros_like(X)
    u[:, 0] = -(z - zc) * dw
    u[:, 2] = w
    u += _uniform_noise(rng, X.shape, noise_amp)
    return u


def cantilever_beam(cells=(200, 20, 20), cell_edge: float = 0.05, seed: int = 2,
                    vseed: int = 12, pseed: int = 22, nq: int = 5,
                    damping: float = 1e3) -> Workload:
    """10 x 1 x 1 m cantilever (at the default cells), Kuhn T10, neo-Hookean
    mu=3.8e6 lam=5.8e6, Kelvin-Voigt mu_v = damping, lam_v = 0.

    Positions: a smooth bending field with tip deflection 5 % of the length
    (0.5 m at L = 10 m) plus U(+-0.1 % of the cell edge) noise; velocities
    N(0, 0.01^2) m/s per component."""
    nx, ny, nz = cells
    size = (nx * cell_edge, ny * cell_edge, nz * cell_edge)
    m = box_mesh(T10, cells, size)
    rng = np.random.default_rng(seed)
    u = _bending_field(m.X, size[0], 0.05 * size[0], rng, 0.001 * cell_edge)
    udot = 0.01 * np.random.default_rng(vseed).standard_normal(m.X.shape)
    v = np.random.default_rng(pseed).standard_normal(m.X.shape)
    return Workload(
        name=f"beam{nx}x{ny}x{nz}_T10_Q{nq}_NH_KV", X=m.X,
        blocks=[Block(T10, nq, m.conn, m.body)],
        model=np.array([NEOHOOKE], np.int32),
        params=np.array([[3.8e6, 5.8e6, damping, 0.0, 1000.0]]),
        u=u, udot=udot, v=v)


def q27_beam(cells=(8, 2, 2), cell_edge: float = 0.05, seed: int = 6, vseed: int = 16,
             pseed: int = 26, model: int = 1, damping: float = 1e3, mu01: float = 0.0,
             curve: float = 0.0) -> Workload:
    """Cantilever of Q27 bricks (one brick per cell, 3x3x3 Gauss points):
    neo-Hookean (model 1) or another law code, mu=3.8e6 lam=5.8e6, Kelvin-Voigt
    mu_v = damping. The same bending field as cantilever_beam (tip deflection
    5 % of the length) plus U(+-0.1 % of the cell edge) noise; velocities
    N(0, 0.01^2) m/s; probe v ~ N(0, 1). curve > 0 moves every node of the
    reference by U(+-curve * cell_edge), making the bricks non-affine."""
    nx, ny, nz = cells
    size = (nx * cell_edge, ny * cell_edge, nz * cell_edge)
    m = box_mesh(Q27, cells, size)
    rng = np.random.default_rng(seed)
    X = m.X.copy()
    if curve > 0:
        X += _uniform_noise(rng, X.shape, curve * cell_edge)
    u = _bending_field(X, size[0], 0.05 * size[0], rng, 0.001 * cell_edge)
    udot = 0.01 * np.random.default_rng(vseed).standard_normal(X.shape)
    v = np.random.default_rng(pseed).standard_normal(X.shape)
    params = np.array([[3.8e6, 5.8e6, damping, 0.0, 1000.0]])
    if mu01 != 0.0:
        params = np.concatenate([params, [[mu01]]], axis=1)
    return Workload(
        name=f"beam{nx}x{ny}x{nz}_Q27", X=X,
        blocks=[Block(Q27, 27, m.conn, m.body)],
        model=np.array([model], np.int32), params=params,
        u=u, udot=udot, v=v)


def small_beam(cells=(20, 2, 2), **kw) -> Workload:
    return cantilever_beam(cells=cells, **kw)


def _near_cube_cells(n_cells):
    n = max(1, int(round(n_cells ** (1.0 / 3.0))))
    m = max(1, int(round(n_cells / float(n * n))))
    return (n, n, m)


def batch_bodies(n_bodies: int = 512, seed: int = 3, ne_range=(1e3, 2e5),
                 cell_edge: float = 0.05) -> Workload:
    """Uneven batch: per body N_e ~ logU(ne_range), element type uniform in
    {T4 (1 qp), T10 (5 qp), H8 (8 qp)}, model uniform in {SVK, neo-Hookean},
    E ~ logU[1e6, 1e9] Pa, nu ~ U[0.2, 0.45]; near-cube blocks; state =
    reference + random symmetric 5 % affine stretch + U(+-1 % cell edge)."""
    rng = np.random.default_rng(seed)
    per_type = {T4: [], T10: [], H8: []}
    models = np.empty(n_bodies, np.int32)
    params = np.zeros((n_bodies, 5))
    X_all, u_all = [], []
    node_off = 0
    lo, hi = np.log(ne_range[0]), np.log(ne_range[1])
    for b in range(n_bodies):
        ne = float(np.exp(rng.uniform(lo, hi)))
        et = int(rng.integers(0, 3))
        models[b] = int(rng.integers(0, 2))
        E = float(np.exp(rng.uniform(np.log(1e6), np.log(1e9))))
        nu = float(rng.uniform(0.2, 0.45))
        mu, lam = lame_from_young(E, nu)
        params[b] = (mu, lam, 0.0, 0.0, 1000.0)
        ncell = ne / 6.0 if et in (T4, T10) else ne
        cells = _near_cube_cells(ncell)
        size = tuple(c * cell_edge for c in cells)
        m = box_mesh(et, cells, size, origin=(0.0, 0.0, 0.0))
        S = rng.uniform(-1.0, 1.0, size=(3, 3))
        A = np.eye(3) + 0.05 * 0.5 * (S + S.T)
        u = m.X @ (A - np.eye(3)).T + _uniform_noise(rng, m.X.shape, 0.01 * cell_edge)
        per_type[et].append((m.conn.astype(np.int64) + node_off, b))
        X_all.append(m.X)
        u_all.append(u)
        node_off += m.n_nodes
    blocks = []
    for et in (T4, T10, H8):
        if not per_type[et]:
            continue
        conn = np.concatenate([c for c, _ in per_type[et]]).astype(np.int32)
        body = np.concatenate([np.full(c.shape[0], b, np.int32) for c, b in per_type[et]])
        blocks.append(Block(et, DEFAULT_NQ[et], conn, body))
    X = np.concatenate(X_all)
    v = np.random.default_rng(seed + 100).standard_normal(X.shape)
    return Workload(name=f"batch{n_bodies}_mixed", X=X, blocks=blocks, model=models,
                    params=params, u=np.concatenate(u_all), udot=None, v=v)


def diff_block(cells: int = 55, seed: int = 4, tseed: int = 14, vseed: int = 24,
               nq: int = 5, damping: float = 1e3) -> Workload:
    """1 m cube of cells^3 x 6 Kuhn T10 elements, neo-Hookean with per-element
    mu ~ logN(ln 4e6, 0.25^2), lam ~ logN(ln 6e6, 0.25^2), Kelvin-Voigt
    mu_v = damping. State: U(+-1 % cell edge) noise, velocities N(0, 0.01^2).
    extra['theta_target'] = theta * (1 + 0.05 N(0, 1)) per element."""
    m = box_mesh(T10, (cells, cells, cells), (1.0, 1.0, 1.0))
    h = 1.0 / cells
    rng = np.random.default_rng(seed)
    mu = np.exp(rng.normal(np.log(4e6), 0.25, size=m.n_elem))
    lam = np.exp(rng.normal(np.log(6e6), 0.25, size=m.n_elem))
    theta = np.stack([mu, lam], axis=1)
    u = _uniform_noise(rng, m.X.shape, 0.01 * h)
    udot = 0.01 * rng.standard_normal(m.X.shape)
    trng = np.random.default_rng(tseed)
    theta_t = theta * (1.0 + 0.05 * trng.standard_normal(theta.shape))
    v = np.random.default_rng(vseed).standard_normal(m.X.shape)
    return Workload(
        name=f"diffblock{cells}^3_T10_Q{nq}_NH_KV", X=m.X,
        blocks=[Block(T10, nq, m.conn, m.body)],
        model=np.array([NEOHOOKE], np.int32),
        params=np.array([[4e6, 6e6, damping, 0.0, 1000.0]]),
        u=u, udot=udot, v=v, elem_mu_lambda=theta,
        extra={"theta_target": theta_t})


def newton_beams(n_bodies: int = 64, seed: int = 5, ne_range=(2e4, 3e5),
                 cell_edge: float = 0.05, nq: int = 5) -> Workload:
    """Implicit-step batch: beams with a 5:1:1 cell ratio and N_e ~
    logU(ne_range) Kuhn T10 elements, neo-Hookean mu=3.8e6 lam=5.8e6,
    rho=1000, no damping, the x = 0 face clamped; at rest in the reference
    configuration (u = 0, v = 0). Gravity and the step size are step
    parameters, not part of the workload."""
    rng = np.random.default_rng(seed)
    X_all, conns, bodies, fixed = [], [], [], []
    off = 0
    lo, hi = np.log(ne_range[0]), np.log(ne_range[1])
    for b in range(n_bodies):
        ne = float(np.exp(rng.uniform(lo, hi)))
        mcell = max(1, int(round((ne / 30.0) ** (1.0 / 3.0))))
        cells = (5 * mcell, mcell, mcell)
        size = tuple(c * cell_edge for c in cells)
        m = box_mesh(T10, cells, size)
        X_all.append(m.X)
        conns.append(m.conn.astype(np.int64) + off)
        bodies.append(np.full(m.n_elem, b, np.int32))
        fixed.append((np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8))
        off += m.n_nodes
    X = np.concatenate(X_all)
    params = np.tile(np.array([[3.8e6, 5.8e6, 0.0, 0.0, 1000.0]]), (n_bodies, 1))
    return Workload(
        name=f"newton{n_bodies}beams_T10_Q{nq}_NH", X=X,
        blocks=[Block(T10, nq, np.concatenate(conns).astype(np.int32), np.concatenate(bodies))],
        model=np.full(n_bodies, NEOHOOKE, np.int32), params=params,
        u=np.zeros_like(X), udot=np.zeros_like(X), v=None,
        fixed=np.concatenate(fixed))


def split_bodies(wl: Workload) -> List[Workload]:
    """One single-body workload per body of a one-block workload whose bodies
    own contiguous node ranges (as newton_beams builds them); node ids are
    renumbered from zero and per-node arrays sliced."""
    assert len(wl.blocks) == 1
    blk = wl.blocks[0]
    out = []
    for b in range(wl.n_bodies):
        sel = blk.body == b
        conn = blk.conn[sel]
        lo, hi = int(conn.min()), int(conn.max()) + 1
        sl = slice(lo, hi)
        pick = lambda a: None if a is None else np.ascontiguousarray(a[sl])  # noqa: E731
        out.append(Workload(
            name=f"{wl.name}_body{b}", X=np.ascontiguousarray(wl.X[sl]),
            blocks=[Block(blk.etype, blk.nq, (conn - lo).astype(np.int32), np.zeros(conn.shape[0], np.int32))],
            model=wl.model[b:b + 1].copy(), params=wl.params[b:b + 1].copy(),
            u=pick(wl.u), udot=pick(wl.udot), v=pick(wl.v), fixed=pick(wl.fixed)))
    return out
