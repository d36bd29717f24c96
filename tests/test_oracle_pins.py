"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these tests re-types an oracle formula: each checks the oracle against
a closed form, an invariant, a finite difference, exact integration, a printed
table or brute force, chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""

import math
import os
from itertools import product

import numpy as np
import pytest

import oracle
import synth
from synth import T4, T10, H8, Q27
from synth.workloads import DEFAULT_NQ, Block, Workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ATOL = 1e-12


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


def _rand_F(rng, scale=0.2):
    return np.eye(3) + scale * rng.uniform(-1, 1, size=(3, 3))


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ------------------------------------------------------------------------
# Appendix A: shape functions and parent gradients
# ------------------------------------------------------------------------

def test_t10_kronecker_at_printed_nodes():
    tab = _load_golden("t10_parent_nodes.txt")
    assert tab.shape == (10, 8)
    for j in range(10):
        L, xi = tab[j, 1:5], tab[j, 5:8]
        # barycentric relation of Appendix A.1: xi = L2, eta = L3, zeta = L4
        assert np.allclose(xi, L[1:4]) and abs(L.sum() - 1.0) < 1e-15
        s = oracle.shape(T10, xi)
        e = np.zeros(10)
        e[j] = 1.0
        assert np.allclose(s, e, atol=1e-15), (j, s)


@pytest.mark.parametrize("etype", [T4, T10, H8, Q27])
def test_partition_of_unity_and_gradient_by_fd(etype):
    rng = np.random.default_rng(0)
    for _ in range(20):
        if etype in (H8, Q27):
            xi = rng.uniform(-1, 1, 3)
        else:
            xi = rng.dirichlet(np.ones(4))[1:]
        s = oracle.shape(etype, xi)
        g = oracle.shape_grad(etype, xi)
        assert abs(s.sum() - 1.0) < 1e-14
        assert np.abs(g.sum(axis=0)).max() < 1e-13
        # the printed gradient table equals the derivative of the printed s
        h = 1e-6
        for k in range(3):
            d = np.zeros(3)
            d[k] = h
            fd = (oracle.shape(etype, xi + d) - oracle.shape(etype, xi - d)) / (2 * h)
            assert np.abs(fd - g[:, k]).max() < 1e-8


def test_t10_is_barycentric_quadratic_lagrange():
    # corners L_k (2 L_k - 1), edges 4 L_a L_b with the Appendix A.1 node table
    edges = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
    rng = np.random.default_rng(1)
    for _ in range(20):
        L = rng.dirichlet(np.ones(4))
        s = oracle.shape(T10, L[1:])
        ref = [L[k] * (2 * L[k] - 1) for k in range(4)] + [4 * L[a] * L[b] for a, b in edges]
        assert np.allclose(s, ref, atol=1e-15)


def test_q27_kronecker_at_printed_nodes():
    tab = _load_golden("q27_parent_nodes.txt")
    assert tab.shape == (27, 7)
    for row in tab:
        n = int(row[0]) - 1
        assert n == int(row[1]) + 3 * int(row[2]) + 9 * int(row[3])
        s = oracle.shape(Q27, row[4:7])
        e = np.zeros(27)
        e[n] = 1.0
        assert np.allclose(s, e, atol=1e-15), (n, s)


def test_q27_matches_printed_expanded_shape_functions():
    # a few entries of the printed expanded vector s(xi, eta, zeta) (App., Q27)
    rng = np.random.default_rng(13)
    for _ in range(10):
        x, y, z = rng.uniform(-1, 1, 3)
        s = oracle.shape(Q27, np.array([x, y, z]))
        s1 = (y**2 * x**2 * z**2 / 8 - y**2 * x**2 * z / 8 - y**2 * x * z**2 / 8 + y**2 * x * z / 8
              - y * x**2 * z**2 / 8 + y * x**2 * z / 8 + y * x * z**2 / 8 - y * x * z / 8)
        s14 = (-y**2 * x**2 * z**2 + y**2 * x**2 + y**2 * z**2 - y**2 + x**2 * z**2 - x**2 - z**2 + 1)
        s27 = (y**2 * x**2 * z**2 / 8 + y**2 * x**2 * z / 8 + y**2 * x * z**2 / 8 + y**2 * x * z / 8
               + y * x**2 * z**2 / 8 + y * x**2 * z / 8 + y * x * z**2 / 8 + y * x * z / 8)
        s5 = (y**2 * x**2 * z**2 / 2 - y**2 * x**2 * z / 2 - y**2 * z**2 / 2 + y**2 * z / 2
              - x**2 * z**2 / 2 + x**2 * z / 2 + z**2 / 2 - z / 2)
        for got, ref in ((s[0], s1), (s[13], s14), (s[26], s27), (s[4], s5)):
            assert abs(got - ref) < 1e-14


def test_q27_gauss_rule_exact_to_degree_5():
    pts, w = oracle.quad_rule(Q27, 27)
    for a, b, c in product(range(7), repeat=3):
        ex = np.prod([0.0 if k % 2 else 2.0 / (k + 1) for k in (a, b, c)])
        val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        if max(a, b, c) <= 5:
            assert abs(val - ex) < 1e-14
        elif (a, b, c) == (6, 0, 0):
            assert abs(val - ex) > 1e-3      # and no further


def test_h8_kronecker_q27_ordering():
    for k, j, i in product(range(2), repeat=3):
        xi = np.array([2 * i - 1, 2 * j - 1, 2 * k - 1], float)
        s = oracle.shape(H8, xi)
        assert abs(s[i + 2 * j + 4 * k] - 1.0) < 1e-15 and abs(s.sum() - 1) < 1e-15


# ------------------------------------------------------------------------
# Section 6: quadrature
# ------------------------------------------------------------------------

def _tet_monomial(a, b, c):
    # int over the unit tetrahedron of xi^a eta^b zeta^c = a! b! c! / (a+b+c+3)!
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


@pytest.mark.parametrize("nq,deg", [(1, 1), (4, 2), (5, 3)])
def test_tet_rules_exact_to_their_degree(nq, deg):
    pts, w = oracle.quad_rule(T10, nq)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15
    for a, b, c in product(range(deg + 2), repeat=3):
        d = a + b + c
        if d > deg + 1:
            continue
        val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        if d <= deg:
            assert abs(val - _tet_monomial(a, b, c)) < 1e-15, (a, b, c)
    # and not exact one degree higher (the rule is what it claims, no more)
    errs = [abs(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c) - _tet_monomial(a, b, c))
            for a, b, c in product(range(deg + 2), repeat=3) if a + b + c == deg + 1]
    assert max(errs) > 1e-6


def test_t10_five_point_rule_has_negative_centroid_weight():
    pts, w = oracle.quad_rule(T10, 5)
    assert np.allclose(pts[0], 0.25) and abs(w[0] + 2.0 / 15.0) < 1e-15
    assert np.allclose(w[1:], 3.0 / 40.0)


def test_hex_gauss_and_exact_rules():
    pts, w = oracle.quad_rule(H8, 8)
    for a, b, c in product(range(5), repeat=3):
        ex = np.prod([0.0 if k % 2 else 2.0 / (k + 1) for k in (a, b, c)])
        val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        if max(a, b, c) <= 3:
            assert abs(val - ex) < 1e-14
    for order in (4, 5):
        pts, w = oracle.exact_rule(T10, order)
        for a, b, c in product(range(7), repeat=3):
            if a + b + c <= 2 * order - 3:
                val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(val - _tet_monomial(a, b, c)) < 1e-15


# ------------------------------------------------------------------------
# Section 6: H = Hp (U Hp)^{-1}, J_p
# ------------------------------------------------------------------------

@pytest.mark.parametrize("etype,nq", [(T4, 1), (T10, 4), (T10, 5), (H8, 8), (Q27, 27)])
def test_precompute_UH_identity_and_volume(etype, nq):
    m = synth.box_mesh(etype, (2, 2, 1), (0.8, 0.6, 0.3))
    rng = np.random.default_rng(2)
    X = m.X.copy()
    if etype == T10:  # curve the reference a little: still U H = I
        X += rng.uniform(-0.01, 0.01, X.shape)
    H, wJ, bad = oracle.precompute(etype, nq, m.conn, X)
    assert bad == 0
    for e in range(m.n_elem):
        Xe = X[m.conn[e]]
        for q in range(nq):
            UH = Xe.T @ H[e, q]
            assert np.abs(UH - np.eye(3)).max() < 1e-13
            assert np.abs(H[e, q].sum(axis=0)).max() < 1e-11
    if etype != T10:
        # affine / trilinear-box elements: the rule integrates 1 exactly
        assert abs(wJ.sum() - 0.8 * 0.6 * 0.3) < 1e-14
    else:
        m0 = synth.box_mesh(etype, (2, 2, 1), (0.8, 0.6, 0.3))
        _, wJ0, _ = oracle.precompute(etype, nq, m0.conn, m0.X)
        assert abs(wJ0.sum() - 0.8 * 0.6 * 0.3) < 1e-14


def test_precompute_flags_inverted_elements():
    m = synth.box_mesh(T4, (1, 1, 1), (1, 1, 1))
    conn = m.conn.copy()
    conn[0, [1, 2]] = conn[0, [2, 1]]
    _, _, bad = oracle.precompute(T4, 1, conn, m.X)
    assert bad == 1


# ------------------------------------------------------------------------
# Section 3: constitutive laws
# ------------------------------------------------------------------------

MU, LAM = 3.8e6, 5.8e6
MU01 = 0.3 * MU / 2          # Mooney-Rivlin: mu10 = mu/2 - mu01 = 0.7 mu/2


def _mat(model):
    """SVK (0), neo-Hookean (1) or Mooney-Rivlin (2) with the test constants."""
    return oracle.material(model, MU, LAM, mu01=MU01 if model == 2 else 0.0)


def mr_beam(cells=(4, 2, 2)):
    """small_beam with a Mooney-Rivlin body (mu01 = 0.3 mu/2), no damping."""
    wl = synth.small_beam(cells=cells, damping=0.0)
    wl.model = np.full(wl.n_bodies, 2, np.int32)
    wl.params = np.concatenate([wl.params, np.full((wl.n_bodies, 1), MU01)], axis=1)
    return wl


@pytest.mark.parametrize("model", [0, 1, 2])
def test_stress_is_energy_gradient(model):
    mat = _mat(model)
    rng = np.random.default_rng(3)
    for _ in range(5):
        F = _rand_F(rng)
        P, st = oracle.stress(mat, F)
        assert st == 0
        h = 1e-6
        G = np.zeros((3, 3))
        for a, b in product(range(3), repeat=2):
            d = np.zeros((3, 3))
            d[a, b] = h
            G[a, b] = (oracle.strain_energy(mat, F + d) - oracle.strain_energy(mat, F - d)) / (2 * h)
        assert np.abs(G - P).max() < 1e-7 * np.abs(P).max()


def test_svk_uniaxial_closed_form():
    mat = oracle.material(0, MU, LAM)
    for l1 in (0.7, 1.0, 1.05, 1.6):
        P, _ = oracle.stress(mat, np.diag([l1, 1.0, 1.0]))
        e = 0.5 * (l1 * l1 - 1.0)
        assert abs(P[0, 0] - l1 * (LAM + 2 * MU) * e) < 1e-8 * (abs(P[0, 0]) + 1)
        assert abs(P[1, 1] - LAM * e) < 1e-8 * (abs(P[1, 1]) + 1)
        assert abs(P[2, 2] - LAM * e) < 1e-8 * (abs(P[1, 1]) + 1)
        assert np.abs(P - np.diag(np.diag(P))).max() == 0.0


def test_neohooke_uniaxial_closed_form():
    mat = oracle.material(1, MU, LAM)
    mu10, k = MU / 2, LAM + 2 * MU / 3
    for l1 in (0.7, 1.0, 1.05, 1.6):
        P, _ = oracle.stress(mat, np.diag([l1, 1.0, 1.0]))
        J, I1 = l1, l1 * l1 + 2
        p11 = 2 * mu10 * J ** (-2 / 3) * (l1 - I1 / (3 * l1)) + k * (J - 1)
        p22 = 2 * mu10 * J ** (-2 / 3) * (1 - I1 / 3) + k * (J - 1) * J
        assert abs(P[0, 0] - p11) < 1e-8 * (abs(p11) + 1)
        assert abs(P[1, 1] - p22) < 1e-8 * (abs(p22) + 1)
        assert abs(P[2, 2] - p22) < 1e-8 * (abs(p22) + 1)


def test_mooney_rivlin_uniaxial_closed_form():
    # F = diag(l, 1, 1): J = l, I1 = l^2 + 2, I2 = 2 l^2 + 1; both isochoric
    # terms reduce to (2 l^2 - 2) / (3 l) along x and (1 - l^2) / 3 across
    mat = _mat(2)
    mu10, k = MU / 2 - MU01, LAM + 2 * MU / 3
    for l1 in (0.7, 1.0, 1.05, 1.6):
        P, _ = oracle.stress(mat, np.diag([l1, 1.0, 1.0]))
        a = 2 * mu10 * l1 ** (-2 / 3) + 2 * MU01 * l1 ** (-4 / 3)
        p11 = a * (2 * l1 * l1 - 2) / (3 * l1) + k * (l1 - 1)
        p22 = a * (1 - l1 * l1) / 3 + k * (l1 - 1) * l1
        assert abs(P[0, 0] - p11) < 1e-8 * (abs(p11) + 1)
        assert abs(P[1, 1] - p22) < 1e-8 * (abs(p22) + 1)
        assert abs(P[2, 2] - p22) < 1e-8 * (abs(p22) + 1)
        assert np.abs(P - np.diag(np.diag(P))).max() < 1e-9 * (abs(p11) + 1)


def test_mooney_rivlin_with_zero_mu01_is_neohooke():
    rng = np.random.default_rng(12)
    mr0 = oracle.material(2, MU, LAM, mu01=0.0)
    nh = _mat(1)
    for _ in range(4):
        F = _rand_F(rng)
        assert np.array_equal(oracle.stress(mr0, F)[0], oracle.stress(nh, F)[0])
        assert oracle.strain_energy(mr0, F) == oracle.strain_energy(nh, F)


@pytest.mark.parametrize("model", [1, 2])
def test_small_strain_limit_is_lame(model):
    # linearisation about F = I gives sigma = lam tr(eps) I + 2 mu eps
    # (Mooney-Rivlin: shear modulus 2 (mu10 + mu01) = mu)
    mat = _mat(model)
    rng = np.random.default_rng(4)
    G = 1e-7 * rng.uniform(-1, 1, (3, 3))
    P, _ = oracle.stress(mat, np.eye(3) + G)
    eps = 0.5 * (G + G.T)
    lin = LAM * np.trace(eps) * np.eye(3) + 2 * MU * eps
    assert np.abs(P - lin).max() < 1e-5 * np.abs(lin).max()


@pytest.mark.parametrize("model", [0, 1, 2])
def test_objectivity_and_rigid_rotation(model):
    mat = _mat(model)
    rng = np.random.default_rng(5)
    R = _rotation(rng)
    P0, _ = oracle.stress(mat, np.eye(3))
    assert np.abs(P0).max() < 1e-6
    PR, _ = oracle.stress(mat, R)
    assert np.abs(PR).max() < 1e-6 * MU
    F = _rand_F(rng)
    P, _ = oracle.stress(mat, F)
    PRF, _ = oracle.stress(mat, R @ F)
    assert np.abs(PRF - R @ P).max() < 1e-9 * np.abs(P).max()
    tau = P @ F.T
    assert np.abs(tau - tau.T).max() < 1e-9 * np.abs(tau).max()


def test_kelvin_voigt_rigid_spin_and_dissipation():
    mat = oracle.material(1, MU, LAM, mu_v=1e3, lam_v=2e2)
    rng = np.random.default_rng(6)
    F = _rand_F(rng)
    Pe, _ = oracle.stress(mat, F)
    W = rng.standard_normal((3, 3))
    W = W - W.T
    P, _ = oracle.stress(mat, F, W @ F)  # rigid spin: Edot = 0
    assert np.abs(P - Pe).max() < 1e-9 * np.abs(Pe).max()
    for _ in range(10):
        Fd = rng.standard_normal((3, 3))
        P, _ = oracle.stress(mat, F, Fd)
        Ed = 0.5 * (Fd.T @ F + F.T @ Fd)
        # stress power of the viscous branch P^v : Fdot = S^v : Edot >= 0 (Sec. 3.2.3)
        assert np.sum((P - Pe) * Fd) >= 0.0
        Sv = 2e3 * Ed + 2e2 * np.trace(Ed) * np.eye(3)
        assert abs(np.sum((P - Pe) * Fd) - np.sum(Sv * Ed)) < 1e-9 * abs(np.sum(Sv * Ed)) + 1e-12
    # closed form: F = I, Fdot = diag(d, 0, 0) -> P^v = 2 mu_v d e1 e1^T + lam_v d I
    d = 0.3
    P, _ = oracle.stress(mat, np.eye(3), np.diag([d, 0, 0]))
    assert abs(P[0, 0] - (2e3 * d + 2e2 * d)) < 1e-9 and abs(P[1, 1] - 2e2 * d) < 1e-9


def test_neohooke_inverted_point_is_flagged():
    mat = oracle.material(1, MU, LAM)
    P, st = oracle.stress(mat, np.diag([-1.0, 1.0, 1.0]))
    assert st == 1 and np.abs(P).max() == 0.0


# ------------------------------------------------------------------------
# Section 4.3: internal force
# ------------------------------------------------------------------------

def _affine_state(wl, A, b=(0.1, -0.2, 0.3)):
    return wl.X @ (A - np.eye(3)).T + np.asarray(b)


@pytest.mark.parametrize("etype,nq,model", [(T4, 1, 0), (T10, 4, 0), (T10, 5, 1), (H8, 8, 1), (Q27, 27, 1)])
def test_patch_test_uniform_F_zero_interior_force(etype, nq, model):
    cells = (3, 3, 3)
    m = synth.box_mesh(etype, cells, (1.0, 1.0, 1.0))
    wl = synth.workloads.Workload("patch", m.X, [synth.workloads.Block(etype, nq, m.conn, m.body)],
                                  np.array([model], np.int32),
                                  np.array([[MU, LAM, 0, 0, 1000.0]]), u=None)
    rng = np.random.default_rng(7)
    A = np.eye(3) + 0.05 * rng.uniform(-1, 1, (3, 3))
    wl.u = _affine_state(wl, A)
    # F = A at every quadrature point (displacement and literal forms)
    H, wJ, _ = oracle.precompute(etype, nq, m.conn, m.X)
    x = m.X + wl.u
    for e in range(0, m.n_elem, 7):
        for q in range(nq):
            F = x[m.conn[e]].T @ H[e, q]
            assert np.abs(F - A).max() < 1e-13
    f, _ = oracle.internal_force(wl)
    f0, _ = oracle.internal_force(wl, kin_form=0)
    tol = 1e-9 * np.abs(f).max()
    on_bdry = np.any((m.X < 1e-12) | (m.X > 1 - 1e-12), axis=1)
    assert np.abs(f[~on_bdry]).max() < tol
    assert np.abs(f - f0).max() < tol
    # boundary nodes carry the traction P n: the net force on the x=1 face
    # equals P e1 times the face area (1 m^2)
    P, _ = oracle.stress(oracle.material(model, MU, LAM), A)
    face = m.X[:, 0] > 1 - 1e-12
    inner_face = face & ~np.any((m.X[:, 1:] < 1e-12) | (m.X[:, 1:] > 1 - 1e-12), axis=1)
    assert inner_face.any()
    tot = f[m.X[:, 0] > 1 - 1e-12].sum(axis=0)
    # forces on the x=1 face sum to P e1 minus edge contributions shared with
    # other faces; take the full slab of nodes with x = 1
    assert np.abs(tot - P[:, 0]).max() < 1e-8 * np.abs(P).max() + 1e-9 * np.abs(P).max()


@pytest.mark.parametrize("builder", ["beam", "block"])
def test_force_balance_and_energy_gradient(builder):
    if builder == "beam":
        wl = synth.small_beam(cells=(4, 2, 2), damping=0.0)
    else:
        wl = synth.block_t10_svk(cells=2)
    f, bad = oracle.internal_force(wl)
    assert bad == 0
    x = wl.X + wl.u
    # linear and angular momentum balance of the internal forces
    assert np.abs(f.sum(axis=0)).max() < 1e-9 * np.abs(f).max()
    assert np.abs(np.cross(x, f).sum(axis=0)).max() < 1e-9 * np.abs(f).max() * np.abs(x).max()
    # f = d/dx sum_e sum_q wJ psi(F) (App. C.1.1 definition of the internal force)
    blk = wl.blocks[0]
    H, wJ, _ = oracle.precompute(blk.etype, blk.nq, blk.conn, wl.X)
    mats = oracle.block_materials(wl, 0)

    def energy(xx):
        tot = 0.0
        for e in range(blk.n_elem):
            for q in range(blk.nq):
                F = xx[blk.conn[e]].T @ H[e, q]
                tot += wJ[e, q] * oracle.strain_energy(mats[e:e + 1], F)
        return tot

    rng = np.random.default_rng(8)
    for _ in range(3):
        d = rng.standard_normal(x.shape)
        h = 1e-6
        fd = (energy(x + h * d) - energy(x - h * d)) / (2 * h)
        assert abs(fd - np.sum(f * d)) < 1e-6 * np.abs(f).max() * np.abs(d).sum() / 100 + 1e-6 * abs(fd)


def test_internal_force_t4_closed_form():
    # one T4 under uniform F: f_i = V P h_i with h_i the constant gradients
    m = synth.box_mesh(T4, (1, 1, 1), (1, 1, 1))
    conn = m.conn[:1]
    Xe = m.X[conn[0]]
    Dm = np.stack([Xe[1] - Xe[0], Xe[2] - Xe[0], Xe[3] - Xe[0]], axis=1)
    V = np.linalg.det(Dm) / 6
    Hh = np.vstack([-np.ones(3) @ np.linalg.inv(Dm), np.linalg.inv(Dm)])  # rows h_i^T
    F = np.eye(3) + np.array([[0.02, 0.01, 0], [0, -0.03, 0.01], [0.005, 0, 0.04]])
    wl = synth.workloads.Workload("t4", m.X, [synth.workloads.Block(T4, 1, conn, m.body[:1])],
                                  np.array([0], np.int32), np.array([[MU, LAM, 0, 0, 1e3]]),
                                  u=m.X @ (F - np.eye(3)).T)
    f, _ = oracle.internal_force(wl)
    P, _ = oracle.stress(oracle.material(0, MU, LAM), F)
    for i in range(4):
        assert np.abs(f[conn[0, i]] - V * P @ Hh[i]).max() < 1e-8 * np.abs(P).max() * V


# ------------------------------------------------------------------------
# App. C: tangent blocks
# ------------------------------------------------------------------------

@pytest.mark.parametrize("builder", ["svk", "nh_kv", "mr"])
def test_tangent_matches_fd_and_symmetry(builder):
    """Closed-form blocks (Eqs. svk_tangent, mr_tangent incl. dt3-dt5, derived
    KV blocks) against central differences of the force, symmetry, rigid
    translation and the transpose."""
    if builder == "svk":
        wl = synth.block_t10_svk(cells=2)
    elif builder == "mr":
        wl = mr_beam()
    else:
        wl = synth.small_beam(cells=(4, 2, 2))
    rng = np.random.default_rng(9)
    v = rng.standard_normal(wl.X.shape)
    w = rng.standard_normal(wl.X.shape)
    Kv = oracle.operator_apply(wl, v)
    h = 1e-7
    fp, _ = oracle.internal_force(wl, u=wl.u + h * v)
    fm, _ = oracle.internal_force(wl, u=wl.u - h * v)
    assert np.abs((fp - fm) / (2 * h) - Kv).max() < 1e-7 * np.abs(Kv).max()
    # elastic K is symmetric; K (rigid translation) = 0
    Ke_v = oracle.operator_apply(wl, v, sym_only=True)
    Ke_w = oracle.operator_apply(wl, w, sym_only=True)
    assert abs(np.sum(w * Ke_v) - np.sum(v * Ke_w)) < 1e-10 * abs(np.sum(w * Ke_v))
    t = np.tile(np.array([0.3, -1.0, 2.0]), (wl.n_nodes, 1))
    assert np.abs(oracle.operator_apply(wl, t)).max() < 1e-7 * np.abs(Kv).max()
    # transpose application is the adjoint
    KTw = oracle.operator_apply(wl, w, transpose=True)
    assert abs(np.sum(w * Kv) - np.sum(KTw * v)) < 1e-10 * abs(np.sum(w * Kv))
    if builder == "nh_kv":
        Cv = oracle.operator_apply(wl, v, a_K=0.0, a_C=1.0)
        fp, _ = oracle.internal_force(wl, udot=wl.udot + h * v)
        fm, _ = oracle.internal_force(wl, udot=wl.udot - h * v)
        assert np.abs((fp - fm) / (2 * h) - Cv).max() < 1e-7 * np.abs(Cv).max()
        Cw = oracle.operator_apply(wl, w, a_K=0.0, a_C=1.0)
        assert abs(np.sum(w * Cv) - np.sum(v * Cw)) < 1e-10 * abs(np.sum(w * Cv))
        assert np.sum(v * Cv) > 0


def _damped_block(etype, cells, model=1, seed=31):
    """A small damped body of one element type with a random state: bending
    displacement + noise, random velocities (Kelvin-Voigt mu_v, lam_v > 0 so
    that every viscous block is non-zero)."""
    m = synth.box_mesh(etype, cells, tuple(0.05 * c for c in cells))
    rng = np.random.default_rng(seed)
    u = 2e-3 * rng.standard_normal(m.X.shape)
    udot = 0.05 * rng.standard_normal(m.X.shape)
    return Workload(name=f"damped_{etype}", X=m.X, blocks=[Block(etype, DEFAULT_NQ[etype],
                                                                            m.conn, m.body)],
                          model=np.array([model], np.int32),
                          params=np.array([[MU, LAM, 2e3, 7e2, 1000.0]]), u=u, udot=udot,
                          v=rng.standard_normal(m.X.shape))


@pytest.mark.parametrize("etype,cells", [(T10, (2, 1, 1)), (H8, (2, 2, 1))])
def test_jacobi_diag_is_the_diagonal_of_the_symmetric_operator(etype, cells):
    """Sec. 2.2 Newton matrix, Jacobi preconditioner: jacobi_diag[k] equals
    e_k . (a_M M + a_K K^e + a_C C) e_k, the operator applied to every unit
    vector (a wrong DOF in the diagonal's scatter, or a term dropped from it
    but not from the operator, fails here)."""
    wl = _damped_block(etype, cells)
    n3 = 3 * wl.n_nodes
    for aM, aK, aC in ((0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (1e3, 0.7, 1.9)):
        d = oracle.jacobi_diag(wl, a_M=aM, a_K=aK, a_C=aC).ravel()
        ref = np.zeros(n3)
        for k in range(n3):
            e = np.zeros(n3)
            e[k] = 1.0
            y = oracle.operator_apply(wl, e.reshape(-1, 3), a_M=aM, a_K=aK, a_C=aC, sym_only=True)
            ref[k] = y.ravel()[k]
        assert np.abs(d - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.all(ref > 0)          # the diagonal of an SPD operator


@pytest.mark.parametrize("etype,cells", [(T10, (2, 1, 1)), (H8, (2, 2, 1)), (T4, (2, 2, 2))])
def test_symmetric_operator_is_the_elastic_stiffness(etype, cells):
    """The CG operator's stiffness K^e (Sec. 7 reading: the viscous stiffness
    K^v left out) against central differences of the force with the velocity
    switched off, which is the elastic force alone (P^v = 0 when Fdot = 0):
    K^e v = d/de f(u + e v, udot = 0). It must not depend on the velocity,
    and with mu_v = lam_v = 0 it equals the full K_t."""
    wl = _damped_block(etype, cells)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(wl.X.shape)
    Ke_v = oracle.operator_apply(wl, v, sym_only=True)
    h = 1e-7
    z = np.zeros_like(wl.X)
    fp, _ = oracle.internal_force(wl, u=wl.u + h * v, udot=z)
    fm, _ = oracle.internal_force(wl, u=wl.u - h * v, udot=z)
    assert np.abs((fp - fm) / (2 * h) - Ke_v).max() < 1e-7 * np.abs(Ke_v).max()
    # independent of the velocity at which it is evaluated
    Ke_v0 = oracle.operator_apply(wl, v, sym_only=True, udot=z)
    assert np.abs(Ke_v0 - Ke_v).max() <= 1e-12 * np.abs(Ke_v).max()
    # the full K_t differs by the viscous stiffness, which is not zero here
    Kt_v = oracle.operator_apply(wl, v)
    assert np.abs(Kt_v - Ke_v).max() > 1e-6 * np.abs(Ke_v).max()
    # undamped: the symmetric operator is the full one
    wl.params[:, 2:4] = 0.0
    assert np.abs(oracle.operator_apply(wl, v, sym_only=True) - oracle.operator_apply(wl, v)).max() <= \
        1e-13 * np.abs(Ke_v).max()
    # the damping product C is the same in both (C v = d/de f(u, udot + e v))
    wl.params[:, 2:4] = (2e3, 7e2)
    Cv = oracle.operator_apply(wl, v, a_K=0.0, a_C=1.0, sym_only=True)
    fp, _ = oracle.internal_force(wl, udot=wl.udot + h * v)
    fm, _ = oracle.internal_force(wl, udot=wl.udot - h * v)
    assert np.abs((fp - fm) / (2 * h) - Cv).max() < 1e-7 * np.abs(Cv).max()


def test_vjp_parameter_gradient_by_fd():
    wl = synth.diff_block(cells=2)
    rng = np.random.default_rng(10)
    r = rng.standard_normal(wl.X.shape)
    _, _, gth = oracle.vjp(wl, r)
    th = wl.elem_mu_lambda.copy()
    for k in range(2):
        d = np.zeros_like(th)
        d[:, k] = 1e-6 * th[:, k] * rng.standard_normal(th.shape[0])
        wl.elem_mu_lambda = th + d
        lp = np.sum(oracle.internal_force(wl)[0] * r)
        wl.elem_mu_lambda = th - d
        lm = np.sum(oracle.internal_force(wl)[0] * r)
        wl.elem_mu_lambda = th
        fd = (lp - lm) / 2
        assert abs(fd - np.sum(gth[:, k] * d[:, k])) < 1e-6 * abs(fd)


# ------------------------------------------------------------------------
# Sec. 4.1 / 4.2: mass and force field
# ------------------------------------------------------------------------

def _bary_integral(exps, V):
    # int L1^a L2^b L3^c L4^d dV = a! b! c! d! 3! V / (a+b+c+d+3)!
    num = math.prod(math.factorial(k) for k in exps) * 6
    return num * V / math.factorial(sum(exps) + 3)


def _t10_poly():
    # each shape function as {exponent tuple of (L1..L4): coefficient}
    polys = []
    for k in range(4):
        e2 = [0] * 4
        e2[k] = 2
        e1 = [0] * 4
        e1[k] = 1
        polys.append({tuple(e2): 2.0, tuple(e1): -1.0})
    for a, b in [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]:
        e = [0] * 4
        e[a] += 1
        e[b] += 1
        polys.append({tuple(e): 4.0})
    return polys


def test_t10_consistent_mass_by_barycentric_formula():
    m = synth.box_mesh(T10, (1, 1, 1), (0.7, 0.5, 0.9))
    rho = 1200.0
    polys = _t10_poly()
    for e in range(6):
        Xc = m.X[m.conn[e, :4]]
        V = np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]], 1)) / 6
        Mref = np.zeros((10, 10))
        for i in range(10):
            for j in range(10):
                for ei, ci in polys[i].items():
                    for ej, cj in polys[j].items():
                        Mref[i, j] += ci * cj * _bary_integral([x + y for x, y in zip(ei, ej)], V)
        _, _, Me = oracle.element_matrices(T10, 5, m.conn[e], m.X, np.zeros_like(m.X), None,
                                           oracle.material(1, MU, LAM, rho=rho))
        assert np.abs(Me[0::3, 0::3] - rho * Mref).max() < 1e-12 * rho * V
        assert abs(Me[0::3, 0::3].sum() - rho * V) < 1e-12 * rho * V


def test_q27_box_mass_is_kronecker_of_1d_quadratic_masses():
    # on a box the triquadratic shape functions factor, so m_ij = rho int s_i s_j dV
    # is the Kronecker product of the 1D quadratic Lagrange mass matrices
    # (L/30)[[4, 2, -1], [2, 16, 2], [-1, 2, 4]] (node n = i + 3 j + 9 k)
    a, b, c = 0.7, 0.5, 0.9
    m = synth.box_mesh(Q27, (1, 1, 1), (a, b, c))
    rho = 1200.0
    m1 = np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0
    Mref = rho * np.kron(np.kron(c * m1, b * m1), a * m1)
    _, _, Me = oracle.element_matrices(Q27, 27, m.conn[0], m.X, np.zeros_like(m.X), None,
                                       oracle.material(1, MU, LAM, rho=rho))
    V = a * b * c
    assert np.abs(Me[0::3, 0::3] - Mref).max() < 1e-13 * rho * V
    assert np.abs(Me[1::3, 1::3] - Mref).max() < 1e-13 * rho * V
    assert np.abs(Me[0::3, 1::3]).max() == 0.0
    # gravity weights int s_i dV: Kronecker of the 1D (1/6, 2/3, 1/6) L
    w1 = np.array([1.0, 4.0, 1.0]) / 6.0
    wl = synth.workloads.Workload("q27", m.X, [synth.workloads.Block(Q27, 27, m.conn, np.zeros(1, np.int32))],
                                  np.array([1], np.int32), np.array([[MU, LAM, 0.0, 0.0, rho]]),
                                  u=np.zeros_like(m.X))
    f = oracle.gravity_load(wl, np.array([0.0, 0.0, -9.81]))
    wref = np.kron(np.kron(c * w1, b * w1), a * w1)
    assert np.abs(f[m.conn[0], 2] / (-9.81 * rho) - wref).max() < 1e-14


def test_gravity_weights_t10_and_mass_totals():
    wl = synth.small_beam(cells=(2, 1, 1))
    g = np.array([0.0, 0.0, -9.81])
    f = oracle.gravity_load(wl, g)
    blk = wl.blocks[0]
    V = np.prod(wl.X.max(0) - wl.X.min(0))
    assert abs(f[:, 2].sum() + 9.81 * 1000.0 * V) < 1e-9 * 9.81 * 1000 * V
    # one isolated T10: corners -V/20, edges V/5 (of rho g)
    one = synth.workloads.Workload("one", wl.X, [synth.workloads.Block(T10, 5, blk.conn[:1],
                                                                       blk.body[:1])],
                                   wl.model, wl.params, u=wl.u)
    f1 = oracle.gravity_load(one, g)
    Xc = wl.X[blk.conn[0, :4]]
    Ve = np.linalg.det(np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]], 1)) / 6
    w = f1[blk.conn[0], 2] / (-9.81 * 1000.0 * Ve)
    assert np.allclose(w[:4], -1 / 20, atol=1e-13) and np.allclose(w[4:], 1 / 5, atol=1e-13)
    mr = oracle.mass_row_sums(wl)
    assert abs(mr.sum() - 1000.0 * V) < 1e-9 * 1000 * V


# ------------------------------------------------------------------------
# Section 7: backward-Euler Newton step
# ------------------------------------------------------------------------

def test_newton_free_fall_is_exact():
    # no clamps, start at rest in the reference: v = h g solves g(v) = 0
    # exactly (rigid translation: f_int = 0, and f_ff = M g since sum s_j = 1)
    wl = synth.small_beam(cells=(3, 1, 1), damping=0.0)
    h = 1e-3
    grav = np.array([0.0, 0.0, -9.81])
    v, rep = oracle.newton_step(wl, np.zeros_like(wl.X), np.zeros_like(wl.X), h, grav,
                                newton_rtol=1e-12)
    assert rep["status"] == 0
    assert np.abs(v - h * grav).max() < 1e-10


def test_newton_residual_is_gradient_and_converges():
    wl = synth.small_beam(cells=(4, 1, 1), damping=0.0)
    fixed = (np.abs(wl.X[:, 0]) < 1e-12).astype(np.uint8)
    h = 1e-3
    grav = np.array([0.0, 0.0, -9.81])
    u_n = np.zeros_like(wl.X)
    v_n = np.zeros_like(wl.X)
    v, rep = oracle.newton_step(wl, u_n, v_n, h, grav, fixed=fixed, newton_rtol=1e-10)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    assert np.abs(v[fixed == 1]).max() == 0.0
    # independent residual: g = M/h (v - v_n) + f_int(u_n + h v) - f_ff
    f_ff = oracle.gravity_load(wl, grav)

    def g_of(vv):
        g = oracle.operator_apply(wl, vv - v_n, a_M=1 / h, a_K=0.0, u=u_n + h * vv, udot=None)
        g += oracle.internal_force(wl, u=u_n + h * vv, udot=None)[0] - f_ff
        g[fixed == 1] = 0
        return g

    g0 = np.linalg.norm(g_of(v_n))
    assert np.linalg.norm(g_of(v)) <= 1e-9 * g0
    # g = grad_v Phi (Eq. gradient_equals_residual), Phi from the energy density
    blk = wl.blocks[0]
    H, wJ, _ = oracle.precompute(blk.etype, blk.nq, blk.conn, wl.X)
    mats = oracle.block_materials(wl, 0)

    def Phi(vv):
        dv = vv - v_n
        Mdv = oracle.operator_apply(wl, dv, a_M=1.0, a_K=0.0, udot=None)
        x = wl.X + u_n + h * vv
        Pi = sum(wJ[e, q] * oracle.strain_energy(mats[e:e + 1], x[blk.conn[e]].T @ H[e, q])
                 for e in range(blk.n_elem) for q in range(blk.nq))
        return 0.5 / h * np.sum(dv * Mdv) + Pi / h - np.sum(f_ff * vv)

    rng = np.random.default_rng(11)
    vt = 0.01 * rng.standard_normal(v.shape)
    vt[fixed == 1] = 0
    d = rng.standard_normal(v.shape)
    d[fixed == 1] = 0
    e = 1e-5
    fd = (Phi(vt + e * d) - Phi(vt - e * d)) / (2 * e)
    assert abs(fd - np.sum(g_of(vt) * d)) < 1e-6 * abs(fd)


# ------------------------------------------------------------------------
# colouring
# ------------------------------------------------------------------------

def test_splitmix64_published_vector():
    # first output of the splitmix64 generator seeded with 1234567
    assert oracle.splitmix64(1234567) == 6457827717110365317


def test_greedy_colouring_valid_and_equal_to_brute_force():
    m = synth.box_mesh(T10, (2, 2, 2), (1, 1, 1))
    seed = 0x1234
    col, nc = oracle.color_greedy(m.conn, m.n_nodes, seed)
    # brute force: pure-Python greedy in descending priority
    pr = [oracle.splitmix64(e ^ seed) for e in range(m.n_elem)]
    order = sorted(range(m.n_elem), key=lambda e: -pr[e])
    ref = [-1] * m.n_elem
    sets = [set(r) for r in m.conn.tolist()]
    for e in order:
        used = {ref[o] for o in range(m.n_elem) if ref[o] >= 0 and sets[o] & sets[e]}
        c = 0
        while c in used:
            c += 1
        ref[e] = c
    assert col.tolist() == ref and nc == max(ref) + 1
    for c in range(nc):
        nodes = m.conn[col == c].ravel()
        assert len(nodes) == len(set(nodes.tolist()))


def test_kinematic_forms_agree_and_rigid_translation_is_exact():
    # Eq. expression-F with U H = I and sum_i h_i = 0: the three forms are equal
    wl = synth.block_t10_svk()
    f2, _ = oracle.internal_force(wl, kin_form=2)
    for form in (0, 1):
        f, _ = oracle.internal_force(wl, kin_form=form)
        assert np.abs(f - f2).max() < 1e-12 * np.abs(f2).max()
    # a rigid translation by a large offset: the element-relative form sees
    # exactly zero strain, hence exactly zero force
    wl.u = np.tile(np.array([123.456, -7.25, 0.3]), (wl.n_nodes, 1))
    f2, _ = oracle.internal_force(wl, kin_form=2)
    assert np.abs(f2).max() == 0.0
    f1, _ = oracle.internal_force(wl, kin_form=1)
    assert np.abs(f1).max() > 0.0          # the plain displacement form rounds


# ------------------------------------------------------------------------
# Sec. 4: pointwise loads and surface tractions
# ------------------------------------------------------------------------

def _outward_normals(etype, X, conn, elem, face):
    """Unit outward normals and areas of flat boundary faces (geometry of the
    corner nodes; the element's other corners lie on the inner side)."""
    n_out, area = [], []
    for e, f in zip(elem, face):
        cs = synth.face_corners(etype, f)
        P = X[conn[e, cs]]
        if etype in (H8, Q27):   # corners in tensor order: (0, 1, 3, 2) walks the quad
            P = P[[0, 1, 3, 2]]
            nv = 0.5 * np.cross(P[2] - P[0], P[3] - P[1])
        else:
            nv = 0.5 * np.cross(P[1] - P[0], P[2] - P[0])
        inner = X[conn[e, [c for c in range(conn.shape[1]) if c not in cs]]].mean(axis=0)
        if np.dot(nv, inner - P[0]) > 0:
            nv = -nv
        a = np.linalg.norm(nv)
        n_out.append(nv / a)
        area.append(a)
    return np.array(n_out), np.array(area)


@pytest.mark.parametrize("etype,nq", [(T4, 1), (T10, 5), (H8, 8), (Q27, 27)])
def test_traction_of_uniform_stress_balances_internal_force(etype, nq):
    """A homogeneous deformation F = A is in equilibrium under the boundary
    traction t0 = P(A) n0 (Sec. 4, the nominal traction induced by a stress):
    the assembled traction load equals f_int at every node (interior nodes
    carry neither). Also: each face's load sums to t0 times its area."""
    m = synth.box_mesh(etype, (2, 2, 3), (1.0, 1.2, 1.5), origin=(0.3, -0.2, 0.1))
    from synth.workloads import Block, Workload
    rng = np.random.default_rng(31)
    A = np.eye(3) + 0.1 * rng.uniform(-1, 1, (3, 3))
    u = m.X @ (A - np.eye(3)).T
    wl = Workload("uniform", m.X, [Block(etype, nq, m.conn, np.zeros(m.n_elem, np.int32))],
                  np.array([1], np.int32), np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=u, udot=None)
    f_int, bad = oracle.internal_force(wl)
    assert bad == 0
    P, _ = oracle.stress(_mat(1), A)
    elem, face = synth.boundary_faces(etype, m.conn)
    nrm, area = _outward_normals(etype, m.X, m.conn, elem, face)
    t0 = nrm @ P.T                                       # t0 = P n0 per face
    f_tr = oracle.surface_traction(wl, 0, elem, face, t0)
    assert np.abs(f_tr - f_int).max() < 1e-9 * np.abs(f_int).max()
    for k in (0, len(elem) // 2, len(elem) - 1):
        one = oracle.surface_traction(wl, 0, elem[k:k + 1], face[k:k + 1], t0[k:k + 1])
        assert np.abs(one.sum(axis=0) - t0[k] * area[k]).max() < 1e-12 * np.abs(t0[k]).max() * area[k]


@pytest.mark.parametrize("etype,nq", [(T4, 1), (T10, 5), (H8, 8), (Q27, 27)])
def test_point_loads_partition_and_kronecker(etype, nq):
    m = synth.box_mesh(etype, (2, 1, 1), (1.0, 1.0, 1.0))
    from synth.workloads import Block, Workload
    wl = Workload("pl", m.X, [Block(etype, nq, m.conn, np.zeros(m.n_elem, np.int32))],
                  np.array([1], np.int32), np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=np.zeros_like(m.X))
    rng = np.random.default_rng(32)
    k = 7
    elem = rng.integers(0, m.n_elem, k).astype(np.int32)
    if etype in (H8, Q27):
        xi = rng.uniform(-1, 1, (k, 3))
    else:
        L = rng.dirichlet(np.ones(4), k)
        xi = L[:, 1:]
    force = rng.standard_normal((k, 3))
    f = oracle.point_loads(wl, 0, elem, xi, force)
    assert np.abs(f.sum(axis=0) - force.sum(axis=0)).max() < 1e-12
    # a load at a node of the parent element goes to that node only
    node_xi = {T4: [0, 0, 0], T10: [0.5, 0, 0], H8: [1, -1, -1], Q27: [0, 1, 0]}[etype]
    node_id = {T4: 0, T10: 4, H8: 1, Q27: 16}[etype]
    f1 = oracle.point_loads(wl, 0, np.array([0], np.int32), np.array([node_xi], float), np.array([[1.0, 2.0, 3.0]]))
    g = m.conn[0, node_id]
    assert np.abs(f1[g] - [1.0, 2.0, 3.0]).max() < 1e-14
    assert np.abs(np.delete(f1, g, axis=0)).max() < 1e-14


# ------------------------------------------------------------------------
# Sec. 3 constraint primitives and the augmented-Lagrangian step (Sec. 7)
# ------------------------------------------------------------------------

def _two_beams():
    """Two T10 beams (bodies 0 and 1) side by side, with seeded displacements."""
    from synth.workloads import Block, Workload
    m1 = synth.box_mesh(T10, (4, 1, 1), (0.2, 0.05, 0.05))
    m2 = synth.box_mesh(T10, (4, 1, 1), (0.2, 0.05, 0.05), origin=(0.0, 0.1, 0.0))
    m = synth.concat_meshes([m1, m2])
    rng = np.random.default_rng(41)
    u = 0.002 * rng.standard_normal(m.X.shape)
    return Workload("two", m.X, [Block(T10, 5, m.conn, m.body)], np.array([1, 1], np.int32),
                    np.array([[MU, LAM, 0.0, 0.0, 1000.0]] * 2), u=u, udot=None)


def _random_constraints(wl, rng):
    ne = wl.blocks[0].n_elem
    half = ne // 2

    def pt(body):
        e = int(rng.integers(0, half)) + (half if body else 0)
        return e, rng.dirichlet(np.ones(4))[1:]
    items = []
    for t in (oracle.CD, oracle.DIST, oracle.DP1, oracle.DP2):
        np_ = 2 if t in (oracle.CD, oracle.DIST) else 4
        bodies = [0, 1] if np_ == 2 else ([0, 0, 1, 1] if t == oracle.DP1 else [0, 0, 0, 1])
        pts = [pt(b) for b in bodies]
        items.append({"type": t, "elem": [p[0] for p in pts], "xi": [p[1] for p in pts],
                      "d": (0.0, 1.0, 0.0), "f": 0.03})
    # a ground point (clamp-like coordinate difference)
    e, xi = pt(0)
    items.append({"type": oracle.CD, "elem": [e, -1], "xi": [xi, [0.05, 0.02, 0.01]], "d": (1.0, 0.0, 0.0)})
    return oracle.constraints(items)


def test_constraint_jacobian_blocks_match_central_differences():
    """C_q v (the element blocks of Eqs. cd_blocks, dist_blocks, dp1_block_P,
    dp2_blocks) equals the central difference of c along v, and C_q^T is its
    adjoint."""
    wl = _two_beams()
    rng = np.random.default_rng(42)
    cons = _random_constraints(wl, rng)
    v = rng.standard_normal(wl.X.shape)
    w = rng.standard_normal(len(cons))
    Jv = oracle.constraint_j(wl, cons, v)
    h = 1e-6
    fd = (oracle.constraint_eval(wl, cons, wl.u + h * v) - oracle.constraint_eval(wl, cons, wl.u - h * v)) / (2 * h)
    assert np.abs(Jv - fd).max() < 1e-8 * np.abs(fd).max()
    JTw = oracle.constraint_jt(wl, cons, w)
    assert abs(np.sum(JTw * v) - np.sum(w * Jv)) < 1e-12 * abs(np.sum(w * Jv))


def test_constraint_values_closed_form():
    """c of each primitive at nodes, where point evaluation returns the node."""
    from synth.workloads import Block, Workload
    m = synth.box_mesh(T4, (1, 1, 1), (1.0, 1.0, 1.0))
    u = np.zeros_like(m.X)
    wl = Workload("c", m.X, [Block(T4, 1, m.conn, np.zeros(m.n_elem, np.int32))], np.array([1], np.int32),
                  np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=u)
    c0 = m.conn[0]
    X = m.X
    node_xi = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]   # T4 corners in parent coordinates
    cons = oracle.constraints([
        {"type": oracle.CD, "elem": [0, 0], "xi": [node_xi[0], node_xi[1]], "d": (1, 0, 0), "f": 0.25},
        {"type": oracle.DIST, "elem": [0, 0], "xi": [node_xi[0], node_xi[2]], "f": 0.5},
        {"type": oracle.DP1, "elem": [0, 0, 0, 0], "xi": node_xi, "f": 0.1},
    ])
    c = oracle.constraint_eval(wl, cons)
    a01 = X[c0[1]] - X[c0[0]]
    a02 = X[c0[2]] - X[c0[0]]
    b23 = X[c0[3]] - X[c0[2]]
    assert abs(c[0] - (a01[0] - 0.25)) < 1e-14
    assert abs(c[1] - 0.5 * (a02 @ a02 - 0.25)) < 1e-14
    assert abs(c[2] - (a01 @ b23 - 0.1)) < 1e-14


def test_alm_clamp_by_coordinate_differences_reproduces_the_projected_clamp():
    """Clamping the x = 0 face by three CD constraints per node to ground
    points (Sec. 3 CD, Sec. 7 ALM with multiplier updates) converges to the
    step with the clamped DOFs projected out."""
    from synth.workloads import Block, Workload
    m = synth.box_mesh(T10, (4, 1, 1), (0.2, 0.05, 0.05))
    wl = Workload("b", m.X, [Block(T10, 5, m.conn, np.zeros(m.n_elem, np.int32))], np.array([1], np.int32),
                  np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=np.zeros_like(m.X))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    g = np.array([0.0, 0.0, -9.81])
    z = np.zeros_like(m.X)
    v_proj, rep = oracle.newton_step(wl, z, z, 1e-3, g, fixed=fixed, newton_rtol=1e-10, cg_rtol=1e-10)
    assert rep["status"] == 0
    # one element holding each clamped node, and that node's parent coordinates
    nxi = _load_golden("t10_parent_nodes.txt")[:, 5:8]      # App. A.1 node table: parent (xi, eta, zeta)
    items = []
    for node in np.nonzero(fixed)[0]:
        e, i = [(e, i) for e in range(m.n_elem) for i in range(10) if m.conn[e, i] == node][0]
        for d in range(3):
            dv = [0.0, 0.0, 0.0]
            dv[d] = 1.0
            items.append({"type": oracle.CD, "elem": [e, -1], "xi": [nxi[i], m.X[node]], "d": dv, "f": 0.0})
    cons = oracle.constraints(items)
    v, lam, r = oracle.newton_step_alm(wl, z, z, 1e-3, g, cons, rho=1e10, newton_rtol=1e-10, cg_rtol=1e-10,
                                       alm_tol=1e-12, max_outer=20)
    assert r["status"] == 0 and r["c_norm"] <= 1e-12
    assert np.abs(v - v_proj).max() <= 1e-7 * np.abs(v_proj).max()
    # the multipliers carry the support reactions: C_q^T lam h balances the load at the clamp
    assert np.abs(lam).max() > 0


def test_row_weights_closed_form():
    """Eq. row_weights at nodes (point evaluation returns the node): a DP1
    row gets 1 / sqrt(|a0|^2 + |b0|^2), every other row 1."""
    from synth.workloads import Block, Workload
    m = synth.box_mesh(T4, (1, 1, 1), (0.3, 0.7, 1.1))
    wl = Workload("w", m.X, [Block(T4, 1, m.conn, np.zeros(m.n_elem, np.int32))], np.array([1], np.int32),
                  np.array([[MU, LAM, 0.0, 0.0, 1000.0]]), u=np.zeros_like(m.X))
    c0, X = m.conn[0], m.X
    node_xi = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    cons = oracle.constraints([
        {"type": oracle.CD, "elem": [0, 0], "xi": [node_xi[0], node_xi[1]], "d": (1, 0, 0), "f": 0.0},
        {"type": oracle.DIST, "elem": [0, 0], "xi": [node_xi[0], node_xi[2]], "f": 0.5},
        {"type": oracle.DP1, "elem": [0, 0, 0, 0], "xi": node_xi, "f": 0.0},
        {"type": oracle.DP2, "elem": [0, 0, 0, 0], "xi": node_xi, "f": 0.0},
    ])
    w = oracle.constraint_row_weights(wl, cons)
    a0, b0 = X[c0[1]] - X[c0[0]], X[c0[3]] - X[c0[2]]
    assert w[0] == 1.0 and w[1] == 1.0 and w[3] == 1.0
    assert abs(w[2] - 1.0 / np.sqrt(a0 @ a0 + b0 @ b0)) < 1e-15


def _revolute_problem(delta):
    """Two T10 beams along x: body 0 clamped at x = 0, body 1 beside it (y
    offset) and free; a revolute-type joint at their far ends: three CD rows
    between coincident-in-x/z points, and two DP1 rows keeping body 1's
    x-fibre perpendicular to body 0's y- and z-fibres (fibres of length
    delta)."""
    from synth.workloads import Block, Workload
    m1 = synth.box_mesh(T10, (4, 1, 1), (0.2, 0.05, 0.05))
    m2 = synth.box_mesh(T10, (4, 1, 1), (0.2, 0.05, 0.05), origin=(0.2, 0.0, 0.0))
    m = synth.concat_meshes([m1, m2])
    wl = Workload("rev", m.X, [Block(T10, 5, m.conn, m.body)], np.array([1, 1], np.int32),
                  np.array([[MU, LAM, 0.0, 0.0, 1000.0]] * 2), u=np.zeros_like(m.X))
    fixed = (np.abs(m.X[:, 0]) < 1e-12).astype(np.uint8)
    conn = m.conn

    def locate(body, p):
        """(element, parent xi) of physical point p inside a body's elements."""
        for e in np.nonzero(m.body == body)[0]:
            Xc = m.X[conn[e, :4]]
            J = np.stack([Xc[1] - Xc[0], Xc[2] - Xc[0], Xc[3] - Xc[0]], axis=1)
            xi = np.linalg.solve(J, p - Xc[0])
            if xi.min() >= -1e-12 and xi.sum() <= 1 + 1e-12:
                return int(e), xi
        raise AssertionError("point outside the body")
    j = np.array([0.2, 0.025, 0.025])      # the joint: the shared end face centre
    p0, p1 = locate(0, j - [0.01, 0, 0]), locate(1, j + [0.01, 0, 0])
    items = []
    for d in np.eye(3):
        items.append({"type": oracle.CD, "elem": [p0[0], p1[0]], "xi": [p0[1], p1[1]], "d": tuple(d),
                      "f": float(d @ np.array([0.02, 0.0, 0.0]))})
    c0 = j - [0.01, 0, 0]
    for fib in (np.array([0, 1.0, 0]), np.array([0, 0, 1.0])):
        P, Q = locate(0, c0 - 0.5 * delta * fib), locate(0, c0 + 0.5 * delta * fib)
        R, T = locate(1, j + [0.01 - 0.5 * delta, 0, 0]), locate(1, j + [0.01 + 0.5 * delta, 0, 0])
        items.append({"type": oracle.DP1, "elem": [P[0], Q[0], R[0], T[0]], "xi": [P[1], Q[1], R[1], T[1]],
                      "f": 0.0})
    return wl, fixed, oracle.constraints(items)


def test_row_normalised_alm_converges_to_a_penalty_independent_solution():
    """A revolute-type joint with 2 cm DP1 fibres (Eqs. row_weights,
    rev_normalized). With the row weights (about 1 / (sqrt(2) delta) on the
    DP1 rows) the augmented-Lagrangian step converges for two penalties rho
    and reaches the same velocities and multipliers: the constrained solution
    does not depend on rho. With raw rows, the same settings stall above the
    tolerance: the scale mismatch the weights remove."""
    delta = 0.02
    wl, fixed, cons = _revolute_problem(delta)
    w = oracle.constraint_row_weights(wl, cons)
    assert np.allclose(w[:3], 1.0) and np.allclose(w[3:], 1.0 / (np.sqrt(2.0) * delta), rtol=1e-12)
    g = np.array([0.0, 0.0, -9.81])
    z = np.zeros_like(wl.X)
    kw = dict(fixed=fixed, newton_rtol=1e-10, cg_rtol=1e-10, max_newton=30, max_cg=5000, max_outer=40, alm_tol=1e-10)
    runs = [oracle.newton_step_alm(wl, z, z, 1e-3, g, cons, rho=rho, row_norm=True, **kw) for rho in (1e8, 1e9)]
    for v, lam, r in runs:
        assert r["status"] == 0 and r["c_norm"] <= 1e-10
        assert np.abs(oracle.constraint_eval(wl, cons, 1e-3 * v)).max() <= 1e-10
    # each run stops at ||c^|| <= alm_tol: a position residual of alm_tol over
    # one step of h bounds the velocity difference by alm_tol / h; the
    # multipliers agree to the inner Newton tolerance
    (v1, lam1, _), (v2, lam2, _) = runs
    assert np.abs(v1 - v2).max() <= kw["alm_tol"] / 1e-3
    assert np.abs(lam1 - lam2).max() <= 1e-4 * np.abs(lam1).max()
    _, _, r_raw = oracle.newton_step_alm(wl, z, z, 1e-3, g, cons, rho=1e8, row_norm=False,
                                         **dict(kw, alm_tol=1e-10 / w.max()))
    assert r_raw["status"] != 0 and r_raw["outer_iters"] == 40
