"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (relative, max-norm, normalised by the oracle's max |value|):
FP64 mode 1e-12, FP32 mode 2e-5; connectivity-derived integers (colours)
bit-exact.
"""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}  # keyed by precision: FP64 = 0, FP32 = 1
PATHS = [0, 1]             # element path: auto (affine blocks on the affine path), slab


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def dev(a, dt):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def relerr(got, ref):
    got = got.double().cpu().numpy() if hasattr(got, "cpu") else got
    den = np.abs(ref).max()
    return np.abs(got - ref).max() / (den if den > 0 else 1.0)


def run_all(wl, prec, scatter=0, aM=0.0, aK=1.0, aC=0.0, diag=True, path=0):
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec, scatter=scatter, element_path=path)
    dt = mesh.torch_dtype
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
    out = {"f": mesh.internal_force(u, ud), "y": mesh.tangent_matvec(u, ud, v, aM, aK, aC)}
    out["gu"], out["gud"], out["gth"] = mesh.vjp(u, ud, v)
    if diag:
        out["d"] = mesh.jacobi_diag(u, ud, aM, aK, aC)
    mesh.sync()
    torch.cuda.synchronize()
    return mesh, out


def check_all(wl, out, prec, aM=0.0, aK=1.0, aC=0.0, diag=True):
    tol = TOL[prec]
    f_ref, _ = oracle.internal_force(wl)
    assert relerr(out["f"], f_ref) <= tol
    y_ref = oracle.operator_apply(wl, wl.v, a_M=aM, a_K=aK, a_C=aC)
    assert relerr(out["y"], y_ref) <= tol
    gu, gud, gth = oracle.vjp(wl, wl.v)
    assert relerr(out["gu"], gu) <= tol
    if wl.udot is not None and np.abs(gud).max() > 0:
        assert relerr(out["gud"], gud) <= tol
    assert relerr(out["gth"], gth) <= tol
    if diag:
        d_ref = oracle.jacobi_diag(wl, a_M=aM, a_K=aK, a_C=aC)
        assert relerr(out["d"], d_ref) <= tol


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_block_t10_svk(prec, path):
    wl = synth.block_t10_svk()
    mesh, out = run_all(wl, prec, path=path)
    assert mesh.info["n_affine_blocks"] == (1 if path == 0 else 0)
    check_all(wl, out, prec)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_small_beam_nh_kv_full_operator(prec, path):
    wl = synth.small_beam(cells=(10, 2, 2))
    h = 1e-3
    _, out = run_all(wl, prec, aM=1.0 / h, aK=h, aC=1.0, path=path)
    check_all(wl, out, prec, aM=1.0 / h, aK=h, aC=1.0)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_batch_t4_t10_h8(prec, path):
    wl = synth.batch_bodies(n_bodies=9, seed=7, ne_range=(40, 400))
    assert len(wl.blocks) >= 2
    _, out = run_all(wl, prec, path=path)
    check_all(wl, out, prec)


def _mixed_law_batch():
    """A batch whose blocks mix SVK, neo-Hookean and Mooney-Rivlin bodies,
    some of them damped (with a velocity field)."""
    wl = synth.batch_bodies(n_bodies=12, seed=11, ne_range=(40, 300))
    model = np.asarray(wl.model).copy()
    model[::4] = 2                                        # Mooney-Rivlin, mu01 = 0.3 mu / 2
    params = np.concatenate([wl.params, 0.15 * wl.params[:, :1]], axis=1)
    params[1::3, 2] = 1e3                                 # Kelvin-Voigt mu_v on every third body
    wl.model, wl.params = model, params
    wl.udot = 0.01 * np.random.default_rng(31).standard_normal(wl.X.shape)
    return wl


@pytest.mark.parametrize("scatter", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_law_blocks_run_one_pass_per_law(prec, scatter):
    """Each block is laid out as one tile range per elastic law (per colour
    and law in colour mode) and each range is launched with its law's kernel:
    the pass count is the number of such groups, every output matches the
    oracle, and colour mode repeats bit for bit."""
    wl = _mixed_law_batch()
    mesh, out = run_all(wl, prec, scatter=scatter, aK=1.0, aC=1.0)
    check_all(wl, out, prec, aK=1.0, aC=1.0)
    law = np.asarray(wl.model)
    if scatter == 0:
        groups = sum(len(np.unique(law[b.body])) for b in wl.blocks if len(b.body))
    else:
        col, k0, groups = mesh.colors(), 0, 0
        for b in wl.blocks:
            n = len(b.body)
            groups += len({(int(c), int(m)) for c, m in zip(col[k0:k0 + n], law[b.body])})
            k0 += n
    assert groups > len(wl.blocks)            # the mix really splits blocks
    assert mesh.info["n_passes"] == groups
    if scatter == 1:
        dt = mesh.torch_dtype
        u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
        y1 = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0).cpu().numpy()
        y2 = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0).cpu().numpy()
        assert np.array_equal(y1, y2)
        assert np.array_equal(y1, out["y"].cpu().numpy())


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_sorted_scatter_matches_oracle_and_repeats_bit_for_bit(prec, path):
    """Sorted scatter (tile partials summed per node in a fixed order) on a
    mixed T4 / T10 / H8 batch with mixed laws and damping: every output
    matches the oracle, and a second evaluation gives the same bits."""
    wl = _mixed_law_batch()
    tl = T()
    mesh, out = run_all(wl, prec, scatter=tl.SCATTER_SORTED, aK=1.0, aC=1.0, path=path)
    check_all(wl, out, prec, aK=1.0, aC=1.0)
    assert mesh.info["n_colors"] == 0
    dt = mesh.torch_dtype
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
    again = {"f": mesh.internal_force(u, ud), "y": mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)}
    again["gu"], again["gud"], again["gth"] = mesh.vjp(u, ud, v)
    again["d"] = mesh.jacobi_diag(u, ud, 0.0, 1.0, 1.0)
    for k, a in again.items():
        assert torch.equal(a, out[k]), k


def test_sorted_scatter_leaves_nodes_outside_elements_at_zero():
    """Nodes no element uses get exactly 0 from the node sums (they replace the
    zero fill of the atomic modes), also with an empty block in the mesh."""
    base = synth.small_beam(cells=(4, 2, 2))
    blk = base.blocks[0]
    keep = blk.conn[: blk.n_elem // 2]
    wl = Workload("half", base.X, [Block(blk.etype, blk.nq, keep, blk.body[: len(keep)]),
                                   Block(synth.T4, 1, np.zeros((0, 4), np.int32), np.zeros(0, np.int32))],
                  base.model, base.params, u=base.u, udot=base.udot, v=base.v)
    tl = T()
    for prec in (0, 1):
        _, out = run_all(wl, prec, scatter=tl.SCATTER_SORTED)
        check_all(wl, out, prec)
        unused = np.setdiff1d(np.arange(wl.n_nodes), np.unique(keep))
        assert unused.size > 0
        for k in ("f", "y", "gu", "d"):
            assert not out[k].cpu().numpy()[unused].any(), k


@pytest.mark.parametrize("scatter", [0, 1, 2])
def test_blocks_sharing_nodes(scatter):
    """One body split into two blocks that share the nodes of their interface:
    every scatter mode (atomic, colour, sorted) sums both blocks there."""
    base = synth.small_beam(cells=(6, 2, 2))
    blk = base.blocks[0]
    h = blk.n_elem // 2
    wl = Workload("split", base.X, [Block(blk.etype, blk.nq, blk.conn[:h], blk.body[:h]),
                                    Block(blk.etype, blk.nq, blk.conn[h:], blk.body[h:])],
                  base.model, base.params, u=base.u, udot=base.udot, v=base.v)
    assert np.intersect1d(blk.conn[:h], blk.conn[h:]).size > 0
    for prec in (0, 1):
        _, out = run_all(wl, prec, scatter=scatter, aK=1.0, aC=1.0)
        check_all(wl, out, prec, aK=1.0, aC=1.0)


def test_single_law_block_is_one_pass():
    wl = synth.small_beam(cells=(6, 2, 2))
    tl = T()
    assert tl.Mesh.from_workload(wl, precision=tl.FP32).info["n_passes"] == 1


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_per_element_parameters_and_damping(prec, path):
    wl = synth.diff_block(cells=3)
    _, out = run_all(wl, prec, aK=1.0, aC=2.0, path=path)
    check_all(wl, out, prec, aK=1.0, aC=2.0)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n_elem", [1, 31, 33, 65])
def test_ragged_tiles(n_elem, path):
    base = synth.small_beam(cells=(6, 2, 2))
    blk = base.blocks[0]
    wl = Workload("ragged", base.X, [Block(blk.etype, blk.nq, blk.conn[:n_elem], blk.body[:n_elem])],
                  base.model, base.params, u=base.u, udot=base.udot, v=base.v)
    for prec in (0, 1):
        _, out = run_all(wl, prec, path=path)
        check_all(wl, out, prec)


def _curved(wl, amp, seed):
    """Move every mid-edge T10 node (and, for H8, every node) off its straight
    position: the elements become genuinely isoparametric (non-affine)."""
    X = wl.X.copy()
    rng = np.random.default_rng(seed)
    for blk in wl.blocks:
        if blk.etype == synth.T10:
            mids = np.unique(blk.conn[:, 4:])
            X[mids] += rng.uniform(-amp, amp, (mids.size, 3))
        elif blk.etype == synth.H8:
            nodes = np.unique(blk.conn)
            X[nodes] += rng.uniform(-amp, amp, (nodes.size, 3))
    return Workload(wl.name + "_curved", X, wl.blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v,
                    elem_mu_lambda=wl.elem_mu_lambda)


@pytest.mark.parametrize("prec", [0, 1])
def test_curved_elements_use_the_slab_path(prec):
    """Non-affine T10 (curved edges) and H8 (distorted bricks): the automatic
    path streams per-point h_i, and results match the isoparametric oracle;
    forcing the affine path on them is refused."""
    base = synth.batch_bodies(n_bodies=6, seed=9, ne_range=(60, 300))
    wl = _curved(base, 0.004, 5)           # cells of 0.05 m: up to 8 % of the edge
    mesh, out = run_all(wl, prec, path=0)
    n_t4 = sum(b.etype == synth.T4 for b in wl.blocks)
    assert mesh.info["n_affine_blocks"] == n_t4    # only the T4 block stays affine
    check_all(wl, out, prec)
    if n_t4 < len(wl.blocks):
        tl = T()
        with pytest.raises(tl.TLFEError) as ei:
            tl.Mesh.from_workload(wl, precision=prec, element_path=tl.PATH_AFFINE)
        assert ei.value.code == 7


def test_empty_block_in_multiblock_mesh():
    base = synth.small_beam(cells=(4, 1, 1))
    blk = base.blocks[0]
    wl = Workload("empty", base.X, [Block(blk.etype, blk.nq, blk.conn, blk.body),
                                    Block(synth.T4, 1, np.zeros((0, 4), np.int32), np.zeros(0, np.int32))],
                  base.model, base.params, u=base.u, udot=base.udot, v=base.v)
    _, out = run_all(wl, 0)
    check_all(wl, out, 0)


def test_colour_scatter_matches_oracle_greedy_and_is_deterministic():
    wl = synth.small_beam(cells=(12, 3, 3))
    seed = 0xC0FFEE
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=tl.SCATTER_COLOR, color_seed=seed)
    col = mesh.colors()
    ref, nc = oracle.color_greedy(wl.blocks[0].conn, wl.n_nodes, seed)
    assert np.array_equal(col, ref)
    assert mesh.info["n_colors"] == nc
    dt = mesh.torch_dtype
    u, ud = dev(wl.u, torch.float64), dev(wl.udot, dt)
    f1 = mesh.internal_force(u, ud).cpu().numpy()
    f2 = mesh.internal_force(u, ud).cpu().numpy()
    assert np.array_equal(f1.view(np.uint32), f2.view(np.uint32))
    f_ref, _ = oracle.internal_force(wl)
    assert relerr(f1, f_ref) <= 2e-5


def _typed_meshes():
    """One workload per element type (T4, T10, H8 and Q27 on the warp-per-element
    path, Q27 curved on the tile path) and one multi-block batch."""
    out = {}
    for name, et in (("T4", synth.T4), ("H8", synth.H8)):
        m = synth.box_mesh(et, (7, 3, 2), (0.35, 0.15, 0.1))
        rng = np.random.default_rng(41 + et)
        out[name] = Workload(name, m.X, [Block(et, synth.workloads.DEFAULT_NQ[et], m.conn, m.body)],
                             np.array([1], np.int32), np.array([[3.8e6, 5.8e6, 0.0, 0.0, 1000.0]]),
                             u=1e-3 * rng.standard_normal(m.X.shape), udot=None, v=rng.standard_normal(m.X.shape))
    out["T10"] = synth.small_beam(cells=(6, 3, 2))
    out["Q27"] = synth.q27_beam(cells=(5, 3, 2))
    out["Q27_curved"] = synth.q27_beam(cells=(5, 3, 2), curve=0.05)
    out["batch"] = synth.batch_bodies(n_bodies=7, seed=13, ne_range=(30, 500))
    return out


@pytest.mark.parametrize("name", ["T4", "T10", "H8", "Q27", "Q27_curved", "batch"])
def test_colours_bit_exact_every_element_type(name):
    """Colouring (two elements conflict iff they share a node; colour = the
    smallest not used by a higher-priority conflicting element of the block,
    priority splitmix64(e xor seed)) equals the oracle's sequential greedy run
    on every block, for every element type and a multi-block batch."""
    wl = _typed_meshes()[name]
    seed = 0x5EED + len(name)
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=tl.SCATTER_COLOR, color_seed=seed)
    col = mesh.colors()
    k0, nc_max = 0, 0
    for blk in wl.blocks:
        ref, nc = oracle.color_greedy(blk.conn, wl.n_nodes, seed)
        assert np.array_equal(col[k0:k0 + blk.n_elem], ref)
        nc_max = max(nc_max, nc)
        k0 += blk.n_elem
    assert mesh.info["n_colors"] == nc_max
    mesh.close()


@pytest.mark.parametrize("scatter", [0, 1, 2])
@pytest.mark.parametrize("name", ["T4", "T10", "H8", "Q27", "Q27_curved", "batch"])
def test_gather_and_scatter_indices_bit_exact(name, scatter):
    """The node every (element, local node) is gathered from and scattered to,
    read back from the kernels' device tables (metadata records, node-sorted
    positions, the sorted-scatter transpose, the warp-per-element
    connectivity), equals conn[e][i] bit for bit: the scatter target of
    component d is 3 conn[e][i] + d."""
    wl = _typed_meshes()[name]
    tl = T()
    for prec in (0, 1):
        mesh = tl.Mesh.from_workload(wl, precision=prec, scatter=scatter)
        g, s = mesh.scatter_targets()
        for blk, gb, sb in zip(wl.blocks, g, s):
            assert np.array_equal(gb, blk.conn)
            assert np.array_equal(sb, blk.conn)
        mesh.close()


def test_inverted_points_are_counted():
    wl = synth.small_beam(cells=(4, 1, 1), damping=0.0)
    # squash the beam through itself along x: J < 0 everywhere
    u = wl.X * np.array([-2.0, 0.0, 0.0])
    wl.u = u
    _, bad = oracle.internal_force(wl)
    assert bad > 0
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP64)
    mesh.internal_force(dev(u, torch.float64), None)
    with pytest.raises(tl.TLFEError) as ei:
        mesh.sync()
    assert ei.value.code == 4
    assert mesh.sync() == 0  # cleared


def test_inverted_reference_rejected():
    tl = T()
    m = synth.box_mesh(synth.T4, (1, 1, 1), (1, 1, 1))
    conn = m.conn.copy()
    conn[0, [1, 2]] = conn[0, [2, 1]]
    with pytest.raises(tl.TLFEError) as ei:
        tl.Mesh(m.X, [(synth.T4, 1, conn, None)], [(0, 1e6, 1e6, 0, 0, 1e3)])
    assert ei.value.code == 4


def test_host_buffer_call_matches_device_call():
    wl = synth.small_beam(cells=(8, 2, 2))
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    u = np.ascontiguousarray(wl.u, np.float64)
    ud = np.ascontiguousarray(wl.udot, np.float32)
    f_h = np.zeros_like(ud)
    mesh.internal_force_host(u, ud, f_h)
    f_d = mesh.internal_force(dev(u, torch.float64), dev(ud, torch.float32)).cpu().numpy()
    assert np.array_equal(f_h, f_d) or relerr(f_h, f_d) < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_host_step_matches_device_calls(prec):
    """tlfe_step_host on pinned host buffers: three calls in a row on two
    different states (the staging sets alternate, transfers overlap), then
    one wait; every output equals the device calls on the same state up to
    the atomic scatter's summation order."""
    wl = synth.small_beam(cells=(8, 2, 2))
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    dt = mesh.torch_dtype
    rng = np.random.default_rng(4)
    states = [(wl.u, wl.udot, wl.v), (wl.u + 1e-4 * rng.standard_normal(wl.X.shape),
                                       wl.udot + 1e-3 * rng.standard_normal(wl.X.shape),
                                       rng.standard_normal(wl.X.shape))]
    pin = lambda a, d: torch.from_numpy(np.ascontiguousarray(a)).to(d).pin_memory()  # noqa: E731
    outs = []
    for k in range(3):
        u, ud, v = states[k % 2]
        hu, hud, hv = pin(u, torch.float64), pin(ud, dt), pin(v, dt)
        o = {n: torch.empty((wl.n_nodes, 3), dtype=dt).pin_memory() for n in ("f", "y", "gu", "gud")}
        o["gth"] = torch.empty((wl.n_elem, 2), dtype=torch.float64).pin_memory()
        mesh.step_host(hu, hud, hv, hv, f=o["f"], y=o["y"], g_u=o["gu"], g_udot=o["gud"], g_mu_lambda=o["gth"],
                       a_M=0.0, a_K=1.0, a_C=1.0)
        outs.append((o, (hu, hud, hv)))
    mesh.step_host_wait()
    mesh.sync()
    for k, (o, _) in enumerate(outs):
        u, ud, v = states[k % 2]
        du, dud, dv = dev(u, torch.float64), dev(ud, dt), dev(v, dt)
        f = mesh.internal_force(du, dud)
        y = mesh.tangent_matvec(du, dud, dv, 0.0, 1.0, 1.0)
        gu, gud, gth = mesh.vjp(du, dud, dv)
        torch.cuda.synchronize()
        for name, ref in (("f", f), ("y", y), ("gu", gu), ("gud", gud), ("gth", gth)):
            r = ref.double().cpu().numpy()
            assert relerr(o[name].double().numpy(), r) <= (1e-12 if prec == 0 else 1e-6), (k, name)
    mesh.close()


def _subset(wl, mask):
    blk = wl.blocks[0]
    return Workload("sub", wl.X, [Block(blk.etype, blk.nq, blk.conn[mask], blk.body[mask])], wl.model, wl.params,
                    u=wl.u, udot=wl.udot, v=wl.v,
                    elem_mu_lambda=None if wl.elem_mu_lambda is None else wl.elem_mu_lambda[mask])


def test_beam_full_size_bench_configuration():
    """The 480k-T10 beam the benchmark times, in its launch configuration:
    force against the oracle everywhere; K v and the adjoint at sampled nodes
    (a node's value depends only on the elements holding it)."""
    wl = synth.cantilever_beam()
    tl = T()
    f_ref, bad = oracle.internal_force(wl)
    assert bad == 0
    for prec, tol, path in ((1, 2e-5, 0), (1, 2e-5, 1), (0, 1e-12, 0)):
        mesh = tl.Mesh.from_workload(wl, precision=prec, element_path=path)
        dt = mesh.torch_dtype
        u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
        f = mesh.internal_force(u, ud)
        y = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)
        gu, gud, gth = mesh.vjp(u, ud, v)
        mesh.sync()
        assert relerr(f, f_ref) <= tol
        rng = np.random.default_rng(8)
        ks = rng.choice(wl.n_nodes, 300, replace=False)
        sub = _subset(wl, np.isin(wl.blocks[0].conn, ks).any(axis=1))
        y_ref = oracle.operator_apply(sub, wl.v, a_K=1.0, a_C=1.0)
        g_ref, gd_ref, _ = oracle.vjp(sub, wl.v)
        assert relerr(y.double().cpu().numpy()[ks], y_ref[ks]) <= tol
        assert relerr(gu.double().cpu().numpy()[ks], g_ref[ks]) <= tol
        assert relerr(gud.double().cpu().numpy()[ks], gd_ref[ks]) <= tol
        mesh.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_schedules_keep_parity(prec):
    """tlfe_autotune picks CTA size and tile assignment by measurement; the
    results stay within the parity bars afterwards (with and without udot,
    i.e. both material modes of a damped block)."""
    wl = synth.small_beam(cells=(12, 3, 3))
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    dt = mesh.torch_dtype
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
    mesh.autotune(u, ud, v)
    mesh.autotune(u, None, v)
    out = {"f": mesh.internal_force(u, ud), "y": mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)}
    out["gu"], out["gud"], out["gth"] = mesh.vjp(u, ud, v)
    f0 = mesh.internal_force(u, None)
    mesh.sync()
    check_all(wl, out, prec, aK=1.0, aC=1.0, diag=False)
    f_ref0, _ = oracle.internal_force(wl, udot=None)
    assert relerr(f0, f_ref0) <= TOL[prec]


def _mooney_rivlin(wl, mu01_frac=0.3):
    """The workload with every body switched to Mooney-Rivlin, mu01 = frac * mu/2."""
    wl.model = np.full(wl.n_bodies, 2, np.int32)
    wl.params = np.concatenate([wl.params, (mu01_frac * 0.5 * wl.params[:, :1])], axis=1)
    return wl


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("prec", [0, 1])
def test_mooney_rivlin_with_damping(prec, path):
    """Full Mooney-Rivlin (App. C, mu01 != 0) with Kelvin-Voigt damping:
    force, K_t v + C v, adjoint and diagonal against the oracle."""
    wl = _mooney_rivlin(synth.small_beam(cells=(10, 2, 2)))
    mesh, out = run_all(wl, prec, aK=1.0, aC=1.0, path=path)
    check_all(wl, out, prec, aK=1.0, aC=1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_mooney_rivlin_per_element_parameters(prec):
    wl = _mooney_rivlin(synth.diff_block(cells=3), 0.2)
    _, out = run_all(wl, prec)
    check_all(wl, out, prec)


def test_bounded_wait_times_out_and_the_context_stays_usable():
    """A device-side wait that nothing completes (tlfe_selftest_wait_timeout:
    the element kernels' bounded mbarrier wait on 16 bytes no copy delivers)
    gives TLFE_E_TIMEOUT at the next sync, without a fault; the status is then
    clear and the same mesh evaluates correctly."""
    tl = T()
    wl = synth.small_beam(cells=(4, 2, 2))
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    with pytest.raises(tl.TLFEError):
        mesh.selftest_wait_timeout(0)
    mesh.selftest_wait_timeout(4096)
    with pytest.raises(tl.TLFEError) as ei:
        mesh.sync()
    assert ei.value.code == 6
    dt = mesh.torch_dtype
    u, ud = dev(wl.u, torch.float64), dev(wl.udot, dt)
    f = mesh.internal_force(u, ud)
    assert mesh.sync() == 0
    f_ref, _ = oracle.internal_force(wl)
    assert relerr(f, f_ref) <= TOL[1]
    mesh.close()
