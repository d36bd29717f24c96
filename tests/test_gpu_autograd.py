"""Differentiation through the hand-written adjoint: torch.autograd around
tlfe_internal_force / tlfe_vjp against central finite differences of the FP64
oracle loss, and the adjoint at the full differentiation-workload size against
the oracle on sampled outputs."""

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fd_directions(wl, theta0, rng):
    """(name, direction, FD step) for u, udot and the per-element parameters."""
    return [("u", rng.standard_normal(wl.X.shape), 1e-7),
            ("udot", rng.standard_normal(wl.X.shape), 1e-4),
            ("theta", rng.standard_normal(theta0.shape) * theta0, 1e-6)]


def _oracle_f(wl, base, name, step):
    """FP64 oracle force with one of (u, udot, theta) moved by `step`."""
    u0, ud0, th0 = base
    wl.u, wl.udot, wl.elem_mu_lambda = u0.copy(), ud0.copy(), th0.copy()
    if name == "u":
        wl.u = u0 + step
    elif name == "udot":
        wl.udot = ud0 + step
    else:
        wl.elem_mu_lambda = th0 + step
    f, _ = oracle.internal_force(wl)
    wl.u, wl.udot, wl.elem_mu_lambda = u0, ud0, th0
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_matches_central_differences(prec):
    """The hand-written adjoint (tlfe_vjp) for a fixed cotangent r against
    central differences of the FP64 oracle's r . f along random directions of
    u, udot and the per-element (mu, lambda): relative error <= 1e-4."""
    from paper_2602_17002_gb300 import tlfe
    wl = synth.diff_block(cells=3)
    theta0 = wl.elem_mu_lambda.copy()
    base = (wl.u.copy(), wl.udot.copy(), theta0)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(wl.X.shape)
    mesh = tlfe.Mesh.from_workload(wl, precision=prec)
    dt = mesh.torch_dtype
    gu, gud, gth = mesh.vjp(torch.tensor(wl.u, dtype=torch.float64, device="cuda"),
                            torch.tensor(wl.udot, dtype=dt, device="cuda"), torch.tensor(r, dtype=dt, device="cuda"))
    g = {"u": gu.double().cpu().numpy(), "udot": gud.double().cpu().numpy(), "theta": gth.cpu().numpy()}
    for name, d, e in _fd_directions(wl, theta0, rng):
        fd = (np.sum(r * _oracle_f(wl, base, name, e * d)) - np.sum(r * _oracle_f(wl, base, name, -e * d))) / (2 * e)
        an = float(np.sum(g[name] * d))
        assert abs(an - fd) <= 1e-4 * abs(fd), (name, an, fd)


def test_loss_gradient_through_autograd():
    """Loss 1/2 |f - f_target|^2 through torch.autograd (forward
    tlfe_internal_force, backward tlfe_vjp). FP64 mesh: against central
    differences of the oracle loss (1e-4). FP32 mesh: against the oracle's
    gradient for the same cotangent f - f_target (1e-4); the cotangent then
    carries the FP32 forward's rounding, which a random-direction difference
    of this loss amplifies through the stiffness, so there the finite
    differences measure the forward, not the adjoint."""
    from paper_2602_17002_gb300 import tlfe
    from paper_2602_17002_gb300.autograd import internal_force
    wl = synth.diff_block(cells=3)
    theta0 = wl.elem_mu_lambda.copy()
    base = (wl.u.copy(), wl.udot.copy(), theta0)
    wl.elem_mu_lambda = wl.extra["theta_target"]
    f_target, _ = oracle.internal_force(wl)
    wl.elem_mu_lambda = theta0
    for prec in (0, 1):
        mesh = tlfe.Mesh.from_workload(wl, precision=prec)
        u = torch.tensor(wl.u, dtype=torch.float64, device="cuda", requires_grad=True)
        ud = torch.tensor(wl.udot, dtype=mesh.torch_dtype, device="cuda", requires_grad=True)
        th = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
        ft = torch.tensor(f_target, device="cuda")
        f = internal_force(mesh, u, ud, th)
        loss = 0.5 * ((f.double() - ft) ** 2).sum()     # FP64 reduction
        loss.backward()
        g = {"u": u.grad.double().cpu().numpy(), "udot": ud.grad.double().cpu().numpy(),
             "theta": th.grad.cpu().numpy()}
        rng = np.random.default_rng(3)
        if prec == 0:
            for name, d, e in _fd_directions(wl, theta0, rng):
                lp = 0.5 * np.sum((_oracle_f(wl, base, name, e * d) - f_target) ** 2)
                lm = 0.5 * np.sum((_oracle_f(wl, base, name, -e * d) - f_target) ** 2)
                fd = (lp - lm) / (2 * e)
                an = float(np.sum(g[name] * d))
                assert abs(an - fd) <= 1e-4 * abs(fd), (name, an, fd)
        else:
            cot = f.detach().double().cpu().numpy() - f_target
            ref = dict(zip(("u", "udot", "theta"), oracle.vjp(wl, cot)))
            for name, d, _ in _fd_directions(wl, theta0, rng):
                an, rf = float(np.sum(g[name] * d)), float(np.sum(ref[name] * d))
                assert abs(an - rf) <= 1e-4 * abs(rf), (name, an, rf)


def test_adjoint_at_full_size_on_sampled_outputs():
    from paper_2602_17002_gb300 import tlfe
    wl = synth.diff_block()            # 998,250 T10, 1,367,631 nodes
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32)
    rng = np.random.default_rng(21)
    r = rng.standard_normal(wl.X.shape)
    dt = torch.float32
    gu, gud, gth = mesh.vjp(torch.tensor(wl.u, dtype=torch.float64, device="cuda"),
                            torch.tensor(wl.udot, dtype=dt, device="cuda"),
                            torch.tensor(r, dtype=dt, device="cuda"))
    gu, gud, gth = gu.double().cpu().numpy(), gud.double().cpu().numpy(), gth.cpu().numpy()
    blk = wl.blocks[0]
    # sampled elements: their parameter gradients are element-local
    es = np.sort(rng.choice(blk.n_elem, 3000, replace=False))
    sub = Workload("s", wl.X, [Block(blk.etype, blk.nq, blk.conn[es], blk.body[es])], wl.model, wl.params,
                   u=wl.u, udot=wl.udot, elem_mu_lambda=wl.elem_mu_lambda[es])
    _, _, th_ref = oracle.vjp(sub, r)
    assert np.abs(gth[es] - th_ref).max() <= 2e-5 * np.abs(th_ref).max()
    # sampled nodes: g at node k depends only on the elements holding k
    ks = rng.choice(wl.n_nodes, 200, replace=False)
    mask = np.isin(blk.conn, ks).any(axis=1)
    sub = Workload("s", wl.X, [Block(blk.etype, blk.nq, blk.conn[mask], blk.body[mask])], wl.model, wl.params,
                   u=wl.u, udot=wl.udot, elem_mu_lambda=wl.elem_mu_lambda[mask])
    gu_ref, gud_ref, _ = oracle.vjp(sub, r)
    assert np.abs(gu[ks] - gu_ref[ks]).max() <= 2e-5 * np.abs(gu_ref[ks]).max()
    assert np.abs(gud[ks] - gud_ref[ks]).max() <= 2e-5 * np.abs(gud_ref[ks]).max()
