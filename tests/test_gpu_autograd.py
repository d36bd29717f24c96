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


def test_loss_gradient_matches_finite_differences():
    from paper_2602_17002_gb300 import tlfe
    from paper_2602_17002_gb300.autograd import internal_force
    wl = synth.diff_block(cells=3)
    theta0 = wl.elem_mu_lambda.copy()
    wl.elem_mu_lambda = wl.extra["theta_target"]
    f_target, _ = oracle.internal_force(wl)
    wl.elem_mu_lambda = theta0
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32)
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda", requires_grad=True)
    ud = torch.tensor(wl.udot, dtype=torch.float32, device="cuda", requires_grad=True)
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    ft = torch.tensor(f_target, device="cuda")
    f = internal_force(mesh, u, ud, th)
    loss = 0.5 * ((f.double() - ft) ** 2).sum()     # FP64 reduction of the FP32 force
    loss.backward()
    gu, gud, gth = u.grad.double().cpu().numpy(), ud.grad.double().cpu().numpy(), th.grad.cpu().numpy()

    def L(du=0.0, dud=0.0, dth=0.0):
        wl.u, wl.udot, wl.elem_mu_lambda = wl_u + du, wl_ud + dud, theta0 + dth
        f64, _ = oracle.internal_force(wl)
        wl.u, wl.udot, wl.elem_mu_lambda = wl_u, wl_ud, theta0
        return 0.5 * np.sum((f64 - f_target) ** 2)

    wl_u, wl_ud = wl.u.copy(), wl.udot.copy()
    rng = np.random.default_rng(3)
    for name, g, scale in (("u", gu, 1e-7), ("udot", gud, 1e-4), ("theta", gth, 1e-6)):
        for _ in range(2):
            shape = theta0.shape if name == "theta" else wl.X.shape
            d = rng.standard_normal(shape) * (theta0 if name == "theta" else 1.0)
            e = scale
            kw = {"u": "du", "udot": "dud", "theta": "dth"}[name]
            fd = (L(**{kw: e * d}) - L(**{kw: -e * d})) / (2 * e)
            an = float(np.sum(g * d))
            assert abs(an - fd) <= 1e-4 * abs(fd), (name, an, fd)


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
