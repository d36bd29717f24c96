"""Measured error of every result against the FP64 oracle, per benchmark
configuration at its full size (sampled nodes where the oracle cannot do
the whole mesh: a node's value depends only on the elements holding it, an
element's parameter gradient only on that element).

Each entry is max |gpu - oracle| / max |oracle| over the compared values
(per body for the batch). The test asserts the parity bars (FP32 2e-5,
FP64 1e-12) and prints the table; with TLFE_ERROR_TABLE set it also writes
the table there as JSON."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import Block, Workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAR = {0: 1e-12, 1: 2e-5}
TABLE = {}


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def dev(a, dt):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def rel(got, ref):
    got = got.double().cpu().numpy() if hasattr(got, "cpu") else np.asarray(got, np.float64)
    den = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (den if den > 0 else 1.0))


def _subset(wl, ks):
    blocks, masks = [], []
    for blk in wl.blocks:
        sel = np.isin(blk.conn, ks).any(axis=1)
        masks.append(sel)
        blocks.append(Block(blk.etype, blk.nq, blk.conn[sel], blk.body[sel]))
    eml = None
    if wl.elem_mu_lambda is not None:
        eml = wl.elem_mu_lambda[np.concatenate(masks)]
    return Workload("sub", wl.X, blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v,
                    elem_mu_lambda=eml), np.concatenate(masks)


def _record(config, prec, **errs):
    key = f"{config} ({'FP64' if prec == 0 else 'FP32'})"
    TABLE[key] = {k: v for k, v in errs.items() if v is not None}
    for name, e in TABLE[key].items():
        assert e <= BAR[prec], (key, name, e)


def _operators(wl, prec, ks=None):
    """Every element result of the library on wl, compared with the oracle on
    all nodes (ks None) or on the nodes ks (and the elements holding them)."""
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec)
    dt = mesh.torch_dtype
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, dt), dev(wl.v, dt)
    f = mesh.internal_force(u, ud).double().cpu().numpy()
    kv = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 0.0).double().cpu().numpy()
    cv = mesh.tangent_matvec(u, ud, v, 0.0, 0.0, 1.0).double().cpu().numpy() if wl.udot is not None else None
    gu, gud, gth = (None if x is None else x.double().cpu().numpy() for x in mesh.vjp(u, ud, v))
    dg = mesh.jacobi_diag(u, ud, 0.0, 1.0, 1.0).double().cpu().numpy()
    one_pass = bool(mesh.info["force_matvec_fused"])
    if one_pass:   # the same results from the one-pass force + operator product (tlfe_force_matvec)
        f1, y1 = (x.double().cpu().numpy() for x in mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0))
    mesh.sync()
    mesh.close()
    sub, emask = (wl, np.ones(wl.n_elem, bool)) if ks is None else _subset(wl, ks)
    sel = slice(None) if ks is None else ks
    f_ref, _ = oracle.internal_force(sub)
    kv_ref = oracle.operator_apply(sub, wl.v, a_K=1.0)
    cv_ref = oracle.operator_apply(sub, wl.v, a_K=0.0, a_C=1.0) if wl.udot is not None else None
    gu_ref, gud_ref, gth_ref = oracle.vjp(sub, wl.v)
    dg_ref = oracle.jacobi_diag(sub, a_K=1.0, a_C=1.0)
    damped = wl.udot is not None and np.abs(wl.params[:, 2:4]).max() > 0
    out = {"f": rel(f[sel], f_ref[sel]), "Kv": rel(kv[sel], kv_ref[sel]),
           "Cv": rel(cv[sel], cv_ref[sel]) if damped else None,
           "g_u": rel(gu[sel], gu_ref[sel]), "g_udot": rel(gud[sel], gud_ref[sel]) if damped else None,
           "g_theta": rel(gth[emask], gth_ref), "diag": rel(dg[sel], dg_ref[sel])}
    if one_pass:
        y_ref = kv_ref + cv_ref if cv_ref is not None else kv_ref
        out["f_one_pass"] = rel(f1[sel], f_ref[sel])
        out["Kv+Cv_one_pass"] = rel(y1[sel], y_ref[sel])
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_errors_block(prec):
    """384-element T10 block, SVK, 4-point rule (every node)."""
    _record("block 4^3 T10 SVK", prec, **_operators(synth.block_t10_svk(), prec))


@pytest.mark.parametrize("prec", [0, 1])
def test_errors_beam(prec):
    """480k-element beam, neo-Hookean + Kelvin-Voigt (400 sampled nodes)."""
    wl = synth.cantilever_beam()
    ks = np.random.default_rng(31).choice(wl.n_nodes, 400, replace=False)
    _record("beam 480k T10 NH+KV", prec, **_operators(wl, prec, ks))


def test_errors_diff_block():
    """1 M-element block with per-element (mu, lambda), FP32 (400 nodes)."""
    wl = synth.diff_block()
    ks = np.random.default_rng(32).choice(wl.n_nodes, 400, replace=False)
    _record("diff 1M T10 NH+KV per-element", 1, **_operators(wl, 1, ks))


def test_errors_batch():
    """512-body batch (mixed types, SVK / neo-Hookean), FP32, force and K v
    at 4 nodes of every body, each body normalised on its own."""
    tl = T()
    wl = synth.batch_bodies(512)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    u, v = dev(wl.u, torch.float64), dev(wl.v, torch.float32)
    f, y = mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0)
    mesh.sync()
    f, y = f.clone(), y.clone()
    # the same step as the benchmark runs it after autotuning: one pass per block and law
    mesh.set_launch_mode(tl.LAUNCH_PER_PASS)
    assert mesh.info["force_matvec_fused"] == 1
    f1, y1 = mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0)
    mesh.sync()
    lo = np.full(wl.n_bodies, np.iinfo(np.int64).max)
    hi = np.full(wl.n_bodies, -1)
    for blk in wl.blocks:
        np.minimum.at(lo, blk.body, blk.conn.min(axis=1))
        np.maximum.at(hi, blk.body, blk.conn.max(axis=1))
    rng = np.random.default_rng(33)
    ks, owner = [], []
    for b in range(wl.n_bodies):
        pick = [lo[b]] + list(lo[b] + rng.choice(hi[b] - lo[b] + 1, 3, replace=False))
        ks += pick
        owner += [b] * 4
    ks, owner = np.array(ks), np.array(owner)
    sub, _ = _subset(wl, ks)
    f_ref, _ = oracle.internal_force(sub)
    y_ref = oracle.operator_apply(sub, wl.v, a_K=1.0)
    errs = {}
    for name, got, ref in (("f", f, f_ref), ("Kv", y, y_ref), ("f_one_pass", f1, f_ref), ("Kv_one_pass", y1, y_ref)):
        g = got.double().cpu().numpy()[ks]
        r = ref[ks]
        den = np.zeros(wl.n_bodies)
        np.maximum.at(den, owner, np.abs(r).max(axis=1))
        errs[name] = float((np.abs(g - r).max(axis=1) / den[owner]).max())
    mesh.close()
    _record("batch 512 bodies", 1, **errs)


def test_errors_newton_velocity():
    """64-beam implicit step (FP32 operator, FP64 residual, Newton 1e-8):
    velocity of the smallest body against the oracle's step of that body
    solved to 1e-10."""
    tl = T()
    wl = synth.newton_beams(64)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = torch.from_numpy(wl.fixed).cuda()
    G = np.array([0.0, 0.0, -9.81])
    v, rep = mesh.newton_step(z, z.clone(), 1e-3, gravity=G, fixed=fx, newton_rtol=1e-8, cg_rtol=1e-4,
                              max_newton=20, max_cg=4000, use_graph=True)
    assert rep["status"] == 0
    bodies = synth.split_bodies(wl)
    k = int(np.argmin([b.n_elem for b in bodies]))
    b = bodies[k]
    lo = int(wl.blocks[0].conn[wl.blocks[0].body == k].min())
    zb = np.zeros_like(b.X)
    v_ref, rep_ref = oracle.newton_step(b, zb, zb, 1e-3, G, fixed=b.fixed, newton_rtol=1e-10, cg_rtol=1e-8,
                                        max_newton=20, max_cg=20000)
    err = rel(v.cpu().numpy()[lo:lo + b.n_nodes], v_ref)
    TABLE["Newton 64 beams (FP32 operator, FP64 residual, rtol 1e-8)"] = {"v": err}
    assert err <= 1e-6
    mesh.close()


def test_zz_write_table():
    """Print (and optionally store) the table gathered above."""
    for k, row in TABLE.items():
        print(k, " ".join(f"{n}={e:.2e}" for n, e in row.items()))
    path = os.environ.get("TLFE_ERROR_TABLE")
    if path:
        with open(path, "w") as fh:
            json.dump(TABLE, fh, indent=1)
