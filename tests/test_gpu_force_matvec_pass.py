"""The one-pass force + operator product (tlfe_force_matvec on FP32 T4 / T10 /
H8 meshes): one kernel per element block and law gathers the nodal inputs,
forms F, Fdot and the stress once, and accumulates both element vectors, the
internal force (Sec. 4.3, Eq. internal_force_universal) and the operator
product (App. C tangents, consistent mass of Sec. 4.1). It matches the two
separate passes to FP32 rounding and the FP64 oracle at the FP32 bar, in
every scatter mode, on both element paths, with mixed types and laws; the
sorted scatter repeats bit for bit; meshes without the pass report so and
fall back to two passes."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-5
H = 1e-3


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def dev(a, dt):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def relerr(got, ref):
    got = got.double().cpu().numpy() if hasattr(got, "cpu") else got
    ref = ref.double().cpu().numpy() if hasattr(ref, "cpu") else ref
    den = np.abs(ref).max()
    return np.abs(got - ref).max() / (den if den > 0 else 1.0)


def _mixed(seed=11):
    """Mixed T4 / T10 / H8 bodies, SVK and neo-Hookean, some damped, moving."""
    wl = synth.batch_bodies(n_bodies=12, seed=seed, ne_range=(40, 400))
    params = wl.params.copy()
    params[1::3, 2] = 1e3
    wl.params = params
    wl.udot = 0.01 * np.random.default_rng(seed + 20).standard_normal(wl.X.shape)
    return wl


CASES = [("beam", 0, 2), ("beam", 1, 2), ("beam", 2, 2), ("beam", 0, 1), ("mixed", 0, 0), ("mixed", 2, 0)]


@pytest.mark.parametrize("name,scatter,path", CASES)
@pytest.mark.parametrize("coeffs", [(0.0, 1.0, 1.0), (1.0 / H, H, 1.0)])
def test_one_pass_equals_two_passes_and_the_oracle(name, scatter, path, coeffs):
    tl = T()
    wl = synth.small_beam(cells=(9, 2, 3)) if name == "beam" else _mixed()
    a_M, a_K, a_C = coeffs
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32, scatter=scatter, element_path=path)
    mesh.set_launch_mode(tl.LAUNCH_PER_PASS)
    assert mesh.info["force_matvec_fused"] == 1   # (the beam's elements are affine: a_M != 0 is defined on both paths)
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, torch.float32), dev(wl.v, torch.float32)
    f, y = torch.empty_like(v), torch.empty_like(v)
    for _ in range(2):                         # direct evaluation and capture, then a replay
        f.fill_(7.0)
        y.fill_(7.0)
        mesh.force_matvec(u, ud, v, a_M, a_K, a_C, f=f, y=y)
    f2 = mesh.internal_force(u, ud)
    y2 = mesh.tangent_matvec(u, ud, v, a_M, a_K, a_C)
    assert mesh.sync() == 0
    assert relerr(f, f2) <= 1e-6 and relerr(y, y2) <= 1e-6
    f_ref, _ = oracle.internal_force(wl)
    y_ref = oracle.operator_apply(wl, wl.v, a_M=a_M, a_K=a_K, a_C=a_C)
    assert relerr(f, f_ref) <= TOL32 and relerr(y, y_ref) <= TOL32
    if scatter == 2:                           # node-ordered partial sums: bit for bit
        a, b = f.cpu().numpy().copy(), y.cpu().numpy().copy()
        mesh.force_matvec(u, ud, v, a_M, a_K, a_C, f=f, y=y)
        mesh.sync()
        assert np.array_equal(a.view(np.uint32), f.cpu().numpy().view(np.uint32))
        assert np.array_equal(b.view(np.uint32), y.cpu().numpy().view(np.uint32))
    mesh.close()


def test_one_pass_without_velocity_and_the_host_buffer_step():
    """No udot (the elastic operator alone); tlfe_step_host with f and y takes
    the same pass and returns what the device call returns."""
    tl = T()
    wl = synth.small_beam(cells=(8, 2, 2))
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    assert mesh.info["force_matvec_fused"] == 1
    u, v = dev(wl.u, torch.float64), dev(wl.v, torch.float32)
    f, y = mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0)
    mesh.sync()
    assert relerr(f, oracle.internal_force(wl, udot=None)[0]) <= TOL32
    assert relerr(y, oracle.operator_apply(wl, wl.v, a_K=1.0, udot=None)) <= TOL32
    uh = np.ascontiguousarray(wl.u)
    udh = np.ascontiguousarray(wl.udot, dtype=np.float32)
    vh = np.ascontiguousarray(wl.v, dtype=np.float32)
    fh = np.zeros_like(vh)
    yh = np.zeros_like(vh)
    mesh.step_host(uh, udh, vh, None, f=fh, y=yh, a_M=0.0, a_K=1.0, a_C=1.0)
    mesh.step_host_wait()
    fd = mesh.internal_force(u, dev(wl.udot, torch.float32)).cpu().numpy()
    yd = mesh.tangent_matvec(u, dev(wl.udot, torch.float32), v, 0.0, 1.0, 1.0).cpu().numpy()
    assert relerr(fh, fd) <= 1e-6 and relerr(yh, yd) <= 1e-6
    mesh.close()


def test_autotune_keeps_a_correct_choice_and_meshes_without_the_pass_fall_back():
    tl = T()
    wl = _mixed(seed=5)
    mesh = tl.Mesh.from_workload(wl, precision=tl.FP32)
    u, ud, v = dev(wl.u, torch.float64), dev(wl.udot, torch.float32), dev(wl.v, torch.float32)
    mesh.autotune(u, ud, v)
    assert mesh.info["force_matvec_fused"] in (0, 1)
    f, y = mesh.force_matvec(u, ud, v, 0.0, 1.0, 1.0)
    mesh.sync()
    assert relerr(f, oracle.internal_force(wl)[0]) <= TOL32
    assert relerr(y, oracle.operator_apply(wl, wl.v, a_K=1.0, a_C=1.0)) <= TOL32
    mesh.close()
    # FP64 meshes and meshes holding Q27 bricks run two passes
    m64 = tl.Mesh.from_workload(wl, precision=tl.FP64)
    assert m64.info["force_matvec_fused"] == 0
    f, y = m64.force_matvec(u, dev(wl.udot, torch.float64), dev(wl.v, torch.float64), 0.0, 1.0, 1.0)
    m64.sync()
    assert relerr(f, oracle.internal_force(wl)[0]) <= 1e-12
    m64.close()
    q = synth.q27_beam(cells=(4, 2, 2))
    mq = tl.Mesh.from_workload(q, precision=tl.FP32)
    assert mq.info["force_matvec_fused"] == 0
    uq, vq = dev(q.u, torch.float64), dev(q.v, torch.float32)
    udq = dev(q.udot, torch.float32)
    f, y = mq.force_matvec(uq, udq, vq, 0.0, 1.0, 1.0)
    mq.sync()
    assert relerr(f, oracle.internal_force(q)[0]) <= TOL32
    assert relerr(y, oracle.operator_apply(q, q.v, a_K=1.0, a_C=1.0)) <= TOL32
    mq.close()
