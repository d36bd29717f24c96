"""The bounds-checked build (libtlfe_checked.so: every index the element
kernels read from a device table range-checked into the status word) runs
every element type, path, scatter mode and precision without a single
out-of-range index, and gives the oracle's results. It runs in a child
process, which loads that build through TLFE_LIB."""

import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import oracle, synth
from synth.workloads import Block, Workload
from paper_2602_17002_gb300 import tlfe
assert tlfe.LIB_PATH.endswith("libtlfe_checked.so"), tlfe.LIB_PATH

def rel(got, ref):
    return float(np.abs(got.double().cpu().numpy() - ref).max() / max(np.abs(ref).max(), 1e-300))

q27 = synth.q27_beam(cells=(5, 3, 2))
curved = synth.q27_beam(cells=(4, 2, 2), curve=0.05)
batch = synth.batch_bodies(n_bodies=8, seed=19, ne_range=(40, 400))
batch.udot = 0.01 * np.random.default_rng(3).standard_normal(batch.X.shape)
batch.params[1::2, 2] = 1e3
cases = [("beam", synth.small_beam(cells=(10, 3, 2))), ("batch", batch), ("q27", q27), ("q27_curved", curved),
         ("diff", synth.diff_block(cells=3))]
out = {}
for name, wl in cases:
    f_ref, _ = oracle.internal_force(wl)
    y_ref = oracle.operator_apply(wl, wl.v, a_K=1.0, a_C=1.0)
    g_ref, _, th_ref = oracle.vjp(wl, wl.v)
    for prec, tol in ((tlfe.FP32, 2e-5), (tlfe.FP64, 1e-12)):
        for scatter in (tlfe.SCATTER_ATOMIC, tlfe.SCATTER_COLOR, tlfe.SCATTER_SORTED):
            for mode in (tlfe.LAUNCH_PER_PASS, tlfe.LAUNCH_FUSED):
                mesh = tlfe.Mesh.from_workload(wl, precision=prec, scatter=scatter)
                mesh.set_launch_mode(mode)
                dt = mesh.torch_dtype
                u = torch.from_numpy(wl.u).cuda()
                ud = None if wl.udot is None else torch.from_numpy(wl.udot).to("cuda", dt)
                v = torch.from_numpy(wl.v).to("cuda", dt)
                f = mesh.internal_force(u, ud)
                y = mesh.tangent_matvec(u, ud, v, 0.0, 1.0, 1.0)
                gu, gud, gth = mesh.vjp(u, ud, v)
                mesh.jacobi_diag(u, ud, 0.0, 1.0, 1.0)
                n_inv = mesh.sync()        # raises TLFEError on any out-of-range index
                errs = [rel(f, f_ref), rel(y, y_ref), rel(gu, g_ref), rel(gth, th_ref)]
                assert max(errs) <= tol, (name, prec, scatter, mode, errs)
                out[f"{name}/{prec}/{scatter}/{mode}"] = max(errs)
                mesh.close()
print(json.dumps({"cases": len(out), "max_err": max(out.values())}))
'''


def test_bounds_checked_build_finds_no_out_of_range_index():
    from paper_2602_17002_gb300 import build_lib
    lib = build_lib.LIB_CHECKED
    if not os.path.exists(lib):
        build_lib.build(checked=True)
    env = dict(os.environ, TLFE_LIB=lib)
    res = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    rep = json.loads(res.stdout.strip().splitlines()[-1])
    assert rep["cases"] == 5 * 2 * 3 * 2
