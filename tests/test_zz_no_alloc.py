"""tlfe_norm_noalloc, the entry point for callers that cannot allocate device
memory, against tlfe_body_norms (the allocating entry point with the same
chunked FP64 reduction), called through the C ABI twice in a row.

Collected last on purpose: when it fails, a run stopping at the first failure
has already run every other test."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_norm_noalloc_matches_body_norms_twice():
    from paper_2602_17002_gb300 import tlfe
    wl = synth.small_beam(cells=(12, 2, 2))
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32)
    rng = np.random.default_rng(17)
    for _ in range(2):
        x = torch.from_numpy(rng.standard_normal(wl.X.shape)).cuda()
        ref = mesh.body_norms(x)                       # one body: the norm of the whole array
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        tlfe.tlfe_norm_noalloc(x.reshape(-1), out)
        torch.cuda.synchronize()
        r, o = float(ref[0]), float(out[0])
        assert abs(o - r) <= 1e-12 * r
        assert abs(o - float(np.linalg.norm(x.cpu().numpy()))) <= 1e-12 * r


def test_norm_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2602_17002_gb300 import tlfe
    big = torch.zeros(4096 * 4096 + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tlfe.TLFEError) as ei:
        tlfe.tlfe_norm_noalloc(big, out)
    assert ei.value.code == 1 and "exceeds the maximum" in str(ei.value)
