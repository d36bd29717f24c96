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

CHUNK = 4096                  # values per partial sum of the entry point
LIMIT = 4096 * 4096           # largest n it accepts


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
    mesh.close()


def test_norm_noalloc_several_chunks_ragged_tail_and_limit():
    """Many partial sums (a ragged last chunk, and n at the limit) and the
    empty vector, each twice in a row, against body_norms on a mesh of that
    many values and against numpy."""
    from paper_2602_17002_gb300 import tlfe
    rng = np.random.default_rng(23)
    for n in (3 * CHUNK + 17, LIMIT):
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        ref_np = float(np.linalg.norm(x.cpu().numpy()))
        for _ in range(2):
            out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            tlfe.tlfe_norm_noalloc(x, out)
            torch.cuda.synchronize()
            assert abs(float(out[0]) - ref_np) <= 1e-12 * ref_np, n
    # a mesh whose node array holds 3 * CHUNK + 17 values is not possible
    # (multiples of 3); compare a multi-chunk node array with body_norms
    wl = synth.small_beam(cells=(40, 4, 4))           # > 12,288 values: several chunks
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32)
    for _ in range(2):
        x = torch.from_numpy(rng.standard_normal(wl.X.shape)).cuda()
        assert x.numel() > 3 * CHUNK and x.numel() % CHUNK != 0
        ref = float(mesh.body_norms(x)[0])
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        tlfe.tlfe_norm_noalloc(x.reshape(-1), out)
        torch.cuda.synchronize()
        assert abs(float(out[0]) - ref) <= 1e-12 * ref
    mesh.close()
    # n = 0: the norm of the empty vector, with scratch left over from above
    for _ in range(2):
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        tlfe.tlfe_norm_noalloc(torch.zeros(0, dtype=torch.float64, device="cuda"), out)
        torch.cuda.synchronize()
        assert float(out[0]) == 0.0


def test_norm_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2602_17002_gb300 import tlfe
    big = torch.zeros(LIMIT + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tlfe.TLFEError) as ei:
        tlfe.tlfe_norm_noalloc(big, out)
    assert ei.value.code == 1 and "exceeds the maximum" in str(ei.value)
