"""Node-patch layouts of the tile kernels: the banked layout (each tile's node
list permuted so that a quarter warp's 16-byte patch loads hit distinct bank
groups) and the plain ascending layout give bit-identical results in the
deterministic (sorted) scatter mode, on every element type and path, and the
banked layout's patch loads take about one shared-memory pass each."""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T():
    from paper_2602_17002_gb300 import tlfe
    return tlfe


def _run(wl, layout, prec, path):
    tl = T()
    mesh = tl.Mesh.from_workload(wl, precision=prec, scatter=tl.SCATTER_SORTED, element_path=path,
                                 patch_layout=layout)
    dt = mesh.torch_dtype
    u = torch.from_numpy(wl.u).cuda()
    ud = None if wl.udot is None else torch.from_numpy(wl.udot).to("cuda", dt)
    v = torch.from_numpy(wl.v).to("cuda", dt)
    out = [mesh.internal_force(u, ud), mesh.tangent_matvec(u, ud, v, 0.5, 1.0, 1.0)]
    out += [x for x in mesh.vjp(u, ud, v) if x is not None]
    out.append(mesh.jacobi_diag(u, ud, 0.5, 1.0, 1.0))
    mesh.sync()
    info = mesh.info
    mesh.close()
    return [x.cpu() for x in out], info


def _batch():
    wl = synth.batch_bodies(n_bodies=12, seed=41, ne_range=(60, 900))
    wl.udot = 0.01 * np.random.default_rng(4).standard_normal(wl.X.shape)
    wl.params[1::2, 2] = 1e3
    return wl


CASES = {
    "beam": lambda: synth.small_beam(cells=(12, 3, 3)),
    "diff": lambda: synth.diff_block(cells=4),
    "batch": _batch,
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("path", [1, 2])
def test_banked_and_sorted_layouts_agree_bit_for_bit(name, prec, path):
    tl = T()
    wl = CASES[name]()
    if path == tl.PATH_AFFINE and name == "batch":
        path = tl.PATH_AUTO
    a, ia = _run(wl, tl.PATCH_BANKED, prec, path)
    b, ib = _run(wl, tl.PATCH_SORTED, prec, path)
    assert ia["patch_layout"] == tl.PATCH_BANKED and ib["patch_layout"] == tl.PATCH_SORTED
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert ia["patch_passes"] <= ib["patch_passes"]
    if name != "batch":                  # Kuhn T10 tiles
        assert ia["patch_passes"] <= 1.1 < 1.5 < ib["patch_passes"], (ia["patch_passes"], ib["patch_passes"])


def test_banked_layout_is_conflict_free_on_the_full_beam():
    """480k-element beam: a quarter-warp patch load takes at most 1.05
    passes, against about 1.9 in ascending node order."""
    tl = T()
    wl = synth.cantilever_beam()
    info = {}
    for layout in (tl.PATCH_BANKED, tl.PATCH_SORTED):
        m = tl.Mesh.from_workload(wl, precision=tl.FP32, patch_layout=layout)
        info[layout] = m.info
        m.close()
    assert info[tl.PATCH_BANKED]["patch_passes"] <= 1.05
    assert 1.7 < info[tl.PATCH_SORTED]["patch_passes"] < 2.1
    # the banked lists are permutations of the ascending ones: the same memory
    assert info[tl.PATCH_BANKED]["device_bytes"] == info[tl.PATCH_SORTED]["device_bytes"]


def test_bad_patch_layout_is_rejected():
    tl = T()
    wl = synth.small_beam(cells=(2, 1, 1))
    with pytest.raises(tl.TLFEError):
        tl.Mesh.from_workload(wl, patch_layout=7)
