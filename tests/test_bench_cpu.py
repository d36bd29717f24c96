"""Host-side logic of bench.py (no GPU): the kernel-source hash that keys the
committed ncu traffic figures, the per-law FLOP table of the batch workload,
and the command line."""

import os
import subprocess
import sys

import numpy as np

import bench
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_comment_stripping_keeps_code_and_literals():
    src = ('int a = 1; // trailing note\n'
           '/* block\n   comment */ float b = 2.0f;\n'
           'const char *s = "a // not a comment /* nor this */";\n'
           "char c = '/';\n\n\n"
           'return a; /* one */ /* two */\n')
    out = bench._strip_comments(src)
    assert "trailing note" not in out and "block" not in out and "one" not in out
    assert 'int a = 1;' in out and 'float b = 2.0f;' in out and 'return a;' in out
    assert '"a // not a comment /* nor this */"' in out
    assert "'/'" in out
    assert "\n\n" not in out                      # blank lines dropped


def test_comment_only_edits_keep_the_stripped_text():
    a = "x = y + z; // sum\n/* about it */\nw = 2 * x;\n"
    b = "x = y + z;   // the sum, reworded\n\n// a new comment line\nw = 2 * x;  /* more */\n"
    c = "x = y - z; // sum\nw = 2 * x;\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)


def test_kernel_source_hash_is_stable_and_covers_existing_files():
    csrc = os.path.join(ROOT, "paper_2602_17002_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    h1, h2 = bench.kernel_source_hash(), bench.kernel_source_hash()
    assert h1 == h2 and len(h1) == 16


def test_batch_flop_table_covers_every_type_and_law():
    wl = synth.batch_bodies(n_bodies=24, seed=3)
    law = np.asarray(wl.model)
    for b in wl.blocks:
        for lw in np.unique(law[b.body]):
            ent = bench.FLOP_PER_QP_BATCH[(b.etype, int(lw))]
            assert 0 < ent["force"] < ent["matvec"]
            # one pass does the operator product's work and less than both passes
            assert ent["matvec"] < ent["force_matvec"] < ent["force"] + ent["matvec"]
    beam = bench.FLOP_PER_QP["beam"]
    assert beam["matvec"] < beam["force_matvec"] < beam["force"] + beam["matvec"]


def test_streamed_bytes_of_the_one_pass_kernel():
    """The one pass reads the element data and the inputs once and writes f
    and y: the operator product's bytes plus one written node array."""
    wl = synth.small_beam(cells=(6, 2, 2))
    sb = bench.streamed_bytes(wl)
    assert sb["force_matvec"] == sb["matvec"] + 3 * 4 * wl.n_nodes
    assert sb["force_matvec"] < sb["force"] + sb["matvec"]


def test_command_line_lists_the_workloads_and_modes():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, timeout=120)
    assert out.returncode == 0
    for flag in ("--workload", "--scatter", "--bodies", "--log", "--impl", "--steps", "--warmup", "--gpus"):
        assert flag in out.stdout
    for mode in ("atomic", "colour", "sorted"):
        assert mode in out.stdout


def test_bench_shards_cover_the_workloads():
    """bench.py's split for N GPUs: one body in slabs (elements once each,
    interface nodes shared) and bodies bin-packed (each body on one GPU)."""
    import numpy as np

    import bench
    import synth
    wl = synth.small_beam(cells=(10, 2, 2))
    shares = [bench.shard_one_body(wl, r, 3) for r in range(3)]
    assert sum(sh.n_elem for sh, _, _ in shares) == wl.n_elem
    assert all(itf.n == shares[0][1].n > 0 for _, itf, _ in shares)
    bw = synth.batch_bodies(n_bodies=11, seed=2, ne_range=(30, 200))
    parts = [bench.shard_bodies(bw, r, 4) for r in range(4)]
    assert np.array_equal(np.sort(np.concatenate([p for _, p in parts])), np.arange(11))
    assert sum(sh.n_elem for sh, _ in parts) == bw.n_elem
    assert sum(sh.n_nodes for sh, _ in parts) == bw.n_nodes
    assert bench.parallelism("beam", 1) == "1 GPU" and "slab" in bench.parallelism("beam", 2)


def test_case_file_sets_option_defaults_and_flags_override_it(tmp_path):
    import json

    import pytest
    case = tmp_path / "case.json"
    case.write_text(json.dumps({"workload": "batch", "scatter": "sorted", "steps": 7, "sub-steps": 4,
                                "headline_only": True}))
    a = bench.parse_args(bench.make_parser(), ["--case", str(case)])
    assert (a.workload, a.scatter, a.steps, a.sub_steps, a.headline_only) == ("batch", "sorted", 7, 4, True)
    assert a.warmup == 3 and a.gpus == 1                     # untouched defaults
    a = bench.parse_args(bench.make_parser(), ["--case", str(case), "--steps", "9", "--scatter", "colour"])
    assert (a.steps, a.scatter, a.workload) == (9, "colour", "batch")
    assert bench.parse_args(bench.make_parser(), []).workload == "beam"
    for bad in ({"workloads": "beam"}, {"scatter": "smem"}, {"steps": "many"}, ["beam"]):
        case.write_text(json.dumps(bad))
        with pytest.raises(SystemExit):
            bench.parse_args(bench.make_parser(), ["--case", str(case)])
