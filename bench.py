"""Benchmark of the TL-FEA hot path on GB300.

Default workload (--workload beam): the 10 x 1 x 1 m cantilever beam,
200 x 20 x 20 cells split into 480,000 Kuhn T10 tetrahedra (674,081 nodes),
5-point quadrature, compressible neo-Hookean (mu = 3.8e6, lambda = 5.8e6 Pa)
with Kelvin-Voigt damping (mu_v = 1e3 Pa s), seeded bending field + 0.1 %
noise, seeded velocities; FP32 element arithmetic, FP64 displacement state.

One step = one pass of the element hot path over the beam:
  internal force f(u, udot)                       (tlfe_internal_force)
  full tangent product y = K_t v + C v            (tlfe_tangent_matvec)
  adjoint g_u, g_udot, g_(mu, lambda) of f . r    (tlfe_vjp)
value = quadrature points processed through that pass per second (whole job).
The same step is also timed with FP64 element arithmetic ("fp64_plain").

Other workloads (one JSON line each):
  --workload newton  64 clamped neo-Hookean beams (6.75 M T10) under gravity:
                     one backward-Euler step, Newton to relative residual 1e-8
                     with Jacobi-PCG; batched FP32 operator + FP64 residual in
                     one CUDA graph, against the FP64 library one body at a time
                     with a host-driven loop.
  --workload batch   512 bodies of uneven size, mixed T4/T10/H8, SVK or
                     neo-Hookean: force + K v of every body, replayed as one
                     CUDA graph.
  --workload diff    1 M-element T10 block with per-element (mu, lambda):
                     loss 1/2 |f - f_target|^2, forward + adjoint through the
                     torch.autograd.Function.
  --workload q27     the beam's 200 x 20 x 20 cells as 80,000 Q27 triquadratic
                     bricks (the same 674,081 nodes), 3 x 3 x 3 Gauss points:
                     the same step as the default workload.

L2: inputs and streamed element data are larger than L2 (129 MB) in every
workload, and a 512 MiB memset flushes L2 before every timed step, outside
the step's CUDA-event pair.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload on the host cores (the benchmark's reference arm).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "quad-pt force evals/s & % HBM roofline; batched FP32 fwd+VJP vs plain FP64"
UNIT = "quad-pt/s"
WORKLOADS = {
    "beam": "cantilever beam 10x1x1 m, 200x20x20 cells -> 480k T10 (674,081 nodes), Q=5, neo-Hookean + "
            "Kelvin-Voigt, FP32",
    "newton": "implicit step: 64 clamped neo-Hookean beams (5:1:1, N_e ~ logU[2e4, 3e5], 6.75 M T10, Q=5), "
              "gravity, h = 1e-3 s, Newton rel. residual 1e-8, Jacobi-PCG rtol 1e-4",
    "batch": "512 bodies, N_e ~ logU[1e3, 2e5], mixed T4 Q1 / T10 Q5 / H8 Q8, SVK or neo-Hookean, "
             "E ~ logU[1e6, 1e9], FP32, graph-captured force + K v",
    "diff": "1 m^3 block 55^3 cells -> 998,250 T10, Q=5, neo-Hookean per-element (mu, lambda) + Kelvin-Voigt, "
            "loss 1/2 |f - f_target|^2, forward + VJP, FP32",
    "q27": "cantilever beam 10x1x1 m, 200x20x20 cells -> 80k Q27 (674,081 nodes), Q=27 (3x3x3 Gauss), "
           "neo-Hookean + Kelvin-Voigt, FP32",
}
GRAVITY = (0.0, 0.0, -9.81)
# Algorithmic FP32 FLOPs per quadrature point of the neo-Hookean + Kelvin-Voigt
# kernels on the affine path: T10 Q5 for the beam workload, Q27 for the q27
# workload. force, matvec, vjp: 2 FFMA + FADD + FMUL thread instructions counted
# by ncu on the scalar build of these kernels; force_matvec (the one-pass force +
# operator product): 2 FFMA + FADD + FMUL + 4 FFMA2 + 2 FADD2 + 2 FMUL2 counted
# by ncu on the packed build (the same count gives the adjoint 1820, against
# 1786 on the scalar build)
FLOP_PER_QP = {"beam": {"force": 852, "matvec": 1589, "vjp": 1786, "force_matvec": 1934},
               "q27": {"force": 1932, "matvec": 3026, "vjp": 3567}}
# batch workload (affine path, no damping): FP32 FLOP per point by (element
# type, law, op), law 0 = SVK, 1 = neo-Hookean; ncu counts of the per-law
# kernels of one timed step (force, matvec: 2 FFMA + FADD + FMUL on the scalar
# build, 512-body batch; force_matvec: with the packed instructions as above,
# 64-body batch)
FLOP_PER_QP_BATCH = {(0, 0): {"force": 288.3, "matvec": 503.3, "force_matvec": 652.3},
                     (0, 1): {"force": 359.3, "matvec": 690.3, "force_matvec": 839.4},
                     (1, 0): {"force": 483.7, "matvec": 865.7, "force_matvec": 1096.7},
                     (1, 1): {"force": 552.3, "matvec": 1048.3, "force_matvec": 1279.3},
                     (2, 0): {"force": 540.0, "matvec": 942.3, "force_matvec": 1188.5},
                     (2, 1): {"force": 610.4, "matvec": 1124.7, "force_matvec": 1370.7}}
# how the end-to-end measurements move data
OVERLAP = ("copies on their own streams: the next step's inputs are copied in while a step computes (two device "
           "staging sets), outputs are copied out as their operations end")
# FP32 FMA roof: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz (maximum SM clock)
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ---------------------------------------------------------------------------
# shared helpers
# ---------------------------------------------------------------------------

_ALU = {}


def alu_peaks():
    """Measured FMA peaks of this GPU (tlfe_peak_probe: independent FMA chains on
    every lane, CUDA events, best of 5 launches), FP32 and FP64, in TFLOP/s,
    with the SM clock sampled while the FP32 probe ran. Cached per process."""
    if not _ALU:
        import torch
        from paper_2602_17002_gb300 import tlfe
        tlfe.load()
        with ClockSampler(torch.cuda.current_device()) as clk:
            f32, ms32 = clk.timed(lambda: tlfe.peak_probe(tlfe.FP32, ctas_per_sm=4, iters=1 << 16))
        f64, ms64 = tlfe.peak_probe(tlfe.FP64, ctas_per_sm=4, iters=1 << 12)
        c = clk.summary()
        _ALU.update(fp32=f32, fp64=f64, sm_mhz=c["sm_mhz"],
                    source=f"measured: tlfe_peak_probe FMA chains, {f32:.1f} TFLOP/s FP32 and {f64:.2f} TFLOP/s FP64 "
                           f"at {c['sm_mhz']} MHz SM clock (derived nominal FP32: 152 x 128 x 2 x 2.07 GHz = "
                           f"{ALU_PEAK_TFLOPS:.1f})")
    return _ALU


def streamed_bytes(wl, s=4):
    """Algorithmic bytes of one force / operator product / adjoint by the
    minimum-traffic count with streamed reference data: connectivity 4 n,
    reference gradients 3 n Q s and weights Q s per element (2 s more with
    per-element parameters); each input node array read once and each output
    node array written once (3 s per node); the adjoint also writes the
    parameter gradient (2 s per element). Node arrays count at the element
    precision s."""
    npe = {0: 4, 1: 10, 2: 8, 3: 27}
    el = sum(b.n_elem * (4 * npe[b.etype] + 3 * npe[b.etype] * b.nq * s + b.nq * s) for b in wl.blocks)
    if wl.elem_mu_lambda is not None:
        el += 2 * s * wl.n_elem
    node = 3 * s * wl.n_nodes
    n_in = 2 if wl.udot is not None else 1
    return {"force": el + node * (n_in + 1), "matvec": el + node * (n_in + 2),
            "force_matvec": el + node * (n_in + 3),   # one pass: u (+udot) and v read, f and y written
            "vjp": el + node * (n_in + 1 + n_in) + 2 * s * wl.n_elem}


def step_launches(info):
    """Element-kernel launches of one force + K v call (tlfe_force_matvec):
    one per pass of the one-pass kernel, else those of both operations."""
    if info["force_matvec_fused"]:
        return info["launches_matvec"]
    return info["launches_force"] + info["launches_matvec"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that determine the element kernels' code, their parameters,
# the mesh layout they read and their launch schedules (not the Newton,
# constraint or load code): the committed ncu traffic is valid while these
# are unchanged
KERNEL_SOURCES = ("k_elem.cuh", "k_wpe.cuh", "k_fused.cuh", "tlfe_fused.h", "tlfe_elem.cuh", "tlfe_math.cuh",
                  "tlfe_internal.h", "tlfe_mesh.h", "api.cu", "k_setup.cu", "k_force.cu", "k_matvec.cu", "k_vjp.cu",
                  "k_diag.cu", "k_fm.cu", "k_fused_force.cu", "k_fused_matvec.cu")


def _strip_comments(src):
    """C/C++ source without comments and blank-line runs, so that the hash
    follows the code, not its prose (string and character literals kept)."""
    import re
    pat = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'', re.S)
    out = pat.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", src)
    return "\n".join(ln.rstrip() for ln in out.splitlines() if ln.strip())


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_17002_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            h.update(name.encode() + _strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary,
    or None when the kernel sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    ent = d.get(kernel_key)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples (every 20 ms) around the timed region. Each sample
    is stamped with the host time it arrived; timed() marks the region, and
    summary() keeps the samples that fall inside it (widened by 50 ms, the
    reporting lag), or, when the region is shorter than the sampling period,
    the sample nearest to it."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.win = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)                      # the first samples arrive before the timed region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def timed(self, fn):
        """Run fn() as the timed region and remember its host-time window."""
        t0 = time.perf_counter()
        out = fn()
        self.win = (t0, time.perf_counter())
        time.sleep(0.1)
        return out

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ts, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((ts, float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        sel, how = rows, "all samples"
        if self.win and rows:
            t0, t1 = self.win
            sel = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
            how = "inside the timed region"
            if not sel:
                mid = 0.5 * (t0 + t1)
                sel = [min(rows, key=lambda r: abs(r[0] - mid))]
                how = f"nearest sample, {abs(sel[0][0] - mid) * 1e3:.0f} ms from the timed region's middle"
        reasons = set()
        for r in sel:
            for nm, val in zip(names, r[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median([r[1] for r in sel]) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "reasons": sorted(reasons), "samples": len(sel),
                "selection": how,
                "timed_region_ms": (self.win[1] - self.win[0]) * 1e3 if self.win else None}


def dist_setup():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    """Max of a host scalar over all ranks (NCCL: through a CUDA tensor;
    gloo: a CPU tensor)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(x, world):
    """Sum of a host scalar over all ranks."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(units_per_rank, world, step_ms_max):
    """Whole-job throughput when every rank processes units_per_rank per step
    and the job takes the slowest rank's time."""
    return world * units_per_rank / (step_ms_max * 1e-3)


SPLIT = {"beam": "slab", "q27": "slab", "diff": "slab", "batch": "bodies", "newton": "bodies"}


def parallelism(workload, world):
    if world == 1:
        return "1 GPU"
    if SPLIT[workload] == "slab":
        return (f"slab split x{world}: the body's elements in {world} equal slabs along x, one per GPU; the "
                f"duplicated interface nodes' partial results summed by one NCCL all-reduce of a compact buffer "
                f"per operation")
    return f"bodies bin-packed x{world} by cost (largest first onto the least-loaded GPU); no exchange"


def base_line(args, world, workload, value, unit, step_ms, dtype, higher=True, **config):
    return {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": higher, "scaling": "strong",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded)",
            "config": dict({"workload": WORKLOADS[workload],
                            "l2": "inputs > L2; 512 MiB memset flush before every timed step, outside its events",
                            "parallelism": parallelism(workload, world)}, **config)}


def shard_one_body(wl, rank, world):
    """This rank's slab of a one-body workload: (share, interface, element mask)."""
    from paper_2602_17002_gb300 import shard
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    masks = shard.slab_partition(wl.X, blocks, world)
    nodes_all = [shard.local_blocks(blocks, m)[0] for m in masks]
    itf = shard.interfaces(nodes_all)[rank]
    share, _ = shard.sub_workload(wl, masks[rank])
    return share, itf, masks[rank]


def shard_bodies(wl, rank, world):
    """This rank's bodies of a many-body workload (cost-based bin packing):
    (share with its bodies renumbered, their global ids)."""
    from paper_2602_17002_gb300 import shard
    blocks = [(b.etype, b.nq, b.conn, b.body) for b in wl.blocks]
    parts = shard.pack_bodies(shard.body_costs(blocks, wl.n_bodies), world)
    share, _ = shard.sub_workload(wl, shard.body_masks(blocks, parts[rank]), bodies=parts[rank])
    return share, parts[rank]


def timed_steps(step, steps, flush, stream, n_ev=2, label="timed"):
    """Run `steps` calls of step(ev) with an L2 flush before each; step records
    its own events ev[0..n_ev-1]; returns the per-step event lists. The steps
    run inside the NVTX range `label` (profilers can select it)."""
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(steps)]
    torch.cuda.nvtx.range_push(label)
    for k in range(steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return evs


# ---------------------------------------------------------------------------
# CPU oracle samples (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def _compact_sample(wl, n):
    """The first n / n_blocks elements of every block as a self-contained
    workload holding only the nodes they use (renumbered), for shipping to
    worker processes."""
    import numpy as np
    from synth.workloads import Block, Workload
    nb = -(-n // len(wl.blocks))
    parts, ml, off = [], [], 0
    for blk in wl.blocks:
        k = min(nb, blk.n_elem)
        parts.append((blk, k))
        if wl.elem_mu_lambda is not None:
            ml.append(wl.elem_mu_lambda[off:off + k])
        off += blk.n_elem
    nodes = np.unique(np.concatenate([blk.conn[:k].ravel() for blk, k in parts]))
    remap = lambda c: np.searchsorted(nodes, c).astype(c.dtype)
    pick = lambda a: None if a is None else np.ascontiguousarray(a[nodes])
    return Workload("sample", pick(wl.X), [Block(blk.etype, blk.nq, remap(blk.conn[:k]), blk.body[:k])
                                          for blk, k in parts], wl.model, wl.params,
                    u=pick(wl.u), udot=pick(wl.udot), v=pick(wl.v),
                    elem_mu_lambda=np.concatenate(ml) if ml else None)


def _sample_text(wl, sub):
    names = 'T4 T10 H8 Q27'.split()
    if len(sub.blocks) == 1:
        b = sub.blocks[0]
        return f"first {b.n_elem} of {wl.n_elem} elements ({names[b.etype]} block)"
    return "first " + ", ".join(f"{b.n_elem} {names[b.etype]}" for b in sub.blocks) + \
        f" of the {len(sub.blocks)} blocks ({wl.n_elem} elements)"


_WORKER_WL = None


def _oracle_worker_init(sub):
    global _WORKER_WL
    _WORKER_WL = sub
    import oracle
    oracle.lib()


def _oracle_ops(workload, sub):
    import oracle
    if workload in ("beam", "q27"):
        oracle.internal_force(sub)
        oracle.operator_apply(sub, sub.v, a_K=1.0, a_C=1.0)
        oracle.vjp(sub, sub.v)
        return "force + closed-form K_t v + C v + adjoint"
    if workload == "batch":
        oracle.internal_force(sub)
        oracle.operator_apply(sub, sub.v, a_K=1.0)
        return "force + closed-form K v"
    oracle.internal_force(sub)
    oracle.vjp(sub, sub.v)
    return "force + adjoint"


def _oracle_worker_chunk(workload, k, procs):
    """One worker's share of the sample: the k-th of procs equal element
    ranges of every block."""
    import numpy as np
    from synth.workloads import Block, Workload
    wl = _WORKER_WL
    blocks, ml, off = [], [], 0
    for blk in wl.blocks:
        i0, i1 = blk.n_elem * k // procs, blk.n_elem * (k + 1) // procs
        if i1 > i0:
            blocks.append(Block(blk.etype, blk.nq, blk.conn[i0:i1], blk.body[i0:i1]))
            if wl.elem_mu_lambda is not None:
                ml.append(wl.elem_mu_lambda[off + i0:off + i1])
        off += blk.n_elem
    if not blocks:
        return 0.0
    sub = Workload("chunk", wl.X, blocks, wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v,
                   elem_mu_lambda=np.concatenate(ml) if ml else None)
    t0 = time.perf_counter()
    _oracle_ops(workload, sub)
    return time.perf_counter() - t0


def oracle_pool(workload, wl, n_sample):
    """Spawned worker processes (one per host core, up to 64) holding the
    compact sample, for the all-core oracle timing; None for the Newton
    workload (one body, not split). Spawned, not forked: the parent has
    touched the GPU by then."""
    if workload == "newton":
        return None
    import multiprocessing as mp
    procs = max(1, min(64, os.cpu_count() or 1))
    sub = _compact_sample(wl, _sample_size(workload, n_sample))
    return mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init, initargs=(sub,)), procs, sub


def _sample_size(workload, n_sample):
    if workload == "q27":   # a Q27 brick costs the oracle about 40 T10 elements (27 points x 27 nodes)
        return max(64, n_sample // 40)
    return n_sample


def cpu_sample_parallel(workload, wl, pool_info):
    """The oracle on the same bounded sample as cpu_sample, split in equal
    element ranges over the pool's processes; wall time from the first
    dispatch to the last result. Returns (value, seconds, processes, text)."""
    pool, procs, sub = pool_info
    chunks = [(workload, k, procs) for k in range(procs)]
    t0 = time.perf_counter()
    pool.starmap(_oracle_worker_chunk, chunks, chunksize=1)
    dt = time.perf_counter() - t0
    what = {"beam": "force + closed-form K_t v + C v + adjoint", "q27": "force + closed-form K_t v + C v + adjoint",
            "batch": "force + closed-form K v"}.get(workload, "force + adjoint")
    nqp = sum(b.n_elem * b.nq for b in sub.blocks)
    return (nqp / dt, dt, procs, f"{_sample_text(wl, sub)}, {what}, split over {procs} processes, {dt:.2f} s wall")


def cpu_sample(workload, wl, n_sample):
    """Time the oracle on a bounded sample of the workload on one host core.
    Returns (value in the workload's unit, seconds, threads, sample text)."""
    import numpy as np
    import oracle
    oracle.lib()
    if workload == "newton":
        import synth
        bodies = synth.split_bodies(wl)
        b = min(bodies, key=lambda x: x.n_elem)
        z = np.zeros_like(b.X)
        t0 = time.perf_counter()
        _, rep = oracle.newton_step(b, z, z, 1e-3, np.array(GRAVITY), fixed=b.fixed, newton_rtol=1e-8,
                                    cg_rtol=1e-4, max_newton=20, max_cg=4000)
        dt = time.perf_counter() - t0
        # steps/s of the whole batch, extrapolated per element from the smallest body
        val = 1.0 / (dt * wl.n_elem / b.n_elem)
        return val, dt, 1, (f"oracle Newton step of the smallest body ({b.n_elem} T10), extrapolated per element "
                            f"to {wl.n_elem}, {dt:.1f} s")
    sub = _compact_sample(wl, _sample_size(workload, n_sample))
    t0 = time.perf_counter()
    what = _oracle_ops(workload, sub)
    dt = time.perf_counter() - t0
    nqp = sum(b.n_elem * b.nq for b in sub.blocks)
    return nqp / dt, dt, 1, f"{_sample_text(wl, sub)}, {what}, {dt:.1f} s"


def scatter_mode(args):
    from paper_2602_17002_gb300 import tlfe
    return {"atomic": tlfe.SCATTER_ATOMIC, "colour": tlfe.SCATTER_COLOR, "sorted": tlfe.SCATTER_SORTED}[args.scatter]


def build_workload(workload, bodies=512):
    import synth
    if workload == "beam":
        return synth.cantilever_beam()
    if workload == "q27":
        return synth.q27_beam(cells=(200, 20, 20))
    if workload == "newton":
        return synth.newton_beams(64)
    if workload == "batch":
        return synth.batch_bodies(bodies)
    return synth.diff_block()


def diff_cotangent(wl):
    import numpy as np
    return np.random.default_rng(24).standard_normal(wl.X.shape)


def run_reference(args):
    """CPU oracle arm: rank 0 only; each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    wl = build_workload(args.workload, args.bodies)
    if args.workload == "diff":
        wl.v = diff_cotangent(wl)
    # all host cores (spawned processes over element ranges); the Newton
    # sample, one body, on one core
    pool_info = oracle_pool(args.workload, wl, args.ref_sample)
    step = ((lambda: cpu_sample_parallel(args.workload, wl, pool_info)) if pool_info
            else (lambda: cpu_sample(args.workload, wl, args.ref_sample)))
    ts, vals = [], []
    what, thr = "", 1
    try:
        if pool_info:
            for _ in range(max(0, args.warmup)):
                step()
        for _ in range(1 if args.workload == "newton" else args.steps):
            v, dt, thr, what = step()
            ts.append(dt)
            vals.append(v)
    finally:
        if pool_info:
            pool_info[0].close()
            pool_info[0].join()
    value = float(np.mean(vals))
    unit = "steps/s" if args.workload == "newton" else UNIT
    line = base_line(args, 1, args.workload, value, unit, float(np.mean(ts)) * 1e3, "f64")
    line.update({"impl": "reference", "n_gpus": args.gpus,
                 "cpu_baseline": {"value": value, "unit": unit, "cores": thr, "kind": "oracle", "sample": what},
                 "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    line["config"]["parallelism"] = f"host, {thr} core{'s' if thr > 1 else ''}"
    line["config"]["workload"] = WORKLOADS[args.workload].replace(", FP32", "") + \
        " (the FP64 CPU oracle on a bounded sample of it)"
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# workload: beam (default)
# ---------------------------------------------------------------------------

def run_beam(args, rank, world, workload="beam"):
    import numpy as np
    import torch

    from paper_2602_17002_gb300 import tlfe
    full = build_workload(workload)
    wl, itf = full, None
    if world > 1:   # this GPU's slab; interface rows summed over the GPUs after every operation
        wl, itf, _ = shard_one_body(full, rank, world)
    xs_cache = {}

    def xsum(t):
        if itf is None:
            return
        if t.dtype not in xs_cache:
            from paper_2602_17002_gb300 import shard
            xs_cache[t.dtype] = shard.InterfaceSum(itf, t.dtype, "cuda")
        xs_cache[t.dtype](t)

    tag = workload
    fpq = FLOP_PER_QP[workload]
    pre = "" if workload == "beam" else workload + "_"   # traffic keys of the committed ncu summary
    L = tlfe.load()
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    sp = tlfe._stream(stream)
    u = torch.from_numpy(wl.u).to("cuda", torch.float64)   # displacement state: FP64 in both precisions

    def make(prec, path=0):
        mesh = tlfe.Mesh.from_workload(wl, precision=prec, element_path=path, scatter=scatter_mode(args))
        dt = mesh.torch_dtype
        ud = torch.from_numpy(wl.udot).to("cuda", dt)
        v = torch.from_numpy(wl.v).to("cuda", dt)
        outs = [torch.empty_like(ud) for _ in range(4)]
        gth = torch.empty((wl.n_elem, 2), dtype=torch.float64, device="cuda")
        return mesh, ud, v, outs, gth

    def make_step(mesh, u_, ud, v, outs, gth):
        """The step's calls and the names of its timed phases: force and
        operator product in one pass (tlfe_force_matvec, graph-replayed) where
        the mesh takes it after autotuning, else in two; then the adjoint."""
        h = mesh.handle
        f, y, gu, gud = outs
        one_pass = bool(mesh.info["force_matvec_fused"])
        names = ["force_matvec", "vjp"] if one_pass else ["force", "matvec", "vjp"]

        def step(ev=None):
            if ev:
                ev[0].record(stream)
            if one_pass:
                tlfe._check(L.tlfe_force_matvec(h, tlfe._ptr(u_), tlfe._ptr(ud), tlfe._ptr(v), 0.0, 1.0, 1.0,
                                                tlfe._ptr(f), tlfe._ptr(y), sp))
                xsum(f)
                xsum(y)
            else:
                tlfe._check(L.tlfe_internal_force(h, tlfe._ptr(u_), tlfe._ptr(ud), tlfe._ptr(f), sp))
                xsum(f)
                if ev:
                    ev[1].record(stream)
                tlfe._check(L.tlfe_tangent_matvec(h, tlfe._ptr(u_), tlfe._ptr(ud), tlfe._ptr(v), 0.0, 1.0, 1.0,
                                                  tlfe._ptr(y), sp))
                xsum(y)
            if ev:
                ev[len(names) - 1].record(stream)
            tlfe._check(L.tlfe_vjp(h, tlfe._ptr(u_), tlfe._ptr(ud), tlfe._ptr(v), tlfe._ptr(gu), tlfe._ptr(gud),
                                   tlfe._ptr(gth), sp))
            xsum(gu)
            xsum(gud)
            if ev:
                ev[len(names)].record(stream)
        return step, names

    def time_step(mesh, ud, v, outs, gth, steps, label):
        mesh.autotune(u, ud, v)
        step, nm = make_step(mesh, u, ud, v, outs, gth)
        for _ in range(args.warmup):
            step()
        mesh.sync()
        torch.cuda.synchronize()
        evs = timed_steps(step, steps, flush, stream, len(nm) + 1, label)
        return np.array([[e[j].elapsed_time(e[j + 1]) for j in range(len(nm))] for e in evs]), nm

    def phase_bytes(info_, nm):
        return [info_["stream_bytes_" + n] for n in nm]

    peak, peak_kind = peaks()

    # the isoparametric (slab) path on the same mesh: per-point h_i streamed
    ms_, ud_, v_, outs_, gth_ = make(tlfe.FP32, tlfe.PATH_SLAB)
    per_s, names_s = time_step(ms_, ud_, v_, outs_, gth_, max(3, args.steps // 2), tag + "_slab_timed")
    info_s = ms_.info
    ms_.close()
    ks = per_s.mean(axis=0)
    bytes_s = phase_bytes(info_s, names_s)
    js = int(np.argmax(ks))
    ach_s = bytes_s[js] / (ks[js] * 1e-3) / 1e9
    slab = {"kernels_ms": {n: float(t) for n, t in zip(names_s, ks)}, "ms_per_step": float(per_s.sum(axis=1).mean()),
            "kernels_gbs": {n: b / (t * 1e-3) / 1e9 for n, b, t in zip(names_s, bytes_s, ks)},
            "roofline": {"bound": "hbm", "achieved": ach_s, "peak": peak, "unit": "GB/s", "frac": ach_s / peak,
                         "traffic": ncu_traffic(pre + "slab_" + names_s[js]), "kernel": names_s[js],
                         "peak_source": peak_kind,
                         "algorithmic_bytes": bytes_s[js]}}

    # the default (affine) path: the timed step, launch schedules autotuned first
    mesh, ud, v, outs, gth = make(tlfe.FP32)
    mesh.autotune(u, ud, v)
    info = mesh.info
    step, names = make_step(mesh, u, ud, v, outs, gth)
    for _ in range(args.warmup):
        step()
    mesh.sync()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        evs = clk.timed(lambda: timed_steps(step, args.steps, flush, stream, len(names) + 1,
                                            tag + "_affine_timed"))
    barrier(world)
    st = mesh.sync()
    per = np.array([[evs[k][j].elapsed_time(evs[k][j + 1]) for j in range(len(names))]
                    for k in range(args.steps)])
    step_ms = allmax(float(per.sum(axis=1).mean()), world)
    kern_ms = per.mean(axis=0)
    units = wl.n_qp                     # this GPU's points (all of them on one GPU)
    value = full.n_qp / (step_ms * 1e-3)  # the whole body per step, at the slowest GPU's time

    # roofline of the dominant kernel: FP32 FMA roof (bound), HBM fraction beside it
    bytes_alg = phase_bytes(info, names)
    j = int(np.argmax(kern_ms))
    flops = fpq[names[j]] * units if fpq[names[j]] else None
    achieved = flops / (kern_ms[j] * 1e-3) / 1e12 if flops else None
    hbm = bytes_alg[j] / (kern_ms[j] * 1e-3) / 1e9
    alu = alu_peaks()
    roof = {"bound": "alu", "achieved": achieved, "peak": alu["fp32"], "unit": "TFLOP/s",
            "frac": achieved / alu["fp32"] if achieved else None,
            "traffic": ncu_traffic(pre + names[j]), "kernel": names[j],
            "peak_source": alu["source"],
            "algorithmic_flops": flops, "flop_per_qp": fpq[names[j]],
            "algorithmic_bytes": bytes_alg[j], "hbm_achieved_gbs": hbm, "hbm_peak_gbs": peak,
            "hbm_frac": hbm / peak, "hbm_peak_source": peak_kind}
    # the same kernels against HBM by the minimum-traffic byte count with
    # streamed reference gradients (what the slab path moves); the affine
    # path forms those gradients instead of reading them
    sb = streamed_bytes(wl)
    roof["streamed_bytes"] = sb[names[j]]
    roof["streamed_hbm_frac"] = sb[names[j]] / (kern_ms[j] * 1e-3) / 1e9 / peak
    kernels_streamed_frac = {n: sb[n] / (t * 1e-3) / 1e9 / peak for n, t in zip(names, kern_ms)}

    # end to end through the C ABI with host buffers (tlfe_step_host, pinned
    # memory), copies timed: every step copies u, udot and v in and f, K v,
    # g_u, g_udot and g_theta out. The library alternates two device staging
    # sets and copies on two streams of its own, so each call's transfers
    # overlap its neighbours' computation; step_host_wait ends the region.
    hu, hud, hv = u.cpu().pin_memory(), ud.cpu().pin_memory(), v.cpu().pin_memory()
    hf, hy, hgu, hgud = (torch.empty(ud.shape, dtype=ud.dtype).pin_memory() for _ in range(4))
    hgth = torch.empty(gth.shape, dtype=torch.float64).pin_memory()

    def e2e_run(n):
        if itf is None:
            for _ in range(n):
                mesh.step_host(hu, hud, hv, hv, f=hf, y=hy, g_u=hgu, g_udot=hgud, g_mu_lambda=hgth,
                               a_M=0.0, a_K=1.0, a_C=1.0, stream=stream)
            mesh.step_host_wait()
            return
        # split body: the interface sums act on device arrays, so the inputs
        # are copied in, the step (with its sums) runs, and the outputs are
        # copied out, on the compute stream
        for _ in range(n):
            for d, hsrc in zip((u, ud, v), (hu, hud, hv)):
                d.copy_(hsrc, non_blocking=True)
            step()
            for hdst, d in zip((hf, hy, hgu, hgud, hgth), outs + [gth]):
                hdst.copy_(d, non_blocking=True)
        torch.cuda.synchronize()

    e2e_run(3)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps, world)
    st_e2e = mesh.sync()
    # the host copies against one device-only step on the same inputs (the
    # atomic scatter's order varies, so within the FP32 bar, not bit for bit)
    chk = [x.clone().double() for x in (hf, hy, hgu, hgud, hgth)]
    step()
    torch.cuda.synchronize()
    e2e_err = max(float((c - o.cpu().double()).abs().max() / o.cpu().double().abs().max().clamp_min(1e-300))
                  for c, o in zip(chk, outs + [gth]))
    h2d = u.numel() * 8 + 2 * ud.numel() * 4
    d2h = 4 * ud.numel() * 4 + gth.numel() * 8
    mesh.close()

    # the same step with FP64 element arithmetic (the plain path)
    m64, ud64, v64, outs64, gth64 = make(tlfe.FP64)
    per64, names64 = time_step(m64, ud64, v64, outs64, gth64, max(3, args.steps // 4), tag + "_fp64_timed")
    ms64 = float(per64.sum(axis=1).mean())
    st64 = m64.sync()
    m64.close()

    line = base_line(args, world, workload, value, UNIT, step_ms, "f32",
                     step="internal force + K_t v + C v + VJP (u, udot, mu, lambda)", n_elem=full.n_elem,
                     n_nodes=full.n_nodes, n_qp=full.n_qp, schedule="autotuned (tlfe_autotune) before the warm-up")
    if itf is not None:
        line["config"]["per_gpu"] = {"n_elem": wl.n_elem, "n_nodes": wl.n_nodes, "interface_nodes": itf.n}
    line.update({
        "kernels_ms": {n: float(t) for n, t in zip(names, kern_ms)},
        "kernels_gbs": {n: b / (t * 1e-3) / 1e9 for n, b, t in zip(names, bytes_alg, kern_ms)},
        "kernels_streamed_hbm_frac": kernels_streamed_frac,
        "phases": names,
        ("force_qps" if names[0] == "force" else "force_matvec_qps"): full.n_qp / (kern_ms[0] * 1e-3),
        "kernels_tflops": {n: fpq[n] * units / (t * 1e-3) / 1e12 if fpq[n] else None
                           for n, t in zip(names, kern_ms)},
        "roofline": roof,
        "element_path": "affine (Sec. 6 affine case: J^-1 and det J per element)",
        "patch": {"layout": "banked" if info["patch_layout"] == tlfe.PATCH_BANKED else "sorted",
                  "passes_per_quarter_warp_load": info["patch_passes"]},
        "slab_path": slab,
        "fp64_plain": {"ms_per_step": ms64, "kernels_ms": {n: float(t) for n, t in zip(names64, per64.mean(axis=0))},
                       "speedup_fp32_over_fp64": ms64 / step_ms, "device_status": st64},
        "e2e": {"value": full.n_qp / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": ("tlfe_step_host (C ABI, host buffers)" if itf is None else
                         "pinned-host copies around the device calls and interface sums"),
                "overlap": OVERLAP,
                "max_rel_diff_vs_device_step": e2e_err, "device_status": st_e2e},
        "gpu_launches": len(names) * args.steps,
        "clocks": clk.summary(),
        "device_status": st})
    return line, wl


# ---------------------------------------------------------------------------
# workload: newton (batched graph-captured FP32 step vs plain FP64 per body)
# ---------------------------------------------------------------------------

def run_newton(args, rank, world):
    import numpy as np
    import torch

    import synth
    from paper_2602_17002_gb300 import tlfe
    full = build_workload("newton")
    wl = full
    if world > 1:   # this GPU's bodies (cost-based bin packing); the bodies do not interact
        wl, _ = shard_bodies(full, rank, world)
    h = 1e-3
    kw = dict(gravity=GRAVITY, newton_rtol=1e-8, cg_rtol=1e-4, max_newton=20, max_cg=4000)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32, scatter=scatter_mode(args))   # the batched step
    z = torch.zeros((wl.n_nodes, 3), dtype=torch.float64, device="cuda")
    fx = torch.from_numpy(wl.fixed).cuda()
    mesh.autotune(z, None, torch.zeros((wl.n_nodes, 3), dtype=torch.float32, device="cuda"))
    v_out = torch.empty_like(z)
    reps = []

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        _, rep = mesh.newton_step(z, z, h, fixed=fx, use_graph=True, v_out=v_out, **kw)
        if ev:
            ev[1].record(stream)
        reps.append(rep)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        evs = clk.timed(lambda: timed_steps(step, args.steps, flush, stream))
    barrier(world)
    ms = allmax(float(np.mean([e[0].elapsed_time(e[1]) for e in evs])), world)
    rep = reps[-1]
    v_b = v_out.cpu().numpy()

    # e2e: state from pinned host memory, velocity back to the host
    hz = z.cpu().pin_memory()
    hv = torch.empty_like(hz).pin_memory()
    du, dv = torch.empty_like(z), torch.empty_like(z)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        du.copy_(hz, non_blocking=True)
        dv.copy_(hz, non_blocking=True)
        mesh.newton_step(du, dv, h, fixed=fx, use_graph=True, v_out=v_out, **kw)
        hv.copy_(v_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps, world)
    # one more, untimed step through the host-driven loop (the same kernels,
    # launched one by one) in its own NVTX range: kernel-level profilers do
    # not see inside a graph with conditional nodes
    torch.cuda.nvtx.range_push("newton_host_step")
    mesh.newton_step(z, z, h, fixed=fx, use_graph=False, v_out=v_out, **kw)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    mesh.close()

    # plain path: the FP64 library, one body at a time, host-driven Newton/CG loop
    bodies = synth.split_bodies(wl)
    plain = []
    for b in bodies:
        mb = tlfe.Mesh.from_workload(b, precision=tlfe.FP64)
        zb = torch.zeros((b.n_nodes, 3), dtype=torch.float64, device="cuda")
        plain.append((mb, zb, torch.from_numpy(b.fixed).cuda(), torch.empty_like(zb)))

    def plain_step():
        out = []
        for mb, zb, fb, vb in plain:
            _, r = mb.newton_step(zb, zb, h, fixed=fb, use_graph=False, v_out=vb, **kw)
            out.append(r)
        return out

    plain_step()                                   # warm-up (per-body kernels and workspaces)
    torch.cuda.synchronize()
    flush.zero_()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    p0.record(stream)
    preps = plain_step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_plain = allmax(p0.elapsed_time(p1), world)
    wall_plain = (time.perf_counter() - t0) * 1e3
    v_p = np.concatenate([vb.cpu().numpy() for _, _, _, vb in plain])
    for mb, *_ in plain:
        mb.close()
    dv_rel = float(np.abs(v_b - v_p).max() / max(np.abs(v_p).max(), 1e-300))

    line = base_line(args, world, "newton", 1e3 / ms, "steps/s", ms, "f32",
                     n_bodies=full.n_bodies, n_elem=full.n_elem, n_nodes=full.n_nodes,
                     step="one backward-Euler step of all bodies from rest (h = 1e-3 s, gravity, x = 0 clamped)")
    line.update({
        "batched": {"ms_per_step": ms, "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"],
                    "rel_residual": rep["rel_residual"], "bodies_converged": rep["n_bodies_converged"],
                    "status": rep["status"],
                    "precision": "FP32 element kernels and CG vectors (dots: double-float per thread, FP64 per "
                                 "chunk and body), FP64 residual and update",
                    "graph": True},
        "plain_fp64": {"ms_per_step": ms_plain, "host_wall_ms": wall_plain,
                       "newton_iters_max": max(r["newton_iters"] for r in preps),
                       "cg_iters_sum": int(sum(r["cg_iters"] for r in preps)),
                       "rel_residual_max": max(r["rel_residual"] for r in preps),
                       "bodies_converged": int(sum(r["status"] == 0 for r in preps)),
                       "precision": "FP64 everywhere", "graph": False, "schedule": "one body at a time"},
        "speedup_batched_over_plain": ms_plain / ms,
        "max_rel_diff_v": dv_rel,
        "e2e": {"value": 1e3 / e2e_ms, "unit": "steps/s", "h2d_bytes_per_step": 2 * z.numel() * 8,
                "d2h_bytes_per_step": z.numel() * 8, "ms_per_step": e2e_ms},
        "gpu_launches": None,
        "gpu_launches_note": "graph replays; the kernel count follows the Newton/CG iteration counts",
        "clocks": clk.summary()})
    return line, wl


# ---------------------------------------------------------------------------
# workload: batch (512 uneven bodies, graph-captured force + K v)
# ---------------------------------------------------------------------------

def run_batch(args, rank, world):
    import numpy as np
    import torch

    from paper_2602_17002_gb300 import tlfe
    full = build_workload("batch", args.bodies)
    wl = full
    if world > 1:   # this GPU's bodies (cost-based bin packing); no exchange
        wl, _ = shard_bodies(full, rank, world)
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32, scatter=scatter_mode(args))
    info = mesh.info
    u = torch.from_numpy(wl.u).to("cuda", torch.float64)
    v = torch.from_numpy(wl.v).to("cuda", torch.float32)
    f, y = torch.empty_like(v), torch.empty_like(v)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # schedules by measurement: per pass and CTA size, and the fused launch
    # (one persistent launch per operation over every pass) against the
    # per-pass launches; then the timed step is the library's own graph of
    # force + K v (tlfe_force_matvec: captured on the first call, replayed)
    mesh.autotune(u, None, v)
    info = mesh.info
    mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0, f=f, y=y)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        mesh.force_matvec(u, None, v, 0.0, 1.0, 0.0, f=f, y=y)
        if ev:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        evs = clk.timed(lambda: timed_steps(step, args.steps, flush, stream, label="batch_timed"))
    barrier(world)
    st = mesh.sync()
    ms = allmax(float(np.mean([e[0].elapsed_time(e[1]) for e in evs])), world)
    # the same step in each launch mode (the tuner keeps the faster one per
    # operation in the timed step above)
    modes = {}
    for name, mode in (("fused", tlfe.LAUNCH_FUSED), ("per_pass", tlfe.LAUNCH_PER_PASS)):
        mesh.set_launch_mode(mode)
        for _ in range(2):
            step()
        evs_m = timed_steps(step, max(3, args.steps // 2), flush, stream, label="batch_" + name)
        modes[name] = {"ms_per_step": float(np.mean([e[0].elapsed_time(e[1]) for e in evs_m])),
                       "launches_per_step": step_launches(mesh.info)}
    mesh.set_launch_mode(tlfe.LAUNCH_AUTO)
    units = wl.n_qp
    peak, peak_kind = peaks()
    b_alg = info["stream_bytes_force"] + info["stream_bytes_matvec"]
    hbm = b_alg / (ms * 1e-3) / 1e9
    # every block is affine and ALU-bound (about 26 FLOP per streamed byte,
    # above the FP32 ridge): FP32 FMA roof, HBM beside it
    one_pass = bool(info["force_matvec_fused"])   # force and K v in one pass per block and law
    if one_pass:
        b_alg = info["stream_bytes_force_matvec"]
        hbm = b_alg / (ms * 1e-3) / 1e9
    flops = 0.0
    for b in wl.blocks:
        laws = np.asarray(wl.model)[b.body]
        for law in (0, 1):
            f_qp = FLOP_PER_QP_BATCH[(b.etype, law)]
            per = f_qp.get("force_matvec") if one_pass else f_qp["force"] + f_qp["matvec"]
            flops = None if (flops is None or per is None) else flops + int((laws == law).sum()) * b.nq * per
    achieved = flops / (ms * 1e-3) / 1e12 if flops else None
    # e2e through the C ABI with host buffers (tlfe_step_host): u and v in,
    # f and K v out, every step; the library overlaps each call's transfers
    # with its neighbours' computation
    hu, hv = u.cpu().pin_memory(), v.cpu().pin_memory()
    hf, hy = torch.empty_like(hv).pin_memory(), torch.empty_like(hv).pin_memory()

    def e2e_run(n):
        for _ in range(n):
            mesh.step_host(hu, None, hv, None, f=hf, y=hy, a_M=0.0, a_K=1.0, a_C=0.0, stream=stream)
        mesh.step_host_wait()

    e2e_run(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps, world)
    types = {0: "T4", 1: "T10", 2: "H8"}
    line = base_line(args, world, "batch", full.n_qp / (ms * 1e-3), UNIT, ms, "f32",
                     n_bodies=full.n_bodies, n_elem=full.n_elem, n_nodes=full.n_nodes, n_qp=full.n_qp,
                     elements_by_type={types[b.etype]: b.n_elem for b in full.blocks},
                     step="internal force + K v over all bodies, one replay of the library's CUDA graph "
                          "(tlfe_force_matvec)")
    if full.n_bodies != 512:
        line["config"]["workload"] = WORKLOADS["batch"].replace("512 bodies", f"{full.n_bodies} bodies")
    if world > 1:
        line["config"]["per_gpu"] = {"n_bodies": wl.n_bodies, "n_elem": wl.n_elem, "n_qp": wl.n_qp}
    line.update({
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peaks()["fp32"], "unit": "TFLOP/s",
                     "frac": achieved / alu_peaks()["fp32"] if achieved else None,
                     "traffic": ncu_traffic("batch512_step") if wl.n_bodies == 512 and world == 1 else None,
                     "kernel": ("force + matvec in one pass per block and law (one step)" if one_pass else
                                "force + matvec, all element blocks (one step)"),
                     "peak_source": alu_peaks()["source"],
                     "algorithmic_flops": flops, "algorithmic_bytes": b_alg, "hbm_achieved_gbs": hbm,
                     "hbm_peak_gbs": peak, "hbm_frac": hbm / peak, "hbm_peak_source": peak_kind},
        "e2e": {"value": full.n_qp / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": u.numel() * 8 + v.numel() * 4, "d2h_bytes_per_step": 2 * v.numel() * 4,
                "call": "tlfe_step_host (C ABI, host buffers)", "overlap": OVERLAP},
        "launch": {"force": "fused" if info["launches_force"] == 1 else "per pass",
                   "matvec": "fused" if info["launches_matvec"] == 1 else "per pass",
                   "force_matvec_one_pass": one_pass,
                   "chosen_by": "tlfe_autotune (the faster mode per operation)",
                   "fused_passes": info["n_fused_passes"], "fused_items": info["n_fused_items"],
                   "passes": info["n_passes"], "launches_per_step": step_launches(info),
                   "graph": "tlfe_force_matvec (captured by the library, replayed)", "modes": modes},
        "gpu_launches": step_launches(info) * args.steps,
        "clocks": clk.summary(), "device_status": st})
    mesh.close()
    return line, wl


# ---------------------------------------------------------------------------
# workload: diff (forward + VJP through torch.autograd)
# ---------------------------------------------------------------------------

def run_diff(args, rank, world):
    import numpy as np
    import torch

    from paper_2602_17002_gb300 import autograd, tlfe
    full = build_workload("diff")
    wl, itf, theta_t = full, None, full.extra["theta_target"]
    xs32 = xs64 = None
    owned = None
    if world > 1:
        # this GPU's slab: the forward force is summed over the GPUs at the
        # interface nodes (and, by the adjoint of that sum, so is the loss
        # gradient); the loss counts every node once; the position and
        # velocity gradients are summed at the interface after the backward
        from paper_2602_17002_gb300 import shard
        wl, itf, emask = shard_one_body(full, rank, world)
        theta_t = full.extra["theta_target"][emask[0]]
        xs32 = shard.InterfaceSum(itf, torch.float32, "cuda")
        xs64 = shard.InterfaceSum(itf, torch.float64, "cuda")
        owned = torch.from_numpy(shard.owned_rows(wl.n_nodes, itf)).cuda()
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32, scatter=scatter_mode(args))
    info = mesh.info
    u = torch.from_numpy(wl.u).to("cuda", torch.float64).requires_grad_(True)
    ud = torch.from_numpy(wl.udot).to("cuda", torch.float32).requires_grad_(True)
    theta = torch.from_numpy(wl.elem_mu_lambda).to("cuda", torch.float64).requires_grad_(True)
    mesh.autotune(u.detach(), ud.detach(), ud.detach())

    def force(uu, vv, th):
        f = autograd.internal_force(mesh, uu, vv, th)
        return f if xs32 is None else autograd.interface_sum(f, xs32)

    def loss_of(f):
        r2 = (f.double() - f_t) ** 2
        return 0.5 * (r2.sum() if owned is None else r2[owned].sum())

    def finish_grads(uu, vv):
        if xs64 is not None:
            xs64(uu.grad)
            xs32(vv.grad)

    # f_target from the perturbed parameter field, computed once by the library
    with torch.no_grad():
        f_t = force(u, ud, torch.from_numpy(theta_t).cuda()).double()
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    losses = []

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        for t in (u, ud, theta):
            t.grad = None
        f = force(u, ud, theta)
        loss = loss_of(f)
        if ev:
            ev[1].record(stream)
        loss.backward()
        finish_grads(u, ud)
        if ev:
            ev[2].record(stream)
        losses.append(loss.detach())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        evs = clk.timed(lambda: timed_steps(step, args.steps, flush, stream, 3))
    barrier(world)
    st = mesh.sync()
    ms = allmax(float(np.mean([e[0].elapsed_time(e[2]) for e in evs])), world)
    ms_fwd = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    ms_bwd = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    units = wl.n_qp                     # this GPU's points
    peak, peak_kind = peaks()
    # roofline of the longer half, the backward (the adjoint kernel plus the
    # loss gradient, a few elementwise torch kernels): FP32 FMA roof, HBM beside
    fpq = FLOP_PER_QP["beam"]    # T10 Q5 neo-Hookean + Kelvin-Voigt, as the beam
    flops = fpq["vjp"] * units
    achieved = flops / (ms_bwd * 1e-3) / 1e12
    b_bwd = info["stream_bytes_vjp"]
    hbm = b_bwd / (ms_bwd * 1e-3) / 1e9

    # end to end: u, udot and the parameters from pinned host memory, the
    # loss and the three gradients back to the host, every step. Copies run on
    # their own streams: the next step's inputs come in while a step computes
    # (two sets of leaf tensors), the gradients go out when its backward ends
    hu, hud, hth = (t.detach().cpu().pin_memory() for t in (u, ud, theta))
    hgu, hgud, hgth = (torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (u, ud, theta))
    hloss = torch.empty((), dtype=torch.float64).pin_memory()
    leaves = [tuple(t.detach().clone().requires_grad_(True) for t in (u, ud, theta)) for _ in range(2)]
    h2d_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_run(n):
        in_ready, comp_done, out_done = [torch.cuda.Event(), torch.cuda.Event()], [None, None], [None, None]

        def h2d(b):
            if comp_done[b] is not None:
                h2d_s.wait_event(comp_done[b])          # the last step that read these leaves has ended
            with torch.cuda.stream(h2d_s), torch.no_grad():
                for d, h in zip(leaves[b], (hu, hud, hth)):
                    d.copy_(h, non_blocking=True)
            in_ready[b].record(h2d_s)

        h2d(0)
        for k in range(n):
            b = k & 1
            stream.wait_event(in_ready[b])
            if out_done[b] is not None:
                stream.wait_event(out_done[b])
            lu, lud, lth = leaves[b]
            for t in leaves[b]:
                t.grad = None
            f = force(lu, lud, lth)
            loss = loss_of(f)
            loss.backward()
            finish_grads(lu, lud)
            comp_done[b] = torch.cuda.Event()
            comp_done[b].record(stream)
            if k + 1 < n:
                h2d(b ^ 1)
            res = [t.grad for t in leaves[b]] + [loss.detach()]
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(comp_done[b])
                for h, g in zip((hgu, hgud, hgth, hloss), res):
                    h.copy_(g, non_blocking=True)
                    g.record_stream(d2h_s)                # kept alive until the copy has run
            out_done[b] = torch.cuda.Event()
            out_done[b].record(d2h_s)
        for o in out_done:
            if o is not None:
                stream.wait_event(o)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d_s.wait_event(e0)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps, world)
    h2d = sum(t.numel() * t.element_size() for t in (hu, hud, hth))
    d2h = sum(t.numel() * t.element_size() for t in (hgu, hgud, hgth)) + 8

    line = base_line(args, world, "diff", full.n_qp / (ms * 1e-3), UNIT, ms, "f32",
                     n_elem=full.n_elem, n_nodes=full.n_nodes, n_qp=full.n_qp,
                     step="autograd forward (tlfe_internal_force) + loss in torch + backward (tlfe_vjp)")
    line.update({
        "phases_ms": {"forward_and_loss": ms_fwd, "backward": ms_bwd},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peaks()["fp32"], "unit": "TFLOP/s",
                     "frac": achieved / alu_peaks()["fp32"], "traffic": None,
                     "kernel": "backward: tlfe_vjp (+ the loss gradient)",
                     "peak_source": alu_peaks()["source"],
                     "algorithmic_flops": flops, "flop_per_qp": fpq["vjp"], "algorithmic_bytes": b_bwd,
                     "hbm_achieved_gbs": hbm, "hbm_peak_gbs": peak, "hbm_frac": hbm / peak,
                     "hbm_peak_source": peak_kind},
        "loss": allsum(float(losses[-1].item()), world),
        "e2e": {"value": full.n_qp / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "overlap": OVERLAP},
        "gpu_launches": 2 * args.steps, "clocks": clk.summary(), "device_status": st})
    mesh.close()
    return line, wl


def cpu_baseline(workload, wl, unit, n_sample, single_core=True):
    """The oracle on a bounded sample of the workload on all host cores
    (spawned processes over element ranges), with the one-core time of the
    same sample beside it; the Newton sample (one body) on one core."""
    if workload == "diff":
        wl.v = diff_cotangent(wl)
    base = None
    if single_core or workload == "newton":
        val, secs, thr, what = cpu_sample(workload, wl, n_sample)
        base = {"value": val, "unit": unit, "cores": thr, "kind": "oracle", "sample": what}
    pool_info = oracle_pool(workload, wl, n_sample)
    if not pool_info:
        return base
    try:
        cpu_sample_parallel(workload, wl, pool_info)   # warm-up
        pv, ps, procs, pwhat = cpu_sample_parallel(workload, wl, pool_info)
    finally:
        pool_info[0].close()
        pool_info[0].join()
    out = {"value": pv, "unit": unit, "cores": procs, "kind": "oracle", "sample": pwhat}
    if base:
        out["single_core"] = base
    return out


def parse_args(ap, argv=None):
    """Parse the command line; with --case FILE the file's JSON object gives
    option defaults first (unknown keys and values of the wrong kind are
    errors), so that flags on the command line take precedence."""
    pre = argparse.ArgumentParser(add_help=False)
    pre.add_argument("--case", default=None)
    known, _ = pre.parse_known_args(argv)
    if known.case:
        with open(known.case) as fh:
            case = json.load(fh)
        if not isinstance(case, dict):
            ap.error(f"--case {known.case}: expected a JSON object")
        acts = {a.dest: a for a in ap._actions if a.dest not in ("help", "case")}
        for k, v in case.items():
            key = k.replace("-", "_")
            if key not in acts:
                ap.error(f"--case {known.case}: unknown option {k!r}")
            a = acts[key]
            if a.choices is not None and v not in a.choices:
                ap.error(f"--case {known.case}: {k} = {v!r} is not one of {sorted(a.choices)}")
            if a.type is not None and v is not None and not isinstance(v, bool):
                try:
                    v = a.type(v)
                except (TypeError, ValueError):
                    ap.error(f"--case {known.case}: {k} = {v!r} is not a valid {a.type.__name__}")
            ap.set_defaults(**{key: v})
    return ap.parse_args(argv)


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tlfe", choices=["tlfe", "reference"])
    ap.add_argument("--workload", default="beam", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-sample", type=int, default=10000, help="elements per reference-arm step")
    ap.add_argument("--cpu-sample", type=int, default=40000, help="elements in the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bodies", type=int, default=512, help="bodies in the batch workload (512 = the benchmark)")
    ap.add_argument("--scatter", default="atomic", choices=["atomic", "colour", "sorted"],
                    help="element scatter of the meshes (of the batched step for newton): atomic adds, "
                         "deterministic colour passes, or deterministic node-ordered partial sums")
    ap.add_argument("--log", default=None, help="also append the JSON line to this file (JSON lines)")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: skip the batch, Newton and differentiation sub-measurements")
    ap.add_argument("--sub-steps", type=int, default=5, help="timed steps of each sub-measurement")
    ap.add_argument("--sub-cpu-sample", type=int, default=12000,
                    help="elements in the sub-measurements' cpu_baseline samples")
    ap.add_argument("--case", default=None,
                    help="JSON file of option values (keys: the long option names without the leading dashes, e.g. "
                         '{"workload": "batch", "scatter": "sorted", "steps": 10}); options given on the '
                         "command line override it")
    return ap


def main():
    args = parse_args(make_parser())
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    rank, world, _ = dist_setup()
    runs = {"beam": run_beam, "newton": run_newton, "batch": run_batch, "diff": run_diff,
            "q27": lambda a, r, w: run_beam(a, r, w, "q27")}
    line, wl = runs[args.workload](args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, wl, line["unit"], args.cpu_sample)
    if args.workload == "beam" and not args.headline_only:
        # the other benchmark configurations of the step, each measured here
        # with its own clocks, roofline and CPU baseline, at fewer steps
        sub_args = argparse.Namespace(**vars(args))
        sub_args.steps = max(3, min(args.steps, args.sub_steps))
        sub_args.warmup = 3
        line["configs"] = {}
        for name in ("batch", "newton", "diff"):
            sl, swl = runs[name](sub_args, rank, world)
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                sl["cpu_baseline"] = cpu_baseline(name, swl, sl["unit"], args.sub_cpu_sample, single_core=False)
            sl.pop("metric", None)
            sl.pop("data", None)
            line["configs"][name] = sl
            del swl
        line["gpu_launches"] = line["gpu_launches"] + sum(
            (c.get("gpu_launches") or 0) for c in line["configs"].values())
        line["gpu_launches_note"] = ("element, node-sum and probe kernels of the headline and the configs' timed "
                                     "regions; the Newton step's graph launches follow its iteration counts")
    if args.scatter != "atomic":
        line["config"]["scatter"] = args.scatter + (" (batched step; the plain FP64 path stays atomic)"
                                                    if args.workload == "newton" else "")
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.log:
            with open(args.log, "a") as fh:
                fh.write(json.dumps(dict(line, argv=sys.argv[1:], time=time.strftime("%Y-%m-%dT%H:%M:%S"))) + "\n")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
