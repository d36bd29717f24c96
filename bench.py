"""Benchmark of the TL-FEA hot path on GB300.

Workload: the 10 x 1 x 1 m cantilever beam, 200 x 20 x 20 cells split into
480,000 Kuhn T10 tetrahedra (674,081 nodes), 5-point quadrature,
compressible neo-Hookean (mu = 3.8e6, lambda = 5.8e6 Pa) with Kelvin-Voigt
damping (mu_v = 1e3 Pa s), seeded bending field + 0.1 % noise, seeded
velocities; FP32 element arithmetic.

One step = one pass of the element hot path over the beam:
  internal force f(u, udot)                       (tlfe_internal_force)
  full tangent product y = K_t v + C v            (tlfe_tangent_matvec)
  adjoint g_u, g_udot, g_(mu, lambda) of f . r    (tlfe_vjp)
value = quadrature points processed through that pass per second (whole job).

L2 is flushed (a 512 MiB memset) before every timed step, outside the step's
CUDA-event pair; ms_per_step is the mean of the per-step event times.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload on the host cores (the reference arm of this build).
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
WORKLOAD = "cantilever beam 10x1x1 m, 200x20x20 cells -> 480k T10 (674,081 nodes), Q=5, neo-Hookean + Kelvin-Voigt, FP32"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_17002_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode() + fh.read())
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
    """nvidia-smi samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample_oracle(wl, n_elem_sample):
    """Time the oracle (force + closed-form tangent product + adjoint) on the
    first n_elem_sample elements of the workload; returns (qp/s, seconds, threads)."""
    import numpy as np
    import oracle
    from synth.workloads import Block, Workload
    blk = wl.blocks[0]
    sub = Workload("sample", wl.X, [Block(blk.etype, blk.nq, blk.conn[:n_elem_sample], blk.body[:n_elem_sample])],
                   wl.model, wl.params, u=wl.u, udot=wl.udot, v=wl.v)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.internal_force(sub)
    oracle.operator_apply(sub, wl.v, a_K=1.0, a_C=1.0)
    oracle.vjp(sub, wl.v)
    dt = time.perf_counter() - t0
    return n_elem_sample * blk.nq / dt, dt, 1


def dist_setup(n_gpus):
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
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """CPU oracle arm: rank 0 only; each step a bounded sample of the beam."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import synth
    wl = synth.cantilever_beam()
    n_s = args.ref_sample
    for _ in range(max(0, args.warmup)):
        cpu_sample_oracle(wl, max(64, n_s // 8))
    ts = []
    for _ in range(args.steps):
        q, dt, thr = cpu_sample_oracle(wl, n_s)
        ts.append(dt)
    t = float(np.mean(ts))
    value = n_s * 5 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: first %d elements per step)" % n_s},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {n_s} of 480,000 elements (force + closed-form K_t v + C v + adjoint)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tlfe", choices=["tlfe", "reference"])
    ap.add_argument("--ref-sample", type=int, default=3000)
    ap.add_argument("--cpu-sample", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import synth
    from paper_2602_17002_gb300 import tlfe

    rank, world, local = dist_setup(args.gpus)
    wl = synth.cantilever_beam()
    mesh = tlfe.Mesh.from_workload(wl, precision=tlfe.FP32)
    info = mesh.info
    dt = torch.float32
    u = torch.from_numpy(wl.u).to("cuda", torch.float64)   # displacement state: FP64 in both precisions
    ud = torch.from_numpy(wl.udot).to("cuda", dt)
    v = torch.from_numpy(wl.v).to("cuda", dt)
    f = torch.empty_like(ud)
    y = torch.empty_like(ud)
    gu = torch.empty_like(ud)
    gud = torch.empty_like(ud)
    gth = torch.empty((wl.n_elem, 2), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    L = tlfe.load()
    stream = torch.cuda.current_stream()
    sp = tlfe._stream(stream)
    h = mesh.handle

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        tlfe._check(L.tlfe_internal_force(h, tlfe._ptr(u), tlfe._ptr(ud), tlfe._ptr(f), sp))
        if ev:
            ev[1].record(stream)
        tlfe._check(L.tlfe_tangent_matvec(h, tlfe._ptr(u), tlfe._ptr(ud), tlfe._ptr(v), 0.0, 1.0, 1.0,
                                          tlfe._ptr(y), sp))
        if ev:
            ev[2].record(stream)
        tlfe._check(L.tlfe_vjp(h, tlfe._ptr(u), tlfe._ptr(ud), tlfe._ptr(v), tlfe._ptr(gu), tlfe._ptr(gud),
                               tlfe._ptr(gth), sp))
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    mesh.sync()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            flush.zero_()
            step(evs[k])
        torch.cuda.synchronize()
    barrier(world)
    st = mesh.sync()
    per = np.array([[evs[k][j].elapsed_time(evs[k][j + 1]) for j in range(3)] for k in range(args.steps)])
    step_ms = float(per.sum(axis=1).mean())
    step_ms_max = allmax(step_ms, world)
    kern_ms = per.mean(axis=0)
    units = wl.n_qp
    value = world * units / (step_ms_max * 1e-3)

    # roofline of the dominant kernel
    names = ["force", "matvec", "vjp"]
    bytes_alg = [info["stream_bytes_force"], info["stream_bytes_matvec"], info["stream_bytes_vjp"]]
    j = int(np.argmax(kern_ms))
    peak, peak_kind = peaks()
    achieved = bytes_alg[j] / (kern_ms[j] * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic(names[j]), "kernel": names[j], "peak_source": peak_kind,
            "algorithmic_bytes": bytes_alg[j]}

    # end to end through the public API with host buffers (pinned), copies timed
    hu = u.cpu().pin_memory()
    hud = ud.cpu().pin_memory()
    hv = v.cpu().pin_memory()
    hf, hy, hgu, hgud = (torch.empty(ud.shape, dtype=dt).pin_memory() for _ in range(4))
    hgth = torch.empty(gth.shape, dtype=torch.float64).pin_memory()
    du, dud, dv = torch.empty_like(u), torch.empty_like(ud), torch.empty_like(ud)

    def e2e_step():
        du.copy_(hu, non_blocking=True)
        dud.copy_(hud, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        tlfe._check(L.tlfe_internal_force(h, tlfe._ptr(du), tlfe._ptr(dud), tlfe._ptr(f), sp))
        tlfe._check(L.tlfe_tangent_matvec(h, tlfe._ptr(du), tlfe._ptr(dud), tlfe._ptr(dv), 0.0, 1.0, 1.0,
                                          tlfe._ptr(y), sp))
        tlfe._check(L.tlfe_vjp(h, tlfe._ptr(du), tlfe._ptr(dud), tlfe._ptr(dv), tlfe._ptr(gu), tlfe._ptr(gud),
                               tlfe._ptr(gth), sp))
        hf.copy_(f, non_blocking=True)
        hy.copy_(y, non_blocking=True)
        hgu.copy_(gu, non_blocking=True)
        hgud.copy_(gud, non_blocking=True)
        hgth.copy_(gth, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps, world)
    h2d = u.numel() * 8 + 2 * ud.numel() * 4
    d2h = 4 * u.numel() * 4 + gth.numel() * 8

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "internal force + K_t v + C v + VJP (u, udot, mu, lambda)",
                       "n_elem": wl.n_elem, "n_nodes": wl.n_nodes, "n_qp": units,
                       "l2": "flushed (512 MiB memset) before every step, outside the timed events",
                       "parallelism": f"replicas x{world} (one independent beam per GPU)"},
            "kernels_ms": {n: float(t) for n, t in zip(names, kern_ms)},
            "kernels_gbs": {n: b / (t * 1e-3) / 1e9 for n, b, t in zip(names, bytes_alg, kern_ms)},
            "force_qps": units / (kern_ms[0] * 1e-3),
            "roofline": roof,
            "e2e": {"value": world * units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": 3 * args.steps,
            "clocks": clk.summary(),
            "device_status": st}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        q, secs, thr = cpu_sample_oracle(wl, args.cpu_sample)
        line["cpu_baseline"] = {"value": q, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"first {args.cpu_sample} of {wl.n_elem} elements, force + closed-form "
                                          f"K_t v + C v + adjoint, {secs:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    mesh.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
