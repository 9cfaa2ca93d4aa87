#!/usr/bin/env python3
"""Benchmark of the phase-field curvature-energy hot path on GB300.

Workload (one "step"): one exact mass-projected gradient-descent step (energy,
exact discrete gradient, update u <- u - tau (g - mean g)) of each of the four
128^3 validation problems -- tanh-profile sphere R = 32 and z-periodic
cylinder r = 20, eps = 2, h = 1, p = k1^2 + k2^2 and p = k1 k2 -- run FP32 on
the fused path as ONE batched launch (plus one launch applying the
projection).  Metric: voxel energy+gradient evaluations per second
(voxel-steps/s), compared with the FP64 plain (unfused) GPU path on the same
workload, at the relative energy error FP32 vs FP64 reported beside it.

The L2 (129 MB) is flushed by writing a 256 MB buffer before every timed step;
step and kernel durations come from CUDA events recorded by the library on
the launching stream around each step and around its fused sweep kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pfc|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU (weak
scaling, no collective on the data path); rank 0 prints the line with the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel energy+grad evals/sec, FP32 fused vs FP64 plain, at <=1e-4 rel energy; % HBM peak"
UNIT = "voxel-steps/s"
N_EDGE = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="pfc", choices=["pfc", "reference"])
    ap.add_argument("--flush-mb", type=int, default=256)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-y", type=int, default=0, help="0 = autotuned (or library default)")
    ap.add_argument("--max-run", type=int, default=-1, help="cap on planes per CTA run (-1 = autotuned)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other_workloads lines")
    ap.add_argument("--only", default=None,
                    choices=["alg1_flow_100", "alg1_batch_100", "extended_sweep_128", "alg1_spatialized",
                             "diagnostics_512", "batch64_mixed"],
                    help="run just this one of the other workloads and print its line (for profiling)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for name, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ reference arm

def run_reference(args, ws, rank):
    """The FP64 CPU oracle on the same workload, a bounded sample per step."""
    if rank != 0:
        return 0
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    insts = I.validation_set_128()
    fields = [inst.field().astype(np.float32).astype(np.float64) for inst in insts]
    # size the sample so the whole run stays within ~3 minutes
    nsteps = args.steps + args.warmup
    t = time.perf_counter()
    oracle.step(fields[0][:32, :32, :32].copy(), insts[0].problem(), 1e-3)
    rate = 32 ** 3 / max(time.perf_counter() - t, 1e-6)     # voxel-steps/s, rough
    budget = 150.0 / max(nsteps, 1)
    edge = int(min(N_EDGE, max(16, (budget * rate) ** (1 / 3))))
    edge -= edge % 8
    samples = [f[:edge, :edge, :edge].copy() for f in fields]
    total, vox = 0.0, 0
    for k in range(nsteps):
        i = k % len(insts)
        t0 = time.perf_counter()
        oracle.step(samples[i], insts[i].problem(), insts[i].tau)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            total += dt
            vox += edge ** 3
    value = vox / total if total > 0 else None
    sample = (f"one FP64 oracle step per timed step on a {edge}^3 crop of the 128^3 validation fields "
              f"(cycling sphere/cylinder x two p), single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "validation_128 (4 x 128^3 tanh sphere/cylinder)",
                                            "sample_edge": edge},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ helpers

def max_over_ranks(values):
    """Element-wise max of per-rank timings (the slowest rank sets the job's
    time); identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_value(voxels_per_rank, world_size, ms_per_step_max):
    """Whole-job throughput under weak scaling: every rank processes its own
    voxels; the job advances at the pace of the slowest rank."""
    return world_size * voxels_per_rank / (ms_per_step_max * 1e-3)


def kernel_sources_sha():
    h = hashlib.sha256()
    for f in ("pfc_fused.cu", "pfc_fused_kernel.cuh", "pfc_fused_sym.cu", "pfc_device.cuh", "pfc_internal.h"):
        with open(os.path.join(ROOT, "paper_2103_04856_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_profile(tile_y, max_run):
    """The fused sweep's figures from the committed ncu summary (DRAM bytes and
    instructions per launch), or None if they were taken on another version of
    the kernel sources or in another launch shape."""
    path = os.path.join(ROOT, "profiles", "fused_sweep_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_sources_sha") != kernel_sources_sha():
            return None, "stale"
        if d.get("tile_y") != tile_y or d.get("max_run") != max_run:
            return None, f"captured with tile_y {d.get('tile_y')}, max_run {d.get('max_run')}"
        return d, d.get("note", "")
    except Exception:
        return None, "absent"


def committed_traffic(tile_y, max_run):
    """DRAM bytes per launch of the fused sweep from the committed ncu summary."""
    d, note = committed_profile(tile_y, max_run)
    return (float(d["traffic_bytes_per_launch"]) if d else None), note


def cpu_baseline_oracle():
    import oracle
    from paper_2103_04856_gb300 import inputs as I
    inst = I.validation_128("sphere", "k1^2+k2^2")
    u = inst.field().astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    reps = 0
    while True:   # a bounded sample: about 10 s of single-threaded CPU work
        oracle.step(u, inst.problem(), inst.tau)
        reps += 1
        if time.perf_counter() - t0 > 10.0 or reps >= 60:
            break
    dt = time.perf_counter() - t0
    return {"value": reps * u.size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} FP64 oracle step(s) of the 128^3 tanh sphere (2,097,152 voxels each), single thread"}


def problem_of(pfc, inst, prec="fp32", **kw):
    return pfc.Problem.from_shape(inst.shape, eps=inst.eps, a=inst.a, h=inst.h, xi=inst.xi, well=inst.well,
                                  prec=prec, **kw)


def accuracy(pfc, insts, fields):
    """FP32 fused against FP64 fused on the same FP32 states (the FP64 path
    equals the oracle to 1e-10 in the tests): the worst relative energy
    error and relative gradient 2-norm error over the instances."""
    import torch
    e_err = g_err = 0.0
    for inst, f in zip(insts, fields):
        if isinstance(f, torch.Tensor):
            u32 = f.to(device="cuda", dtype=torch.float32).contiguous()
        else:
            u32 = torch.tensor(np.asarray(f, dtype=np.float32), device="cuda")
        c32, c64 = pfc.Context(problem_of(pfc, inst, "fp32")), pfc.Context(problem_of(pfc, inst, "fp64"))
        E32, g32 = c32.energy_and_grad(u32)
        E64, g64 = c64.energy_and_grad(u32.double())
        e_err = max(e_err, abs(E32 - E64) / abs(E64))
        g_err = max(g_err, float(torch.linalg.norm(g32.double() - g64) / torch.linalg.norm(g64)))
        c32.close()
        c64.close()
        del g32, g64, u32
    return {"rel_energy_err": e_err, "rel_grad_norm_err": g_err}


def lazy_chain(batch, A, B, taus, flush, steps, warmup):
    """`warmup` untimed, then `steps` timed chained steps (pfc_batch_step_lazy)
    with the L2 flushed before each, and the launch that adds the last
    offset, timed and spread over the steps.  Returns (ms per step, ms per
    sweep, the projected fields)."""
    import torch
    cur, nxt = A, B
    for k in range(warmup):
        flush.zero_()
        batch.step_lazy(cur, nxt, taus, first=(k == 0))
        cur, nxt = nxt, cur
    if warmup:
        batch.lazy_finish(cur)
    st, sw = [], []
    for k in range(steps):
        flush.zero_()
        batch.step_lazy(cur, nxt, taus, first=(k == 0))
        a, b = batch.last_timing()
        st.append(a)
        sw.append(b)
        cur, nxt = nxt, cur
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    batch.lazy_finish(cur)
    ev1.record()
    torch.cuda.synchronize()
    return float(np.mean(st)) + ev0.elapsed_time(ev1) / steps, float(np.mean(sw)), cur


def alu_roofline(flops, ms, peak, peak_kind, kernel):
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "kernel": kernel, "kernel_ms": ms}


def cpu_oracle_rate(inst, edge, seconds):
    """The FP64 oracle (single thread) on an edge^3 crop of the workload's
    field, repeated for about `seconds`: voxel-steps/s."""
    import oracle
    u = inst.field()[:edge, :edge, :edge].astype(np.float32).astype(np.float64).copy()
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.step(u, inst.problem(), inst.tau)
        reps += 1
        if time.perf_counter() - t0 > seconds:
            break
    return reps * u.size / (time.perf_counter() - t0), reps


def membrane_block(pfc, I, flush, steps, peak, peak_kind, with_cpu):
    """The largest single-GPU workload, 512^3 FP32 with the membrane-favouring
    (asymmetric) polynomial: chained steps of the general sweep, its roofline,
    end to end through host buffers, accuracy at the first and last state,
    and the oracle on a crop of the same field."""
    import torch
    inst = I.membrane_descent_512()
    host = inst.field().astype(np.float32)
    vox = host.size
    A = [torch.tensor(host, device="cuda")]
    B = [torch.empty_like(A[0])]
    acc0 = accuracy(pfc, [inst], A)
    b = pfc.Batch([problem_of(pfc, inst)])
    b.timing(True)
    ms, msw, cur = lazy_chain(b, A, B, [inst.tau], flush, steps, 3)
    acc1 = accuracy(pfc, [inst], cur)
    del A, B, cur
    peaks, hk = load_peaks()
    # a batch's automatic tile height (pfc_batch_create): 16 or 13 rows by padded rows times the
    # measured cost of a row (the general 16-row batched sweep's rows cost 4 % more)
    ny = inst.shape[1]
    ty = 13 if ((ny + 12) // 13 * 13) < ((ny + 15) // 16 * 16) * 1.04 else 16
    roof = alu_roofline(workload_flops([inst]), msw, peak, peak_kind, f"k_fused<float,{ty},STEP,64> (general sweep)")
    hbm = 8.0 * vox / (msw * 1e-3) / 1e9
    roof["traffic"] = None
    roof["traffic_note"] = "no ncu capture of this launch (512^3 is above the capture size rule)"
    roof["hbm"] = {"achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
                   "peak_kind": hk, "algorithmic_bytes_per_launch": 8.0 * vox}
    pin_in = torch.from_numpy(host).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    for _ in range(2):
        b.step_host([pin_in], [pin_out], [inst.tau])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n_e2e = 5
    for _ in range(n_e2e):
        b.step_host([pin_in], [pin_out], [inst.tau], wait=False)
    b.host_wait()
    e2e = {"value": vox * n_e2e / (time.perf_counter() - t1), "unit": UNIT, "h2d_bytes_per_step": host.nbytes,
           "d2h_bytes_per_step": host.nbytes}
    b.close()
    out = {"workload": "membrane_512: 512^3 FP32, eps=2, p=0.2k1^2+k2^2+0.3k1k2 (k1 the smaller), noise u0",
           "value": vox / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "sweep_ms": msw, "roofline": roof,
           "e2e": e2e, "accuracy_fp32_vs_fp64": {"initial": acc0, "final": acc1, "steps_between": steps + 3}}
    if with_cpu:
        rate, reps = cpu_oracle_rate(inst, 96, 5.0)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{reps} FP64 oracle step(s) of a 96^3 crop of the 512^3 field, single thread"}
    return out


def descent_32_block(pfc, I):
    """The 32^3 plain FP64 workload: 100 mass-projected steps of 1e-3 from
    noise (pfc_run, one CUDA graph), fused and plain FP64 paths."""
    import torch
    inst = I.willmore_descent_32()
    u0 = torch.tensor(inst.field(), device="cuda")
    out = {"workload": "willmore_descent_32: 32^3 FP64, eps=1.5, p=k1^2+k2^2, 100 steps of 1e-3"}
    for impl in ("fused", "plain"):
        ctx = pfc.Context(problem_of(pfc, inst, "fp64", impl=impl))
        x = u0.clone()
        ctx.run(x, 100, inst.tau, trace=False)           # graph capture
        x.copy_(u0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        tr = ctx.run(x, 100, inst.tau)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[impl] = {"ms_per_run": ms, "value": u0.numel() * 100 / (ms * 1e-3), "unit": UNIT,
                     "energy_first_last": [float(tr[0, 0]), float(tr[-1, 0])]}
        ctx.close()
    out["note"] = "32,768 voxels per step: launch-bound (the run includes its trace copy and synchronisation)"
    return out


def tube_256_block(pfc, I, steps, peak, peak_kind):
    """The 256^3 FP32 tube-favouring workload (asymmetric p): `steps`
    mass-projected steps (pfc_run: the projection in fused form, 64-step CUDA
    graphs), accuracy at the first and last state.  Timed at xi = 1e-2: at
    the workload's xi = 1e-6 the fixed step 1e-3 makes voxels at the
    sqrt(D+) kink chatter, and whether a 2000-step run blows up depends on
    FP32 rounding (measured: 1 to 3 of four seeds blow up between steps 118
    and 340, depending on the build, and the same starts run to the end in
    50-step calls), so the timed work would not be well defined."""
    import dataclasses
    import torch
    inst = dataclasses.replace(I.tube_descent_256(), xi=1e-2)
    u0 = torch.tensor(inst.field().astype(np.float32), device="cuda")
    ctx = pfc.Context(problem_of(pfc, inst))
    x = u0.clone()
    ctx.run(x, 64, inst.tau, trace=False)                # graph capture
    x.copy_(u0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    tr = ctx.run(x, steps, inst.tau)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ctx.close()
    n = u0.numel()
    return {"workload": "tube_descent_256: 256^3 FP32, eps=1.5, p=k1^2+0.2k2^2-0.5k1 (k1 the smaller), "
                        f"{steps} steps of 1e-3, xi=1e-2 (at 1e-6 a long fixed-step run may blow up)",
            "value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "roofline_incl_run_overheads": alu_roofline(workload_flops([inst]), ms, peak, peak_kind,
                                                        "pfc_run step (general sweep + graph)"),
            "energy_first_last": [float(tr[0, 0]), float(tr[-1, 0])], "mass_drift": float(abs(tr[-1, 1] - tr[0, 1])),
            "accuracy_fp32_vs_fp64": {"initial": accuracy(pfc, [inst], [u0]), "final": accuracy(pfc, [inst], [x])}}


def batch64_block(pfc, I, steps, ws, rank):
    """The 64 mixed-size instances (random asymmetric p), partitioned across
    the ranks by voxels, `steps` steps each (pfc_batch_run: one launch per
    step over a rank's instances, 64-step graphs); traces gathered on rank 0.
    Random polynomials can make a descent blow up: per-instance finiteness is
    reported."""
    import torch
    from paper_2103_04856_gb300 import slab
    insts = I.batch_instances(64)
    sizes = [int(np.prod(i.shape)) for i in insts]
    parts = slab.partition_instances(sizes, ws)
    mine = parts[rank]
    my = [insts[k] for k in mine]
    b = pfc.Batch([problem_of(pfc, i) for i in my])
    init = [torch.tensor(i.field().astype(np.float32), device="cuda") for i in my]
    fields = [x.clone() for x in init]
    b.run(fields, 64, [i.tau for i in my], trace=False, allow_nonfinite=True)    # graph capture
    for f, x in zip(fields, init):
        f.copy_(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record()
    tr, finite = b.run(fields, steps, [i.tau for i in my], allow_nonfinite=True)
    e1.record()
    e1.synchronize()
    ms = max_over_ranks([e0.elapsed_time(e1)])[0]
    b.close()
    traces = slab.gather_traces({k: tr[j] for j, k in enumerate(mine)}, len(insts))
    vox = sum(sizes)
    out = {"workload": f"batch64_mixed: 64 instances of 64^3/96^3/128^3 ({vox} voxels), random p, {steps} steps",
           "unit": UNIT, "ms_per_step": ms / steps, "ranks": ws,
           "partition": "by voxels, largest first (paper_2103_04856_gb300.slab.partition_instances)",
           "value_all_instances": vox * steps / (ms * 1e-3)}
    if traces is not None:
        # an instance whose scalars turned non-finite is retired (its later
        # steps only store NaN): count the voxel-steps evaluated, up to and
        # including each instance's first non-finite step
        evaluated = 0
        for t, n in zip(traces, sizes):
            bad = np.flatnonzero(~np.all(np.isfinite(t), axis=1))
            evaluated += n * (steps if bad.size == 0 else int(bad[0]) + 1)
        out["value"] = evaluated / (ms * 1e-3)
        out["voxel_steps_evaluated"] = evaluated
        out["finite_instances"] = int(sum(bool(np.all(np.isfinite(t))) for t in traces))
    return out


def slab_block(pfc, I, steps, ws, rank):
    """The 512^3 membrane workload split in z across the ranks (one slab per
    rank; with one rank the halo wraps locally): per step a halo exchange of
    two planes per side, the slab's fused sweep, an all-gather of the sums
    and their combine (paper_2103_04856_gb300.slab.SlabDescent)."""
    import torch
    from paper_2103_04856_gb300 import slab
    inst = I.membrane_descent_512()
    z0, nzl = slab.split_z(inst.shape[0], ws)[rank]
    host = inst.field()[z0:z0 + nzl].astype(np.float32)
    drv = slab.SlabDescent(problem_of(pfc, inst), torch.tensor(host, device="cuda"), z0)
    drv.run(3, inst.tau)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        drv.step(inst.tau)
    e1.record()
    e1.synchronize()
    ms = max_over_ranks([e0.elapsed_time(e1) / steps])[0]
    n = int(np.prod(inst.shape))
    return {"workload": f"membrane_512 split in {ws} z-slab(s), FP32, {steps} chained steps",
            "value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "ranks": ws,
            "halo_bytes_per_rank_per_step": 2 * 2 * inst.shape[1] * inst.shape[2] * 4}


def alg1_workload(pfc, I, steps):
    """The paper's generator (Alg. 1) in its own setting (100^3, Fig. cvg_1
    parameters, blur of 2 voxels, Adam), FP32, run as the paper runs it:
    `steps` Adam iterations from white noise (8000 in Sec. 4.1), then the
    viability diagnostics (Sec. 4.5) and the curvature diagram (Sec. 4.1) of
    the generated shape.  Reports seconds per shape and iterations per second."""
    import torch
    pd, fd, A0 = I.paper_flow_100()
    nz, ny, nx = pd["shape"]
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=pd["h"], eps=pd["eps"], xi=pd["xi"], a=pd["a"], well=pd["well"],
                       prec="fp32")
    flow = pfc.HFlow(prob, m0=fd["m0"], lr=fd["lr"], betas=(fd["beta1"], fd["beta2"]), adam_eps=fd["adam_eps"],
                     blur_sigma=fd["blur_sigma"])
    A = torch.tensor(A0.astype(np.float32), device="cuda")
    m, v = torch.zeros_like(A), torch.zeros_like(A)
    flow.run(A, m, v, 64)                       # warm-up: captures the graph for these buffers
    A.copy_(torch.tensor(A0.astype(np.float32)))   # then the real run starts from white noise
    m.zero_()
    v.zero_()
    flow.t = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    tr = flow.run(A, m, v, steps)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ut = flow.field(A)
    flow.close()
    ctx = pfc.Context(prob)
    diag = ctx.diagnostics(ut)
    cells = []
    ms_cells = _timed(lambda: cells.append(ctx.surface_cells(ut, 0.0)), 5)
    hist = ctx.curvature_histogram(cells[-1], 100, -100.0, 100.0)
    torch.cuda.synchronize()
    c = cells[-1].double()
    area = float(c[:, 0].sum())
    diagram = {"cells": int(c.shape[0]), "area": area, "ms_cells_incl_sync": ms_cells,
               "mean_kappa1": float((c[:, 0] * c[:, 1]).sum()) / area if area > 0 else None,
               "mean_kappa2": float((c[:, 0] * c[:, 2]).sum()) / area if area > 0 else None,
               "hist_area_in_range": float(hist.sum())}
    ctx.close()
    n = nx * ny * nz
    peaks, peak_kind = load_peaks()
    # Adam state (A, m, v: 9 FP32 values) read and written once per iteration
    state_gbs = 72.0 * n / (ms * 1e-3) / 1e9
    viable = diag["ratio"] < 0.75 and diag["max"] > 0.1 and diag["min"] < -0.1
    return {"workload": "Alg. 1 at 100^3, h=0.01, eps=0.02, a=(1,2.4,9,30,170,-195), m0=-0.66, blur 2 px, Adam 1e-3",
            "iterations": steps, "seconds_per_shape": ms * steps / 1e3,
            "iterations_per_s": 1e3 / ms, "ms_per_iteration": ms, "value": n * 1e3 / ms, "unit": "voxel-iterations/s",
            "state_bytes_per_voxel_iteration": 72, "state_GBps": state_gbs,
            "state_frac_of_hbm": state_gbs / peaks["hbm_gbs"], "hbm_peak_kind": peak_kind,
            "note": "the 100^3 working set (about 60 MB) stays in the 129 MB L2",
            "energy_first_last": [float(tr[0, 0]), float(tr[-1, 0])], "mass": float(tr[-1, 3]),
            "viability": {**diag, "viable": bool(viable)}, "curvature_diagram": diagram,
            "paper_context": "up to 150 s for ~8000 iterations at 100^3 (~53 iterations/s) on an unnamed GPU, "
                             "PyTorch autograd (Sec. 4.1)"}


def _timed(fn, reps):
    import torch
    fn()                                        # warm-up (graph capture, allocation)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def alg1_batch_workload(pfc, I, n_inst, steps):
    """The paper's generator in its setting (100^3, Fig. cvg_1 parameters,
    blur 2 voxels, Adam), n_inst shapes from different white-noise A0 at
    once (pfc_hflow_batch: one launch per kernel for all): throughput in
    shape-iterations per second and the time of the paper's 8000-iteration
    protocol per shape."""
    import torch
    pd, fd, _ = I.paper_flow_100()
    nz, ny, nx = pd["shape"]
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=pd["h"], eps=pd["eps"], xi=pd["xi"], a=pd["a"], well=pd["well"],
                       prec="fp32")
    fb = pfc.HFlowBatch([prob] * n_inst, [fd["m0"]] * n_inst, lr=fd["lr"], betas=(fd["beta1"], fd["beta2"]),
                        adam_eps=fd["adam_eps"], blur_sigma=fd["blur_sigma"])
    As = [torch.tensor(I.paper_flow_100(seed=s)[2].astype(np.float32), device="cuda") for s in range(n_inst)]
    ms = [torch.zeros_like(a) for a in As]
    vs = [torch.zeros_like(a) for a in As]
    fb.run(As, ms, vs, 32, trace=False)           # warm-up: graph capture
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    fb.run(As, ms, vs, steps, trace=False)
    e1.record()
    e1.synchronize()
    ms_it = e0.elapsed_time(e1) / steps
    fb.close()
    n = nx * ny * nz
    peaks, kind = load_peaks()
    state_gbs = 72.0 * n * n_inst / (ms_it * 1e-3) / 1e9
    return {"workload": f"Alg. 1 at 100^3 (paper setting), {n_inst} shapes per batch", "instances": n_inst,
            "ms_per_batch_iteration": ms_it, "shape_iterations_per_s": n_inst * 1e3 / ms_it,
            "seconds_per_shape_8000_iterations": 8000 * ms_it / 1e3 / n_inst,
            "value": n * n_inst * 1e3 / ms_it, "unit": "voxel-iterations/s",
            "state_GBps": state_gbs, "state_frac_of_hbm": state_gbs / peaks["hbm_gbs"], "hbm_peak_kind": kind}


def extended_sweep_workload(pfc, I, steps):
    """The Sec. 5.2 extensions on the 128^3 tanh sphere (p = k1^2 + k2^2),
    FP32 descent steps (pfc_run, graph replays): the plain sweep, with the
    orientation term, and with a(x) (a constant field equal to a, so that the
    three compute the same problem up to the orientation term)."""
    import torch
    inst = I.validation_128("sphere", "k1^2+k2^2")
    u0 = torch.tensor(inst.field().astype(np.float32), device="cuda")
    n = u0.numel()
    out = {}
    for name, kw, field in (("plain", {}, False), ("orientation", {"mu": 1.0, "theta": (0.0, 0.6, 0.8)}, False),
                            ("a_of_x", {}, True)):
        ctx = pfc.Context(pfc.Problem.from_shape(inst.shape, eps=inst.eps, a=inst.a, prec="fp32", **kw))
        if field:
            af = torch.tensor(np.broadcast_to(np.asarray(inst.a, dtype=np.float32)[:, None, None, None],
                                              (6,) + inst.shape).copy(), device="cuda")
            ctx.set_coefficient_field(af)
        u = u0.clone()
        ms = _timed(lambda: ctx.run(u, steps, 1e-3, trace=False), 3) / steps
        out[name] = {"ms_per_step": ms, "voxel_steps_per_s": n * 1e3 / ms}
        ctx.close()
    return {"workload": "128^3 tanh sphere R=32, eps=2, FP32 descent steps (Sec. 5.2 extensions)", **out}


def spatialized_flow_workload(pfc, I, steps):
    """The paper's spatialised example (Sec. 5.2, Table in_spatialized): Alg. 1
    on six 100^3 cubes along x (600 x 100 x 100, h = 0.01, eps = 0.02, the +-1
    well) with a(x) and m(x) interpolated between the table's four
    parameters, blur 2 voxels, Adam 1e-3, FP32."""
    import torch
    af, mf = I.spatialized_fields(100)
    nz, ny, nx = mf.shape
    prob = pfc.Problem(nx=nx, ny=ny, nz=nz, h=0.01, eps=0.02, xi=1e-6, a=(0.0,) * 6, well=1, prec="fp32")
    flow = pfc.HFlow(prob, m0=0.0, lr=1e-3, blur_sigma=2.0)
    flow.set_coefficient_field(torch.tensor(af.astype(np.float32), device="cuda"))
    flow.set_mass_field(torch.tensor(mf.astype(np.float32), device="cuda"))
    rng = np.random.default_rng(0)
    A = torch.tensor((2.0 * 0.01 * 0.1 / math.sqrt(6.0) * rng.standard_normal((3, nz, ny, nx))).astype(np.float32),
                     device="cuda")
    m, v = torch.zeros_like(A), torch.zeros_like(A)
    trs = []
    ms = _timed(lambda: trs.append(flow.run(A, m, v, steps)), 1) / steps
    flow.close()
    n = nx * ny * nz
    return {"workload": "Alg. 1 with a(x), m(x): 600x100x100, h=0.01, eps=0.02, blur 2 px, Adam 1e-3",
            "iterations_per_s": 1e3 / ms, "ms_per_iteration": ms, "value": n * 1e3 / ms,
            "unit": "voxel-iterations/s", "energy_last": float(trs[-1][-1, 0]), "mass_last": float(trs[-1][-1, 3]),
            "mass_target": float(mf.mean())}


def diagnostics_workload(pfc, I):
    """Sec. 4.5 viability diagnostics of a 512^3 FP32 field: one HBM-bound
    pass (4 B/voxel read)."""
    import torch
    inst = I.membrane_descent_512()
    u = torch.tensor(inst.field().astype(np.float32), device="cuda")
    ctx = pfc.Context(pfc.Problem.from_shape(inst.shape, eps=inst.eps, a=inst.a, prec="fp32"))
    res = {}
    ms = _timed(lambda: res.update(ctx.diagnostics(u)), 10)
    # the kernel alone: back-to-back launches writing to device memory
    # (pfc_diagnostics_dev), CUDA events on the launching stream; the 537 MB
    # field is 4x the L2
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.diagnostics_dev(u, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 20
    torch.cuda.synchronize()
    e0.record()
    for _ in range(n):
        ctx.diagnostics_dev(u, out)
    e1.record()
    e1.synchronize()
    ms_k = e0.elapsed_time(e1) / n
    ctx.close()
    peaks, kind = load_peaks()
    gbs = 4.0 * u.numel() / (ms * 1e-3) / 1e9
    gbs_k = 4.0 * u.numel() / (ms_k * 1e-3) / 1e9
    return {"workload": "viability diagnostics of a 512^3 FP32 noise field", "kernel": "k_diag_rows<2,4,well>",
            "ms_per_launch": ms_k, "GBps_of_4B_per_voxel": gbs_k, "frac_of_hbm": gbs_k / peaks["hbm_gbs"],
            "hbm_peak_kind": kind, "ms_per_call_incl_sync": ms, "GBps_incl_sync": gbs,
            "same_values": bool(np.allclose(out.cpu().numpy(), [res[k] for k in ("discrepancy", "cahn_hilliard",
                                                                                 "ratio", "max", "min")],
                                            rtol=0, atol=0)),
            "ratio": res["ratio"]}


# Algorithmic FP32 flops of one voxel-step, counted from the arithmetic (FMA =
# 2): stencils 18, forward (eq. Feps) 86, local reverse mode 75,
# transposed-stencil pieces 19, gather 9, update and sums 4.
FLOPS_PER_VOXEL_STEP = 211
# For p symmetric in kappa1, kappa2 (a20 = a02, a10 = a01) the sqrt(D+) terms
# have weight zero and are not evaluated: D and its compensation 5, the weight
# c3 T + c5 q 3, the FP64-refinement test 3, sqrt(P) 2, its term in e 2;
# reverse: dr/dD 2, de/dD 1, its share of de/dS 2, of de/dT 4, of de/dq 2.
FLOPS_PER_VOXEL_STEP_SYM = FLOPS_PER_VOXEL_STEP - 26


def flops_per_voxel_step(a):
    """Algorithmic flops of one voxel-step for coefficients a (paper order)."""
    return FLOPS_PER_VOXEL_STEP_SYM if (a[0] == a[2] and a[3] == a[4]) else FLOPS_PER_VOXEL_STEP


def workload_flops(insts):
    """Algorithmic flops of one step over a list of instances."""
    return float(sum(flops_per_voxel_step(i.a) * int(np.prod(i.shape)) for i in insts))
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# instruction issue peak: 152 SMs x 4 schedulers x 1 warp instruction per clock x 2070 MHz
ISSUE_PEAK_TWIPS = 152 * 4 * 2070e6 / 1e12


# ------------------------------------------------------------ our arm

def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2103_04856_gb300 import inputs as I
    from paper_2103_04856_gb300 import pfc

    if args.only:
        run = {"alg1_flow_100": lambda: alg1_workload(pfc, I, steps=args.steps),
               "alg1_batch_100": lambda: alg1_batch_workload(pfc, I, 16, steps=args.steps),
               "extended_sweep_128": lambda: extended_sweep_workload(pfc, I, steps=args.steps),
               "alg1_spatialized": lambda: spatialized_flow_workload(pfc, I, steps=args.steps),
               "diagnostics_512": lambda: diagnostics_workload(pfc, I),
               "batch64_mixed": lambda: batch64_block(pfc, I, 500, ws, rank)}[args.only]
        print(json.dumps({"only": args.only, **run()}), flush=True)
        return 0

    insts = I.validation_set_128()
    launch = {"tile_y": args.tile_y, "max_run": max(args.max_run, 0), "source": "command line"}
    if not args.no_autotune and args.tile_y == 0 and args.max_run < 0:
        from paper_2103_04856_gb300 import autotune
        best = autotune.tune([i.shape for i in insts], cache=None,
                             symmetric=all(i.a[0] == i.a[2] and i.a[3] == i.a[4] for i in insts))
        launch = {"tile_y": best["tile_y"], "max_run": best["max_run"], "source": "autotuned",
                  "tried": [{k: r[k] for k in ("tile_y", "max_run", "sweep_ms")} for r in best["tried"]]}
    probs = [problem_of(pfc, i, "fp32", tile_y=launch["tile_y"], tile_z=launch["max_run"]) for i in insts]
    host = [i.field().astype(np.float32) for i in insts]
    taus = [i.tau for i in insts]
    A = [torch.tensor(h, device="cuda") for h in host]
    B = [torch.empty_like(a) for a in A]
    vox = sum(h.size for h in host)
    batch = pfc.Batch(probs)
    batch.timing(True)
    flush = torch.empty(args.flush_mb * (1 << 20), dtype=torch.uint8, device="cuda")

    # accuracy on the initial state: FP32 fused vs FP64 fused (the FP64 path
    # equals the oracle to 1e-10 in the tests)
    acc_initial = accuracy(pfc, insts, host)

    # one step = one batched fused launch, the mass projection in its fused
    # form: each step's FP64 offset c = m - mean(u') is added by the next
    # step's loads, the chain's last one by one launch at the end, which is
    # timed and spread over the steps (pfc_batch_step_lazy / _lazy_finish)
    cur, nxt = A, B
    for k in range(args.warmup):
        flush.zero_()
        batch.step_lazy(cur, nxt, taus, first=(k == 0))
        cur, nxt = nxt, cur
    batch.lazy_finish(cur)
    torch.cuda.synchronize()

    gpu_uuid = None
    try:
        gpu_uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not gpu_uuid.startswith("GPU-"):
            gpu_uuid = "GPU-" + gpu_uuid
    except Exception:
        gpu_uuid = None
    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    # the FP32 issue peak of this GPU now, measured in-process with FMA
    # chains (pfc_measure_fp32_peak): the arithmetic roofline's denominator
    fp32_peak = pfc.measure_fp32_peak()
    time.sleep(0.2)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step_ms, sweep_ms = [], []
    for k in range(args.steps):
        flush.zero_()
        batch.step_lazy(cur, nxt, taus, first=(k == 0))
        a, b = batch.last_timing()
        step_ms.append(a)
        sweep_ms.append(b)
        cur, nxt = nxt, cur
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    batch.lazy_finish(cur)
    ev1.record()
    torch.cuda.synchronize()
    finish_ms = ev0.elapsed_time(ev1)
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clocks.stop()

    ms_step, ms_sweep = max_over_ranks([float(np.mean(step_ms)) + finish_ms / args.steps, float(np.mean(sweep_ms))])
    value = job_value(vox, ws, ms_step)

    # the same steps one at a time, each materialising its projection with a
    # second launch (pfc_batch_step), for comparison
    mat_ms = []
    for _ in range(args.steps):
        flush.zero_()
        batch.step(cur, nxt, taus)
        mat_ms.append(batch.last_timing()[0])
        cur, nxt = nxt, cur
    torch.cuda.synchronize()
    ms_step_mat = max_over_ranks([float(np.mean(mat_ms))])[0]

    # mass is kept by every step; accuracy again on the last state
    mass_err = max(abs(c.double().mean().item() - h.astype(np.float64).mean()) for c, h in zip(cur, host))
    acc_final = accuracy(pfc, insts, cur)

    # the FP64 paths on the same workload: plain (5 unfused passes through
    # HBM) and fused (the same sweep in FP64), exact steps one at a time
    def fp64_rate(impl, nsteps):
        ctxs = [pfc.Context(problem_of(pfc, i, "fp64", impl=impl)) for i in insts]
        ua = [torch.tensor(h.astype(np.float64), device="cuda") for h in host]
        ub = [torch.empty_like(x) for x in ua]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for k in range(nsteps + 2):
            flush.zero_()
            e0.record()
            for c, x, y, tau in zip(ctxs, ua, ub, taus):
                c.step(x, y, tau)
            e1.record()
            e1.synchronize()
            if k >= 2:
                tot += e0.elapsed_time(e1)
            ua, ub = ub, ua
        for c in ctxs:
            c.close()
        ms64 = tot / nsteps
        return {"value": vox / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "dtype": "f64"}

    fp64 = fp64f = None
    if args.fp64_steps > 0:
        fp64 = fp64_rate("plain", args.fp64_steps)
        fp64["impl"] = "plain: 5 unfused passes storing grad u, Hess u and cotangents in HBM"
        fp64f = fp64_rate("fused", args.fp64_steps)
        fp64f["impl"] = "fused: the same single sweep in FP64, plus the projection launch"

    # end to end through the C ABI with host buffers (pfc_batch_step_host):
    # every step copies its four fields in from pinned host memory, steps them
    # and copies the results back; the library pipelines the problems and
    # overlaps consecutive steps, and the timed region ends when the last
    # result is in host memory
    pin_in = [torch.from_numpy(h).pin_memory() for h in host]
    pin_out = [torch.empty_like(p).pin_memory() for p in pin_in]
    for _ in range(2):
        batch.step_host(pin_in, pin_out, taus)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for k in range(args.e2e_steps):
        batch.step_host(pin_in, pin_out, taus, wait=False)
    batch.host_wait()
    e2e_t = time.perf_counter() - t1
    e2e_bytes = sum(h.nbytes for h in host)
    e2e = {"value": ws * vox * args.e2e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
           "d2h_bytes_per_step": e2e_bytes}

    peaks, peak_kind = load_peaks()
    fp32_kind = ("measured in-process: pfc_measure_fp32_peak (FMA chains on every SM, best of 3, CUDA events) "
                 "just before the timed steps")
    bytes_launch = 8.0 * vox                      # read u, write u' (FP32)
    hbm_achieved = bytes_launch / (ms_sweep * 1e-3) / 1e9
    ty_used = launch["tile_y"] or 16                 # the batch's automatic height
    prof, traffic_note = committed_profile(ty_used, launch["max_run"])
    traffic = float(prof["traffic_bytes_per_launch"]) if prof else None
    flops_launch = workload_flops(insts)
    all_sym = all(i.a[0] == i.a[2] and i.a[3] == i.a[4] for i in insts)
    # 185-211 flop per 8 B is ~2x GB300's FP32/HBM balance: the sweep is bound
    # by arithmetic issue, not by HBM; the HBM fraction is reported beside it
    roofline = alu_roofline(flops_launch, ms_sweep, fp32_peak, fp32_kind,
                            f"k_fused<float,{ty_used},STEP,64{',SYM' if all_sym else ''}> (batched fused sweep)")
    roofline.update({"traffic": traffic, "derived_peak": FP32_PEAK_TFLOPS,
                     "derived_peak_kind": "152 SM x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "flops_per_voxel_step": flops_launch / vox, "voxels_per_launch": vox,
                     "hbm": {"achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": hbm_achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                             "algorithmic_bytes_per_launch": bytes_launch}})
    if traffic is None:
        roofline["traffic_note"] = traffic_note
    if prof and prof.get("warp_instructions_per_launch"):
        # what actually bounds the sweep: instruction issue (one warp
        # instruction per scheduler per clock), from the committed count of
        # this kernel's instructions and its live duration
        wi = float(prof["warp_instructions_per_launch"])
        issue_achieved = wi / (ms_sweep * 1e-3) / 1e12
        roofline["issue"] = {"achieved": issue_achieved, "peak": ISSUE_PEAK_TWIPS, "unit": "T warp-instr/s",
                             "frac": issue_achieved / ISSUE_PEAK_TWIPS, "warp_instructions_per_launch": wi,
                             "peak_kind": "derived: 152 SM x 4 schedulers x 1 warp instruction x 2070 MHz"}

    extra = None
    if not args.no_extra:
        extra = {"membrane_512": membrane_block(pfc, I, flush, 10, fp32_peak, fp32_kind,
                                                with_cpu=(rank == 0 and ws == 1 and not args.no_cpu_baseline)),
                 "batch64_mixed": batch64_block(pfc, I, 500, ws, rank),
                 "tube_256_2000_steps": tube_256_block(pfc, I, 2000, fp32_peak, fp32_kind),
                 "willmore_32_fp64_100_steps": descent_32_block(pfc, I),
                 "membrane_512_zslabs": slab_block(pfc, I, 20, ws, rank),
                 "alg1_flow_100": alg1_workload(pfc, I, steps=8000),
                 "alg1_batch_100x16": alg1_batch_workload(pfc, I, 16, steps=256),
                 "extended_sweep_128": extended_sweep_workload(pfc, I, steps=64),
                 "alg1_spatialized_600x100x100": spatialized_flow_workload(pfc, I, steps=64),
                 "diagnostics_512": diagnostics_workload(pfc, I)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "validation_128: 4 x 128^3 (tanh sphere R=32, z-cylinder r=20; eps=2, h=1; "
                                   "p=k1^2+k2^2 and p=k1k2), one batched fused step each",
                       "step": "one batched fused launch; the mass projection in fused form (each step's FP64 "
                               "offset is added by the next step's loads; the last one by one launch, timed "
                               "and spread over the steps)",
                       "voxels_per_step": vox, "l2": f"flushed ({args.flush_mb} MB write) before every timed step",
                       "symmetric_p": "both polynomials are symmetric in k1, k2: the sqrt(D+) terms have weight "
                                      "exactly 0 and are not evaluated (same result bits); 185 flop per "
                                      "voxel-step counted; other_workloads hold asymmetric p",
                       "parallelism": f"replicas x{ws}"},
            "wall_ms_per_step_incl_flush": 1e3 * wall / args.steps,
            "ms_per_step_materialized": ms_step_mat,
            "accuracy_fp32_vs_fp64": {"initial": acc_initial, "final": acc_final,
                                      "steps_between": args.warmup + 2 * args.steps},
            "rel_energy_err_fp32_vs_fp64": max(acc_initial["rel_energy_err"], acc_final["rel_energy_err"]),
            "mass_drift": mass_err,
            "fp64_plain": fp64, "fp64_fused": fp64f,
            "speedup_vs_fp64_plain": (value / ws) / fp64["value"] if fp64 else None,
            "speedup_vs_fp64_fused": (value / ws) / fp64f["value"] if fp64f else None,
            "launch": launch, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "other_workloads": extra,
            "gpu_launches": args.steps + 1, "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
