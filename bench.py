#!/usr/bin/env python
"""Throughput of the periodic FMM with a neutralising background charge.

One step = one pass of the whole hot path on one batch: leaf sort, P2M, M2M,
level-0 lattice (Eq. 12), M2L + L2L on every level, L2P with gradient, near
field, background-charge terms (Eq. Velecfull), forces, and the reduced-far-
field solute-solvent energy (Eq. FMMcalc) -- one fmm_evaluate call.

Default workload: Na+ + 333,333 rigid TIP3P waters (N = 1,000,000, L = 215.3 A),
depth 6, p = 12, ws = 1, mixed precision (FP32 near field and expansions,
FP64 lattice operator, background terms and reductions).  The FP64 path on
the same input is timed beside it and the mixed path's error against it is
reported.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run: every rank evaluates its own
replica of the workload (the single-box path does not shard; weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-evals/s, FMM energy+forces @1M charges: mixed vs FP64 at ≤1e-6 rel err"
UNIT = "particle-evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) of one level-6 tensor-core M2L launch (fp16x2
# split, fused L2L, CTA pairs) of the na_1m workload, from the ncu capture of
# that launch summarised under profiles/, with the sha256 of the kernel's device
# code it was taken on: the value is reported only while that code is unchanged.
M2L_TRAFFIC = {"src": "paper_2003_13218_gb300/csrc/fmm_m2l_tc.cu",
               "sha256": "711fa46ddc82e4c3acf198ceac77e93d844a0a4abb2a2d0c76207d4d088579b9",
               "workload": "na_1m", "level": 6, "split": "fp16x2", "ws": 1, "p": 12,
               "bytes_per_launch": 360.280320e6 + 160.011776e6}
ION_LABEL = {"Na": "Na+", "Cl": "Cl-", "Mg": "Mg2+"}
KERNEL_BEGIN = "// ------------------------------------------------------------------ the kernel"
KERNEL_END = "// ------------------------------------------------------------------ operand preparation"


def n_il(ws: int) -> int:
    """Interaction-list length: (4 ws + 2)^3 - (2 ws + 1)^3 (189 for ws = 1, 875 for ws = 2)."""
    return (4 * ws + 2) ** 3 - (2 * ws + 1) ** 3


def m2l_flops(d: int, p: int, levels=None, fused_l2l=False, ws: int = 1) -> float:
    """Algorithmic flops of M2L: 2 C^2 per (target, source) pair, 189 sources per target,
    plus one dense C x C product per target when the L2L is fused into the same launch."""
    C = (p + 1) ** 2
    levels = range(1, d + 1) if levels is None else levels
    pairs = (n_il(ws) + (1 if fused_l2l else 0)) * sum(8 ** l for l in levels)
    return 2.0 * C * C * pairs


GRADE_DEFAULT = (4, 8)  # the library's default M2L grading (FMM_GRADE_DEFAULT): degrees 4..7 two products, >= 8 one


def mmas_per_offset(p: int, grade, products: int = 3) -> tuple[int, int]:
    """K16 MMA steps (128-row units) per interaction-list offset of the fp16x2 tensor-core M2L and per
    fused L2L offset: K chunks of 64 coefficients, chunk kc graded by its lowest degree floor(sqrt(64 kc))
    (1 product from degree D1, 2 from D2, else 3); in a 3-product chunk the K16 steps whose lowest degree
    floor(sqrt(64 kc + 16 s)) reaches D2 take 2."""
    C = (p + 1) ** 2
    ksteps = (C + 15) // 16
    kchunks = ((C + 63) // 64 * 64) // 64
    d2, d1 = grade
    m2l = 0
    for kc in range(kchunks):
        lam = int(math.isqrt(64 * kc))
        np_ = 1 if (d1 > 0 and lam >= d1) else 2 if (d2 > 0 and lam >= d2) else products
        for st in range(min(4, ksteps - 4 * kc)):
            if np_ == 3 and d2 > 0 and int(math.isqrt(64 * kc + 16 * st)) >= d2:
                m2l += 2
            else:
                m2l += np_
    return m2l, products * ksteps


def kernel_sha(rel):
    try:
        with open(os.path.join(ROOT, rel)) as f:
            s = f.read()
        return hashlib.sha256(s[s.index(KERNEL_BEGIN):s.index(KERNEL_END)].encode()).hexdigest()
    except (OSError, ValueError):
        return None


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time: every rank returns the maximum of `ms` over the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, steps: int, world: int, ms_total: float) -> float:
    """Whole-job particle-evals/s: every rank evaluates its own replica `steps` times; the job
    takes the slowest rank's time."""
    return n_per_rank * steps * world / (ms_total / 1e3)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def src_sha(rel):
    try:
        with open(os.path.join(ROOT, rel), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None


# --------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2003_13218_gb300 import boxes
    from paper_2003_13218_gb300.fmm import FMMPlan

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    box, d, p = boxes.workload(args.workload, seed=rank)
    if args.p is not None:
        p = args.p
    if args.depth is not None:
        d = args.depth
    N = box.N
    pos = torch.from_numpy(box.pos).to(dev)
    q = torch.from_numpy(box.q).to(dev)
    sol = torch.from_numpy(box.is_solute).to(dev)
    F = torch.empty((N, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    grade = GRADE_DEFAULT if args.m2l_grade is None else tuple(int(x) for x in args.m2l_grade.split(","))
    plan = FMMPlan(box.L, N, d, p, precision="mixed", split=args.split, timings=True, ws=args.ws,
                   overlap=bool(args.overlap), m2l_grade=None if args.m2l_grade is None else grade,
                   acc_group=args.acc_group)
    for _ in range(args.warmup):
        plan.evaluate(pos, q, sol, forces=F)
    torch.cuda.synchronize()
    launches = plan.last_launch_count()
    backend = plan.m2l_backend(d)

    jgen = torch.Generator(device=dev)
    jgen.manual_seed(1234 + rank)
    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    stream = torch.cuda.current_stream()
    ms_total = 0.0
    m2l_ms = []
    terms = uv = None
    for k in range(args.steps):
        if args.jitter > 0 and k > 0:  # new coordinates every call, as in a trajectory (before e0: not timed)
            pos.add_(torch.randn(pos.shape, generator=jgen, device=dev, dtype=torch.float64) * args.jitter)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        terms, uv = plan.evaluate(pos, q, sol, forces=F)
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        tm = plan.timings()
        m2l_ms.append((tm["m2l_top"], tm["m2l_kernels"]))
        flush.zero_()  # L2 flush between timed steps (not timed)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if ws > 1:
        ms_total = max_over_ranks(ms_total, dev)
        dist.barrier()
    stage = plan.timings()
    F_mixed = F.cpu().numpy()

    # end to end through the public API with host buffers (copies inside the call)
    hpos, hq, hsol = box.pos, box.q, box.is_solute
    hF = np.empty((N, 3))
    plan.evaluate(hpos, hq, hsol, forces=hF)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.evaluate(hpos, hq, hsol, forces=hF)
    e2e_s = time.perf_counter() - t0

    # cost of the solute-solvent energy: the reduced scheme (Eq. FMMcalc, one extra sparse pass)
    # against the conventional three passes (Eq. FMMconv: u+v, u alone, v alone), energies only
    def ev_ms(fn, k=3):
        fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k
    qu = torch.where(sol == 1, q, torch.zeros_like(q))
    qv = q - qu
    t_e = ev_ms(lambda: plan.evaluate(pos, q, None, forces=None))
    t_uv = ev_ms(lambda: plan.evaluate(pos, q, sol, forces=None))
    t_u = ev_ms(lambda: plan.evaluate(pos, qu, None, forces=None))
    t_v = ev_ms(lambda: plan.evaluate(pos, qv, None, forces=None))
    uv_cost = {"energy_only_ms": t_e, "energy_and_e_uv_reduced_ms": t_uv, "three_pass_ms": t_e + t_u + t_v,
               "e_uv_extra_reduced_ms": t_uv - t_e, "e_uv_extra_three_pass_ms": t_u + t_v}
    plan.close()

    # the FP64 path on the same input
    fp64 = None
    if args.fp64_steps > 0:
        p64 = FMMPlan(box.L, N, d, p, precision="fp64", timings=True, ws=args.ws)
        F64 = torch.empty_like(F)
        t64, uv64 = p64.evaluate(pos, q, sol, forces=F64)
        torch.cuda.synchronize()
        ms64 = 0.0
        for _ in range(args.fp64_steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t64, uv64 = p64.evaluate(pos, q, sol, forces=F64)
            e1.record(stream)
            e1.synchronize()
            ms64 += e0.elapsed_time(e1)
            flush.zero_()
        F64h = F64.cpu().numpy()
        p64.close()
        fp64 = {
            "value": N * args.fp64_steps / (ms64 / 1e3) * ws,
            "ms_per_step": ms64 / args.fp64_steps,
            "steps": args.fp64_steps,
            "rel_err_energy_mixed_vs_fp64": abs(terms["total"] - t64["total"]) / abs(t64["total"]),
            "rel_rms_force_err_mixed_vs_fp64": float(np.sqrt(np.mean((F_mixed - F64h) ** 2)) /
                                                     np.sqrt(np.mean(F64h ** 2))),
            "abs_err_e_uv_mixed_vs_fp64": abs(uv["e_uv"] - uv64["e_uv"]),
        }

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    value = job_throughput(N, args.steps, ws, ms_total)
    peaks, peak_kind = load_peaks()
    uses_tc = backend == "tcgen05"
    fused = uses_tc and args.split == "fp16x2"  # the fp16 split fuses the L2L into each level's launch
    stage_flops = m2l_flops(d, p, fused_l2l=fused, ws=args.ws)
    stage_ms = statistics.mean(x[1] for x in m2l_ms)
    if uses_tc:
        # the dominant launch: the tensor-core M2L of the finest level
        flops = m2l_flops(d, p, levels=[d], fused_l2l=fused, ws=args.ws)
        launch_ms = statistics.mean(x[0] for x in m2l_ms)
        peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
        roof = {"bound": "tensor", "peak_source": peak_kind + " bf16 dense burst (MEASURED_PEAKS.json)",
                "kernel": "k_m2l_tc, level %d (one launch%s)" % (d, ", M2L + fused L2L" if fused else "")}
        traffic = None
        if (M2L_TRAFFIC and M2L_TRAFFIC["workload"] == args.workload and M2L_TRAFFIC["level"] == d
                and M2L_TRAFFIC.get("ws", 1) == args.ws and M2L_TRAFFIC.get("p", p) == p
                and M2L_TRAFFIC["split"] == args.split and kernel_sha(M2L_TRAFFIC["src"]) == M2L_TRAFFIC["sha256"]):
            traffic = M2L_TRAFFIC["bytes_per_launch"]
    else:
        flops, launch_ms = stage_flops, stage_ms
        peak = FP32_ALU_TFLOPS
        roof = {"bound": "alu", "peak_source": "FP32 CUDA-core peak from unit counts and max clock",
                "kernel": "k_m2l_simt<float> (all levels, one evaluation)"}
        traffic = None
    achieved = flops / (launch_ms / 1e3) / 1e12
    if uses_tc:
        # tensor work actually issued by the launch: every target row runs one 128 x npad x 16 MMA per
        # K step (K = (p+1)^2 padded to 16), split product and offset
        C = (p + 1) ** 2
        ksteps, npad = (C + 15) // 16, (C + 15) // 16 * 16
        products = {"fp16x2": 3, "bf16x3": 6, "bf16a2b3": 4, "bf16x2": 3}.get(args.split, 0)
        if args.split == "fp16x2":
            per_m2l, per_l2l = mmas_per_offset(p, grade, products)
        else:
            per_m2l, per_l2l = products * ksteps, products * ksteps
        issued = 8 ** d * (n_il(args.ws) * per_m2l + (per_l2l if fused else 0)) * 2.0 * npad * 16
        roof["mma_steps_per_offset"] = {"m2l": per_m2l, "fused_l2l": per_l2l if fused else 0,
                                        "ungraded": products * ksteps}
        roof["issued_flops_per_launch"] = issued
        roof["issued_tflops"] = issued / (launch_ms / 1e3) / 1e12
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                 "algorithmic_flops_per_launch": flops, "avg_launch_ms": launch_ms,
                 "m2l_all_levels": {"ms": stage_ms, "tflops": stage_flops / (stage_ms / 1e3) / 1e12}})
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32+%s-tensor+f64" % args.split) if uses_tc else "f32+f64",
        "data": "synthetic (seeded ion-in-water boxes standing in for the paper's MD snapshots)",
        "config": {"workload": "%s: %s + %d TIP3P waters, N=%d, L=%.2f A, depth %d, p %d, ws %d, mixed precision, "
                               "energy+forces+solute-solvent per step" % (args.workload, ION_LABEL[box.ion], box.n_waters, N,
                                                                          box.L, d, p, args.ws),
                   "l2": "flushed between timed steps (256 MB write)", "jitter_A": args.jitter, "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "m2l_split": args.split, "overlap": bool(args.overlap),
                   "m2l_grade": {"d2": grade[0], "d1": grade[1], "note": "K16 steps of input degree >= d2 with two fp16 products, K chunks of degree >= d1 with one"},
                   "acc_group": args.acc_group if args.acc_group is not None else "library default (2)"},
        "roofline": roof,
        "solute_solvent_cost": uv_cost,
        "e2e": {"value": N * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": N * (24 + 8 + 1),
                "d2h_bytes_per_step": N * 24 + 29 * 8 + 4},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "stage_ms": stage,
        "fp64_path": fp64,
    }
    if ws == 1 and args.batch_leg:
        # the batched lambda-window workload (64 boxes of uneven size), timed here so that every default
        # run carries it
        m = measure_batch(max(3, args.steps // 2), 3, rank, local, serial=False)
        out["lambda64"] = {"value": m["Ntot"] / m["t_graph"], "unit": UNIT, "ms_per_step": m["t_graph"] * 1e3,
                           "workload": m["workload"], "timing": "host wall time around the synchronous batch call",
                           **m["batch"]}
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------- the oracle
def sample_box(workload: str, shrink: int):
    """A sub-box of the workload with the same density, leaf occupancy and order p:
    1/shrink^3 of the waters in a box 1/shrink the side, depth reduced by log2(shrink)."""
    from paper_2003_13218_gb300 import boxes
    w = boxes.WORKLOADS[workload]
    L = w["L"] if w["L"] is not None else (w["n_waters"] / boxes.WATER_DENSITY) ** (1 / 3)
    k = int(round(math.log2(shrink)))
    b = boxes.ion_in_water(w["n_waters"] // shrink ** 3, w["ion"], seed=0, L=L / shrink)
    return b, w["depth"] - k, w["p"]


def oracle_step(b, d, p):
    import oracle
    oracle.fmm(b.pos, b.q, b.L, d, p, forces=True)
    oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, d, p)


BATCH_TOL = 1e-6  # relative energy error budget of the batch tuner's order choice (the metric's 1e-6)

SAMPLE_SHRINK = 8  # the oracle's bounded sample: a 1/512 sub-box (both the cpu_baseline leg and --impl reference)


def one_core_seconds(workload: str):
    """One oracle step on the sample sub-box with a single OpenMP thread (fresh process)."""
    code = ("import sys, time; sys.path.insert(0, %r); import bench; b, d, p = bench.sample_box(%r, %d); "
            "t = time.perf_counter(); bench.oracle_step(b, d, p); print(time.perf_counter() - t)" %
            (ROOT, workload, SAMPLE_SHRINK))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        return float(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def cpu_baseline(workload: str):
    import oracle
    b, d, p = sample_box(workload, SAMPLE_SHRINK)
    oracle_step(b, d, p)  # builds the oracle's tables once
    n, t0 = 0, time.perf_counter()
    while True:  # about 10 s of the oracle on all host cores
        oracle_step(b, d, p)
        n += 1
        dt = time.perf_counter() - t0
        if dt > 10.0:
            break
    t1 = one_core_seconds(workload)
    return {"value": b.N * n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d energy+forces+solute-solvent evaluations of a 1/512 sub-box of the workload "
                      "(N=%d, L=%.2f A, depth %d, p %d: same density, leaf occupancy and order), %.1f s; "
                      "the same sub-box as --impl reference" % (n, b.N, b.L, d, p, dt),
            "one_core": None if t1 is None else {"value": b.N / t1, "unit": UNIT, "cores": 1, "seconds": t1}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    b, d, p = sample_box(args.workload, SAMPLE_SHRINK)
    for _ in range(args.warmup):
        oracle_step(b, d, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(b, d, p)
    dt = time.perf_counter() - t0
    value = b.N * args.steps / dt
    sample = ("per step one energy+forces+solute-solvent evaluation of a 1/512 sub-box of the workload "
              "(N=%d, L=%.2f A, depth %d, p %d: same density, leaf occupancy and order)" % (b.N, b.L, d, p))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + " (bounded CPU sample, see cpu_baseline.sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def measure_batch(steps: int, warmup: int, rank: int, local: int, serial: bool = True, shard_world: int = 0):
    """The batched free-energy workload: 64 ion-in-water boxes of uneven size (lambda
    windows, ion charge scaled by lambda), per box E_total, E_uv, V_lambda and dV/dlambda_C
    through fmm_batch_*; the recorded-graph path is timed, beside the stream path and (serial)
    the same boxes on single plans one after the other."""
    import torch

    from paper_2003_13218_gb300 import boxes
    from paper_2003_13218_gb300.fmm import FMMBatch, FMMPlan

    dev = torch.device("cuda", local)
    if shard_world > 1:
        # one 64-box batch split across the ranks by estimated cost (each rank evaluates its share)
        from paper_2003_13218_gb300 import shard
        allwin = boxes.lambda_windows(64, seed=0)
        mine = shard.partition_boxes([shard.box_cost(b.N) for b, _ in allwin], shard_world)[rank]
        win = [allwin[i] for i in mine]
    else:
        win = boxes.lambda_windows(64, seed=rank)
    Ntot = sum(b.N for b, _ in win)
    lam = np.array([l for _, l in win])
    pos = [torch.from_numpy(b.pos).to(dev) for b, _ in win]
    q = [torch.from_numpy(b.q).to(dev) for b, _ in win]
    sol = [torch.from_numpy(b.is_solute).to(dev) for b, _ in win]
    t0 = time.perf_counter()
    # depth, order (within BATCH_TOL relative energy error) and launch form chosen by the batch tuner
    bt = FMMBatch([b.L for b, _ in win], [b.N for b, _ in win], None, [-1] * len(win), precision="mixed",
                  energy_rel_tol=BATCH_TOL, sweep="auto", tiles=True)
    create_s = time.perf_counter() - t0
    depths = [bt.info(i)["depth"] for i in range(len(win))]
    orders = [bt.info(i)["p"] for i in range(len(win))]
    tune = bt.tune_info()
    bricks = sorted({"d%d: %dx%dx%d" % (l, *bk) for l, bk in (bt.brick(i) for i in range(len(win)))})

    def timed(fn, k):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(k):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / k

    sampler = ClockSampler(local)
    for _ in range(warmup):
        r = bt.lambda_energies(pos, q, sol, lam)
    sampler.start()
    t_graph = timed(lambda: bt.lambda_energies(pos, q, sol, lam), steps)
    clocks = sampler.stop()
    info = bt.info(0)
    r_graph = bt.lambda_energies(pos, q, sol, lam)
    # the same graph with the other launch form (A/B of the persistent sweep)
    sweep_was = tune["sweep_on"]
    bt.set_sweep(not sweep_was)
    sweep = bt.sweep_info() if not sweep_was else None
    bt.lambda_energies(pos, q, sol, lam)
    r_other = bt.lambda_energies(pos, q, sol, lam)
    t_other = timed(lambda: bt.lambda_energies(pos, q, sol, lam), steps)
    bt.set_sweep(sweep_was)
    if sweep is None:
        sweep = bt.sweep_info()
    bt.set_graph(False)
    bt.lambda_energies(pos, q, sol, lam)
    t_stream = timed(lambda: bt.lambda_energies(pos, q, sol, lam), steps)
    r_stream = bt.lambda_energies(pos, q, sol, lam)
    bt.close()
    batch = {"graph_ms": t_graph * 1e3, "stream_path_ms": t_stream * 1e3, "plan_create_s": create_s,
             "depths": depths, "replays": info["replays"],
             "orders": sorted(set(orders)),
             "tuner": {"energy_rel_tol": BATCH_TOL, "p_err_vs_p15_on_water_test_box": {str(k): v for k, v in
                                                                                   tune["p_err"].items()},
                       "p_chosen": tune["p_chosen"], "tile_bricks": bricks,
                       "graph_ms_sweep_off": tune["ms_sweep_off"],
                       "graph_ms_sweep_on": tune["ms_sweep_on"], "sweep_chosen": tune["sweep_on"],
                       "note": "timed on uniform test charges at batch creation"},
             "sweep": {"boxes": sweep["boxes"], "first_levels": sorted(set(sweep["first_level"])),
                       "in_use": sweep_was,
                       ("graph_ms_per_level_launches" if sweep_was else "graph_ms_with_sweep"): t_other * 1e3,
                       "bitwise_equal_to_the_other_form": bool(
                           all(np.array_equal(r_graph[k], r_other[k]) for k in ("e_total", "e_uv")))}}
    if serial:
        # the same boxes and depths on single plans, one after the other
        plans = [FMMPlan(b.L, b.N, d, pi, precision="mixed") for (b, _), d, pi in zip(win, depths, orders)]
        def serial_run():
            for pl, x, y, z in zip(plans, pos, q, sol):
                pl.evaluate(x, y, z, forces=None)
        serial_run()
        t_serial = timed(serial_run, max(1, steps // 2))
        e_single = np.array([pl.evaluate(x, y, z, forces=None)[1]["e_uv"] for pl, x, y, z in zip(plans, pos, q, sol)])
        for pl in plans:
            pl.close()
        batch["single_plans_serial_ms"] = t_serial * 1e3
        # the tuned order on the actual boxes: the smallest and the largest box against FP64 at the same
        # order (the metric's arithmetic error) and against FP64 at p = 15 (the change the order makes)
        acc = {}
        for i in (int(np.argmin([b.N for b, _ in win])), int(np.argmax([b.N for b, _ in win]))):
            b = win[i][0]
            row = {}
            for pr, key in ((orders[i], "vs_fp64_same_p"), (15, "vs_fp64_p15")):
                ref = FMMPlan(b.L, b.N, depths[i], pr, precision="fp64")
                e64 = ref.evaluate(pos[i], q[i], sol[i], forces=None)[0]["total"]
                ref.close()
                row[key] = abs(r_stream["e_total"][i] - e64) / abs(e64)
            acc["box%d_N%d" % (i, b.N)] = row
        batch["rel_err_e_total"] = acc
        batch["max_rel_diff_e_uv_vs_single_plans"] = float(np.max(np.abs(r_stream["e_uv"] - e_single) /
                                                                  np.maximum(np.abs(e_single), 1e-30)))
    workload = ("lambda64: 64 boxes, %d charges in all (%d..%d per box), species Mg/Na/Cl, lambda = (b mod 16)/15, "
                "order p, depth, tile bricks and launch form chosen by the batch tuner" % (Ntot, min(b.N for b, _ in win),
                                                                  max(b.N for b, _ in win)))
    out = {"Ntot": Ntot, "t_graph": t_graph, "batch": batch, "clocks": clocks, "workload": workload}
    if shard_world > 1:
        from paper_2003_13218_gb300 import shard
        out["gathered"] = shard.gather_box_results({"e_total": r_stream["e_total"], "e_uv": r_stream["e_uv"]},
                                                   mine, 64)
    return out


def run_batch(args):
    import torch
    rank = int(os.environ.get("RANK", 0))
    ws = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    sharded = args.shard and ws > 1
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")  # host-side gather of per-box FP64 results only
    m = measure_batch(args.steps, args.warmup, rank, local, shard_world=ws if sharded else 0)
    t_graph = m["t_graph"]
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([t_graph], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_graph = float(t.item())
        n = torch.tensor([float(m["Ntot"])], dtype=torch.float64)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        n_all = float(n.item())
        dist.destroy_process_group()
    else:
        n_all = float(m["Ntot"])
    if rank != 0:
        return
    Ntot = m["Ntot"]
    out = {
        "metric": "particle-evals/s, batched lambda windows: E_total, E_uv, V_lambda, dV/dlambda_C per box",
        "value": n_all / t_graph, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_graph * 1e3, "higher_is_better": True, "scaling": "strong" if sharded else "weak",
        "vs_baseline": None,
        "dtype": "f32+fp16x2-tensor+f64", "data": "synthetic (seeded ion-in-water boxes, lambda-scaled ion charge)",
        "config": {"workload": m["workload"], "l2": "inputs (%.0f MB) larger than L2" % (Ntot * 33 / 1e6),
                   "parallelism": ("boxes sharded by cost across %d GPUs" % ws) if sharded else
                   ("replicas" if ws > 1 else "1 GPU")},
        "roofline": None,
        "batch": m["batch"],
        "note": "host wall time around the synchronous batch call (results read back); the batch owns its streams",
        "clocks": m["clocks"],
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="na_1m")
    ap.add_argument("--split", default="fp16x2", choices=["fp16x2", "bf16x3", "bf16x2", "bf16a2b3", "fp32"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="lambda64 on N GPUs: split one 64-box batch across the ranks (else every rank its own)")
    ap.add_argument("--batch-leg", type=int, default=1, choices=[0, 1],
                    help="1: also time the 64-box lambda-window batch and add it to the line")
    ap.add_argument("--ws", type=int, default=1, choices=[1, 2], help="well-separatedness (2: the paper's setting)")
    ap.add_argument("--p", type=int, default=None, help="expansion order (default: the workload's)")
    ap.add_argument("--depth", type=int, default=None, help="tree depth (default: the workload's)")
    ap.add_argument("--m2l-grade", default=None, help="D2,D1 of FMM_OPT_M2L_GRADE (default: the library's 4,8)")
    ap.add_argument("--acc-group", type=int, default=None, help="FMM_OPT_M2L_ACC_GROUP (default: the library's)")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="1: near field and sparse solute pass beside the far field (plan-owned streams)")
    ap.add_argument("--jitter", type=float, default=0.0,
                    help="jitter every position by N(0, jitter^2) A between timed calls (untimed)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "lambda64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
