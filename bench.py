#!/usr/bin/env python
"""Benchmark of the SpAMM dual-channel Newton-Schulz solve (S^{1/2} and S^{-1/2}).

Workload (one "step" = one full solve): Kac-Murdock-Szego matrix
S_ij = 0.9^|i-j|, N = 4096, leaf tiles N_b = 64, 30 iterations of the
dual-channel iteration with SpAMM products at tau (y channel tau_s =
0.01 tau).  The headline tau is the largest power of ten for which the
oracle's solve meets ||Z S Z - I||_F <= 1e-8 at this size; the tau sweep
{1e-4, 1e-6, 1e-8} (task counts, residual, solves/s) is reported beside it.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Multi-GPU (torchrun): every rank solves its own copy (independent problems,
weak scaling, no collective on the data path); value = all solves / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 4096
RHO = 0.9
LEAF = 64
MAXIT = 30
MAP = 0  # 0: NS map with alpha = 1; 1: damped, stabilised h_alpha (--map scaled)
TOL = 0.0  # > 0: a solve stops once |t_k| <= TOL (at most MAXIT iterations), on the device
CHANNEL = 0  # 0: dual channel, Eq. (cannonical); 1: single channel, Eq. (single)
TAU_HEADLINE = 1e-14
TAU_SWEEP = (1e-4, 1e-6, 1e-8)
GATE = 1e-8
METRIC = "NS sqrt/invsqrt solves/s at ||ZSZ-I||_F<=1e-8 (KMS N=4096)"
UNIT = "solves/s"


def workload_name(tau: float, precision: str) -> str:
    mp = (", damped stabilised map h_alpha" if MAP else "") + (", single channel" if CHANNEL else "")
    steps = f"{MAXIT}" if TOL <= 0 else f"until |t_k| <= {TOL:g} (at most {MAXIT})"
    return (f"KMS rho={RHO} N={N} N_b={LEAF} tau={tau:g} tau_s={0.01 * tau:g} {steps} NS iterations{mp}, "
            f"{precision} leaf products")


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Largest x over the ranks of the job (x itself for a single process).  The bench's
    timed region ends when the slowest rank ends."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, steps: int, t_max: float) -> float:
    """Whole-job throughput: every rank solves `steps` problems; the job takes t_max seconds."""
    return ws * steps / t_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle timing


def oracle_solve_rate(S, tau: float, budget_s: float, min_solves: int = 1) -> tuple[float, int, float, dict]:
    """Full oracle solves of S for about budget_s seconds: (solves/s, solves, seconds, the last solve)."""
    import oracle
    t0 = time.perf_counter()
    cnt = 0
    while True:
        ref = oracle.sqrt_invsqrt(S, LEAF, tau, MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
        cnt += 1
        el = time.perf_counter() - t0
        if cnt >= min_solves and el >= budget_s:
            break
        if el > 0 and cnt >= min_solves and el / cnt * (cnt + 1) > 3 * budget_s:
            break
    return cnt / el, cnt, el, ref


def rel_err(a, b) -> float:
    import numpy as np
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / nb if nb > 0 else float(np.linalg.norm(a))


def err_vs_oracle(Y, Z, st, ref) -> dict:
    """Relative Frobenius errors of a GPU solve against the oracle's solve of the same input, and whether the
    per-iteration task counts of its three products equal the oracle's."""
    import numpy as np
    out = {"Z": rel_err(Z, ref["Z"]), "Y": rel_err(Y, ref["Y"]), "iters_equal": bool(st["iters"] == ref["iters"])}
    if "task_hist" in st:
        out["task_hist_equal"] = bool(np.array_equal(np.asarray(st["task_hist"]), ref["task_hist"]))
    return out


def run_reference(args, ws, rank):
    """The oracle as it stands, timed on this host's cores on the bench workload."""
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    S = synth.kms(N, RHO)
    tau = args.tau
    for _ in range(args.warmup):
        oracle.sqrt_invsqrt(S, LEAF, tau, MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sqrt_invsqrt(S, LEAF, tau, MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = len(times) / tot
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(tau, "FP64 CPU oracle"), "n": N, "leaf": LEAF, "tau": tau,
                       "maxit": MAXIT, "tol_t": TOL, "map": args.map, "channel": args.channel},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(times)} full solves of the workload on {cores} OpenMP threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm


def measure_dgemm_tflops(torch, dev) -> float:
    """cuBLAS FP64 GEMM throughput on this GPU (denominator of the FP64 roofline)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def lens_summary(h, bins: int, channel: int) -> dict:
    """Share (%) of each product's surviving tile triples lying on each plane diagonal (distance 0) and within
    one tile of it, at the first and the last iteration: the collapse of the volume the paper calls lensing."""
    names = ("z", "s z", "x") if channel else ("y", "z", "x")
    planes = ("i=j", "j=k", "i=k")
    out = {"bins": bins, "iterations": int(h.shape[0])}
    for label, k in (("first", 0), ("last", h.shape[0] - 1)):
        rec = {}
        for p, nm in enumerate(names):
            tot = float(h[k, p, 0].sum())
            rec[nm] = {pl: {"on": round(100.0 * h[k, p, q, 0] / tot, 2) if tot else None,
                            "within_1": round(100.0 * h[k, p, q, :2].sum() / tot, 2) if tot else None}
                       for q, pl in enumerate(planes)}
        out[label] = rec
    return out


def source_digest(sources) -> str | None:
    """sha256 over the source text a captured kernel is built from, in order: each entry is a whole file
    ({"file": path}) or the span of a file from the first occurrence of a start marker up to the next
    occurrence of an end marker ({"file", "from", "to"}); None when a file or marker is missing."""
    import hashlib
    h = hashlib.sha256()
    for part in sources:
        path = os.path.join(ROOT, part["file"])
        if not os.path.exists(path):
            return None
        text = open(path, "rb").read()
        if "from" in part:
            a = text.find(part["from"].encode())
            b = text.find(part["to"].encode(), a + 1) if a >= 0 else -1
            if a < 0 or b < 0:
                return None
            text = text[a:b]
        h.update(text)
    return h.hexdigest()


def captured_traffic(kernel: str, tasks_per_launch: float):
    """DRAM bytes (read + write) per launch from the committed ncu capture of `kernel`, scaled by tasks
    to this run's mean launch; None when the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec or source_digest(rec["sources"]) != rec["sources_sha256"]:
        return None
    per_task = (rec["dram_read_bytes"] + rec["dram_write_bytes"]) / rec["tasks"]
    return per_task * tasks_per_launch


def run_gpu(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1508_05856_gb300 as sp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sp.lib()
    prec = sp.EMU64 if args.precision == "emu64" else sp.FP64
    tau = args.tau

    S = synth.kms(N, RHO)
    Sd = torch.from_numpy(S).to(dev)
    Yd = torch.empty_like(Sd)
    Zd = torch.empty_like(Sd)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve(t, profile=False, residual=False, raise_on=True):
        return sp.sqrt_invsqrt(Sd, t, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, profile=profile, map=MAP,
                               tol_t=TOL, residual=residual, channel=CHANNEL, raise_on=raise_on)

    # verification solve (untimed): residual against the gate, FP64 dense; its Y and Z are compared with the
    # oracle's solve of the same input on rank 0
    _, _, vst = solve(tau, residual=True, raise_on=False)
    Yv, Zv = (Yd.cpu().numpy(), Zd.cpu().numpy()) if rank == 0 else (None, None)
    lensing = None
    if args.lens_bins > 0:
        # plane-diagonal profile of every product (untimed): volume share on each plane diagonal per iteration
        _, _, lst = sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, map=MAP, tol_t=TOL,
                                    channel=CHANNEL, lens_bins=args.lens_bins)
        lensing = lens_summary(lst["lens_hist"], args.lens_bins, CHANNEL)
        if args.lens_npz:
            np.savez(args.lens_npz, lens_hist=lst["lens_hist"], task_hist=lst["task_hist"], t_hist=lst["t_hist"])
            lensing["npz"] = args.lens_npz
    for _ in range(max(args.warmup, 3)):
        solve(tau)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = sp.kernel_launches()
    step_s = []
    gemm_ms = 0.0
    gemm_launches = 0
    gemm_flops = 0.0
    tensor_units = 0
    phase = {k: [0.0, 0] for k in ("cull", "tree", "slice")}
    n_prof = max(1, min(args.steps, 3))
    for _ in range(args.steps):
        flush.zero_()                       # L2 (129 MB) flushed between timed solves
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve(tau)
        e1.record(stream)
        e1.synchronize()
        step_s.append(e0.elapsed_time(e1) / 1e3)
    launches = sp.kernel_launches() - l0
    barrier()
    clk = clocks.stop()
    # leaf-product kernel timings: separate solves with per-launch events (not part of the timed steps)
    prof_s = 0.0
    for _ in range(n_prof):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, st = solve(tau, profile=True)
        e1.record(stream)
        e1.synchronize()
        prof_s += e0.elapsed_time(e1) / 1e3
        gemm_ms += st["gemm_ms"]
        gemm_launches += st["gemm_launches"]
        gemm_flops += st["flops"]
        tensor_units += st["tensor_units"]
        for k in phase:
            phase[k][0] += st[f"{k}_ms"]
            phase[k][1] += st[f"{k}_launches"]
    tot = sum(step_s)
    tot_max = max_over_ranks(tot, ws, dev)
    value = job_rate(ws, args.steps, tot_max)

    # end to end through the C ABI with pinned host buffers (H2D of S, D2H of Y and Z inside the region)
    Sh = torch.from_numpy(S).pin_memory()
    Yh = torch.empty((N, N), dtype=torch.float64).pin_memory()
    Zh = torch.empty((N, N), dtype=torch.float64).pin_memory()
    sp.sqrt_invsqrt(Sh, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yh, Z=Zh, map=MAP, tol_t=TOL, channel=CHANNEL)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sp.sqrt_invsqrt(Sh, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yh, Z=Zh, map=MAP, tol_t=TOL, channel=CHANNEL)
        e2e_t.append(time.perf_counter() - t0)
    e2e_tot = max_over_ranks(sum(e2e_t), ws, dev)

    # the same solves stopped once |t_k| <= tol (the trace-error monitor of Sec. 4.2; the iteration is a
    # WHILE node of the solve's graph, so only the iterations that run are launched): a secondary figure,
    # the headline keeps the configuration's fixed iteration count
    to_tol = None
    if TOL <= 0 and args.tol_report > 0:
        _, _, tst = sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, map=MAP,
                                    tol_t=args.tol_report, residual=True, raise_on=False, channel=CHANNEL)
        tt = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, map=MAP, tol_t=args.tol_report,
                            raise_on=False, channel=CHANNEL)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1) / 1e3)
        to_tol = {"value": job_rate(ws, len(tt), max_over_ranks(sum(tt), ws, dev)), "unit": UNIT,
                  "tol_t": args.tol_report, "iters": tst["iters"], "t_final": tst["t_final"],
                  "resid_F": tst["resid_F"], "gate_met": bool(tst["resid_F"] <= GATE), "status": tst["status"]}

    # the plain FP64-pipe method on the same workload, for comparison with the tensor-core path
    fp64_path = None
    if prec == sp.EMU64 and not args.no_fp64_path:
        _, _, fst = sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=sp.FP64, Y=Yd, Z=Zd, residual=True,
                                         map=MAP, tol_t=TOL, channel=CHANNEL)
        ft = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=sp.FP64, Y=Yd, Z=Zd, map=MAP, tol_t=TOL,
                            channel=CHANNEL)
            e1.record(stream)
            e1.synchronize()
            ft.append(e0.elapsed_time(e1) / 1e3)
        fp64_path = {"value": job_rate(ws, len(ft), max_over_ranks(sum(ft), ws, dev)), "unit": UNIT,
                     "resid_F": fst["resid_F"], "gate_met": bool(fst["resid_F"] <= GATE),
                     "_out": (Yd.cpu().numpy(), Zd.cpu().numpy(), fst) if rank == 0 else None}

    # the other schedule of one solve (the batched engine with one problem: the y and z products share each
    # launch) and the schedule the autotuner picks for this input
    schedules = None
    if TOL <= 0 and MAP == 0 and CHANNEL == 0:
        sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, schedule=sp.SCHED_STAGES)
        tt = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, sst = sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd,
                                        schedule=sp.SCHED_STAGES)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1) / 1e3)
        _, _, ast = sp.sqrt_invsqrt(Sd, tau, MAXIT, leaf=LEAF, precision=prec, Y=Yd, Z=Zd, schedule=sp.SCHED_AUTO)
        schedules = {"branches": {"value": value, "unit": UNIT},
                     "stages": {"value": job_rate(ws, len(tt), max_over_ranks(sum(tt), ws, dev)), "unit": UNIT,
                                "ran_as": "stages" if sst["schedule"] == sp.SCHED_STAGES else "branches"},
                     "autotuned": "stages" if ast["schedule"] == sp.SCHED_STAGES else "branches"}

    # tau sweep (the configuration's cull-count / error study)
    sweep = []
    if not args.no_sweep:
        for ts in TAU_SWEEP:
            _, _, rs = solve(ts, residual=True, raise_on=False)
            out_s = (Yd.cpu().numpy(), Zd.cpu().numpy(), rs) if rank == 0 else None
            tt = []
            for _ in range(3):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                solve(ts, raise_on=False)
                e1.record(stream)
                e1.synchronize()
                tt.append(e0.elapsed_time(e1) / 1e3)
            sweep.append({"tau": ts, "solves_per_s": 3 / sum(tt), "resid_F": rs["resid_F"],
                          "tasks": rs["tasks_total"], "volume_pct": 100.0 * rs["tasks_total"] / rs["tasks_dense"],
                          "gate_met": bool(rs["resid_F"] <= GATE), "status": sp.STATUS.get(rs["status"]),
                          "_out": out_s})

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel (the leaf-product kernel).  Its per-launch duration comes from profiled
    # solves (branches serialised, events around each launch); its time per unprofiled solve is that average
    # times the launches of one solve, next to ms_per_step.  In the unprofiled solve the Y and Z products run
    # on two branches at once, so the kernel-time sum can exceed the solve's critical path.
    ms_per_step = 1e3 * tot_max / args.steps
    avg_ms = gemm_ms / max(1, gemm_launches)
    flops_per_launch = gemm_flops / max(1, gemm_launches)
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
    launches_per_solve = gemm_launches / n_prof
    kernel_ms_per_solve = avg_ms * launches_per_solve
    if prec == sp.FP64:
        peak = measure_dgemm_tflops(torch, dev)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": None,
                "kernel": f"k_gemm_f64<{LEAF}>",
                "peak_source": "cuBLAS FP64 GEMM 4096^3 measured in this run (FP64 pipe)",
                "avg_launch_ms": avg_ms, "launches_per_solve": launches_per_solve,
                "kernel_ms_per_solve": kernel_ms_per_solve, "share_of_step": kernel_ms_per_solve / ms_per_step}
    else:
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
        peak = peaks.get("bf16_tflops", 1900.0)
        # the FP16 tensor work the kernel issued, as it counts it: (stack, slice) units of 2*128*64*64 flop,
        # 12 per task
        per_launch = tensor_units * (2.0 * 128 * 64 * 64) / max(1, gemm_launches)
        issued = per_launch / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        tasks_per_launch = gemm_flops / max(1, gemm_launches) / (2.0 * LEAF ** 3)
        roof = {"bound": "tensor", "achieved": issued, "peak": peak, "unit": "TFLOP/s",
                "frac": issued / peak if peak else None,
                "traffic": captured_traffic("k_gemm_emu", tasks_per_launch), "kernel": "spamm::emu::k_gemm_emu",
                "achieved_counts": "FP16 tensor-pipe flops issued (counted by the kernel: 2*128*64*64 per (stack, "
                                   "slice) unit, 12 units per task: 24x the FP64-equivalent useful flops)",
                "units_per_task": tensor_units / max(1.0, tasks_per_launch * gemm_launches),
                "useful_fp64_equiv_tflops": achieved,
                "useful_frac": achieved / peak if peak else None,
                "peak_source": ("bf16_tflops of measured x 1.0 (FP16 and BF16 dense rates are equal)" if peaks
                                else "fallback 1.9 PFLOP/s"),
                "avg_launch_ms": avg_ms, "launches_per_solve": launches_per_solve,
                "kernel_ms_per_solve": kernel_ms_per_solve, "share_of_step": kernel_ms_per_solve / ms_per_step}

    # the norm-tree, cull and slicing kernels of the products: algorithmic bytes per launch over their mean
    # duration.  m tiles per side; cull: both operands' leaf norms read (2 * 8 m^2), task counts written
    # (4 m^2) and 4 bytes per surviving task; tree: the leaf level read (8 m^2) and the upper levels written
    # (8 m^2 / 3).
    m = (N + LEAF - 1) // LEAF
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = (json.load(open(peaks_path)).get("hbm_gbs") if os.path.exists(peaks_path) else None) or 6800.0
    tasks_per_product = vst["tasks_total"] / max(1, 3 * vst["iters"])
    setup = {"peak_gbs": hbm, "peak_source": "hbm_gbs of measured" if os.path.exists(peaks_path) else "fallback"}
    for k, nbytes in (("cull", 20.0 * m * m + 4.0 * tasks_per_product), ("tree", 8.0 * m * m * 4.0 / 3.0),
                      ("slice", None)):
        ms_k, cnt_k = phase[k]
        if cnt_k == 0:
            continue
        avg_k = ms_k / cnt_k
        rec = {"avg_launch_us": 1e3 * avg_k, "launches_per_solve": cnt_k / n_prof,
               "ms_per_solve": avg_k * cnt_k / n_prof}
        if nbytes is not None:
            gbs = nbytes / (avg_k / 1e3) / 1e9
            rec.update({"bytes_per_launch": nbytes, "achieved_gbs": gbs, "frac": gbs / hbm})
        setup[k] = rec

    import oracle
    oracle.build()
    cpu = None
    ref = None
    if not args.no_cpu_baseline and ws == 1:
        rate, cnt, el, ref = oracle_solve_rate(S, tau, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{cnt} full solve(s) of the same workload in {el:.1f} s"}
    # error of every reported GPU result against the oracle's solve of the same input
    oracle_err = None
    if not args.no_oracle_error:
        if ref is None:
            ref = oracle.sqrt_invsqrt(S, LEAF, tau, MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
        oracle_err = err_vs_oracle(Yv, Zv, vst, ref)
        if fp64_path is not None:
            fy, fz, fst = fp64_path["_out"]
            fp64_path["err_vs_oracle"] = err_vs_oracle(fy, fz, fst, ref)
        for row in sweep:
            sy, sz, sst = row["_out"]
            row["err_vs_oracle"] = err_vs_oracle(sy, sz, sst, oracle.sqrt_invsqrt(S, LEAF, row["tau"], MAXIT, map=MAP,
                                                                                   tol_t=TOL, channel=CHANNEL))
    if fp64_path is not None:
        fp64_path.pop("_out", None)
    for row in sweep:
        row.pop("_out", None)

    nbytes = N * N * 8
    p50 = statistics.median(step_s) * 1e3
    p99 = sorted(step_s)[min(len(step_s) - 1, int(math.ceil(0.99 * len(step_s))) - 1)] * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == sp.FP64 else "f16-split",
            "data": "synthetic",
            "config": {"workload": workload_name(tau, args.precision.upper()), "n": N, "leaf": LEAF, "tau": tau,
                       "tau_s": 0.01 * tau, "maxit": MAXIT, "tol_t": TOL, "precision": args.precision,
                       "map": args.map, "channel": args.channel,
                       "l2": "flushed by a 256 MB write before every timed solve",
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": p50, "p99": p99},
            "resid_F": vst["resid_F"], "gate": GATE, "gate_met": bool(vst["resid_F"] <= GATE),
            "tasks_per_solve": vst["tasks_total"], "volume_pct": 100.0 * vst["tasks_total"] / vst["tasks_dense"],
            "t_final": vst["t_final"], "iters": vst["iters"], "status": sp.STATUS.get(vst["status"]),
            "err_vs_oracle": oracle_err,
            "err_tolerance": {"Z": 1e-9 if prec == sp.EMU64 else 1e-10, "Y": 1e-9 if prec == sp.EMU64 else 1e-10},
            "roofline": roof,
            "norm_cull_kernels": setup,
            "fp64_path": fp64_path,
            "schedules": schedules,
            "to_tolerance": to_tol,
            "lensing": lensing,
            "cpu_baseline": cpu,
            "e2e": {"value": job_rate(ws, args.steps, e2e_tot), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": 2 * nbytes},
            "gpu_launches": launches,
            "clocks": clk,
            "tau_sweep": sweep}
    if ws == 1 and not args.no_extra:
        # the other single-GPU configurations, each with its own CPU baseline and errors against the oracle
        del Sd, Yd, Zd, flush, Sh, Yh, Zh
        sp.release()
        torch.cuda.empty_cache()
        extra = {}
        for name, fn in (("c3", lambda: c3_config(args, local, taus=[args.c3_tau_default])),
                         ("c4", lambda: batched_config(args, local)),
                         ("c5", lambda: serve_config(args, local, seq_requests=args.serve_seq))):
            t0 = time.perf_counter()
            extra[name] = fn()
            extra[name]["bench_seconds"] = time.perf_counter() - t0
            sp.release()
            torch.cuda.empty_cache()
        line["configs"] = extra
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def batched_config(args, local) -> dict:
    """Batched configuration: many independent SPD decay matrices of mixed sizes in one call (one graph over
    the whole batch: every stage of the iteration one launch of each kernel over all matrices), against the
    same matrices solved one call at a time; errors against the oracle on a sample of the matrices, and the
    oracle's rate over the same list on the host cores."""
    import numpy as np
    import torch

    import paper_1508_05856_gb300 as sp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = sp.EMU64 if args.precision == "emu64" else sp.FP64
    specs = synth.batch_mix(args.batch, lo=128, hi=2048, seed=0)
    host = [synth.make(sp_) for sp_ in specs]
    Ss = [torch.from_numpy(S).to(dev) for S in host]
    Ys = [torch.empty_like(S) for S in Ss]
    Zs = [torch.empty_like(S) for S in Ss]
    taus = [args.batch_tau] * len(Ss)
    kw = dict(leaf=LEAF, precision=prec, map=MAP, tol_t=TOL, channel=CHANNEL)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the first call builds the batch (buffers and graph); the timed calls replay it
    _, _, sts = sp.sqrt_invsqrt_batched(Ss, taus, MAXIT, raise_on=False, Ys=Ys, Zs=Zs, **kw)
    torch.cuda.synchronize()
    l0 = sp.kernel_launches()
    tb = []
    for _ in range(args.batch_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, sts = sp.sqrt_invsqrt_batched(Ss, taus, MAXIT, raise_on=False, Ys=Ys, Zs=Zs, **kw)
        e1.record(stream)
        e1.synchronize()
        tb.append(e0.elapsed_time(e1) / 1e3)
    launches = (sp.kernel_launches() - l0) / max(1, args.batch_steps)
    # one call per matrix, the same matrices
    for S, t, Y, Z in list(zip(Ss, taus, Ys, Zs))[:8]:
        sp.sqrt_invsqrt(S, t, MAXIT, raise_on=False, Y=Y, Z=Z, **kw)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for S, t, Y, Z in zip(Ss, taus, Ys, Zs):
        sp.sqrt_invsqrt(S, t, MAXIT, raise_on=False, Y=Y, Z=Z, **kw)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    # errors against the oracle on a sample spread over the sizes, from a fresh batched call
    _, _, sts = sp.sqrt_invsqrt_batched(Ss, taus, MAXIT, raise_on=False, Ys=Ys, Zs=Zs, **kw)
    torch.cuda.synchronize()
    order = np.argsort([S.shape[0] for S in host])
    sample = [int(order[q]) for q in np.linspace(0, len(order) - 1, args.batch_oracle_sample).astype(int)]
    errs = None
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ez, ey, ti = [], [], []
        for q in sample:
            ref = oracle.sqrt_invsqrt(host[q], LEAF, taus[q], MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
            ez.append(rel_err(Zs[q].cpu().numpy(), ref["Z"]))
            ey.append(rel_err(Ys[q].cpu().numpy(), ref["Y"]))
            ti.append(sts[q]["tasks_total"] == int(ref["task_hist"].sum()))
        errs = {"matrices": len(sample), "sizes": [int(host[q].shape[0]) for q in sample], "Z_max": max(ez),
                "Y_max": max(ey), "task_totals_equal": int(sum(ti))}
        # the oracle over the batch list in order, on the host cores, for about cpu_budget seconds
        t0 = time.perf_counter()
        done = 0
        for q in range(len(host)):
            oracle.sqrt_invsqrt(host[q], LEAF, taus[q], MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
            done += 1
            if time.perf_counter() - t0 >= args.batch_cpu_budget:
                break
        el = time.perf_counter() - t0
        cpu = {"value": done / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"the first {done} matrices of the batch list in {el:.1f} s (list order, sizes as drawn)"}
    t_batch = sum(tb) / len(tb)
    out = {"metric": "batched NS solves/s (mixed KMS / 3D Gaussian, N in [128, 2048])", "value": len(Ss) / t_batch,
           "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f64" if prec == sp.FP64 else "f16-split",
           "data": "synthetic",
           "config": {"workload": f"{len(Ss)} matrices, sizes log-uniform in [128, 2048] (multiples of 32), "
                                  f"50% KMS rho~U(0.5,0.95), 50% Gaussian sigma~U(0.6,0.9), tau={args.batch_tau:g}, "
                                  + (f"{MAXIT} iterations" if TOL <= 0
                                     else f"until |t_k| <= {TOL:g} (at most {MAXIT})"),
                      "precision": args.precision, "map": args.map, "channel": args.channel,
                      "l2": "flushed by a 256 MB write before every timed batch"},
           "ms_per_batch": 1e3 * t_batch, "timed_batches": len(tb), "gpu_launches_per_batch": launches,
           "one_call_per_matrix": {"value": len(Ss) / t_seq, "unit": UNIT},
           "tasks": int(sum(st["tasks_total"] for st in sts)),
           "iters_mean": float(sum(st["iters"] for st in sts)) / max(1, len(sts)),
           "call_status": sp.STATUS.get(sts[0]["call_status"]),
           "err_vs_oracle": errs, "cpu_baseline": cpu}
    del Ss, Ys, Zs, flush
    torch.cuda.empty_cache()
    return out


def run_batched(args, local):
    print(json.dumps(batched_config(args, local)), flush=True)
    return 0


def serve_config(args, local, requests=None, seq_requests=None) -> dict:
    """Serving configuration: Poisson arrivals of square-root requests on 3D Gaussian-decay matrices, served by
    the request server (queued device-resident requests are solved together, sharing every launch); p50/p99
    latency from arrival to completion and solves/s, against the same requests solved one at a time.

    Each request's matrix is built on the device when it arrives, from its own seeded point set (input
    generation, not part of the solve).  The client keeps at most --serve-outstanding-gb of request matrices
    (S, Y, Z) alive; a request arriving beyond that waits on the client and its wait counts in its latency."""
    import collections

    import numpy as np
    import torch

    import paper_1508_05856_gb300 as sp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = sp.EMU64 if args.precision == "emu64" else sp.FP64
    R = requests or args.requests
    trace = synth.serving_trace(R, rate=args.rate, lo=256, hi=args.serve_max_n, seed=0)

    def make(r):
        # S_ij = exp(-|r_i - r_j|^2 / (2 sigma^2)), built in row blocks; finished before the request is
        # handed to the server, whose workers run on their own streams
        pts = torch.from_numpy(synth.lattice_points(r["n"], r["seed"])).to(dev)
        n = r["n"]
        S = torch.empty((n, n), dtype=torch.float64, device=dev)
        c = -1.0 / (2.0 * r["sigma"] * r["sigma"])
        for a in range(0, n, 2048):
            d = pts[a:a + 2048, None, :] - pts[None, :, :]
            S[a:a + 2048] = torch.exp((d * d).sum(-1) * c)
        torch.cuda.current_stream(dev).synchronize()
        return S

    cap = int(args.serve_outstanding_gb * (1 << 30))
    nbytes = [3 * r["n"] * r["n"] * 8 for r in trace]
    lat = [0.0] * R
    status = [None] * R
    keep_out = {}
    sample = {q for q in range(R) if trace[q]["n"] <= 1024 and q < 200}
    sample = set(sorted(sample)[:args.serve_oracle_sample])
    with sp.Server(bytes_budget=int(args.budget_gb * (1 << 30)), max_active=args.max_active, leaf=LEAF,
                   precision=prec) as srv:
        for r in trace[:4]:
            srv.wait(srv.submit(make(r), r["tau"], MAXIT), raise_on=False)     # warm-up
        torch.cuda.synchronize()
        pending = collections.deque()
        outstanding = {}
        out_bytes = 0
        nxt = 0
        t0 = time.perf_counter()
        t_last = t0
        while nxt < R or pending or outstanding:
            now = time.perf_counter() - t0
            while nxt < R and trace[nxt]["arrival"] <= now:
                pending.append(nxt)
                nxt += 1
            busy = False
            while pending and (out_bytes + nbytes[pending[0]] <= cap or not outstanding):
                q = pending.popleft()
                S = make(trace[q])
                rid = srv.submit(S, trace[q]["tau"], MAXIT)
                outstanding[rid] = (q, time.perf_counter() - t0, S)
                out_bytes += nbytes[q]
                busy = True
            for rid in list(outstanding):
                if srv.poll(rid) == 2:
                    q, t_sub, S = outstanding.pop(rid)
                    Y, Z, st, l = srv.wait(rid, raise_on=False)
                    lat[q] = t_sub + l - trace[q]["arrival"]
                    status[q] = st["status"]
                    t_last = max(t_last, t0 + t_sub + l)
                    if q in sample:
                        keep_out[q] = (S.cpu().numpy(), Y.cpu().numpy(), Z.cpu().numpy())
                    out_bytes -= nbytes[q]
                    busy = True
            if not busy:
                time.sleep(0.0005)
        t_all = t_last - (t0 + trace[0]["arrival"])
    # the same requests one at a time (a prefix of the trace when the run asks for fewer)
    Rs = min(R, seq_requests or R)
    seq_status = []
    seq_lat = []
    same_out = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(Rs):
        a = time.perf_counter()
        S = make(trace[q])
        Y, Z, st = sp.sqrt_invsqrt(S, trace[q]["tau"], MAXIT, leaf=LEAF, precision=prec, raise_on=False, map=MAP,
                                   tol_t=TOL, channel=CHANNEL)
        torch.cuda.synchronize()
        seq_lat.append(time.perf_counter() - a)
        seq_status.append(st["status"])
        if q in keep_out:
            same_out += int(np.array_equal(keep_out[q][1], Y.cpu().numpy()) and
                            np.array_equal(keep_out[q][2], Z.cpu().numpy()))
        del S, Y, Z
    t_seq = time.perf_counter() - t0
    errs = None
    if keep_out and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ez = []
        for q, (S, Y, Z) in sorted(keep_out.items()):
            ref = oracle.sqrt_invsqrt(S, LEAF, trace[q]["tau"], MAXIT, map=MAP, tol_t=TOL, channel=CHANNEL)
            ez.append(max(rel_err(Z, ref["Z"]), rel_err(Y, ref["Y"])))
        errs = {"requests": len(ez), "max_rel_err_YZ": max(ez)}
    la = np.array(lat) * 1e3
    out = {"metric": "served NS requests: solves/s with p50/p99 latency", "value": R / t_all, "unit": UNIT,
           "n_gpus": 1, "higher_is_better": True, "dtype": "f64" if prec == sp.FP64 else "f16-split",
           "data": "synthetic",
           "config": {"workload": f"{R} requests, Poisson arrivals at {args.rate:g}/s, N log-uniform in "
                                  f"[256, {args.serve_max_n}] (multiples of 32), 3D Gaussian decay sigma~U(0.6,0.9) "
                                  f"on each request's own seeded lattice, tau in {{1e-4, 1e-6, 1e-8}}, {MAXIT} "
                                  "iterations", "max_active": args.max_active, "budget_gb": args.budget_gb,
                      "client_outstanding_gb": args.serve_outstanding_gb, "precision": args.precision,
                      "map": args.map},
           "latency_ms": {"p50": float(np.percentile(la, 50)), "p99": float(np.percentile(la, 99)),
                          "from": "arrival to completion"},
           "requests": {"ok": int(sum(1 for x in status if x == 0)),
                        "diverged": int(sum(1 for x in status if x == -3)),
                        "other_error": int(sum(1 for x in status if x not in (0, -3))),
                        "same_status_as_alone": bool(status[:Rs] == seq_status),
                        "status_mismatches": [{"q": q, "n": trace[q]["n"], "tau": trace[q]["tau"],
                                               "served": status[q], "alone": seq_status[q]}
                                              for q in range(Rs) if status[q] != seq_status[q]][:10],
                        "bitwise_same_as_alone": f"{same_out} of {len([q for q in keep_out if q < Rs])} sampled"},
           "one_request_at_a_time": {"value": Rs / t_seq, "unit": UNIT, "requests": Rs,
                                     "p50_service_ms": float(np.percentile(np.array(seq_lat) * 1e3, 50))},
           "err_vs_oracle": errs}
    torch.cuda.empty_cache()
    return out


def run_serve(args, local):
    print(json.dumps(serve_config(args, local)), flush=True)
    return 0


def c3_config(args, local, taus=None) -> dict:
    """Large configuration: 3D Gaussian decay on N jittered Morton-ordered lattice points (default N = 16384),
    N_b = 64, one or more tau, optional Tikhonov shift mu = mu_rel * c.  Solves/s, residual and cull volume per
    tau.  The oracle cannot solve this size in the time of a run: its rate is the measured time of a random
    sample of the solve's own leaf products, scaled by the solve's task count (labelled extrapolated), and the
    GPU result is checked by properties that hold at any size: ||ZSZ - I||_F (FP64, dense) and Y^2 = S on a
    sample of rows."""
    import numpy as np
    import torch

    import paper_1508_05856_gb300 as sp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = sp.EMU64 if args.precision == "emu64" else sp.FP64
    taus = list(taus if taus is not None else args.c3_tau)
    S = synth.gaussian_lattice(args.c3_n, args.c3_sigma, seed=0)
    Sd = torch.from_numpy(S).to(dev)
    Yd, Zd = torch.empty_like(Sd), torch.empty_like(Sd)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(0)
    rows = torch.from_numpy(np.sort(rng.choice(args.c3_n, size=64, replace=False))).to(dev)
    rows_out = []
    for tau in taus:
        kw = dict(leaf=LEAF, precision=prec, Y=Yd, Z=Zd, mu_rel=args.c3_mu, map=MAP, tol_t=TOL, channel=CHANNEL,
                  raise_on=False)
        _, _, vst = sp.sqrt_invsqrt(Sd, tau, MAXIT, residual=True, **kw)
        # Y^2 = S on 64 sampled rows, FP64 (verification only; without a shift)
        y2 = float(torch.linalg.norm(Yd[rows] @ Yd - Sd[rows]) / torch.linalg.norm(Sd[rows]))
        sp.sqrt_invsqrt(Sd, tau, MAXIT, **kw)
        ts = []
        for _ in range(args.c3_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sp.sqrt_invsqrt(Sd, tau, MAXIT, **kw)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        rows_out.append({"tau": tau, "solves_per_s": len(ts) / sum(ts), "ms_per_solve": 1e3 * sum(ts) / len(ts),
                         "resid_F": vst["resid_F"], "gate_met": bool(vst["resid_F"] <= GATE),
                         "y2_rows_rel_err": y2 if not args.c3_mu else None,
                         "tasks": vst["tasks_total"], "volume_pct": 100.0 * vst["tasks_total"] / vst["tasks_dense"],
                         "iters": vst["iters"], "t_final": vst["t_final"], "status": sp.STATUS.get(vst["status"])})
    best = max((r for r in rows_out if r["gate_met"]), key=lambda r: r["solves_per_s"], default=rows_out[-1])
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # a random sample of the leaf products of one product of the solve (X0 X0 at the best tau), timed in
        # the oracle, per task, times the solve's tasks
        c = oracle.gershgorin(S)
        X0 = S * (1.0 / c)
        X0d = torch.from_numpy(X0).to(dev)
        tasks, _, ntask = sp.cull(X0d, X0d, best["tau"], LEAF)
        del X0d
        pick = tasks[rng.choice(len(tasks), size=min(len(tasks), args.c3_oracle_tasks), replace=False)]
        t0 = time.perf_counter()
        oracle.leaf_products(X0, X0, LEAF, pick)
        el = time.perf_counter() - t0
        per_task = el / len(pick)
        cpu = {"value": 1.0 / (per_task * best["tasks"]), "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle", "extrapolated": True,
               "sample": f"{len(pick)} leaf products of X0 (x) X0 at tau={best['tau']:g} in {el:.2f} s, scaled to "
                         f"the solve's {best['tasks']} leaf products (the culls, trees and maps left out)"}
    out = {"metric": f"NS solves/s at ||ZSZ-I||_F<=1e-8 (3D Gaussian N={args.c3_n})", "value": best["solves_per_s"],
           "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
           "dtype": "f64" if prec == sp.FP64 else "f16-split", "data": "synthetic",
           "config": {"workload": f"3D Gaussian decay sigma={args.c3_sigma} on {args.c3_n} jittered Morton-ordered "
                                  f"lattice points, N_b={LEAF}, "
                                  + (f"{MAXIT} iterations" if TOL <= 0
                                     else f"until |t_k| <= {TOL:g} (at most {MAXIT})")
                                  + f", mu_rel={args.c3_mu}",
                      "precision": args.precision, "map": args.map, "channel": args.channel,
                      "tau_best": best["tau"], "l2": "flushed by a 256 MB write before every timed solve"},
           "per_tau": rows_out, "cpu_baseline": cpu}
    del Sd, Yd, Zd, flush
    torch.cuda.empty_cache()
    return out


def run_c3(args, local):
    print(json.dumps(c3_config(args, local)), flush=True)
    return 0


def run_product_rep(args, local):
    """Product representation of the regularised inverse factor (Sec. 6): slices at tau0 with shifts mus
    (relative to the Gershgorin bound), residual products at tau1, on a 3D Gaussian decay; against one
    regularised NS solve to the last shift.  The residual ||Z^T (S + mu_last c0 I) Z - I||_F is checked
    outside the timed region with dense FP64 products."""
    import torch

    import paper_1508_05856_gb300 as sp
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = sp.EMU64 if args.precision == "emu64" else sp.FP64
    n, mus, tau0, tau1 = args.pr_n, args.pr_mu, args.pr_tau0, args.pr_tau1
    S = synth.gaussian_lattice(n, args.pr_sigma, seed=0)
    Sd = torch.from_numpy(S).to(dev)
    Zd = torch.empty_like(Sd)
    Yd = torch.empty_like(Sd)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    c0 = float(Sd.abs().sum(dim=1).max())
    Smu = Sd + mus[-1] * c0 * torch.eye(n, dtype=torch.float64, device=dev)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return ts

    def resid(Z):
        M = Z.T @ Smu @ Z
        return float(torch.linalg.norm(M - torch.eye(n, dtype=torch.float64, device=dev)))

    def kappa(M):
        ev = torch.linalg.eigvalsh(0.5 * (M + M.T))
        return float(ev.max() / ev.min()) if float(ev.min()) > 0 else float("inf")

    kappa_s = kappa(Smu)

    kw = dict(leaf=LEAF, precision=prec, map=MAP, channel=CHANNEL, tol_t=TOL, raise_on=False)
    _, info = sp.invsqrt_product(Sd, mus, tau0, tau1, MAXIT, Z=Zd, **kw)
    r_prod = resid(Zd)
    k_prod = kappa(Zd.T @ Smu @ Zd)
    ts = timed(lambda: sp.invsqrt_product(Sd, mus, tau0, tau1, MAXIT, Z=Zd, **kw), args.steps)
    # one regularised solve to the last shift at the products' threshold, for comparison
    _, _, st1 = sp.sqrt_invsqrt(Sd, tau1, MAXIT, Y=Yd, Z=Zd, mu_rel=mus[-1], **kw)
    r_one = resid(Zd)
    k_one = kappa(Zd.T @ Smu @ Zd)
    t1 = timed(lambda: sp.sqrt_invsqrt(Sd, tau1, MAXIT, Y=Yd, Z=Zd, mu_rel=mus[-1], **kw), args.steps)
    line = {"metric": f"product representation of (S + mu I)^-1/2 per second (3D Gaussian N={n})",
            "value": len(ts) / sum(ts), "unit": "factors/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64" if prec == sp.FP64 else "f16-split", "data": "synthetic",
            "config": {"workload": f"3D Gaussian decay sigma={args.pr_sigma} on {n} jittered Morton-ordered lattice "
                                   f"points, N_b={LEAF}, slices at tau0={tau0:g} with shifts {mus} x Gershgorin "
                                   f"bound, residual products at tau1={tau1:g}, {MAXIT} iterations per slice",
                       "precision": args.precision, "levels": len(mus)},
            "ms_per_factor": 1e3 * sum(ts) / len(ts), "slice_iters": info["iters"], "status": info["status"],
            "resid_F": r_prod, "kappa_S_mu": kappa_s, "kappa_ZtSZ": k_prod,
            "single_solve": {"value": len(t1) / sum(t1), "unit": "solves/s", "tau": tau1, "mu_rel": mus[-1],
                             "resid_F": r_one, "kappa_ZtSZ": k_one, "iters": st1["iters"], "status": st1["status"]}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    global N, MAXIT, MAP, TOL, CHANNEL
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "emu64"], default="emu64",
                    help="leaf-product arithmetic: emu64 (FP64-class products on the BF16 tensor cores, the "
                         "default) or fp64 (FP64 pipe)")
    ap.add_argument("--tau", type=float, default=TAU_HEADLINE)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--size", type=int, default=N, help="matrix size N (a smaller case for profiler captures)")
    ap.add_argument("--maxit", type=int, default=MAXIT, help="iterations per solve (fewer for profiler captures)")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the FP64-pipe solve beside EMU64")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the oracle solves that give every result's error against the oracle")
    ap.add_argument("--c3", action="store_true", help="large 3D Gaussian configuration instead of the headline solve")
    ap.add_argument("--emu-layout", choices=["auto", "fixed", "alternating"], default="auto",
                    help="accumulator layout of the tensor-core leaf products (auto: alternating from 128 tiles "
                         "per side); both give the same bits")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: leave out the large, batched and served configurations")
    ap.add_argument("--c3-tau-default", type=float, default=1e-15,
                    help="tau of the large configuration inside the default run (the largest meeting the gate)")
    ap.add_argument("--serve-seq", type=int, default=500,
                    help="requests of the trace also solved one at a time inside the default run")
    ap.add_argument("--c3-n", type=int, default=16384)
    ap.add_argument("--c3-sigma", type=float, default=0.7)
    ap.add_argument("--c3-tau", type=float, nargs="+", default=[1e-10, 1e-12, 1e-14])
    ap.add_argument("--c3-mu", type=float, default=0.0)
    ap.add_argument("--c3-steps", type=int, default=2)
    ap.add_argument("--c3-oracle-tasks", type=int, default=3000,
                    help="leaf products the oracle times for the extrapolated CPU rate")
    ap.add_argument("--batched", action="store_true", help="batched configuration instead of the headline solve")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--batch-tau", type=float, default=1e-6)
    ap.add_argument("--batch-steps", type=int, default=3, help="timed batched calls")
    ap.add_argument("--batch-oracle-sample", type=int, default=6, help="matrices compared with the oracle")
    ap.add_argument("--batch-cpu-budget", type=float, default=8.0, help="seconds of oracle time over the list")
    ap.add_argument("--serve", action="store_true", help="serving configuration instead of the headline solve")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--serve-outstanding-gb", type=float, default=96.0,
                    help="request matrices (S, Y, Z) the client keeps alive at most")
    ap.add_argument("--serve-oracle-sample", type=int, default=4, help="small requests compared with the oracle")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--serve-max-n", type=int, default=8192)
    ap.add_argument("--max-active", type=int, default=2)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--map", choices=["ns", "scaled"], default="ns",
                    help="NS map: alpha = 1, or the damped, stabilised h_alpha of Sec. 4.2")
    ap.add_argument("--tol-t", type=float, default=0.0,
                    help="stop a solve once |t_k| <= tol (Sec. 4.2 trace error); 0 runs exactly --maxit steps")
    ap.add_argument("--channel", choices=["dual", "single"], default="dual",
                    help="instance of the iteration: dual channel, Eq. (cannonical), or single, Eq. (single)")
    ap.add_argument("--product-rep", action="store_true",
                    help="product representation of the regularised inverse factor (Sec. 6) instead of the headline")
    ap.add_argument("--pr-n", type=int, default=4096)
    ap.add_argument("--pr-sigma", type=float, default=0.9)
    ap.add_argument("--pr-mu", type=float, nargs="+", default=[0.1, 0.01, 0.001])
    ap.add_argument("--pr-tau0", type=float, default=1e-3)
    ap.add_argument("--pr-tau1", type=float, default=1e-5)
    ap.add_argument("--lens-bins", type=int, default=0,
                    help="also profile the products' volumes about the plane diagonals (Sec. 7.2), this many bins")
    ap.add_argument("--lens-npz", default="", help="write the full plane-diagonal profile to this .npz")
    ap.add_argument("--tol-report", type=float, default=1e-12,
                    help="with fixed-step solves, also time solves stopped at |t_k| <= this (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    N, MAXIT = args.size, args.maxit
    MAP = 1 if args.map == "scaled" else 0
    TOL = args.tol_t
    CHANNEL = 1 if args.channel == "single" else 0
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.emu_layout != "auto" and args.impl != "reference":
        import paper_1508_05856_gb300 as sp
        sp.lib().spamm_test_emu_alternate(1 if args.emu_layout == "alternating" else 0)
    if args.c3:
        return run_c3(args, local)
    if args.product_rep:
        return run_product_rep(args, local)
    if args.batched:
        return run_batched(args, local)
    if args.serve:
        return run_serve(args, local)
    return run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
