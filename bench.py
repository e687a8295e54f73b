#!/usr/bin/env python
"""Throughput benchmark: Tersoff MD on one GB300 (mixed and FP64 paths).

Workload: Si diamond 40x40x40 cubic cells (512,000 atoms, a = 5.432 A),
Gaussian displacements sigma = 0.05 A, Maxwell velocities at 1000 K,
velocity-Verlet NVE with dt = 1 fs, neighbour list radius 4.0 A (cutoff 3.0 A
+ skin 1.0 A) rebuilt every 10 steps. One benchmark step = one rebuild period
= 10 MD steps (kick, drift, [rebuild], forces, kick), so every step includes
one neighbour build. Metric: atom-steps/s = atoms x MD steps / device time.

The L2 cache is flushed (a 512 MiB write) before every timed step, outside the
timed events. With N GPUs (torchrun) each rank runs its own replica of the
workload (the metric's workload is one periodic cell; there is no data-path
collective); value = all ranks' atom-steps / slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Tersoff atom-steps/s on 1 GB300, mixed vs FP64 path, at stated force error"
UNIT = "atom-steps/s"
MD_PER_STEP = 10
DT = 0.001
R_LIST = 4.0
RC_SI = 3.0  # largest f_C outer cutoff of the Tersoff 1989 Si / C tables (R + D)
NPARAM_TABLE_SI = 14
# Derived from unit counts and the maximum clock, for cross-checking the
# measured peaks (tersoff_pipe_peaks: FFMA, DFMA and MUFU loop kernels, run at
# the start of every benchmark); the roofline fractions use the measured ones.
PEAK_FP32_TFLOPS_DERIVED = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
PEAK_ISSUE_WARP_INST = 152 * 4 * 2.07e9  # SMs x schedulers (one warp instruction each) x clock
# warp instructions of one force launch on this workload (ncu smsp__inst_executed.sum, the same
# capture as the traffic); like the traffic, valid only for the sources it was taken with
FORCE_WARP_INST = 25_201_239

# Algorithmic FP32 operations of the force evaluation per unit of work
# (additions and multiplications, an FMA counting 2; special-function ops
# counted separately): per bond inside the cutoffs (bond vector, length, unit
# vector, its share of the force and virial epilogue), per pair term and per
# three-body term. The filter pass over the skin list (FLOP_SKIN per entry)
# is not the method's work and is reported on its own.
FLOP_SKIN, FLOP_SHORT, FLOP_PAIR, FLOP_TRIPLET = 15, 36, 63, 61
MUFU_SHORT, MUFU_PAIR, MUFU_TRIPLET = 1, 7, 1

# DRAM bytes (read + write) of one launch of the mixed force kernel on this
# workload, from an ncu capture (profiles/k_tersoff_si512k_mixed.md). Valid only
# for the kernel sources it was taken with, identified by their SHA-256; once
# those change the traffic is reported as null until it is measured again.
FORCE_TRAFFIC_BYTES = 23_687_680 + 2_466_048
FORCE_TRAFFIC_SOURCES = ("tersoff_fwd.cuh", "fwd_launch.cuh", "fwd_f32.cu")
FORCE_TRAFFIC_SHA256 = "5efc65b2dcff08db97c3937c7257cb7f397ef6382c488f13dc0b93038baad181"


def mufu_peak(pk):
    """Largest measured special-function rate (1e12 ops/s): a lower bound on
    the time of any mix of rsqrt, ex2 and lg2."""
    return max(pk["rsqrt_tops"], pk["ex2_tops"], pk["lg2_tops"])


def ceilings_us(flop, mufu, peaks, pk, kern_ms):
    """Lower bounds on one force launch (us) from each resource, beside the
    measured time: FP32 arithmetic (the FLOP model over the measured FFMA
    peak), special-function operations (over the measured MUFU rate), DRAM
    traffic (ncu bytes over the measured copy bandwidth), and instruction issue
    (ncu warp instructions over 4 per SM per clock)."""
    out = {"fp32_flops": flop / (pk["fp32_tflops"] * 1e12) * 1e6,
           "mufu": mufu / (mufu_peak(pk) * 1e12) * 1e6,
           "measured": kern_ms * 1e3}
    tr = force_traffic()
    if tr is not None and peaks.get("hbm_gbs"):
        out["dram"] = tr / (peaks["hbm_gbs"] * 1e9) * 1e6
        out["issue"] = FORCE_WARP_INST / PEAK_ISSUE_WARP_INST * 1e6
    return out


def force_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in FORCE_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1607_02904_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return FORCE_TRAFFIC_BYTES if h.hexdigest() == FORCE_TRAFFIC_SHA256 else None


def workload_name():
    return ("si-diamond-40x40x40-512000-atoms-1000K-dt1fs-rlist4.0-rebuild10-"
            "10-md-steps-per-step")


def chosen_options(summary):
    """The options of an autotuner summary ("chosen scatter=... split=...
    waves=... block=... (...)") as a dict."""
    head = summary.split("(")[0].replace("chosen", "").split()
    return dict(kv.split("=") for kv in head)


def apply_options(ctx, T, opt):
    ctx.set_scatter(T.SCATTER_ATOMIC if opt["scatter"] == "atomic" else T.SCATTER_GATHER)
    split = {"auto": -1, "off": 0, "on": 1}[opt["split"]]
    ctx.set_launch(int(opt["waves"]), split, int(opt["block"]))
    ctx.set_lanes({"auto": 0, "1": 1, "4": 4}[opt.get("lanes", "auto")])


def base_config(n, world):
    return {"workload": workload_name(), "atoms_per_gpu": n, "md_steps_per_step": MD_PER_STEP,
            "dt_ps": DT, "neighbor_rebuild_every": MD_PER_STEP, "r_list_A": R_LIST,
            "l2": "flushed before each timed step (512 MiB write, outside the timed events)",
            "parallelism": f"replicas x{world}"}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_ms: float, local_units: float, world: int):
    """Max of the per-rank times and the sum of units over ranks."""
    if world == 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        """Starts sampling and waits until the first sample is written, so the
        sampler's start-up does not fall inside the timed region."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for _, _, r in rows for q in range(4) if r[q] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def smi_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].strip().isdigit():
            return int(ids[local_rank])
    return local_rank


def work_counts(x, types, box, cnt, nbr, table, ns):
    """Skin entries, short-list entries, pairs and three-body terms inside their
    cutoffs (FLOP model bookkeeping, from the library's exported list)."""
    import numpy as np
    t = np.asarray(table).reshape(ns, ns, ns, 14)
    rout = t[..., 10] + t[..., 11]  # R + D per record
    n = x.shape[0]
    mask = nbr >= 0
    j = np.where(mask, nbr, 0)
    d = x[j] - x[:, None, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(-1))
    ti = types[:, None]
    tj = types[j]
    pair_cut = rout[ti, tj, tj]
    filt = np.zeros((ns, ns))
    for a in range(ns):
        for b in range(ns):
            filt[a, b] = max(rout[a, b, b], rout[a, :, b].max())
    short = mask & (r <= filt[ti, tj])
    pairs = short & (r < pair_cut)
    skin = int(mask.sum())
    nshort = int(short.sum())
    npair = int(pairs.sum())
    # three-body terms: ordered (j, k), j in pairs, k short and inside its cutoff
    trip = 0
    zmax = int(short.sum(1).max()) if n else 0
    order = np.argsort(~short, axis=1, kind="stable")[:, :zmax]
    rs = np.take_along_axis(r, order, 1)
    ok = np.take_along_axis(short, order, 1)
    okp = np.take_along_axis(pairs, order, 1)
    tjs = np.take_along_axis(tj, order, 1)
    for qj in range(zmax):
        for qk in range(zmax):
            if qj == qk:
                continue
            cut = rout[types, tjs[:, qj], tjs[:, qk]]
            trip += int((okp[:, qj] & ok[:, qk] & (rs[:, qk] < cut)).sum())
    return skin, nshort, npair, trip


def run_ours(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_1607_02904_gb300 as T

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cells, gen_s = (generate_batch_cells(W) if (rank == 0 and not args.no_extra)
                    else (None, 0.0))
    x, v, t, box, names = W.config_si_md()
    n = x.shape[0]
    table = T.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def setup(prec):
        ctx = T.Context(prec)
        ctx.params(table)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        vd = torch.tensor(v, dtype=torch.float64, device=dev)
        td = torch.tensor(t, dtype=torch.int32, device=dev)
        ctx.neighbor_build(xd, td, box, R_LIST)
        fd = torch.zeros_like(xd)
        e = torch.zeros(1, dtype=torch.float64, device=dev)
        w = torch.zeros(6, dtype=torch.float64, device=dev)
        ctx.compute(xd, e, fd, w)
        return ctx, xd, vd, td, fd, e, w

    def timed(ctx, xd, vd, fd, steps, warmup, sampler=None, instrument=False):
        """Sum of per-step device times (CUDA events on the launching stream,
        L2 flushed before each step). instrument: also record CUDA events
        around the force kernel, neighbour builds and integration kernels
        inside the steps (this slows the steps, so it is a separate pass)."""
        for _ in range(warmup):
            ctx.md_step(xd, vd, fd, mass, DT, MD_PER_STEP, MD_PER_STEP)
        torch.cuda.synchronize()
        ctx.set_timing(instrument)
        l0 = ctx.launch_count()
        stream = torch.cuda.current_stream()
        ms = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.md_step(xd, vd, fd, mass, DT, MD_PER_STEP, MD_PER_STEP)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop() if sampler else None
        launches = ctx.launch_count() - l0
        kern = ctx.timing(0)
        build = ctx.timing(1)
        integ = ctx.timing(2)
        ctx.set_timing(False)
        return sum(ms), launches, kern, build, integ, clocks

    # arithmetic-pipe peaks of this device, measured now (loop kernels)
    pk = T.pipe_peaks()
    out = {}
    # ---------------- accuracy of the mixed path against the FP64 path (same start)
    ctx64, xd64, vd64, td, f64, e64, w64 = setup(T.FP64)
    ctxm, xdm, vdm, _, fm, em, wm = setup(T.MIXED)
    torch.cuda.synchronize()
    fr = f64.cpu().numpy()
    fmm = fm.cpu().numpy()
    force_rms_rel = float(np.sqrt(((fmm - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean()))
    energy_rel = float(abs(em.item() - e64.item()) / abs(e64.item()))
    virial_rel = float((wm - w64).abs().max().item() / w64.abs().max().item())

    # FLOP model inputs from the exported skin list
    cap, mx = ctxm.neighbor_capacity()
    cnt, nbr, _ = ctxm.neighbor_export(mx)
    skin, nshort, npair, ntrip = work_counts(x, t, box, cnt.cpu().numpy(), nbr.cpu().numpy(),
                                             table, len(names))
    del cnt, nbr
    flop_launch = FLOP_SHORT * nshort + FLOP_PAIR * npair + FLOP_TRIPLET * ntrip
    filter_flop_launch = FLOP_SKIN * skin
    mufu_launch = MUFU_SHORT * nshort + MUFU_PAIR * npair + MUFU_TRIPLET * ntrip

    # ---------------- launch options chosen by the library's autotuner (MD
    # periods on copies of the state; the timed state is not advanced)
    tune_m = ctxm.autotune(xdm, vdm, mass, DT, MD_PER_STEP)
    tune_d = ctx64.autotune(xd64, vd64, mass, DT, MD_PER_STEP)
    best = chosen_options(tune_m)
    best64 = chosen_options(tune_d)

    # ---------------- timed: mixed (headline), then FP64; then instrumented
    # passes of the same length for the kernel durations
    sampler = ClockSampler(smi_index(local))
    ms_m, launches_m, _, _, _, clocks = timed(ctxm, xdm, vdm, fm, args.steps, args.warmup,
                                              sampler)
    ms_d, launches_d, _, _, _, _ = timed(ctx64, xd64, vd64, f64, args.steps, args.warmup)
    ms_mi, _, kern_m, build_m, integ_m, _ = timed(ctxm, xdm, vdm, fm, args.steps, 1,
                                                  instrument=True)
    ms_di, _, kern_d, build_d, integ_d, _ = timed(ctx64, xd64, vd64, f64, args.steps, 1,
                                                  instrument=True)
    units = float(n) * MD_PER_STEP * args.steps
    tmax_m, units_all = aggregate(ms_m, units, world)
    tmax_d, _ = aggregate(ms_d, units, world)
    value = units_all / (tmax_m * 1e-3)
    value_d = units_all / (tmax_d * 1e-3)

    # ---------------- end to end through the host-buffer entry point (mixed)
    xh = xdm.cpu().pin_memory()
    vh = vdm.cpu().pin_memory()
    fh = fm.cpu().pin_memory()
    for _ in range(max(1, args.warmup)):
        ctxm.md_step_host(xh, vh, fh, mass, DT, MD_PER_STEP, MD_PER_STEP)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ms_e = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a.record(stream)
        ctxm.md_step_host(xh, vh, fh, mass, DT, MD_PER_STEP, MD_PER_STEP)
        b.record(stream)
        b.synchronize()
        ms_e += a.elapsed_time(b)
    wall_e = time.perf_counter() - t0
    tmax_e, _ = aggregate(ms_e, units, world)
    value_e = units_all / (tmax_e * 1e-3)

    kern_ms = kern_m[0] / max(kern_m[1], 1)
    achieved = flop_launch / (kern_ms * 1e-3) / 1e12
    kern_ms_d = kern_d[0] / max(kern_d[1], 1)

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}

    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax_m / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "accumulate_dtype": "f64",
        "data": "synthetic",
        "config": dict(base_config(n, world), launch=best),
        "autotune": {"mixed": tune_m, "fp64": tune_d},
        "force_error": {
            "reference": "FP64 GPU path (itself within 1e-10 of the FP64 CPU oracle in tests)",
            "force_rms_rel": force_rms_rel,
            "energy_rel": energy_rel,
            "virial_max_rel": virial_rel,
        },
        "fp64": {
            "value": value_d,
            "unit": UNIT,
            "ms_per_step": tmax_d / args.steps,
            "dtype": "f64",
            "launch": best64,
            "force_kernel_ms": kern_ms_d,
            "roofline": {
                "bound": "fp64",
                "kernel": "k_tersoff<double>",
                "achieved": flop_launch / (kern_ms_d * 1e-3) / 1e12,
                "peak": pk["fp64_tflops"],
                "unit": "TFLOP/s",
                "frac": flop_launch / (kern_ms_d * 1e-3) / 1e12 / pk["fp64_tflops"],
                "peak_source": "measured in this run: DFMA loop kernel (tersoff_pipe_peaks)",
                "flop_per_launch": flop_launch,
            },
            "gpu_launches": launches_d,
        },
        "mixed_over_fp64": value / value_d,
        "roofline": {
            "bound": "alu",
            "kernel": "k_tersoff<float> (fused zeta/bond-order/force)",
            "achieved": achieved,
            "peak": pk["fp32_tflops"],
            "unit": "TFLOP/s",
            "frac": achieved / pk["fp32_tflops"],
            "peak_source": "measured in this run: FFMA loop kernel (tersoff_pipe_peaks)",
            "peak_derived": PEAK_FP32_TFLOPS_DERIVED,
            "peak_derived_source": "152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz max clock",
            "flop_model": {"per_bond_in_cutoff": FLOP_SHORT, "per_pair_term": FLOP_PAIR,
                           "per_three_body_term": FLOP_TRIPLET,
                           "formula": "short_entries x 36 + pairs x 63 + triplets x 61"},
            "filter_flop_per_launch": filter_flop_launch,
            "mufu": {"ops_per_launch": mufu_launch,
                     "achieved_tops": mufu_launch / (kern_ms * 1e-3) / 1e12,
                     "peak_tops": mufu_peak(pk),
                     "frac": mufu_launch / (kern_ms * 1e-3) / 1e12 / mufu_peak(pk)},
            "traffic": force_traffic(),
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "ceilings_us": ceilings_us(flop_launch, mufu_launch, peaks, pk, kern_ms),
            "flop_per_launch": flop_launch,
            "mufu_per_launch": mufu_launch,
            "work_per_launch": {"skin_entries": skin, "short_entries": nshort, "pairs": npair,
                                "triplets": ntrip},
            "kernel_ms": kern_ms,
            "kernel_launches_timed": kern_m[1],
            "kernel_timing": "CUDA events around each force-kernel launch on its stream, in an "
                             "instrumented pass of the same steps right after the headline pass",
        },
        "breakdown_ms_per_step": {
            "note": "instrumented pass (CUDA events inside the steps; that pass took "
                    f"{ms_mi / args.steps:.3f} ms per step)",
            "force_kernel": kern_m[0] / args.steps,
            "neighbor_build": build_m[0] / args.steps,
            "integrate": integ_m[0] / args.steps,
        },
        "e2e": {
            "value": value_e,
            "unit": UNIT,
            "h2d_bytes_per_step": 3 * n * 3 * 8,
            "d2h_bytes_per_step": 3 * n * 3 * 8,
            "wall_s": wall_e,
        },
        "gpu_launches": launches_m,
        "clocks": clocks,
        "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None,
        "pipe_peaks": pk,
    }
    if world > 1 and not args.no_extra:
        # the sharded fitting step needs every rank (collectives)
        sf = sharded_fit(T, W, dev, flush, world, rank)
        if rank == 0:
            out["sharded_fit"] = sf
    if rank == 0 and not args.no_extra:
        out["backward"] = time_backward(T, ctxm, xdm, ctx64, xd64, flush)
    ctxm.close()
    ctx64.close()
    if rank == 0 and not args.no_extra:
        out["single_evaluations"] = single_evaluations(T, W, dev, flush, cpu=not args.no_cpu_baseline)
        out["batched_fit"] = batched_fit(T, W, dev, flush, cells, gen_s)
        del flush
        torch.cuda.empty_cache()
        out["large_md"] = large_md(T, W, dev, best64)
        if args.accuracy_steps > 0:
            out["accuracy"] = accuracy_run(T, W, args.accuracy_steps, with_fp32_sums=False)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(x, v, t, box, names, table)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _event_time(fn, reps, flush, stream):
    """Mean device time (ms) of fn() over reps calls, L2 flushed before each."""
    import torch
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def time_backward(T, ctxm, xdm, ctx64, xd64, flush, reps=10):
    """tersoff_backward (parameter VJP of energy and forces) on the MD system,
    both paths, against one force evaluation of the same path."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    out = {"what": "tersoff_backward: d/dtheta [gE E + sum gF . F] for all table entries, "
                   "random gF (backward_ms), and d/dx of the same loss = -gE F - H gF "
                   "(position_grad_ms: forces plus the Hessian-vector product); "
                   "forward = tersoff_compute (energy, forces, virial)",
           "atoms": int(xdm.shape[0])}
    for name, ctx, xd in (("mixed", ctxm, xdm), ("fp64", ctx64, xd64)):
        n = xd.shape[0]
        rng = np.random.Generator(np.random.Philox(7))
        gE = torch.tensor([1.0], dtype=torch.float64, device=xd.device)
        gF = torch.tensor(rng.normal(0.0, 1.0, size=(n, 3)), dtype=torch.float64,
                          device=xd.device)
        grad = torch.empty(NPARAM_TABLE_SI, dtype=torch.float64, device=xd.device)
        e = torch.empty(1, dtype=torch.float64, device=xd.device)
        f = torch.empty_like(xd)
        w = torch.empty(6, dtype=torch.float64, device=xd.device)
        gx = torch.empty_like(xd)
        for _ in range(2):
            ctx.backward(xd, gE, gF, None, grad)
            ctx.backward(xd, gE, gF, gx, None)
            ctx.compute(xd, e, f, w)
        torch.cuda.synchronize()
        bw = _event_time(lambda: ctx.backward(xd, gE, gF, None, grad), reps, flush, stream)
        px = _event_time(lambda: ctx.backward(xd, gE, gF, gx, None), reps, flush, stream)
        fw = _event_time(lambda: ctx.compute(xd, e, f, w), reps, flush, stream)
        out[name] = {"backward_ms": bw, "position_grad_ms": px, "forward_ms": fw,
                     "backward_over_forward": bw / fw, "position_grad_over_forward": px / fw,
                     "backward_atoms_per_s": n / (bw * 1e-3)}
    return out


def generate_batch_cells(W):
    """The 256-cell fitting workload's packings, generated in spawn-started
    worker processes (before any GPU use)."""
    import multiprocessing as mp
    t0 = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        cells = W.batched_cells(n_cells=256, map_fn=pool.map)
    return cells, time.time() - t0


def batched_fit(T, W, dev, flush, cells, gen_seconds, reps=20):
    """256 independent periodic Si/C cells (64-4096 atoms, random packings at
    2.3 g/cm^3): one fitting step = energies and forces of every cell in one
    launch, the loss sum_s (E_s - E0_s)^2 + sum_a |F_a - F0_a|^2 and its gradient
    with respect to the whole parameter table (autograd Function, adjoint
    kernel), mixed path, captured in one CUDA graph and replayed. Targets E0,
    F0: the FP64 path at a parameter table perturbed by 1% (seeded)."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    names = ["Si", "C"]
    table = T.mix_tersoff89(*W.element_records(names))
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    n = x.shape[0]
    xd = torch.tensor(x, dtype=torch.float64, device=dev)
    # targets at a perturbed table (continuous fields, m and lambda3 = 0 kept)
    rng = np.random.Generator(np.random.Philox(1607029044))
    pert = table.copy()
    cont = np.arange(table.size) % T.NPARAM != 0
    pert[cont] *= 1.0 + 0.01 * rng.normal(0.0, 1.0, size=int(cont.sum()))
    ref = T.TersoffBatch(t, off, boxes, R_LIST, precision=T.FP64)
    with torch.no_grad():
        e0, f0 = T.energy_forces(ref, xd, torch.tensor(pert, dtype=torch.float64))
    e0, f0 = e0.clone(), f0.clone()
    ref.ctx.close()
    system = T.TersoffBatch(t, off, boxes, R_LIST, precision=T.MIXED)
    tab = torch.tensor(table, dtype=torch.float64, device=dev, requires_grad=True)
    with torch.no_grad():
        T.energy_forces(system, xd, tab)  # uploads the table, builds the lists
    tune = system.ctx.autotune(xd)

    def step():
        E, F = T.energy_forces(system, xd, tab)
        loss = ((E - e0) ** 2).sum() + ((F - f0) ** 2).sum()
        loss.backward()
        return loss

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            tab.grad = None
            step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    tab.grad = None
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        static_loss = step()
    fit_ms = _event_time(graph.replay, reps, flush, stream)
    # the pieces, timed alone (same buffers)
    e = torch.empty(len(cells), dtype=torch.float64, device=dev)
    f = torch.empty_like(xd)
    gE = torch.ones(len(cells), dtype=torch.float64, device=dev)
    gF = torch.ones_like(xd)
    grad = torch.empty(table.size, dtype=torch.float64, device=dev)
    fwd_ms = _event_time(lambda: system.ctx.compute_batched(xd, e, f), reps, flush, stream)
    bwd_ms = _event_time(lambda: system.ctx.backward(xd, gE, gF, None, grad), reps, flush, stream)
    out = {"workload": "256 periodic Si/C cells, 64-4096 atoms each (random packings, 2.3 g/cm^3, "
                       "min separation 1.8 A), loss on energies and forces, gradient with respect "
                       "to all table entries; mixed path; one CUDA graph per step",
           "cells": len(cells), "atoms": int(n), "cell_generation_s": gen_seconds,
           "fit_step_ms": fit_ms, "atoms_per_s": n / (fit_ms * 1e-3),
           "forward_ms": fwd_ms, "backward_ms": bwd_ms, "autotune": tune,
           "loss": float(static_loss.item()),
           "grad_norm": float(tab.grad.norm().item())}
    system.ctx.close()
    return out


def sharded_fit(T, W, dev, flush, world, rank, reps=20):
    """The 256-cell fitting step sharded over the ranks (one GPU each): every
    rank takes its cost-balanced share of the cells (shard.shard_cells),
    generates only those, and runs the same fitting step as batched_fit on them
    (forward, loss on energies and forces, parameter VJP; captured in one CUDA
    graph); the loss and the table gradient are then summed over ranks with one
    NCCL all-reduce each (shard.fit_step). The time of a step is the slowest
    rank's; the work is all ranks' atoms."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1607_02904_gb300 import shard
    stream = torch.cuda.current_stream()
    t0 = time.time()
    sizes, _ = W.batched_cell_sizes(256)
    mine = shard.shard_cells(sizes, world, rank)
    cells = W.batched_cells(n_cells=256, subset=mine)
    gen_s = time.time() - t0
    names = ["Si", "C"]
    table = T.mix_tersoff89(*W.element_records(names))
    off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
    x = np.concatenate([c[0] for c in cells])
    t = np.concatenate([c[1] for c in cells]).astype(np.int32)
    boxes = np.stack([c[2] for c in cells])
    xd = torch.tensor(x, dtype=torch.float64, device=dev)
    rng = np.random.Generator(np.random.Philox(1607029044))
    pert = table.copy()
    cont = np.arange(table.size) % T.NPARAM != 0
    pert[cont] *= 1.0 + 0.01 * rng.normal(0.0, 1.0, size=int(cont.sum()))
    ref = T.TersoffBatch(t, off, boxes, R_LIST, precision=T.FP64)
    with torch.no_grad():
        e0, f0 = T.energy_forces(ref, xd, torch.tensor(pert, dtype=torch.float64))
    e0, f0 = e0.clone(), f0.clone()
    ref.ctx.close()
    system = T.TersoffBatch(t, off, boxes, R_LIST, precision=T.MIXED)
    tab = torch.tensor(table, dtype=torch.float64, device=dev, requires_grad=True)
    with torch.no_grad():
        T.energy_forces(system, xd, tab)

    def step():
        E, F = T.energy_forces(system, xd, tab)
        loss = ((E - e0) ** 2).sum() + ((F - f0) ** 2).sum()
        loss.backward()
        return loss

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            tab.grad = None
            step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    tab.grad = None
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        static_loss = step()
    loss_sum = static_loss.detach().reshape(1)
    for _ in range(3):
        graph.replay()
        shard.fit_step(lambda: (loss_sum, tab.grad))
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(reps):
        flush.zero_()
        dist.barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        shard.fit_step(lambda: (loss_sum, tab.grad))
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    ms /= reps
    atoms = float(len(x))
    tmax, atoms_all = aggregate(ms, atoms, world)
    out = {"workload": "256 periodic Si/C cells (the batched fitting workload) sharded over "
                       f"{world} ranks by cost (atoms x 16); one NCCL all-reduce of the loss "
                       "and of the table gradient per step",
           "ranks": world, "cells_this_rank": len(mine), "atoms_this_rank": int(atoms),
           "atoms_all_ranks": int(atoms_all), "fit_step_ms": tmax,
           "atoms_per_s": atoms_all / (tmax * 1e-3), "cell_generation_s_this_rank": gen_s,
           "loss": float(loss_sum.item()), "grad_norm": float(tab.grad.norm().item())}
    system.ctx.close()
    return out


def large_md(T, W, dev, opt64, steps_mixed=1000, steps_fp64=1000, chunk=100):
    """Si diamond 160x160x80 cells (16,384,000 atoms) at 1000 K: NVE velocity
    Verlet, dt 1 fs, r_list 4.0 A (skin 1.0), rebuilds triggered by the
    displacement (half the skin), all steps of a call in one CUDA graph. Reports
    atom-steps/s per path and the total-energy drift per atom per ns (least-squares
    slope of E_tot / N over the run)."""
    import numpy as np
    import torch
    x, v, t, box, names = W.config_si_large()
    n = x.shape[0]
    table = T.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    stream = torch.cuda.current_stream()
    out = {"workload": "si-diamond-160x160x80-16384000-atoms-1000K-dt1fs-rlist4.0-"
                       "rebuild-on-half-skin", "atoms": n}
    for name, prec, steps in (("mixed", T.MIXED, steps_mixed), ("fp64", T.FP64, steps_fp64)):
        ctx = T.Context(prec)
        ctx.params(table)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        vd = torch.tensor(v, dtype=torch.float64, device=dev)
        td = torch.tensor(t, dtype=torch.int32, device=dev)
        ctx.neighbor_build(xd, td, box, R_LIST)
        if prec == T.MIXED:
            out["autotune_mixed"] = ctx.autotune(xd, vd, mass, DT, MD_PER_STEP)
        else:
            apply_options(ctx, T, opt64)
        fd = torch.zeros_like(xd)
        ctx.compute(xd, None, fd)
        th = torch.zeros((chunk, 3), dtype=torch.float64, device=dev)
        # one untimed call captures the graph
        ctx.md_step(xd, vd, fd, mass, DT, chunk, -1, th)
        torch.cuda.synchronize()
        ms, etot, rebuilds = 0.0, [], 0
        for _ in range(steps // chunk):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.md_step(xd, vd, fd, mass, DT, chunk, -1, th)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
            rebuilds += ctx.md_rebuilds()
            etot.extend(th[:, 2].cpu().numpy().tolist())
        e = np.asarray(etot) / n
        tt = np.arange(e.size) * DT * 1e-3  # ns
        slope = float(np.polyfit(tt, e, 1)[0])
        out[name] = {"steps": steps, "ms": ms, "atom_steps_per_s": n * steps / (ms * 1e-3),
                     "rebuilds": rebuilds, "etot_drift_eV_per_atom_per_ns": slope,
                     "etot_first_last_eV_per_atom": [float(e[0]), float(e[-1])]}
        ctx.close()
        del xd, vd, td, fd, th
        torch.cuda.empty_cache()
    out["mixed_over_fp64"] = out["mixed"]["atom_steps_per_s"] / out["fp64"]["atom_steps_per_s"]
    return out


def single_evaluations(T, W, dev, flush, cpu=True, reps=20):
    """The single-evaluation workloads: Si 8x8x8 cells (4,096 atoms) in FP64, and
    SiC zincblende 64x64x64 cells (2,097,152 atoms) in the mixed path with its
    error against the FP64 oracle (host cores)."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    cases = [("si-diamond-8x8x8-4096-atoms-fp64", W.config_si_small(), T.FP64, RC_SI + 1.0),
             ("sic-zincblende-64x64x64-2097152-atoms-mixed", W.config_sic(), T.MIXED, RC_SI + 1.0)]
    for name, (x, t, box, names), prec, r_list in cases:
        table = T.mix_tersoff89(*W.element_records(names))
        ctx = T.Context(prec)
        ctx.params(table)
        xd = torch.tensor(x, dtype=torch.float64, device=dev)
        td = torch.tensor(t, dtype=torch.int32, device=dev)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        f = torch.empty_like(xd)
        w = torch.empty(6, dtype=torch.float64, device=dev)
        ctx.neighbor_build(xd, td, box, r_list)
        ctx.compute(xd, e, f, w)
        torch.cuda.synchronize()
        build_ms = _event_time(lambda: ctx.neighbor_build(xd, td, box, r_list), 5, flush, stream)
        eval_ms = _event_time(lambda: ctx.compute(xd, e, f, w), reps, flush, stream)
        n = x.shape[0]
        row = {"atoms": n, "precision": "fp64" if prec == T.FP64 else "mixed",
               "r_list_A": r_list, "eval_ms": eval_ms, "atom_evals_per_s": n / (eval_ms * 1e-3),
               "neighbor_build_ms": build_ms}
        if prec == T.MIXED:
            ctx.set_precision(T.FP64)
            ctx.compute(xd, e, f, w)
            ctx.set_precision(T.MIXED)
            f64 = f.cpu().numpy()
            ctx.compute(xd, e, f, w)
            fm = f.cpu().numpy()
            row["force_rms_rel_vs_fp64_gpu"] = float(np.sqrt(((fm - f64) ** 2).mean()) /
                                                     np.sqrt((f64 ** 2).mean()))
        if cpu:
            import oracle
            cores = os.cpu_count() or 1
            t0 = time.perf_counter()
            nl = oracle.neighbors(x, box, RC_SI)
            er, fr, wr = oracle.compute(x, t, box, table, nl, nthreads=cores)
            row["oracle_seconds"] = time.perf_counter() - t0
            ctx.compute(xd, e, f, w)
            torch.cuda.synchronize()
            fg = f.cpu().numpy()
            row["vs_fp64_oracle"] = {
                "energy_rel": abs(e.item() - er) / abs(er),
                "force_rms_rel": float(np.sqrt(((fg - fr) ** 2).mean()) / np.sqrt((fr ** 2).mean())),
                "virial_max_rel": float(np.abs(w.cpu().numpy() - wr).max() / np.abs(wr).max())}
        ctx.close()
        del xd, td, f
        out[name] = row
    return out


def cpu_baseline(x, v, t, box, names, table, nsteps=100):
    """The FP64 oracle on the host cores: full 512,000-atom system, velocity
    Verlet for nsteps steps (rebuild every 10) minus its own setup (one list
    build and one force evaluation), scaled to atom-steps/s."""
    import oracle
    import workloads as W
    mass = [W.MASS_AMU[s] for s in names]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.md_run(x, v, t, box, table, mass, DT, 0, R_LIST, MD_PER_STEP, cap=48,
                  nthreads=cores)
    t1 = time.perf_counter()
    oracle.md_run(x, v, t, box, table, mass, DT, nsteps, R_LIST, MD_PER_STEP, cap=48,
                  nthreads=cores)
    t2 = time.perf_counter()
    per = (t2 - t1) - (t1 - t0)
    return {"value": x.shape[0] * nsteps / per, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle MD on the full {x.shape[0]}-atom system: {nsteps} VV steps "
                      f"(rebuild every {MD_PER_STEP}), setup subtracted, {cores} OpenMP threads",
            "seconds": t2 - t0}


def run_reference(args):
    """The oracle on the host cores (there is no reference implementation to
    install), on the benchmark's own system: Si diamond 40x40x40 cells,
    512,000 atoms, same recipe. Each step is one oracle md_run call of
    MD_PER_STEP velocity-Verlet steps continuing the trajectory of the previous
    call; a call also builds its list and evaluates its forces once before the
    first step (two list builds and 11 force evaluations per 10 steps, against
    one build and 10 evaluations on the GPU), so the oracle's rate is, if
    anything, understated by about a tenth."""
    world, rank, local = dist_info()
    if rank != 0:
        return
    import oracle
    import workloads as W
    x, v, t, box, names = W.config_si_md()
    table = oracle.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        x, v, _, _ = oracle.md_run(x, v, t, box, table, mass, DT, MD_PER_STEP, R_LIST,
                                   MD_PER_STEP, cap=48, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x, v, _, _ = oracle.md_run(x, v, t, box, table, mass, DT, MD_PER_STEP, R_LIST,
                                   MD_PER_STEP, cap=48, nthreads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    units = x.shape[0] * MD_PER_STEP * args.steps
    value = units / total
    sample = (f"each step: oracle md_run of {MD_PER_STEP} VV steps on the full {x.shape[0]}-atom "
              f"benchmark system, continuing the previous step's trajectory, including the "
              f"call's own list build and first force evaluation, {cores} OpenMP threads")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": base_config(x.shape[0], world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def accuracy_run(T, W, steps, with_fp32_sums=True):
    """Long-run accuracy of the mixed path (the paper's accuracy experiment,
    Sec. V-D): Si diamond 20x20x10 cells (32,000 atoms) at 1000 K, the same
    initial state integrated by the FP64 and the mixed path for `steps`
    velocity-Verlet steps (dt 1 fs, rebuilds on half the skin), total energy
    recorded every step; the largest relative deviation of the mixed path's
    total energy from the FP64 path's, and each path's drift. Optionally the
    same for the mixed path with single-precision force sums (the paper's
    all-single mode, ABLATE_FP32_SUMS)."""
    import numpy as np
    import torch
    names = ["Si"]
    x, t, box = W.diamond(20, 20, 10, 5.432)
    rng = W.rng_for(6)
    x = W.jitter_gaussian(x, 0.05, rng)
    v = W.maxwell_velocities(t, np.array([W.MASS_AMU["Si"]]), 1000.0, rng)
    n = x.shape[0]
    table = T.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    chunk = 1000
    out = {"metric": "total-energy deviation of the mixed path from the FP64 path",
           "atoms": int(n), "steps": steps, "dt_ps": DT, "temperature_K": 1000.0,
           "rebuild": "on half the skin (r_list 4.0 A)"}
    series = {}
    variants = [("fp64", T.FP64, 0), ("mixed", T.MIXED, 0)]
    if with_fp32_sums:
        variants.append(("fp32_sums", T.MIXED, T.ABLATE_FP32_SUMS))
    for name, prec, abl in variants:
        ctx = T.Context(prec)
        ctx.set_ablation(abl)
        ctx.set_scatter(T.SCATTER_GATHER)
        ctx.params(table)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        vd = torch.tensor(v, dtype=torch.float64, device="cuda")
        ctx.neighbor_build(xd, torch.tensor(t, dtype=torch.int32, device="cuda"), box, R_LIST)
        fd = torch.zeros_like(xd)
        ctx.compute(xd, None, fd)
        th = torch.zeros((chunk, 3), dtype=torch.float64, device="cuda")
        etot = []
        t0 = time.perf_counter()
        for _ in range(steps // chunk):
            ctx.md_step(xd, vd, fd, mass, DT, chunk, -1, th)
            etot.append(th[:, 2].cpu().numpy().copy())
        torch.cuda.synchronize()
        series[name] = np.concatenate(etot)
        out[name + "_seconds"] = time.perf_counter() - t0
        ctx.close()
    e64, em = series["fp64"], series["mixed"]
    tt = np.arange(e64.size) * DT * 1e-3  # ns
    out["max_rel_deviation"] = float(np.abs(em - e64).max() / np.abs(e64).max())
    out["final_rel_deviation"] = float(abs(em[-1] - e64[-1]) / abs(e64[-1]))
    if with_fp32_sums:
        es = series["fp32_sums"]
        out["fp32_sums_max_rel_deviation"] = float(np.abs(es - e64).max() / np.abs(e64).max())
        out["fp32_sums_final_rel_deviation"] = float(abs(es[-1] - e64[-1]) / abs(e64[-1]))
    out["paper_bound_rel"] = 2e-5
    for name, e in series.items():
        out[name + "_drift_eV_per_atom_per_ns"] = float(np.polyfit(tt, e / n, 1)[0])
        out[name + "_etot_first_last_eV"] = [float(e[0]), float(e[-1])]
    return out


def run_accuracy(args):
    """--accuracy: the long-run accuracy experiment for --steps MD steps, with
    the single-precision force-sum variant (one JSON line)."""
    import workloads as W
    import paper_1607_02904_gb300 as T
    print(json.dumps(accuracy_run(T, W, args.steps)), flush=True)


def run_ablations(args):
    """The paper's design choices measured on the benchmark workload (mixed
    path, default launch options): the stored short list (Sec. IV-D) and the
    register-resident neighbourhood with pre-computed derivatives (Sec. IV-A),
    each switched off alone and together, the compensated force sums replaced
    by plain float sums (the paper's all-single accumulation), and no list
    filtering at all with the fast-forward lane scheme (Sec. IV-C); and, under
    the atomic scatter, each atom's own sums in plain float (the default)
    against compensated sums carried into double. Reports
    ms per 10 MD steps and per force evaluation, and the force error against
    the default mixed path and against the FP64 path (the first three leave
    the forces unchanged up to rounding order)."""
    import numpy as np
    import torch
    import workloads as W
    import paper_1607_02904_gb300 as T
    x, v, t, box, names = W.config_si_md()
    table = T.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"metric": "ablations of the paper's design choices (mixed path)",
           "workload": workload_name(), "md_ms_per_10_steps": {}, "force_eval_ms": {},
           "force_rms_rel_vs_default": {}, "force_rms_rel_vs_fp64": {},
           "energy_rel_vs_fp64": {}, "virial_max_rel_vs_fp64": {}}
    ref = None
    ctx = T.Context(T.FP64)
    ctx.params(table)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ctx.neighbor_build(xd, torch.tensor(t, dtype=torch.int32, device="cuda"), box, R_LIST)
    fd = torch.zeros_like(xd)
    e64 = torch.zeros(1, dtype=torch.float64, device="cuda")
    w64 = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(xd, e64, fd, w64)
    f64 = fd.cpu().numpy()
    e64, w64 = e64.item(), w64.cpu().numpy()
    ctx.close()
    for name, flags in (("default", 0), ("no_short_list", T.ABLATE_NO_SHORT),
                        ("general_path", T.ABLATE_GENERAL),
                        ("both", T.ABLATE_NO_SHORT | T.ABLATE_GENERAL),
                        ("fp32_sums", T.ABLATE_FP32_SUMS),
                        ("fast_forward", T.ABLATE_FASTFWD),
                        ("atomic_scatter", "atomic"),
                        ("atomic_scatter_comp_atom_sums", T.ABLATE_COMP_ATOM_SUMS)):
        ctx = T.Context(T.MIXED)
        ctx.set_ablation(0 if flags == "atomic" else flags)
        ctx.set_scatter(T.SCATTER_ATOMIC if flags in ("atomic", T.ABLATE_COMP_ATOM_SUMS)
                        else T.SCATTER_GATHER)
        ctx.params(table)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        vd = torch.tensor(v, dtype=torch.float64, device="cuda")
        ctx.neighbor_build(xd, torch.tensor(t, dtype=torch.int32, device="cuda"), box, R_LIST)
        fd = torch.zeros_like(xd)
        ee = torch.zeros(1, dtype=torch.float64, device="cuda")
        ww = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.compute(xd, ee, fd, ww)
        fr = fd.cpu().numpy()
        out["energy_rel_vs_fp64"][name] = abs(ee.item() - e64) / abs(e64)
        out["virial_max_rel_vs_fp64"][name] = float(np.abs(ww.cpu().numpy() - w64).max() /
                                                    np.abs(w64).max())
        if ref is None:
            ref = fr
        out["force_rms_rel_vs_default"][name] = float(np.sqrt(((fr - ref) ** 2).mean()) /
                                                      np.sqrt((ref ** 2).mean()))
        out["force_rms_rel_vs_fp64"][name] = float(np.sqrt(((fr - f64) ** 2).mean()) /
                                                   np.sqrt((f64 ** 2).mean()))
        out["force_eval_ms"][name] = _event_time(lambda: ctx.compute(xd, None, fd), args.steps,
                                                 flush, stream)
        for _ in range(3):
            ctx.md_step(xd, vd, fd, mass, DT, MD_PER_STEP, MD_PER_STEP)
        out["md_ms_per_10_steps"][name] = _event_time(
            lambda: ctx.md_step(xd, vd, fd, mass, DT, MD_PER_STEP, MD_PER_STEP), args.steps,
            flush, stream)
        ctx.close()
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """The benchmark workload without timing, for profiler captures."""
    import numpy as np
    import torch
    import workloads as W
    import paper_1607_02904_gb300 as T
    if args.only == "backward-batch":
        cells = W.batched_cells(n_cells=64)
        off = np.cumsum([0] + [len(c[0]) for c in cells]).astype(np.int32)
        x = np.concatenate([c[0] for c in cells])
        t = np.concatenate([c[1] for c in cells]).astype(np.int32)
        boxes = np.stack([c[2] for c in cells])
        ctx = T.Context(T.MIXED if args.precision == "mixed" else T.FP64)
        ctx.params(T.mix_tersoff89(*W.element_records(["Si", "C"])))
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        ctx.neighbor_build_batched(xd, torch.tensor(t, device="cuda"), off, boxes, R_LIST)
        gE = torch.ones(len(cells), dtype=torch.float64, device="cuda")
        gF = torch.ones_like(xd)
        g = torch.empty(14 * 8, dtype=torch.float64, device="cuda")
        for _ in range(args.steps):
            ctx.backward(xd, gE, gF, None, g)
        torch.cuda.synchronize()
        ctx.close()
        return
    if args.only == "force-sic":
        x, t, box, names = W.config_sic()
        v = None
    else:
        x, v, t, box, names = W.config_si_md()
    table = T.mix_tersoff89(*W.element_records(names))
    mass = [W.MASS_AMU[s] for s in names]
    ctx = T.Context(T.MIXED if args.precision == "mixed" else T.FP64)
    ctx.set_scatter(T.SCATTER_ATOMIC if args.scatter == "atomic" else T.SCATTER_GATHER)
    ctx.params(table)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    vd = torch.tensor(v, dtype=torch.float64, device="cuda") if v is not None else None
    td = torch.tensor(t, dtype=torch.int32, device="cuda")
    ctx.neighbor_build(xd, td, box, R_LIST)
    fd = torch.zeros_like(xd)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    gE = torch.ones(1, dtype=torch.float64, device="cuda")
    gF = torch.ones_like(xd)
    g = torch.empty(table.size, dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        if args.only in ("force", "force-sic"):
            ctx.compute(xd, e, fd)
        elif args.only == "backward":
            ctx.backward(xd, gE, gF, None, g)
        elif args.only == "hvp":
            ctx.backward(xd, gE, gF, fd, None)
        else:
            ctx.md_step(xd, vd, fd, mass, DT, MD_PER_STEP, MD_PER_STEP)
    torch.cuda.synchronize()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the single-evaluation workloads and the backward timing")
    ap.add_argument("--only", choices=["force", "md", "force-sic", "backward", "backward-batch", "hvp"],
                    default=None,
                    help="profiling case: K force evaluations, K MD rebuild periods, K "
                         "parameter backward passes or K position gradients (hvp) of the "
                         "benchmark workload, K force evaluations of the 2.1M-atom SiC "
                         "workload, or K backward passes of 64 packing cells; nothing printed")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--ablations", action="store_true",
                    help="the paper's design choices switched off one at a time (one JSON line)")
    ap.add_argument("--accuracy", action="store_true",
                    help="long-run accuracy of the mixed path against the FP64 path "
                         "(32,000 atoms, --steps MD steps; one JSON line)")
    ap.add_argument("--scatter", choices=["gather", "atomic"], default="gather")
    ap.add_argument("--accuracy-steps", type=int, default=1_000_000,
                    help="MD steps of the long-run accuracy leg of the default run (32,000 "
                         "atoms, FP64 and mixed paths; 0 skips it)")
    args = ap.parse_args()
    if args.only:
        run_profile_case(args)
        return
    if args.accuracy:
        run_accuracy(args)
        return
    if args.ablations:
        run_ablations(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
