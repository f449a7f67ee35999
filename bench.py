#!/usr/bin/env python
"""Benchmark of the Rotne-Prager-Blake Brownian-dynamics hot path on GB300.

One step = one stochastic Adams-Bashforth step (Eq. AB) of a synthetic roller monolayer: forces,
the fused wall-RPY product M_tt F + M_tr T, Philox noise, Lanczos M^{1/2} W, the RFD drift and the
update -- every part in the CUDA library, called through its C ABI.

Default workload: the large monolayer, N = 65536 spheres (a = eta = kT = 1, area fraction 0.4,
z = a + Exp(0.5 a)), gravity -1 z, torque +1 y, soft repulsion U0 = 1, b = 0.1 a, dt = 0.01,
Lanczos tol 1e-3, float32 pair arithmetic with float64 Lanczos.

Prints one JSON line (rank 0).  value = wall-RPY pair evaluations per second over the whole step
(N^2 per pair pass; a step makes 3 + m passes: the fused product, m Lanczos products and two RFD
products), summed over ranks.  --impl reference times the FP64 CPU oracle instead (a bounded
sample of the same workload on the host cores).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wall-RPY matvec Gpairs/s; BD steps/s at N=65536; p50/p99 solve latency"


def read_flops(path=os.path.join(ROOT, "FLOPS.md")):
    """The fixed per-pair work of the pair block (FLOPS.md): {key: count} for its FLOPS_* / MUFU_* rows."""
    out = {}
    with open(path) as f:
        for line in f:
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) >= 2 and (cells[0].startswith("FLOPS_") or cells[0].startswith("MUFU_")):
                out[cells[0]] = int(cells[1])
    return out


_FLOPS = read_flops()
FLOPS_TT = _FLOPS["FLOPS_TT"]          # one direction, translation-translation, per ordered pair
FLOPS_FUSED = _FLOPS["FLOPS_FUSED"]    # one direction with the translation-rotation coupling
FLOPS_SYM = _FLOPS["FLOPS_SYM"]        # per unordered pair, applied both ways (reciprocity)
# FP32 lane operations (an FMA, a multiply or an add is one) that the symmetric translation-translation
# kernel executes per unordered pair, counted from its source (pair_offsets_x2 6, pair_block_x2 34,
# tt_apply_target 16, tt_apply_source 16); a property of the kernel, used only for the pipe-occupancy
# view beside the flop roofline.
OPS_SYM_KERNEL = 72
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25  # dense FP64 rate of a GB300 (vector pipe), for context
# DRAM bytes (read + write) of one launch of the symmetric translation-translation kernel at
# N = 65536, from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` (1 pass) on the
# default workload (profiles/pair_f32x2_sym_kernel_n32768.md gives the command), mean of two launches:
# 3.71 MB read (the packed sources), 165.20 MB written (segment and source-column partials leaving
# L2).  Valid for this kernel build only: reset to {} when the kernel changes.
SYM_TT_TRAFFIC_BYTES = {65536: 3.711e6 + 165.199e6}
SM_MAX_MHZ = 2070.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=None,
                    help="spheres; default 65536 (monolayer, reference arm, bound of the lanczos sweep), 4096 "
                         "(accuracy) or 32768 (fingering)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--delta", type=float, default=None,
                    help="RFD length; default 1e-6 a (fp64) or 5e-3 a (fp32: delta ~ eps^(1/3) a, Sec. II.A)")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="monolayer at N=1: skip the small and batched configurations measured after the headline")
    ap.add_argument("--periodic", action="store_true",
                    help="monolayer: pseudo-periodic boundaries with the monolayer's square as the unit cell")
    ap.add_argument("--split", choices=["replicas", "pairs", "rows"], default="replicas",
                    help="monolayer under torchrun: independent replicas (weak scaling) or one suspension whose "
                         "products are shared among the ranks (strong scaling), by equal runs of the symmetric "
                         "pass's pair triangle summed with an all-reduce (pairs) or by target rows gathered with "
                         "an all-gather (rows)")
    ap.add_argument("--precondition", action="store_true",
                    help="monolayer: block-diagonal Lanczos preconditioner (an option; the paper's runs use none)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--workload", choices=["monolayer", "batched", "serving", "lanczos", "accuracy", "small",
                                           "fingering", "shares"],
                    default="monolayer")
    ap.add_argument("--acc-steps", type=int, default=10, help="accuracy: steps compared with the oracle")
    ap.add_argument("--lanczos-iters", type=int, default=12,
                    help="batched: Lanczos iterations per step inside the step graph (converged instances masked)")
    ap.add_argument("--B", type=int, default=512, help="batched: number of suspensions")
    ap.add_argument("--hg", type=float, default=1.5, help="fingering: gravitational height h_g / a")
    ap.add_argument("--fing-steps", type=int, default=2500, help="fingering: steps of each run (0.016 s each)")
    ap.add_argument("--sample-every", type=int, default=10, help="fingering: steps between front spectra")
    ap.add_argument("--fing-dt", type=float, default=0.016,
                    help="fingering: time step in seconds (the paper's 0.016 s = tau_U / 2; it reports 0.008 s "
                         "giving essentially the same results)")
    ap.add_argument("--equilibrate-s", type=float, default=0.0,
                    help="fingering: seconds of Brownian dynamics without torque in the 60a x 4915a cell with "
                         "pseudo-periodic boundaries before each realization (an equilibrium sample of the "
                         "two-periodic suspension, as the paper's initial states); 0: sequential addition only")
    ap.add_argument("--realizations", type=int, default=1,
                    help="fingering: independent realizations (initial state and noise seeds seed, seed + 1, ...); "
                         "t* and t1/2 come from their mean band power")
    ap.add_argument("--requests", type=int, default=500, help="serving: number of requests")
    ap.add_argument("--serial-sample-s", type=float, default=60.0,
                    help="serving: seconds of real serial FP64 service measured on a sample of the requests")
    ap.add_argument("--load", type=float, default=0.85, help="serving: offered load relative to measured capacity")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: device-memory budget for resident state")
    ap.add_argument("--max-batch", type=int, default=256, help="serving: requests per batched step")
    ap.add_argument("--max-spheres", type=int, default=262144, help="serving: spheres per batched step")
    return ap.parse_args(argv)


def cell_side(N, phi=0.4):
    """Side of the square the monolayer generator fills (a = 1)."""
    return math.sqrt(N * math.pi / phi)


def workload_name(args):
    per = (f", pseudo-periodic {cell_side(args.N):.2f}a x {cell_side(args.N):.2f}a cell (unit cell + 8 neighbours)"
           if args.periodic else "")
    pc = ", block-diagonal Lanczos preconditioner" if getattr(args, "precondition", False) else ""
    return (f"roller monolayer N={args.N} (phi=0.4, z=a+Exp(0.5a), gravity -1 z, torque +1 y, U0=1, b=0.1a), "
            f"AB step dt={args.dt}, RFD delta={args.delta}, Lanczos tol={args.tol}, {args.precision} pairs{per}{pc}")


def oracle_sample(N, seed, seconds, periodic=None):
    """Time the FP64 oracle's fused product on a row sample of the workload; returns Gpairs/s and info
    (pair evaluations: nine per pair with pseudo-periodic boundaries)."""
    import oracle as O
    from paper_1612_00474_gb300 import inputs

    pos = inputs.monolayer(N, seed=seed)
    F = np.tile([0.0, 0.0, -1.0], (N, 1))
    T = np.tile([0.0, 1.0, 0.0], (N, 1))
    images = 9 if periodic else 1
    O.mobility_apply(pos, F, T, rows=(0, 4), periodic=periodic)  # start the OpenMP pool
    rows = 64  # 16 chunks of 4 rows: every OpenMP thread of the host busy while calibrating
    t0 = time.perf_counter()
    O.mobility_apply(pos, F, T, rows=(0, rows), periodic=periodic)
    dt = time.perf_counter() - t0
    rows = int(max(8, min(N, rows * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    O.mobility_apply(pos, F, T, rows=(0, rows), periodic=periodic)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return images * rows * N / dt / 1e9, dict(rows=rows, seconds=dt, cores=cores)


def clocks_start(device_index):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                                 "-i", str(device_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except (FileNotFoundError, OSError):
        return None


def clocks_stop(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def measure_peaks(device_index):
    """Measured fused-multiply-add rates of this GPU (rpb_fma_peak), with the clocks sampled meanwhile."""
    from paper_1612_00474_gb300 import rpb

    clk = clocks_start(device_index)
    out = {}
    for kind in ("ffma2", "ffma", "dfma"):
        t, ms = rpb.fma_peak(kind)
        out[kind + "_tflops"] = t
        out[kind + "_ms"] = ms
    out["clocks"] = clocks_stop(clk)
    return out


def cpu_baseline_line(args, N):
    """The FP64 oracle's fused product on a row sample of an N-sphere monolayer, as a cpu_baseline entry."""
    if args.no_cpu_baseline:
        return None
    v, info = oracle_sample(N, args.seed, min(args.cpu_seconds, 10.0))
    return {"value": v, "unit": "Gpairs/s", "cores": info["cores"], "kind": "oracle",
            "sample": (f"fused M_tt F + M_tr T of an N={N} monolayer on {info['rows']} target rows x {N} sources "
                       f"({info['seconds']:.1f} s, FP64 oracle, OpenMP over target rows)")}


def run_reference(args, rank, world):
    if rank != 0:
        return
    N = args.N
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        v, info = oracle_sample(N, args.seed, per_step,
                                periodic=(cell_side(N), cell_side(N)) if args.periodic else None)
        if k >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"fused M_tt F + M_tr T of the N={N} monolayer on {info['rows']} target rows x {N} sources "
              f"per step (FP64 oracle, OpenMP over target rows)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": info["seconds"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "N": N},
        "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": info["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate(dist, max_vals, sum_vals, device="cpu"):
    """Combine per-rank measurements: the maximum over ranks of each entry of max_vals (times) and
    the sum of each entry of sum_vals (work).  dist is torch.distributed (initialised) or None."""
    import torch

    mx = [float(v) for v in max_vals]
    sm = [float(v) for v in sum_vals]
    if dist is None:
        return mx, sm
    a = torch.tensor(mx, dtype=torch.float64, device=device)
    b = torch.tensor(sm, dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.cpu().tolist(), b.cpu().tolist()


def init_dist(world):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group("nccl", init_method="env://")
    return dist


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    torch.cuda.set_device(local_rank)
    dist = init_dist(world)

    N = args.N
    shared = args.split in ("pairs", "rows") and world > 1
    rows = shared and args.split == "rows"
    if shared:  # one suspension, its products shared among the ranks (same seed and state on every rank)
        from paper_1612_00474_gb300.split import SplitContext

        seed = args.seed
        ctx = SplitContext(N, mode=args.split, precision=args.precision, max_iter=64)
    else:
        seed = args.seed + rank  # independent replicas, one suspension per rank
        ctx = rpb.Context(max_N=N, precision=args.precision, max_iter=64)
    images = 1
    if args.periodic:
        ctx.set_periodic(cell_side(N), cell_side(N))
        images = 9  # each source at its minimum image and the eight neighbour-cell shifts
    if args.precondition:
        ctx.set_preconditioner("block-diagonal")
    pos0 = inputs.monolayer(N, seed=seed)
    q = torch.tensor(inputs.to_soa(pos0), dtype=torch.float64, device="cuda")
    Up = torch.zeros_like(q)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    kw = dict(dt=args.dt, delta=args.delta, tol=args.tol, max_iter=64)

    step = 0
    for _ in range(args.warmup):
        ctx.ab_step(q, Up, step, seed, **kw)
        step += 1
    torch.cuda.synchronize()
    peaks = measure_peaks(local_rank)
    if dist:
        dist.barrier()

    clk = clocks_start(local_rank)
    launches0 = rpb.launch_count()
    ms, ms_list = [], []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.ab_step(q, Up, step, seed, **kw)
        e1.record(stream)
        ms.append((e0, e1))
        ms_list.append(st["m"])
        step += 1
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = rpb.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ms]
    total_s = sum(step_ms) / 1e3
    pairs = images * float(N) * N * sum(3 + m for m in ms_list)

    # end to end through the C ABI with host buffers: copy state in, step, copy state out
    h_q = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
    h_U = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
    h_q.copy_(q)
    h_U.copy_(Up)
    e2e_ms, e2e_m = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.copy_(h_q, non_blocking=True)
        Up.copy_(h_U, non_blocking=True)
        st = ctx.ab_step(q, Up, step, seed, **kw)
        h_q.copy_(q, non_blocking=True)
        h_U.copy_(Up, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_m.append(st["m"])
        step += 1
    clocks = clocks_stop(clk)
    e2e_pairs = images * float(N) * N * sum(3 + m for m in e2e_m)
    e2e_s = sum(e2e_ms) / 1e3

    # dominant kernel: the translation-translation pair pass (m + 2 of the 3 + m passes per step),
    # timed live through the C ABI on this stream; and the fused pass for reference
    def time_product(F, T, reps=3):
        out = torch.empty_like(q)
        ctx.mobility_apply(q, F, T, out=out)
        durs = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.mobility_apply(q, F, T, out=out)
            b.record(stream)
            b.synchronize()
            durs.append(a.elapsed_time(b) / 1e3)
        return statistics.mean(durs)

    W = ctx.philox_normal(N, seed, 0, 0)
    Tq = torch.tensor(inputs.to_soa(np.tile([0.0, 1.0, 0.0], (N, 1))), dtype=torch.float64, device="cuda")
    t_tt = time_product(W, None)
    t_fused = time_product(W, Tq)

    # max of the times and sum of the work over ranks
    # max of the times over ranks; the work summed over ranks for replicas, once for a shared suspension
    (total_s, e2e_s), (pairs, e2e_pairs) = aggregate(dist, [total_s, e2e_s], [pairs, e2e_pairs], device="cuda")
    if shared:
        pairs, e2e_pairs = pairs / world, e2e_pairs / world
    if dist:
        dist.barrier()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per = (cell_side(N), cell_side(N)) if args.periodic else None
        v, info = oracle_sample(N, args.seed, args.cpu_seconds, periodic=per)
        cpu = {"value": v, "unit": "Gpairs/s", "cores": info["cores"], "kind": "oracle",
               "sample": (f"fused M_tt F + M_tr T of the N={N} monolayer on {info['rows']} target rows x {N} "
                          f"sources ({info['seconds']:.1f} s, FP64 oracle, OpenMP over target rows)")}

    if rank == 0:
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        fp32_peak = max(peaks["ffma2_tflops"], peaks["ffma_tflops"])
        if args.precision == "fp32":
            peak = fp32_peak
            peak_basis = (f"measured on this GPU by rpb_fma_peak: FFMA2 {peaks['ffma2_tflops']:.1f}, FFMA "
                          f"{peaks['ffma_tflops']:.1f} TFLOP/s (best of 3 launches on all SMs; nominal "
                          f"{sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz = "
                          f"{sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12:.1f})")
        else:
            peak = peaks["dfma_tflops"]
            peak_basis = (f"measured on this GPU by rpb_fma_peak: DFMA {peak:.3f} TFLOP/s (nominal "
                          f"{FP64_NOMINAL_TFLOPS})")
        sym = args.precision == "fp32" and os.environ.get("RPB_FP32_SYM") != "0" and N >= 256 and not rows
        share = 1.0 / world if shared else 1.0  # rank 0's share of the triangle's tile units (pairs split)
        diag = float(N) * 128
        if args.periodic and sym:  # nine images of each unordered pair once, both ways
            flops_tt = 9.0 * (FLOPS_SYM * (float(N) * N - diag) / 2 + FLOPS_TT * diag)
            kernel = "pair_f32x2_sym_kernel, pseudo-periodic form (translation-translation, reciprocity, 9 images)"
        elif args.periodic:
            flops_tt = 9.0 * N * N * FLOPS_TT
            kernel = f"pair_periodic_f{args.precision[2:]}_kernel<false,true> (translation-translation, 9 images)"
        elif sym:  # each unordered pair once (135 flop) except inside the 128-wide diagonal tiles (106 flop each way)
            flops_tt = share * (FLOPS_SYM * (float(N) * N - diag) / 2 + FLOPS_TT * diag)
            kernel = "pair_f32x2_sym_kernel (translation-translation, reciprocity)"
            if shared:
                kernel += (f" over rank 0's share (1/{world} of the triangle's tile units), timed with the "
                           f"all-reduce of the partial products")
        elif rows:  # this rank's rows against all sources, timed with the all-gather of the other rows
            a_, b_ = ctx.split(N).mine
            flops_tt = float(b_ - a_) * N * FLOPS_TT
            kernel = (f"pair_f{'32x2' if args.precision == 'fp32' else '64'}_kernel<false> over rank 0's rows "
                      f"[{a_}, {b_}) of {N}, timed with the all-gather of the row blocks")
        else:
            flops_tt = float(N) * N * FLOPS_TT
            kernel = f"pair_f{args.precision[2:]}_kernel<false> (translation-translation)"
        achieved = flops_tt / t_tt / 1e12
        ops_view = None
        if sym:
            # the FP32 pipe's operation rate: one lane operation per lane per clock, whether an FMA, a
            # multiply or an add (a third of the pair's operations are multiplies and adds that cannot be
            # fused, so the flop fraction understates how busy the pipe is)
            ops = share * (9.0 if args.periodic else 1.0) * OPS_SYM_KERNEL * (float(N) * N - diag) / 2
            ops_peak = fp32_peak / 2  # one FMA is one lane operation
            ops_view = {"per_unordered_pair": OPS_SYM_KERNEL, "basis": "the kernel's own operation count",
                        "achieved": ops / t_tt / 1e12, "peak": ops_peak, "unit": "Top/s",
                        "frac": ops / t_tt / 1e12 / ops_peak}
        value = pairs / total_s / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "Gpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong" if shared else "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "N": N, "precision": args.precision,
                       "pair_arith": args.precision, "lanczos_arith": "f64", "parallelism": f"{args.split} x{world}" if shared else f"replicas x{world}",
                       "l2": "256 MB buffer written between timed steps",
                       "periodic": [cell_side(N)] * 2 if args.periodic else None,
                       "pair_evaluations_per_product": images * N * N},
            "steps_per_s": args.steps * (1 if shared else world) / total_s,
            "lanczos_m": ms_list,
            "step_ms": [round(x, 3) for x in step_ms],
            "matvec": {"tt_ms": t_tt * 1e3, "fused_ms": t_fused * 1e3,
                       "tt_gpairs_s": images * N * N / t_tt / 1e9, "fused_gpairs_s": images * N * N / t_fused / 1e9},
            "roofline": {"bound": "alu", "kernel": kernel,
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_basis": peak_basis,
                         "flops_per_launch": flops_tt,
                         "flops_per_pair": FLOPS_SYM / 2 if sym else FLOPS_TT,
                         "traffic": SYM_TT_TRAFFIC_BYTES.get(N) if sym and not args.periodic and not shared else None,
                         "traffic_unit": "bytes per launch",
                         "fp32_ops": ops_view},
            "peaks": peaks,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_pairs / e2e_s / 1e9, "unit": "Gpairs/s", "h2d_bytes_per_step": 2 * 3 * N * 8,
                    "d2h_bytes_per_step": 2 * 3 * N * 8},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s_timed": t_wall,
        }
        if world == 1 and not args.no_secondary:
            line["secondary"] = secondary_configs(args, local_rank)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def secondary_configs(args, local_rank):
    """The small (N = 256, FP64) and batched (512 suspensions) configurations measured in the same run
    as the headline, after it (a few seconds each; their own workloads add the oracle timings)."""
    sm = measure_small(local_rank, 20, 3)
    bargs = argparse.Namespace(**vars(args))
    bargs.delta = 5e-3 if args.precision == "fp32" else 1e-6
    b = measure_batched(bargs, 0, 1, local_rank, None, 10, 3)
    return {
        "small": {"workload": "N=256 monolayer (seed 0), FP64 pairs, AB step dt=0.01, delta=1e-6, tol=1e-3",
                  "us_per_step_rpb_ab_step": b_round(sm["gpu_us"]), "us_per_step_rpb_run": b_round(sm["graph_us"]),
                  "lanczos_m": sm["ms_m"][-1], "clocks": sm["clocks"]},
        "batched": {"workload": f"{b['B']} suspensions, N log-uniform in [64, 2048] (sum N = {sum(b['sizes'])}), "
                                f"{args.precision} pairs, 10 graph-replayed AB steps",
                    "instance_steps_per_s": b["B"] * 10 / b["total_s"], "gpairs_s": b["pairs"] / b["total_s"] / 1e9,
                    "e2e_gpairs_s": b["e2e_pairs"] / b["e2e_s"] / 1e9,
                    "loop_instance_steps_per_s": b["B"] / b["loop_s"], "tiles": b["tuned"]["best"],
                    "unconverged_instance_steps": b["unconv"], "gpu_launches": b["launches"], "clocks": b["clocks"]},
    }


def b_round(x):
    return round(float(x), 2)


def _base_line(args, world, metric_value, unit, ms_per_step, dtype, config):
    return {"metric": METRIC, "value": metric_value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}


def measure_batched(args, rank, world, local_rank, dist, steps, warmup):
    """512 independent suspensions, N log-uniform in [64, 2048] (seeds 0..511), advanced together by
    rpb_batch_run (graph-replayed steps); the tile schedule from the batch tuner; the same timed end to
    end from pinned host memory, and a loop over the single-suspension rpb_ab_step for comparison."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    B = args.B
    sizes = [int(n) for n in inputs.batch_sizes(B, seed=args.seed)]
    seeds = [args.seed + rank * B + k for k in range(B)]
    bt = rpb.BatchContext(max_total_N=sum(sizes), max_B=B, precision=args.precision, max_iter=64)
    q = [torch.tensor(inputs.to_soa(inputs.monolayer(N, seed=s)), dtype=torch.float64, device="cuda")
         for N, s in zip(sizes, seeds)]
    U = [torch.zeros_like(t) for t in q]
    kw = dict(dt=args.dt, delta=args.delta, tol=args.tol, max_iter=64)
    stream = torch.cuda.current_stream()
    tuned = bt.tune(q, reps=3)  # the tile schedule of this size mix, kept by the context
    step = 0
    for _ in range(warmup):
        bt.ab_step(q, U, [step] * B, seeds, **kw)
        step += 1
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # host-driven steps (one rpb_batch_ab_step call per step), for comparison
    ms_call = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = bt.ab_step(q, U, [step] * B, seeds, **kw)
        e1.record(stream)
        e1.synchronize()
        ms_call.append(e0.elapsed_time(e1))
        step += 1
    m_used = max(s["m"] for s in st)
    # timed: all K steps in one rpb_batch_run call (one gather, the step graph replayed K times)
    clk = clocks_start(local_rank)
    launches0 = rpb.launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, unconv = bt.run(q, U, [step] * B, seeds, nsteps=steps, lanczos_iters=args.lanczos_iters,
                        dt=args.dt, delta=args.delta, tol=args.tol)
    torch.cuda.synchronize()
    total_s = time.perf_counter() - t0
    clocks = clocks_stop(clk)
    launches = rpb.launch_count() - launches0
    step += steps
    # pair evaluations: each instance's converged iteration count (m of the last step as the estimate)
    pairs = steps * sum(float(N) * N * (3 + s["m"]) for N, s in zip(sizes, st))
    # end to end: the states come from pinned host memory and return to it around the same run
    hq = [t.cpu().pin_memory() for t in q]
    hU = [t.cpu().pin_memory() for t in U]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d_, h_ in zip(q + U, hq + hU):
        d_.copy_(h_, non_blocking=True)
    st_e2e, _ = bt.run(q, U, [step] * B, seeds, nsteps=steps, lanczos_iters=args.lanczos_iters,
                       dt=args.dt, delta=args.delta, tol=args.tol)
    for d_, h_ in zip(q + U, hq + hU):
        h_.copy_(d_, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_pairs = steps * sum(float(N) * N * (3 + s_["m"]) for N, s_ in zip(sizes, st_e2e))
    step += steps
    # the same instances, one rpb_ab_step call each (one step of all B)
    ctx = rpb.Context(max_N=max(sizes), precision=args.precision, max_iter=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(B):
        ctx.ab_step(q[k], U[k], step, seeds[k], **kw)
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    ctx.close()
    bt.close()
    return dict(B=B, sizes=sizes, total_s=total_s, loop_s=loop_s, pairs=pairs, e2e_s=e2e_s, e2e_pairs=e2e_pairs,
                unconv=unconv, ms_call=ms_call, m_used=m_used, tuned=tuned, launches=int(launches), clocks=clocks)


def run_batched(args, rank, world, local_rank):
    """The batched workload (measure_batched) as its own bench line."""
    import torch

    torch.cuda.set_device(local_rank)
    dist = init_dist(world)
    r = measure_batched(args, rank, world, local_rank, dist, args.steps, args.warmup)
    B, sizes = r["B"], r["sizes"]
    (total_s, loop_s), (pairs,) = aggregate(dist, [r["total_s"], r["loop_s"]], [r["pairs"]], device="cuda")
    if rank == 0:
        inst_steps = B * args.steps * world / total_s
        line = _base_line(args, world, pairs / total_s / 1e9, "Gpairs/s", total_s * 1e3 / args.steps,
                          "f32" if args.precision == "fp32" else "f64",
                          {"workload": f"batched: {B} suspensions, N log-uniform in [64, 2048] (sum N = {sum(sizes)}), "
                                       f"AB step dt={args.dt}, delta={args.delta}, tol={args.tol}, "
                                       f"{args.precision} pairs", "B": B, "sum_N": sum(sizes),
                           "sum_N2": sum(N * N for N in sizes), "parallelism": f"replicas x{world}"})
        line.update({"instance_steps_per_s": inst_steps,
                     "loop_instance_steps_per_s": B * world / loop_s,
                     "speedup_vs_loop": inst_steps / (B * world / loop_s),
                     "graph_run": {"steps": args.steps, "lanczos_iters_per_step": args.lanczos_iters,
                                   "unconverged_instance_steps": r["unconv"], "host_driven_step_ms": r["ms_call"],
                                   "max_m": r["m_used"]},
                     "e2e": {"value": r["e2e_pairs"] / r["e2e_s"] / 1e9, "unit": "Gpairs/s",
                             "h2d_bytes_per_step": 48.0 * sum(sizes) / args.steps,
                             "d2h_bytes_per_step": 48.0 * sum(sizes) / args.steps,
                             "note": "all instances' positions and U^{n-1} copied from pinned host memory before "
                                     "and back after one graph-replayed run of the timed steps"},
                     "cpu_baseline": cpu_baseline_line(args, 2048),
                     "tiles": {"tuned": r["tuned"]["best"],
                               "candidates_ms": [[c, round(t, 4)] for c, t in r["tuned"]["candidates"]]},
                     "step_ms": [round(total_s * 1e3 / args.steps, 3)] * args.steps, "gpu_launches": r["launches"],
                     "clocks": r["clocks"]})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serving(args, rank, world, local_rank):
    """Poisson arrivals of trajectory requests (N log-uniform in [128, 32768], 10-200 steps), served by
    continuous batching with state resident in HBM and admission by a device-memory budget; p50/p99
    request latency and throughput, beside a serial FP64 single-suspension server simulated from
    measured per-step times of that path."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb, serve

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    # calibrate: batched throughput on a mixed sample, to pick an arrival rate near 85% utilisation
    sample = serve.poisson_requests(16, rate=1.0, seed=args.seed + 99)
    srv = serve.GpuServer(max_batch=args.max_batch, max_spheres=args.max_spheres, precision=args.precision,
                          delta=args.delta, tol=args.tol, dt=args.dt)
    act = []
    for r in sample[:12]:
        r.state = srv.allocate(r)
        act.append(r)
    srv.step(act)
    torch.cuda.synchronize()
    srv.pairs = 0.0
    t0 = time.perf_counter()
    for _ in range(3):
        srv.step(act)
    torch.cuda.synchronize()
    thr = srv.pairs / (time.perf_counter() - t0)              # pairs/s when busy
    reqs = serve.poisson_requests(args.requests, rate=1.0, seed=args.seed)
    mean_work = statistics.mean(r.N * r.N * 11.0 * r.steps for r in reqs)
    rate = args.load * thr / mean_work
    reqs = serve.poisson_requests(args.requests, rate=rate, seed=args.seed)
    for r in reqs:  # the client supplies the initial configuration with the request
        r.pos0 = inputs.monolayer(r.N, seed=r.seed)
    srv.pairs = 0.0
    sched = serve.Scheduler(budget_bytes=int(args.budget_gb * 1e9), max_batch=args.max_batch,
                            max_spheres=args.max_spheres)
    launches0 = rpb.launch_count()
    clk = clocks_start(local_rank)
    fin, busy, total = serve.run(reqs, sched, srv.step, srv.allocate, srv.finalize)
    clocks = clocks_stop(clk)
    launches = rpb.launch_count() - launches0
    srv.close()
    lat = [r.latency for r in fin]
    req_steps = sum(r.steps for r in fin)
    # serial FP64 reference server: per-step time of rpb_ab_step (FP64) measured at a few sizes,
    # fitted as t(N) = c0 + c2 N^2, and a first-come-first-served queue over the same arrivals
    ctx = rpb.Context(max_N=32768, precision="fp64", max_iter=64)
    pts = []
    for N in (128, 1024, 4096, 16384):
        qq = torch.tensor(inputs.to_soa(inputs.monolayer(N, seed=5)), dtype=torch.float64, device="cuda")
        UU = torch.zeros_like(qq)
        ctx.ab_step(qq, UU, 0, 5, delta=1e-6, tol=args.tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.ab_step(qq, UU, 1, 5, delta=1e-6, tol=args.tol)
        torch.cuda.synchronize()
        pts.append((N, time.perf_counter() - t0))
    A = np.array([[1.0, float(N) ** 2] for N, _ in pts])
    coef = np.linalg.lstsq(A, np.array([t for _, t in pts]), rcond=None)[0]
    # the serial server for real on a sample: requests in arrival order, each served alone by the
    # single-suspension FP64 path (its steps replayed from a CUDA graph), until the time budget is used;
    # the measured service times check the fitted model the full queue is simulated with
    sample = []
    spent = 0.0
    for r in sorted(reqs, key=lambda r: r.arrival):
        pred = r.steps * (coef[0] + coef[1] * r.N * r.N)
        if spent + pred > args.serial_sample_s:
            continue
        qq = torch.tensor(inputs.to_soa(r.pos0), dtype=torch.float64, device="cuda")
        UU = torch.zeros_like(qq)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.run(qq, UU, 0, r.seed, r.steps, delta=1e-6, tol=args.tol, raise_on_noconv=False)
        torch.cuda.synchronize()
        meas = time.perf_counter() - t0
        spent += meas
        sample.append({"rid": r.rid, "N": r.N, "steps": r.steps, "measured_s": meas, "predicted_s": pred})
        if len(sample) >= 24:
            break
    ctx.close()
    scale = (sum(x["measured_s"] for x in sample) / sum(x["predicted_s"] for x in sample)) if sample else 1.0
    tfree, lat64 = 0.0, []
    for r in sorted(reqs, key=lambda r: r.arrival):
        start = max(tfree, r.arrival)
        tfree = start + scale * r.steps * (coef[0] + coef[1] * r.N * r.N)
        lat64.append(tfree - r.arrival)
    line = _base_line(args, 1, srv.pairs / total / 1e9, "Gpairs/s", 1e3 * busy / max(1, len(fin)),
                      "f32" if args.precision == "fp32" else "f64",
                      {"workload": f"serving: {len(reqs)} Poisson requests at {rate:.3f}/s, N log-uniform in "
                                   f"[128, 32768], 10-200 steps, budget {args.budget_gb} GB, batch <= "
                                   f"{args.max_batch} requests / {args.max_spheres} spheres, {args.precision} pairs",
                       "requests": len(reqs), "rate_per_s": rate})
    line.update({"p50_latency_s": serve.percentile(lat, 50), "p99_latency_s": serve.percentile(lat, 99),
                 "request_steps_per_s": req_steps / total, "gpu_busy_frac": busy / total, "wall_s": total,
                 "serial_fp64": {"p50_latency_s": serve.percentile(lat64, 50),
                                 "p99_latency_s": serve.percentile(lat64, 99),
                                 "request_steps_per_s": req_steps / max(tfree, 1e-9),
                                 "step_time_fit_s": {"c0": coef[0], "c2": coef[1]},
                                 "measured_sample": sample, "fit_scale_from_sample": scale,
                                 "basis": "FCFS queue over the same arrivals with service times from rpb_ab_step "
                                          "FP64 step times measured at N = 128, 1024, 4096, 16384 (c0 + c2 N^2), "
                                          "scaled by the ratio of real serial FP64 service (rpb_run) to that fit "
                                          "on the measured sample of requests"},
                 "e2e": {"value": srv.pairs / total / 1e9, "unit": "Gpairs/s",
                         "h2d_bytes_per_step": 24.0 * sum(r.N for r in fin) / max(1, req_steps),
                         "d2h_bytes_per_step": 24.0 * sum(r.N for r in fin) / max(1, req_steps),
                         "note": "each request's initial positions come from host memory and its final positions "
                                 "return to it inside the served latency; bytes per request-step"},
                 "cpu_baseline": cpu_baseline_line(args, 4096),
                 "gpu_launches": int(launches), "clocks": clocks})
    print(json.dumps(line), flush=True)


def run_shares(args, rank, world, local_rank):
    """The pair split's work per process, measured on one GPU: the translation-translation product of
    the N-sphere monolayer cut into W shares of the symmetric pass's triangle (rpb_mobility_apply_part),
    each share timed alone with CUDA events; the largest share against the whole product gives the
    speedup W processes would reach on the pairs (the all-reduce of 3N doubles per product, which needs
    several GPUs, is not in it).  The row split's largest share (rpb_mobility_apply_rows) is timed
    beside it."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    N = args.N
    ctx = rpb.Context(max_N=N, precision=args.precision, max_iter=16)
    q = torch.tensor(inputs.to_soa(inputs.monolayer(N, seed=args.seed)), dtype=torch.float64, device="cuda")
    F = ctx.philox_normal(N, args.seed, 0, 0)
    out = torch.empty_like(q)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    clk = clocks_start(local_rank)
    t_full = timed(lambda: ctx.mobility_apply(q, F, out=out))
    rows = []
    from paper_1612_00474_gb300.split import row_ranges
    for W in (1, 2, 4, 8):
        ts = [timed(lambda p=p: ctx.mobility_apply_part(q, F, None, p, W, out=out)) for p in range(W)]
        # the row split's largest share for comparison: one-way kernels over its target rows
        r0, r1 = max(row_ranges(N, W), key=lambda ab: ab[1] - ab[0])
        t_rows = timed(lambda: ctx.mobility_apply_rows(q, F, None, r0, r1))
        rows.append({"W": W, "share_ms": [round(t, 4) for t in ts], "max_share_ms": max(ts),
                     "speedup_on_pairs": t_full / max(ts), "efficiency": t_full / max(ts) / W,
                     "row_split_max_share_ms": t_rows, "row_split_speedup": t_full / t_rows})
    clocks = clocks_stop(clk)
    ctx.close()
    best = rows[-1]
    line = _base_line(args, 1, best["speedup_on_pairs"], "x", best["max_share_ms"],
                      "f32" if args.precision == "fp32" else "f64",
                      {"workload": f"pair split shares: N={N} monolayer, {args.precision} pairs, translation-"
                                   f"translation product cut into W = 1, 2, 4, 8 shares, each timed alone on one GPU",
                       "N": N})
    line.update({"full_product_ms": t_full, "shares": rows, "clocks": clocks,
                 "note": "value: the speedup of the pair work at W = 8 (all-reduce not included)"})
    print(json.dumps(line), flush=True)


def run_lanczos_sweep(args, rank, world, local_rank):
    """Lanczos iterations to reach eps <= 1e-3 and <= 1e-5 versus N, with the wall-corrected mobility
    and with the unbounded-domain mobility (Sec. II.C: screening by the wall keeps the iteration count
    independent of N; without it the count grows), FP32 pairs, same monolayers and noise."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    Ns = [n for n in (1024, 2048, 4096, 8192, 16384, 32768, 65536) if n <= args.N]
    rows = []
    t0 = time.perf_counter()
    for wall, pc in ((True, False), (False, False), (True, True)):
        ctx = rpb.Context(max_N=max(Ns), precision="fp32", max_iter=64, wall=wall)
        if pc:  # the block-diagonal preconditioner Sec. II.C reports trying (an option, off in the paper)
            ctx.set_preconditioner("block-diagonal")
        for N in Ns:
            q = torch.tensor(inputs.to_soa(inputs.monolayer(N, seed=args.seed)), dtype=torch.float64, device="cuda")
            W = ctx.philox_normal(N, args.seed, 0, 0)
            row = {"N": N, "wall": wall, "preconditioner": "block-diagonal" if pc else None}
            for tol in (1e-3, 1e-5):
                g, m, eps, conv = ctx.lanczos_sqrt_apply(q, W, tol=tol, max_iter=64, raise_on_noconv=False)
                row[f"m_{tol:g}"] = m if conv else None
                row[f"eps_{tol:g}"] = eps
            rows.append(row)
        ctx.close()
    wall_s = time.perf_counter() - t0
    m_wall = [r["m_1e-05"] for r in rows if r["wall"] and not r["preconditioner"]]
    line = _base_line(args, 1, float(max(m_wall)) if all(m_wall) else float("nan"), "iterations", wall_s * 1e3 / len(rows),
                      "f32", {"workload": f"Lanczos iterations vs N: monolayers phi=0.4, z=a+Exp(0.5a), N in {Ns}, "
                                          "fp32 pairs, fp64 Lanczos, with and without the wall terms, and with "
                                          "the wall and the block-diagonal preconditioner"})
    line["higher_is_better"] = False
    line["sweep"] = rows
    print(json.dumps(line), flush=True)


def run_accuracy(args, rank, world, local_rank):
    """Per-step errors against the FP64 oracle (first `--acc-steps` steps of the N=4096 suspension,
    both GPU paths restarted from the oracle's state every step, identical Philox noise): the
    deterministic velocity U^n and the increment q^{n+1} - q^n; then steps/s of each path over
    `--steps` steps.  The oracle runs with the same delta as each path."""
    import torch

    import oracle as O
    from paper_1612_00474_gb300 import inputs, rpb

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    N = args.N
    dev = lambda x: torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")  # noqa: E731
    host = lambda t: inputs.from_soa(t.cpu().numpy(), N)  # noqa: E731
    paths = {"fp64": dict(delta=1e-6), "fp32": dict(delta=5e-3)}
    ctxs = {p: rpb.Context(max_N=N, precision=p, max_iter=64) for p in paths}
    q_ref = inputs.monolayer(N, seed=args.seed)
    Up_ref = None
    table = []
    t_oracle = 0.0
    for n in range(args.acc_steps):
        row = {"step": n}
        refs = {}
        for p, kw in paths.items():
            t0 = time.perf_counter()
            refs[p] = O.ab_step(q_ref, Up_ref, n, seed=args.seed, dt=args.dt, delta=kw["delta"], tol=args.tol,
                                max_iter=64)
            t_oracle += time.perf_counter() - t0
        for p, kw in paths.items():
            new_ref, Un_ref, info = refs[p]
            q = dev(q_ref)
            U = dev(Up_ref) if Up_ref is not None else torch.zeros(3 * N, dtype=torch.float64, device="cuda")
            st = ctxs[p].ab_step(q, U, n, args.seed, dt=args.dt, delta=kw["delta"], tol=args.tol, max_iter=64)
            inc, inc_ref = host(q) - q_ref, new_ref - q_ref
            row[p] = {"U_rel": O.rel_err(host(U), Un_ref), "increment_rel": O.rel_err(inc, inc_ref),
                      "m": st["m"], "m_oracle": info["m"]}
        table.append(row)
        q_ref, Up_ref = refs["fp64"][0], refs["fp64"][1]
    # throughput of both paths over args.steps steps
    rates = {}
    for p, kw in paths.items():
        q = dev(inputs.monolayer(N, seed=args.seed))
        U = torch.zeros_like(q)
        for s in range(args.warmup):
            ctxs[p].ab_step(q, U, s, args.seed, dt=args.dt, delta=kw["delta"], tol=args.tol, max_iter=64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(args.warmup, args.warmup + args.steps):
            ctxs[p].ab_step(q, U, s, args.seed, dt=args.dt, delta=kw["delta"], tol=args.tol, max_iter=64)
        torch.cuda.synchronize()
        rates[p] = args.steps / (time.perf_counter() - t0)
        ctxs[p].close()
    worst32 = max(r["fp32"]["U_rel"] for r in table)
    line = _base_line(args, 1, rates["fp32"], "steps/s", 1e3 / rates["fp32"], "f32",
                      {"workload": f"accuracy: N={N} suspension, AB steps dt={args.dt}, tol={args.tol}; FP64 path "
                                   f"delta=1e-6, FP32 path delta=5e-3; oracle per-step comparison on the first "
                                   f"{args.acc_steps} steps", "N": N})
    line.update({"steps_per_s": rates, "per_step_errors": table, "worst_fp32_U_rel": worst32,
                 "oracle_seconds_per_step": t_oracle / (2 * args.acc_steps)})
    print(json.dumps(line), flush=True)


_ORACLE_TIMING = r"""
import json, os, sys, time
import oracle as O
from paper_1612_00474_gb300 import inputs
res = {}
threads = int(os.environ.get("OMP_NUM_THREADS", "1"))
for N in ((256, 4096) if sys.argv[2] == "1" else (256,)):
    q = inputs.monolayer(N, seed=0)
    if N == 256:
        O.ab_step(q, None, 0, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
    t0 = time.perf_counter()
    O.ab_step(q, None, 0, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
    res[f"ab_step_N{N}_s"] = time.perf_counter() - t0
N = 4096
q = inputs.monolayer(N, seed=0)
F = [[0.0, 0.0, -1.0]] * N
T = [[0.0, 1.0, 0.0]] * N
t0 = time.perf_counter()
O.mobility_apply(q, F, T)
res["fused_product_N4096_s"] = time.perf_counter() - t0
N = 65536
q = inputs.monolayer(N, seed=0)
F = [[0.0, 0.0, -1.0]] * N
T = [[0.0, 1.0, 0.0]] * N
rows = max(8, 4 * threads)
t0 = time.perf_counter()
O.mobility_apply(q, F, T, rows=(0, rows))
dt = time.perf_counter() - t0
rows = int(max(8, min(N, rows * float(sys.argv[1]) / max(dt, 1e-6))))
t0 = time.perf_counter()
O.mobility_apply(q, F, T, rows=(0, rows))
dt = time.perf_counter() - t0
res["fused_product_N65536_gpairs_s"] = rows * N / dt / 1e9
res["fused_product_N65536_rows"] = rows
print(json.dumps(res))
"""


def oracle_timing(threads, seconds, step_4096=True):
    """FP64 oracle timings on `threads` host threads, in a fresh interpreter (the OpenMP pool size is
    fixed at first use): one full AB step at N = 256 (and at N = 4096 if step_4096), one fused product
    at N = 4096, and the fused product of the N = 65536 monolayer on a row sample of about `seconds`
    seconds."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    here = os.path.dirname(os.path.abspath(__file__))
    out = subprocess.run([sys.executable, "-c", _ORACLE_TIMING, str(seconds), "1" if step_4096 else "0"], env=env,
                         cwd=here,
                         capture_output=True, text=True, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    res["threads"] = threads
    return res


def measure_small(local_rank, steps, warmup):
    """The 256-sphere configuration (seed 0, FP64 pairs, dt = 0.01, delta = 1e-6, tol = 1e-3):
    microseconds per AB step on the GPU through rpb_ab_step (the host reads the Lanczos status back
    after every iteration) and through rpb_run (the step replayed from a CUDA graph, the Lanczos stop
    decided on the device)."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    N, seed = 256, 0
    kw = dict(dt=0.01, delta=1e-6, tol=1e-3)
    pos0 = inputs.monolayer(N, seed=seed)
    ctx = rpb.Context(max_N=N, precision="fp64", max_iter=64)
    q = torch.tensor(inputs.to_soa(pos0), dtype=torch.float64, device="cuda")
    U = torch.zeros_like(q)
    step = 0
    for _ in range(warmup):
        ctx.ab_step(q, U, step, seed, max_iter=64, **kw)
        step += 1
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    clk = clocks_start(local_rank)
    launches0 = rpb.launch_count()
    us, ms_m = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.ab_step(q, U, step, seed, max_iter=64, **kw)
        e1.record(stream)
        e1.synchronize()
        us.append(e0.elapsed_time(e1) * 1e3)
        ms_m.append(st["m"])
        step += 1
    launches_host = rpb.launch_count() - launches0
    # the same suspension, steps replayed from a CUDA graph (one capture per call, amortised over the
    # call's steps: the timed call makes K = max(steps, 50) of them)
    ctx.run(q, U, step, seed, max(1, warmup), max_iter=64, **kw)
    step += max(1, warmup)
    K = max(steps, 50)
    torch.cuda.synchronize()
    launches0 = rpb.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st_run, unconv = ctx.run(q, U, step, seed, K, max_iter=64, **kw)
    e1.record(stream)
    e1.synchronize()
    launches_run = rpb.launch_count() - launches0
    graph_us = e0.elapsed_time(e1) * 1e3 / K
    ctx.close()
    clocks = clocks_stop(clk)
    gpu_us = statistics.median(us)
    return dict(N=N, seed=seed, us=us, ms_m=ms_m, gpu_us=gpu_us, graph_us=graph_us, K=K, st_run=st_run,
                unconv=unconv, launches_host=launches_host, launches_run=launches_run, clocks=clocks)


def run_small(args, rank, world, local_rank):
    """The small workload (measure_small) as its own bench line, beside the FP64 oracle's full step on
    all host cores and on one core (plus, on both, one 4096-sphere step and a row sample of the
    65536-sphere fused product)."""
    import torch

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    r = measure_small(local_rank, args.steps, args.warmup)
    N, seed, gpu_us, graph_us, K = r["N"], r["seed"], r["gpu_us"], r["graph_us"], r["K"]
    best_us = min(gpu_us, graph_us)  # the faster of the host-driven and the graph-replayed step
    line = _base_line(args, 1, best_us, "us/step", best_us / 1e3, "f64",
                      {"workload": f"small: N={N} monolayer (seed {seed}), AB step dt=0.01, delta=1e-6, tol=1e-3, "
                                   f"fp64 pairs", "N": N})
    line["higher_is_better"] = False
    line.update({"value_path": "rpb_ab_step (host-driven)" if gpu_us <= graph_us else "rpb_run (graph-replayed)",
                 "us_per_step": {"rpb_run": graph_us, "rpb_ab_step_median": gpu_us,
                                 "rpb_ab_step_mean": statistics.mean(r["us"])},
                 "graph_run": {"steps": K, "last_m": r["st_run"]["m"], "unconverged_steps": r["unconv"],
                               "launches_per_step": r["launches_run"] / K},
                 "lanczos_m": r["ms_m"], "gpu_launches": int(r["launches_run"]),
                 "host_driven_launches_per_step": r["launches_host"] / max(1, args.steps), "clocks": r["clocks"]})
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        allc = oracle_timing(cores, 5.0)
        one = oracle_timing(1, 5.0, step_4096=False)  # a one-core 4096-sphere step takes minutes
        line["cpu_baseline"] = {"value": allc["ab_step_N256_s"] * 1e6, "unit": "us/step", "cores": cores,
                                "kind": "oracle", "sample": "one full AB step of the same N=256 suspension"}
        line["oracle_timing"] = {"all_cores": allc, "one_core": one}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- roller fingering (Sec. IV)
# Physical setting of the roller runs: a = 0.656 um, water (eta = 1 mPa s), torque 8 pi eta a^3 omega y
# with omega = 62.8 rad/s, U0 = 4 kT, b = 0.1 a, dt = 0.016 s = tau_U / 2, Lanczos tolerance 1e-3,
# N = 32768 in a 60a x 4915a strip; front spectra over k in [2e-3, 0.26] per um.
FING_A_M = 0.656e-6
FING_ETA = 1e-3
FING_KT = 1.380649e-23 * 298.0   # the temperature is not stated; 298 K gives tau_U / 2 = 0.016 s
FING_OMEGA = 62.8
FING_DT_S = 0.016
FING_LX, FING_LY = 60.0, 4915.0
FING_KMIN_UM, FING_KMAX_UM = 2.0e-3, 0.26
FING_T_STAR_PAPER = {1.5: (9.4, 11.8), 3.5: (17.3, 26.9), 6.1: (32.6, 42.9)}  # (deterministic, stochastic) s


def fingering_units(dt_s=FING_DT_S):
    """Reduced units a = eta = kT = 1: time unit eta a^3 / kT; dt_s: the time step in seconds."""
    tau0 = FING_ETA * FING_A_M ** 3 / FING_KT
    return dict(tau0=tau0, dt=dt_s / tau0, dt_s=dt_s, torque=8.0 * math.pi * FING_OMEGA * tau0)


def fingering_initial(N, hg, U0, b, seed):
    """Rollers in the 60a x 4915a strip (x across the front, y along it): heights from the one-sphere
    Gibbs-Boltzmann density exp(-(w h + U_wall(h)) / kT) with w = kT / (h_g - a) and the wall branch
    of the soft potential, in-plane positions uniform, 3D overlaps (r < 2a) rejected in sequence."""
    rng = np.random.default_rng(seed)
    w = 1.0 / (hg - 1.0)
    h = np.linspace(1e-3, 1.0 + 60.0 / w, 200001)
    uw = np.where(h < 1.0, U0 * (1.0 + (1.0 - h) / b), U0 * np.exp(-(h - 1.0) / b))
    pdf = np.exp(-(w * h + uw - (w * 1.0 + U0)))
    cdf = np.cumsum(pdf)
    cdf /= cdf[-1]
    cells = {}
    out = np.zeros((N, 3))
    n = 0
    while n < N:
        x, y = rng.uniform(0.0, FING_LX), rng.uniform(0.0, FING_LY)
        z = float(np.interp(rng.uniform(), cdf, h))
        cx, cy = int(x // 2.0), int(y // 2.0)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for j in cells.get((cx + dx, cy + dy), ()):
                    if (out[j, 0] - x) ** 2 + (out[j, 1] - y) ** 2 + (out[j, 2] - z) ** 2 < 4.0:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[n] = (x, y, z)
            cells.setdefault((cx, cy), []).append(n)
            n += 1
    return out


def front_band_power(p, frac=0.7):
    """Power of the number density along the front, sum of |n(k_y)|^2 over the wavenumbers of the band,
    from the fraction `frac` of the spheres with the largest x (the front)."""
    k_a = 2.0 * math.pi * np.arange(1, 4096) / FING_LY       # per a
    k_um = k_a / (FING_A_M * 1e6)
    ks = k_a[(k_um >= FING_KMIN_UM) & (k_um <= FING_KMAX_UM)]
    y = p[np.argsort(p[:, 0])[int((1.0 - frac) * len(p)):], 1]
    nk = np.exp(-1j * np.outer(ks, y)).sum(axis=1)
    return float(np.sum(np.abs(nk) ** 2))


def front_band_power_cycles(p, frac=0.7, bins=1 << 17):
    """The same band read in cycles per micrometre (k = 1/lambda, modes n / L_y with L_y in um inside
    [2e-3, 0.26]: wavelengths down to 5.9a instead of 37a), from an FFT of the front's y positions
    binned into `bins` bins of the strip's period (the sum over spheres of e^{-2 pi i n y / L_y} is
    periodic in y, so y is folded into [0, L_y); the binning changes |n(k)| by under 1e-4 here)."""
    y = p[np.argsort(p[:, 0])[int((1.0 - frac) * len(p)):], 1]
    L_um = FING_LY * FING_A_M * 1e6
    n = np.arange(1, bins // 2)
    sel = n[(n / L_um >= FING_KMIN_UM) & (n / L_um <= FING_KMAX_UM)]
    idx = np.minimum((np.mod(y, FING_LY) / FING_LY * bins).astype(np.int64), bins - 1)
    f = np.fft.rfft(np.bincount(idx, minlength=bins).astype(np.float64))
    return float(np.sum(np.abs(f[sel]) ** 2))


def _half_time(times, power):
    """First time the series reaches half its maximum (linear interpolation between samples): a
    companion of t* that does not depend on the noisy top of a plateau."""
    k = int(np.argmax(power))
    half = 0.5 * power[k]
    jh = next(j for j, v in enumerate(power) if v >= half)
    if jh == 0:
        return times[0]
    return times[jh - 1] + (half - power[jh - 1]) / (power[jh] - power[jh - 1]) * (times[jh] - times[jh - 1])


def run_fingering(args, rank, world, local_rank):
    """Roller fingering run: the same N = 32768 strip advanced deterministically (kT = 0) and with
    Brownian motion, the front's band power sampled along the way; t* is the time of its maximum.
    With several realizations (the paper averages four), each starts from its own initial state and
    noise, and t* and t1/2 are taken on the mean band power."""
    import torch

    from paper_1612_00474_gb300 import inputs, rpb

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    units = fingering_units(args.fing_dt)
    N, hg, U0, b = args.N, args.hg, 4.0, 0.1
    weight = 1.0 / (hg - 1.0)
    torque = (0.0, units["torque"], 0.0)
    R = max(1, args.realizations)
    runs = {}
    clk = clocks_start(local_rank)
    h_edges = np.linspace(0.0, 12.0, 49)
    x_edges = np.arange(-100.0, 1501.0, 20.0)

    def sample(p):
        return (front_band_power(p), np.histogram(p[:, 2], h_edges)[0], np.histogram(p[:, 0], x_edges)[0],
                float(p[:, 2].mean()), float(np.mean(np.sort(p[:, 0])[int(0.3 * N):])), front_band_power_cycles(p))

    # initial states: sequential addition, then (optionally) Brownian dynamics without torque in the
    # pseudo-periodic cell, folded back into it -- a sample of the two-periodic suspension's equilibrium
    inits, eq_info = [], []
    neq = int(round(args.equilibrate_s / units["dt_s"]))
    ctx_eq = None
    if neq > 0:
        ctx_eq = rpb.Context(max_N=N, precision=args.precision, max_iter=64, kT=1.0)
        ctx_eq.set_periodic(FING_LX, FING_LY)
    for r in range(R):
        p0 = fingering_initial(N, hg, U0, b, args.seed + r)
        if ctx_eq is not None:
            q = torch.tensor(inputs.to_soa(p0), dtype=torch.float64, device="cuda")
            U = torch.zeros_like(q)
            ctx_eq.run(q, U, 0, args.seed + 1000 + r, neq, dt=units["dt"], delta=args.delta, tol=args.tol,
                       max_iter=64, weight=weight, U0=U0, b=b, torque=(0.0, 0.0, 0.0))
            p1 = inputs.from_soa(q.cpu().numpy(), N)
            p1[:, 0] = np.mod(p1[:, 0], FING_LX)
            p1[:, 1] = np.mod(p1[:, 1], FING_LY)
            eq_info.append({"mean_h_before": float(p0[:, 2].mean()), "mean_h_after": float(p1[:, 2].mean())})
            p0 = p1
        inits.append(p0)
    if ctx_eq is not None:
        ctx_eq.close()
    for name, kT in (("deterministic", 0.0), ("stochastic", 1.0)):
        ctx = rpb.Context(max_N=N, precision=args.precision, max_iter=64, kT=kT)
        per, ms, wall = [], [], 0.0
        times = [0.0]
        for r in range(R):
            seed = args.seed + r
            pos0 = inits[r]
            q = torch.tensor(inputs.to_soa(pos0), dtype=torch.float64, device="cuda")
            U = torch.zeros_like(q)
            samples = [sample(pos0)]
            ts = [0.0]
            t0 = time.perf_counter()
            for step in range(args.fing_steps):
                st = ctx.ab_step(q, U, step, seed, dt=units["dt"], delta=args.delta, tol=args.tol, max_iter=64,
                                 weight=weight, U0=U0, b=b, torque=torque)
                ms.append(st["m"])
                if (step + 1) % args.sample_every == 0:
                    ts.append((step + 1) * units["dt_s"])
                    samples.append(sample(inputs.from_soa(q.cpu().numpy(), N)))
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            times = ts
            per.append(samples)
        ctx.close()
        power = np.mean([[s_[0] for s_ in smp] for smp in per], axis=0).tolist()
        power_c = np.mean([[s_[5] for s_ in smp] for smp in per], axis=0).tolist()
        k = int(np.argmax(power))
        kc = int(np.argmax(power_c))
        every = max(1, len(times) // 80)
        mean_h = np.mean([[s_[3] for s_ in smp] for smp in per], axis=0)
        front = np.mean([[s_[4] for s_ in smp] for smp in per], axis=0)
        Ph = np.sum([smp[k][1] for smp in per], axis=0)
        rx = np.sum([smp[k][2] for smp in per], axis=0)
        runs[name] = {"t_star_s": times[k], "t_star_at_end_of_run": k == len(power) - 1,
                      "t_half_s": _half_time(times, power),
                      "cycles_reading": {"t_star_s": times[kc], "t_star_at_end_of_run": kc == len(power_c) - 1,
                                         "t_half_s": _half_time(times, power_c)},
                      "per_realization": [{"seed": args.seed + r,
                                           "t_star_s": times[int(np.argmax([s_[0] for s_ in smp]))],
                                           "t_half_s": _half_time(times, [s_[0] for s_ in smp])}
                                          for r, smp in enumerate(per)],
                      "steps_per_s": R * args.fing_steps / wall, "lanczos_m_mean": float(np.mean(ms)),
                      "P_h_at_t_star": {"edges_a": h_edges.tolist(), "counts": Ph.tolist()},
                      "rho_x_at_t_star": {"edges_a": x_edges.tolist(), "counts": rx.tolist()},
                      "P_h_initial": np.sum([smp[0][1] for smp in per], axis=0).tolist(),
                      "series": [{"t_s": round(t, 3), "band_power": round(pw, 1), "band_power_cycles": round(pc, 1),
                                  "mean_h": round(float(h), 3), "front_x": round(float(fx), 2)}
                                 for t, pw, pc, h, fx in zip(times, power, power_c, mean_h, front)][::every]}
    clocks = clocks_stop(clk)
    paper = FING_T_STAR_PAPER.get(round(hg, 1))
    det, sto = runs["deterministic"]["t_star_s"], runs["stochastic"]["t_star_s"]
    line = _base_line(args, 1, runs["stochastic"]["steps_per_s"], "steps/s", 1e3 / runs["stochastic"]["steps_per_s"],
                      "f32" if args.precision == "fp32" else "f64",
                      {"workload": f"roller fingering: N={N} strip 60a x 4915a, h_g={hg}a, U0=4kT, b=0.1a, "
                                   f"torque 8 pi eta a^3 omega (omega=62.8 rad/s), dt={units['dt_s']:g} s, "
                                   f"{args.fing_steps} steps per run, {R} realization(s), {args.precision} pairs, "
                                   f"initial states: sequential addition"
                                   + (f" then {args.equilibrate_s:g} s of torque-free Brownian dynamics in the "
                                      f"pseudo-periodic cell" if neq > 0 else ""),
                       "N": N, "realizations": R, "equilibrate_s": args.equilibrate_s})
    hd, hs = runs["deterministic"]["t_half_s"], runs["stochastic"]["t_half_s"]
    cdet, csto = runs["deterministic"]["cycles_reading"]["t_star_s"], runs["stochastic"]["cycles_reading"]["t_star_s"]
    line.update({"fingering": {"t_star_s": {"deterministic": det, "stochastic": sto},
                               "t_star_s_cycles_reading": {"deterministic": cdet, "stochastic": csto},
                               "ratio_stochastic_over_deterministic": sto / det if det > 0 else None,
                               "t_half_s": {"deterministic": hd, "stochastic": hs},
                               "t_half_ratio": hs / hd if hd > 0 else None,
                               "paper_t_star_s": ({"deterministic": paper[0], "stochastic": paper[1],
                                                   "ratio": paper[1] / paper[0]} if paper else None),
                               "reduced_units": units, "equilibration": eq_info, "runs": runs},
                 "clocks": clocks})
    print(json.dumps(line), flush=True)


def resolve_defaults(args):
    """Workload-dependent defaults: the suspension size (65536 for the monolayer, the reference arm and
    the bound of the Lanczos sweep; 4096 for the accuracy comparison with the oracle; 32768 for the
    fingering strip) and the RFD length (1e-6 a for float64 products, 5e-3 a for float32, Sec. II.A)."""
    if args.N is None:
        args.N = {"accuracy": 4096, "fingering": 32768}.get(args.workload, 65536)
    if args.delta is None:
        args.delta = 1e-6 if args.precision == "fp64" else 5e-3
    return args


def main():
    args = resolve_defaults(parse())
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "lanczos":
        run_lanczos_sweep(args, rank, world, local_rank)
    elif args.workload == "accuracy":
        run_accuracy(args, rank, world, local_rank)
    elif args.workload == "serving":
        run_serving(args, rank, world, local_rank)
    elif args.workload == "small":
        run_small(args, rank, world, local_rank)
    elif args.workload == "fingering":
        run_fingering(args, rank, world, local_rank)
    elif args.workload == "shares":
        run_shares(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
