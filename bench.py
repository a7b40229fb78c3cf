#!/usr/bin/env python3
"""Throughput benchmark of the GB300 one-way quantum computer simulator.

One step = one full simulation of the brickwork cluster pattern, 28 rows x
40 columns (1120 qubits, 1092 measurements, angles k pi/4, |+>^28 input,
forced seeded outcomes) under the greedy reordering (peak 29 live qubits):
1092 measure passes over 2^28 complex64 amplitudes plus the output pass.
The metric is amplitude-updates per second: every command counts 2^(live
width) amplitude updates (N after it, M before elimination), summed by the
library over the schedule.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl owqs|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload family instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-updates/s and % HBM peak, FP32 vs FP64 GPU at ≤2e-5 amp error"
UNIT = "amplitude-updates/s"
ROWS, COLS = 28, 40
WORKLOAD = ("brickwork cluster 28x40 (1120 qubits, 1092 measurements), angles k*pi/4, |+>^28 input, "
            "forced seeded outcomes, greedy reordering (peak 29 live qubits, 2^28 complex64 amplitudes)")


def workload_name(rows: int, cols: int) -> str:
    if (rows, cols) == (ROWS, COLS):
        return WORKLOAD
    return (f"brickwork cluster {rows}x{cols} ({rows * cols} qubits), angles k*pi/4, |+>^{rows} input, "
            f"forced seeded outcomes, greedy reordering (a reduced size of the 28x40 workload)")
FALLBACK_HBM_GBS = 6800.0
# ncu DRAM bytes (read + write) per launch of the dominant kernel, keyed by the
# sha256 prefix of the pass-group sources they were measured on (a changed
# kernel reports null; comments do not count).  Both are pass groups on the full brickwork workload:
# c64, the mean over all 105 group launches of one run (k_group on 2-, 3- and
# 4-qubit registers, 2^28 complex64 amplitudes in and out, the first one
# reading the virtual input; 2127.2 MB read + 2094.4 MB written), and c128,
# the mean of three k_group64<3, 0, 0> launches (2^28 complex128; 4298.3 MB
# read + 4246.9 MB written).  profiles/k_group_c64_brickwork28x40_dram.md.
NCU_TRAFFIC = {("c92668ad8a6f4fb2", "c64"): (223356161792 + 219915724544) / 105.0,
               ("c92668ad8a6f4fb2", "c128"): (12894790144 + 12740737536) / 3.0}
# nominal GB300 FP64 rate (no measured FP64 peak exists for this machine)
FP64_PEAK_TFLOPS = 1.25
# FP64 flops per output amplitude of the complex128 pass: complex multiply-add
# (2 DMUL + 4 DFMA = 10 flops) and the squared-norm sum (DMUL + DFMA + DADD = 4)
FP64_FLOPS_PER_OUTPUT = 14
# inside a pass group: per butterfly (two outputs) the complex product
# (2 DMUL + 2 DFMA = 6 flops), two amplitude updates (4 DFMA = 8) and the
# squared norms (4 DFMA = 8): 11 flops per output; 7 in a group whose every
# probability is exactly 1/2, which sums no norms
FP64_FLOPS_PER_GROUP_OUTPUT = 11
FP64_FLOPS_PER_HALF_GROUP_OUTPUT = 7


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["owqs", "reference"], default="owqs")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end calls timed (0: --steps)")
    ap.add_argument("--cpu-meas", type=int, default=10,
                    help="measurements of the workload in each CPU-oracle sample (all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=ROWS)
    ap.add_argument("--cols", type=int, default=COLS)
    ap.add_argument("--legs", default="c64,c128,e2e,sampled,cpu,rec,learned,qft,small,substates,m",
                    help="comma list of c64 (always run), c128, e2e, sampled, cpu, rec, learned, qft, small, "
                         "substates, m; fewer legs for profiler runs")
    ap.add_argument("--sampled-steps", type=int, default=3, help="sampled-outcome runs per mode")
    ap.add_argument("--learned-count", type=int, default=200, help="held-out patterns in the learned leg")
    ap.add_argument("--rec-branches", type=int, default=64, help="outcome branches per pattern in the recognition leg")
    ap.add_argument("--rec-count", type=int, default=256, help="patterns in the recognition leg")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t: float, dist=None, device: str = "cpu") -> float:
    """Slowest rank's time (every rank gets it); t itself without a group."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(units_per_step: float, steps: int, world: int, t_max: float) -> float:
    """Whole-job throughput of N independent replicas (weak scaling): the
    units every rank processed over the slowest rank's time."""
    return units_per_step * steps * world / t_max


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="owqs_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_code(text: str) -> str:
    """C++/CUDA source without its comments and with whitespace collapsed:
    what the compiler sees, so that editing a comment keeps the key."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """sha256 prefix of the code of the pass-group sources (the dominant
    kernels), comments and whitespace left out."""
    h = hashlib.sha256()
    for name in ("owqs_group.cu", "owqs_group_c64.cuh", "owqs_group_seq.cu", "owqs_device.cuh",
                 "owqs_group_sequences.inc"):
        with open(os.path.join(ROOT, "paper_1604_05659_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(kernel_code(f.read()).encode())
    return h.hexdigest()[:16]


def oracle_sample(rows: int, cols: int, target_s: float):
    """Time the FP64 oracle (as it is) on a prefix of a brickwork pattern from
    the same generator; returns (amp-updates/s, description, seconds)."""
    from oracle import counting, proa, substate
    from owqs_inputs import workloads
    from owqs_inputs.patterns import Pattern
    wl = workloads.brickwork(rows, cols)
    p = wl.pattern
    order, _, _ = proa.proa(p)
    rp = proa.reorder_commands(p, order)
    outs = {q: int(wl.outcomes[k]) for k, q in enumerate(p.measured())}
    # calibrate on a short prefix, then size the sample to target_s
    t0 = time.perf_counter()
    substate.run(rp, None, outcomes=outs, stop_after=4)
    t4 = time.perf_counter() - t0
    nmeas = max(4, min(p.K, int(4 * target_s / max(t4, 1e-3))))
    t0 = time.perf_counter()
    substate.run(rp, None, outcomes=outs, stop_after=nmeas)
    dt = time.perf_counter() - t0
    cut, seen = 0, 0
    for i, c in enumerate(rp.cmds):
        if c.kind == "M":
            seen += 1
            if seen == nmeas:
                cut = i + 1
                break
    prefix = Pattern(rp.nqubits, list(rp.inputs), [], rp.cmds[:cut])
    upd = counting.amplitude_updates(prefix)
    desc = (f"FP64 oracle (numpy, sub-state simulator) on brickwork {rows}x{cols} from the same generator, "
            f"first {nmeas} of {p.K} measurements (live width up to {rows + 1}), {upd} amplitude updates")
    return upd / dt, desc, dt


class OraclePrefix:
    """The first `nmeas` measurements of the brickwork rows x cols pattern
    itself, under the oracle's own PROA order, as a workload for the C oracle
    (O-A with its amplitude loops on every host core): the pattern, the
    forced outcomes by label and the amplitude updates of the prefix."""

    def __init__(self, rows: int, cols: int, nmeas: int):
        from oracle import counting, proa
        from owqs_inputs import workloads
        from owqs_inputs.patterns import Pattern
        wl = workloads.brickwork(rows, cols)
        p = wl.pattern
        order, _, _ = proa.proa(p)
        self.pattern = proa.reorder_commands(p, order)
        self.outcomes = {q: int(wl.outcomes[k]) for k, q in enumerate(p.measured())}
        self.nmeas = min(nmeas, p.K)
        cut, seen = 0, 0
        for i, c in enumerate(self.pattern.cmds):
            if c.kind == "M":
                seen += 1
                if seen == self.nmeas:
                    cut = i + 1
                    break
        prefix = Pattern(self.pattern.nqubits, list(self.pattern.inputs), [], self.pattern.cmds[:cut])
        self.updates = counting.amplitude_updates(prefix)
        self.desc = (f"FP64 oracle (C sub-state simulator, OpenMP loops) on brickwork {rows}x{cols} itself, "
                     f"first {self.nmeas} of {p.K} measurements under PROA (live width {rows + 1}), "
                     f"{self.updates} amplitude updates")

    def time(self, threads: int = 0) -> float:
        from oracle import substate_c
        t0 = time.perf_counter()
        substate_c.run(self.pattern, None, outcomes=self.outcomes, stop_after=self.nmeas, threads=threads)
        return time.perf_counter() - t0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import substate_c
    cores = substate_c.max_threads()
    wl = OraclePrefix(args.rows, args.cols, args.cpu_meas)
    times = []
    for i in range(args.warmup + args.steps):
        dt = wl.time()
        if i >= args.warmup:
            times.append(dt)
    tot_t = sum(times)
    value = wl.updates * len(times) / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": workload_name(args.rows, args.cols), "sample": wl.desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": wl.desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def readout_leg(args, owqs, torch, timed):
    """Sampled OWQS on patterns without a gflow: the brickwork rows x cols
    with all of its outputs, or half of them, measured as well at seeded
    random angles (these last measurements have probabilities other than
    1/2).  Complex64, one array.  Times, per run: the forced run of one
    outcome vector, the sampled run by checked launches (a new seed every
    run; relaunches and host checks reported) and the one-measurement-at-a-
    time draw (one run)."""
    import numpy as np
    from owqs_inputs import workloads
    res = {}
    for kept in (0, args.rows // 2):
        wl = workloads.brickwork_readout(args.rows, args.cols, kept=kept)
        h = owqs.load(wl.pattern)
        _, info = h.reorder()
        out = torch.empty(1 << h.nout, dtype=torch.complex64, device="cuda")
        steps = args.sampled_steps
        forced = lambda: h.run(None, dtype="c64", outcomes=wl.outcomes, out=out, layout="one_array", check=False)
        forced()
        tf = timed(forced, steps)
        seeds = iter(range(3000, 4000))
        infos, devs = [], []

        def sampled():
            _, _, ps, _ = h.run(None, dtype="c64", policy="sampled", seed=next(seeds), out=out, layout="one_array")
            infos.append(h.last_sample_info())
            devs.append(float(np.max(np.abs(ps - 0.5))))

        sampled()
        infos.clear()
        ts = timed(sampled, steps)
        one = lambda: h.run(None, dtype="c64", policy="sampled", seed=3999, out=out, layout="one_array",
                            sequential_sampling=True)
        t1 = timed(one, 1)
        res[f"outputs_kept_{kept}"] = {
            "workload": f"brickwork {args.rows}x{args.cols} with {args.rows - kept} of its {args.rows} outputs measured "
                        f"at seeded random angles (no gflow), |+> inputs, {wl.pattern.K} measurements, peak live "
                        f"{info['peak_live']}, {info['amp_updates']} amplitude updates",
            "forced_ms_per_run": 1e3 * tf / steps,
            "checked_launches_ms_per_run": 1e3 * ts / steps,
            "one_at_a_time_ms_per_run": 1e3 * t1,
            "checked_over_forced": ts / tf,
            "paths": sorted({i["path"] for i in infos}),
            "relaunches_per_run": [i["relaunches"] for i in infos],
            "checks_per_run": [i["checks"] for i in infos],
            "max_abs_prob_minus_half": max(devs)}
        del out
        h.close()
    return res


def table3_leg(owqs):
    """The paper's m (peak sub-state at a measurement, Table III) of the
    greedy PROA order with OWQS dependencies and with every qubit ready
    (EOWQS, Section 4.5), side by side, with the width of one array over
    every live qubit, on the synthetic pattern families (host only)."""
    from owqs_inputs import workloads
    fams = {"3-wire depth-10 circuit": [workloads.small_random()],
            "brickwork 28x40": [workloads.brickwork(28, 40)],
            "QFT-24": [workloads.qft(24, with_input=False)],
            "random J/CZ 6-14 wires": workloads.random_batch(16, 6, 14, 10, 40),
            "random J/CZ 16-30 wires": workloads.random_batch(16, 16, 30, 20, 60, config_index=4, start=2000,
                                                              with_input=False)}
    out = {}
    for name, wls in fams.items():
        rows = []
        for wl in wls:
            h = owqs.load(wl.pattern)
            n = max(1, h.nout)
            r = {}
            for mode in ("owqs", "eowqs"):
                _, info = h.reorder(mode=mode, sweep=(mode == "owqs"),
                                    weights=(float(n), float(n), 0.5, float(n)))
                r[mode] = (info["peak_m"], info["peak_live"])
            rows.append(r)
        out[name] = {"patterns": len(rows),
                     "owqs_m_mean": statistics.mean(r["owqs"][0] for r in rows),
                     "eowqs_m_mean": statistics.mean(r["eowqs"][0] for r in rows),
                     "owqs_m_max": max(r["owqs"][0] for r in rows),
                     "eowqs_m_max": max(r["eowqs"][0] for r in rows),
                     "owqs_one_array_width_mean": statistics.mean(r["owqs"][1] for r in rows),
                     "eowqs_one_array_width_mean": statistics.mean(r["eowqs"][1] for r in rows)}
    return out


def recognition_leg(args, owqs, torch):
    """Batched recognition: the full unitary (all 2^n basis columns) of every
    pattern of the uneven random J/CZ set (widths 6..14, depths 10..40) in
    complex64.  Items whose arrays fit a shared-memory column block run in one
    persistent launch; wider ones are streamed through the pass kernels with
    one reused output buffer.  The plain complex128 path (owqs_unitary per
    pattern) is timed on the widths up to 10 with the c64 batch's error.
    Determinism: 64 random outcome branches per pattern on one random input,
    complex64 and complex128, one batch call each, with every branch's
    fidelity to the pattern's first branch computed on the device."""
    import numpy as np
    from owqs_inputs import workloads
    wls = workloads.random_batch(count=args.rec_count)
    small = []
    for wl in wls:
        if len(wl.pattern.inputs) <= 12:
            h = owqs.load(wl.pattern)
            h.reorder()
            small.append((h, wl))
    wide = [wl for wl in wls if len(wl.pattern.inputs) > 12]
    outs = [torch.empty(1 << (2 * len(wl.pattern.inputs)), dtype=torch.complex64, device="cuda") for _, wl in small]
    items = [{"handle": h, "outcomes": wl.outcomes, "psi_in": None, "out": o, "ref": -1}
             for (h, wl), o in zip(small, outs)]
    owqs.run_batch(items, dtype="c64")  # first call tunes the column block
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    info, _ = owqs.run_batch(items, dtype="c64")
    e1.record()
    torch.cuda.synchronize()
    t_small = e0.elapsed_time(e1) / 1e3
    # wide items one at a time (each handle's workspace is released after use);
    # the first unitary call of a handle captures its graph, the timed second
    # call replays it
    t_wide = 0.0
    upd = sum(h.info()["amp_updates"] << len(wl.pattern.inputs) for h, wl in small)
    if wide:
        nmax = max(len(wl.pattern.inputs) for wl in wide)
        buf = torch.empty(1 << (2 * nmax), dtype=torch.complex64, device="cuda")
        for wl in wide:
            n = len(wl.pattern.inputs)
            h = owqs.load(wl.pattern)
            h.reorder()
            upd += h.info()["amp_updates"] << n
            h.unitary(dtype="c64", outcomes=wl.outcomes, out=buf[: 1 << (2 * n)])
            e0.record()
            h.unitary(dtype="c64", outcomes=wl.outcomes, out=buf[: 1 << (2 * n)])
            e1.record()
            torch.cuda.synchronize()
            t_wide += e0.elapsed_time(e1) / 1e3
            h.close()
        del buf
    cols = sum(1 << len(wl.pattern.inputs) for wl in wls)
    # plain complex128 path on the widths up to 10, and the c64 error there
    sub = [(i, h, wl) for i, (h, wl) in enumerate(small) if len(wl.pattern.inputs) <= 10]
    e0.record()
    refs = [h.unitary(dtype="c128", outcomes=wl.outcomes, use_graph=False)[0] for _, h, wl in sub]
    e1.record()
    torch.cuda.synchronize()
    t128 = e0.elapsed_time(e1) / 1e3
    err = 0.0
    for (i, h, wl), r in zip(sub, refs):
        err = max(err, torch.max(torch.abs(outs[i].to(torch.complex128) - r)).item())
    e0.record()
    sub_items = [items[i] for i, _, _ in sub]
    owqs.run_batch(sub_items, dtype="c64")
    e1.record()
    torch.cuda.synchronize()
    t64_sub = e0.elapsed_time(e1) / 1e3
    # determinism: 64 random outcome branches of every pattern on one random
    # input, in one batch call per precision, each branch's output compared
    # with the pattern's first branch on the device (<ref|out> and norms)
    from owqs_inputs.rng import SplitMix64, random_state
    branches = {}
    handles = [(h, wl) for h, wl in small]
    for wl in wide:
        h = owqs.load(wl.pattern)
        h.reorder()
        handles.append((h, wl))
    for dtype, tdt, npdt in (("c64", torch.complex64, np.complex64), ("c128", torch.complex128, np.complex128)):
        bitems, bufs = [], []
        rng = SplitMix64(1604)
        for h, wl in handles:
            nin, nout = len(wl.pattern.inputs), len(wl.pattern.outputs)
            psi = torch.from_numpy(random_state(rng, nin).astype(npdt)).cuda()
            first = len(bitems)
            for b in range(args.rec_branches):
                o = torch.empty(1 << nout, dtype=tdt, device="cuda")
                bufs.append((psi, o))
                bitems.append({"handle": h, "outcomes": rng.bits(h.K), "psi_in": psi, "out": o,
                               "ref": -1 if b == 0 else first})
        # the first call of a batch shape tunes the column block (kept for the process)
        owqs.run_batch(bitems, dtype=dtype, overlaps=True, use_graph=False)
        torch.cuda.synchronize()
        e0.record()
        w0 = time.perf_counter()
        # every branch item has its own outcomes: graphs would never be replayed
        binfo, ov = owqs.run_batch(bitems, dtype=dtype, overlaps=True, use_graph=False)
        e1.record()
        torch.cuda.synchronize()
        tw = time.perf_counter() - w0
        tb = e0.elapsed_time(e1) / 1e3
        fid = [ov[i, 0] ** 2 + ov[i, 1] ** 2 for i, it in enumerate(bitems) if it["ref"] >= 0]
        fid = [f / (ov[i, 2] * ov[i, 3]) for f, i in zip(fid, [i for i, it in enumerate(bitems) if it["ref"] >= 0])]
        # seconds: CUDA events around the call; the call's own host time and its
        # compile share are in batch_info (call_ms, compile_ms), the binding's
        # marshalling of the item list is the rest of wall_seconds
        branches[dtype] = {"items": len(bitems), "seconds": tb, "wall_seconds": tw, "batch_info": binfo,
                           "min_branch_fidelity": float(min(fid)), "bound": 1 - 4e-5 if dtype == "c64" else 1 - 1e-12}
        del bufs, bitems
    for h, wl in handles[len(small):]:
        h.close()
    return {"patterns": len(wls), "widths": "6..14", "columns": cols, "amp_updates": upd,
            "branches_per_pattern": args.rec_branches, "determinism": branches,
            "seconds": t_small + t_wide, "smem_batch_seconds": t_small, "wide_seconds": t_wide,
            "amp_updates_per_s": upd / (t_small + t_wide), "batch_info": info,
            "c128_plain_subset": {"patterns": len(sub), "seconds_c128_per_pattern_calls": t128,
                                  "seconds_c64_batch": t64_sub, "speedup": t128 / t64_sub if t64_sub else None,
                                  "c64_max_abs_err_vs_c128": err, "bound": 2e-5}}


def qft_leg(args, owqs, torch):
    """QFT-shaped pattern on 24 logical qubits (2784 measurements, peak 25
    live qubits), random normalised input, forced seeded outcomes, complex64
    and complex128 (FP64 groups, and double-float groups).  The pattern has no final swaps, so the exact output is
    the inverse DFT (numpy FFT) of the bit-reversed input times 2^(n/2); per
    output the max-abs error after global-phase alignment and the fidelity
    |<ref|out>|^2 are reported for both precisions."""
    import numpy as np
    from owqs_inputs import workloads
    wl = workloads.qft(24)
    h = owqs.load(wl.pattern)
    _, rinfo = h.reorder()
    n = 24
    upd = int(h.info()["amp_updates"])
    idx = np.arange(1 << n, dtype=np.int64)
    rev = np.zeros_like(idx)
    for b in range(n):
        rev |= ((idx >> b) & 1) << (n - 1 - b)
    ref = np.fft.ifft(wl.psi_in[rev]) * math.sqrt(1 << n)
    res = {"workload": "QFT-shaped J/CZ pattern, 24 logical qubits, random normalised input",
           "measurements": wl.pattern.K, "peak_m": rinfo["peak_m"], "amp_updates_per_run": upd}
    for key, dtype, tdt in (("c64", "c64", torch.complex64), ("c128", "c128", torch.complex128),
                            ("c128_double_float", "c128", torch.complex128)):
        psi = torch.from_numpy(wl.psi_in.astype(np.complex64 if dtype == "c64" else np.complex128)).cuda()
        out = torch.empty(1 << n, dtype=tdt, device="cuda")
        run = lambda: h.run(psi, dtype=dtype, outcomes=wl.outcomes, out=out,
                            double_float=key.endswith("double_float"))
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 3
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        got = out.cpu().numpy().astype(np.complex128)
        ov = np.vdot(got, ref)
        aligned = got * (ov / abs(ov))
        res[key] = {"ms_per_run": 1e3 * t, "amp_updates_per_s": upd / t,
                      "max_abs_err_vs_exact": float(np.max(np.abs(aligned - ref))),
                      "fidelity": float(abs(ov) ** 2 / (np.vdot(got, got).real * np.vdot(ref, ref).real))}
        del out, psi
    res["c64_speedup_over_c128"] = res["c128"]["ms_per_run"] / res["c64"]["ms_per_run"]
    h.close()
    return res


def small_leg(args, owqs, torch):
    """The small case: random 3-wire J/CZ circuit of depth 10 (33 qubits, 30
    measurements, peak 4 live), complex128, forced seeded outcomes.  Latency
    of one run replayed from the CUDA graph (host schedule compile included,
    as in every owqs_run call); its parity with the oracle is a test."""
    import numpy as np
    from owqs_inputs import workloads
    wl = workloads.small_random()
    h = owqs.load(wl.pattern)
    h.reorder()
    psi = torch.from_numpy(wl.psi_in).cuda()
    out = torch.empty(1 << len(wl.pattern.outputs), dtype=torch.complex128, device="cuda")
    run = lambda: h.run(psi, dtype="c128", outcomes=wl.outcomes, out=out)
    for _ in range(5):
        run()
    torch.cuda.synchronize()
    n = 200
    t0 = time.perf_counter()
    for _ in range(n):
        run()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / n
    ms, _, _, _ = h.profile(psi, dtype="c128", outcomes=wl.outcomes)
    res = {"workload": "random 3-wire J/CZ circuit, depth 10 (30 measurements)", "us_per_run": 1e6 * dt,
           "launches_per_run": int(len(ms))}
    h.close()
    return res


def learned_leg(args, owqs, torch, hbm_gbs):
    """The committed learned proposal against the best greedy order on the
    held-out random J/CZ patterns (16..30 qubits, depth 20..60; the first
    --learned-count of the 200 held out from training).  Per pattern, host
    side: the greedy EOWQS order (every qubit ready) and the greedy OWQS
    sweep order (which waits for every domain, so it is valid with
    preselected outcomes too), each with the paper's m and the one-array
    width; then owqs_reorder with the proposal, which keeps it only if it is
    no worse than the better greedy order by (peak live width, amplitude
    updates).  GPU side, wherever the order fits: complex64, EOWQS, all-zero
    branch, one array, CUDA-event time of the kept order and of the best
    greedy order (one warm-up and one timed run each)."""
    import numpy as np
    from owqs_inputs import workloads
    path = os.path.join(ROOT, "paper_1604_05659_gb300", "reorder_mlp.json")
    if not os.path.exists(path):
        return {"unavailable": "no trained weights committed"}
    meta = json.load(open(path))
    model = owqs.Model(weights=np.array(meta["params"], dtype=np.float32))
    free = torch.cuda.mem_get_info()[0]

    def gpu_seconds(h):
        width = h.info()["peak_live"]
        if (1 << min(width, 62)) * 8 * 2.2 > 0.8 * free:
            return None
        out = torch.empty(1 << h.nout, dtype=torch.complex64, device="cuda")
        run = lambda: h.run(None, dtype="c64", mode="eowqs", policy="zero", out=out, check=False, layout="one_array")
        run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        del out
        return e0.elapsed_time(e1) / 1e3

    def m_of_active(h):
        """The paper's m of the active order (its widest sub-state at a
        measurement); None when a sub-state exceeds 62 qubits."""
        try:
            return h.plan_memory(real_input=True)["peak_m"]
        except owqs.OwqsError:
            return None

    rows = []
    for i in range(1_000_000, 1_000_000 + args.learned_count):
        wl = workloads.random_pattern(i, 16, 30, 20, 60, 4, with_input=False)
        h = owqs.load(wl.pattern)
        k = float(max(1, h.nout))
        w = (k, k, 0.5, k)
        oe, ie = h.reorder(mode="eowqs", sweep=False, weights=w)
        me = ie["peak_m"]  # PROA's own MS bookkeeping (the order is too wide to plan)
        oo, io = h.reorder(mode="owqs", sweep=True)
        mo = m_of_active(h)
        t_owqs = gpu_seconds(h)
        t0 = time.perf_counter()
        _, il = h.reorder(mode="eowqs", sweep=False, weights=w, model=model)
        t_reorder = time.perf_counter() - t0
        sat = lambda v: None if v >= (1 << 64) - 1 else v   # the count saturates past 2^64
        row = {"n": h.nin, "K": h.K,
               "eowqs_greedy": {"m": me, "peak_live": ie["peak_live"], "amp_updates": sat(ie["amp_updates"])},
               "owqs_greedy": {"m": mo, "peak_live": io["peak_live"], "amp_updates": io["amp_updates"]},
               "best_greedy": "owqs" if il["greedy_best_owqs"] else "eowqs",
               "learned": {"peak_live": il["learned_peak_live"], "amp_updates": il["learned_amp_updates"]},
               "accepted": il["learned_accepted"],
               "kept": {"m": m_of_active(h), "peak_live": il["peak_live"], "amp_updates": il["amp_updates"]},
               "reorder_seconds": t_reorder}
        best = (il["greedy_peak_live"], il["greedy_amp_updates"])
        row["kept_not_worse"] = (il["peak_live"], il["amp_updates"]) <= best
        if il["learned_accepted"]:
            row["kept_gpu_seconds"] = gpu_seconds(h)
        elif il["greedy_best_owqs"]:
            row["kept_gpu_seconds"] = t_owqs
        row["best_greedy_gpu_seconds"] = t_owqs if il["greedy_best_owqs"] else None
        h.close()
        rows.append(row)
    timed = [r for r in rows if r.get("kept_gpu_seconds") and r.get("best_greedy_gpu_seconds")]
    acc = [r for r in rows if r["accepted"]]
    return {"patterns": len(rows), "accepted": len(acc),
            "kept_never_worse_than_best_greedy": all(r["kept_not_worse"] for r in rows),
            "best_greedy_is_owqs_sweep": sum(r["best_greedy"] == "owqs" for r in rows),
            "mean_m": {"eowqs_greedy": float(np.mean([r["eowqs_greedy"]["m"] for r in rows])),
                       "owqs_greedy": float(np.mean([r["owqs_greedy"]["m"] for r in rows if r["owqs_greedy"]["m"]])),
                       "kept": float(np.mean([r["kept"]["m"] for r in rows if r["kept"]["m"]]))},
            "mean_peak_live": {"eowqs_greedy": float(np.mean([r["eowqs_greedy"]["peak_live"] for r in rows])),
                               "owqs_greedy": float(np.mean([r["owqs_greedy"]["peak_live"] for r in rows])),
                               "learned": float(np.mean([r["learned"]["peak_live"] for r in rows])),
                               "kept": float(np.mean([r["kept"]["peak_live"] for r in rows]))},
            "geomean_update_ratio_best_greedy_over_kept": float(np.exp(np.mean(
                [np.log(max(1, min(r["owqs_greedy"]["amp_updates"], r["eowqs_greedy"]["amp_updates"] or 2**64)) /
                        max(1, r["kept"]["amp_updates"])) for r in rows]))),
            "gpu_timed_patterns": len(timed),
            "geomean_gpu_time_best_greedy_over_kept": float(np.exp(np.mean(
                [np.log(r["best_greedy_gpu_seconds"] / r["kept_gpu_seconds"]) for r in timed]))) if timed else None,
            "gpu_seconds_total": {"kept": float(sum(r["kept_gpu_seconds"] for r in timed)),
                                  "best_greedy": float(sum(r["best_greedy_gpu_seconds"] for r in timed))},
            "trained": {k: v for k, v in meta.items() if k not in ("params", "heldout")},
            "rows_shown": f"first 8 of {len(rows)}", "rows": rows[:8]}


def run_owqs(args):
    import numpy as np
    import torch

    from owqs_inputs import workloads
    from paper_1604_05659_gb300 import owqs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    owqs.library()

    wl = workloads.brickwork(args.rows, args.cols)
    p = wl.pattern
    h = owqs.load(p)
    order, rinfo = h.reorder()
    info = h.info()
    upd = int(info["amp_updates"])
    nout = len(p.outputs)
    stream = torch.cuda.current_stream()
    out64 = torch.empty(1 << nout, dtype=torch.complex64, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, "cuda")

    # the workload as defined: every pass over one array of all live qubits
    # (2^28 amplitudes once the greedy order has prepared 28 rows); the
    # separate-sub-state layout, which a default run of this |+>-input
    # pattern would take, is its own leg below
    run64 = lambda: h.run(None, dtype="c64", outcomes=wl.outcomes, out=out64, layout="one_array")
    for _ in range(args.warmup):
        run64()
    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    sampler = ClockSampler(gpu_id)
    sampler.start()
    t64 = timed(run64, args.steps)
    clocks = sampler.stop()
    value = replica_throughput(upd, args.steps, world, t64)

    # per-launch CUDA-event timing of one run: roofline of the dominant kernel
    hbm, peak_kind = measured_peaks()

    def roofline(dtype):
        ms, by, kd, _ = h.profile(None, dtype=dtype, outcomes=wl.outcomes,
                                  out=out64 if dtype == "c64" else None, layout="one_array")
        kinds = sorted(set(int(k) for k in kd))
        tot = {k: float(ms[kd == k].sum()) for k in kinds}
        dom = max(tot, key=tot.get)
        sel = kd == dom
        secs = float(ms[sel].sum()) / 1e3
        share = tot[dom] / sum(tot.values())
        common = {"kernel": owqs.KERNEL_KIND[dom], "launches": int(sel.sum()), "share_of_step": share,
                  "bytes_per_launch": float(by[sel].mean()), "avg_launch_ms": float(ms[sel].mean())}
        if dtype == "c128":
            # FP64-bound on GB300.  A launch of k measurements on 2^n amplitudes
            # (in and out) produces k 2^n outputs: FP64 flops per output are
            # FP64_FLOPS_PER_OUTPUT for a single pass and FP64_FLOPS_PER_GROUP_OUTPUT
            # inside a pass group (scales and signs carried, not multiplied)
            nm = h.profile_meas[sel].astype(np.float64)
            outputs = by[sel] / 32.0 * nm
            fpo = np.full(len(outputs), float(FP64_FLOPS_PER_OUTPUT))
            if owqs.KERNEL_KIND[dom] == "group_pass":
                halves = [g["half"] for g in h.describe_groups(wl.outcomes, dtype="c128")]
                fpo[:] = FP64_FLOPS_PER_GROUP_OUTPUT
                if len(halves) == len(fpo):
                    fpo[np.array(halves)] = FP64_FLOPS_PER_HALF_GROUP_OUTPUT
            achieved = float((outputs * fpo).sum()) / secs / 1e12
            return dict({"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get((kernel_source_hash(), dtype)),
                         "hbm_gbs": float(by[sel].sum()) / secs / 1e9,
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (no measured FP64 peak)"}, **common), len(ms)
        achieved = float(by[sel].sum()) / secs / 1e9
        traffic = NCU_TRAFFIC.get((kernel_source_hash(), dtype))
        return dict({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs (copy, burst)"}, **common), len(ms)

    legs = set(args.legs.split(","))
    # the end-to-end leg runs right after the device-resident one, before the
    # seconds-long complex128 leg can leave the GPU at its power limit
    e2e = None
    if "e2e" in legs:
        # end to end through the public call with host vectors: the |+>^28
        # input is copied in from pinned memory and the output copied back
        # every step
        nin = len(p.inputs)
        host_in = torch.full((1 << nin,), complex(2.0 ** (-nin / 2.0), 0.0), dtype=torch.complex64).pin_memory()
        host_out = torch.empty(1 << nout, dtype=torch.complex64).pin_memory()
        run_e2e = lambda: h.run_host(host_in, host_out, dtype="c64", outcomes=wl.outcomes)
        run_e2e()
        e2e_steps = args.e2e_steps or args.steps
        # the host link of this machine on the same pinned buffers: one plain copy
        # each way (the end-to-end call moves these bytes before its first
        # launch and after its last), before and after the end-to-end loops,
        # and the copies alone for as many steps as the loops (the host link
        # is shared with other work on the machine and can be slower while
        # the loops run than in a single copy)
        dev_in = torch.empty(1 << nin, dtype=torch.complex64, device="cuda")

        def link_now():
            res = {}
            for name, fn in (("h2d", lambda: dev_in.copy_(host_in, non_blocking=True)),
                             ("d2h", lambda: host_out.copy_(out64, non_blocking=True))):
                fn()
                tl = timed(fn, 3) / 3
                nbytes = (1 << nin) * 8 if name == "h2d" else (1 << nout) * 8
                res[name] = {"GBps": nbytes / tl / 1e9, "ms": 1e3 * tl}
            return res

        def copies_only():
            dev_in.copy_(host_in, non_blocking=True)
            host_out.copy_(out64, non_blocking=True)

        link_before = link_now()
        sampler_e = ClockSampler(gpu_id)
        sampler_e.start()
        te = timed(run_e2e, e2e_steps)
        clocks_e2e = sampler_e.stop()
        tc = timed(copies_only, e2e_steps)
        link = link_now()
        # the same steps through owqs_run_async / owqs_wait with two runs in
        # flight: every step still copies its own input in and its output out
        # (two pinned output buffers in turn), but a step's input copy
        # overlaps the previous step's launches and its output copy the next
        # step's
        host_out2 = torch.empty(1 << nout, dtype=torch.complex64).pin_memory()
        outs = (host_out, host_out2)

        def run_pipe(n):
            h.run_async(host_in, outs[0], dtype="c64", outcomes=wl.outcomes)
            for i in range(1, n):
                h.run_async(host_in, outs[i % 2], dtype="c64", outcomes=wl.outcomes)
                h.wait()
            h.wait()

        run_pipe(2)
        sampler_p = ClockSampler(gpu_id)
        sampler_p.start()
        tp = timed(lambda: run_pipe(e2e_steps), 1)
        clocks_p = sampler_p.stop()
        pipe_ok = bool(torch.equal(host_out2, host_out))  # both hold the same step's result
        del host_out2, outs, dev_in
        e2e = {"value": replica_throughput(upd, e2e_steps, world, tp), "unit": UNIT,
               "h2d_bytes_per_step": (1 << nin) * 8, "d2h_bytes_per_step": (1 << nout) * 8 + 8 * (p.K + 3),
               "ms_per_step": 1e3 * tp / e2e_steps, "steps": e2e_steps, "clocks": clocks_p,
               "api": "owqs_run_async + owqs_wait, two runs in flight, pinned host vectors",
               "outputs_equal": pipe_ok,
               "sync": {"value": replica_throughput(upd, e2e_steps, world, te), "unit": UNIT,
                        "api": "owqs_run with OWQS_IO_HOST, one call per step",
                        "ms_per_step": 1e3 * te / e2e_steps, "clocks": clocks_e2e},
               "host_link": link, "host_link_before": link_before,
               "copies_only_ms_per_step": 1e3 * tc / e2e_steps,
               "device_step_plus_copies_ms": 1e3 * t64 / args.steps + link["h2d"]["ms"] + link["d2h"]["ms"]}

    roof64, launches_per_step = roofline("c64")

    sampled = None
    if "sampled" in legs:
        # sampled outcomes on the same workload, a new seed (a new branch,
        # schedule and graph) every run: OWQS (the guess u > 1/2 checked
        # against the probabilities the run computes) and EOWQS (drawn first)
        sampled = {"runs": args.sampled_steps, "seeds": "1000 + run index"}
        for mode in ("owqs", "eowqs"):
            seeds = iter(range(1000, 2000))
            dev = []

            def run_s():
                _, _, ps, _ = h.run(None, dtype="c64", mode=mode, policy="sampled", seed=next(seeds), out=out64,
                                    layout="one_array")
                dev.append(float(np.max(np.abs(ps - 0.5))) if len(ps) else 0.0)

            run_s()
            ts = timed(run_s, args.sampled_steps)
            sampled[mode] = {"value": replica_throughput(upd, args.sampled_steps, world, ts), "unit": UNIT,
                             "ms_per_run": 1e3 * ts / args.sampled_steps, "max_abs_prob_minus_half": max(dev)}
        sampled["no_gflow"] = readout_leg(args, owqs, torch, timed)

    fp64, accuracy = None, None
    if "c128" in legs:
        # FP64 (complex128) path on the same workload
        out128 = torch.empty(1 << nout, dtype=torch.complex128, device="cuda")
        run128 = lambda: h.run(None, dtype="c128", outcomes=wl.outcomes, out=out128, layout="one_array")
        run128()
        t128 = timed(run128, args.fp64_steps)
        roof128, _ = roofline("c128")
        _, _, p128, _ = run128()
        _, _, p64, _ = run64()
        a = out64.to(torch.complex128)
        ov = torch.vdot(a, out128)
        amp_err = torch.max(torch.abs(a * (ov / abs(ov)) - out128)).item()
        prob_err = float(np.max(np.abs(p64 - p128)))
        del a
        fp64 = {"dtype": "c128", "value": replica_throughput(upd, args.fp64_steps, world, t128),
                "ms_per_step": 1e3 * t128 / args.fp64_steps, "roofline": roof128}
        # the same complex128 arrays with the pass groups in double-float
        # arithmetic on the FP32 pipes (GB300's FP64 rate is 1/64 of FP32)
        outdf = torch.empty(1 << nout, dtype=torch.complex128, device="cuda")
        rundf = lambda: h.run(None, dtype="c128", outcomes=wl.outcomes, out=outdf, layout="one_array",
                              double_float=True)
        rundf()
        tdf = timed(rundf, args.fp64_steps)
        _, _, pdf, _ = rundf()
        fp64["double_float"] = {"value": replica_throughput(upd, args.fp64_steps, world, tdf),
                                "ms_per_step": 1e3 * tdf / args.fp64_steps,
                                "max_abs_amp_diff_vs_fp64": torch.max(torch.abs(outdf - out128)).item(),
                                "max_prob_diff_vs_fp64": float(np.max(np.abs(pdf - p128))),
                                "bound": 1e-12}
        del outdf, out128
        accuracy = {"c64_vs_c128_max_abs_amp_err": amp_err, "c64_vs_c128_max_prob_err": prob_err, "bound": 2e-5}

    subs = None
    if "substates" in legs:
        # the same pattern and branch with separate sub-states (Section 4.1):
        # the |+> inputs are product factors, so a row joins the computation
        # only when the order first touches it and rows stay apart until an E
        # joins them
        plan = h.plan_memory(wl.outcomes, dtype="c64")
        out_s = torch.empty_like(out64)
        run_s = lambda: h.run(None, dtype="c64", outcomes=wl.outcomes, out=out_s, layout="substates")
        run_s()
        ts = timed(run_s, args.steps)
        _, _, p1, _ = run64()
        _, _, p2, _ = run_s()
        ov = torch.vdot(out64.to(torch.complex128), out_s.to(torch.complex128))
        diff = torch.max(torch.abs(out_s.to(torch.complex128) * (ov / abs(ov)) - out64.to(torch.complex128))).item()
        subs = {"ms_per_run": 1e3 * ts / args.steps, "one_array_ms_per_run": 1e3 * t64 / args.steps,
                "peak_m": plan["peak_m"], "components": plan["components"], "joins": plan["joins"],
                "arena_bytes": plan["substate_bytes"], "one_array_bytes": plan["one_array_bytes"],
                "amplitudes_moved": plan["substate_work"], "one_array_amplitudes_moved_estimate": plan["one_array_work"],
                "max_abs_diff_vs_one_array": diff, "max_prob_diff_vs_one_array": float(np.max(np.abs(p1 - p2))),
                "launches_per_run": int(len(h.profile(None, dtype="c64", outcomes=wl.outcomes, out=out_s,
                                                      layout="substates")[0]))}
        del out_s
    m_table = table3_leg(owqs) if "m" in legs else None
    rec = recognition_leg(args, owqs, torch) if "rec" in legs else None
    qft = qft_leg(args, owqs, torch) if "qft" in legs else None
    small = small_leg(args, owqs, torch) if "small" in legs else None
    learned = learned_leg(args, owqs, torch, hbm) if "learned" in legs else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and "cpu" in legs:
        # the C oracle on every host core, on a prefix of this workload; beside
        # it the numpy oracle on one core (a prefix of a 22-row brickwork: its
        # first 29-qubit measurement alone would take minutes on one core)
        from oracle import substate_c
        pre = OraclePrefix(args.rows, args.cols, args.cpu_meas)
        dt = pre.time()
        v1, desc1, dt1 = oracle_sample(22, args.cols, target_s=8.0)
        cpu = {"value": pre.updates / dt, "unit": UNIT, "cores": substate_c.max_threads(), "kind": "oracle",
               "sample": pre.desc, "seconds": dt,
               "one_core": {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc1,
                            "seconds": dt1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t64 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": workload_name(args.rows, args.cols), "rows": args.rows, "cols": args.cols,
                       "measurements": p.K,
                       "peak_m": rinfo["peak_m"], "peak_live": rinfo["peak_live"],
                       "amp_updates_per_step": upd, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "no flush: live arrays of 2 GiB (c64) / 4 GiB (c128) exceed the 129 MB L2",
                       "outcomes": "forced seeded bits, same every step; schedule compiled every call, "
                                   "kernels replayed from a CUDA graph"},
            "roofline": roof64,
            "fp64": fp64,
            "accuracy": accuracy,
            "e2e": e2e,
            "sampled": sampled,
            "recognition": rec,
            "qft24": qft,
            "small": small,
            "learned_reorder": learned,
            "substates": subs,
            "peak_m_owqs_vs_eowqs": m_table,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_owqs(args)


if __name__ == "__main__":
    sys.exit(main())
