"""Benchmark: per-cell chemistry advance on GB300 (one JSON line on stdout).

Workload (N = 1): the FP64 Rodas4 integrator on 2^20 cells of the quasi-DNS-shaped H2/air field
(9 species, 25 reactions; 128^3 grid, first 2^20 cells), one CFD step dt = 5e-7 s, rtol 1e-6,
atol 1e-10.  One step = restore the field from a pristine device copy, flush L2, one
chem_advance over all cells.  Under torchrun each rank advances its own 2^20-cell field (weak
scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

--impl reference times the oracle (plain FP64 CPU implementation) on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DT = 5e-7
RTOL = 1e-6
ATOL = 1e-10
NCELLS = 1 << 20
FIELD_SEED = 12346
METRIC = "chem cell-updates/s, FP64 Rosenbrock vs BF16 MLP at stated error; p50/p99 latency"
WORKLOAD = ("FP64 Rodas4 chemistry advance, 2^20 cells of a 128^3 quasi-DNS H2/air field "
            "(9 species, 25 reactions), dt=5e-7 s, rtol=1e-6, atol=1e-10")

# DRAM traffic of one integrator launch from an ncu capture of the full bench launch
# (profiles/integrator_h2_quasi_dns.md: 2^20 cells of the same field and launch shape, 93.39 MB
# read + 40.90 MB written, one pass), valid only for the kernel source it was measured on (captured
# on sha1 3298e25d; the source has changed since in one comment only).
TRAFFIC = {"bytes_per_launch": 93387520 + 40898560, "source_sha1": "019397584f7777875e6adf89f4f2d58b5794ce18"}

# The paper's chemistry time per step for its H2-air case (Table 1, Section 3.2), in seconds:
# CVODE on one CPU core and DNN inference on one GPU card, on uniform meshes of 32^3, 64^3 and
# 128^3 cells.  Neither the card nor the CPU is named beside the table (the roofline figure of the
# same section shows V100 and T4).  Quoted in the output as context, never used as a target.
PAPER_TABLE1_CHEMISTRY_S = {32: (4.7, 0.007), 64: (34.24, 0.053), 128: (253.86, 0.41)}


def paper_context():
    """Table 1's chemistry columns as rates: cells advanced per second by each side of the
    paper's comparison, and their quotient (the paper's chemistry speedup)."""
    rows = {}
    for side, (cpu_s, gpu_s) in PAPER_TABLE1_CHEMISTRY_S.items():
        n = side ** 3
        rows[f"{side}^3"] = {"cpu_cvode_s": cpu_s, "gpu_dnn_s": gpu_s,
                             "cpu_cvode_cell_updates_per_s_per_core": n / cpu_s,
                             "gpu_dnn_cell_updates_per_s": n / gpu_s, "chemistry_speedup": cpu_s / gpu_s}
    return {"source": "Table 1 (Section 3.2): H2-air, 9 species, per-step chemistry time",
            "hardware": "one GPU card, not named (V100 and T4 in the same section's roofline figure), "
                        "against one CPU core, not named",
            "rows": rows}


def _sha1_of_kernel():
    p = os.path.join(ROOT, "paper_2312_13513_gb300", "csrc", "integrator.cu")
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"chem_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = parse_clock_samples(f)
        os.unlink(self.path)
        return out


def parse_clock_samples(lines):
    """Summary of nvidia-smi samples in ClockSampler.Q's column order (csv, noheader, nounits):
    median SM clock, maximum SM clock, and each throttle reason that was Active in any sample."""
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return out
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    out["samples"] = len(rows)
    out["sm_mhz"] = statistics.median(sm) if sm else None
    try:
        out["sm_max_mhz"] = float(rows[0][2])
    except ValueError:
        pass
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for i, nm in enumerate(names):
        if any(r[5 + i].lower() == "active" for r in rows):
            out["reasons"].append(nm)
    return out


def workload_config(world):
    """The workload both arms report (the reference arm times a bounded sample of it, stated in
    its cpu_baseline)."""
    return {"workload": WORKLOAD, "cells_per_gpu": NCELLS, "dt": DT, "rtol": RTOL, "atol": ATOL,
            "mechanism": "synthetic H2/air-shaped, 9 species, 25 reactions",
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"one field of {world} x 2^20 cells in contiguous ranges per rank, balanced "
                           f"by the warm-up's attempt counts; no collective in the timed steps"}


def shared_field(world):
    """The field a job of world ranks advances: world seeded 2^20-cell quasi-DNS fields end to end
    (one field for a single GPU)."""
    parts = [make_field(r) for r in range(world)]
    if world == 1:
        return parts[0]
    return {"T": np.concatenate([f["T"] for f in parts]), "p": np.concatenate([f["p"] for f in parts]),
            "Y": np.concatenate([f["Y"] for f in parts], axis=1)}


def make_field(rank=0, n=NCELLS):
    from synth.states import load_table, quasi_dns_field
    return quasi_dns_field(load_table("h2_flamelet.npz"), n=n, seed=FIELD_SEED + rank)


def cpu_baseline(field, mech, budget_s=12.0):
    """The oracle as it stands on a seeded sample of the workload's cells, all host cores."""
    import oracle
    om = oracle.OracleMech(mech)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    order = rng.permutation(field["T"].size)
    done = 0
    t0 = time.perf_counter()
    chunk = 2048
    while time.perf_counter() - t0 < budget_s and done < order.size:
        s = np.sort(order[done:done + chunk])
        om.advance(field["T"][s], field["p"][s], field["Y"][:, s], DT, RTOL, ATOL, nthreads=cores)
        done += s.size
    el = time.perf_counter() - t0
    # single-thread rate on a small sample of the same cells
    s1 = np.sort(order[:1024])
    t1 = time.perf_counter()
    om.advance(field["T"][s1], field["p"][s1], field["Y"][:, s1], DT, RTOL, ATOL, nthreads=1)
    el1 = time.perf_counter() - t1
    return {"value": done / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded-uniform cells of the same 2^20-cell field, {el:.1f} s, "
                      f"OpenMP over cells on {cores} threads; rate extrapolates per cell",
            "single_thread_value": s1.size / el1,
            "single_thread_sample": f"{s1.size} cells of the same sample, 1 thread, {el1:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from synth.mechanism import h2_mechanism
    import oracle
    mech = h2_mechanism()
    field = make_field(0)
    om = oracle.OracleMech(mech)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    per_step = 4096
    order = rng.permutation(field["T"].size)
    t_steps = []
    for step in range(args.warmup + args.steps):
        s = np.sort(order[(step * per_step) % order.size:][:per_step])
        t0 = time.perf_counter()
        om.advance(field["T"][s], field["p"][s], field["Y"][:, s], DT, RTOL, ATOL, nthreads=cores)
        if step >= args.warmup:
            t_steps.append(time.perf_counter() - t0)
    tot = sum(t_steps)
    value = per_step * len(t_steps) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(t_steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{per_step} seeded-uniform cells of the 2^20-cell field per step"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """One kernel family on a small case (profiling): the integrator on the quasi-DNS H2 field or
    the LES CH4 field, or the surrogate step on the quasi-DNS H2 field."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.mechanism import ch4_mechanism, h2_mechanism
    from synth.states import les_field, load_table
    if args.case == "h2small":
        print(json.dumps(dict(case=args.case, **extra_h2_small(cg.fp64_fma_peak(), n=args.cells, reps=args.steps,
                                                               group=args.group))),
              flush=True)
        return
    if args.case == "fvm":
        side = max(2, int(round(args.cells ** (1.0 / 3.0))))
        m, kw = _fvm_inputs(side)
        gm = cg.FvMesh(m)
        ms = []
        for k in range(args.warmup + args.steps):
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            gm.assemble(**kw)
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        print(json.dumps({"case": args.case, "cells": m.n_cells, "ms": ms,
                          "gbs": fvm_bytes(m.n_cells, m.owner.size, m.b_cell.size) / (float(np.mean(ms)) * 1e-3) / 1e9}),
              flush=True)
        return
    if args.case == "transport":
        from synth.transport import generate_transport
        mech = ch4_mechanism()
        f = les_field(load_table("ch4_flamelet.npz"), n=args.cells, seed=12347)
        dm = cg.Mechanism(mech)
        gt = cg.Transport(dm, generate_transport(mech))
        T = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        mu = torch.empty_like(T); lam = torch.empty_like(T); D = torch.empty_like(Y)
        ms = []
        for k in range(args.warmup + args.steps):
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            gt(T, p, Y, mu, lam, D)
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        print(json.dumps({"case": args.case, "cells": args.cells, "ms": ms,
                          "cells_per_s": args.cells / (float(np.mean(ms)) * 1e-3)}), flush=True)
        return
    if args.case in ("surrogate", "surrogate_ps"):
        dm = cg.Mechanism(h2_mechanism())
        if args.case == "surrogate":
            model = cg.Surrogate(dm, path=MODEL_PATH)
        else:
            # the per-species networks' shapes with seeded weights (timing only), the single
            # network's normalisation and trust box
            from paper_2312_13513_gb300 import train as trn
            base = trn.load_model_params(MODEL_PATH)
            rng = np.random.default_rng(3)
            dims = [dm.ns + 2, 1600, 800, 400, 1]
            nets = {k: {"W": [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(4)],
                        "b": [np.zeros(dims[i + 1]) for i in range(4)]}
                    for k in range(dm.ns) if base["y_std"][k] > 0}
            prm = {kk: base[kk] for kk in ("x_mean", "x_std", "y_mean", "y_std", "box_lo", "box_hi", "dt")}
            prm.update({"hidden": [1600, 800, 400], "nets": nets})
            model = cg.Surrogate(dm, prm)
        f = make_field(0, args.cells)
        T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        ms = []
        for k in range(args.warmup + args.steps):
            T = T0.clone(); Y = Y0.clone()
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            cg.surrogate_advance(model, T, p, Y, DT, RTOL, ATOL)
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        print(json.dumps({"case": args.case, "cells": args.cells, "ms": ms,
                          "cells_per_s": args.cells / (float(np.mean(ms)) * 1e-3)}), flush=True)
        return
    if args.case == "h2":
        mech, f, dt = h2_mechanism(), make_field(0, args.cells), DT
    else:
        mech = ch4_mechanism()
        f, dt = les_field(load_table("ch4_flamelet.npz"), n=args.cells, seed=12347), 1e-6
    from paper_2312_13513_gb300 import flops as fl
    dm = cg.Mechanism(mech)
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    nsub = torch.zeros(args.cells, dtype=torch.int32, device="cuda"); nrej = torch.zeros_like(nsub)
    opts = cg.options(group_threads=args.group) if args.group else None
    ms = []
    for k in range(args.warmup + args.steps):
        T = T0.clone(); Y = Y0.clone()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        cg.advance(dm, T, p, Y, dt, RTOL, ATOL, nsub=nsub, nrej=nrej, opts=opts)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(a.elapsed_time(b))
    acc = int(nsub.sum()); att = acc + int(nrej.sum())
    _, _, folded = fl.launch_flops(mech, acc, att)
    t = float(np.mean(ms)) * 1e-3
    print(json.dumps({"case": args.case, "cells": args.cells, "group": args.group, "ms": ms,
                      "cells_per_s": args.cells / t, "attempts_per_cell": att / args.cells,
                      "fp64_tflops": folded / t / 1e12,
                      "fp64_frac": folded / t / 1e12 / cg.fp64_fma_peak()}), flush=True)


MODEL_PATH = os.path.join(ROOT, "paper_2312_13513_gb300", "models", "h2_quasi_dns.chemsur")


def _time_ms(fn, stream, reps=1):
    import torch
    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        a.record(stream); fn(); b.record(stream)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return out


def oracle_rate(mech, f, dt, sample, seed=0):
    """The oracle (plain FP64 CPU) on a seeded uniform sample of a field's cells, all host cores:
    its cell-updates/s, which extrapolates per cell to the whole field."""
    import oracle
    om = oracle.OracleMech(mech)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    s = np.sort(rng.choice(f["T"].size, min(sample, f["T"].size), replace=False))
    t0 = time.perf_counter()
    om.advance(f["T"][s], f["p"][s], f["Y"][:, s], dt, RTOL, ATOL, nthreads=cores)
    el = time.perf_counter() - t0
    return {"value": s.size / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{s.size} seeded-uniform cells of the field, {el:.1f} s, extrapolated per cell"}


def extra_ch4(fp64_peak, steps=2, oracle_sample=4096):
    """Config 2: CH4/air-shaped mechanism (53 species, 325 reactions), 262144 LES cells."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import flops as fl
    from synth.mechanism import ch4_mechanism
    from synth.states import les_field, load_table
    mech = ch4_mechanism()
    dm = cg.Mechanism(mech)
    f = les_field(load_table("ch4_flamelet.npz"), n=262144, seed=12347)
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    n = T0.numel()
    ns_ = torch.zeros(n, dtype=torch.int32, device="cuda"); nr_ = torch.zeros_like(ns_)
    T, Y = T0.clone(), Y0.clone()
    stream = torch.cuda.current_stream()

    def run():
        T.copy_(T0); Y.copy_(Y0)
        cg.advance(dm, T, p, Y, 1e-6, RTOL, ATOL, nsub=ns_, nrej=nr_, stream=stream)

    run()
    ms = _time_ms(run, stream, steps)
    acc = int(ns_.sum()); att = acc + int(nr_.sum())
    flo, tr, folded = fl.launch_flops(mech, acc, att)
    t = min(ms) * 1e-3
    out = {"workload": "FP64 Rodas4, 262144 LES-shaped CH4/air cells (53 species, 325 reactions), "
                       "dt=1e-6 s, 128-thread group per cell",
           "ms": min(ms), "cell_updates_per_s": n / t}
    if oracle_sample:
        out["cpu_oracle"] = oracle_rate(mech, f, 1e-6, oracle_sample, seed=2)
    out.update({
            "fp64_frac_plain": flo / t / 1e12 / fp64_peak,
            "fp64_frac_folded": folded / t / 1e12 / fp64_peak,
            "fp64_tflops_plain": flo / t / 1e12, "fp64_tflops_folded": folded / t / 1e12,
            "transcendental_weight": fl.TRANSCENDENTAL_FLOPS, "attempts_mean": att / n})
    return out


def small_h2_states(n=4096, seed=12345):
    """The small H2 case: n H2/air mixing states (Z ~ U[0, 1], T ~ U[900, 2200] K, 1 atm), half of
    them first reacted by this integrator for log-uniform times in [1e-7, 1e-3] s (eight bins of
    the drawn time, each advanced by its bin's geometric centre).  Returns device tensors."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.mechanism import h2_mechanism
    from synth.states import mixing_states
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    st = mixing_states(mech, n, seed)
    T = torch.tensor(st["T"], device="cuda"); p = torch.tensor(st["p"], device="cuda")
    Y = torch.tensor(np.ascontiguousarray(st["Y"]), device="cuda")
    react = np.nonzero(st["react"])[0]
    lt = np.log10(st["t_react"][react])
    edges = np.linspace(-7.0, -3.0, 9)
    bins = np.clip(np.searchsorted(edges, lt, side="right") - 1, 0, 7)
    failed = 0
    for b in range(8):
        sel = react[bins == b]
        if sel.size == 0:
            continue
        idx = torch.tensor(sel.astype(np.int32), device="cuda")
        status = torch.zeros(n, dtype=torch.int8, device="cuda")
        cg.advance(dm, T, p, Y, 10.0 ** (0.5 * (edges[b] + edges[b + 1])), RTOL, ATOL, idx=idx, status=status)
        failed += int((status != 0).sum())
    torch.cuda.synchronize()
    return mech, dm, T, p, Y, failed


def extra_h2_small(fp64_peak, n=4096, reps=10, group=0):
    """Config 0: the small H2 case (4096 cells, dt = 1e-6 s).  Too few cells to fill the GPU (the
    bench launch holds 80 two-thread groups = 80 cells per SM): the time is the sequential
    attempts of the stiffest cells, each attempt's FP64 instructions issued by one warp.  Reported
    with the library's default group (two threads per cell) and, with the default, also with one
    warp per cell (group_threads = 32, a caller's option: fewer instructions per attempt for each
    cell, fewer cells per warp)."""
    import torch
    from paper_2312_13513_gb300 import flops as fl
    import paper_2312_13513_gb300 as cg
    mech, dm, T0, p, Y0, failed = small_h2_states(n)
    T, Y = T0.clone(), Y0.clone()
    ns_ = torch.zeros(n, dtype=torch.int32, device="cuda"); nr_ = torch.zeros_like(ns_)
    stream = torch.cuda.current_stream()

    def timed(g):
        opts = cg.options(group_threads=g) if g else None

        def run():
            T.copy_(T0); Y.copy_(Y0)
            cg.advance(dm, T, p, Y, 1e-6, RTOL, ATOL, nsub=ns_, nrej=nr_, stream=stream, opts=opts)

        for _ in range(3):
            run()
        ms = sorted(_time_ms(run, stream, reps))
        return ms[len(ms) // 2] * 1e-3

    t = timed(group)
    acc = int(ns_.sum()); att = acc + int(nr_.sum())
    _, _, folded = fl.launch_flops(mech, acc, att)
    slots = torch.cuda.get_device_properties(0).multi_processor_count * 80
    out = {"workload": f"FP64 Rodas4, {n} H2/air mixing states (half pre-reacted by this integrator), "
                       "dt=1e-6 s",
           "group_threads": group or 2, "ms": t * 1e3, "cell_updates_per_s": n / t,
           "attempts_mean": att / n, "max_attempts": int((ns_ + nr_).max()),
           "fp64_frac_folded": folded / t / 1e12 / fp64_peak,
           "cell_slot_occupancy": min(n, slots) / slots, "prereact_failed": failed}
    if not group:
        t32 = timed(32)
        out["warp_per_cell"] = {"group_threads": 32, "ms": t32 * 1e3, "cell_updates_per_s": n / t32,
                                "fp64_frac_folded": folded / t32 / 1e12 / fp64_peak}
    return out


def extra_surrogate(peaks, steps=3):
    """Config 3: BF16 MLP surrogate vs the FP64 integrator on 2^22 quasi-DNS H2 cells."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import train as trn
    from synth.mechanism import h2_mechanism
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    trained_here = False
    if not os.path.exists(MODEL_PATH):
        params = trn.train(mech, n_states=1 << 22, epochs=40, log=lambda *a: None, time_budget_s=90)
        os.makedirs(os.path.dirname(MODEL_PATH), exist_ok=True)
        trn.save_model(params, MODEL_PATH)
        trained_here = True
    model = cg.Surrogate(dm, path=MODEL_PATH)
    f = make_field(0, 1 << 22)
    n = f["T"].size
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    stream = torch.cuda.current_stream()
    Tr, Yr = T0.clone(), Y0.clone()

    def fp64():
        Tr.copy_(T0); Yr.copy_(Y0)
        cg.advance(dm, Tr, p, Yr, DT, RTOL, ATOL, stream=stream)

    ms_fp64 = min(_time_ms(fp64, stream, 1))
    cpu = oracle_rate(mech, f, DT, 16384, seed=3)
    Ts, Ys = T0.clone(), Y0.clone()
    route = torch.empty(n, dtype=torch.int8, device="cuda")

    def sur():
        Ts.copy_(T0); Ys.copy_(Y0)
        cg.surrogate_advance(model, Ts, p, Ys, DT, RTOL, ATOL, route=route, stream=stream)

    sur()
    ms_sur = min(_time_ms(sur, stream, steps))
    ms_fwd = min(_time_ms(lambda: cg.surrogate_forward(model, T0, p, Y0, stream=stream), stream, steps))
    qr = cg.heat_release(dm, T0, p, Y0, Yr, DT)
    qs = cg.heat_release(dm, T0, p, Y0, Ys, DT)
    err = float(((qs - qr).abs().sum() / qr.abs().sum()).item())
    err_sum = float(((qs.sum() - qr.sum()).abs() / qr.sum().abs()).item())
    big = qr.abs() > 1e-3 * qr.abs().max()
    rel = ((qs - qr).abs() / qr.abs())[big]
    p99_rel = float(torch.quantile(rel.float()[torch.randperm(rel.numel(), device=rel.device)[:1 << 24]], 0.99).item())
    flop = 2.0 * (11 * 512 + 3 * 512 * 512 + 512 * 9) * n
    tf = flop / (ms_fwd * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    burst = peaks.get("bf16_tflops", 1900.0)
    return {"workload": "BF16 MLP 11-512x4-9 (tcgen05) with projection, Newton T and FP64 fallback, "
                        "2^22 quasi-DNS H2 cells, dt=5e-7 s",
            "model_trained_in_this_run": trained_here, "cpu_oracle_fp64": cpu,
            "fp64_ms": ms_fp64, "fp64_cell_updates_per_s": n / (ms_fp64 * 1e-3),
            "forward_kernel_ms": ms_fwd, "tensor_tflops": tf,
            "tensor_frac_of_burst": tf / burst, "tensor_frac_of_sustained": tf / peak,
            "fallback_fraction": float((route == 1).float().mean().item()),
            "hrr_sum_rel_error_vs_fp64": err_sum, "hrr_p99_cell_rel_error_vs_fp64": p99_rel,
            "surrogate_ms": ms_sur, "surrogate_cell_updates_per_s": n / (ms_sur * 1e-3),
            "speedup_vs_fp64": ms_fp64 / ms_sur, "hrr_l1_rel_error_vs_fp64": err}


def _score_surrogate(cg, dm, model, T0, p, Y0, Yr, stream, steps=3):
    """Step and forward time, heat-release error against the FP64 result Yr, fallback fraction."""
    import torch
    n = T0.numel()
    Ts, Ys = T0.clone(), Y0.clone()
    route = torch.empty(n, dtype=torch.int8, device="cuda")

    def sur():
        Ts.copy_(T0); Ys.copy_(Y0)
        cg.surrogate_advance(model, Ts, p, Ys, DT, RTOL, ATOL, route=route, stream=stream)

    sur()
    ms = min(_time_ms(sur, stream, steps))
    ms_fwd = min(_time_ms(lambda: cg.surrogate_forward(model, T0, p, Y0, stream=stream), stream, steps))
    qr = cg.heat_release(dm, T0, p, Y0, Yr, DT)
    qs = cg.heat_release(dm, T0, p, Y0, Ys, DT)
    err = float(((qs - qr).abs().sum() / qr.abs().sum()).item())
    return {"step_ms": ms, "forward_ms": ms_fwd, "hrr_l1_rel_error_vs_fp64": err,
            "fallback_fraction": float((route == 1).float().mean().item())}


def extra_surrogate_per_species(peaks, n_states=1 << 20, epochs=12):
    """The paper's per-species networks (one 11-1600-800-400-1 GELU network per reactive species)
    against the single 11-512x4-9 network, both trained in this run on the same data with the same
    schedule and epochs, scored on the 2^22-cell quasi-DNS field."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import train as trn
    from synth.mechanism import h2_mechanism
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    data = trn.make_dataset(mech, dm, n_states, DT, 7)
    quiet = lambda *a: None
    t0 = time.time()
    p1 = trn.train(mech, epochs=epochs, log=quiet, data=data)
    t_single = time.time() - t0
    t0 = time.time()
    pps = trn.train_per_species(mech, epochs=epochs, log=quiet, data=data)
    t_ps = time.time() - t0
    f = make_field(0, 1 << 22)
    n = f["T"].size
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    stream = torch.cuda.current_stream()
    Tr, Yr = T0.clone(), Y0.clone()
    cg.advance(dm, Tr, p, Yr, DT, RTOL, ATOL, stream=stream)
    out = {"workload": f"single 11-512x4-9 network vs per-species 11-1600-800-400-1 networks "
                       f"({len(pps['nets'])} reactive species), both trained here on {n_states} states "
                       f"x {epochs} epochs (same data, schedule, batch 4096), scored on 2^22 quasi-DNS "
                       f"H2 cells"}
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    for name, prm, secs in (("single_net", p1, t_single), ("per_species", pps, t_ps)):
        model = cg.Surrogate(dm, prm)
        r = _score_surrogate(cg, dm, model, T0, p, Y0, Yr, stream)
        if name == "single_net":
            flop = 2.0 * (11 * 512 + 3 * 512 * 512 + 512 * 9)
        else:
            h1, h2, h3 = prm["hidden"]
            flop = 2.0 * len(prm["nets"]) * (11 * h1 + h1 * h2 + h2 * h3 + h3)
        tf = flop * n / (r["forward_ms"] * 1e-3) / 1e12
        r.update({"train_s": secs, "mflop_per_cell": flop / 1e6, "forward_tensor_tflops": tf,
                  "forward_tensor_frac_of_sustained": tf / peak,
                  "cell_updates_per_s": n / (r["step_ms"] * 1e-3)})
        out[name] = r
        model.close()
    return out


def extra_train_step(peaks, batch=4096, n_states=1 << 20, steps=256):
    """Training steps of the single 11-512x4-9 network (batch gather, forward, backward, Adam) on
    2^20 states, issued directly and replayed from one captured CUDA graph; both runs start from
    the same weights and visit the same batches, and end with bitwise the same weights."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import parallel
    from paper_2312_13513_gb300 import train as trn
    from synth.mechanism import h2_mechanism
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    data = trn.make_dataset(mech, dm, n_states, DT, 7)
    X, Tt = data["X"], data["T"]
    perm = trn.epoch_order(n_states, 7, 0)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    lrs = [trn.cosine_lr(k, steps, 3e-4, 1e-5) for k in range(steps)]
    out = {"workload": f"11-512x4-9 GELU network, batch {batch}, {steps} Adam steps over {n_states} "
                       f"H2 states (one epoch's first batches)"}
    weights = {}
    for mode in ("direct", "graph"):
        tr = trn.Trainer(mech.ns + 2, mech.ns, batch, seed=7)
        replay = trn._captured_step(tr, X, Tt, batch, loss) if mode == "graph" else None

        def run():
            for k in range(steps):
                idx = perm[k * batch:(k + 1) * batch]
                if replay is not None:
                    replay(idx, lrs[k])
                else:
                    tr.forward(X.index_select(0, idx))
                    tr.backward(Tt.index_select(0, idx), loss)
                    tr.adam(lrs[k])

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms = _time_ms(run, stream, 1)[0]
        wall = time.perf_counter() - t0
        weights[mode] = parallel.flatten_grads(*tr.get(0))
        tr.close()
        out[mode + "_ms_per_step"] = ms / steps
        out[mode + "_host_ms_per_step"] = wall * 1e3 / steps
    p = 11 * 512 + 3 * 512 * 512 + 512 * 9
    # forward 2 flop per weight and sample, backward 4 (input and weight gradients)
    flop = 6.0 * p * batch
    tf = flop / (out["graph_ms_per_step"] * 1e-3) / 1e12
    out.update({"samples_per_s_graph": batch / (out["graph_ms_per_step"] * 1e-3),
                "samples_per_s_direct": batch / (out["direct_ms_per_step"] * 1e-3),
                "graph_speedup": out["direct_ms_per_step"] / out["graph_ms_per_step"],
                "tensor_tflops_graph": tf,
                "tensor_frac_of_sustained": tf / peaks.get("bf16_tflops_sustained", 1700.0),
                "graph_weights_equal_direct": bool(np.array_equal(weights["direct"], weights["graph"]))})
    return out


def _fvm_inputs(n_side, seed=21):
    """A 128^3-style box in face-addressed form (natural numbering, mildly stretched) and seeded
    species-equation inputs of realistic magnitude (cgs), all terms on."""
    import torch
    from synth.mesh import box_mesh
    m = box_mesh(n_side, n_side, n_side, seed=seed, stretch=1.5)
    rng = np.random.default_rng(seed + 1)
    n, nf, nb = m.n_cells, m.owner.size, m.b_cell.size
    dev = lambda a: torch.tensor(a, device="cuda")
    kw = dict(dt=1e-6, rho=dev(rng.uniform(2e-4, 1.2e-3, n)), rho_old=dev(rng.uniform(2e-4, 1.2e-3, n)),
              Y_old=dev(rng.uniform(0.0, 0.3, n)), phi=dev(rng.standard_normal(nf) * 1e-6),
              phi_b=dev(rng.standard_normal(nb) * 1e-6), gamma=dev(rng.uniform(1e-4, 1e-3, n)),
              gamma_b=dev(rng.uniform(1e-4, 1e-3, nb)), Y_b=dev(rng.uniform(0.0, 0.3, nb)),
              S=dev(rng.standard_normal(n)), kappa=dev(rng.uniform(0.0, 1.0, n)))
    return m, kw


def fvm_bytes(n, nf, nb):
    """Algorithmic bytes of one assembly with every term: per cell V, rho, rho_old, Y_old, gamma,
    S, kappa read, diag and source written, its face-index range; per internal face owner,
    neighbour, w, delta, |S|, phi read once, lower and upper written; per boundary face type,
    delta, |S|, phi_b, gamma_b, Y_b; the cell-to-face codes."""
    return n * (7 * 8 + 2 * 8 + 4) + nf * (8 + 4 * 8 + 2 * 8) + nb * (1 + 5 * 8) + (2 * nf + nb) * 4


def extra_fvm(hbm_peak, reps=5):
    """Species-equation assembly (Alg. 1 and the other terms) on a 128^3 box, ldu and CSR, and
    the PaSR factor on the same cells."""
    import torch
    import paper_2312_13513_gb300 as cg
    m, kw = _fvm_inputs(128)
    gm = cg.FvMesh(m)
    s = torch.cuda.current_stream()
    out = gm.assemble(**kw)
    ms = min(_time_ms(lambda: gm.assemble(**kw), s, reps))
    lo, up, dg, _ = out
    ms_csr = min(_time_ms(lambda: gm.to_csr(lo, up, dg), s, reps))
    n, nf, nb = m.n_cells, m.owner.size, m.b_cell.size
    byts = fvm_bytes(n, nf, nb)
    rng = np.random.default_rng(5)
    pin = [torch.tensor(a, device="cuda") for a in (10.0 ** rng.uniform(-7, -2, n), rng.uniform(2e-4, 1.2e-3, n),
                                                     rng.uniform(1e-4, 6e-4, n), 10.0 ** rng.uniform(1, 5, n),
                                                     np.full(n, 1.0 / 128))]
    kap = torch.empty(n, dtype=torch.float64, device="cuda")
    ms_pasr = min(_time_ms(lambda: cg.pasr_kappa(*pin, kappa=kap), s, reps))
    return {"workload": f"species equation (implicit Euler, upwind convection, Alg. 1 Laplacian, fixed-value and "
                        f"zero-gradient patches, PaSR-scaled source) on a 128^3 box: {n} cells, {nf} internal "
                        f"faces, {nb} boundary faces",
            "assemble_ms": ms, "assemble_gbs": byts / (ms * 1e-3) / 1e9,
            "assemble_frac_of_hbm": byts / (ms * 1e-3) / 1e9 / hbm_peak, "algorithmic_bytes": byts,
            "to_csr_ms": ms_csr, "csr_nnz": gm.nnz, "pasr_ms": ms_pasr,
            "pasr_gbs": 6 * 8 * n / (ms_pasr * 1e-3) / 1e9}


def extra_transport(fp64_peak, reps=3):
    """Transport and T-from-h kernels on the LES CH4 field (262144 cells) and the quasi-DNS H2
    field (2^20 cells)."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import flops as fl
    from synth.mechanism import ch4_mechanism, h2_mechanism
    from synth.states import les_field, load_table
    from synth.transport import generate_transport
    out = {}
    for name, mech, f in (("ch4_les", ch4_mechanism(), les_field(load_table("ch4_flamelet.npz"), n=262144, seed=12347)),
                          ("h2_quasi_dns", h2_mechanism(), make_field(0, 1 << 20))):
        dm = cg.Mechanism(mech)
        gt = cg.Transport(dm, generate_transport(mech))
        T = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        n = T.numel()
        mu = torch.empty_like(T); lam = torch.empty_like(T); D = torch.empty_like(Y)
        h = torch.empty_like(T); cp = torch.empty_like(T)
        st = torch.empty(n, dtype=torch.int8, device="cuda")
        s = torch.cuda.current_stream()
        gt(T, p, Y, mu, lam, D)
        ms_tr = min(_time_ms(lambda: gt(T, p, Y, mu, lam, D), s, reps))
        cg.mixture_thermo(dm, T, Y, h, cp)
        Tg = T + 100.0
        ms_T = min(_time_ms(lambda: (Tg.copy_(T + 100.0), cg.temperature_from_enthalpy(dm, h, Y, Tg, st)), s, reps))
        flo, tr = fl.transport_counts(mech.ns)
        folded = n * (flo + fl.TRANSCENDENTAL_FLOPS * tr)
        out[name] = {"cells": n, "transport_ms": ms_tr, "transport_cells_per_s": n / (ms_tr * 1e-3),
                     "transport_fp64_frac": folded / (ms_tr * 1e-3) / 1e12 / fp64_peak,
                     "t_from_h_ms": ms_T, "t_from_h_cells_per_s": n / (ms_T * 1e-3),
                     "t_from_h_converged": int((st == 0).sum())}
    out["workload"] = ("mixture-averaged viscosity (Wilke), conductivity (Mathur-Saxena), diffusion "
                       "coefficients from cubic ln T fits; T from h by Newton from T0 + 100 K")
    return out


def extra_graph(sizes=(4096, 65536), reps=50):
    """The chemistry + thermo step (surrogate route) on small fields, issued back to back: directly
    (about a dozen API calls and launches per step) and as replays of the captured CUDA graph.  At
    these sizes the host's issue rate, not the GPU, sets the direct rate: per-step time of each."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.mechanism import h2_mechanism
    from synth.transport import generate_transport
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    if not os.path.exists(MODEL_PATH):
        return {"skipped": "no trained model"}
    model = cg.Surrogate(dm, path=MODEL_PATH)
    tr = cg.Transport(dm, generate_transport(mech))
    stream = torch.cuda.current_stream()
    out = {"workload": f"chemistry + thermo step (surrogate route) from the field's state, {reps} steps back to "
                       f"back, per step"}
    for n in sizes:
        f = make_field(0, n)
        T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        T, Y = T0.clone(), Y0.clone()
        f64 = lambda *sh: torch.empty(*sh, dtype=torch.float64, device="cuda")
        st = cg.Step(dm, T, p, Y, DT, RTOL, ATOL, model=model, transport=tr, h0=f64(n), cp0=f64(n), q=f64(n),
                     thermo_status=torch.empty(n, dtype=torch.int8, device="cuda"), mu=f64(n), lam=f64(n),
                     D=f64(mech.ns, n))
        st.run(graph=False, stream=stream)
        st.run(graph=True, stream=stream)            # capture
        torch.cuda.synchronize()
        res = {}
        for name, use_graph in (("direct_ms", False), ("graph_ms", True)):
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                T.copy_(T0); Y.copy_(Y0)        # every step from the field's state (two copies in both)
                st.run(graph=use_graph, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            res[name] = a.elapsed_time(b) / reps
        st.close()
        out[f"{n}_cells"] = res
    return out


def extra_step(n=1 << 20, reps=3):
    """One "chemistry + thermo" step (start-state thermo, chemistry, heat release and T from h,
    transport properties) on the 2^20-cell quasi-DNS H2 field, per stage like the paper's Table 1
    (chemistry vs the rest of a step), issued directly and as a replayed CUDA graph, for the FP64
    integrator and for the surrogate."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.mechanism import h2_mechanism
    from synth.transport import generate_transport
    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    tr = cg.Transport(dm, generate_transport(mech))
    f = make_field(0, n)
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    f64 = lambda *sh: torch.empty(*sh, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"workload": f"{n} quasi-DNS H2 cells, dt=5e-7 s: start-state h and cp, chemistry, heat release "
                       "and T from h by Newton, mixture-averaged transport; median of direct runs and of "
                       "graph replays"}
    routes = [("fp64", None)]
    if os.path.exists(MODEL_PATH):
        routes.append(("surrogate", cg.Surrogate(dm, path=MODEL_PATH)))
    for name, model in routes:
        T, Y = T0.clone(), Y0.clone()
        st = cg.Step(dm, T, p, Y, DT, RTOL, ATOL, model=model, transport=tr, h0=f64(n), cp0=f64(n), q=f64(n),
                     thermo_status=torch.empty(n, dtype=torch.int8, device="cuda"), mu=f64(n), lam=f64(n),
                     D=f64(mech.ns, n))

        def timed(use_graph):
            ms = []
            for _ in range(reps):
                T.copy_(T0); Y.copy_(Y0)
                a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream); st.run(graph=use_graph, stream=stream); b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            return float(np.median(ms))

        T.copy_(T0); Y.copy_(Y0); st.run(graph=False, stream=stream)       # warm-up
        T.copy_(T0); Y.copy_(Y0); st.run(graph=True, stream=stream)        # capture + first replay
        torch.cuda.synchronize()
        direct = timed(False)
        stages = st.stage_ms()
        graph = timed(True)
        st.close()
        out[name] = {"thermo_in_ms": stages[0], "chemistry_ms": stages[1], "thermo_out_ms": stages[2],
                     "transport_ms": stages[3], "direct_total_ms": direct, "graph_total_ms": graph,
                     "chemistry_share": stages[1] / max(1e-9, sum(stages))}
    return out


def _serving_setup(seed):
    """The config-4 solvers: 64 states of 1e4-2e6 cells (log-uniform), 70 % H2 / 30 % CH4, routes
    50/50 (H2 only: there is no CH4 surrogate), resident on the device."""
    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import serve
    from synth.mechanism import ch4_mechanism, h2_mechanism
    from synth.states import les_field, load_table
    rng = np.random.default_rng(seed)
    h2, ch4 = h2_mechanism(), ch4_mechanism()
    dm_h2, dm_ch4 = cg.Mechanism(h2), cg.Mechanism(ch4)
    model = cg.Surrogate(dm_h2, path=MODEL_PATH) if os.path.exists(MODEL_PATH) else None
    fh = make_field(7, 1 << 21)
    fc = les_field(load_table("ch4_flamelet.npz"), n=1 << 21, seed=seed)
    solvers = []
    for i in range(64):
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(2e6))))
        is_h2 = rng.uniform() < 0.7
        sur = rng.uniform() < 0.5
        f = fh if is_h2 else fc
        off = int(rng.integers(0, f["T"].size - n + 1))
        route = serve.ROUTE_SURROGATE if (is_h2 and sur and model is not None) else serve.ROUTE_FP64
        label = ("h2" if is_h2 else "ch4") + ("_surrogate" if route == serve.ROUTE_SURROGATE else "_fp64")
        solvers.append({"route": route, "dt": DT if is_h2 else 1e-6, "cells": n, "mech": "h2" if is_h2 else "ch4",
                        "label": label, "off": off,
                        "T0": torch.tensor(f["T"][off:off + n], device="cuda"),
                        "p": torch.tensor(f["p"][off:off + n], device="cuda"),
                        "Y0": torch.tensor(np.ascontiguousarray(f["Y"][:, off:off + n]), device="cuda")})
        solvers[-1]["T"] = solvers[-1]["T0"].clone()
        solvers[-1]["Y"] = solvers[-1]["Y0"].clone()
    return dm_h2, dm_ch4, model, solvers


def _service_s_per_cell(dm_h2, dm_ch4, model):
    """Idle-GPU time per cell of each request class (FP64 H2, FP64 CH4, surrogate H2)."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.states import les_field, load_table
    stream = torch.cuda.current_stream()
    out = {}
    fh = make_field(8, 1 << 18)
    fc = les_field(load_table("ch4_flamelet.npz"), n=1 << 15, seed=5)
    for label, dm, f, dt in (("h2_fp64", dm_h2, fh, DT), ("ch4_fp64", dm_ch4, fc, 1e-6)):
        T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        T, Y = T0.clone(), Y0.clone()

        def run():
            T.copy_(T0); Y.copy_(Y0)
            cg.advance(dm, T, p, Y, dt, RTOL, ATOL, stream=stream)
        run()
        out[label] = min(_time_ms(run, stream, 2)) * 1e-3 / T0.numel()
    if model is not None:
        f = make_field(8, 1 << 20)
        T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
        Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
        T, Y = T0.clone(), Y0.clone()

        def run_s():
            T.copy_(T0); Y.copy_(Y0)
            cg.surrogate_advance(model, T, p, Y, DT, RTOL, ATOL, stream=stream)
        run_s()
        out["h2_surrogate"] = min(_time_ms(run_s, stream, 2)) * 1e-3 / T0.numel()
    return out


def _serving_run(dm_h2, dm_ch4, model, solvers, think, duration_s, seed, slice_ms=0.0):
    from paper_2312_13513_gb300 import serve
    import torch
    srv = serve.Server(150 << 30, n_streams=4, slice_ms=slice_ms)
    run_solvers = []

    def flow_step(s_):
        # the solver's own step between two chemistry sub-steps: here it brings the state back to
        # the field's (a chemistry-only loop would drift towards equilibrium, out of the surrogate's
        # training distribution, which a real flow step keeps it in)
        def run():
            s_["T"].copy_(s_["T0"]); s_["Y"].copy_(s_["Y0"])
            torch.cuda.current_stream().synchronize()
        return run

    for s_ in solvers:
        s_["T"].copy_(s_["T0"]); s_["Y"].copy_(s_["Y0"])
        sid = srv.register(dm_h2 if s_["mech"] == "h2" else dm_ch4, s_["T"], s_["p"], s_["Y"],
                           model=model if s_["mech"] == "h2" else None)
        d = {"state_id": sid, "route": s_["route"], "dt": s_["dt"], "cells": s_["cells"], "label": s_["label"],
             "flow": flow_step(s_)}
        if think is not None:
            d["think_s"] = think(s_)
        run_solvers.append(d)
    res = serve.run_closed_loop(srv, run_solvers, duration_s=duration_s, mean_gap_s=2e-3, seed=seed)
    st = srv.stats()
    srv.close()
    lat = np.array(res["latencies"]) * 1e3
    labels = np.array(res["labels"])
    by_class = {}
    for c in sorted(set(labels.tolist())):
        lc = lat[labels == c]
        by_class[c] = [int(lc.size), round(float(np.percentile(lc, 50)), 1), round(float(np.percentile(lc, 99)), 1)]
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "cell_updates_per_s": res["cells"] / res["wall_s"], "wall_s": res["wall_s"],
            "by_class_requests_p50_p99_ms": by_class, "fp64_time_slices": st["slices"],
            "launches": st["launches"], "requests_per_launch": st["requests_launched"] / max(1, st["launches"]),
            "fp64_joined_running_job": st["joined"], "max_concurrent_launches": st["max_concurrent"],
            "failed": st["failed"]}


def extra_serving(duration_s=10.0, seed=12349, duty=1.0 / 128.0, slice_ms=0.0):
    """Config 4 at two loads: (a) sustainable -- each solver spends 1/duty - 1 times its idle-GPU
    chemistry time on its own flow solve between requests, so the 64 solvers together offer about
    64 duty = 50 % of the GPU; (b) overload -- Exp(2 ms) gaps between a solver's result and its next
    request (the workload as stated: far more work than the GPU can serve)."""
    dm_h2, dm_ch4, model, solvers = _serving_setup(seed)
    per_cell = _service_s_per_cell(dm_h2, dm_ch4, model)
    offered = sum(s_["cells"] * per_cell[s_["label"]] for s_ in solvers)
    think = lambda s_: s_["cells"] * per_cell[s_["label"]] * (1.0 / duty - 1.0)
    sustainable = _serving_run(dm_h2, dm_ch4, model, solvers, think, duration_s, seed, slice_ms)
    sustainable["load"] = (f"each solver thinks {1.0 / duty - 1.0:.0f}x its idle-GPU service time "
                           f"(offered ~{64 * duty:.0%} of the GPU)")
    overload = _serving_run(dm_h2, dm_ch4, model, solvers, None, duration_s, seed, slice_ms)
    overload["load"] = "Exp(2 ms) think time (offered work far above capacity)"
    return {"workload": "64 closed-loop solvers, 1e4-2e6 cells log-uniform, 70/30 H2/CH4, routes 50/50 "
                        "(H2 only), 150 GB budget, 10 s of submissions per load, FP64 jobs in 20 ms time "
                        "slices that requests join, surrogate requests gathered into one pass per model; "
                        "each solver's flow step restores its state to the field's before it submits",
            "idle_service_us_per_kcell": {k: round(v * 1e9, 3) for k, v in per_cell.items()},
            "all_solvers_once_idle_s": offered,
            "cells_h2": int(sum(s_["cells"] for s_ in solvers if s_["mech"] == "h2")),
            "cells_ch4": int(sum(s_["cells"] for s_ in solvers if s_["mech"] == "ch4")),
            "overload": overload, "sustainable": sustainable,
            "p50_ms": overload["p50_ms"], "p99_ms": overload["p99_ms"],
            "cell_updates_per_s": overload["cell_updates_per_s"],
            "sustainable_surrogate_p99_ms": sustainable["by_class_requests_p50_p99_ms"].get("h2_surrogate", [0, None, None])[2]}


def summary(line):
    """The headline figures of every config in a few hundred bytes (the last key of the line)."""
    ex = line.get("extras", {})
    c0, c2, c3, c4 = ex.get("h2_small", {}), ex.get("ch4_les", {}), ex.get("surrogate", {}), ex.get("serving", {})
    r = lambda v, d=4: None if v is None else round(float(v), d)
    return {"cfg0_h2_small_ms": r(c0.get("ms"), 3), "cfg0_fp64_frac_folded": r(c0.get("fp64_frac_folded")),
            "cfg1_h2_cells_per_s": r(line["value"], 0), "cfg1_fp64_frac_folded": r(line["roofline"]["frac"]),
            "cfg2_ch4_cells_per_s": r(c2.get("cell_updates_per_s"), 0),
            "cfg2_fp64_frac_plain": r(c2.get("fp64_frac_plain")), "cfg2_fp64_frac_folded": r(c2.get("fp64_frac_folded")),
            "cfg3_surrogate_cells_per_s": r(c3.get("surrogate_cell_updates_per_s"), 0),
            "cfg3_speedup_vs_fp64": r(c3.get("speedup_vs_fp64"), 2),
            "cfg3_hrr_l1_rel_error": r(c3.get("hrr_l1_rel_error_vs_fp64"), 5),
            "cfg3_forward_frac_burst": r(c3.get("tensor_frac_of_burst")),
            "cfg4_p50_ms": r(c4.get("p50_ms"), 1), "cfg4_p99_ms": r(c4.get("p99_ms"), 1),
            "cfg4_cells_per_s": r(c4.get("cell_updates_per_s"), 0),
            "cfg4_sustainable_surrogate_p99_ms": r(c4.get("sustainable_surrogate_p99_ms"), 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=["h2", "h2small", "ch4", "surrogate", "surrogate_ps", "transport", "fvm"],
                    default=None,
                    help="time one kernel family on a small case (profiling)")
    ap.add_argument("--cells", type=int, default=65536)
    ap.add_argument("--group", type=int, default=0, help="threads per cell (profiling mode; 0 = auto)")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2312_13513_gb300 as cg
    from paper_2312_13513_gb300 import flops as fl
    from synth.mechanism import h2_mechanism

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    mech = h2_mechanism()
    dm = cg.Mechanism(mech)
    dev = torch.device("cuda", local)
    # one shared field of world x 2^20 cells; each rank advances a contiguous range of it, first
    # equal, then balanced by the attempt counts measured in the warm-up (weak scaling: 2^20 cells
    # per GPU on average, no collective inside the timed steps)
    from paper_2312_13513_gb300 import parallel
    field_all = shared_field(world)
    n_total = field_all["T"].size
    S = {}

    def take(a, b):
        S["range"] = (a, b)
        S["T0"] = torch.tensor(field_all["T"][a:b], device=dev)
        S["p"] = torch.tensor(field_all["p"][a:b], device=dev)
        S["Y0"] = torch.tensor(np.ascontiguousarray(field_all["Y"][:, a:b]), device=dev)
        S["T"], S["Y"] = S["T0"].clone(), S["Y0"].clone()
        m = b - a
        S["nsub"] = torch.zeros(m, dtype=torch.int32, device=dev)
        S["nrej"] = torch.zeros(m, dtype=torch.int32, device=dev)
        S["status"] = torch.zeros(m, dtype=torch.int8, device=dev)

    take(*parallel.shard(n_total, rank, world))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        T, Y, T0, Y0, p = S["T"], S["Y"], S["T0"], S["Y0"], S["p"]
        T.copy_(T0); Y.copy_(Y0)
        flush.fill_(1)
        if ev is not None:
            ev[0].record(stream)
        cg.advance(dm, T, p, Y, DT, RTOL, ATOL, status=S["status"], nsub=S["nsub"], nrej=S["nrej"], stream=stream)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        # the next steps' ranges from this step's per-cell attempts (parallel.rebalance), then one
        # more untimed step on the new range
        w = (S["nsub"] + S["nrej"] + 1).to(torch.float64)
        take(*parallel.rebalance(w, S["range"][0], n_total))
        step()
        torch.cuda.synchronize()
    T, Y, T0, Y0, p = S["T"], S["Y"], S["T0"], S["Y0"], S["p"]
    nsub, nrej, status = S["nsub"], S["nrej"], S["status"]
    n = T.numel()
    a0, b0 = S["range"]
    field = {"T": field_all["T"][a0:b0], "p": field_all["p"][a0:b0], "Y": field_all["Y"][:, a0:b0]}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        step(kev[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n_total * args.steps / (total_ms * 1e-3)
    bad = int((status != 0).sum().item())
    acc = int(nsub.sum().item())
    att = acc + int(nrej.sum().item())
    flops, trans, folded = fl.launch_flops(mech, acc, att)

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    Th = torch.tensor(field["T"]).pin_memory()
    ph = torch.tensor(field["p"]).pin_memory()
    Yh = torch.tensor(np.ascontiguousarray(field["Y"])).pin_memory()
    To = torch.empty_like(Th).pin_memory()
    Yo = torch.empty_like(Yh).pin_memory()
    Td = torch.empty_like(T0); pd = torch.empty_like(p); Yd = torch.empty_like(Y0)

    def e2e_step():
        Td.copy_(Th, non_blocking=True); pd.copy_(ph, non_blocking=True); Yd.copy_(Yh, non_blocking=True)
        cg.advance(dm, Td, pd, Yd, DT, RTOL, ATOL, stream=stream)
        To.copy_(Td, non_blocking=True); Yo.copy_(Yd, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = (Th.numel() + ph.numel() + Yh.numel()) * 8
    d2h = (To.numel() + Yo.numel()) * 8

    fp64_peak = cg.fp64_fma_peak()
    achieved = folded / (kernel_ms * 1e-3) / 1e12
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["source_sha1"] == _sha1_of_kernel() else None
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(world),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": traffic,
                     "peak_source": "FP64 FMA-chain probe measured in this run (chem_fp64_fma_peak)",
                     "kernel_ms": kernel_ms, "flops_per_launch": flops,
                     "transcendentals_per_launch": trans,
                     "transcendental_weight": fl.TRANSCENDENTAL_FLOPS},
        "e2e": {"value": n_total * args.steps / (e2e_ms * 1e-3), "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clk,
        "substeps": {"accepted_mean": acc / n, "attempts_mean": att / n, "non_ok_cells": bad},
        "paper_context": paper_context(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(field, mech)
    if rank == 0 and world == 1 and not args.no_extras:
        # configs 2 and 3 are printed last: the end of the line is what a truncated log keeps
        extras = {}
        for name, fn in (("surrogate_per_species", lambda: extra_surrogate_per_species(_peaks())),
                         ("train_step", lambda: extra_train_step(_peaks())),
                         ("fvm_species_assembly", lambda: extra_fvm(_peaks().get("hbm_gbs", 6800.0))),
                         ("graph_small_step", extra_graph),
                         ("chemistry_thermo_step", extra_step),
                         ("thermo_transport", lambda: extra_transport(fp64_peak)),
                         ("serving", extra_serving),
                         ("h2_small", lambda: extra_h2_small(fp64_peak)),
                         ("ch4_les", lambda: extra_ch4(fp64_peak)),
                         ("surrogate", lambda: extra_surrogate(_peaks()))):
            try:
                extras[name] = fn()
            except Exception as e:      # an extra measurement never hides the headline line
                extras[name] = {"error": f"{type(e).__name__}: {e}"}
        line["extras"] = extras
        line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
