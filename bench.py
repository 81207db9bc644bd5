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

# DRAM traffic of one integrator launch from an ncu capture (profiles/), valid only for the
# kernel source it was measured on.
TRAFFIC = {"bytes_per_launch": None, "source_sha1": None}


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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
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
    return {"value": done / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded-uniform cells of the same 2^20-cell field, {el:.1f} s, "
                      f"OpenMP over cells on {cores} threads; rate extrapolates per cell"}


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
            "config": {"workload": WORKLOAD, "sample_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{per_step} seeded-uniform cells of the 2^20-cell field per step"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """Integrator only, on a small case: the quasi-DNS H2 field or the LES CH4 field."""
    import torch
    import paper_2312_13513_gb300 as cg
    from synth.mechanism import ch4_mechanism, h2_mechanism
    from synth.states import les_field, load_table
    if args.case == "h2":
        mech, f, dt = h2_mechanism(), make_field(0, args.cells), DT
    else:
        mech = ch4_mechanism()
        f, dt = les_field(load_table("ch4_flamelet.npz"), n=args.cells, seed=12347), 1e-6
    dm = cg.Mechanism(mech)
    T0 = torch.tensor(f["T"], device="cuda"); p = torch.tensor(f["p"], device="cuda")
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device="cuda")
    ms = []
    for k in range(args.warmup + args.steps):
        T = T0.clone(); Y = Y0.clone()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        cg.advance(dm, T, p, Y, dt, RTOL, ATOL)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(a.elapsed_time(b))
    print(json.dumps({"case": args.case, "cells": args.cells, "ms": ms,
                      "cells_per_s": args.cells / (np.mean(ms) * 1e-3)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=["h2", "ch4"], default=None,
                    help="time only the integrator on a small case (profiling)")
    ap.add_argument("--cells", type=int, default=65536)
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
    field = make_field(rank)
    dev = torch.device("cuda", local)
    T0 = torch.tensor(field["T"], device=dev)
    p = torch.tensor(field["p"], device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(field["Y"]), device=dev)
    T = T0.clone(); Y = Y0.clone()
    n = T.numel()
    nsub = torch.zeros(n, dtype=torch.int32, device=dev)
    nrej = torch.zeros(n, dtype=torch.int32, device=dev)
    status = torch.zeros(n, dtype=torch.int8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        T.copy_(T0); Y.copy_(Y0)
        flush.fill_(1)
        if ev is not None:
            ev[0].record(stream)
        cg.advance(dm, T, p, Y, DT, RTOL, ATOL, status=status, nsub=nsub, nrej=nrej, stream=stream)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
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
    value = world * n * args.steps / (total_ms * 1e-3)
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
        "config": {"workload": WORKLOAD, "cells_per_gpu": n, "dt": DT, "rtol": RTOL, "atol": ATOL,
                   "mechanism": "synthetic H2/air-shaped, 9 species, 25 reactions",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"cells sharded, {world} rank(s), no collective"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": traffic,
                     "peak_source": "FP64 FMA-chain probe measured in this run (chem_fp64_fma_peak)",
                     "kernel_ms": kernel_ms, "flops_per_launch": flops,
                     "transcendentals_per_launch": trans,
                     "transcendental_weight": fl.TRANSCENDENTAL_FLOPS},
        "e2e": {"value": world * n * args.steps / (e2e_ms * 1e-3), "unit": "cell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clk,
        "substeps": {"accepted_mean": acc / n, "attempts_mean": att / n, "non_ok_cells": bad},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(field, mech)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
