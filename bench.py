#!/usr/bin/env python
"""Benchmark of one exact-exchange + ACE step on GB300.

Default workload (one step), the slab of the paper's scale: 72 x 72 x 144 grid, periodic
x and y, Dirichlet z with the top 30% of z vacuum, h = 0.2 bohr, 12th-order FD,
erfc-screened kernel omega = 0.106, 1024 orthonormal synthetic orbitals of which 800 are
fractionally occupied (Fermi-Dirac, kT = 0.01 Ha):
    VxPsi = exx_apply(Psi_occ = 800, Psi_in = all 1024)   (499,600 unique pair solves)
    E_x   = exx_energy(...)
    xi    = ace_build(Psi, VxPsi)
Metric: pair-Poisson solves per second (unique orbital pairs of the workload solved per
second of step time; each solve is one batched Kronecker solve, Sec. II.B) and the
exx_apply time.  Every arm (GPU, FP64 leg, CPU oracle, reference) reports this unit.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--prec auto|fp64|bf16x3|tf32x3|bf16x6|bf16x10|bf16x7]
                       [--workload slab|periodic48|batch48|sweep|precision]
Other workloads (not the default line):
  periodic48 48^3 periodic grid, 128 orbitals (every output compared with the full oracle).
  batch48   48 independent systems (grids of 20-64 points per axis, 8-160 orbitals) solved
            by one exx_apply_batched call (one CUDA graph) per step, beside the same work
            issued as one exx_apply call per system.
  sweep     exx_apply of the 48^3 workload for pair batches n_c = 1 (one pair per solve
            sequence, the unbatched Kronecker solver) up to 1024.
  precision 48^3 grid with 256 orbitals: every precision mode against the FP64 path
            (VxPsi, xi, E_x errors and times).
For N > 1 launch with torchrun; every rank runs an independent replica (the pair
solves shard with no exchange), so the whole-job value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-Poisson solves/s & exx_apply time: FP64 vs split-precision at stated error"
UNIT = "pair-Poisson solves/s"
WORKLOAD = ("periodic48_erfc_128: 48x48x48 periodic grid, h=0.25, 12th-order FD, erfc kernel "
            "omega=0.106, 128 orbitals, Fermi-Dirac occupations; step = exx_apply + exx_energy + ace_build")
SLAB_WORKLOAD = ("slab72x72x144_erfc_1024: 72x72x144 grid, periodic x,y, Dirichlet z (top 30% of z vacuum), "
                 "h=0.2, 12th-order FD, erfc kernel omega=0.106, 1024 orbitals, 800 fractionally occupied "
                 "(Fermi-Dirac kT=0.01); step = exx_apply + exx_energy + ace_build")
L2_FLUSH_BYTES = 512 << 20
BATCH_WORKLOAD = ("batch48: 48 independent systems, seeded grid draws of 20-64 points per axis, "
                  "mixed Dirichlet/periodic axes, h=0.3, 12th-order FD, Coulomb kernel with any Dirichlet "
                  "axis else erfc omega=0.106, 8-160 orbitals with Fermi-Dirac occupations; "
                  "step = exx_apply of every system in one exx_apply_batched call")
FP64_PEAK_NOTE = "FP64 CUDA-core peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-vs-split comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="library default settings instead of the autotuner's")
    ap.add_argument("--set-tuning", default="",
                    help="six comma-separated settings for exx_plan_set_tuning instead of the autotuner "
                         "(pairs per batch, block orbitals, z block, z buffers, staging, pipeline)")
    ap.add_argument("--n-orb", type=int, default=128)
    ap.add_argument("--slab-orbitals", type=int, default=1024,
                    help="orbitals of the slab workload (occupied: 800/1024 of them); smaller values "
                         "make small cases of the same grid for profiling")
    ap.add_argument("--batch", type=int, default=0, help="pairs per batch (0 = library default)")
    ap.add_argument("--workload", default="slab", choices=["slab", "periodic48", "batch48", "sweep", "precision", "capacity"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler for the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait (at most 5 s) until the sampler writes, so the timed region starts with it live;
        # the samples already written were taken before the region and are skipped
        self.skip = 0
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            self.fh.flush()
            with open(self.path) as fh:
                n = sum(1 for _ in fh)
            if n:
                self.skip = n
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm_mhz, max_mhz = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            rows.append((sm_mhz, max_mhz, {nm for nm, v in zip(names, parts[5:9]) if v.lower().startswith("active")}))
        os.unlink(self.path)
        skip = getattr(self, "skip", 0)
        inside = rows[skip:]
        note = None
        if not inside:
            if not rows:
                return None
            # the region was shorter than the sampling interval: the last sample before it
            inside, note = rows[-1:], "timed region shorter than the 200 ms sampling interval; last sample before it"
        rec = {"sm_mhz": statistics.median(r[0] for r in inside), "sm_max_mhz": max(r[1] for r in inside),
               "samples": len(rows[skip:]), "reasons": sorted(set().union(*(r[2] for r in inside)))}
        if note:
            rec["note"] = note
        return rec


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def code_text(src):
    """Source text without // comments and blank lines: edits to comments alone leave the
    compiled kernel, and so its recorded counters, valid."""
    lines = []
    for line in src.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return "\n".join(lines)


def src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(code_text(open(os.path.join(ROOT, p), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except Exception:
        return None
    if rec.get("src_hash") != src_hash(rec["sources"]):
        return None
    return rec


def prec_code(exx, name):
    return {"fp64": exx.EXX_PREC_FP64, "bf16x3": exx.EXX_PREC_BF16X3, "tf32x3": exx.EXX_PREC_TF32X3,
            "bf16x6": exx.EXX_PREC_BF16X6, "bf16x10": exx.EXX_PREC_BF16X10, "bf16x7": exx.EXX_PREC_BF16X7}[name]


def pick_precision(exx, s, dev):
    """'auto': the fastest split-precision form that meets both error targets (VxPsi <= 1e-6,
    E_x <= 1e-8 relative) and supports the grid, else FP64."""
    for name in ("bf16x7", "bf16x10"):
        try:
            p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
            p.set_precision(prec_code(exx, name))
            p.close()
            return name
        except Exception:
            continue
    return "fp64"


def workload(args):
    """(system, description, flush L2 between steps) of the workload named by --workload."""
    import synth
    if args.workload == "periodic48":
        return synth.config2(args.n_orb), WORKLOAD, True
    if args.slab_orbitals != 1024:
        n = args.slab_orbitals
        s = synth.config5(n_orb=n, n_occ=max(1, (n * 800) // 1024))
        return s, SLAB_WORKLOAD.replace("1024 orbitals, 800", f"{n} orbitals, {s.n_occ}"), False
    return synth.config5(), SLAB_WORKLOAD, False


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2501_16572_gb300 as exx

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    t_gen = time.perf_counter()
    s, wl_text, flush_l2 = workload(args)
    t_gen = time.perf_counter() - t_gen
    occ = s.n_occ
    unique = s.unique_pairs()
    ordered = s.ordered_pairs()
    psi = torch.from_numpy(s.psi).to(dev)
    f = torch.from_numpy(s.f).to(dev)
    prec_name = args.prec if args.prec != "auto" else pick_precision(exx, s, dev)

    def make_plan(name):
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec_code(exx, name))
        if args.batch:
            p.set_batch(args.batch, 0)
        return p

    plan = make_plan(prec_name)
    W = torch.empty_like(psi)
    xi = torch.empty_like(psi)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev) if flush_l2 else None
    stream = torch.cuda.current_stream()
    # the library's autotuner picks the batch, block and kernel settings on this grid (untimed)
    tuning = None
    if args.set_tuning:
        v = [int(x) for x in args.set_tuning.split(",")]
        plan.set_tuning(*v)
        tuning = plan.tuning()
    elif not args.batch and not args.no_tune:
        t0 = time.perf_counter()
        tuning = plan.autotune(psi[:occ], f, psi, out=W)
        tuning["seconds"] = time.perf_counter() - t0

    def step(p, t_apply=None):
        launches = 0
        if t_apply is not None:
            t_apply[0].record(stream)
        p.apply(psi[:occ], f, psi, out=W)
        launches += p.launch_count()
        if t_apply is not None:
            t_apply[1].record(stream)
        e = p.energy(psi[:occ], f, W)
        launches += p.launch_count()
        p.ace_build(psi, W, xi=xi)
        launches += p.launch_count()
        return e, launches

    def timed(p, steps, warmup, with_kernel_timing):
        for _ in range(warmup):
            step(p)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms, apply_ms, launches = [], [], 0
        if with_kernel_timing:
            p.set_timing(True)
        clocks = Clocks(local)
        clocks.start()
        for _ in range(steps):
            if flush is not None:
                flush.fill_(1.0)             # evict L2 between timed steps (untimed)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            e, nl = step(p, (ev[2], ev[3]))
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
            apply_ms.append(ev[2].elapsed_time(ev[3]))
            launches += nl
        clk = clocks.stop()
        kt = p.timing() if with_kernel_timing else {}
        if with_kernel_timing:
            p.set_timing(False)
        tot = torch.tensor([sum(ms), sum(apply_ms)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        return tot[0].item(), tot[1].item(), e, launches, kt, clk

    total_ms, apply_total_ms, e_main, launches, ktimes, clk = timed(plan, args.steps, args.warmup, True)
    K = args.steps
    value = world * unique * K / (total_ms / 1e3)
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec_name, "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
        "config": {"workload": wl_text, "grid": list(s.n), "n_orb": s.n_orb, "n_occ": occ,
                   "unique_pair_solves_per_step": unique, "ordered_pairs_per_step": ordered,
                   "precision": prec_name,
                   "l2": ("flushed between timed steps (512 MB write, untimed)" if flush_l2 else
                          f"inputs larger than L2 (Psi {s.psi.nbytes / 1e9:.1f} GB)"),
                   "parallelism": f"replicas x{world}"},
        "exx_apply_ms": apply_total_ms / K,
        "gpu_launches": launches,
        "E_x": e_main,
        "input_generation_s": t_gen,
        "autotune": tuning,
    }
    # -- rooflines: the dominant kernel class and the whole apply (CUDA events, timed region) --
    peaks = measured_peaks()
    if ktimes:
        dom = max(ktimes, key=lambda k: ktimes[k][0])
        dom_ms, dom_n = ktimes[dom]
        rec["kernel_times_ms"] = {k: round(v[0] / K, 4) for k, v in ktimes.items()}
        rec["roofline"] = roofline(s, prec_name, dom, dom_ms, dom_n, K, peaks)
        rec["roofline_apply"] = roofline_apply(s, prec_name, apply_total_ms / K, peaks)
        rec["tensor_roofline"] = tensor_roofline(s, prec_name, apply_total_ms / K, peaks)
    rec["ordered_pair_solves_per_s"] = value * ordered / unique
    rec["clocks"] = clk
    W_split = W.clone()
    # -- FP64 path on sampled output columns (the slab) or on all of them (48^3) --
    if not args.no_compare and prec_name != "fp64":
        cols = (list(range(0, s.n_orb, s.n_orb // 16))[:16] if s.n_orb > 256 else list(range(s.n_orb)))
        p64 = make_plan("fp64")
        sub = psi[cols].contiguous()
        ref64 = torch.empty_like(sub)
        p64.apply(psi[:occ], f, sub, out=ref64)      # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.apply(psi[:occ], f, sub, out=ref64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        solves64 = occ * len(cols)
        # the same unit: unique pairs of the workload per second, from the FP64 solve rate
        rate64 = solves64 / (ms64 / 1e3) * unique / ordered
        rec["fp64"] = {"output_columns": len(cols), "pair_solves": solves64, "exx_apply_ms": ms64,
                       "value": world * rate64, "unit": UNIT,
                       "sample": f"{len(cols)} output column(s) x {occ} occupied partners on the FP64 path; value "
                                 "= its solve rate x unique/ordered pairs of the workload"}
        fl64 = 4.0 * s.N * sum(s.n) * solves64 / (ms64 / 1e3) / 1e12
        pk64 = 152 * 2 * 2 * 2.07e9 / 1e12
        rec["fp64"]["roofline"] = {"bound": "alu", "achieved": fl64, "peak": pk64, "unit": "TFLOP/s",
                                   "frac": fl64 / pk64, "peak_source": FP64_PEAK_NOTE + " (derived, not measured)",
                                   "rule": "4 N (n1 + n2 + n3) flops per pair solve over the FP64 apply time"}
        rec["split_vs_fp64_speedup"] = value / (world * rate64)
        rec["vxpsi_rel_fro_vs_fp64_sampled"] = float(torch.linalg.norm(W_split[cols] - ref64) / torch.linalg.norm(ref64))
        p64.close()
    # -- CPU oracle: baseline throughput and the error of this run against it --
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, oracle_cols = cpu_baseline(s, budget_s=15.0)
        rec["cpu_baseline"] = cb
        rec["error_vs_oracle"] = error_vs_oracle(s, W_split, xi, e_main, oracle_cols, args.workload)
    # -- end to end through the host-buffer entry point --
    if not args.no_e2e:
        rec["e2e"] = e2e(plan, s, 2 if s.N * s.n_orb > 2e8 else K, world)
    plan.close()
    if rank == 0:
        print(json.dumps(rec), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batch48(args):
    """Many small systems: one graph-captured exx_apply_batched call per step against
    one exx_apply call per system, same stream, same buffers."""
    import torch
    import torch.distributed as dist

    import synth
    import paper_2501_16572_gb300 as exx

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    specs = synth.config4_specs()
    mine = [i for i in range(len(specs)) if i % world == rank]   # systems shard over ranks
    systems = [synth.config4_system(i, specs) for i in mine]
    prec_name = args.prec if args.prec != "auto" else "bf16x7"
    plans, bufs = [], []
    for s in systems:
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec_code(exx, prec_name))
        plans.append(p)
        psi = torch.from_numpy(s.psi).to(dev)
        bufs.append((psi, torch.from_numpy(s.f).to(dev), torch.empty_like(psi)))
    bargs = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    unique = sum(s.unique_pairs() for s in systems)
    # every system's settings from the library's autotuner, on its own grid and data (untimed)
    tuning = None
    if not args.no_tune:
        import collections
        t0 = time.perf_counter()
        picks = collections.Counter()
        for p, (po, f, pi, out) in zip(plans, bargs):
            t = p.autotune(po, f, pi, out=out)
            picks[f"pairs {t['pairs_per_batch']}, block {t['block_orbitals']}, z {t['z_block']}/{t['z_buffers']}, "
                  f"staging {t['staging']}, pipeline {t['pipeline']}"] += 1
        tuning = {"systems_tuned": len(plans), "seconds": time.perf_counter() - t0,
                  "choices": dict(picks.most_common())}
    side = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def graph_step():
        exx.exx_apply_batched(plans, bargs, stream=side)

    def loop_step():
        for p, (po, f, pi, out) in zip(plans, bargs):
            p.apply(po, f, pi, out=out, stream=side)

    def launches():
        return sum(p.launch_count() for p in plans)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms, nl = [], 0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(side)
            fn()
            e1.record(side)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            nl += launches()
        tot = torch.tensor([sum(ms)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        return tot.item(), nl

    K = args.steps
    clocks = Clocks(local)
    clocks.start()
    t_graph, nl_graph = timed(graph_step, K, args.warmup)
    clk = clocks.stop()
    t_loop, _ = timed(loop_step, K, args.warmup)
    ref = [out.clone() for (_, _, out) in bufs]
    graph_step()
    torch.cuda.synchronize()
    identical = all(torch.equal(r, out) for r, (_, _, out) in zip(ref, bufs))
    # whole job: every rank's systems over the slowest rank's time
    u = torch.tensor([float(unique)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(u)
    value = u.item() * K / (t_graph / 1e3)
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_graph / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": prec_name, "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
        "config": {"workload": BATCH_WORKLOAD, "systems": len(specs), "systems_this_rank": len(systems),
                   "unique_pair_solves_per_step": int(u.item()), "precision": prec_name,
                   "l2": "flushed between timed steps (512 MB write, untimed)",
                   "parallelism": f"systems sharded over {world} rank(s)"},
        "gpu_launches": nl_graph,
        "per_system_loop": {"ms_per_step": t_loop / K, "value": u.item() * K / (t_loop / 1e3)},
        "graph_vs_loop_speedup": t_loop / t_graph,
        "graph_equals_loop_bitwise": identical,
        "autotune": tuning,
        "clocks": clk,
    }
    # per-kernel times: one more step with CUDA events around every launch (timing issues
    # the launches one by one instead of through the graph)
    for p in plans:
        p.set_timing(True)
    graph_step()
    torch.cuda.synchronize()
    per_kind, bytes_kind = {}, {}
    for p, s in zip(plans, systems):
        for kind, (ms, n) in p.timing().items():
            a = per_kind.setdefault(kind, [0.0, 0])
            a[0] += ms
            a[1] += n
            if kind.startswith("pass") and prec_name != "fp64":
                b = pass_bytes(kind) * s.N * s.unique_pairs() + (8 * s.N * n if kind == "pass3" else 0)
                bytes_kind[kind] = bytes_kind.get(kind, 0.0) + b
        p.set_timing(False)
    rec["kernel_times_ms"] = {k: round(v[0], 4) for k, v in per_kind.items()}
    dom = max(per_kind, key=lambda k: per_kind[k][0])
    peaks = measured_peaks()
    if dom in bytes_kind:
        ms, n = per_kind[dom]
        achieved = bytes_kind[dom] / (ms / 1e3) / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        rec["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
                           "traffic": None, "kernel": kernel_name(prec_name, dom), "launches": n,
                           "avg_launch_ms": ms / n, "algorithmic_bytes_per_launch": bytes_kind[dom] / n,
                           "timing": "one extra step with CUDA events around each launch (launches issued "
                                     "one by one, not through the graph)",
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                           else "fallback 6800 GB/s"}
    # end to end: pinned host orbitals in, host VxPsi out, every step
    if not args.no_e2e:
        host_in = [(torch.from_numpy(s.psi.copy()).pin_memory(), torch.from_numpy(s.f.copy()).pin_memory())
                   for s in systems]
        host_out = [torch.empty_like(h[0]).pin_memory() for h in host_in]

        def e2e_step():
            with torch.cuda.stream(side):
                for (ph, fh), (psi, f, _) in zip(host_in, bufs):
                    psi.copy_(ph, non_blocking=True)
                    f.copy_(fh, non_blocking=True)
                graph_step()
                for ho, (_, _, out) in zip(host_out, bufs):
                    ho.copy_(out, non_blocking=True)
            side.synchronize()

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        dt = (time.perf_counter() - t0) / K
        rec["e2e"] = {"value": u.item() / dt, "unit": UNIT,
                      "ms_per_step": dt * 1e3,
                      "h2d_bytes_per_step": int(sum(h[0].numel() * 8 + h[1].numel() * 8 for h in host_in)),
                      "d2h_bytes_per_step": int(sum(h.numel() * 8 for h in host_out)),
                      "entry": "exx_apply_batched with host copies of every system's Psi, f and VxPsi"}
    if rank == 0 and world == 1 and not args.no_cpu:
        rec["cpu_baseline"] = cpu_baseline(systems[1])[0]
        rec["cpu_baseline"]["sample"] += f" of system 1 ({'x'.join(map(str, systems[1].n))}, {systems[1].n_orb} orbitals)"
    for p in plans:
        p.close()
    if rank == 0:
        print(json.dumps(rec), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _apply_ms(exx, plan, psi_occ, f, psi_in, out, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        plan.apply(psi_occ, f, psi_in, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.apply(psi_occ, f, psi_in, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_sweep(args):
    """Batching study (Sec. II.B, Figs. 1-2): per-solve time of the original formalism (Eq. 8,
    one pair per solve, 4 n_z + 2 GEMM launches) against the batched solver over the pair
    batch size n_c, on the 48^3 periodic grid and on the 72x72x144 slab grid."""
    import torch
    import synth
    import paper_2501_16572_gb300 as exx
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    grids = [("periodic48", synth.config2(16)),
             ("slab72x72x144", synth.make_system("slab_sweep", (72, 72, 144), 0.2, (1, 1, 0), 16, synth.KERNEL_ERFC,
                                                 synth.HSE_OMEGA, "fd", synth.SEED_BASE + 5, slab_axis=2,
                                                 fermi_index=12))]
    out_rows = []
    for gname, s in grids:
        psi = torch.from_numpy(s.psi).cuda()
        f = torch.from_numpy(s.f).cuda()
        out = torch.empty_like(psi)
        unique = s.unique_pairs()
        rows = []
        # original formalism on the first 4 orbitals (10 pair solves)
        sub = 4
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        o4 = torch.empty_like(psi[:sub])
        p.apply_original(psi[:sub], f, psi[:sub], out=o4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.apply_original(psi[:sub], f, psi[:sub], out=o4)
        e1.record(stream)
        torch.cuda.synchronize()
        n_sub = sub * (sub + 1) // 2
        rows.append({"solver": "original (Eq. 8), FP64", "n_c": 1, "pair_solves": n_sub,
                     "launches": p.launch_count(), "ms_per_solve": e0.elapsed_time(e1) / n_sub})
        p.close()
        for prec_name, ncs in (("fp64", (1, 16, 0)), ("bf16x7", (1, 16, 64, 0))):
            for nc in ncs:
                p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
                p.set_precision(prec_code(exx, prec_name))
                p.set_batch(nc, 1 if nc == 1 else (4 if nc == 16 else 0))
                ms = _apply_ms(exx, p, psi, f, psi, out, 1, 1, stream)
                rows.append({"solver": f"batched, {prec_name}", "n_c": nc if nc else "default",
                             "pair_solves": unique, "launches": p.launch_count(), "ms_per_solve": ms / unique})
                p.close()
        base = rows[0]["ms_per_solve"]
        for r in rows:
            r["speedup_vs_original"] = base / r["ms_per_solve"]
        out_rows.append({"grid": gname, "n": list(s.n), "orbitals": s.n_orb, "rows": rows})
    best = min(out_rows[0]["rows"], key=lambda r: r["ms_per_solve"])
    rec = {"metric": METRIC, "value": 1e3 / best["ms_per_solve"], "unit": UNIT, "n_gpus": 1, "steps": 1,
           "warmup": 1, "ms_per_step": best["ms_per_solve"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "mixed", "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": "batching study: original formalism vs batched solver over n_c, 16 orbitals, "
                                  "48^3 periodic and 72x72x144 slab grids", "l2": "not flushed (back-to-back applies)"},
           "sweep": out_rows}
    print(json.dumps(rec), flush=True)


def run_precision(args):
    """Every precision mode on the 48^3 grid with 256 orbitals, against the FP64 path."""
    import torch
    import synth
    import paper_2501_16572_gb300 as exx
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    s = synth.config3()
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    stream = torch.cuda.current_stream()
    res = {}
    for name in ("fp64", "bf16x7", "bf16x10", "bf16x6", "tf32x3", "bf16x3"):
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec_code(exx, name))
        W = torch.empty_like(psi)
        ms = _apply_ms(exx, p, psi[:s.n_occ], f, psi, W, max(1, args.steps), 1, stream)
        e = p.energy(psi[:s.n_occ], f, W)
        xi = p.ace_build(psi, W)
        res[name] = (ms, W, xi, e)
        p.close()
    ms64, W64, xi64, e64 = res["fp64"]
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    table = []
    for name, (ms, W, xi, e) in res.items():
        table.append({"precision": name, "exx_apply_ms": ms, "pair_solves_per_s": s.unique_pairs() / (ms / 1e3),
                      "vxpsi_rel_fro_vs_fp64": rel(W, W64), "xi_rel_fro_vs_fp64": rel(xi, xi64),
                      "E_x_rel_vs_fp64": abs(e - e64) / abs(e64), "E_x": e})
    b7 = [r for r in table if r["precision"] == "bf16x7"][0]   # the default mode
    rec = {"metric": METRIC, "value": b7["pair_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": 1, "ms_per_step": b7["exx_apply_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16x7", "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": "precision study: 48x48x48 periodic grid, erfc omega=0.106, 256 orbitals, "
                                  "Fermi-Dirac occupations; exx_apply timed per precision",
                      "unique_pair_solves": s.unique_pairs(), "l2": "not flushed (back-to-back applies)"},
           "precisions": table}
    print(json.dumps(rec), flush=True)


# Algorithmic bytes per grid element and pair field of each kernel class, as the method's
# pipeline stages them: FP32, 4 B in and 4 B out per element per pass.  The five-pass modes
# have five such passes (BF16X10 also stores hi+lo pairs: that is executed traffic, not
# algorithmic); the three-pass mode has three; the accumulation reads each field once.
# Pass 3 of every mode also reads f(Lambda) (8 B per grid point) once per launch.
def pass_bytes(kind):
    return {"pass1": 8, "pass2": 8, "pass3": 8, "pass4": 8, "pass5": 8, "accum": 4}.get(kind)


# kernel behind each timing class, per mode family
def kernel_name(prec, kind):
    if prec == "fp64":
        return "fp64_pass_kernel" if kind.startswith("pass") else kind
    if prec == "bf16x7":
        return {"pass1": "slice_pass_kernel (pass A)", "pass3": "zpass_kernel (pass B)",
                "pass5": "slice_pass_kernel (pass C)", "accum": "tc_accum_kernel"}.get(kind, kind)
    return {"accum": "tc_accum_kernel"}.get(kind, f"tc_pass_kernel ({kind})")


def roofline(s, prec, kind, ms, nlaunch, K, peaks):
    """Achieved throughput of the dominant kernel class from its live CUDA-event time:
    algorithmic bytes per launch (pass_bytes x N x pair fields per launch, + f(Lambda)) over
    the average launch time, against the measured HBM copy bandwidth."""
    N = s.N
    unique = s.unique_pairs()
    fields_per_launch = unique * K / max(1, nlaunch)
    avg_s = ms / max(1, nlaunch) / 1e3
    name = kernel_name(prec, kind)
    out = {"kernel": name, "launches": nlaunch, "avg_launch_ms": ms / max(1, nlaunch),
           "fields_per_launch": fields_per_launch}
    if prec == "fp64" and kind.startswith("pass"):
        n = s.n
        axis_K = {"pass1": n[2], "pass2": n[0], "pass3": n[1], "pass4": n[0], "pass5": n[2]}[kind]
        flops = 2.0 * N * axis_K * fields_per_launch
        achieved = flops / avg_s / 1e12
        peak = 152 * 2 * 2 * 2.07e9 / 1e12
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": FP64_PEAK_NOTE + " (derived from unit counts and clock, not measured)",
                    "algorithmic_flops_per_launch": flops, "traffic": None})
        return out
    pb = pass_bytes(kind)
    if pb is None:
        out.update({"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None})
        return out
    byt = pb * N * fields_per_launch + (8 * N if kind == "pass3" else 0)
    achieved = byt / avg_s / 1e9
    pk = peaks.get("hbm_gbs", 6800.0)
    out.update({"bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s",
                "algorithmic_bytes_per_launch": byt,
                "algorithmic_bytes_rule": "FP32: 4 B in + 4 B out per grid element per pair field per pass "
                                          "(accumulation: 4 B read), + f(Lambda) 8 B per point for the pass "
                                          "holding the scaling"})
    tr = traffic_for(name.split(" ")[0] + ":" + kind + ":" + prec)
    if tr:
        out["traffic"] = tr["bytes_per_field"] * fields_per_launch
        out["traffic_source"] = tr["source"]
    else:
        out["traffic"] = None
    return out


def roofline_apply(s, prec, apply_ms, peaks):
    """The whole exx_apply against HBM: the method's staged bytes (16 N per unique pair: the
    three-pass pipeline's FP32 intermediates) plus the compulsory bytes (read Psi, write the
    output, FP64) over the apply time."""
    staged = 16.0 * s.N * s.unique_pairs()
    compulsory = 8.0 * s.N * (s.n_orb + s.n_orb)
    achieved = (staged + compulsory) / (apply_ms / 1e3) / 1e9
    pk = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
            "bytes_per_apply": staged + compulsory,
            "rule": "16 N B per unique pair (staged FP32 pipeline) + 8 N B per orbital read and per output written"}


# digit products executed per mode product, and the tensor dtype's share of the bf16 peak
TENSOR_PRODUCTS = {"bf16x7": (7, 1.0), "bf16x10": (10, 1.0), "bf16x6": (7, 1.0), "tf32x3": (3, 0.5),
                   "bf16x3": (3, 1.0)}


def tensor_roofline(s, prec, apply_ms, peaks):
    """The apply's mode products against the tensor-core roof: algorithmic flops 4 N (n1+n2+n3)
    per unique pair (the six mode products), executed flops = algorithmic x the digit products
    of one mode product, over the exx_apply time, against the measured sustained bf16 rate
    (TF32X3: half of it, the nominal dense ratio)."""
    algo = 4.0 * s.N * sum(s.n) * s.unique_pairs()
    out = {"algorithmic_tflops": algo / (apply_ms / 1e3) / 1e12,
           "algorithmic_flops_per_apply": algo, "rule": "4 N (n1 + n2 + n3) flops per unique pair"}
    if prec in TENSOR_PRODUCTS:
        nprod, ratio = TENSOR_PRODUCTS[prec]
        pk = peaks.get("bf16_tflops_sustained", 1700.0) * ratio
        ex = algo * nprod / (apply_ms / 1e3) / 1e12
        out.update({"bound": "tensor", "digit_products": nprod, "executed_tflops": ex, "peak": pk, "unit": "TFLOP/s",
                    "frac": ex / pk, "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"
                    + (" x 0.5 (tf32 nominal ratio)" if ratio != 1.0 else "")})
    return out


def e2e(plan, s, steps, world):
    import torch
    psi_h = torch.from_numpy(s.psi.copy()).pin_memory()
    f_h = torch.from_numpy(s.f.copy()).pin_memory()
    xi_h = torch.empty_like(psi_h).pin_memory()
    plan.ace_step_host(psi_h, s.n_occ, f_h, xi_h)       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        plan.ace_step_host(psi_h, s.n_occ, f_h, xi_h)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"value": world * s.unique_pairs() / dt, "unit": UNIT, "ms_per_step": dt * 1e3, "steps": steps,
            "h2d_bytes_per_step": int(psi_h.numel() * 8 + f_h.numel() * 8),
            "d2h_bytes_per_step": int(xi_h.numel() * 8 + 8),
            "entry": "exx_ace_step_host (pinned host Psi, f in; xi, E_x out)"}


def cpu_sample(s, budget_s=15.0, partners=None):
    """Time the CPU oracle on whole output columns of the workload (each column = its
    occupied partners' pair solves, all of them or the first `partners`) until about
    budget_s seconds of work have run.  Returns (solves/s, columns, solves, seconds, threads,
    {column: values})."""
    import oracle
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    no = s.n_occ if partners is None else min(partners, s.n_occ)
    cols, got = 0, {}
    # columns spread over the orbitals: occupied and (for the slab) empty outputs alike
    order = [(i * 389) % s.n_orb for i in range(s.n_orb)]
    t0 = time.perf_counter()
    while True:
        c = order[cols % s.n_orb]
        got[c] = orc.exx_apply(s.psi[:no], s.f[:no], s.psi, cols=[c])[0]
        cols += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or cols >= s.n_orb:
            break
    solves = cols * no
    return solves / dt, cols, solves, dt, oracle.num_threads(), got


def cpu_baseline(s, budget_s=15.0):
    """The oracle's throughput in the metric's unit: its full apply would take n_orb columns
    x (sample time / sampled columns); unique pairs of the workload / that time."""
    rate, cols, solves, dt, cores, got = cpu_sample(s, budget_s)
    full_s = dt / cols * s.n_orb
    rec = {"value": s.unique_pairs() / full_s, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{cols} whole output column(s) of the workload ({solves} ordered pair solves, {dt:.1f} s, "
                     f"plain C FP64 oracle); value = unique pairs of the workload / ({s.n_orb} columns x "
                     f"{dt / cols:.2f} s per column)",
           "ordered_solves_per_s": rate, "full_apply_s_extrapolated": full_s}
    return rec, got


def golden_energy(s):
    """Stored oracle E_x of the slab workload when the stored input fingerprint matches the
    inputs regenerated here (tests/golden/make_slab_energy.py), else None."""
    path = os.path.join(ROOT, "tests", "golden", "slab72x72x144_energy.json")
    try:
        g = json.load(open(path))
    except Exception:
        return None
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_slab_energy as mk
    if not mk.stored_matches(g, s, s.psi):
        return None
    return g["E_x"]


def error_vs_oracle(s, W, xi, e_gpu, oracle_cols, workload_name):
    """Errors of this run against the oracle: VxPsi on the columns the CPU baseline computed
    (every column for the 48^3 workload), E_x against the full oracle energy, xi against the
    oracle's ACE where the full oracle W is affordable."""
    import numpy as np
    import oracle
    cols = sorted(oracle_cols)
    Wn = W[cols].cpu().numpy()
    ref = np.stack([oracle_cols[c] for c in cols])
    out = {"vxpsi_rel_fro": float(np.linalg.norm(Wn - ref) / np.linalg.norm(ref)), "vxpsi_columns": len(cols)}
    if workload_name == "periodic48":
        orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        full = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi)
        e_ref = orc.energy(s.psi[:s.n_occ], s.f, full)
        _, _, xi_ref = oracle.ace(s.psi, full, s.dV)
        Wa = W.cpu().numpy()
        out.update({"vxpsi_rel_fro": float(np.linalg.norm(Wa - full) / np.linalg.norm(full)),
                    "vxpsi_columns": s.n_orb, "E_x_rel": abs(e_gpu - e_ref) / abs(e_ref),
                    "xi_rel_fro": float(np.linalg.norm(xi.cpu().numpy() - xi_ref) / np.linalg.norm(xi_ref))})
    else:
        e_ref = golden_energy(s)
        out["E_x_rel"] = None if e_ref is None else abs(e_gpu - e_ref) / abs(e_ref)
        out["E_x_source"] = ("stored full oracle run (tests/golden/slab72x72x144_energy.json), fingerprint "
                             "matched" if e_ref is not None else "no stored oracle energy for these inputs")
        out["xi_rel_fro"] = None
        out["xi_note"] = "the oracle's xi needs its full W (all 1024 columns); compared at 48^3 (--workload periodic48)"
    return out


def run_reference(args):
    """The reference arm of this build is the CPU oracle: each step computes one output column
    of the workload against a bounded number of its occupied partners."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s, wl_text, _ = workload(args)
    partners = 64 if s.N * s.n_occ > 1e8 else None
    for _ in range(min(args.warmup, 1)):
        cpu_sample(s, budget_s=0.0, partners=partners)
    tot_solves, tot_t, cores = 0, 0.0, 1
    for _ in range(args.steps):
        rate, cols, solves, dt, cores, _ = cpu_sample(s, budget_s=0.0, partners=partners)
        tot_solves += solves
        tot_t += dt
    # unique pairs of the workload per second: the ordered solve rate x unique / ordered
    value = tot_solves / tot_t * s.unique_pairs() / s.ordered_pairs()
    sample = (f"each step: one output column of the workload against "
              f"{partners if partners else s.n_occ} occupied partners ({tot_solves // args.steps} ordered pair "
              f"solves); value = ordered solve rate x unique/ordered pairs of the workload")
    rec = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": wl_text, "grid": list(s.n), "n_orb": s.n_orb, "n_occ": s.n_occ,
                      "unique_pair_solves_per_step": s.unique_pairs(), "ordered_pairs_per_step": s.ordered_pairs(),
                      "precision": "f64", "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec), flush=True)


def run_capacity(args):
    """Capacity run on the paper-scale mixed-boundary slab (117 x 117 x 119, 1848 orbitals,
    1440 occupied): one timed step (exx_apply + exx_energy + ace_build) in the fastest
    precision form that supports the grid, the device memory it held, and the VxPsi error of
    two sampled output columns (one occupied, one empty) against the CPU oracle."""
    import numpy as np
    import torch

    import oracle
    import paper_2501_16572_gb300 as exx
    import synth

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    s = synth.capacity_slab()
    t_gen = time.perf_counter() - t0
    free0, total = torch.cuda.mem_get_info(dev)
    psi = torch.from_numpy(s.psi).to(dev)
    f = torch.from_numpy(s.f).to(dev)
    prec_name = args.prec if args.prec != "auto" else pick_precision(exx, s, dev)
    plan = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    plan.set_precision(prec_code(exx, prec_name))
    W = torch.empty_like(psi)
    xi = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    plan.set_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    plan.apply(psi[:s.n_occ], f, psi, out=W)
    ev[1].record(stream)
    e_x = plan.energy(psi[:s.n_occ], f, W)
    plan.ace_build(psi, W, xi=xi)
    ev[2].record(stream)
    torch.cuda.synchronize()
    step_ms, apply_ms = ev[0].elapsed_time(ev[2]), ev[0].elapsed_time(ev[1])
    kt = plan.timing()
    free1, _ = torch.cuda.mem_get_info(dev)
    cols = [7, s.n_orb - 5]
    t1 = time.perf_counter()
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    ref = orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=cols)
    t_orc = time.perf_counter() - t1
    got = W[cols].cpu().numpy()
    err = {f"col{c}": float(np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])) for i, c in enumerate(cols)}
    rec = {"workload": s.name, "grid": list(s.n), "n_orb": s.n_orb, "n_occ": s.n_occ,
           "unique_pair_solves": s.unique_pairs(), "precision": prec_name,
           "ms_per_step": step_ms, "exx_apply_ms": apply_ms, "value": s.unique_pairs() / (apply_ms * 1e-3),
           "unit": UNIT + " (exx_apply)", "E_x": e_x,
           "kernel_times_ms": {k: round(v[0], 3) for k, v in kt.items() if v[1]},
           "device_bytes_held": int(free0 - free1), "device_bytes_total": int(total),
           "vxpsi_rel_vs_oracle": err, "oracle_seconds": t_orc, "oracle_threads": oracle.num_threads(),
           "input_generation_s": t_gen}
    plan.close()
    print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch48":
        run_batch48(a)
    elif a.workload == "sweep":
        run_sweep(a)
    elif a.workload == "precision":
        run_precision(a)
    elif a.workload == "capacity":
        run_capacity(a)
    else:
        run_ours(a)
