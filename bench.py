#!/usr/bin/env python
"""Benchmark of one exact-exchange + ACE step on GB300.

Workload (one step): the 48^3 periodic grid, h = 0.25 bohr, 12th-order FD, erfc-screened
kernel omega = 0.106, 128 orthonormal synthetic orbitals with Fermi-Dirac occupations
(Fermi level at orbital 100):
    VxPsi = exx_apply(Psi_occ = all 128, Psi_in = all 128)   (8256 unique pair solves)
    E_x   = exx_energy(...)
    xi    = ace_build(Psi, VxPsi)
Metric: pair-Poisson solves per second (each solve is one batched Kronecker solve of
one orbital pair, Sec. II.B) and the exx_apply time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--prec auto|fp64|bf16x3|tf32x3|bf16x6|bf16x10]
                       [--workload periodic48|batch48|sweep|precision|slab]
Other workloads (not the default line):
  batch48   48 independent systems (grids of 20-64 points per axis, 8-160 orbitals) solved
            by one exx_apply_batched call (one CUDA graph) per step, beside the same work
            issued as one exx_apply call per system.
  sweep     exx_apply of the 48^3 workload for pair batches n_c = 1 (one pair per solve
            sequence, the unbatched Kronecker solver) up to 1024.
  precision 48^3 grid with 256 orbitals: every precision mode against the FP64 path
            (VxPsi, xi, E_x errors and times).
  slab      72x72x144 slab (periodic x, y; Dirichlet z), 1024 orbitals, 800 occupied:
            BF16X10 step timed, FP64 path on 16 sampled output orbitals for the error.
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
L2_FLUSH_BYTES = 512 << 20
BATCH_WORKLOAD = ("batch48: 48 independent systems, seeded grid draws of 20-64 points per axis, "
                  "mixed Dirichlet/periodic axes, h=0.3, 12th-order FD, Coulomb kernel with any Dirichlet "
                  "axis else erfc omega=0.106, 8-160 orbitals with Fermi-Dirac occupations; "
                  "step = exx_apply of every system in one exx_apply_batched call")
FP64_PEAK_NOTE = "FP64 CUDA-core peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-vs-split comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n-orb", type=int, default=128)
    ap.add_argument("--batch", type=int, default=0, help="pairs per batch (0 = library default)")
    ap.add_argument("--workload", default="periodic48", choices=["periodic48", "batch48", "sweep", "precision", "slab"])
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
            "bf16x6": exx.EXX_PREC_BF16X6, "bf16x10": exx.EXX_PREC_BF16X10}[name]


def pick_precision(exx, s, dev):
    """'auto': the split-precision form that meets both error targets (VxPsi <= 1e-6,
    E_x <= 1e-8 relative), else FP64."""
    for name in ("bf16x10",):
        try:
            p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
            p.set_precision(prec_code(exx, name))
            p.close()
            return name
        except Exception:
            continue
    return "fp64"


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2501_16572_gb300 as exx

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    s = synth.config2(args.n_orb)
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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

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
            flush.fill_(1.0)                 # evict L2 between timed steps (untimed)
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
        "config": {"workload": WORKLOAD, "grid": list(s.n), "n_orb": s.n_orb, "n_occ": occ,
                   "unique_pair_solves_per_step": unique, "ordered_pairs_per_step": ordered,
                   "precision": prec_name, "l2": "flushed between timed steps (512 MB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "exx_apply_ms": apply_total_ms / K,
        "ordered_pairs_per_s": world * ordered * K / (total_ms / 1e3),
        "gpu_launches": launches,
        "E_x": e_main,
    }
    # -- roofline of the dominant kernel (CUDA events around every launch, timed region) --
    peaks = measured_peaks()
    if ktimes:
        dom = max(ktimes, key=lambda k: ktimes[k][0])
        dom_ms, dom_n = ktimes[dom]
        rec["kernel_times_ms"] = {k: round(v[0] / K, 4) for k, v in ktimes.items()}
        rec["roofline"] = roofline(exx, plan, s, prec_name, dom, dom_ms, dom_n, K, peaks, clk)
    rec["clocks"] = clk
    # -- FP64 vs split comparison --
    if not args.no_compare and prec_name != "fp64":
        W_split = W.clone()
        xi_split = xi.clone()
        p64 = make_plan("fp64")
        t64, a64, e64, _, _, _ = timed(p64, max(1, min(2, K)), 1, False)
        k64 = max(1, min(2, K))
        rec["fp64"] = {"ms_per_step": t64 / k64, "exx_apply_ms": a64 / k64,
                       "pair_solves_per_s": world * unique * k64 / (t64 / 1e3)}
        rec["split_vs_fp64_speedup"] = (t64 / k64) / (total_ms / K)
        rec["split_vs_fp64_apply_speedup"] = (a64 / k64) / (apply_total_ms / K)
        rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        rec["error_vs_fp64"] = {"vxpsi_rel_fro": rel(W_split, W), "xi_rel_fro": rel(xi_split, xi),
                                "E_x_rel": abs(e_main - e64) / abs(e64)}
        p64.close()
    # -- end to end through the host-buffer entry point --
    if not args.no_e2e:
        rec["e2e"] = e2e(exx, plan, s, K, world, dev)
    # -- CPU oracle baseline (rank 0, N = 1) --
    if rank == 0 and world == 1 and not args.no_cpu:
        rec["cpu_baseline"] = cpu_baseline(s)
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
    prec_name = args.prec if args.prec != "auto" else "bf16x10"
    plans, bufs = [], []
    for s in systems:
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec_code(exx, prec_name))
        plans.append(p)
        psi = torch.from_numpy(s.psi).to(dev)
        bufs.append((psi, torch.from_numpy(s.f).to(dev), torch.empty_like(psi)))
    bargs = [(psi[:s.n_occ], f, psi, out) for (psi, f, out), s in zip(bufs, systems)]
    unique = sum(s.unique_pairs() for s in systems)
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
                b = pass_bytes(prec_name, kind) * s.N * s.unique_pairs() + (8 * s.N * n if kind == "pass3" else 0)
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
                           "traffic": None, "kernel": f"tc_pass_kernel ({dom})", "launches": n,
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
        rec["cpu_baseline"] = cpu_baseline(systems[1])
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
    """exx_apply time of the 48^3 / 128-orbital workload against the pair batch size n_c."""
    import torch
    import synth
    import paper_2501_16572_gb300 as exx
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    s = synth.config2(args.n_orb)
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    prec_name = args.prec if args.prec != "auto" else "bf16x10"
    rows = []
    for nc, blk in [(1, 1), (4, 2), (16, 4), (64, 8), (256, 8), (512, 8), (1024, 8), (1024, 16), (1024, 32)]:
        p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
        p.set_precision(prec_code(exx, prec_name))
        p.set_batch(nc, blk)
        ms = _apply_ms(exx, p, psi, f, psi, out, max(1, args.steps), max(1, args.warmup if nc > 16 else 1), stream)
        launches = p.launch_count()
        p.set_timing(True)
        p.apply(psi, f, psi, out=out)
        kt = {k: round(v[0], 3) for k, v in p.timing().items()}
        p.set_timing(False)
        rows.append({"n_c": nc, "block_orbitals": blk, "exx_apply_ms": ms, "launches": launches,
                     "pair_solves_per_s": s.unique_pairs() / (ms / 1e3), "kernel_ms": kt})
        p.close()
    best = max(rows, key=lambda r: r["pair_solves_per_s"])
    rec = {"metric": METRIC, "value": best["pair_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": best["exx_apply_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": prec_name, "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": "n_c sweep of exx_apply on " + WORKLOAD.split(";")[0], "n_orb": s.n_orb,
                      "unique_pair_solves": s.unique_pairs(), "l2": "not flushed (back-to-back applies)"},
           "sweep": rows}
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
    for name in ("fp64", "bf16x10", "bf16x6", "tf32x3", "bf16x3"):
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
    b10 = [r for r in table if r["precision"] == "bf16x10"][0]
    rec = {"metric": METRIC, "value": b10["pair_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": 1, "ms_per_step": b10["exx_apply_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16x10", "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": "precision study: 48x48x48 periodic grid, erfc omega=0.106, 256 orbitals, "
                                  "Fermi-Dirac occupations; exx_apply timed per precision",
                      "unique_pair_solves": s.unique_pairs(), "l2": "not flushed (back-to-back applies)"},
           "precisions": table}
    print(json.dumps(rec), flush=True)


def run_slab(args):
    """72x72x144 slab, 1024 orbitals (800 occupied): BF16X10 step (exx_apply + energy +
    ACE) timed; the FP64 path recomputes 16 sampled output orbitals for the error."""
    import torch
    import synth
    import paper_2501_16572_gb300 as exx
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    s = synth.config5()
    t_synth = time.perf_counter() - t0
    psi = torch.from_numpy(s.psi).cuda()
    f = torch.from_numpy(s.f).cuda()
    occ = s.n_occ
    stream = torch.cuda.current_stream()
    prec_name = args.prec if args.prec != "auto" else "bf16x10"
    p = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    p.set_precision(prec_code(exx, prec_name))
    W = torch.empty_like(psi)
    xi = torch.empty_like(psi)
    for _ in range(args.warmup):
        p.apply(psi[:occ], f, psi, out=W)
    torch.cuda.synchronize()
    ms, apply_ms, e = [], [], 0.0
    clocks = Clocks(local)
    clocks.start()
    for _ in range(args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        p.apply(psi[:occ], f, psi, out=W)
        ev[1].record(stream)
        e = p.energy(psi[:occ], f, W)
        p.ace_build(psi, W, xi=xi)
        ev[2].record(stream)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[2]))
        apply_ms.append(ev[0].elapsed_time(ev[1]))
    clk = clocks.stop()
    cols = list(range(0, s.n_orb, s.n_orb // 16))[:16]
    p64 = exx.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    sub = psi[cols].contiguous()
    ref = torch.empty_like(sub)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    p64.apply(psi[:occ], f, sub, out=ref)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    rel = float(torch.linalg.norm(W[cols] - ref) / torch.linalg.norm(ref))
    unique = s.unique_pairs()
    K = args.steps
    rec = {"metric": METRIC, "value": unique * K / (sum(ms) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K,
           "warmup": args.warmup, "ms_per_step": sum(ms) / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": prec_name, "data": "synthetic (seeded Gaussian orbitals in the bottom 70% of z, orthonormalised)",
           "config": {"workload": "slab 72x72x144, periodic x,y, Dirichlet z, h=0.2, erfc omega=0.106, 1024 orbitals, "
                                  "800 occupied; step = exx_apply + exx_energy + ace_build",
                      "unique_pair_solves_per_step": unique, "ordered_pairs_per_step": s.ordered_pairs(),
                      "l2": "inputs (6.1 GB) larger than L2"},
           "exx_apply_ms": sum(apply_ms) / K, "E_x": e, "clocks": clk,
           "fp64_sampled": {"output_orbitals": cols, "pair_solves": occ * len(cols), "exx_apply_ms": ms64,
                            "pair_solves_per_s": occ * len(cols) / (ms64 / 1e3),
                            "vxpsi_rel_fro_of_sampled_vs_fp64": rel},
           "input_generation_s": t_synth}
    print(json.dumps(rec), flush=True)


# bytes per grid element a pass must read and write (its input and output planes); pass 1
# reads the FP32 hi/lo planes of both orbitals, pass 3 also reads f(Lambda) (hi/lo) once
# per launch.  BF16X10 keeps hi+lo intermediates (8 B), the other split modes FP32 (4 B).
def pass_bytes(prec, kind):
    inter = 8 if prec in ("bf16x10", "fp64") else 4
    if prec == "fp64":
        return {"pass1": 16 + 8, "pass2": 16, "pass3": 32, "pass4": 16, "pass5": 16}[kind]
    return {"pass1": 16 + inter, "pass2": 2 * inter, "pass3": 2 * inter, "pass4": 2 * inter, "pass5": 2 * inter}[kind]


def roofline(exx, plan, s, prec, kind, ms, nlaunch, K, peaks, clk):
    """Achieved throughput of the dominant kernel class from its live CUDA-event time."""
    n = s.n
    N = s.N
    unique = s.unique_pairs()
    fields_per_launch = unique * K / max(1, nlaunch) * (2 if (prec == "fp64" and kind == "pass3") else 1)
    axis_K = {"pass1": n[2], "pass2": n[0], "pass3": n[1], "pass4": n[0], "pass5": n[2]}
    avg_s = ms / max(1, nlaunch) / 1e3
    out = {}
    if kind in axis_K and prec == "fp64":
        contractions = 1   # FP64 pass 3 is two launches, one contraction each
        flops = 2.0 * N * axis_K[kind] * contractions * fields_per_launch
        achieved = flops / avg_s / 1e12
        peak = 152 * 2 * 2 * 2.07e9 / 1e12
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "kernel": f"fp64_pass_kernel ({kind})",
               "peak_source": FP64_PEAK_NOTE + " (derived from unit counts and clock, not measured)",
               "algorithmic_flops_per_launch": flops}
    elif kind in axis_K:
        byt = pass_bytes(prec, kind) * N * fields_per_launch + (8 * N if kind == "pass3" else 0)
        achieved = byt / avg_s / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        contractions = 2 if kind == "pass3" else 1
        nprod = {"bf16x10": 10, "bf16x6": 7, "bf16x3": 3, "tf32x3": 3}.get(prec, 1)
        flops = 2.0 * N * axis_K[kind] * contractions * fields_per_launch
        out = {"bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
               "kernel": f"tc_pass_kernel ({kind})",
               "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s",
               "algorithmic_bytes_per_launch": byt,
               "fields_per_launch": fields_per_launch,
               "algorithmic_tflops": flops / avg_s / 1e12,
               "tensor_executed_tflops": nprod * flops / avg_s / 1e12,
               "tensor_executed_frac_of_bf16": nprod * flops / avg_s / 1e12 / peaks.get("bf16_tflops_sustained", 1751.7)}
    else:
        out = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "kernel": kind}
    out["launches"] = nlaunch
    out["avg_launch_ms"] = ms / max(1, nlaunch)
    tr = traffic_for(out["kernel"].split(" ")[0] + ":" + kind + ":" + prec)
    if tr:
        # DRAM bytes per launch from the committed ncu capture, scaled to this launch size
        out["traffic"] = tr["bytes_per_field"] * fields_per_launch
        out["traffic_source"] = tr["source"]
    else:
        out["traffic"] = None
    return out


def e2e(exx, plan, s, K, world, dev):
    import torch
    psi_h = torch.from_numpy(s.psi.copy()).pin_memory()
    f_h = torch.from_numpy(s.f.copy()).pin_memory()
    xi_h = torch.empty_like(psi_h).pin_memory()
    plan.ace_step_host(psi_h, s.n_occ, f_h, xi_h)       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        plan.ace_step_host(psi_h, s.n_occ, f_h, xi_h)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / K
    return {"value": world * s.unique_pairs() / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(psi_h.numel() * 8 + f_h.numel() * 8),
            "d2h_bytes_per_step": int(xi_h.numel() * 8 + 8),
            "entry": "exx_ace_step_host (pinned host Psi, f in; xi, E_x out)"}


def cpu_sample(s, budget_s=15.0):
    """Time the CPU oracle on whole output columns of the workload (each column = n_occ
    pair solves) until about budget_s seconds of work have run."""
    import oracle
    orc = oracle.Plan(s.n, s.h, s.bc, s.fd_order, s.kernel, s.omega)
    cols = 0
    t0 = time.perf_counter()
    while True:
        orc.exx_apply(s.psi[:s.n_occ], s.f, s.psi, cols=[cols % s.n_orb])
        cols += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or cols >= s.n_orb:
            break
    solves = cols * s.n_occ
    return solves / dt, cols, solves, dt, oracle.num_threads()


def cpu_baseline(s):
    v, cols, solves, dt, cores = cpu_sample(s)
    rec = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{cols} output column(s) of the workload = {solves} pair Poisson solves "
                     f"(plain C FP64 oracle, {dt:.1f} s)"}
    # one core on the 24^3 Dirichlet workload (16 orbitals, f = 2): the whole apply
    import oracle
    import synth
    c1 = synth.config1()
    orc = oracle.Plan(c1.n, c1.h, c1.bc, c1.fd_order, c1.kernel, c1.omega)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        orc.exx_apply(c1.psi, c1.f, c1.psi)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    rec["single_core_24cube_16orb"] = {"value": c1.n_orb * c1.n_occ / dt1, "unit": UNIT, "cores": 1,
                                       "seconds": dt1, "pair_solves": c1.n_orb * c1.n_occ}
    return rec


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    s = synth.config2(args.n_orb)
    budget = 8.0
    for _ in range(args.warmup):
        cpu_sample(s, budget_s=1.0)
    vals, tot_solves, tot_t = [], 0, 0.0
    for _ in range(args.steps):
        v, cols, solves, dt, cores = cpu_sample(s, budget_s=budget)
        vals.append(v)
        tot_solves += solves
        tot_t += dt
    value = tot_solves / tot_t
    rec = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Gaussian + plane-wave orbitals, orthonormalised)",
           "config": {"workload": WORKLOAD, "grid": list(s.n), "n_orb": s.n_orb, "n_occ": s.n_occ,
                      "sample": "each step: whole output columns of the workload for about 8 s"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} steps x ~{budget:.0f} s of whole output columns "
                                      f"({tot_solves} pair solves)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    elif a.workload == "slab":
        run_slab(a)
    else:
        run_ours(a)
