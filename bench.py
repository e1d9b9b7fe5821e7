#!/usr/bin/env python
"""Benchmark of the per-column Krylov Green's-function path on GB300.

One step = one whole energy + force evaluation of the 4096-atom disordered diamond system
(8x8x8 cells, sigma 0.1 A, cluster radius 6 A, nu 30, 16384 columns, kT 0.1 eV): neighbour
and cluster lists and Slater-Koster H, S (a1, a2), every Green's-function column (a3-a6), the
chemical-potential bisection (a7), the density matrix (a8), energies (a9) and forces (a10).
Positions are resident in HBM when the timed region starts (value); the e2e figure runs the
same step through the public API from pinned host positions, with the host->device copy of the
positions and the device->host read of forces and energies inside the timed region.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun) each rank runs an independent replica (the path has no exchange step on
one system); value is the total columns of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Green's-fn columns/sec & energy+force steps/sec at |drho|<=1e-10, batched vs plain"
WORKLOAD = "diamond_4096"
DESCRIPTION = {"diamond_4096": "disordered diamond (8x8x8 cells, sigma 0.1 A)",
               "composite_32768": "graphite with diamond grains (sp2-sp3 composite)",
               "amorphous_1m": "dense disordered carbon (3.0 g/cm3, sigma 0.3 A)",
               "diamond_64": "disordered diamond (2x2x2 cells, sigma 0.05 A)"}
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07     # SMs x FP64 FMA/clk/SM x 2 flops x GHz
# DRAM bytes (read + write) of one k_krylov launch on the 4096-atom step, from the ncu capture in
# profiles/k_krylov_diamond4096.md; valid only while krylov.cu is the source that was captured.
# DRAM bytes (read + write) of the k_krylov launches of one 4096-atom step, from one ncu capture
# of the source whose sha256 prefix (krylov.cu + krylov.cuh) is given; reported per launch, null
# once that source changes
KRYLOV_TRAFFIC = {"krylov_sha256_prefix": "1dea01a43985331b", "bytes_per_step": 176.29e9,
                  "launches_per_step": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--k3-ctas", type=int, default=0, help="Krylov CTAs per SM (0: as many as fit)")
    ap.add_argument("--no-exact", action="store_true",
                    help="skip the energy + exact-force step (gradient through the truncated Krylov build)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- oracle timing
def _oracle_worker(args):
    name, cols = args
    os.environ["OMP_NUM_THREADS"] = "1"
    import workloads as wl
    from oracle import pipeline
    w = wl.make(name)
    t0 = time.perf_counter()
    res = pipeline.columns(w, cols)
    mu = 0.0
    for c in res:
        pipeline.rho_column(c, mu, w.kT)
    return time.perf_counter() - t0, len(res)


def oracle_columns_per_s(name: str, n_sample: int):
    """The oracle as it stands on a bounded seeded sample of columns, on every host core."""
    import multiprocessing as mp

    import workloads as wl
    w = wl.make(name)
    cols = wl.sample_columns(4 * w.n_atoms, n_sample)
    cores = os.cpu_count() or 1
    chunks = [(name, cols[i::cores]) for i in range(cores) if len(cols[i::cores])]
    ctx = mp.get_context("spawn")
    env_prev = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with ctx.Pool(len(chunks)) as pool:
            pool.map(_oracle_worker, [(name, c[:1]) for _, c in chunks])      # import / setup
            t0 = time.perf_counter()
            out = pool.map(_oracle_worker, chunks)
            wall = time.perf_counter() - t0
    finally:
        for k, v in env_prev.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    n = sum(o[1] for o in out)
    return n / wall, len(chunks), f"{n} seeded columns of {name} (Krylov build, projected eigenproblem, spectra, rho column), one process per core"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            for name, v in zip(names, r[3:]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


# ----------------------------------------------------------------------------- algorithmic flops
def aggregate(ms_local, units_local, world, dist=None, device=None):
    """Whole-job figures of N independent replicas: (max step time over ranks in ms, total
    units of all ranks per second). world == 1 needs no process group."""
    if world == 1 or dist is None:
        return ms_local, units_local / (ms_local * 1e-3)
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(u.item()) / (ms * 1e-3)


def krylov_traffic():
    import hashlib
    h = hashlib.sha256()
    for name in ("krylov.cu", "krylov.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1210_1531_gb300", "csrc", name), "rb").read())
    h = h.hexdigest()[:16]
    if h != KRYLOV_TRAFFIC["krylov_sha256_prefix"]:
        return None
    return KRYLOV_TRAFFIC["bytes_per_step"] / KRYLOV_TRAFFIC["launches_per_step"]


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # spawn pool before any CUDA work of this process
        v, cores, sample = oracle_columns_per_s(args.workload, args.cpu_sample)
        cpu_base = {"value": v, "unit": "columns/s", "cores": cores, "kind": "oracle", "sample": sample}

    from paper_1210_1531_gb300 import build
    build.build()
    import paper_1210_1531_gb300 as eg
    import workloads as wl

    w = wl.make(args.workload)
    M = 4 * w.n_atoms
    stream = torch.cuda.current_stream()
    pos_dev = torch.tensor(w.pos, dtype=torch.float64, device="cuda")
    forces = torch.empty((w.n_atoms, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make(schedule, exact_forces=False, autotune=False, graph=False):
        return eg.System(pos_dev, w.box, w.sk, w.r_cluster, w.nu, w.kT, w.n_electrons,
                         nu_classes=w.nu_classes, schedule=schedule, timing=True,
                         k3_ctas_per_sm=args.k3_ctas, exact_forces=exact_forces,
                         autotune=autotune and args.k3_ctas == 0, graph=graph)

    def step(s):
        s.rebuild(pos_dev)
        return s.energy_force(forces)

    keys = ("launches", "krylov_launches", "t_krylov_ms", "t_eig_ms", "t_bisect_ms",
            "t_density_ms", "t_force_ms", "krylov_flops", "t_adjoint_ms")

    def timed(s, k, w_steps, barrier=False):
        """w_steps untimed steps, then k steps each timed with CUDA events on the stream; the
        counters of each step (reset by its rebuild) are accumulated."""
        for _ in range(w_steps):
            step(s)
        torch.cuda.synchronize()
        if barrier:
            dist.barrier()
            torch.cuda.synchronize()
        acc = dict.fromkeys(keys, 0.0)
        times, out = [], None
        for _ in range(k):
            flush.zero_()                       # L2 flush between timed steps (not timed)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = step(s)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            st = s.stats()
            for key in keys:
                acc[key] += st[key]
        torch.cuda.synchronize()
        if barrier:
            dist.barrier()
            torch.cuda.synchronize()
        acc["bisect_steps"] = s.stats()["bisect_steps"]
        return times, acc, out

    # the production form: launch shape tuned at build (before timing), the step replayed as a
    # CUDA graph (captured during the warm-up steps)
    batched = make(1, autotune=True, graph=True)
    tuned = batched.autotune_shapes()
    with ClockSampler(local) as clk:
        times, stats, out = timed(batched, args.steps, args.warmup, barrier=world > 1)
    ms, value = aggregate(sum(times) / len(times), M, world, dist if world > 1 else None, "cuda")
    mu, e_band, f_free, _ = out

    # kernel roofline of the dominant kernel (Krylov build + projection), event-timed per launch
    # algorithmic flops counted by the kernel per column (formula in include/elses.h, elses_stats)
    k_launch_ms = stats["t_krylov_ms"] / max(1, stats["krylov_launches"])
    flops_per_launch = stats["krylov_flops"] / max(1.0, stats["krylov_launches"])
    achieved = flops_per_launch / (k_launch_ms * 1e-3) / 1e9      # GFLOP/s
    peak_probe = eg.probe_fp64()

    # plain schedule, same step, fewer repetitions (reported beside the batched form)
    plain = make(0)
    pt, _, _ = timed(plain, max(3, args.steps // 2), 1)
    plain_ms = sum(pt) / len(pt)
    plain.close()

    # end to end through the public API from pinned host memory
    pos_host = torch.tensor(w.pos, dtype=torch.float64).pin_memory()
    f_host = torch.empty((w.n_atoms, 3), dtype=torch.float64).pin_memory()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pos_dev.copy_(pos_host, non_blocking=True)
        batched.rebuild(pos_dev)
        res = batched.energy_force(forces)
        f_host.copy_(forces, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            e2e_times.append(a.elapsed_time(b))
    e2e_ms = sum(e2e_times) / len(e2e_times)

    # the same step with exact forces (the gradient through the truncated Krylov build)
    exact = None
    if not args.no_exact:
        ex = make(1, exact_forces=True)
        xt, xst, _ = timed(ex, 2, 1)
        x_ms = sum(xt) / len(xt)
        exact = {"ms_per_step": x_ms, "value": M / (x_ms * 1e-3), "unit": "columns/s",
                 "t_adjoint_ms": xst["t_adjoint_ms"] / 2,
                 "note": "forces = exact gradient of Omega through the truncated Krylov build "
                         "(finite-difference gated at 1e-5); 2 timed steps after 1 warm-up"}
        ex.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "columns/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "steps_per_s": 1e3 / ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, w, world),
            "plain": {"ms_per_step": plain_ms, "value": M / (plain_ms * 1e-3), "unit": "columns/s"},
            "exact_forces": exact,
            "autotuned_shapes": {f"{k}-atom clusters": f"{b} CTAs/SM, queue by {o}"
                                 for k, (b, o) in tuned.items()},
            "phases_ms_per_step": {k: stats[k] / args.steps for k in
                                   ("t_krylov_ms", "t_eig_ms", "t_bisect_ms", "t_density_ms", "t_force_ms")},
            "e2e": {"value": world * M / (e2e_ms * 1e-3), "unit": "columns/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(pos_host.numel() * 8),
                    "d2h_bytes_per_step": int(f_host.numel() * 8 + 3 * 8)},
            "gpu_launches": int(stats["launches"]),
            "roofline": {"bound": "alu", "kernel": "k_krylov (a3 Krylov build + a4 projection)",
                         "achieved": achieved, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_NOMINAL_GFLOPS,
                         "traffic": krylov_traffic() if args.workload == WORKLOAD else None,
                         "peak_probe": peak_probe, "flops_per_launch": flops_per_launch,
                         "launch_ms": k_launch_ms, "ctas_per_sm": batched.stats()["k3_ctas_per_sm"],
                         "launches_per_step": stats["krylov_launches"] / args.steps,
                         "peak_note": "FP64 FMA pipe: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s); peak_probe = measured FMA-chain throughput"},
            "clocks": clk.summary(),
            "result": {"mu": mu, "e_band": e_band, "f_free": f_free, "bisect_steps": stats["bisect_steps"]},
        }
        if cpu_base is not None:
            line["cpu_baseline"] = cpu_base
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def bench_config(args, w, world):
    """The workload configuration both arms report."""
    M = 4 * w.n_atoms
    nu = "/".join(str(v) for _, v in w.nu_classes) + " by cluster size" if w.nu_classes else str(w.nu)
    cl = f"{w.r_cluster:g} A" if w.r_cluster > 0 else "= whole system"
    return {"workload": f"{args.workload}: {DESCRIPTION.get(args.workload, 'synthetic system')}, "
                        f"{w.n_atoms} atoms, cluster {cl}, nu {nu}, {M} columns, "
                        f"kT {w.kT} eV, full energy+force step",
            "columns_per_step": M,
            "schedule": "batched (persistent, size-sorted queue, autotuned launch shape, CUDA graph)",
            "l2": "256 MB buffer written between timed steps",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import workloads as wl
    w = wl.make(args.workload)
    M = 4 * w.n_atoms
    per_step = max(64, min(args.cpu_sample, M) // 4)
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, sample = oracle_columns_per_s(args.workload, per_step)
        if i >= args.warmup:
            vals.append(v)
    v = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "columns/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": M / v * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, w, args.gpus),
        "cpu_baseline": {"value": v, "unit": "columns/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
