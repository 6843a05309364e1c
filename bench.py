#!/usr/bin/env python3
"""Throughput benchmark of the pgen graph generators on GB300.

One step = one full pass of the generation path over the workload:
  pba_n2p30_b1024_m5  two-phase PBA, 2^30 new vertices in 1024 blocks, m = 5
                      (prefix -> phase 1 -> count scan -> phase 2 + substitution)
  kron_k20_m16x_csr   stochastic Kronecker k = 20, 16 * 2^20 edges, then CSR
  ba_n100k_m4         serial BA, 100,000 new vertices, m = 4
Prints ONE JSON line (rank 0). Under torchrun every rank generates its own
instance (seed + rank): replicas, weak scaling, no collective on the data path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference    # the CPU oracle on a bounded sample
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

from paper_1003_3684_gb300 import workloads as W  # noqa: E402

DEFAULT_WORKLOAD = "pba_n2p30_b1024_m5"

# Algorithmic work per unit (32-bit lane operations and bytes), per kernel.
# A Philox4x32-10 call is 60 lane ops (10 rounds of two 32x32->64 multiplies,
# counted as two ops each, and two three-input XORs); a 64-bit uniform draw
# adds 4. Where a kernel's counters keep words 1..3 fixed (phase 1's (j, 0, p, 1),
# the serial method's (i, 0, 0, 2)), two of the twenty multiplies are done once
# per fixed prefix, so such a draw counts 56. Chain links recomputed beyond the
# first draw of a unit are NOT counted: they are the implementation's overhead,
# not the method's work.
PHILOX_OPS = 60
PHILOX_HEADED_OPS = 56
KERNEL_WORK = {
    # unit = one phase-1 entry: its own draw (coin + uniform index) + select
    "pba_phase1": dict(ops=PHILOX_HEADED_OPS + 4 + 6, bytes=2),
    # unit = one edge: its endpoint draw + uniform + sigma/E index arithmetic
    # and the rank bookkeeping; bytes = the (src, dst) pair written
    "pba_emit": dict(ops=PHILOX_OPS + 4 + 16, bytes=8),
    "ba_chain": dict(ops=PHILOX_HEADED_OPS + 4 + 16, bytes=8),
}


# Sorting kernels of the CSR step: HBM-bound; unit = one edge per launch, bytes
# = what one launch must move at least (a radix pass reads and writes every
# pair; the histogram pass and the sortedness check read every pair once).
CSR_WORK = {
    "csr_radix_scatter": dict(ops=0, bytes=16),
    "csr_radix_hist": dict(ops=0, bytes=8),
    "csr_check": dict(ops=0, bytes=8),
    "csr_finish": dict(ops=0, bytes=12),
}


def dram_traffic_table():
    """DRAM bytes per unit measured by ncu, from profiles/dram_traffic.json.

    Each entry names the kernel, the source file it is compiled from and that
    file's sha256 prefix at capture time; an entry whose file has changed since
    is ignored (the counters no longer describe the kernel that runs).
    """
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    table = {}
    try:
        with open(path) as fh:
            rows = json.load(fh)["kernels"]
    except (OSError, ValueError, KeyError):
        return table
    for row in rows:
        try:
            with open(os.path.join(ROOT, row["source"]), "rb") as fh:
                cur = hashlib.sha256(fh.read()).hexdigest()[:12]
            if cur == row["sha256"]:
                table[row["kernel"]] = float(row["bytes_per_unit"])
        except (OSError, KeyError, TypeError, ValueError):
            continue
    return table


def kron_work(k: int, id_bytes: int = 4):
    # ceil(k/4) Philox calls + per level: 3 threshold compares + 2 shift-ors
    return dict(ops=PHILOX_OPS * ((k + 3) // 4) + 5 * k, bytes=2 * id_bytes)


def kron_det_work(k: int, id_bytes: int = 4):
    # per level: one base-e0 digit (a fixed-point divide), one seed lookup,
    # two multiply-adds into the ids; no random draws
    return dict(ops=6 * k, bytes=2 * id_bytes)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)),
                    source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


# --------------------------------------------------------------------------
# several GPUs: independent replicas (no collective on the data path)
# --------------------------------------------------------------------------
def replica_seed(base_seed: int, rank: int) -> int:
    """Rank r generates its own instance of the workload, seeded base + r."""
    return base_seed + rank


def max_over_ranks(value: float, device, world: int) -> float:
    """The largest value over the ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Units of the whole job per second: every rank's units over the slowest time."""
    return units_per_rank_step * steps * world / (ms_max / 1000.0)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[0]), smax=float(parts[1]),
                                 hw=parts[4], hwt=parts[5], swt=parts[6], swp=parts[7],
                                 util=float(parts[8]) if parts[8] not in ("", "[N/A]") else 0.0))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in load),
                    sm_max_mhz=max(r["smax"] for r in rows), reasons=sorted(reasons),
                    samples=len(load))


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# --------------------------------------------------------------------------
def all_cores_estimate(value: float) -> dict:
    """The one-core oracle rate scaled by the host's core count: a labelled
    estimate (the blocks of the workload are independent), not a measurement."""
    n = os.cpu_count() or 1
    return dict(value=value * n, host_cores=n, note="estimate: one-core rate x host cores")


def oracle_sample(name: str, cfg: dict, budget_s: float):
    """Time the oracle, as it stands, on samples of the workload.

    PBA: the full two-phase oracle on 2 blocks of the workload's own block size
    (same n_b, m, n0, f, W): per-edge work is that of the full graph, which
    only has more blocks. Kronecker: the oracle descent for 2^20 edges of the
    same initiator and k, plus CSR of them. Returns (edges/s, description,
    seconds, samples).
    """
    import numpy as np

    import oracle as o
    t_total, edges_total, samples = 0.0, 0, 0
    if cfg["kind"] == "batch":
        jobs = W.batch_jobs(cfg["n_jobs"], seed=cfg["seed"])
    if cfg["kind"] == "serve":
        from paper_1003_3684_gb300 import serve
        trace = serve.poisson_workload(cfg["rate"], 2.0, seed=cfg["seed"])
    if cfg["kind"] == "bfs":
        # the oracle BFS over the undirected CSR of a 2-block graph of the same
        # block size (built once, not timed), from a new source each sample
        nb = cfg["n"] // cfg["blocks"]
        e, _, _ = o.pba(2 * nb, cfg["m"], 2, cfg["n0"], 1, cfg["inter_frac"], cfg["seed"])
        Ns = 2 * (cfg["n0"] + nb)
        rp, col = o.csr_opts(e, Ns, o.CSR_SYMMETRIZE)
    while samples == 0 or t_total < budget_s:
        if cfg["kind"] == "bfs":
            t0 = time.perf_counter()
            _, _, sc = o.bfs(rp, col, (samples * 2654435761) % Ns)
            t_total += time.perf_counter() - t0
            edges_total += sc
            desc = (f"or_bfs over the undirected CSR of a 2-block PBA graph (n_b={nb}, "
                    f"m={cfg['m']}); adjacency entries scanned per sample")
        elif cfg["kind"] == "serve":
            _, j = trace[(samples * 97) % len(trace)]
            t0 = time.perf_counter()
            e = (o.ba(j["n"], j["m"], j["n0"], j["seed"]) if j["kind"] == "pba"
                 else o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"]))
            o.csr(e, serve.job_vertices(j))
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = "oracle graph + CSR of requests of the trace (every 97th)"
        elif cfg["kind"] == "batch":
            j = jobs[(samples * 97) % len(jobs)]
            t0 = time.perf_counter()
            e = (o.ba(j["n"], j["m"], j["n0"], j["seed"]) if j["kind"] == "pba"
                 else o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"]))
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = "oracle on jobs of the batch (every 97th job)"
        elif cfg["kind"] == "kron_xor":
            M, Mr = 2**20, 2**20 * cfg["n_random"] // cfg["n_edges"]
            t0 = time.perf_counter()
            pk = o.kron(cfg["initiator"], cfg["k"], M, cfg["seed"] + samples)
            rnd = o.random_cells(2 ** cfg["k"], Mr, cfg["seed"] + samples)
            o.csr_opts(np.concatenate([pk, rnd]), 2 ** cfg["k"], o.CSR_ODD)
            t_total += time.perf_counter() - t0
            edges_total += M + Mr
            desc = (f"or_kron k={cfg['k']} ({M} edges) + or_random_cells ({Mr}) + "
                    "or_csr_opts (odd multiplicity) per sample")
        elif cfg["kind"] == "kron_det":
            ks = min(cfg["k"], 6)
            t0 = time.perf_counter()
            e, _ = o.kron_det(cfg["initiator"], ks)
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = (f"or_kron_det (the literal meta-edge stack) of the same seed at k={ks} "
                    f"({e.shape[0]} edges) per sample")
        elif cfg["kind"] == "pba" and cfg["blocks"] > 1 and cfg.get("factions"):
            B = 2
            n = B * (cfg["n"] // cfg["blocks"])
            t0 = time.perf_counter()
            e, _, _ = o.pba_factions(n, cfg["m"], B, cfg["n0"], W.ring_factions(B, 3),
                                     cfg["inter_frac"], cfg["seed"] + samples)
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = (f"or_pba_factions, 2 blocks of n_b={cfg['n'] // cfg['blocks']} with ring "
                    f"lists, m={cfg['m']}, f={cfg['inter_frac']}: {e.shape[0]} edges per sample")
        elif cfg["kind"] == "pba" and cfg["blocks"] > 1:
            B = 2
            n = B * (cfg["n"] // cfg["blocks"])
            t0 = time.perf_counter()
            e, _, _ = o.pba(n, cfg["m"], B, cfg["n0"], cfg["faction_width"] if
                            cfg["faction_width"] < B else 1, cfg["inter_frac"],
                            cfg["seed"] + samples)
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = (f"or_pba, 2 blocks of n_b={cfg['n'] // cfg['blocks']}, m={cfg['m']}, "
                    f"n0={cfg['n0']}, f={cfg['inter_frac']}: {e.shape[0]} edges per sample")
        elif cfg["kind"] == "pba":
            t0 = time.perf_counter()
            e = o.ba(cfg["n"], cfg["m"], cfg["n0"], cfg["seed"] + samples)
            t_total += time.perf_counter() - t0
            edges_total += e.shape[0]
            desc = f"or_ba, the full workload ({e.shape[0]} edges) per sample"
        else:
            M = 2**20
            t0 = time.perf_counter()
            e = o.kron(cfg["initiator"], cfg["k"], M, cfg["seed"] + samples)
            if cfg.get("csr"):
                o.csr(e, 2 ** cfg["k"])
            t_total += time.perf_counter() - t0
            edges_total += M
            desc = f"or_kron k={cfg['k']}, {M} edges per sample" + (" + or_csr" if cfg.get("csr") else "")
        samples += 1
    return edges_total / t_total, desc, t_total, samples


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    cfg = W.CONFIGS[args.workload]
    times, eps = [], []
    desc = ""
    for _ in range(args.warmup):
        oracle_sample(args.workload, cfg, 0.0)
    for _ in range(args.steps):
        v, desc, t, _ = oracle_sample(args.workload, cfg, 0.0)
        times.append(t)
        eps.append(v)
    value = sum(v * t for v, t in zip(eps, times)) / sum(times)
    metric, unit = (("traversed_entries/sec", "entries/s") if cfg["kind"] == "bfs"
                    else ("edges/sec", "edges/s"))
    line = dict(impl="reference", metric=metric, value=value, unit=unit,
                n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * statistics.mean(times), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="u32", data="synthetic",
                config=dict(workload=args.workload, sample=desc),
                cpu_baseline=dict(kind="oracle", value=value, unit=unit, cores=1,
                                  sample=desc, all_cores_estimate=all_cores_estimate(value)),
                e2e=dict(value=value, unit=unit, h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def batch_work(jobs):
    """Algorithmic int32 ops of a batch (one draw per edge, as KERNEL_WORK)."""
    ops = 0
    for j in jobs:
        if j["kind"] == "pba":
            ops += j["n"] * j["m"] * KERNEL_WORK["ba_chain"]["ops"]
        else:
            ops += j["n_edges"] * kron_work(j["k"])["ops"]
    return ops


def run_batch(args, rank: int, world: int, local_rank: int):
    """Batched workload: one CUDA-graph replay of the persistent batch kernel
    per step, against the same jobs launched one graph at a time."""
    import torch
    import torch.distributed as dist

    from paper_1003_3684_gb300 import autotune
    from paper_1003_3684_gb300 import build as pbuild
    pbuild.build()
    import paper_1003_3684_gb300 as pg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cfg = W.CONFIGS[args.workload]
    jobs = W.batch_jobs(cfg["n_jobs"], seed=cfg["seed"] + rank)
    if args.batch_jobs:
        jobs = jobs[:args.batch_jobs // 2] + jobs[cfg["n_jobs"] // 2:][:args.batch_jobs // 2]
    total = sum(j["n"] * j["m"] + j["n0"] * (j["n0"] - 1) // 2 if j["kind"] == "pba"
                else j["n_edges"] for j in jobs)
    free, _ = torch.cuda.mem_get_info()
    # waves: split the jobs so that one wave's arena fits in free memory
    waves = 1
    while total * 8 / waves > 0.8 * free and waves < 8:
        waves += 1
    chunks = [jobs[i::waves] for i in range(waves)]
    tune = autotune.tune_batch(chunks[0], reps=1, tiles=(2048, 4096, 8192), fractions=(1.0,))
    plans = [pg.BatchPlan(c, tile_edges=tune["tile_edges"]) for c in chunks]
    # one arena serves both arms; the per-graph arm places every job at an
    # even edge offset (16-byte aligned output, as gen_pba/gen_kronecker need)
    arena = torch.empty((max(p.total_edges for p in plans) + len(jobs) + 2, 2), dtype=torch.int32,
                        device=dev)
    ws = torch.empty(pg.pg_batch_workspace_size(), dtype=torch.uint8, device=dev)
    graphs = []
    for p in plans:
        pg.gen_batch(p, arena=arena, workspace=ws, grid_ctas=tune["grid_ctas"])
        torch.cuda.synchronize()
        gph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gph):
            pg.gen_batch(p, arena=arena, workspace=ws, grid_ctas=tune["grid_ctas"])
        graphs.append(gph)

    def step():
        for gph in graphs:
            gph.replay()

    # per-graph baseline: every job its own gen_pba / gen_kronecker call
    def per_graph():
        for c, p in zip(chunks, plans):
            a = 0
            for i, j in enumerate(c):
                size = int(p.offsets[i + 1] - p.offsets[i])
                if j["kind"] == "pba":
                    pg.gen_pba(j["n"], j["m"], 1, j["n0"], 1, 0.0, j["seed"],
                               out=arena[a:a + size])
                else:
                    pg.gen_kronecker(j["initiator"], j["k"], j["n_edges"], j["seed"],
                                     out=arena[a:a + size])
                a += size + (size & 1)

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    per_graph()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        dist.barrier()
    pg.pg_trace_dump()
    pg.pg_trace_enable(True)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    pg.pg_trace_enable(False)
    kernels = pg.pg_trace_dump()
    ms = ev0.elapsed_time(ev1)
    # per-graph launches, timed the same way
    pg_steps = max(1, min(args.steps, 3))
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(pg_steps):
        per_graph()
    ev3.record(stream)
    torch.cuda.synchronize()
    ms_pg = ev2.elapsed_time(ev3) / pg_steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = total * args.steps * world / (ms_max / 1000.0)
    peaks = load_peaks()
    sms = pg.pg_device_sm_count()
    alu_peak = sms * 128 * peaks["sm_max_mhz"] * 1e6
    # inside a graph replay the library's trace does not run: the replays are
    # timed by the events above, one persistent launch (plus a 8-byte counter
    # reset) per wave per step
    launches = args.steps * waves
    kernels = {"batch_persistent (graph replay)": (launches, ms_max)}
    per_launch = ms_max / launches / 1000.0
    ops = batch_work(jobs) / waves
    roof = dict(bound="alu", kernel="batch_persistent", achieved=ops / per_launch / 1e12,
                peak=alu_peak / 1e12, unit="Tops/s (int32 lane ops)",
                frac=ops / per_launch / alu_peak, traffic=None,
                hbm=dict(achieved=total * 8 / waves / per_launch / 1e9, peak=peaks["hbm_gbs"],
                         unit="GB/s", frac=total * 8 / waves / per_launch / (peaks["hbm_gbs"] * 1e9)),
                ms_per_launch=per_launch * 1000.0,
                peak_source=f"{sms} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz")
    line = dict(metric="edges/sec", value=value, unit="edges/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_max / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="u32", data="synthetic",
                config=dict(workload=args.workload, n_jobs=len(jobs), edges_per_step=total,
                            waves=waves, tile_edges=tune["tile_edges"],
                            grid_ctas=tune["grid_ctas"], autotune_cached=tune["cached"],
                            launch="CUDA graph of one persistent kernel per wave",
                            l2=f"no flush: each step writes {total * 8 / 1e9:.1f} GB"),
                per_graph=dict(value=total * world / (ms_pg / 1000.0), unit="edges/s",
                               ms_per_step=ms_pg, launches=len(jobs),
                               speedup_batched=ms_pg / (ms_max / args.steps)),
                roofline=roof, gpu_launches=launches,
                kernels={kk: [v[0], round(v[1], 4)] for kk, v in kernels.items()},
                clocks=clocks)
    if not args.no_e2e:
        # end to end: the batch plus the device-to-host copy of the arena
        out_bytes = total * 8 // waves
        chunk = min(out_bytes, 4 << 30)
        host = torch.empty(chunk, dtype=torch.uint8, pin_memory=True)
        flat = arena.view(torch.uint8).view(-1)
        t0 = time.perf_counter()
        for gph in graphs:
            gph.replay()
            for off in range(0, out_bytes, chunk):
                n = min(chunk, out_bytes - off)
                host[:n].copy_(flat[off:off + n], non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        line["e2e"] = dict(value=total / dt, unit="edges/s", h2d_bytes_per_step=0,
                           d2h_bytes_per_step=total * 8, steps=1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as o
        t_cpu, e_cpu, i = 0.0, 0, 0
        while t_cpu < args.cpu_budget and i < len(jobs):
            j = jobs[(i * 97) % len(jobs)]
            t0 = time.perf_counter()
            if j["kind"] == "pba":
                e_cpu += o.ba(j["n"], j["m"], j["n0"], j["seed"]).shape[0]
            else:
                e_cpu += o.kron(j["initiator"], j["k"], j["n_edges"], j["seed"]).shape[0]
            t_cpu += time.perf_counter() - t0
            i += 1
        line["cpu_baseline"] = dict(value=e_cpu / t_cpu, unit="edges/s", cores=1, kind="oracle",
                                    sample=f"{i} jobs of the batch (every 97th), {t_cpu:.1f} s",
                                    all_cores_estimate=all_cores_estimate(e_cpu / t_cpu))
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


def run_serve(args, rank: int, world: int, local_rank: int):
    """Served workload: a Poisson trace replayed in real time against the
    continuous-batching server, then against a per-graph server (one
    generation call per request, one stream) on the same trace."""
    import numpy as np
    import torch

    from paper_1003_3684_gb300 import build as pbuild
    pbuild.build()
    import paper_1003_3684_gb300 as pg
    from paper_1003_3684_gb300 import serve

    torch.cuda.set_device(local_rank)
    cfg = W.CONFIGS[args.workload]
    duration = args.serve_seconds or cfg["duration"]
    trace = serve.poisson_workload(cfg["rate"], duration, seed=cfg["seed"] + rank)
    warm = serve.poisson_workload(cfg["rate"], 0.5, seed=cfg["seed"] + 1000 + rank)

    def replay(per_graph, arrivals, max_wall=None):
        srv = serve.Server(budget_bytes=cfg["budget"], n_streams=1 if per_graph else 3,
                           max_batch_jobs=1 if per_graph else 256, per_graph=per_graph)
        t0 = time.perf_counter()
        done = serve.run_open_loop(srv, arrivals, max_wall=max_wall)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in done]) * 1000.0
        edges = sum(serve.job_edges(r.job) for r in done)
        if srv.failed:
            raise RuntimeError(f"serving: {len(srv.failed)} request(s) failed: "
                               f"{srv.failed[0].error}")
        return dict(value=edges / wall, unit="edges/s", completed=len(done),
                    offered=len(arrivals), wall_s=wall,
                    p50_ms=float(np.percentile(lat, 50)) if lat.size else None,
                    p99_ms=float(np.percentile(lat, 99)) if lat.size else None,
                    launches=srv.launches, peak_budget_used=srv.peak_in_use)

    replay(False, warm)
    pg.pg_trace_dump()
    pg.pg_trace_enable(True)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    launch0 = pg.pg_launch_count()
    served = replay(False, trace)
    launches = pg.pg_launch_count() - launch0
    clocks = sampler.stop() if sampler else None
    pg.pg_trace_enable(False)
    kernels = pg.pg_trace_dump()
    per_graph = replay(True, trace, max_wall=args.serve_per_graph_wall * duration)
    offered = sum(serve.job_edges(j) for _, j in trace) / duration
    line = dict(metric="edges/sec", value=served["value"], unit="edges/s", n_gpus=world,
                steps=1, warmup=1, ms_per_step=served["wall_s"] * 1000.0, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="u32", data="synthetic",
                config=dict(workload=args.workload, rate_per_s=cfg["rate"], duration_s=duration,
                            requests=len(trace), offered_edges_per_s=offered,
                            budget_bytes=cfg["budget"], csr="kept on device until released",
                            streams=3),
                latency_ms=dict(p50=served["p50_ms"], p99=served["p99_ms"]),
                served=served, per_graph=per_graph,
                gpu_launches=launches,
                kernels={kk: [v[0], round(v[1], 3)] for kk, v in kernels.items()},
                clocks=clocks)
    return line if rank == 0 else None


def run_pgen(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    from paper_1003_3684_gb300 import build as pbuild
    pbuild.build()
    import paper_1003_3684_gb300 as pg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cfg = dict(W.CONFIGS[args.workload])
    if args.blocks and cfg["kind"] == "pba":
        # a smaller case of the same workload: fewer blocks of the same size
        cfg["n"] = cfg["n"] // cfg["blocks"] * args.blocks
        cfg["blocks"] = args.blocks
    seed = replica_seed(cfg["seed"], rank)
    stream = torch.cuda.current_stream()
    kind = cfg["kind"]
    csr_call = None   # (workspace, edges, vertices, flags) of a timed CSR call
    e2e_outs = None   # every buffer a step writes, when more than `out`
    e2e_split = None  # (generate, build the CSR): the edges can leave while the CSR runs

    if kind == "pba":
        n, m, B, n0 = cfg["n"], cfg["m"], cfg["blocks"], cfg["n0"]
        E = pg.pg_pba_edge_count(n, m, B, n0)
        parts = cfg.get("parts", 1)
        out = torch.empty((E // parts if parts > 1 else E, 2), dtype=torch.int32, device=dev)
        ws_bytes = pg.pg_pba_workspace_size(n, m, B)
        ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
        factions = None
        if cfg.get("factions") == "ring3":
            factions = W.ring_factions(B, 3)
            table = torch.from_numpy(pg.pba_faction_table(factions)).to(dev)

        if factions is not None:
            def step():
                pg.gen_pba_factions(n, m, factions, n0=n0, inter_frac=cfg["inter_frac"], seed=seed,
                                    out=out, workspace=ws, table=table)
        elif parts > 1:
            per = B // parts

            def step():
                pg.pg_pba_prepare(n, m, B, n0, cfg["faction_width"], cfg["inter_frac"], seed,
                                  workspace=ws)
                for r in range(parts):
                    pg.gen_pba_blocks(ws, n, m, B, r * per, (r + 1) * per, n0=n0, seed=seed,
                                      out=out)
        else:
            def step():
                pg.gen_pba(n, m, B, n0, cfg["faction_width"], cfg["inter_frac"], seed, out=out,
                           workspace=ws if B > 1 else None)
        units = {"pba_phase1": B * (n // B) * m, "pba_emit": B * (n // B) * m // parts,
                 "ba_chain": n * m}
        work = dict(KERNEL_WORK)
        out_bytes = E * 8
        cfg_json = dict(workload=args.workload + (f" (blocks={B})" if args.blocks else ""),
                        n=n, m=m, blocks=B, n0=n0,
                        faction_width=cfg["faction_width"], inter_frac=cfg["inter_frac"],
                        seed=cfg["seed"], edges_per_step=E, id_width=32,
                        workspace_bytes=ws_bytes)
        if factions is not None:
            cfg_json["factions"] = "ring: block p lists p-1, p, p+1 (mod B)"
        if parts > 1:
            cfg_json["parts"] = (f"{parts} ranges of {B // parts} blocks through one buffer of "
                                 f"{out.numel() * 4 / 1e9:.2f} GB")
    elif kind == "bfs":
        n, m, B, n0 = cfg["n"], cfg["m"], cfg["blocks"], cfg["n0"]
        Ep = pg.pg_pba_edge_count(n, m, B, n0)
        N = B * (n0 + n // B)
        edges = pg.gen_pba(n, m, B, n0, cfg["faction_width"], cfg["inter_frac"], seed)
        row_ptr, col = pg.edges_to_csr_opts(edges, N, pg.CSR_SYMMETRIZE)
        del edges
        torch.cuda.synchronize()
        dist = torch.empty(N, dtype=torch.int32, device=dev)
        bws = torch.empty(pg._analysis_lib().pg_bfs_workspace_size(N), dtype=torch.uint8,
                          device=dev)
        sources = [(i * 2654435761) % N for i in range(cfg["sources"])]
        scanned_per_step = [0]

        def step():
            tot = 0
            for src in sources:
                _, _, sc = pg.bfs(row_ptr, col, src, dist=dist, workspace=bws, undirected=True)
                tot += sc
            scanned_per_step[0] = tot
        step()
        E = scanned_per_step[0]
        units = {"bfs": E / len(sources)}        # one traced launch per search
        work = {"bfs": dict(ops=0, bytes=8)}     # col entry + the distance it tests
        out = dist
        out_bytes = N * 4
        csr_bytes = row_ptr.numel() * 8 + col.numel() * 4
        cfg_json = dict(workload=args.workload, n=n, m=m, blocks=B, n0=n0, vertices=N,
                        csr_entries=2 * Ep, sources=len(sources),
                        metric_note="adjacency entries of the reached vertices (what a "
                                    "top-down search reads) per second over BFS from each "
                                    "source; the CSR is symmetric, so wide levels run "
                                    "bottom-up and read fewer. The roofline counts the "
                                    "top-down reads.", id_width=32)
    elif kind == "kron_det":
        k, P = cfg["k"], cfg["initiator"]
        N = len(P) ** k
        E = pg.pg_kron_edge_count(P, k, 0, deterministic=True)
        out = torch.empty((E, 2), dtype=torch.int32, device=dev)

        def step():
            pg.gen_kronecker(P, k, deterministic=True, out=out)
        units = {"kron_det": E}
        work = {"kron_det": kron_det_work(k)}
        out_bytes = E * 8
        cfg_json = dict(workload=args.workload, initiator="Fig. 2(b) seed: 5 vertices, 11 edges",
                        k=k, vertices=N, edges_per_step=E, order="stack (seed-digit) order",
                        id_width=32)
    elif kind == "kron_xor":
        k, M, Mr = cfg["k"], cfg["n_edges"], cfg["n_random"]
        N = 2**k
        E = M + Mr
        out = torch.empty((E, 2), dtype=torch.int32, device=dev)
        row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
        col = torch.empty(E, dtype=torch.int32, device=dev)
        ws_bytes = pg._opts_lib().pg_csr_opts_workspace_size(E, N, pg.CSR_ODD)
        ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)

        def gen():
            pg.gen_kronecker(cfg["initiator"], k, M, seed, out=out[:M])
            pg.gen_random_cells(N, Mr, seed, out=out[M:])

        def csr():
            pg.edges_to_csr_opts(out, N, pg.CSR_ODD, row_ptr=row_ptr, col=col, workspace=ws)

        def step():
            gen()
            csr()
        csr_call = (ws, E, N, pg.CSR_ODD)
        e2e_outs = [out, row_ptr, col]
        e2e_split = (gen, csr)
        units = {"kron_descent_n0_2": M}
        work = {"kron_descent_n0_2": kron_work(k)}
        units.update({kk: E for kk in CSR_WORK})
        work.update(CSR_WORK)
        out_bytes = E * 8 + (N + 1) * 8 + E * 4
        cfg_json = dict(workload=args.workload, initiator=cfg["initiator"], k=k, n_edges=M,
                        n_random=Mr, seed=cfg["seed"], csr="odd multiplicity (XOR)",
                        edges_per_step=E, id_width=32)
    else:
        k, M = cfg["k"], cfg["n_edges"]
        N = 2**k
        E = M
        out = torch.empty((M, 2), dtype=torch.int32, device=dev)
        row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
        col = torch.empty(M, dtype=torch.int32, device=dev)
        ws_bytes = pg.pg_csr_workspace_size(M, N) if cfg.get("csr") else 0
        ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)

        def gen():
            pg.gen_kronecker(cfg["initiator"], k, M, seed, out=out)

        def csr():
            pg.edges_to_csr(out, N, row_ptr=row_ptr, col=col, workspace=ws)

        def step():
            gen()
            if cfg.get("csr"):
                csr()
        if cfg.get("csr"):
            csr_call = (ws, M, N, 0)
            e2e_outs = [out, row_ptr, col]
            e2e_split = (gen, csr)
        units = {"kron_descent_n0_2": M}
        work = {"kron_descent_n0_2": kron_work(k)}
        if cfg.get("csr"):
            units.update({kk: M for kk in CSR_WORK})
            work.update(CSR_WORK)
        out_bytes = M * 8 + ((N + 1) * 8 + M * 4 if cfg.get("csr") else 0)
        cfg_json = dict(workload=args.workload, initiator=cfg["initiator"], k=k, n_edges=M,
                        seed=cfg["seed"], csr=bool(cfg.get("csr")), edges_per_step=M,
                        id_width=32)
    cfg_json["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    L2_BYTES = 129e6
    flush = None
    if kind == "bfs":
        cfg_json["l2"] = (f"no flush: each search reads the {csr_bytes / 1e9:.2f} GB CSR, more "
                          "than the 129 MB L2")
    elif out_bytes > 2 * L2_BYTES:
        cfg_json["l2"] = (f"no flush: each step writes {out_bytes / 1e9:.2f} GB of output, more "
                          "than the 129 MB L2")
    else:
        flush = torch.empty(int(2 * L2_BYTES), dtype=torch.uint8, device=dev)
        cfg_json["l2"] = (f"flushed: each step ({out_bytes / 1e6:.1f} MB of output) is timed alone "
                          "after a write of a 258 MB buffer")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    pg.pg_trace_dump()              # drop anything recorded so far
    pg.pg_trace_enable(True)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launch0 = pg.pg_launch_count()  # the library's kernel launches from here on
    if flush is None:
        # one event between consecutive steps: the region's time and each step's
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        ms = evs[0].elapsed_time(evs[-1])
        per_step = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    else:
        # each step timed alone, after a write of a buffer twice the L2 size
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        per_step = [a.elapsed_time(b) for a, b in evs]
        ms = sum(per_step)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    pg.pg_trace_enable(False)
    kernels = pg.pg_trace_dump()
    csr_wait = None
    if csr_call is not None:
        # the sort's bounded waits: a nonzero word means the last timed CSR
        # is unspecified, so the run is not a measurement
        csr_wait = pg.csr_wait_error(csr_call[0], csr_call[1], csr_call[2], flags=csr_call[3])
        if csr_wait:
            raise RuntimeError("edges_to_csr: a bounded wait of the sort gave up (PG_ETIMEOUT)")
    ms_max = max_over_ranks(ms, dev, world)
    value = job_throughput(E, args.steps, world, ms_max)
    # every kernel the library launched in the timed steps (the trace above
    # groups some launches under one name, e.g. all phase-1 levels of a step)
    launches = pg.pg_launch_count() - launch0

    # roofline of the dominant kernel
    peaks = load_peaks()
    sms = pg.pg_device_sm_count()
    alu_peak = sms * 128 * peaks["sm_max_mhz"] * 1e6       # int32 lane ops / s
    hbm_peak = peaks["hbm_gbs"] * 1e9
    dom = max((kname for kname in kernels if kname in work), key=lambda x: kernels[x][1],
              default=None)
    roof = None
    if dom:
        nl, tot_ms = kernels[dom]
        per_launch_s = tot_ms / nl / 1000.0
        u = units[dom]
        ops_rate = u * work[dom]["ops"] / per_launch_s
        byte_rate = u * work[dom]["bytes"] / per_launch_s
        t_alu = u * work[dom]["ops"] / alu_peak
        t_hbm = u * work[dom]["bytes"] / hbm_peak
        per_unit = dram_traffic_table().get(dom)
        traffic = per_unit * u if per_unit is not None else None
        if t_alu >= t_hbm:
            roof = dict(bound="alu", kernel=dom, achieved=ops_rate / 1e12, peak=alu_peak / 1e12,
                        unit="Tops/s (int32 lane ops)", frac=ops_rate / alu_peak, traffic=traffic,
                        hbm=dict(achieved=byte_rate / 1e9, peak=peaks["hbm_gbs"], unit="GB/s",
                                 frac=byte_rate / hbm_peak),
                        peak_source=f"{sms} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz")
        else:
            roof = dict(bound="hbm", kernel=dom, achieved=byte_rate / 1e9, peak=peaks["hbm_gbs"],
                        unit="GB/s", frac=byte_rate / hbm_peak, traffic=traffic,
                        peak_source=f"{peaks['source']} MEASURED_PEAKS hbm_gbs")
        if roof["bound"] == "alu":
            # the same fraction against the measured Philox ceiling of this GPU
            rate = pg.philox_rate()
            meas = rate * PHILOX_OPS
            roof["alu_measured"] = dict(philox_per_s=rate, peak=meas / 1e12,
                                        unit="Tops/s (int32 lane ops)", frac=ops_rate / meas,
                                        source="pg_philox_probe: Philox4x32-10 calls/s x 60 ops")
            # per-SM-per-clock rates of the operations Philox is made of
            clk = peaks["sm_max_mhz"] * 1e6
            roof["int_pipes_per_sm_clk"] = {
                k: round(v / sms / clk, 1) for k, v in pg.int_pipe_rates().items()}
        roof["ms_per_launch"] = per_launch_s * 1000.0
        roof["units_per_launch"] = u
        roof["ops_per_unit"] = work[dom]["ops"]
        roof["bytes_per_unit"] = work[dom]["bytes"]
        # whole-step roofline: slower of output bytes at HBM peak and the
        # algorithmic integer work of every kernel at the int32 peak
        step_alu = sum(units[kk] * work[kk]["ops"] for kk in kernels if kk in work) / alu_peak
        step_hbm = out_bytes / hbm_peak
        roof["step_bound_ms"] = 1000.0 * max(step_alu, step_hbm)
        roof["step_frac"] = roof["step_bound_ms"] / (ms_max / args.steps)

    metric, unit = (("traversed_entries/sec", "entries/s") if kind == "bfs"
                    else ("edges/sec", "edges/s"))
    line = dict(metric=metric, value=value, unit=unit, n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=ms_max / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="u32",
                data="synthetic", config=cfg_json, roofline=roof, gpu_launches=launches,
                kernels={kk: [v[0], round(v[1], 4)] for kk, v in kernels.items()},
                clocks=clocks, csr_wait_error=csr_wait,
                step_ms=dict(best=round(min(per_step), 4),
                             median=round(statistics.median(per_step), 4),
                             mean=round(ms / args.steps, 4), rank=0))
    if kind == "pba" and cfg["blocks"] > 1:
        line["paper_context"] = ("PBA 1e9 vertices / 5e9 edges in 12.39 s on 1,000 CPUs "
                                 "(~4.0e8 edges/s): context, other hardware")

    # end to end through the public API with host buffers: the step plus the
    # device-to-host copy of everything it produced into pinned host memory
    if not args.no_e2e and kind != "bfs":
        if kind == "pba" and cfg.get("parts", 1) > 1:
            line["e2e"] = measure_e2e_parts(args, cfg, seed, out, ws, E, dev, world)
        elif kind == "pba" and not cfg.get("factions") and world == 1:
            # one rank: a pinned host buffer of the whole graph, copies
            # overlapped with generation; with several ranks on one host the
            # copies go through a 4 GB pinned buffer per rank instead
            line["e2e"] = measure_e2e_pba(args, cfg, seed, out, ws, E, dev, world)
        else:
            line["e2e"] = measure_e2e(args, step, e2e_outs or [out], cfg, E, dev, world, rank,
                                      split=e2e_split)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, tsec, ns = oracle_sample(args.workload, cfg, args.cpu_budget)
        line["cpu_baseline"] = dict(value=v, unit=unit, cores=1, kind="oracle",
                                    sample=f"{desc}; {ns} samples, {tsec:.1f} s",
                                    all_cores_estimate=all_cores_estimate(v))
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


def measure_e2e_pba(args, cfg, seed, out, ws, E, dev, world):
    """End to end through the public API with a host destination: each step
    is one gen_pba_to_host call (generation with the edge list copied into
    pinned host memory, overlapped) and a stream synchronisation."""
    import torch
    import torch.distributed as dist

    import paper_1003_3684_gb300 as pg
    host = torch.empty(tuple(out.shape), dtype=out.dtype, pin_memory=True)
    B = cfg["blocks"]

    def e2e_step():
        pg.gen_pba_to_host(host, cfg["n"], cfg["m"], B, cfg["n0"], cfg["faction_width"],
                           cfg["inter_frac"], seed, out=out, workspace=ws if B > 1 else None)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    steps = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dt = float(t.item())
    out_bytes = out.numel() * out.element_size()
    return dict(value=E * steps * world / dt, unit="edges/s", h2d_bytes_per_step=0,
                d2h_bytes_per_step=out_bytes, steps=steps,
                host_buffer=f"pinned {out_bytes / 2**30:.1f} GiB; copy overlapped with "
                            "generation (gen_pba_to_host)")


def measure_e2e_parts(args, cfg, seed, out, ws, E, dev, world):
    """End to end for generation in parts: prepare, then each block range into
    the device buffer and on to its place in one pinned host buffer of the
    whole graph (range r+1 is generated while range r is copied)."""
    import torch
    import torch.distributed as dist

    import paper_1003_3684_gb300 as pg
    B, parts = cfg["blocks"], cfg["parts"]
    per = B // parts
    rows = out.shape[0]
    host = torch.empty((rows * parts, 2), dtype=out.dtype, pin_memory=True)
    bufs = [out, torch.empty_like(out)]
    copy = torch.cuda.Stream(device=dev)
    main = torch.cuda.current_stream(dev)
    done = [torch.cuda.Event() for _ in range(2)]

    def e2e_step():
        pg.pg_pba_prepare(cfg["n"], cfg["m"], B, cfg["n0"], cfg["faction_width"],
                          cfg["inter_frac"], seed, workspace=ws)
        for r in range(parts):
            b = bufs[r % 2]
            if r >= 2:
                main.wait_event(done[r % 2])           # buffer free again
            pg.gen_pba_blocks(ws, cfg["n"], cfg["m"], B, r * per, (r + 1) * per, n0=cfg["n0"],
                              seed=seed, out=b)
            ev = torch.cuda.Event()
            ev.record(main)
            copy.wait_event(ev)
            with torch.cuda.stream(copy):
                host[r * rows:(r + 1) * rows].copy_(b, non_blocking=True)
            done[r % 2].record(copy)
        copy.synchronize()
        main.synchronize()

    e2e_step()
    steps = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dt = float(t.item())
    return dict(value=E * steps * world / dt, unit="edges/s", h2d_bytes_per_step=0,
                d2h_bytes_per_step=E * 8, steps=steps,
                host_buffer=f"pinned {E * 8 / 2**30:.1f} GiB; two device buffers of "
                            f"{rows * 8 / 2**30:.1f} GiB, each range copied while the next is made")


def measure_e2e(args, step, outs, cfg, E, dev, world, rank, split=None):
    """End to end through the public calls: the step, then every output
    buffer copied into pinned host memory. With split = (generate, build the
    CSR) and room for the whole output in one pinned buffer, the edge list is
    copied on a second stream while the CSR is built from it (the sort only
    reads the list); row_ptr and col follow the CSR."""
    import torch
    import torch.distributed as dist
    flats = [o.reshape(-1).view(torch.uint8) for o in outs]
    out_bytes = sum(f.numel() for f in flats)
    if split is not None and out_bytes > (16 << 30):
        split = None
    chunk = out_bytes if split is not None else min(out_bytes, 4 << 30)
    host = torch.empty(chunk, dtype=torch.uint8, pin_memory=True)
    h2d = 0
    if cfg["kind"] in ("kron", "kron_det"):
        init = torch.tensor(cfg["initiator"], dtype=torch.float64).pin_memory()
        h2d = init.numel() * 8

    side = torch.cuda.Stream(dev) if split is not None else None
    edges_done = torch.cuda.Event() if split is not None else None

    def e2e_step_split():
        main = torch.cuda.current_stream(dev)
        if h2d:
            init.to(dev, non_blocking=True)
        split[0]()
        edges_done.record(main)
        side.wait_event(edges_done)
        with torch.cuda.stream(side):
            host[:flats[0].numel()].copy_(flats[0], non_blocking=True)
        split[1]()
        pos = flats[0].numel()
        for flat in flats[1:]:
            host[pos:pos + flat.numel()].copy_(flat, non_blocking=True)
            pos += flat.numel()
        main.synchronize()
        side.synchronize()

    def e2e_step():
        if split is not None:
            e2e_step_split()
            return
        if h2d:
            init.to(dev, non_blocking=True)
        step()
        pos = 0
        for flat in flats:
            for off in range(0, flat.numel(), chunk):
                n = min(chunk, flat.numel() - off)
                if pos + n > chunk:
                    pos = 0
                host[pos:pos + n].copy_(flat[off:off + n], non_blocking=True)
                pos += n
        torch.cuda.current_stream().synchronize()

    e2e_step()
    steps = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    dt = time.perf_counter() - t0
    t = torch.tensor([dt], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dt = float(t.item())
    return dict(value=E * steps * world / dt, unit="edges/s", h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=out_bytes, steps=steps,
                host_buffer=f"pinned {chunk / 2**30:.1f} GiB; "
                            + ("edges, row_ptr and col" if len(flats) == 3 else "the output")
                            + (" copied into it, the edges on a second stream while the CSR "
                               "is built" if split is not None else
                               f" copied into it in {(out_bytes + chunk - 1) // chunk} "
                               "chunk(s) per step"))


# The default run's line also carries the metric's other parts, measured in
# the same process after the headline (N = 1 only): Kronecker k = 20 with CSR,
# the 4096-job batch against per-graph launches, and the Poisson serving
# trace against a per-graph server. Each is a shortened run of its workload.
SUB_RECORDS = (
    ("kron", "kron_k20_m16x_csr", dict(steps=20, warmup=3)),
    ("batch", "batch_4096_mixed", dict(steps=3, warmup=1, no_cpu_baseline=True)),
    ("serve", "serve_poisson_2000", dict(serve_seconds=4.0, serve_per_graph_wall=2.0)),
)
SUB_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config", "roofline",
            "per_graph", "served", "latency_ms", "e2e", "step_ms", "kernels", "gpu_launches",
            "clocks", "csr_wait_error")


def run_sub_records(args, local_rank: int) -> dict:
    import torch
    subs = {}
    for key, workload, over in SUB_RECORDS:
        torch.cuda.empty_cache()
        a = argparse.Namespace(**vars(args))
        a.workload, a.blocks, a.batch_jobs = workload, 0, 0
        a.no_cpu_baseline = True
        for k, v in over.items():
            setattr(a, k, v)
        kind = W.CONFIGS[workload]["kind"]
        runner = run_batch if kind == "batch" else run_serve if kind == "serve" else run_pgen
        line = runner(a, 0, 1, local_rank)
        subs[key] = {k: line[k] for k in SUB_KEYS if k in line}
    torch.cuda.empty_cache()
    return subs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pgen", "reference"], default="pgen")
    ap.add_argument("--workload", choices=sorted(W.CONFIGS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload only: leave out the kron/batch/serve sub-records")
    ap.add_argument("--blocks", type=int, default=0,
                    help="PBA only: run this many blocks of the workload's block size "
                         "(a smaller case, e.g. for profiler captures)")
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="serve workload only: seconds of arrivals (default: the workload's)")
    ap.add_argument("--serve-per-graph-wall", type=float, default=3.0,
                    help="serve workload only: the per-graph server stops after this many "
                         "times the arrival window")
    ap.add_argument("--batch-jobs", type=int, default=0,
                    help="batch workload only: use this many of its jobs (a smaller case)")
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    kind = W.CONFIGS[args.workload]["kind"]
    if kind == "batch":
        line = run_batch(args, rank, world, local_rank)
    elif kind == "serve":
        line = run_serve(args, rank, world, local_rank)
    else:
        line = run_pgen(args, rank, world, local_rank)
    if (line is not None and args.workload == DEFAULT_WORKLOAD and world == 1 and
            not args.no_sub and not args.blocks):
        line.update(run_sub_records(args, local_rank))
        line["sub_records"] = ("kron, batch and serve: the metric's other parts, measured after "
                               "the headline in the same process, each with its own clocks")
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
