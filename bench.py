"""Benchmark: solve time to relative residual 1e-6, FP32-preconditioned vs all-FP64 form.

Timed workload (default ``grf4096``): n = 4096 (4097^2 nodes), k = 1000 (kh = 0.244), smooth
random medium k (1 + 0.3 g) with g a seeded Gaussian random field of correlation length 0.05,
a centre point source of 1/h^2, hybrid (HYB-V) hierarchy of 10 levels, Bi-CGSTAB to relres 1e-6.
A step is one complete solve (every kernel of the hot path) with the inputs resident in HBM; the
library rewrites every Krylov vector from the right-hand side, so no state carries over between
solves. The problem's arrays (3.6 GB) are far larger than L2 (129 MB); L2 is also flushed (a 512 MB
write, untimed) before each timed solve.

Beside the headline: the FP64 form of the same solve, the solve through host buffers (``e2e``),
the per-kernel roofline of one profiled iteration (CUDA events on the library's stream inside
the solve's graph), the measured FP64 FMA rate (the ceiling of the FP64 Krylov kernels), the
batched form (64 right-hand sides over 4 grids) and a prefix of the served Poisson stream, and
for every workload the error of each form's solution against the FP64 oracle (test
infrastructure, run on the host beside the GPU work; the n = 4096 oracle solve takes hours, so
its solution is read from the sampled copy that tests/golden/make_grf4096_oracle.py wrote).

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead: each step is one
whole Bi-CGSTAB iteration of the same workload, and the solve time is that per-iteration time
times the oracle's own iteration count. Multi-GPU (torchrun): every rank solves its own replica
(weak scaling, no collective on the data path); times are the max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1312_2880_gb300 import inputs as I  # noqa: E402

GOLDEN_GRF4096 = os.path.join(ROOT, "tests", "golden", "grf_n4096_k1000_oracle.json")


# Algorithmic (compulsory) HBM bytes per finest-grid node of one launch of each kernel. FP32 form:
# the V-cycle reads and writes FP32 (complex 8 B, k h 4 B) on every level including the finest,
# the FP64 Krylov kernels (complex 16 B, k h 8 B) write the FP32 copies of p and s and read the
# FP32 preconditioned vectors y, z (8 B). FP64 form: 16/8 B throughout. A colour half-sweep
# touches half the nodes for its own row data but all nodes of the other colour.
def kernel_bytes_per_node(kernel: str, fp32: bool) -> float:
    c, r = (8, 4) if fp32 else (16, 8)
    y = 8 if fp32 else 16  # preconditioned vector as the Krylov kernels read it
    w = 8 if fp32 else 0  # FP32 copy of p or s written for the V-cycle
    table = {
        "smooth_restrict": c + r + c + c / 4,      # f, k h; write u and the coarse f
        "prolong_smooth": c + c / 4 + c + r + c,   # u_pre, coarse e, f, k h; write the result
        "gs_first": c / 2 + r / 2 + c,
        "gs_colour": (c + c + r + c) / 2,
        "kacz_colour": (5 * c * 2 + c + r) / 5,
        "kacz_sweep": c + c + r + c,               # u in, f, k h; u out
        "restrict_residual": c + c + r + c / 4,
        "prolong_add": 2 * c + c / 4,
        "export": 2 * c,
        "k_update_p": 64 + w,
        "k_apply_rv": y + 8 + 16 + 16,
        "k_update_s": 48 + w,
        "k_apply_ts": y + 8 + 16 + 16,
        "k_update_r": 16 + 16 + 16 + 16,           # s, t, r^; write r
        "k_update_x": y + 32,                      # y or z; x in and out (one half of the update)
    }
    return table.get(kernel, 0.0)


# FP64 work per node of the Krylov kernels: (flops with an FMA counted 2, FP64-pipe instructions).
# The operator on an interior node: 3 complex adds (6), d = (kh)^2 - 4 (1 FMA), v = nb + d y (2 FMA).
KRYLOV_FP64 = {"k_update_p": (16, 8), "k_apply_rv": (20, 13), "k_update_s": (12, 6), "k_apply_ts": (24, 15),
               "k_update_r": (20, 10), "k_update_x": (8, 4)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

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
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload(name: str):
    if name == "grf4096":
        return I.grf_n4096()
    if name == "wedge512":
        return I.wedge_n512()
    if name == "plain64":
        return I.plain_n64()
    if name.startswith("grf"):
        n = int(name[3:])
        return I.grf_n4096(n=n, k=1000.0 * n / 4096)
    raise ValueError(name)


def dist_setup(n_gpus: int, backend: str = "nccl"):
    """Rank, world size and local GPU from the torchrun environment. One process per GPU; the
    process group only carries the barriers and the max over ranks of the timings (each rank
    solves its own replica). backend="gloo" runs the same path on host cores (no GPU)."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend, rank=rank, world_size=world)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier_max(value: float, world: int) -> float:
    """The maximum of `value` over all ranks, after a barrier (the slowest replica's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], device=dev, dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_fields(world: int, ms: float) -> dict:
    """Whole-job figures of N replicas (weak scaling): every rank completes one solve per step, so
    the job completes `world` solves in the slowest rank's time `ms`."""
    return {"n_gpus": world, "solves_per_s": round(world * 1e3 / ms, 3),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def l2_flush_buffer():
    """A device buffer larger than L2 (129 MB); writing it evicts every line of the solve."""
    import torch

    return torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")


def time_solves(P, rhs, steps: int, warmup: int, world: int, tol: float, maxit: int):
    """Each step: flush L2 (untimed), then one solve bracketed by CUDA events on the caller's
    stream. Returns per-step ms, their sum and the solve infos."""
    import torch

    flush = l2_flush_buffer()
    for _ in range(warmup):
        P.solve(rhs, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    x = None
    for s in range(steps):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        x, info, _ = P.solve(rhs, tol=tol, maxit=maxit)
        ev[s][1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per = [a.elapsed_time(b) for a, b in ev]
    return per, sum(per), infos, x


def time_e2e(P, rhs_host, steps: int, tol: float, maxit: int):
    """The same solve through the host-buffer entry point: the right-hand side is copied in from
    pinned host memory and the solution out to pinned host memory inside every timed call."""
    import torch

    pinned_in = torch.empty(rhs_host.shape, dtype=torch.complex128, pin_memory=True)
    pinned_in.numpy()[...] = rhs_host
    rhs_host = pinned_in.numpy()
    out = torch.empty(rhs_host.shape, dtype=torch.complex128, pin_memory=True).numpy()
    P.solve_host(rhs_host, tol=tol, maxit=maxit, out=out)
    torch.cuda.synchronize()
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        P.solve_host(rhs_host, tol=tol, maxit=maxit, out=out)
        t.append((time.perf_counter() - t0) * 1e3)
    return t, out


def profile(P, rhs, iterations: int = 2):
    """{(kernel, level): [ms per launch]} over `iterations` Bi-CGSTAB iterations captured in one
    CUDA graph with an event node after every kernel (hz_profile_graph): each kernel as it runs
    inside a solve's graph replay, timed with CUDA events on the library's stream."""
    per = {}
    for name, level, ms in P.profile_iteration(rhs, iterations=iterations, graph=True):
        per.setdefault((name, level), []).append(ms)
    return per


def roofline(per, fp32: bool, hbm_peak: float, peak_kind: str, n: int, fp64_peak: dict | None):
    """The dominant kernel (largest total time) of a profile and its achieved rate: an FP64 Krylov
    kernel against the measured FP64 FMA rate, a V-cycle kernel against the measured HBM copy
    rate; the HBM fraction is given beside the FP64 one. An FP64 kernel's rate is its FP64-pipe
    issue rate in FMA-equivalents (every DFMA, DADD or DMUL takes one pipe slot and counts 2
    flops, as the probe's DFMA chains do), its algorithmic flops (an add counted 1) beside."""
    total = sum(sum(v) for v in per.values())
    (name, level), times = max(per.items(), key=lambda kv: sum(kv[1]))
    avg_ms = sum(times) / len(times)
    nodes = ((n >> level) + 1) ** 2
    gbs = kernel_bytes_per_node(name, fp32) * nodes / (avg_ms * 1e-3) / 1e9
    if name.startswith("k_") and fp64_peak:
        flops, instr = KRYLOV_FP64[name]
        secs = avg_ms * 1e-3
        achieved = 2 * instr * nodes / secs / 1e12
        peak = fp64_peak["tflops"]
        roof = {"kernel": name, "level": level, "bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": "measured: hz_measure_fp64_rate in this run (DFMA chains on every SM, CUDA events); "
                               "FMA = 2 flops",
                "achieved_is": "FP64-pipe issue rate in FMA-equivalents (each DFMA, DADD or DMUL one pipe slot = 2 flops)",
                "fp64_instructions_per_node": instr, "algorithmic_flops_per_node": flops,
                "algorithmic_tflops": round(flops * nodes / secs / 1e12, 4), "nodes": nodes,
                "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4), "hbm_peak": hbm_peak}
    else:
        roof = {"kernel": name, "level": level, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(gbs / hbm_peak, 4), "peak_source": peak_kind,
                "bytes_per_node": kernel_bytes_per_node(name, fp32), "nodes": nodes}
    roof.update({"traffic": None, "avg_launch_ms": round(avg_ms, 5), "launches": len(times),
                 "share": round(sum(times) / total, 4)})
    return roof


def sweep_rates(per, fp32: bool, hbm_peak: float, n: int):
    """Achieved HBM GB/s (algorithmic bytes / device time) of each V-cycle kernel on the levels
    larger than L2 (n_l >= 2048), and of the Kaczmarz sweeps (L2-resident levels, for reference)."""
    out = {}
    for (name, level), times in per.items():
        nl = n >> level
        if name.startswith("k_") or kernel_bytes_per_node(name, fp32) == 0:
            continue
        if nl < 2048 and not name.startswith("kacz"):
            continue
        avg = sum(times) / len(times)
        gbs = kernel_bytes_per_node(name, fp32) * (nl + 1) ** 2 / (avg * 1e-3) / 1e9
        out[f"{name}@L{level}"] = {"n_l": nl, "gbs": round(gbs, 1), "frac": round(gbs / hbm_peak, 4),
                                   "ms": round(avg, 4), "launches_per_iteration": len(times) // 2}
    return out


def pass_forms(P):
    """Fused-pass forms the tile autotuner picked: {"L<l> n=<n_l>": [pre, post]} per fused level."""
    return {f"L{l} n={d['n']}": [d["pass_down"], d["pass_up"]] for l, d in enumerate(P.schedule())
            if d["pass_down"] >= 0}


def source_digest():
    """SHA-256 of the CUDA sources and headers the kernels are built from."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1312_2880_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, level: int, workload_name: str):
    """DRAM bytes (read + write) per launch of `kernel` on `level` from a committed ncu summary
    under profiles/ (lines "traffic: <kernel>@L<level> <workload> <bytes> sources=<digest>"), or
    None when no summary covers it or the kernel sources have changed since it was taken."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    digest = source_digest()
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(pdir, name)):
            parts = line.strip().strip("`").split()
            if len(parts) == 5 and parts[0] == "traffic:" and parts[1] == f"{kernel}@L{level}" \
                    and parts[2] == workload_name and parts[4] == f"sources={digest}":
                return int(parts[3])
    return None


def shares(per, top: int = 12):
    total = sum(sum(v) for v in per.values())
    rows = sorted(per.items(), key=lambda kv: -sum(kv[1]))[:top]
    return {f"{k[0]}@L{k[1]}": round(sum(v) / total, 4) for k, v in rows}


# --------------------------------------------------------------------------- oracle side (host)
# The oracle is test infrastructure: the benchmark runs it only to state each form's error against
# it and to time the CPU baseline, in worker processes started with "spawn" beside the GPU work.


def oracle_job(spec):
    """One oracle task in a worker process. ("solve", kind, key): the oracle's own solve to relres
    1e-6 of a workload (kind plain64 / wedge512 / batch (problem index, rhs index) / serve (request
    id, stream length, rate)), returning its solution and iteration count. ("sample", workload,
    iterations): the time of that many whole Bi-CGSTAB iterations of the workload (after an
    untimed setup)."""
    import oracle as o

    kind = spec[0]
    if kind == "sample":
        wl = workload(spec[1])
        t0 = time.perf_counter()
        A = o.helmholtz_matrix(wl.n, wl.kfield)
        H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
        setup = time.perf_counter() - t0
        b = wl.rhs.ravel()
        t0 = time.perf_counter()
        o.bicgstab(A, b, lambda v: o.vcycle(H, v), tol=1e-300, maxit=spec[2])
        dt = time.perf_counter() - t0
        return {"per_iter_ms": dt * 1e3 / spec[2], "iterations": spec[2], "setup_s": setup}
    wl = oracle_workload(spec[1], spec[2])
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    res = o.bicgstab(A, wl.rhs.ravel(), lambda v: o.vcycle(H, v), tol=wl.tol, maxit=5000)
    return {"x": res.x, "iterations": res.iterations, "status": res.status, "true_relres": res.true_relres}


def oracle_workload(kind: str, key):
    """The single-right-hand-side workload behind an oracle task (same inputs the GPU side solves)."""
    if kind in ("plain64", "wedge512"):
        return workload(kind)
    if kind == "batch":
        wl = I.batch_problems(rhs_per_k=16)[key[0]]
        return I.Workload(wl.name, wl.n, wl.k_ref, wl.kfield, wl.rhs[key[1]], variant=wl.variant, levels=wl.levels)
    if kind == "serve":
        rid, count, rate = key
        req = I.serving_requests(count, rate)[rid]
        return I.Workload(f"request{rid}", req.n, req.k, I.request_medium(req), I.point_source_rhs(req.n, [req.source]))
    raise ValueError(kind)


def oracle_batch_solve(key):
    """One oracle solve of right-hand side `q` of batched grid `pi` (key = (pi, q)); returns its
    wall time in seconds (worker process)."""
    t0 = time.perf_counter()
    oracle_job(("solve", "batch", key))
    return time.perf_counter() - t0


def allcore_batched_baseline(grids=(0, 1), per_grid: int = 16):
    """The oracle on every host core: the right-hand sides of the batched workload's two smaller
    grids (n = 96, 192) solved by one process per core (spawned), against the same solves on one
    core (their summed single-process times). The oracle's own solve is single-threaded (scipy's
    sparse products hold the GIL), so independent solves are how it uses more cores."""
    import concurrent.futures
    import multiprocessing

    keys = [(pi, q) for pi in grids for q in range(per_grid)]
    cores = os.cpu_count() or 1
    with concurrent.futures.ProcessPoolExecutor(max_workers=cores,
                                                mp_context=multiprocessing.get_context("spawn")) as pool:
        list(pool.map(oracle_batch_solve, [(0, 0)] * cores))  # start every worker (imports)
        t0 = time.perf_counter()
        per = list(pool.map(oracle_batch_solve, keys))
        wall = time.perf_counter() - t0
    return {"kind": "oracle", "cores": cores, "solves": len(keys), "wall_s": round(wall, 2),
            "solves_per_s": round(len(keys) / wall, 3), "one_core_solves_per_s": round(len(keys) / sum(per), 3),
            "sample": f"right-hand sides 0..{per_grid - 1} of the batched grids n = "
                      f"{', '.join(str(I.BATCH_SPECS[g][1]) for g in grids)}, one process per core"}


def rel_err(x, ref) -> float:
    x = np.asarray(x).ravel()
    ref = np.asarray(ref).ravel()
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def grf4096_sampled_errors(xs: dict):
    """max over the sampled nodes of |x - x_oracle| / max |x_oracle| of each form's n = 4096 solution,
    against the oracle's solve stored by tests/golden/make_grf4096_oracle.py (None if absent)."""
    if not os.path.exists(GOLDEN_GRF4096):
        return None
    g = json.load(open(GOLDEN_GRF4096))
    s = np.array(g["sampled"])
    i, j = s[:, 0].astype(int), s[:, 1].astype(int)
    ref = s[:, 2] + 1j * s[:, 3]
    out = {f"{p}_form": float(np.abs(x[j, i] - ref).max() / g["max_abs_x"]) for p, x in xs.items()}
    out.update({"oracle_iterations": g["iterations"], "oracle_true_relres": g["true_relres"],
                "sampled_nodes": int(len(ref)),
                "sample": "every 128th node in each direction plus the 9 x 9 nodes around the source"})
    return out


def serve_sample_ids(count: int, rate: float, sizes=(128, 256, 512), per_size: int = 1):
    """Request ids of the served prefix whose solutions are checked against the oracle: the first
    `per_size` requests of each listed grid size (the oracle's solves of larger grids take minutes)."""
    reqs = I.serving_requests(count, rate)
    out = []
    for n in sizes:
        out += [q.rid for q in reqs if q.n == n][:per_size]
    return out


# --------------------------------------------------------------------------- batched and served forms


def run_batched(precision: str, reps: int = 3, keep=()):
    """Four constant-k problems (k, n) = (50, 96), (100, 192), (200, 384), (300, 576), 16 seeded
    point sources each, solved as one group (every right-hand side of every problem advances in
    the same graph launch per iteration; finished ones retire). Returns timing, counts and the
    solutions of the (problem, rhs) pairs listed in `keep`."""
    import torch

    from paper_1312_2880_gb300 import hz

    wls = I.batch_problems(rhs_per_k=16)
    probs = [hz.Problem(w.n, w.kfield, 0.5, variant=w.variant, precision=precision, k_ref=w.k_ref,
                        batch=w.rhs.shape[0]) for w in wls]
    rhs = [torch.from_numpy(w.rhs).cuda() for w in wls]
    G = hz.Group(probs)
    G.solve(rhs, tol=1e-6, maxit=3000, allow_fail=True)  # warm-up (graph capture)
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        xs, infos = G.solve(rhs, tol=1e-6, maxit=3000, allow_fail=True)
        t.append((time.perf_counter() - t0) * 1e3)
    kept = {(pi, q): xs[pi][q].cpu().numpy() for pi, q in keep}
    its = [i["iterations"] for i in infos]
    conv = sum(1 for i in infos if i["status"] == 0)
    G.close()
    for P in probs:
        P.close()
    ms = statistics.median(t)
    return {"ms": round(ms, 2), "rhs": len(infos), "converged": conv, "iterations_min": min(its),
            "iterations_max": max(its), "solves_per_s": round(len(infos) * 1e3 / ms, 1)}, kept


def run_serving(precision: str, count: int, rate: float, keep=()):
    """The first `count` requests of the served Poisson stream (200 requests/s, n uniform over
    {128, ..., 2048}, kh = 2 pi / 12, wedge or random-field media, one seeded source each) through
    the continuous-batching server. Media are generated before the clock starts."""
    import torch

    from paper_1312_2880_gb300.serve import Job, Server

    reqs = I.serving_requests(count, rate)
    media = {}
    jobs = []
    for q in reqs:
        key = (q.n, q.medium, q.medium_seed)
        if key not in media:
            media[key] = I.request_medium(q)
        jobs.append(Job(q.rid, q.n, key, (lambda key=key: media[key]), q.k, q.source, arrival=q.arrival_s))
    free = torch.cuda.mem_get_info()[0]
    srv = Server(hbm_budget=int(free * 0.6), precision=precision, max_active=32, maxit=4000, keep_solutions=set(keep))
    summ = srv.run(jobs, realtime=True)
    kept = {j.rid: j.result["x"] for j in srv.done if "x" in j.result}
    its = [j.result.get("iterations", 0.0) for j in srv.done]
    srv.close()
    service = sum((j.end - j.start) for j in srv.done)
    waits = [(j.start - j.arrival) * 1e3 for j in srv.done]
    last_arrival = reqs[-1].arrival_s if reqs else 0.0
    summ.update({"rate_hz": rate, "requests": count, "iterations_max": max(its) if its else None,
                 "mean_concurrency": round(service / max(summ["wall_s"], 1e-9), 2),
                 "admission_wait_p50_ms": round(float(np.percentile(waits, 50)), 2) if waits else None,
                 "last_arrival_s": round(last_arrival, 3),
                 # arrivals outpace service: latency is then mostly time spent queued
                 "queue_bound": bool(summ["wall_s"] > 1.5 * last_arrival + 0.05)})
    return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in summ.items()}, kept


# --------------------------------------------------------------------------- the GPU arm


def small_solves(names=("plain64", "wedge512"), tol: float = 1e-6):
    """Both forms' solutions of the small workloads (for their error against the oracle)."""
    import torch

    from paper_1312_2880_gb300 import hz

    out = {}
    for name in names:
        wl = workload(name)
        rhs = torch.from_numpy(wl.rhs).cuda()
        for prec in ("fp32", "fp64"):
            P = hz.Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=prec, levels=wl.levels, k_ref=wl.k_ref)
            x, info, _ = P.solve(rhs, tol=tol, maxit=4000)
            out[(name, prec)] = (x.cpu().numpy(), info["iterations"])
            P.close()
    return out


def start_oracle_pool(args, serve_ids):
    """Worker processes (spawn) for the oracle tasks, submitted before any GPU work."""
    import concurrent.futures
    import multiprocessing

    pool = concurrent.futures.ProcessPoolExecutor(max_workers=args.oracle_workers,
                                                  mp_context=multiprocessing.get_context("spawn"))
    fut = {"sample": pool.submit(oracle_job, ("sample", args.workload, args.cpu_sample_iters))}
    for name in ("plain64", "wedge512"):
        fut[name] = pool.submit(oracle_job, ("solve", name, None))
    if not args.skip_forms:
        for pi in range(4):
            fut[("batch", pi, 0)] = pool.submit(oracle_job, ("solve", "batch", (pi, 0)))
        for rid in serve_ids:
            fut[("serve", rid)] = pool.submit(oracle_job, ("solve", "serve", (rid, args.serve_requests, args.serve_rate)))
    return pool, fut


def run_ours(args):
    import torch

    from paper_1312_2880_gb300 import build, hz

    world, rank, local = dist_setup(args.gpus)
    with_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    serve_ids = serve_sample_ids(args.serve_requests, args.serve_rate) if not args.skip_forms else []
    pool, fut = start_oracle_pool(args, serve_ids) if with_oracle else (None, {})
    build.build()
    wl = workload(args.workload)
    tol = 1e-6
    rhs = torch.from_numpy(wl.rhs).cuda()
    hbm_peak, peak_kind = load_peaks()
    fp64_peak = hz.measure_fp64_rate()
    results, probs = {}, {}
    for prec in ("fp32", "fp64"):
        P = hz.Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision=prec, levels=wl.levels, k_ref=wl.k_ref)
        steps = args.steps if prec == "fp32" else max(1, min(args.steps, args.fp64_steps))
        warm = args.warmup if prec == "fp32" else max(1, min(args.warmup, args.fp64_warmup))
        with ClockSampler(local) as clk:
            per, total, infos, x = time_solves(P, rhs, steps, warm, world, tol, args.maxit)
        results[prec] = {"ms": barrier_max(total / steps, world), "per_step_ms": [round(v, 3) for v in per],
                         "steps": steps, "warmup": warm, "iterations": infos[-1]["iterations"],
                         "relres_true": infos[-1]["relres_true"], "status": infos[-1]["status"],
                         "restarts": infos[-1]["restarts"], "clocks": clk.summary(), "forms": pass_forms(P),
                         "x": x.cpu().numpy()}
        probs[prec] = P
    P32 = probs["fp32"]
    e2e_t, _ = time_e2e(P32, wl.rhs, max(1, min(args.steps, 3)), tol, args.maxit)
    e2e_ms = barrier_max(statistics.mean(e2e_t), world)
    per32 = profile(P32, rhs, 2)
    per64 = profile(probs["fp64"], rhs, 2)
    launches_per_iter = sum(len(v) for v in per32.values()) // 2 + 1  # + the loop-control kernel
    for P in probs.values():
        P.close()
    roof = roofline(per32, True, hbm_peak, peak_kind, wl.n, fp64_peak)
    roof["workload"] = wl.name
    roof["traffic"] = profiled_traffic(roof["kernel"], roof["level"], wl.name)
    it32 = results["fp32"]["iterations"]
    gpu_launches = int(args.steps * (math.ceil(it32) * launches_per_iter + 4))
    batched = serving = None
    kept_b, kept_s = {}, {}
    if not args.skip_forms:
        keep_b = [(pi, 0) for pi in range(4)]
        b32, kb32 = run_batched("fp32", keep=keep_b)
        b64, kb64 = run_batched("fp64", keep=keep_b)
        batched = {"fp32_form": b32, "fp64_form": b64}
        kept_b = {"fp32": kb32, "fp64": kb64}
        s32, ks32 = run_serving("fp32", args.serve_requests, args.serve_rate, keep=serve_ids)
        s64, ks64 = run_serving("fp64", args.serve_requests, args.serve_rate, keep=serve_ids)
        serving = {"fp32_form": s32, "fp64_form": s64,
                   "stream": f"the first {args.serve_requests} requests of the 2000-request stream "
                             f"(Poisson, {args.serve_rate:g}/s, n in 128..2048, kh = 2 pi / 12)"}
        kept_s = {"fp32": ks32, "fp64": ks64}
    small = small_solves() if with_oracle else {}
    replica = replica_fields(world, results["fp32"]["ms"])
    line = headline_line(args, wl, results, replica, e2e_ms, roof, per32, per64, hbm_peak, fp64_peak, gpu_launches,
                         batched, serving)
    if with_oracle:
        line.update(oracle_fields(args, wl, results, fut, small, kept_b, kept_s, serve_ids))
        pool.shutdown()
        if not args.skip_forms:
            line["cpu_baseline"]["all_cores_batched"] = allcore_batched_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def headline_line(args, wl, results, replica, e2e_ms, roof, per32, per64, hbm_peak, fp64_peak, gpu_launches,
                  batched, serving):
    r32, r64 = results["fp32"], results["fp64"]
    nbytes = 16 * (wl.n + 1) ** 2
    return {
        "metric": "solve time to relres 1e-6 (FP32-preconditioned form; FP64 form beside it)",
        "value": round(r32["ms"], 3),
        "unit": "ms",
        "n_gpus": replica["n_gpus"],
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(r32["ms"], 3),
        "per_step_ms": r32["per_step_ms"],
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64 V-cycle / c128 Krylov",
        "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "k": wl.k_ref, "medium": wl.meta.get("medium", ""),
                   "levels": wl.levels, "variant": wl.variant, "tol": wl.tol, "rhs": wl.meta.get("rhs", ""),
                   "l2": "inputs (3.6 GB of arrays) larger than L2, and L2 flushed before every timed solve (512 MB write)",
                   "parallelism": replica["parallelism"]},
        "iterations": r32["iterations"],
        "relres_true": r32["relres_true"],
        "status": r32["status"],
        "solves_per_s": replica["solves_per_s"],
        "fp64_form": {"ms": round(r64["ms"], 3), "per_step_ms": r64["per_step_ms"], "steps": r64["steps"],
                      "warmup": r64["warmup"], "iterations": r64["iterations"], "relres_true": r64["relres_true"],
                      "status": r64["status"], "speedup_of_fp32_form": round(r64["ms"] / r32["ms"], 3),
                      "iteration_ms": round(r64["ms"] / max(r64["iterations"], 1), 4),
                      "kernel_share": shares(per64, 8), "clocks": r64["clocks"]},
        "iteration_ms": round(r32["ms"] / max(r32["iterations"], 1), 4),
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "host_buffers": "pinned"},
        "batched": batched,
        "serving": serving,
        "roofline": roof,
        "fp64_peak": {"tflops": round(fp64_peak["tflops"], 4), "probe_ms": round(fp64_peak["ms"], 3),
                      "fmas_per_chain": fp64_peak["iters"]},
        "sweep_hbm": {"workload": wl.name, "kernels": sweep_rates(per32, True, hbm_peak, wl.n),
                      "iteration_ms_profiled": round(sum(sum(v) for v in per32.values()) / 2, 3)},
        "kernel_share": shares(per32),
        "gpu_launches": gpu_launches,
        "tile_autotuner": {"fp32_form": r32["forms"], "fp64_form": r64["forms"],
                           "forms": "0 = shared-memory tiles; v = 1..8: register streaming, 2^v rows per warp"},
        "clocks": r32["clocks"],
    }


def oracle_fields(args, wl, results, fut, small, kept_b, kept_s, serve_ids):
    """error_vs_oracle for every workload and the CPU baseline, from the oracle tasks."""
    err = {wl.name: grf4096_sampled_errors({p: r["x"] for p, r in results.items()})
           if wl.name == "grf_n4096_k1000" else None}
    for name, label in (("plain64", "plain_n64_k20"), ("wedge512", "wedge_n512_k100")):
        ref = fut[name].result()
        err[label] = {f"{p}_form": rel_err(small[(name, p)][0], ref["x"]) for p in ("fp32", "fp64")}
        err[label].update({"oracle_iterations": ref["iterations"],
                           "gpu_iterations": {p: small[(name, p)][1] for p in ("fp32", "fp64")}})
    if kept_b:
        per = {}
        for pi in range(4):
            ref = fut[("batch", pi, 0)].result()
            per[f"n={I.BATCH_SPECS[pi][1]},rhs0"] = {f"{p}_form": rel_err(kept_b[p][(pi, 0)], ref["x"])
                                                     for p in ("fp32", "fp64")}
        err["batched"] = {"max": {f"{p}_form": max(v[f"{p}_form"] for v in per.values()) for p in ("fp32", "fp64")},
                          "cases": per, "sample": "right-hand side 0 of each of the 4 grids"}
    if kept_s:
        per = {}
        for rid in serve_ids:
            ref = fut[("serve", rid)].result()
            per[f"request{rid}"] = {f"{p}_form": (rel_err(kept_s[p][rid], ref["x"]) if rid in kept_s[p] else None)
                                    for p in ("fp32", "fp64")}
        err["served"] = {"cases": per, "sample": "the first request of each of n = 128, 256, 512 in the served prefix"}
    samp = fut["sample"].result()
    g_iters = json.load(open(GOLDEN_GRF4096))["iterations"] if (os.path.exists(GOLDEN_GRF4096) and
                                                                  wl.name == "grf_n4096_k1000") else None
    iters_full = g_iters if g_iters is not None else results["fp64"]["iterations"]
    cpu = {"value": round(samp["per_iter_ms"] * iters_full, 1), "unit": "ms", "cores": 1, "kind": "oracle",
           "sample": f"{samp['iterations']} whole Bi-CGSTAB iterations of the same {wl.name} solve "
                     f"({samp['per_iter_ms']:.0f} ms each, numpy/scipy on one host core; scipy's sparse products "
                     f"hold the GIL, so the oracle uses one core), times the "
                     f"{'oracle' if g_iters is not None else 'FP64 form'}'s {iters_full:g} iterations; "
                     f"untimed setup {samp['setup_s']:.0f} s"}
    return {"error_vs_oracle": err, "cpu_baseline": cpu}


# --------------------------------------------------------------------------- reference arm (the oracle)


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: untimed setup, then `warmup` and `steps` steps of one
    whole Bi-CGSTAB iteration each (o.bicgstab with maxit = 1, from x0 = 0); the solve time is the
    mean step time times the oracle's own iteration count (from its stored solve of the n = 4096
    workload, or from one full solve for the smaller workloads)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as o

    wl = workload(args.workload)
    A = o.helmholtz_matrix(wl.n, wl.kfield)
    H = o.build_hierarchy(wl.n, wl.kfield, wl.k_ref, wl.variant, wl.levels)
    b = wl.rhs.ravel()
    K = lambda v: o.vcycle(H, v)  # noqa: E731
    if wl.name == "grf_n4096_k1000" and os.path.exists(GOLDEN_GRF4096):
        iters_full, source = json.load(open(GOLDEN_GRF4096))["iterations"], "its stored solve"
    else:
        iters_full, source = o.bicgstab(A, b, K, tol=1e-6, maxit=5000).iterations, "one full solve in this run"
    for _ in range(args.warmup):
        o.bicgstab(A, b, K, tol=1e-300, maxit=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.bicgstab(A, b, K, tol=1e-300, maxit=1)
        times.append((time.perf_counter() - t0) * 1e3)
    per_iter = statistics.mean(times)
    value = per_iter * iters_full
    line = {
        "impl": "reference",
        "metric": "solve time to relres 1e-6 (FP32-preconditioned form; FP64 form beside it)",
        "value": round(value, 1), "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per_iter, 1), "value_is": "per-step time x the oracle's iterations to relres 1e-6",
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "k": wl.k_ref, "levels": wl.levels, "variant": wl.variant},
        "iterations": iters_full,
        "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"each step one whole Bi-CGSTAB iteration of the n={wl.n} solve ({per_iter:.0f} ms, "
                                   f"numpy/scipy on one host core), times the oracle's {iters_full:g} iterations to "
                                   f"relres 1e-6 ({source})"},
        "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """One iteration of a workload launched kernel by kernel (for ncu), in the form --profile-precision."""
    import torch

    from paper_1312_2880_gb300 import build, hz

    torch.cuda.set_device(0)
    build.build()
    rw = workload(args.profile_case)
    P = hz.Problem(rw.n, rw.kfield, 0.5, variant=rw.variant, precision=args.profile_precision, levels=rw.levels,
                   k_ref=rw.k_ref, pass_variant=args.pass_variant)
    recs = P.profile_iteration(torch.from_numpy(rw.rhs).cuda(), iterations=1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": rw.name, "launches": len(recs)}))
    P.close()


def run_sweep(args):
    """The fused passes and Kaczmarz sweeps of the FP32 form on a larger grid of the same medium and
    kh (n = --sweep-n; k scaled with n): per-kernel HBM rates from two profiled iterations, as the
    bench line's sweep_hbm, on arrays four or more times the size of config 3's."""
    import torch

    from paper_1312_2880_gb300 import build, hz

    torch.cuda.set_device(0)
    build.build()
    hbm_peak, peak_kind = load_peaks()
    n = args.sweep_n
    wl = I.grf_n4096(n=n, k=1000.0 * n / 4096)
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant=wl.variant, precision="fp32", levels=wl.levels, k_ref=wl.k_ref)
    per = profile(P, torch.from_numpy(wl.rhs).cuda())
    torch.cuda.synchronize()
    print(json.dumps({"sweep_workload": wl.name, "n": n, "hbm_peak": hbm_peak, "peak_source": peak_kind,
                      "sweep_hbm": sweep_rates(per, True, hbm_peak, n), "kernel_share": shares(per),
                      "tile_autotuner": pass_forms(P)}), flush=True)
    P.close()


def run_serving_only(args):
    """The served stream alone (both forms, or --serve-precision): a long run of the config."""
    import torch

    from paper_1312_2880_gb300 import build

    torch.cuda.set_device(0)
    build.build()
    out = {}
    for prec in args.serve_precision.split(","):
        with ClockSampler(0) as clk:
            summ, _ = run_serving(prec, args.serve_requests, args.serve_rate)
        summ["clocks"] = clk.summary()
        out[f"{prec}_form"] = summ
    print(json.dumps({"serving": out, "requests": args.serve_requests, "rate_hz": args.serve_rate}), flush=True)


def run_tables(args):
    """Sec. 6, Tables 1, 2 and 6 re-run on the GPU: Bi-CGSTAB iterations to relres 1e-7 for HYB-V,
    SL-V and HLM-V (no ray correction), and HYB-V with damped Jacobi (omega 0.8) or red-black SOR
    (omega 1.2) on its Gauss-Seidel levels, FP64 and FP32 V-cycle forms; one JSON line per run and a
    summary line with the paper's counts beside ours (context: the paper leaves the boundary
    scheme, smoother ordering and shadow residual unstated, so only trends are comparable)."""
    import torch

    from paper_1312_2880_gb300 import build, hz

    torch.cuda.set_device(0)
    build.build()
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_iterations.json")))
    summary = {}
    runs = [(v, "gs", 0.0) for v in ("hyb", "sl", "hlm")] + [("hyb", "jacobi", 0.0), ("hyb", "sor", 1.2)]
    for variant, smoother, omega in runs:
        tables = ("table1", "table2", "table6") if smoother == "gs" else ("table1", "table2")
        for table, col, wl in I.paper_table_workloads(tables, variant=variant, max_n=args.tables_max_n):
            rhs = torch.from_numpy(wl.rhs).cuda()
            for prec in ("fp64", "fp32"):
                P = hz.Problem(wl.n, wl.kfield, 0.5, variant=variant, precision=prec, k_ref=wl.k_ref,
                               gs_smoother=smoother, omega=omega)
                try:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, info, _ = P.solve(rhs, tol=wl.tol, maxit=args.tables_maxit, allow_fail=True)
                    torch.cuda.synchronize()
                    ms = (time.perf_counter() - t0) * 1e3
                finally:
                    P.close()
                it = info["iterations"] if info["status"] == 0 else None
                name = variant if smoother == "gs" else f"{variant}+{smoother}"
                print(json.dumps({"table": table, "column": col, "variant": name, "precision": prec,
                                  "n": wl.n, "iterations": it, "status": info["status"],
                                  "relres_true": info["relres_true"], "ms": round(ms, 2)}), flush=True)
                summary.setdefault(f"{table} {name} {prec}", []).append(it)
    paper = {}
    for table in ("table1", "table2", "table6"):
        for variant in ("sl", "hyb"):
            paper[f"{table} {variant}"] = golden[table][variant]
    print(json.dumps({"tables": summary, "paper": paper, "tol": 1e-7, "maxit": args.tables_maxit}), flush=True)


def run_table7(args):
    """Sec. 6, Table 7 on the GPU: V-cycle plus ray correction as a stand-alone solver (relres 1e-7,
    kh = 0.3125, centre source) for HLM-V, SL-V and HYB-V, FP64 and FP32 V-cycle forms (the ray
    correction is FP64 in both). One JSON line per run with the cycle count beside the stored
    oracle's and the paper's, the solve time, the ray set-up time and one V-cycle and one ray
    correction timed alone (CUDA events on the library's stream, 20 launches after 3 untimed)."""
    import torch

    from paper_1312_2880_gb300 import build, hz

    torch.cuda.set_device(0)
    build.build()
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "table7_oracle.json")))
    summary = {}
    for ci, (col, wl) in enumerate(I.paper_table7_workloads(max_n=args.tables_max_n)):
        rhs = torch.from_numpy(wl.rhs).cuda()
        for variant in ("hlm", "sl", "hyb"):
            for prec in ("fp64", "fp32"):
                P = hz.Problem(wl.n, wl.kfield, 0.5, variant=variant, precision=prec, k_ref=wl.k_ref)
                R = hz.Ray(P, wl.k_ref)
                try:
                    P.cycle_solve(rhs, R, tol=wl.tol, maxc=60, allow_fail=True)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    xg, info, _ = P.cycle_solve(rhs, R, tol=wl.tol, maxc=60, allow_fail=True)
                    torch.cuda.synchronize()
                    ms = (time.perf_counter() - t0) * 1e3
                    smp = np.array(golden["oracle"][variant][ci]["sampled"])
                    xs = xg.cpu().numpy()[smp[:, 1].astype(int), smp[:, 0].astype(int)]
                    x_err = float(np.abs(xs - (smp[:, 2] + 1j * smp[:, 3])).max()
                                  / golden["oracle"][variant][ci]["max_abs_x"])
                    r = torch.randn(wl.n + 1, wl.n + 1, dtype=torch.complex128, device="cuda")
                    x = torch.zeros_like(r)
                    split = {}
                    g = R.restrict(r)
                    for name, fn in (("vcycle_ms", lambda: P.vcycle(r)), ("ray_correction_ms", lambda: R.correct(r, x)),
                                     ("ray_restrict_ms", lambda: R.restrict(r)), ("ray_solve_ms", lambda: R.coarse_solve(g))):
                        for _ in range(3):
                            fn()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        for _ in range(20):
                            fn()
                        e1.record()
                        torch.cuda.synchronize()
                        split[name] = round(e0.elapsed_time(e1) / 20, 4)
                finally:
                    setup_ms, m, unknowns = R.setup_ms, R.m, R.unknowns
                    R.close()
                    P.close()
                cyc = info["cycles"] if info["status"] == 0 else None
                ref = golden["oracle"][variant][ci]
                print(json.dumps({"table": "table7", "column": col, "variant": variant, "precision": prec, "n": wl.n,
                                  "ray_m": m, "ray_unknowns": unknowns, "cycles": cyc, "status": info["status"],
                                  "oracle_cycles": ref["cycles"], "paper_cycles": golden["paper"][variant][ci],
                                  "relres_true": info["relres_true"], "error_vs_oracle": x_err,
                                  "solve_ms": round(ms, 2),
                                  "ms_per_cycle": round(ms / max(1, info["cycles"]), 3), **split,
                                  "ray_setup_ms": round(setup_ms, 1)}), flush=True)
                summary.setdefault(f"{variant} {prec}", []).append(cyc)
    print(json.dumps({"table7": summary, "oracle": {v: [c["cycles"] for c in golden["oracle"][v]] for v in golden["oracle"]},
                      "paper": golden["paper"], "tol": golden["tol"]}), flush=True)


def run_ray_profile(args):
    """One Table 7 column (k = RAY_PROFILE, HLM-V, FP32 V-cycle): ray set-up, then three ray
    corrections of a seeded residual, each timed with CUDA events (the launches an ncu launch list
    of this command sees after the set-up)."""
    import torch

    from paper_1312_2880_gb300 import build, hz

    torch.cuda.set_device(0)
    build.build()
    wl = next(w for c, w in I.paper_table7_workloads() if c == f"k={args.ray_profile:g}")
    P = hz.Problem(wl.n, wl.kfield, 0.5, variant="hlm", precision="fp32", k_ref=wl.k_ref)
    R = hz.Ray(P, wl.k_ref)
    g = torch.Generator().manual_seed(I.SEED_BASE + 7)
    r = torch.randn(wl.n + 1, wl.n + 1, dtype=torch.complex128, generator=g).cuda()
    x = torch.zeros_like(r)
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R.correct(r, x)
        e1.record()
        torch.cuda.synchronize()
        ms.append(round(e0.elapsed_time(e1), 4))
    print(json.dumps({"ray_profile": f"table7_n{wl.n}_k{wl.k_ref:g}", "m": R.m, "unknowns": R.unknowns,
                      "setup_ms": round(R.setup_ms, 1), "correction_ms": ms}), flush=True)
    R.close()
    P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--fp64-warmup", type=int, default=2)
    ap.add_argument("--maxit", type=int, default=4000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grf4096")
    ap.add_argument("--cpu-sample-iters", type=int, default=2)
    ap.add_argument("--oracle-workers", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip every oracle task (baseline and errors)")
    ap.add_argument("--profile-case", default=None, help="run one profiled iteration of this workload and exit")
    ap.add_argument("--skip-forms", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-only", action="store_true", help="run only the served stream and exit")
    ap.add_argument("--serve-precision", default="fp32,fp64")
    ap.add_argument("--profile-precision", default="fp32")
    ap.add_argument("--pass-variant", type=int, default=-1,
                    help="fused-pass form for --profile-case (-1: tile autotuner; 0: tiles; 1..8: streaming)")
    ap.add_argument("--tables", action="store_true", help="re-run the paper's Tables 1, 2 and 6 and exit")
    ap.add_argument("--table7", action="store_true",
                    help="re-run the paper's Table 7 (V-cycle plus ray correction as a solver) and exit")
    ap.add_argument("--ray-profile", type=float, default=0.0,
                    help="set up the ray correction of one Table 7 column (its k) and time three corrections")
    ap.add_argument("--tables-maxit", type=int, default=400)
    ap.add_argument("--tables-max-n", type=int, default=1024)
    ap.add_argument("--sweep-n", type=int, default=0,
                    help="time the V-cycle passes of the FP32 form on an n = SWEEP_N grid of the same medium and exit")
    args = ap.parse_args()
    if args.tables:
        run_tables(args)
    elif args.table7:
        run_table7(args)
    elif args.ray_profile:
        run_ray_profile(args)
    elif args.sweep_n:
        run_sweep(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.serve_only:
        run_serving_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
