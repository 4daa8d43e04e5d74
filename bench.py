"""Throughput of the fused wetting-LB step on GB300, in MLUPS and as a fraction
of the HBM roofline.

Workload: the 8192x4096 D2Q9 lattice with 64 drops (R ~ U[40, 120], seed 1) on a
heterogeneous wall (thickness 3 + 1.5 sin(2 pi 8 x / nx)), exponential
pseudo-potential G = -5.5, tau = 1, core 0.1 / tail 0.05 wall potential.
A bench "step" is one LB time step over the whole lattice: one launch of the
fused kernel.  Population buffers (2 x 1.2 GB in FP32) are far larger than L2,
so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage fp32|fp16s|bf16s|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

N > 1 (under torch.distributed.run): independent replicas, one per GPU, no
collective on the data path ("scaling": "weak"); value = all ranks' lattice
updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY = 8192, 4096
WORKLOAD = ("8192x4096 D2Q9 pseudo-potential wetting LB, 64 drops R~U[40,120] seed 1 on a "
            "heterogeneous wall (T(x)=3+1.5 sin(2 pi 8x/nx)), exp psi G=-5.5, tau=1, "
            "core 0.1 / tail 0.05")
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f16", "bf16s": "bf16"}
BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2, "bf16s": 2}
# FP64 storage is bound by the FP64 pipe, not by HBM.  Its roofline counts the
# FP64 flops the step executes per node update (2 x DFMA + DADD + DMUL, ncu on
# 4096x2048; about 2% of them are the recomputed halo psi) against the DFMA
# peak: SMs x 2 DFMA per cycle x 2 flops x SM clock (GB300: 152 x 2 x 2 x
# 2.07 GHz = 1.26 TFLOP/s, its nominal FP64 rate).
FP64_FLOPS_PER_NODE = {9: 288, 21: 514}
FP64_DFMA_PER_SM_CLK = 2


def workload_name(nx: int, ny: int, lattice: int) -> str:
    return WORKLOAD.replace("8192x4096", f"{nx}x{ny}").replace("D2Q9", f"D2Q{lattice}")


KERNEL_SOURCES = ["step_kernel.cuh", "node.cuh", "f2.cuh", "tma.cuh", "lattice.cuh", "launch.cuh",
                  "step_impl.cuh", "engine.cu"]


def kernel_hash() -> str:
    """Hash of the code (comments and blank space removed) of the sources that
    shape the step kernel and its launch: a profile taken on other code no
    longer describes it."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1202_6130_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(storage: str, lattice: int = 9):
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"step_{storage}_d2q{lattice}_8192x4096.txt")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_hash:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != kernel_hash():
        return None
    return float(m_tr.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        # raw samples go to LBM_CLOCKS_DIR (default: the temporary directory)
        out_dir = os.environ.get("LBM_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_identifier(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def dist_max(world: int, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------

class OracleBand:
    """The FP64 oracle on rows [0, rows) of the workload: a periodic band of the
    full 8192-wide lattice with its wall (the sample the CPU legs time)."""

    def __init__(self, rows: int, lattice: int = 9):
        import workloads as W
        from oracle import lbm_oracle as O
        self.O = O
        w = W.large_multi_droplet(with_fields=False)
        T = 3.0 + 1.5 * np.sin(2.0 * np.pi * 8.0 * np.arange(NX) / NX)
        rho = W.droplet_density(NX, rows, w.meta["centers"], w.meta["radii"], 2.0, 0.15, 2.0)
        phi, pr, pa = W.wall_core_tail(W.wall_distance_slab(NX, rows), T[None, :])
        self.p = O.Params(lattice=O.LATTICES[lattice], tau=1.0, G=-5.5)
        self.wall = O.Wall(phi, pr, pa, 0.1, 0.05, 1.0)
        z = np.zeros_like(rho)
        self.f = O.initial_populations(self.p, rho, z, z)
        self.nodes = NX * rows

    def step(self, n: int = 1) -> float:
        """Runs n oracle steps; returns their wall time in seconds."""
        t0 = time.perf_counter()
        for _ in range(n):
            self.f = self.O.step(self.p, self.wall, self.f)
        return time.perf_counter() - t0


def _band_worker(job):
    """One process of the all-cores leg: its own band, stepped for about
    `seconds`; returns (node updates, seconds spent stepping)."""
    rows, lattice, seconds = job
    band = OracleBand(rows, lattice)
    dt1 = band.step(1)
    steps = max(1, int(seconds / max(dt1, 1e-3)))
    return band.nodes * steps, band.step(steps)


def cpu_baseline_all_cores(lattice: int = 9, rows: int = 64, seconds: float = 10.0):
    """The same oracle in one process per host core (spawned, so no process is
    forked from the CUDA one), each on its own band; aggregate node updates
    over the wall time of the stepping."""
    import multiprocessing as mp
    n = max(1, min(64, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_band_worker, [(rows, lattice, seconds)] * n)
    ups = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": ups / wall / 1e6, "unit": "MLUPS", "cores": n, "kind": "oracle",
            "sample": f"{n} processes, each the FP64 numpy oracle (D2Q{lattice}) on rows "
                      f"0..{rows - 1} of the 8192-wide workload as a periodic {NX}x{rows} band, "
                      f"about {seconds:.0f} s of steps"}


def cpu_baseline(target_s: float = 15.0, lattice: int = 9):
    rows = 256
    band = OracleBand(rows, lattice)
    dt1 = band.step(1)
    steps = max(1, int(target_s / max(dt1, 1e-3)))
    dt = band.step(steps)
    out = {"value": band.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"FP64 numpy oracle (D2Q{lattice}), rows 0..{rows - 1} of the 8192-wide "
                     f"workload as a periodic {NX}x{rows} band with its wall, {steps} steps, "
                     "one thread"}
    out["all_cores"] = cpu_baseline_all_cores(lattice)
    return out


def run_reference(args, world, rank):
    """The FP64 oracle as the reference arm: each bench step is one oracle step
    on a periodic 8192-wide band of the workload, sized so that warm-up plus
    timed steps take about two and a half minutes of one host thread."""
    if rank != 0:
        return 0
    budget = 150.0
    total = args.steps + args.warmup
    probe = OracleBand(16, args.lattice)
    probe.step(1)
    per_node = probe.step(2) / (2 * probe.nodes)
    rows = int(max(4, min(512, budget / total / per_node / NX)))
    band = OracleBand(rows, args.lattice)
    band.step(args.warmup)
    dt = band.step(args.steps)
    v = band.nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(NX, NY, args.lattice),
                                        "nx": NX, "ny": NY, "lattice": f"D2Q{args.lattice}",
                                        "sample_rows": rows},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"each step: one oracle step on a periodic {NX}x{rows} band "
                                   "(rows 0.. of the workload, wall included)"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measure_serving(pkg, torch, W, n: int = 300, storage: str = "fp32"):
    """Continuous-batching serving against plain sequential solves, on the
    first n requests of the Poisson stream (seed 3; sizes log-uniform 64x32 ..
    2048x1024, budgets 1k..20k steps, random wall parameters).  Two arrival
    rates: the specified 2000 req/s (a burst: throughput and queueing) and
    10 req/s (about 60% of what the batched loop sustains, so p50/p99 reflect
    service rather than backlog).  Time-to-result runs from a request's
    arrival to its measured result (contact angle or slip length) on the host.
    The stream is capped at n requests: the full minute at 2000 req/s offers
    about 57 times what one GPU can update in that time."""
    from paper_1202_6130_gb300 import serve
    out = {"requests": n, "storage": storage,
           "cap": f"first {n} requests of the seed-3 stream at each rate"}
    for label, rate in (("burst_2000_per_s", 2000.0), ("sustained_10_per_s", 10.0)):
        reqs = serve.requests_from_stream(W.serving_stream(rate=rate, duration=1e9, seed=3,
                                                           max_requests=n))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        srv = serve.Server(storage=storage, hbm_budget=100e9, quantum=500)
        res_b = srv.run(reqs, realtime=True)
        srv.close()
        t_b = time.perf_counter() - t0
        t0 = time.perf_counter()
        res_s = serve.run_sequential(reqs, storage=storage, realtime=True)
        t_s = time.perf_counter() - t0
        b = serve.summarize(res_b, t_b)
        q = serve.summarize(res_s, t_s)
        same = all(x.value == y.value or (x.value != x.value and y.value != y.value)
                   for x, y in zip(sorted(res_b, key=lambda r: r.id), sorted(res_s, key=lambda r: r.id)))
        out[label] = {"rate_per_s": rate, "batched": b, "sequential": q,
                      "throughput_ratio": b["mlups"] / q["mlups"], "results_identical": same}
    return out


def measure_batch(pkg, torch, W, storage: str = "fp16s", steps: int = 200, n: int = 256):
    """The batched parameter sweep: n independent lattices, sizes log-uniform in
    64x32 .. 1024x512 (seed 2), each with its own tau, G, G_R, G_A and a drop or
    a sheared film.  Times `steps` steps run one lattice after another (one
    launch per lattice per step) against the same steps of all lattices in one
    batch (one fused launch per 64-lattice chunk per step, chunks on forked
    streams, 16-step CUDA graphs, autotuned tiles)."""
    ws = W.batch_sweep(n=n, seed=2)
    nodes = sum(w.nx * w.ny for w in ws)
    sims = [pkg.Simulation.from_workload(w, storage=storage) for w in ws]
    for sm in sims:
        sm.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sm in sims:
        sm.step(steps)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    b = pkg.Batch()
    for sm in sims:
        b.add(sm)
    tune = b.autotune(steps_per_trial=32)
    launches = b.launches_per_step()
    b.step(36)  # rebuild with the chosen tiling and capture both step graphs
    b.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(b.stream)
    b.step(steps)
    ev1.record(b.stream)
    b.synchronize()
    t_bat = time.perf_counter() - t0
    t_bat_dev = ev0.elapsed_time(ev1) / 1e3
    finite = all(bool(np.isfinite(sm.moments()[0]).all()) for sm in sims[:8])
    b.close()
    for sm in sims:
        sm.close()
    return {"lattices": n, "nodes": nodes, "steps": steps, "storage": storage,
            "sequential_mlups": nodes * steps / t_seq / 1e6,
            "batched_mlups": nodes * steps / t_bat / 1e6,
            "batched_device_mlups": nodes * steps / t_bat_dev / 1e6,
            "speedup": t_seq / t_bat, "tiling": tune, "finite": finite,
            "gpu_launches_batched": steps * launches}


# Storage and lattice variants the default run measures beside the headline
# (D2Q9 FP32), each with the number of timed steps (about 0.1-0.5 s each).
PER_STORAGE = ((9, "fp16s", 400), (9, "bf16s", 400), (9, "fp64", 20),
               (21, "fp32", 100), (21, "fp16s", 150), (21, "bf16s", 150))


def roofline_of(torch, local, lattice: int, storage: str, N: int, steps: int, t: float,
                clocks: dict) -> dict:
    """Roofline of the fused kernel: algorithmic bytes per node update (2 Q s)
    against the measured HBM copy rate, or for FP64 storage the executed FP64
    flops against the DFMA peak derived from the SM count and clock."""
    traffic = ncu_traffic(storage, lattice)
    if storage == "fp64":
        props = torch.cuda.get_device_properties(local)
        mhz = clocks.get("sm_max_mhz") or 2070.0
        fpeak = props.multi_processor_count * FP64_DFMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12
        fach = FP64_FLOPS_PER_NODE[lattice] * N * steps / t / 1e12
        return {"bound": "alu", "achieved": fach, "peak": fpeak, "unit": "TFLOP/s",
                "frac": fach / fpeak, "traffic": traffic,
                "peak_source": f"derived: {props.multi_processor_count} SMs x "
                               f"{FP64_DFMA_PER_SM_CLK} DFMA/clk x 2 flop x {mhz:.0f} MHz",
                "flops_per_node": FP64_FLOPS_PER_NODE[lattice], "kernel": "lbm::step_kernel"}
    peak, peak_kind = measured_peaks()
    b_node = 2 * lattice * BYTES[storage]
    achieved = b_node * N * steps / t / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs",
            "bytes_per_node": b_node, "kernel": "lbm::step_kernel"}


def measure_per_storage(pkg, torch, W, local: int, nx: int, ny: int, variants=PER_STORAGE):
    """The same workload in the other storage precisions and on D2Q21: for each,
    warm-up launches, then timed launches of the fused step (CUDA events on the
    library's stream, inputs far larger than L2), with the clocks sampled
    around each timed region."""
    N = nx * ny
    out = {}
    base = W.large_multi_droplet(nx=nx, ny=ny, noise_amp=0.0)
    for lattice, storage, steps in variants:
        base.lattice = lattice
        sim = pkg.Simulation.from_workload(base, storage=storage)
        stream = torch.cuda.current_stream()
        sim.step(5)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(gpu_identifier(torch, local)) as clk:
            ev0.record(stream)
            sim.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        sim.sync()
        clocks = clk.summary()
        lay = sim.layout()
        sim.close()
        out[f"d2q{lattice}_{storage}"] = {
            "lattice": f"D2Q{lattice}", "storage": storage, "dtype": DTYPE[storage],
            "steps": steps, "ms_per_step": t / steps * 1e3, "mlups": N * steps / t / 1e6,
            "roofline": roofline_of(torch, local, lattice, storage, N, steps, t, clocks),
            "launch": {k: lay[k] for k in ("tile_rows", "grid_x", "grid_y", "stages")},
            "clocks": clocks}
    return out


def run_gpu(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    import paper_1202_6130_gb300 as pkg
    import workloads as W
    pkg.load()

    nx, ny = (int(v) for v in args.size.lower().split("x"))
    w = W.large_multi_droplet(nx=nx, ny=ny, noise_amp=0.0)
    w.lattice = args.lattice
    sim = pkg.Simulation.from_workload(w, storage=args.storage)
    lay = sim.layout()
    stream = torch.cuda.current_stream()
    N = nx * ny

    sim.step(args.warmup)
    torch.cuda.synchronize()

    # ---- device-resident timed region: K launches of the fused step --------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_identifier(torch, local)) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    t_local = ev0.elapsed_time(ev1) / 1e3
    t = dist_max(world, t_local)
    mlups = world * N * args.steps / t / 1e6
    sim.sync()

    # ---- end to end through the public API with pinned host buffers --------
    lbm_per_e2e = 1000
    n_e2e = max(1, args.steps // lbm_per_e2e)
    rho_h = torch.from_numpy(w.rho).pin_memory().numpy()
    z = torch.zeros((ny, nx), dtype=torch.float64).pin_memory().numpy()
    outs = [torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    sim.set_equilibrium(rho_h, z, z)
    sim.step(10)
    sim.moments(outs)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        sim.set_equilibrium(rho_h, z, z)
        sim.step(lbm_per_e2e)
        sim.moments(outs)
    t_e2e = dist_max(world, time.perf_counter() - t0)
    e2e = world * N * lbm_per_e2e * n_e2e / t_e2e / 1e6
    assert np.isfinite(outs[0]).all()

    # ---- roofline of the fused kernel ----------------------------------------
    clocks = clk.summary()
    roofline = roofline_of(torch, local, args.lattice, args.storage, N, args.steps, t_local,
                           clocks)
    sim.close()
    if rank != 0:
        return 0
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.storage], "data": "synthetic",
        "config": {"workload": workload_name(nx, ny, args.lattice), "nx": nx, "ny": ny,
                   "lattice": f"D2Q{args.lattice}",
                   "storage": args.storage, "parallelism": f"replicas{world}",
                   "l2": "no flush: the 2 population buffers (2x%.2f GB) exceed L2" %
                         (args.lattice * BYTES[args.storage] * N / 1e9),
                   "launch": {k: lay[k] for k in ("strip_width", "tile_rows", "grid_x",
                                                   "grid_y", "stages")}},
        "roofline": roofline,
        "e2e": {"value": e2e, "unit": "MLUPS",
                "h2d_bytes_per_step": 3 * N * 8, "d2h_bytes_per_step": 3 * N * 8,
                "lbm_steps_per_e2e_step": lbm_per_e2e, "e2e_steps": n_e2e,
                "path": "Simulation.set_equilibrium(pinned rho,u) -> step -> moments(pinned)"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if not args.no_per_storage:
        line["per_storage"] = measure_per_storage(pkg, torch, W, local, nx, ny)
    if not args.no_batch:
        line["batch"] = measure_batch(pkg, torch, W)
    if not args.no_serving:
        line["serving"] = measure_serving(pkg, torch, W)
    if not args.no_cpu_baseline and world == 1:   # the host-core baseline is an N = 1 figure
        line["cpu_baseline"] = cpu_baseline(lattice=args.lattice)
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--storage", default="fp32", choices=list(DTYPE))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-storage", action="store_true",
                    help="skip the other storage precisions and D2Q21")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched parameter-sweep measurement")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the continuous-batching serving measurement")
    ap.add_argument("--lattice", type=int, default=9, choices=[9, 21],
                    help="velocity set: D2Q9 (the headline) or D2Q21 on the same drops and wall")
    ap.add_argument("--size", default=f"{NX}x{NY}",
                    help="lattice size NXxNY (the same recipe at another size, for profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
