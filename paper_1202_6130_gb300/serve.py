"""Continuous-batching service for wetting simulations.

Requests (a drop on a wall, or a body-force-driven channel) arrive over time.
The server admits them first-come first-served as long as their device
footprint fits its HBM budget, keeps every admitted lattice resident on the
GPU, and advances all of them together: each step quantum is one batch call
(one fused launch per time step for every active lattice).  Between quanta,
finished requests leave the batch (their result is measured on the host from
the final moments: the static contact angle of a drop, the slip length of a
channel) and waiting requests join it, so requests that arrive while others
are running start as soon as memory frees up.

Per-request arithmetic is the same alone and in the mix: the result of a
request does not depend on what else is in the batch.  Host work (building a
request's fields, measuring a result) runs in worker threads and overlaps the
GPU steps.
"""
from __future__ import annotations

import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import analysis
from .sim import Batch, Simulation

_BYTES = {"fp64": 8, "fp32": 4, "fp16s": 2, "bf16s": 2}


@dataclass
class Request:
    id: int
    t_arrival: float          # seconds after the start of the run
    kind: str                 # "droplet" or "channel"
    nx: int
    ny: int
    steps: int
    G_A: float = 0.05
    G_R: float = 0.1
    tau: float = 1.0
    G: float = -5.5
    epsilon: float = 1.0
    extra: dict = field(default_factory=dict)


@dataclass
class Result:
    id: int
    kind: str
    nx: int
    ny: int
    steps: int
    t_arrival: float
    t_admit: float
    t_done: float
    value: float              # contact angle (degrees) or slip length (lattice units)
    rho: Optional[np.ndarray] = None
    ux: Optional[np.ndarray] = None
    uy: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def footprint_bytes(nx: int, ny: int, storage: str, lattice: int = 9) -> int:
    """Device bytes a resident request needs: two padded population buffers,
    the wall fields (phi^eps, S_x, S_y; optional wall velocity counted) and the
    flag words, plus the FP64 staging of its initialisation and read-out."""
    s = _BYTES[storage]
    r = 1 if lattice == 9 else 3
    gx = ((2 * r * s + 15) // 16) * 16 // s
    pitch = ((nx + 2 * gx + 31) // 32) * 32
    pops = 2 * lattice * pitch * (ny + 4 * r) * s
    t = 8 if storage == "fp64" else 4
    wall = 5 * nx * ny * t + ((nx + 31) // 32 + 3) // 4 * 4 * ny * 4
    staging = (lattice + 3) * nx * ny * 8
    return pops + wall + staging


def default_workload(req: Request):
    """Initial and wall fields of a request, from the seeded synthetic recipes of
    the ``workloads`` module (any callable with this signature can replace it)."""
    import workloads as W
    if req.kind == "droplet":
        R = max(4.0, min(req.nx / 4.0, req.ny / 2.0))
        w = W.droplet_on_wall(nx=req.nx, ny=req.ny, R=R, G_A=req.G_A, G_R=req.G_R, tau=req.tau,
                              G=req.G, noise_amp=0.0, steps=req.steps)
    else:
        w = W.poiseuille_channel(nx=req.nx, ny=req.ny, force=1e-6, G_A=req.G_A, G_R=req.G_R,
                                 tau=req.tau, epsilon=req.epsilon, steps=req.steps)
    w.epsilon = req.epsilon
    return w


def measure(req: Request, w, rho, ux, uy) -> float:
    """Contact angle of a drop or slip length of a channel, from final moments."""
    try:
        if req.kind == "droplet":
            return analysis.contact_angle(rho, w.phi_s, w.meta["rho_l"], w.meta["rho_v"]).theta_deg
        return analysis.slip_length(ux, w.phi_s).slip_length
    except Exception:
        return float("nan")


class Server:
    """FIFO admission by device footprint; one resident batch; step quanta.

    Host work overlaps the GPU.  A request's fields are built by a worker
    thread as soon as it is submitted.  While the batch runs a quantum, the
    main thread creates and initialises the simulations of waiting requests
    that fit the budget, on a side stream (they join the batch at the next
    quantum).  Finished requests are read back after the quantum and measured
    by worker threads; a result's t_done is when its measurement completes."""

    def __init__(self, storage: str = "fp32", hbm_budget: float = 64e9, quantum: int = 500,
                 keep_fields: bool = False, workload: Callable = default_workload,
                 tiling: Optional[tuple] = None, host_workers: int = 4):
        import torch
        self.storage = storage
        self.budget = float(hbm_budget)
        self.quantum = int(quantum)
        self.keep_fields = keep_fields
        self.workload = workload
        self.batch = Batch()
        # tiling: (tile_rows, ctas), or None for the tiling an earlier autotune
        # chose for the batch's current size class, when there is one
        self.tiling = tiling
        if tiling is not None:
            self.batch.set_tiling(*tiling)
        self.side = torch.cuda.Stream()
        self.pool = ThreadPoolExecutor(max_workers=max(1, int(host_workers)))
        self.queue: deque = deque()
        self.fields: dict = {}      # id -> future of the request's workload
        self.staged: list = []      # [req, sim, workload, t_admit, bytes], not yet in the batch
        self.active: dict = {}      # id -> [req, sim, workload, steps_left, t_admit, bytes]
        self.measuring: list = []   # futures of Results
        self.used = 0.0
        self.results: list = []
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        if footprint_bytes(req.nx, req.ny, self.storage) > self.budget:
            raise ValueError(f"request {req.id} needs more than the whole HBM budget")
        self.queue.append(req)
        self.fields[req.id] = self.pool.submit(self.workload, req)

    def _stage(self):
        """Creates, on the side stream, the simulations of the waiting requests
        that fit the budget (strict FIFO: the first that does not fit waits).
        Only requests whose fields are ready are taken, except that an idle
        GPU waits for the first one."""
        import torch
        while self.queue:
            req = self.queue[0]
            need = footprint_bytes(req.nx, req.ny, self.storage)
            if self.used + need > self.budget:
                break
            fut = self.fields[req.id]
            if not fut.done() and (self.active or self.staged):
                break
            self.queue.popleft()
            w = self.fields.pop(req.id).result()
            with torch.cuda.stream(self.side):
                sim = Simulation.from_workload(w, storage=self.storage, stream=self.side)
            self.staged.append([req, sim, w, self.now(), need])
            self.used += need

    def _join(self):
        for req, sim, w, t_admit, need in self.staged:
            self.batch.add(sim)
            self.active[req.id] = [req, sim, w, req.steps, t_admit, need]
        self.staged.clear()

    def _finish(self, req, w, t_admit, rho, ux, uy) -> Result:
        res = Result(req.id, req.kind, req.nx, req.ny, req.steps, req.t_arrival, t_admit, 0.0,
                     measure(req, w, rho, ux, uy))
        if self.keep_fields:
            res.rho, res.ux, res.uy = rho, ux, uy
        res.t_done = self.now()
        return res

    def _retire(self):
        done = [k for k, v in self.active.items() if v[3] <= 0]
        for k in done:
            req, sim, w, _, t_admit, need = self.active.pop(k)
            self.batch.remove(sim)
            rho, ux, uy = sim.moments()
            sim.close()
            self.used -= need
            self.measuring.append(self.pool.submit(self._finish, req, w, t_admit, rho, ux, uy))

    def _collect(self, wait: bool = False):
        pending = []
        for f in self.measuring:
            if wait or f.done():
                self.results.append(f.result())
            else:
                pending.append(f)
        self.measuring = pending

    def tick(self) -> bool:
        """Joins the staged simulations, launches one quantum (or up to the
        nearest finish), stages waiting requests while it runs, retires.
        Returns False when nothing is active, staged or waiting."""
        self._join()
        if not self.active:
            self._stage()
            self._join()
            if not self.active:
                self._collect()
                return bool(self.queue)
        q = min(self.quantum, min(v[3] for v in self.active.values()))
        if self.tiling is None:
            self.batch.use_tuned()
        self.batch.step(q)
        self._stage()
        self._collect()
        for v in self.active.values():
            v[3] -= q
        self._retire()
        return bool(self.active or self.staged or self.queue)

    def run(self, requests, realtime: bool = True):
        """Serves `requests` (sorted by arrival).  With realtime, a request is
        released when the wall clock passes its arrival time; otherwise all are
        released at once."""
        pending = deque(sorted(requests, key=lambda r: r.t_arrival))
        self.t0 = time.perf_counter()
        while pending or self.queue or self.active or self.staged:
            t = self.now()
            while pending and (not realtime or pending[0].t_arrival <= t):
                self.submit(pending.popleft())
            if not self.active and not self.queue and not self.staged and pending:
                time.sleep(max(0.0, min(0.01, pending[0].t_arrival - t)))
                continue
            self.tick()
        self._collect(wait=True)
        return self.results

    def close(self):
        for v in self.active.values():
            v[1].close()
        for v in self.staged:
            v[1].close()
        self.active.clear()
        self.staged.clear()
        self._collect(wait=True)
        self.pool.shutdown(wait=True)
        self.batch.close()


def run_sequential(requests, storage: str = "fp32", workload: Callable = default_workload,
                   realtime: bool = True, keep_fields: bool = False):
    """Plain solves, one request at a time in arrival order (the comparison for
    the batched server)."""
    out = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.t_arrival):
        if realtime:
            wait = req.t_arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        t_admit = time.perf_counter() - t0
        w = workload(req)
        sim = Simulation.from_workload(w, storage=storage)
        sim.step(req.steps)
        rho, ux, uy = sim.moments()
        res = Result(req.id, req.kind, req.nx, req.ny, req.steps, req.t_arrival, t_admit,
                     time.perf_counter() - t0, measure(req, w, rho, ux, uy))
        if keep_fields:
            res.rho, res.ux, res.uy = rho, ux, uy
        sim.close()
        out.append(res)
    return out


def summarize(results, wall_time: float) -> dict:
    lat = np.array([r.latency for r in results])
    lups = sum(r.nx * r.ny * r.steps for r in results)
    return {"requests": len(results), "wall_s": wall_time,
            "mlups": lups / wall_time / 1e6 if wall_time > 0 else float("nan"),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else float("nan"),
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else float("nan"),
            "mean_s": float(lat.mean()) if len(lat) else float("nan")}


def requests_from_stream(stream) -> list:
    """Request objects from the dicts of ``workloads.serving_stream``."""
    return [Request(id=d["id"], t_arrival=d["t_arrival"], kind=d["kind"], nx=d["nx"],
                    ny=d["ny"], steps=d["steps"], G_A=d["G_A"], G_R=d["G_R"]) for d in stream]
