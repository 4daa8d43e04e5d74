"""Seeded synthetic inputs for the pseudo-potential wetting model.

This module holds NO arithmetic of the lattice-Boltzmann method itself: it only
draws random numbers and builds the static input fields that the method takes
as given (initial density, initial velocity, population noise, and the wall
fields phi_S, psi_R-bar, psi_A-bar of Sec. II "Fluid-Solid interactions").
Both the CUDA library and the FP64 oracle consume these arrays as data.

The paper evaluates the wall fields with the recursive filter of its Appendix;
the synthetic workloads here instead use a closed-form core/tail profile
(repulsive core of range lambda, attractive tail decaying as r^-3 to a cutoff,
tanh wall probability), which the Appendix explicitly allows ("any integrable
function with a finite value in the solid bulk and null value within the fluid
bulk").  The paper's own filter is part of the method and lives in the library
(``lbm_wall_gaussian_filter``) and, separately, in the oracle.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here from its
published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "splitmix64", "uniform", "droplet_density", "wall_distance_slab",
    "wall_core_tail", "Workload", "droplet_on_wall", "poiseuille_channel",
    "large_multi_droplet", "batch_sweep", "serving_stream",
]

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs (uint64) for a 64-bit seed."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + k * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """n doubles uniform in [lo, hi): the top 53 bits of SplitMix64 scaled."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def droplet_density(nx: int, ny: int, centers, radii, rho_l: float, rho_v: float,
                    width: float) -> np.ndarray:
    """Initial density [ny, nx]: union (max) of tanh-profiled discs.

    rho = rho_v + (rho_l - rho_v) * 0.5 * (1 - tanh(2 (r - R) / width)), with r
    the plain Euclidean distance to the centre (the disc is not wrapped).
    """
    rho = np.full((ny, nx), rho_v, dtype=np.float64)
    # Each cap is evaluated inside its bounding box grown by 12 widths: farther
    # out (rho_l - rho_v)(1 - tanh)/2 < 2e-21, which cannot change rho_v in FP64,
    # so the result is identical to evaluating every cap everywhere.
    margin = 12.0 * width + 1.0
    for (cx, cy), R in zip(centers, radii):
        x0 = max(0, int(math.floor(cx - R - margin)))
        x1 = min(nx, int(math.ceil(cx + R + margin)) + 1)
        y0 = max(0, int(math.floor(cy - R - margin)))
        y1 = min(ny, int(math.ceil(cy + R + margin)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        y, x = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
        cap = rho_v + (rho_l - rho_v) * 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width))
        rho[y0:y1, x0:x1] = np.maximum(rho[y0:y1, x0:x1], cap)
    return rho


def wall_distance_slab(nx: int, ny: int) -> np.ndarray:
    """Periodic distance to the solid row y = 0: d = min(y, ny - y), shape [ny, nx].

    With fully periodic streaming, a wall 'at y = 0' and walls 'at the top and
    bottom' of a channel are the same solid slab across the periodic seam.
    """
    y = np.arange(ny, dtype=np.float64)
    d = np.minimum(y, ny - y)
    return np.repeat(d[:, None], nx, axis=1)


def wall_core_tail(dist: np.ndarray, thickness, core_lambda: float = 1.0,
                   core_cut: float = 4.0, tail_exp: float = 3.0,
                   tail_cut: float = 4.0, phi_cut: float = 1e-16):
    """Closed-form wall fields from a distance-to-solid map.

    phi_S = 0.5 (1 - tanh((d - T/2) / (T/4)))      (tanh profile, T thick)
    psi_R = exp(-d/lambda) - exp(-r_c/lambda)      for d < r_c, else 0
    psi_A = (1+d)^-p - (1+r_c)^-p                   for d < r_c, else 0
    phi_S values below ``phi_cut`` are set to exactly 0 so that the wall
    region is finite (the tanh tail otherwise never reaches 0).
    ``thickness`` is a scalar or an array broadcastable to ``dist``.
    """
    d = np.asarray(dist, dtype=np.float64)
    T = np.broadcast_to(np.asarray(thickness, dtype=np.float64), d.shape)
    phi = 0.5 * (1.0 - np.tanh((d - 0.5 * T) / (0.25 * T)))
    phi = np.where(phi < phi_cut, 0.0, phi)
    psi_r = np.where(d < core_cut, np.exp(-d / core_lambda) - math.exp(-core_cut / core_lambda), 0.0)
    psi_a = np.where(d < tail_cut, (1.0 + d) ** (-tail_exp) - (1.0 + tail_cut) ** (-tail_exp), 0.0)
    return phi, psi_r, psi_a


@dataclass
class Workload:
    """One simulation input: parameters plus initial and wall fields (FP64)."""
    name: str
    nx: int
    ny: int
    lattice: int = 9
    tau: float = 1.0
    G: float = -5.5
    rho0: float = 1.0
    psi_kind: int = 0            # 0: exponential psi, 1: piecewise-linear EOS
    G_R: float = 0.1
    G_A: float = 0.05
    epsilon: float = 1.0
    body_force: tuple = (0.0, 0.0)
    rho: Optional[np.ndarray] = None        # [ny, nx]
    ux: Optional[np.ndarray] = None
    uy: Optional[np.ndarray] = None
    noise: Optional[np.ndarray] = None      # [Q, ny, nx] added to f^eq
    phi_s: Optional[np.ndarray] = None
    psi_r: Optional[np.ndarray] = None
    psi_a: Optional[np.ndarray] = None
    u_wall: Optional[np.ndarray] = None     # [2, ny, nx] or None
    steps: int = 1000
    meta: dict = field(default_factory=dict)


def _noise(seed: int, q: int, ny: int, nx: int, amp: float) -> np.ndarray:
    return uniform(seed, q * ny * nx, -amp, amp).reshape(q, ny, nx)


def droplet_on_wall(nx: int = 128, ny: int = 64, R: float = 20.0, G_A: float = 0.05,
                    G_R: float = 0.1, seed: int = 0, noise_amp: float = 1e-6,
                    steps: int = 1000, lattice: int = 9, tau: float = 1.0,
                    G: float = -5.5, rho_l: float = 2.0, rho_v: float = 0.15,
                    thickness: float = 3.0, name: str = "droplet") -> Workload:
    """Semicircular drop centred on the wall row (nx/2, 0): the 128x64 FP64
    parity case and, at 1024x512 / R = 160, the contact-angle sweep case."""
    rho = droplet_density(nx, ny, [(nx / 2.0, 0.0)], [R], rho_l, rho_v, 2.0)
    phi, pr, pa = wall_core_tail(wall_distance_slab(nx, ny), thickness)
    z = np.zeros((ny, nx))
    return Workload(name=name, nx=nx, ny=ny, lattice=lattice, tau=tau, G=G,
                    G_R=G_R, G_A=G_A, rho=rho, ux=z.copy(), uy=z.copy(),
                    noise=_noise(seed, lattice, ny, nx, noise_amp) if noise_amp else None,
                    phi_s=phi, psi_r=pr, psi_a=pa, steps=steps,
                    meta=dict(R=R, rho_l=rho_l, rho_v=rho_v, seed=seed))


def poiseuille_channel(nx: int = 1024, ny: int = 256, force: float = 1e-6,
                       rho_l: float = 2.0, G_A: float = 0.05, G_R: float = 0.1,
                       tau: float = 1.0, epsilon: float = 1.0, steps: int = 1000,
                       thickness: float = 3.0, lattice: int = 9,
                       name: str = "channel") -> Workload:
    """Liquid-filled channel; the solid slab sits across the periodic y seam
    (walls at the top and bottom), driven by a uniform force density."""
    phi, pr, pa = wall_core_tail(wall_distance_slab(nx, ny), thickness)
    rho = np.full((ny, nx), rho_l)
    z = np.zeros((ny, nx))
    return Workload(name=name, nx=nx, ny=ny, lattice=lattice, tau=tau, G_R=G_R,
                    G_A=G_A, epsilon=epsilon, body_force=(force, 0.0), rho=rho,
                    ux=z.copy(), uy=z.copy(), phi_s=phi, psi_r=pr, psi_a=pa,
                    steps=steps, meta=dict(rho_l=rho_l, force=force))


def large_multi_droplet(nx: int = 8192, ny: int = 4096, n_drops: int = 64,
                        seed: int = 1, rho_l: float = 2.0, rho_v: float = 0.15,
                        noise_amp: float = 0.0, steps: int = 20000,
                        with_fields: bool = True) -> Workload:
    """64 drops, R ~ U[40, 120] (seed 1), centres x_k = (k + 1/2) nx / 64 on
    the wall row; the caps overlap and are merged by max.  The substrate is
    heterogeneous: wall thickness T(x) = 3 + 1.5 sin(2 pi 8 x / nx)."""
    radii = uniform(seed, n_drops, 40.0, 120.0)
    centers = [((k + 0.5) * nx / n_drops, 0.0) for k in range(n_drops)]
    T = 3.0 + 1.5 * np.sin(2.0 * np.pi * 8.0 * np.arange(nx) / nx)
    w = Workload(name="multi_droplet", nx=nx, ny=ny, steps=steps,
                 meta=dict(radii=radii, centers=centers, rho_l=rho_l, rho_v=rho_v))
    if with_fields:
        w.rho = droplet_density(nx, ny, centers, radii, rho_l, rho_v, 2.0)
        w.ux = np.zeros((ny, nx))
        w.uy = np.zeros((ny, nx))
        w.phi_s, w.psi_r, w.psi_a = wall_core_tail(wall_distance_slab(nx, ny), T[None, :])
        if noise_amp:
            w.noise = _noise(seed, 9, ny, nx, noise_amp)
    return w


def batch_sweep(n: int = 256, seed: int = 2, smin: float = 64.0, smax: float = 1024.0,
                steps: int = 10000, with_fields: bool = True):
    """Independent lattices, sizes log-uniform in [smin, smax] (ny = nx/2),
    tau ~ U[0.6, 1.5], G ~ U[-6, -5], G_R, G_A ~ U[0, 0.15]; half drops, half
    sheared films (top wall moving at U_wall = (0.01, 0))."""
    r = uniform(seed, 7 * n, 0.0, 1.0).reshape(n, 7)
    out = []
    for k in range(n):
        s = math.exp(math.log(smin) + (math.log(smax) - math.log(smin)) * r[k, 0])
        nx = max(8, int(round(s)))
        ny = max(8, int(round(s / 2)))
        tau = 0.6 + 0.9 * r[k, 1]
        G = -6.0 + 1.0 * r[k, 2]
        G_R = 0.15 * r[k, 3]
        G_A = 0.15 * r[k, 4]
        film = r[k, 5] < 0.5
        w = Workload(name=f"batch{k}", nx=nx, ny=ny, tau=tau, G=G, G_R=G_R,
                     G_A=G_A, steps=steps, meta=dict(film=bool(film)))
        if with_fields:
            phi, pr, pa = wall_core_tail(wall_distance_slab(nx, ny), 3.0)
            if film:
                # liquid film of height ny/4 on the bottom wall
                y = np.arange(ny, dtype=np.float64)[:, None]
                prof = 0.15 + (2.0 - 0.15) * 0.5 * (1.0 - np.tanh(2.0 * (y - ny / 4.0) / 2.0))
                w.rho = np.repeat(prof, nx, axis=1)
                uw = np.zeros((2, ny, nx))
                # the slab row band nearer the top of the domain moves
                yy = np.arange(ny)
                top = yy >= ny // 2
                uw[0, top, :] = 0.01
                w.u_wall = uw
            else:
                R = ny / 3.0
                w.rho = droplet_density(nx, ny, [(nx / 2.0, 0.0)], [R], 2.0, 0.15, 2.0)
            w.ux = np.zeros((ny, nx))
            w.uy = np.zeros((ny, nx))
            w.phi_s, w.psi_r, w.psi_a = phi, pr, pa
        out.append(w)
    return out


def serving_stream(rate: float = 2000.0, duration: float = 60.0, seed: int = 3,
                   smin: float = 64.0, smax: float = 2048.0, kmin: int = 1000,
                   kmax: int = 20000, max_requests: Optional[int] = None):
    """Poisson arrivals (exponential gaps) of droplet / channel requests with
    log-uniform sizes and uniform step budgets.  Returns a list of dicts with
    arrival time, kind, nx, ny, steps and wall parameters (fields are built
    lazily by the caller with ``droplet_on_wall`` / ``poiseuille_channel``)."""
    n_est = int(rate * duration * 1.5) + 16
    if max_requests is not None:
        n_est = min(n_est, max_requests)
    u = uniform(seed, 6 * n_est, 0.0, 1.0).reshape(n_est, 6)
    t = 0.0
    reqs = []
    for k in range(n_est):
        t += -math.log(1.0 - u[k, 0]) / rate
        if t > duration:
            break
        s = math.exp(math.log(smin) + (math.log(smax) - math.log(smin)) * u[k, 1])
        reqs.append(dict(
            id=k, t_arrival=t,
            kind="droplet" if u[k, 2] < 0.5 else "channel",
            nx=max(8, int(round(s))), ny=max(8, int(round(s / 2))),
            steps=int(kmin + (kmax - kmin) * u[k, 3]),
            G_A=0.15 * u[k, 4], G_R=0.15 * u[k, 5]))
        if max_requests is not None and len(reqs) >= max_requests:
            break
    return reqs
