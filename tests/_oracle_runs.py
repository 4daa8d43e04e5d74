"""Oracle runs used by the physics pins, as module-level functions so that a
spawn-started process pool can run them in parallel.  Measurements are done
here with plain numpy (no package code): pressure from its closed form,
interface points by linear interpolation, an algebraic least-squares circle."""
import math

import numpy as np

from oracle import lbm_oracle as O
import workloads as W


def pressure_exp(rho, G, theta):
    """Bulk pressure of the exponential pseudo-potential fluid (rho0 = 1):
    p = rho theta + G theta psi^2 / 2."""
    psi = 1.0 - np.exp(-rho)
    return rho * theta + 0.5 * G * theta * psi * psi


def laplace_drop(R, n=64, steps=3000, G=-5.5, rho_l=2.3, rho_v=0.105):
    """A free drop (no wall) of initial radius R on an n x n periodic lattice.
    Returns (equilibrium radius from the liquid area, p_in - p_out)."""
    lat = O.D2Q9
    rho = W.droplet_density(n, n, [(n / 2.0, n / 2.0)], [R], rho_l, rho_v, 2.0)
    p = O.Params(lattice=lat, tau=1.0, G=G)
    z = np.zeros_like(rho)
    f = O.run(p, None, O.initial_populations(p, rho, z, z), steps)
    r, _, _ = O.macroscopic(p, None, f)
    mid = 0.5 * (r.max() + r.min())
    # area of the liquid, counting each node by its fraction across the interface
    frac = np.clip((r - r.min()) / (r.max() - r.min()), 0.0, 1.0)
    R_eq = math.sqrt(frac.sum() / math.pi)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    d = np.hypot(x - n / 2.0, y - n / 2.0)
    pr = pressure_exp(r, G, lat.theta)
    return R_eq, float(pr[d < R_eq - 4].mean() - pr[d > R_eq + 6].mean()), float(mid)


def _interface_points(field, level, mask):
    f = field - level
    xs, ys = [], []
    a, b = f[:, :-1], f[:, 1:]
    m = (a * b < 0) & mask[:, :-1] & mask[:, 1:]
    yy, xx = np.nonzero(m)
    xs.append(xx + a[yy, xx] / (a[yy, xx] - b[yy, xx]))
    ys.append(yy.astype(float))
    a, b = f[:-1, :], f[1:, :]
    m = (a * b < 0) & mask[:-1, :] & mask[1:, :]
    yy, xx = np.nonzero(m)
    xs.append(xx.astype(float))
    ys.append(yy + a[yy, xx] / (a[yy, xx] - b[yy, xx]))
    return np.concatenate(xs), np.concatenate(ys)


def _contact_angle(rho, phi_s, rho_l, rho_v):
    """theta = acos((y_b - y_c) / R): circle fitted (algebraically) to the
    rho = (rho_l + rho_v)/2 points with phi_S < 0.01 below mid-height; y_b is
    where phi_S falls through 0.5 above the bottom wall."""
    ny = rho.shape[0]
    mask = phi_s < 0.01
    mask[ny // 2:, :] = False
    x, y = _interface_points(rho, 0.5 * (rho_l + rho_v), mask)
    A = np.column_stack([x, y, np.ones_like(x)])
    (a, b, c), *_ = np.linalg.lstsq(A, x * x + y * y, rcond=None)
    xc, yc = a / 2.0, b / 2.0
    R = math.sqrt(c + xc * xc + yc * yc)
    col = phi_s[:, 0]
    k = int(np.nonzero(col <= 0.5)[0][0])
    yb = (k - 1) + (col[k - 1] - 0.5) / (col[k - 1] - col[k])
    return math.degrees(math.acos(max(-1.0, min(1.0, (yb - yc) / R))))


def sessile_angles(G_A, G_R=0.1, nx=96, ny=48, R=15.0, steps=9000, chunk=1500):
    """Contact angle of a drop on the tanh wall (core 0.1, tail G_A) after each
    chunk of steps."""
    w = W.droplet_on_wall(nx=nx, ny=ny, R=R, G_A=G_A, G_R=G_R, noise_amp=0.0)
    p = O.Params(lattice=O.D2Q9, tau=w.tau, G=w.G)
    wall = O.Wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon)
    f = O.initial_populations(p, w.rho, w.ux, w.uy)
    out = []
    for _ in range(steps // chunk):
        f = O.run(p, wall, f, chunk)
        r, _, _ = O.macroscopic(p, wall, f)
        out.append(_contact_angle(r, w.phi_s, w.meta["rho_l"], w.meta["rho_v"]))
    return out
