"""Host-side FP64 measurements on the engine's moment fields (Sec. III of
arXiv:1202.6130): the static contact angle by a least-squares circle fit in the
hydrodynamic region, the hydrodynamic slip of a pressure-driven channel flow,
the Laplace pressure jump of a drop, and spurious-current magnitude.

These read outputs of ``Simulation.moments()``; they are not part of the time
step.  Conventions: arrays [y][x], the solid slab across the periodic seam
near y = 0, wall probability phi_S; the hydrodynamic region is phi_S < 0.01 and
the solid surface is the line phi_S = 0.5.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def contour_points(field: np.ndarray, level: float, mask: np.ndarray | None = None):
    """Points where ``field`` crosses ``level`` between horizontally or vertically
    adjacent nodes (linear interpolation), optionally only between nodes that are
    both inside ``mask``.  Returns (x, y) arrays (non-periodic: no wrap)."""
    f = field - level
    xs, ys = [], []
    # horizontal neighbours
    a, b = f[:, :-1], f[:, 1:]
    cross = (a * b < 0)
    if mask is not None:
        cross &= mask[:, :-1] & mask[:, 1:]
    yy, xx = np.nonzero(cross)
    t = a[yy, xx] / (a[yy, xx] - b[yy, xx])
    xs.append(xx + t)
    ys.append(yy.astype(float))
    # vertical neighbours
    a, b = f[:-1, :], f[1:, :]
    cross = (a * b < 0)
    if mask is not None:
        cross &= mask[:-1, :] & mask[1:, :]
    yy, xx = np.nonzero(cross)
    t = a[yy, xx] / (a[yy, xx] - b[yy, xx])
    xs.append(xx.astype(float))
    ys.append(yy + t)
    return np.concatenate(xs), np.concatenate(ys)


def fit_circle(x: np.ndarray, y: np.ndarray, iterations: int = 50):
    """Least-squares circle: algebraic (Kasa) start, then Gauss-Newton on the
    geometric distances.  Returns (xc, yc, R)."""
    A = np.column_stack([x, y, np.ones_like(x)])
    rhs = x * x + y * y
    (a, b, c), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = a / 2.0, b / 2.0
    R = math.sqrt(max(c + xc * xc + yc * yc, 1e-300))
    for _ in range(iterations):
        dx, dy = x - xc, y - yc
        d = np.sqrt(dx * dx + dy * dy)
        d = np.where(d == 0, 1e-300, d)
        res = d - R
        J = np.column_stack([-dx / d, -dy / d, -np.ones_like(d)])
        step, *_ = np.linalg.lstsq(J, -res, rcond=None)
        xc, yc, R = xc + step[0], yc + step[1], R + step[2]
        if np.max(np.abs(step)) < 1e-12:
            break
    return float(xc), float(yc), float(R)


def surface_line(phi_col: np.ndarray, level: float = 0.5) -> float:
    """Height above the bottom solid row where phi_S falls through ``level``
    (first crossing going up from y = 0; linear interpolation)."""
    for y in range(1, len(phi_col)):
        if phi_col[y] <= level < phi_col[y - 1]:
            return (y - 1) + (phi_col[y - 1] - level) / (phi_col[y - 1] - phi_col[y])
    return 0.0


@dataclass
class ContactAngle:
    theta_deg: float
    xc: float
    yc: float
    R: float
    y_base: float
    npoints: int


def interface_base(rho: np.ndarray, x: float, rho_mid: float) -> float:
    """Height of the lowest crossing of ``rho_mid`` in the column nearest to x:
    the bottom of the liquid, where the density falls towards the adsorbed
    vapour of the solid (linear interpolation between nodes)."""
    col = rho[:, int(round(x)) % rho.shape[1]]
    f = col - rho_mid
    for y in range(len(col) - 1):
        if f[y] * f[y + 1] < 0:
            return y + f[y] / (f[y] - f[y + 1])
    return 0.0


def contact_angle(rho: np.ndarray, phi_s: np.ndarray, rho_l: float, rho_v: float,
                  x_range=None, y_max=None, base: str = "surface") -> ContactAngle:
    """Static contact angle of a drop resting on the bottom wall.

    The drop's interface is the contour rho = (rho_l + rho_v)/2; only points in
    the hydrodynamic region (phi_S < 0.01) above the bottom wall and below
    ``y_max`` (default ny/2) are fitted.  theta = acos((y_b - y_c)/R), i.e.
    acos(1 - h/R) with h the apex height above the base line y_b (Sec. III,
    static wetting).  The base line: "surface" (default) the solid surface
    phi_S = 0.5; "outer" the domain's outer boundary, the row y = 0 (one
    reading of the Fig. 6 caption); "interface" the bottom liquid-vapour
    interface under the drop's centre (a reading of the text of Sec. III B)."""
    ny, nx = rho.shape
    y_max = ny // 2 if y_max is None else y_max
    mask = phi_s < 0.01
    mask[y_max:, :] = False
    if x_range is not None:
        m2 = np.zeros_like(mask)
        m2[:, x_range[0]:x_range[1]] = True
        mask &= m2
    x, y = contour_points(rho, 0.5 * (rho_l + rho_v), mask)
    if len(x) < 5:
        raise ValueError("too few interface points in the hydrodynamic region")
    xc, yc, R = fit_circle(x, y)
    if base == "surface":
        yb = surface_line(phi_s[:, int(round(xc)) % nx], 0.5)
    elif base == "outer":
        yb = 0.0
    elif base == "interface":
        yb = interface_base(rho, xc, 0.5 * (rho_l + rho_v))
    else:
        raise ValueError(base)
    c = max(-1.0, min(1.0, (yb - yc) / R))
    return ContactAngle(math.degrees(math.acos(c)), xc, yc, R, yb, len(x))


@dataclass
class Slip:
    slip_length: float
    y_w: float
    u_wall: float
    du_wall: float
    curvature: float


def slip_length(ux: np.ndarray, phi_s: np.ndarray) -> Slip:
    """Hydrodynamic slip of a body-force-driven channel (Sec. III, Poiseuille):
    fit u(y) = a y^2 + b y + c over the hydrodynamic region (phi_S < 0.01) of the
    x-averaged profile; the boundary y_w is where phi_S falls through 0.01 above
    the bottom wall; slip length = u(y_w) / |u'(y_w)|."""
    u = ux.mean(axis=1)
    phi = phi_s.mean(axis=1)
    ny = len(u)
    bulk = phi < 0.01
    ys = np.arange(ny, dtype=float)
    a, b, c = np.polyfit(ys[bulk], u[bulk], 2)
    yw = surface_line(phi, 0.01)
    uw = a * yw * yw + b * yw + c
    du = 2 * a * yw + b
    return Slip(float(uw / abs(du)) if du != 0 else float("inf"), float(yw), float(uw),
                float(du), float(2 * a))


def pressure_exp(rho: np.ndarray, G: float, rho0: float = 1.0, theta: float = 1.0 / 3.0):
    """Bulk pressure of the exponential pseudo-potential fluid:
    p = rho theta + G theta psi^2 / 2 (the continuum limit of Eq. force_SC)."""
    psi = rho0 * (1.0 - np.exp(-rho / rho0))
    return rho * theta + 0.5 * G * theta * psi * psi


def laplace_jump(rho: np.ndarray, G: float, center, r_in: float, r_out: float,
                 rho0: float = 1.0, theta: float = 1.0 / 3.0):
    """Pressure inside (r < r_in) minus outside (r > r_out) of a drop centred at
    ``center`` on the periodic lattice."""
    ny, nx = rho.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx = (x - center[0] + nx / 2) % nx - nx / 2
    dy = (y - center[1] + ny / 2) % ny - ny / 2
    r = np.hypot(dx, dy)
    p = pressure_exp(rho, G, rho0, theta)
    return float(p[r < r_in].mean() - p[r > r_out].mean())


def spurious_current(ux: np.ndarray, uy: np.ndarray) -> float:
    """max |u| over the lattice."""
    return float(np.sqrt(ux * ux + uy * uy).max())


def recenter_x(rho: np.ndarray, rho_mid: float):
    """Rolls a periodic field in x so that the liquid's circular-mean column is
    at nx/2 (a moving drop may straddle the periodic seam).  Returns the
    shift applied (columns) so that other fields can be rolled the same way."""
    ny, nx = rho.shape
    w = np.clip(rho - rho_mid, 0.0, None).sum(axis=0)
    ang = 2.0 * np.pi * np.arange(nx) / nx
    c = math.atan2(float((w * np.sin(ang)).sum()), float((w * np.cos(ang)).sum()))
    xc = (c / (2.0 * np.pi) * nx) % nx
    return int(round(nx / 2.0 - xc))


@dataclass
class DynamicAngles:
    theta_adv_deg: float
    theta_rec_deg: float
    x_apex: float
    h: float
    front: tuple
    rear: tuple
    npoints: tuple
    theta_adv_hR_deg: float = float("nan")
    theta_rec_hR_deg: float = float("nan")


def dynamic_angles(rho: np.ndarray, phi_s: np.ndarray, rho_l: float, rho_v: float,
                   y_max=None, direction: int = 1) -> DynamicAngles:
    """Advancing and receding angles of a drop moving along +x (direction=1):
    the interface contour rho = (rho_l + rho_v)/2 in the hydrodynamic region is
    split at the apex; one circle is fitted to the points ahead of it (front)
    and one to those behind it (rear), and each angle is acos((y_b - y_c)/R)
    with y_b the solid surface phi_S = 0.5 (Sec. III C).  Also returned, as
    theta_*_hR_deg: acos(1 - h/R) with the common apex height h above y_b and
    each circle's radius R (the wording of the Fig. 9 caption)."""
    ny, nx = rho.shape
    shift = recenter_x(rho, 0.5 * (rho_l + rho_v))
    rho = np.roll(rho, shift, axis=1)
    phi_s = np.roll(phi_s, shift, axis=1)
    y_max = ny // 2 if y_max is None else y_max
    mask = phi_s < 0.01
    mask[y_max:, :] = False
    x, y = contour_points(rho, 0.5 * (rho_l + rho_v), mask)
    if len(x) < 10:
        raise ValueError("too few interface points")
    ia = int(np.argmax(y))
    xa = float(x[ia])
    front = (x - xa) * direction >= 0
    rear = ~front
    yb = surface_line(phi_s[:, nx // 2], 0.5)
    out = []
    for sel in (front, rear):
        xc, yc, R = fit_circle(x[sel], y[sel])
        c = max(-1.0, min(1.0, (yb - yc) / R))
        out.append((math.degrees(math.acos(c)), (xc - shift) % nx, yc, R))
    h = float(y[ia] - yb)
    hr = [math.degrees(math.acos(max(-1.0, min(1.0, 1.0 - h / o[3])))) for o in out]
    return DynamicAngles(out[0][0], out[1][0], (xa - shift) % nx, h,
                         out[0][1:], out[1][1:], (int(front.sum()), int(rear.sum())),
                         hr[0], hr[1])


def drop_velocity(rho: np.ndarray, ux: np.ndarray, rho_mid: float, phi_s=None) -> float:
    """Mass-weighted mean x velocity of the liquid (rho > rho_mid), outside the
    solid (phi_S < 0.5) when phi_S is given."""
    m = rho > rho_mid
    if phi_s is not None:
        m &= phi_s < 0.5
    return float((rho[m] * ux[m]).sum() / rho[m].sum())


def _liquid_runs(rho, phi_s, rho_l, rho_v, y_max, min_height):
    """Periodic runs of columns with at least ``min_height`` liquid nodes in the
    hydrodynamic region (phi_S < 0.01, below y_max): the columns under drops or
    ridges, not those under a wetting film alone.  Returns (shift, runs) with
    the runs [x0, x1) in a frame rolled by ``shift`` so that none wraps."""
    mid = 0.5 * (rho_l + rho_v)
    liquid = (rho > mid) & (phi_s < 0.01)
    liquid[y_max:, :] = False
    cols = liquid.sum(axis=0) >= min_height
    if cols.all() or not cols.any():
        raise ValueError("no separate drops: every column or none holds liquid")
    shift = -int(np.argmin(cols))          # roll a dry column to x = 0
    cols = np.roll(cols, shift)
    edges = np.flatnonzero(np.diff(np.concatenate(([0], cols.astype(np.int8), [0]))))
    return shift, list(zip(edges[0::2].tolist(), edges[1::2].tolist()))


def contact_angles_of_drops(rho: np.ndarray, phi_s: np.ndarray, rho_l: float, rho_v: float,
                            y_max: int | None = None, min_width: int = 12,
                            min_height: int = 3):
    """Static angles of every drop resting on the bottom wall of a periodic
    lattice holding many of them.  A column belongs to a drop when at least
    ``min_height`` of its nodes in the hydrodynamic region (phi_S < 0.01, below
    ``y_max``) are liquid (rho above the mid density), so a wetting film along
    the wall does not join the drops; each periodic run of such columns at
    least ``min_width`` wide gets the circle fit of ``contact_angle`` over its
    own columns.  Returns a list of (x_centre, theta_deg, R), sorted by
    x_centre."""
    ny, nx = rho.shape
    y_max = ny // 2 if y_max is None else y_max
    shift, runs = _liquid_runs(rho, phi_s, rho_l, rho_v, y_max, min_height)
    rho_r = np.roll(rho, shift, axis=1)
    phi_r = np.roll(phi_s, shift, axis=1)
    out = []
    for x0, x1 in runs:
        if x1 - x0 < min_width:
            continue
        try:
            c = contact_angle(rho_r, phi_r, rho_l, rho_v, x_range=(max(0, x0 - 2), min(nx, x1 + 2)),
                              y_max=y_max)
        except ValueError:
            continue
        out.append((float((c.xc - shift) % nx), c.theta_deg, c.R))
    return sorted(out)


def contact_line_angles(rho: np.ndarray, phi_s: np.ndarray, rho_l: float, rho_v: float,
                        y_max: int | None = None, window: int = 40, min_height: int = 3):
    """Angle at every contact line of a periodic lattice whose drops may have
    merged into ridges: for each end of each run of liquid columns (see
    ``contact_angles_of_drops``), a circle is fitted to the interface contour
    over the ``window`` columns next to the line (hydrodynamic region only),
    and the angle is acos((y_b - y_c)/R) with y_b the solid surface.  Returns a
    list of (x_line, side, theta_deg) sorted by x_line, side -1 for a left
    (rising) and +1 for a right (falling) contact line."""
    ny, nx = rho.shape
    y_max = ny // 2 if y_max is None else y_max
    shift, runs = _liquid_runs(rho, phi_s, rho_l, rho_v, y_max, min_height)
    rho_r = np.roll(rho, shift, axis=1)
    phi_r = np.roll(phi_s, shift, axis=1)
    out = []
    for x0, x1 in runs:
        if x1 - x0 < window:
            continue
        for side, xr in ((-1, (max(0, x0 - 3), x0 + window)), (+1, (x1 - window, min(nx, x1 + 3)))):
            try:
                c = contact_angle(rho_r, phi_r, rho_l, rho_v, x_range=xr, y_max=y_max)
            except ValueError:
                continue
            xl = x0 if side < 0 else x1
            out.append((float((xl - shift) % nx), side, c.theta_deg))
    return sorted(out)
