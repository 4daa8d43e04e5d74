"""Plain FP64 restatement of one time step of the pseudo-potential wetting model.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.  Written from Colosqui, Kavousanakis, Papathanasiou & Kevrekidis,
"A mesoscopic model for microscale hydrodynamics and interfacial phenomena"
(arXiv:1202.6130), Sec. II, in the paper's order and notation.  numpy is used
only for whole-array arithmetic and for periodic shifts (``np.roll``); every
sum over lattice states is an explicit loop in table order.

State convention: ``f[i, y, x]`` is the population f_i(x, t) *before*
collision at time t (just after streaming).  Arrays are [y][x], y = 0 at the
bottom, fully periodic in x and y (the solid exists only through the wall
fields phi_S, psi_R-bar, psi_A-bar).

Readings of the paper taken here (each is listed with its justification in
the design notes of the repository):
  * Table I's third row is read as (+-2,0),(0,+-2) (the printed row repeats
    (+-2,0)); with it the weights sum to 1 and reproduce theta = 2/3.
  * F_FF = -G psi(x) sum_i w_i psi(x + r_i) r_i.  For the EOS pseudo-potential
    the paper's continuous force psi grad(w * psi) ~ psi grad psi is recovered
    with G = -1/theta, because sum_i w_i r_i r_i = theta I.
  * psi_FS = G_A psi_A-bar - G_R psi_R-bar, with G_R, G_A >= 0 strengths: the
    core repels fluid from the solid and the tail attracts it (the reading that
    matches "forces reverse direction as the solid is approached").
  * Delta u_wall = U_wall - u - F_FF dt / rho (a velocity), u the bare j / rho.
  * rho g = F_FF + F_FS (F_FS including Delta F_S) + a uniform body-force
    density; u* = u + rho g dt / rho (exact difference method).
  * The optional projection (Eq. f2) acts after streaming, before collision.
  * Reported velocity u_phys = (j + F/2) / rho.

What pins it (tests/test_oracle_pins.py): Table I exactly, the equilibrium
moments, the EDM closed form at tau = 1, streaming, the force operator against
an O(N^2) brute-force pair sum, conservation laws, the flat film, Laplace's
law, the Poiseuille curvature, Couette flow, coexistence densities, the
adsorbed-fraction trend of Sec. III and the trend of the contact angle with
G_A.  Parity unpinned: the magnitude of the fluid-solid terms under the
readings above (the sign of psi_FS, the F_FF term of Delta u_wall, rho rather
than psi multiplying the long-range sum) is pinned in sign and trend only; with
them the paper's own fluid and walls give static angles 8-35 degrees below the
table printed in Sec. III B, and no reading tried reproduces it.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction as Fr
from typing import Optional

import numpy as np

# ----------------------------------------------------------------------------
# Lattices (Sec. II A, Table I).  The oracle keeps its own copy of the tables.
# ----------------------------------------------------------------------------


@dataclass(frozen=True)
class Lattice:
    name: str
    c: tuple          # ((cx, cy), ...) in table order
    w_exact: tuple    # Fractions
    theta_exact: Fr

    @property
    def Q(self) -> int:
        return len(self.c)

    @property
    def w(self) -> np.ndarray:
        return np.array([float(v) for v in self.w_exact])

    @property
    def theta(self) -> float:
        return float(self.theta_exact)

    @property
    def reach(self) -> int:
        return max(max(abs(cx), abs(cy)) for cx, cy in self.c)


# D2Q9 (not in the paper; the standard 9-state set, theta = 1/3), rest state first.
D2Q9 = Lattice(
    "D2Q9",
    ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)),
    (Fr(4, 9),) + (Fr(1, 9),) * 4 + (Fr(1, 36),) * 4,
    Fr(1, 3),
)

# D2Q21, Table I: states 1-4 speed one on the axes, 5-8 diagonals, 9-12 speed
# two on the axes, 13-16 (+-2,+-2), 17-20 speed three on the axes, 21 at rest.
# Within each group the order is counter-clockwise starting on +x.
D2Q21 = Lattice(
    "D2Q21",
    ((1, 0), (0, 1), (-1, 0), (0, -1),
     (1, 1), (-1, 1), (-1, -1), (1, -1),
     (2, 0), (0, 2), (-2, 0), (0, -2),
     (2, 2), (-2, 2), (-2, -2), (2, -2),
     (3, 0), (0, 3), (-3, 0), (0, -3),
     (0, 0)),
    (Fr(1, 12),) * 4 + (Fr(2, 27),) * 4 + (Fr(7, 360),) * 4 + (Fr(1, 432),) * 4
    + (Fr(1, 1620),) * 4 + (Fr(91, 324),),
    Fr(2, 3),
)

LATTICES = {9: D2Q9, 21: D2Q21}


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------


@dataclass
class Params:
    """Problem statement of Sec. II: lattice, tau, fluid-fluid coupling, body force."""
    lattice: Lattice = D2Q9
    tau: float = 1.0
    G: float = -5.5
    psi_kind: str = "exp"              # "exp": rho0 (1 - exp(-rho/rho0)); "eos": Eq. EOS
    rho0: float = 1.0
    eos_theta_v: float = 0.25 / 3.0    # slopes of Eq. EOS (absolute values, not / theta)
    eos_theta_u: float = -0.25 / 3.0
    eos_theta_l: float = 1.0 / 3.0
    eos_rho1: float = 0.222
    eos_rho2: float = 0.869
    body_force: tuple = (0.0, 0.0)     # force density per node
    project: bool = False


@dataclass
class Wall:
    """Static wall fields (Sec. II "Fluid-Solid interactions", Appendix)."""
    phi_s: Optional[np.ndarray] = None     # wall probability phi_S, [ny, nx]
    psi_r: Optional[np.ndarray] = None     # repulsive potential psi_R-bar
    psi_a: Optional[np.ndarray] = None     # attractive potential psi_A-bar
    G_R: float = 0.0
    G_A: float = 0.0
    epsilon: float = 1.0
    u_wall: Optional[np.ndarray] = None    # [2, ny, nx] or None (solid at rest)


# ----------------------------------------------------------------------------
# Building blocks
# ----------------------------------------------------------------------------


def neighbour(field: np.ndarray, cx: int, cy: int) -> np.ndarray:
    """field(x + c) on the periodic lattice: out[y, x] = field[y + cy, x + cx]."""
    return np.roll(field, shift=(-cy, -cx), axis=(0, 1))


def moments(lat: Lattice, f: np.ndarray):
    """M0 = rho = sum_i f_i and M1 = j = sum_i f_i c_i (Eqs. M0, M1), table order."""
    rho = np.zeros(f.shape[1:])
    jx = np.zeros(f.shape[1:])
    jy = np.zeros(f.shape[1:])
    for i, (cx, cy) in enumerate(lat.c):
        rho = rho + f[i]
        jx = jx + f[i] * cx
        jy = jy + f[i] * cy
    return rho, jx, jy


def second_moment(lat: Lattice, f: np.ndarray):
    """M2 = Pi = sum_i f_i c_i c_i (Eq. M2): returns Pi_xx, Pi_xy, Pi_yy."""
    pxx = np.zeros(f.shape[1:])
    pxy = np.zeros(f.shape[1:])
    pyy = np.zeros(f.shape[1:])
    for i, (cx, cy) in enumerate(lat.c):
        pxx = pxx + f[i] * (cx * cx)
        pxy = pxy + f[i] * (cx * cy)
        pyy = pyy + f[i] * (cy * cy)
    return pxx, pxy, pyy


def equilibrium(lat: Lattice, rho, ux, uy) -> np.ndarray:
    """Lattice form of the Maxwell-Boltzmann equilibrium, Eq. feqc truncated at
    second Hermite order (Eq. f2 with M1 = rho u, M2 = rho u u + rho theta I):

        f_i^eq = w_i rho [1 + (c_i.u)/theta + (c_i.u)^2/(2 theta^2) - u^2/(2 theta)]
    """
    th = lat.theta
    rho = np.asarray(rho, dtype=np.float64)
    usq = ux * ux + uy * uy
    out = np.empty((lat.Q,) + rho.shape)
    for i, (cx, cy) in enumerate(lat.c):
        cu = cx * ux + cy * uy
        out[i] = lat.w[i] * rho * (1.0 + cu / th + cu * cu / (2.0 * th * th) - usq / (2.0 * th))
    return out


def project(lat: Lattice, f: np.ndarray) -> np.ndarray:
    """Projection step (Sec. II, after Eq. f2): replace f by its second-order
    Hermite expansion built from its own M0, M1, M2:

        f_i = w_i [M0 + M1.c_i/theta + (M2 - M0 theta I):(c_i c_i - theta I)/(2 theta^2)]
    """
    th = lat.theta
    rho, jx, jy = moments(lat, f)
    pxx, pxy, pyy = second_moment(lat, f)
    axx = pxx - rho * th
    ayy = pyy - rho * th
    out = np.empty_like(f)
    for i, (cx, cy) in enumerate(lat.c):
        contr = axx * (cx * cx - th) + 2.0 * pxy * (cx * cy) + ayy * (cy * cy - th)
        out[i] = lat.w[i] * (rho + (jx * cx + jy * cy) / th + contr / (2.0 * th * th))
    return out


def p_eos(p: Params, rho):
    """Piecewise-linear equation of state, Eq. EOS: vapour, unstable, liquid
    branches with slopes theta_V > 0, theta_U < 0, theta_L > 0."""
    r1, r2 = p.eos_rho1, p.eos_rho2
    p1 = r1 * p.eos_theta_v
    p2 = r1 * p.eos_theta_v + (r2 - r1) * p.eos_theta_u
    return np.where(rho <= r1, rho * p.eos_theta_v,
                    np.where(rho <= r2, p1 + (rho - r1) * p.eos_theta_u,
                             p2 + (rho - r2) * p.eos_theta_l))


def pseudo_potential(p: Params, rho):
    """psi_FF from rho: "exp" -> rho0 (1 - exp(-rho/rho0)) (Shan-Chen form);
    "eos" -> sqrt(2 [rho theta - p_EOS(rho)]) (Sec. II "Fluid-Fluid interactions")."""
    if p.psi_kind == "exp":
        return p.rho0 * (1.0 - np.exp(-rho / p.rho0))
    if p.psi_kind == "eos":
        th = p.lattice.theta
        return np.sqrt(2.0 * (rho * th - p_eos(p, rho)))
    raise ValueError(p.psi_kind)


def weighted_sum(lat: Lattice, field: np.ndarray):
    """sum_i w_i field(x + r_i) r_i over all states in table order (the discrete
    operator of Eqs. force_SC and force_SC_FS; the rest state adds zero)."""
    sx = np.zeros(field.shape)
    sy = np.zeros(field.shape)
    for i, (cx, cy) in enumerate(lat.c):
        nb = neighbour(field, cx, cy)
        sx = sx + lat.w[i] * nb * cx
        sy = sy + lat.w[i] * nb * cy
    return sx, sy


@dataclass
class Forces:
    ff: tuple          # F_FF
    fs_long: tuple     # rho sum_i w_i psi_FS(x + r_i) r_i
    dfs: tuple         # Delta F_S
    total: tuple       # F = F_FF + F_FS + body force


def forces(p: Params, wall: Optional[Wall], rho, ux, uy) -> Forces:
    """Interaction force rho g = F_FF + F_FS (Eqs. force_SC, force_SC_FS,
    pseudopotential, wall_shift) plus the body-force density."""
    lat = p.lattice
    psi = pseudo_potential(p, rho)
    sx, sy = weighted_sum(lat, psi)
    ffx = -p.G * psi * sx
    ffy = -p.G * psi * sy
    zero = np.zeros_like(rho)
    flx, fly, dfx, dfy = zero, zero, zero, zero
    if wall is not None:
        psi_fs = zero
        if wall.psi_a is not None:
            psi_fs = psi_fs + wall.G_A * wall.psi_a
        if wall.psi_r is not None:
            psi_fs = psi_fs - wall.G_R * wall.psi_r
        gx, gy = weighted_sum(lat, psi_fs)
        flx = rho * gx
        fly = rho * gy
        if wall.phi_s is not None:
            phie = wall.phi_s ** wall.epsilon
            uwx = wall.u_wall[0] if wall.u_wall is not None else zero
            uwy = wall.u_wall[1] if wall.u_wall is not None else zero
            dfx = rho * phie * (uwx - ux - ffx / rho)
            dfy = rho * phie * (uwy - uy - ffy / rho)
    bx, by = p.body_force
    fx = ffx + flx + dfx + bx
    fy = ffy + fly + dfy + by
    return Forces((ffx, ffy), (flx, fly), (dfx, dfy), (fx, fy))


def collide(p: Params, f, rho, ux, uy, usx, usy):
    """BGK relaxation plus the exact-difference-method force term (Eq. BE-BGK
    with delta f = f^eq(rho, u*) - f^eq(rho, u)):

        f_i^post = f_i - (f_i - f_i^eq(rho, u)) / tau + [f_i^eq(rho, u*) - f_i^eq(rho, u)]
    """
    feq = equilibrium(p.lattice, rho, ux, uy)
    feq_star = equilibrium(p.lattice, rho, usx, usy)
    return f - (f - feq) / p.tau + (feq_star - feq)


def stream(lat: Lattice, fpost: np.ndarray) -> np.ndarray:
    """Periodic streaming: f_i(x + c_i, t + 1) = f_i^post(x, t)."""
    out = np.empty_like(fpost)
    for i, (cx, cy) in enumerate(lat.c):
        out[i] = np.roll(fpost[i], shift=(cy, cx), axis=(0, 1))
    return out


def step(p: Params, wall: Optional[Wall], f: np.ndarray) -> np.ndarray:
    """One time step in the paper's order: moments, psi, forces, (projection),
    EDM-BGK collision, streaming."""
    lat = p.lattice
    rho, jx, jy = moments(lat, f)
    ux = jx / rho
    uy = jy / rho
    F = forces(p, wall, rho, ux, uy)
    usx = ux + F.total[0] / rho
    usy = uy + F.total[1] / rho
    if p.project:
        f = project(lat, f)
    fpost = collide(p, f, rho, ux, uy, usx, usy)
    return stream(lat, fpost)


def run(p: Params, wall: Optional[Wall], f: np.ndarray, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        f = step(p, wall, f)
    return f


def macroscopic(p: Params, wall: Optional[Wall], f: np.ndarray):
    """rho and the reported velocity u_phys = (j + F/2)/rho of the state f."""
    rho, jx, jy = moments(p.lattice, f)
    ux = jx / rho
    uy = jy / rho
    F = forces(p, wall, rho, ux, uy)
    return rho, (jx + 0.5 * F.total[0]) / rho, (jy + 0.5 * F.total[1]) / rho


def initial_populations(p: Params, rho, ux, uy, noise=None) -> np.ndarray:
    """f = f^eq(rho, u) plus an optional per-population perturbation."""
    f = equilibrium(p.lattice, rho, ux, uy)
    if noise is not None:
        f = f + noise
    return f


def totals(p: Params, wall: Optional[Wall], f: np.ndarray):
    """Total mass sum(rho) and momentum sum(j + F/2) (math.fsum, exact-rounded)."""
    import math
    rho, jx, jy = moments(p.lattice, f)
    F = forces(p, wall, rho, jx / rho, jy / rho)
    return (math.fsum(rho.ravel()),
            math.fsum((jx + 0.5 * F.total[0]).ravel()),
            math.fsum((jy + 0.5 * F.total[1]).ravel()))


def bare_momentum(p: Params, f: np.ndarray):
    """Sum of j = sum_i f_i c_i over the lattice (math.fsum)."""
    import math
    _, jx, jy = moments(p.lattice, f)
    return math.fsum(jx.ravel()), math.fsum(jy.ravel())


def paper_profile(lat: Lattice = D2Q21, tau: float = 1.0, project_step: bool = True) -> Params:
    """The paper's fluid: Eq. EOS with theta_V = 0.25 theta, theta_U = -0.25 theta,
    theta_L = theta, rho_1 = 0.222, rho_2 = 0.869, and G = -1/theta (see the
    module docstring for the 1/theta reading)."""
    th = lat.theta
    return Params(lattice=lat, tau=tau, G=-1.0 / th, psi_kind="eos",
                  eos_theta_v=0.25 * th, eos_theta_u=-0.25 * th, eos_theta_l=1.0 * th,
                  eos_rho1=0.222, eos_rho2=0.869, project=project_step)
