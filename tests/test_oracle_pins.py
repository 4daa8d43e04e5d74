"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: exact
rational identities of the quadrature (Table I), closed forms of the
equilibrium and of the exact-difference-method collision, an O(N^2) brute-force
pair sum for the discrete force operator, conservation laws, the analytic
Poiseuille curvature, mechanical coexistence of a flat interface, the
numbers printed in the paper (Eq. EOS parameters, the hydrodynamic boundary
y_w of Fig. 3, the adsorbed fraction of Sec. III), and the trends it reports
(the contact angle against the attraction strength, the capillary slip against
the wall exponent).
"""
import itertools
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import lbm_oracle as O
from oracle import wall_filter as WF
import workloads as W
from tests import _golden

LATS = [O.D2Q9, O.D2Q21]


# --------------------------------------------------------------------------
# Quadrature (Sec. II A, Table I)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_lattice_isotropy_exact(lat):
    """Exact rational moments: sum w = 1, odd moments 0, sum w c c = theta I,
    4th order 3 theta^2 / theta^2; D2Q21 also 6th order (15, 3) theta^3."""
    th = lat.theta_exact
    w = lat.w_exact

    def mom(px, py):
        return sum(wi * Fr(cx) ** px * Fr(cy) ** py for wi, (cx, cy) in zip(w, lat.c))

    assert mom(0, 0) == 1
    for px, py in itertools.product(range(6), range(6)):
        if (px + py) % 2 == 1 and px + py <= 7:
            assert mom(px, py) == 0
    assert mom(2, 0) == th and mom(0, 2) == th and mom(1, 1) == 0
    assert mom(4, 0) == 3 * th ** 2 and mom(2, 2) == th ** 2 and mom(0, 4) == 3 * th ** 2
    if lat.Q == 21:
        assert mom(6, 0) == 15 * th ** 3
        assert mom(4, 2) == 3 * th ** 3
        assert mom(2, 4) == 3 * th ** 3


def test_d2q21_matches_table1():
    groups, theta = _golden.table1()
    lat = O.D2Q21
    assert lat.theta_exact == theta
    speeds = {"speed1_axes": {1}, "diagonal_1": {2}, "speed2_axes": {4},
              "diagonal_2": {8}, "speed3_axes": {9}, "rest": {0}}
    for g, (a, b, wt) in groups.items():
        for s in range(a, b + 1):
            i = s - 1                      # paper states are 1-based
            cx, cy = lat.c[i]
            assert lat.w_exact[i] == wt, (g, s)
            assert cx * cx + cy * cy in speeds[g], (g, s)
    # every velocity appears once
    assert len(set(lat.c)) == 21


# --------------------------------------------------------------------------
# Equilibrium (Eq. feqc / f2), projection, collision (Eq. BE-BGK with EDM)
# --------------------------------------------------------------------------

def _rand_state(lat, ny=5, nx=7, seed=11):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.5, (ny, nx))
    ux = rng.uniform(-0.1, 0.1, (ny, nx))
    uy = rng.uniform(-0.1, 0.1, (ny, nx))
    return rho, ux, uy


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_equilibrium_moments(lat):
    """sum f^eq = rho, sum f^eq c = rho u, sum f^eq c c = rho u u + rho theta I."""
    rho, ux, uy = _rand_state(lat)
    feq = O.equilibrium(lat, rho, ux, uy)
    r, jx, jy = O.moments(lat, feq)
    pxx, pxy, pyy = O.second_moment(lat, feq)
    th = lat.theta
    np.testing.assert_allclose(r, rho, rtol=1e-14)
    np.testing.assert_allclose(jx, rho * ux, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(jy, rho * uy, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pxx, rho * ux * ux + rho * th, rtol=1e-13)
    np.testing.assert_allclose(pyy, rho * uy * uy + rho * th, rtol=1e-13)
    np.testing.assert_allclose(pxy, rho * ux * uy, rtol=1e-12, atol=1e-15)


def test_equilibrium_weights_at_rest():
    """u = 0: f_i^eq = w_i rho exactly (Eq. feqc at zero velocity)."""
    for lat in LATS:
        rho = np.array([[1.7]])
        feq = O.equilibrium(lat, rho, np.zeros((1, 1)), np.zeros((1, 1)))
        np.testing.assert_array_equal(feq[:, 0, 0], lat.w * 1.7)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_projection_keeps_m0_m1_m2_and_is_idempotent(lat):
    rng = np.random.default_rng(3)
    rho, ux, uy = _rand_state(lat)
    f = O.equilibrium(lat, rho, ux, uy) + rng.uniform(-1e-3, 1e-3, (lat.Q,) + rho.shape)
    g = O.project(lat, f)
    for a, b in zip(O.moments(lat, f) + O.second_moment(lat, f),
                    O.moments(lat, g) + O.second_moment(lat, g)):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(O.project(lat, g), g, rtol=1e-12, atol=1e-15)
    feq = O.equilibrium(lat, rho, ux, uy)
    np.testing.assert_allclose(O.project(lat, feq), feq, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_edm_tau_one_is_shifted_equilibrium(lat):
    """tau = 1: f^post = f^eq(rho, u*) whatever f is (closed form of EDM-BGK)."""
    rng = np.random.default_rng(5)
    rho, ux, uy = _rand_state(lat)
    f = O.equilibrium(lat, rho, ux, uy) + rng.uniform(-1e-3, 1e-3, (lat.Q,) + rho.shape)
    r, jx, jy = O.moments(lat, f)
    u0x, u0y = jx / r, jy / r
    usx, usy = u0x + 0.01, u0y - 0.02
    p = O.Params(lattice=lat, tau=1.0)
    post = O.collide(p, f, r, u0x, u0y, usx, usy)
    np.testing.assert_allclose(post, O.equilibrium(lat, r, usx, usy), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_collision_conserves_mass_and_adds_force(tau):
    """sum f^post = rho and sum f^post c = rho u* = j + F (EDM momentum balance)."""
    lat = O.D2Q9
    rng = np.random.default_rng(7)
    rho, ux, uy = _rand_state(lat)
    f = O.equilibrium(lat, rho, ux, uy) + rng.uniform(-1e-3, 1e-3, (lat.Q,) + rho.shape)
    r, jx, jy = O.moments(lat, f)
    Fx = rng.uniform(-1e-3, 1e-3, r.shape)
    Fy = rng.uniform(-1e-3, 1e-3, r.shape)
    p = O.Params(lattice=lat, tau=tau)
    post = O.collide(p, f, r, jx / r, jy / r, jx / r + Fx / r, jy / r + Fy / r)
    r2, jx2, jy2 = O.moments(lat, post)
    np.testing.assert_allclose(r2, r, rtol=1e-14)
    np.testing.assert_allclose(jx2, jx + Fx, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(jy2, jy + Fy, rtol=1e-11, atol=1e-15)


# --------------------------------------------------------------------------
# Streaming and the discrete force operator (Eqs. force_SC, force_SC_FS)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_stream_moves_each_population_by_its_velocity(lat):
    ny, nx = 9, 11
    f = np.zeros((lat.Q, ny, nx))
    x0, y0 = 2, 7
    f[:, y0, x0] = np.arange(1, lat.Q + 1)
    g = O.stream(lat, f)
    for i, (cx, cy) in enumerate(lat.c):
        assert g[i, (y0 + cy) % ny, (x0 + cx) % nx] == i + 1
        assert np.count_nonzero(g[i]) == 1


def _brute_force_sum(lat, field):
    """sum over every lattice node y of w(y - x) field(y) (y - x), with the
    minimal-image offset and w = 0 for offsets that are not lattice velocities:
    an O(N^2) pair sum written without the stencil."""
    ny, nx = field.shape
    wmap = {c: float(wi) for c, wi in zip(lat.c, lat.w_exact)}
    sx = np.zeros_like(field)
    sy = np.zeros_like(field)
    for (ya, xa) in itertools.product(range(ny), range(nx)):
        ax = ay = 0.0
        for (yb, xb) in itertools.product(range(ny), range(nx)):
            dx = (xb - xa + nx // 2) % nx - nx // 2
            dy = (yb - ya + ny // 2) % ny - ny // 2
            wgt = wmap.get((dx, dy), 0.0)
            ax += wgt * field[yb, xb] * dx
            ay += wgt * field[yb, xb] * dy
        sx[ya, xa] = ax
        sy[ya, xa] = ay
    return sx, sy


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_force_operator_matches_brute_force_pair_sum(lat):
    rng = np.random.default_rng(13)
    field = rng.uniform(0.0, 1.0, (8, 8))
    sx, sy = O.weighted_sum(lat, field)
    bx, by = _brute_force_sum(lat, field)
    np.testing.assert_allclose(sx, bx, atol=1e-15)
    np.testing.assert_allclose(sy, by, atol=1e-15)


def test_force_ff_brute_force_8x8_full_step():
    """F_FF = -G psi(x) sum_y w(y-x) psi(y) (y-x) from a brute-force pair sum on
    the 8x8 lattice equals the oracle's force for a random density field."""
    lat = O.D2Q9
    rng = np.random.default_rng(17)
    rho = rng.uniform(0.2, 2.2, (8, 8))
    p = O.Params(lattice=lat, G=-5.5)
    F = O.forces(p, None, rho, np.zeros_like(rho), np.zeros_like(rho))
    psi = 1.0 - np.exp(-rho)
    bx, by = _brute_force_sum(lat, psi)
    np.testing.assert_allclose(F.ff[0], 5.5 * psi * bx, atol=1e-15)
    np.testing.assert_allclose(F.ff[1], 5.5 * psi * by, atol=1e-15)


def test_pseudo_potentials_closed_forms():
    rho = np.array([0.05, 0.1, 0.222, 0.5, 0.869, 1.0, 2.0])
    p = O.Params(lattice=O.D2Q9, rho0=1.0)
    np.testing.assert_allclose(O.pseudo_potential(p, rho), 1.0 - np.exp(-rho), rtol=1e-15)
    pv = _golden.paper_values()
    lat = O.D2Q21
    pp = O.paper_profile(lat)
    th = lat.theta
    assert pp.eos_theta_v == pv["eos_theta_v_over_theta"][0] * th
    assert pp.eos_theta_u == pv["eos_theta_u_over_theta"][0] * th
    assert pp.eos_theta_l == pv["eos_theta_l_over_theta"][0] * th
    assert pp.eos_rho1 == pv["eos_rho_1"][0] and pp.eos_rho2 == pv["eos_rho_2"][0]
    # continuity of Eq. EOS at the knots
    e = 1e-12
    for knot in (pp.eos_rho1, pp.eos_rho2):
        a, b = O.p_eos(pp, np.array([knot - e, knot + e]))
        assert abs(a - b) < 1e-11
    # the printed coexistence densities have (nearly) equal EOS pressure
    pv_, pl_ = O.p_eos(pp, np.array([pv["eos_rho_v"][0], pv["eos_rho_l"][0]]))
    assert abs(pv_ - pl_) / pl_ < 0.02
    # psi_FF = sqrt(2 (rho theta - p)) is real on all branches and constant
    # on the liquid branch (theta_L = theta: ideal behaviour)
    psi = O.pseudo_potential(pp, np.array([0.9, 1.0, 1.5]))
    np.testing.assert_allclose(psi, psi[0], rtol=1e-12)
    assert np.all(np.isfinite(O.pseudo_potential(pp, np.linspace(0.0, 3.0, 301))))


# --------------------------------------------------------------------------
# Whole-step invariants
# --------------------------------------------------------------------------

def _params_for(w):
    return O.Params(lattice=O.LATTICES[w.lattice], tau=w.tau, G=w.G, rho0=w.rho0,
                    body_force=tuple(w.body_force))


def _wall_for(w):
    return O.Wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_uniform_rest_state_is_a_fixed_point(lat):
    p = O.Params(lattice=lat, tau=0.8, G=-5.5)
    rho = np.full((6, 10), 0.7)
    z = np.zeros_like(rho)
    f = O.equilibrium(lat, rho, z, z)
    F = O.forces(p, None, rho, z, z)
    assert np.all(F.total[0] == 0.0) and np.all(F.total[1] == 0.0)
    g = O.run(p, None, f, 20)
    np.testing.assert_allclose(g, f, rtol=4e-15, atol=0)


def test_mass_conserved_on_the_128x64_droplet_1000_steps():
    w = W.droplet_on_wall()
    p, wall = _params_for(w), _wall_for(w)
    f = O.initial_populations(p, w.rho, w.ux, w.uy, w.noise)
    m0 = O.totals(p, wall, f)[0]
    f = O.run(p, wall, f, 1000)
    m1 = O.totals(p, wall, f)[0]
    assert abs(m1 - m0) / m0 < 1e-13
    assert np.all(np.isfinite(f))


def test_momentum_conserved_without_walls_and_grows_with_body_force():
    lat = O.D2Q9
    rho = W.droplet_density(40, 32, [(20.0, 16.0)], [8.0], 2.0, 0.15, 2.0)
    z = np.zeros_like(rho)
    noise = W.uniform(9, 9 * rho.size, -1e-4, 1e-4).reshape((9,) + rho.shape)
    p = O.Params(lattice=lat, tau=0.9, G=-5.5)
    f0 = O.initial_populations(p, rho, z, z, noise)
    j0 = O.bare_momentum(p, f0)
    f = O.run(p, None, f0, 100)
    j1 = O.bare_momentum(p, f)
    assert abs(j1[0] - j0[0]) < 1e-12 and abs(j1[1] - j0[1]) < 1e-12
    fb = (2e-6, -1e-6)
    pb = O.Params(lattice=lat, tau=0.9, G=-5.5, body_force=fb)
    f = O.run(pb, None, f0, 50)
    j2 = O.bare_momentum(pb, f)
    n = rho.size
    assert abs(j2[0] - (j0[0] + 50 * n * fb[0])) < 1e-11
    assert abs(j2[1] - (j0[1] + 50 * n * fb[1])) < 1e-11


def test_flat_film_has_exactly_zero_tangential_velocity():
    """Mirror symmetry x -> -x of an x-invariant film: u_x = 0 exactly (the
    relaxation to zero u_y is pinned by the next test)."""
    w = W.poiseuille_channel(nx=6, ny=40, force=0.0)
    y = np.arange(40, dtype=float)[:, None]
    w.rho = np.repeat(0.15 + 1.85 * 0.5 * (1.0 - np.tanh(2.0 * (y - 12.0) / 2.0)), 6, axis=1)
    p, wall = _params_for(w), _wall_for(w)
    f = O.initial_populations(p, w.rho, w.ux, w.uy)
    f = O.run(p, wall, f, 300)
    rho, ux, uy = O.macroscopic(p, wall, f)
    assert np.all(ux == 0.0)
    assert np.all(np.isfinite(uy))


def test_flat_film_equilibrium_has_zero_velocity():
    """A liquid film on the wall (x-invariant) relaxes to rest: u_x stays
    exactly 0 and u_y decays to rounding level (below 1e-10 after 7000 steps)."""
    w = W.poiseuille_channel(nx=6, ny=24, force=0.0)
    y = np.arange(24, dtype=float)[:, None]
    w.rho = np.repeat(0.15 + 1.85 * 0.5 * (1.0 - np.tanh(2.0 * (y - 8.0) / 2.0)), 6, axis=1)
    p, wall = _params_for(w), _wall_for(w)
    f = O.run(p, wall, O.initial_populations(p, w.rho, w.ux, w.uy), 7000)
    rho, ux, uy = O.macroscopic(p, wall, f)
    assert np.all(ux == 0.0)
    assert np.max(np.abs(uy)) < 1e-10


# --------------------------------------------------------------------------
# Physics pins
# --------------------------------------------------------------------------

def _pool(fn, args):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(min(len(args), 8), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, args))


def test_laplace_law_across_droplet_radii():
    """Free drops of radius 8-16 (exponential psi, G = -5.5): the pressure jump
    p_in - p_out (p = rho theta + G theta psi^2 / 2) is linear in 1/R with a
    vanishing intercept (Laplace, dp = gamma / R in 2-D), gamma > 0."""
    from tests import _oracle_runs as R
    res = _pool(R.laplace_drop, [8, 10, 12, 14, 16])
    inv = np.array([1.0 / r[0] for r in res])
    dp = np.array([r[1] for r in res])
    A = np.vstack([inv, np.ones_like(inv)]).T
    (gamma, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    resid = dp - A @ np.array([gamma, c])
    r2 = 1.0 - (resid ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert gamma > 0.0 and r2 > 0.999, (gamma, r2)
    assert abs(c) < 0.05 * dp.mean(), (c, dp)


def test_contact_angle_falls_with_tail_strength():
    """Sessile drop on the tanh wall, core G_R = 0.1, tail G_A in [0, 0.1]:
    the equilibrium angle decreases monotonically with G_A, and cos theta is
    linear in G_A (Sec. III B).  The angles are converged: the last 1500
    steps change them by less than 0.2 deg."""
    from tests import _oracle_runs as R
    gas = [0.0, 0.1 / 3, 0.2 / 3, 0.1]
    hist = _pool(R.sessile_angles, gas)
    th = np.array([h[-1] for h in hist])
    assert all(abs(h[-1] - h[-2]) < 0.2 for h in hist), hist
    assert np.all(np.diff(th) < -1.0), th
    c = np.cos(np.radians(th))
    a1, a0 = np.polyfit(gas, c, 1)
    resid = c - (a1 * np.array(gas) + a0)
    assert 1.0 - (resid ** 2).sum() / ((c - c.mean()) ** 2).sum() > 0.99
    assert 45.0 < th.min() and th.max() < 90.0

def test_poiseuille_bulk_curvature_matches_viscosity():
    """Steady body-force-driven channel: in the hydrodynamic region (phi_S < 0.01)
    u(y) is a parabola with u'' = -f / (rho nu), nu = theta (tau - 1/2)."""
    tau, fb = 1.0, 1e-6
    w = W.poiseuille_channel(nx=1, ny=48, force=fb, tau=tau)
    p, wall = _params_for(w), _wall_for(w)
    f = O.initial_populations(p, w.rho, w.ux, w.uy)
    f = O.run(p, wall, f, 9000)
    rho, ux, uy = O.macroscopic(p, wall, f)
    col_u, col_rho, phi = ux[:, 0], rho[:, 0], w.phi_s[:, 0]
    bulk = phi < 0.01
    # the bulk band is contiguous around the channel centre y = ny/2
    ys = np.arange(48)[bulk].astype(float)
    a2, a1, a0 = np.polyfit(ys, col_u[bulk], 2)
    nu = O.D2Q9.theta * (tau - 0.5)
    rho_bulk = col_rho[bulk].mean()
    expect = -fb / (rho_bulk * nu)
    assert abs(2.0 * a2 - expect) / abs(expect) < 0.01
    # the solid bulk is held at the wall velocity by the momentum exchange
    assert abs(col_u[0]) < 0.05 * col_u.max()


def _channel_slip(eps, G_A, steps=4000):
    """Slip length of the steady 32-row channel (body force 1e-5): the bulk
    parabola u(y) over phi_S < 0.01, extrapolated to the hydrodynamic boundary
    y_w where phi_S falls through 0.01 above the bottom wall, b = u(y_w)/|u'(y_w)|."""
    w = W.poiseuille_channel(nx=2, ny=32, force=1e-5, epsilon=eps, G_A=G_A)
    p, wall = _params_for(w), _wall_for(w)
    f = O.run(p, wall, O.initial_populations(p, w.rho, w.ux, w.uy), steps)
    _, ux, _ = O.macroscopic(p, wall, f)
    u, phi = ux.mean(axis=1), w.phi_s.mean(axis=1)
    ys = np.arange(len(u), dtype=float)
    bulk = phi < 0.01
    a2, a1, a0 = np.polyfit(ys[bulk], u[bulk], 2)
    k = int(np.argmax(bulk))                   # first bulk row above the bottom slab
    yw = (k - 1) + (phi[k - 1] - 0.01) / (phi[k - 1] - phi[k])
    return (a2 * yw * yw + a1 * yw + a0) / abs(2 * a2 * yw + a1)


def test_capillary_slip_grows_with_wall_exponent_and_not_with_attraction():
    """Sec. III A (pressure-driven flow in a capillary): the wall with the
    larger exponent epsilon = 1.3 slips markedly more than epsilon = 1, and the
    slip hardly changes with the attraction strength G_A.  Under this build's
    readings the oracle gives slip lengths 1.82-1.84 (epsilon = 1) and
    2.16-2.19 (1.3) on this channel, 1.4-1.7% apart over G_A = 0.02-0.1.  (The
    paper calls epsilon = 1 a no-slip wall; measured from the phi_S = 0.01
    boundary the slip length there is not zero, so only the ordering and the
    independence are pinned.)  A dropped or misplaced exponent makes the two
    walls slip alike and fails the first assertion."""
    b = {(e, g): _channel_slip(e, g) for e in (1.0, 1.3) for g in (0.02, 0.1)}
    for g in (0.02, 0.1):
        assert b[(1.3, g)] > 1.1 * b[(1.0, g)], b
    for e in (1.0, 1.3):
        assert abs(b[(e, 0.1)] - b[(e, 0.02)]) < 0.03 * b[(e, 0.02)], b
    assert all(v > 0 for v in b.values()), b


def test_flat_interface_mechanical_coexistence_exp_psi():
    """Flat liquid slab (no wall): at equilibrium the bulk pressures
    p = rho theta + G theta psi^2 / 2 of liquid and vapour are equal, and the
    densities separate (G = -5.5 is beyond the critical -4)."""
    lat = O.D2Q9
    ny = 64
    y = np.arange(ny, dtype=float)[:, None]
    rho = np.repeat(0.15 + 1.85 * 0.5 * (np.tanh((y - 16) / 2.0) - np.tanh((y - 48) / 2.0)), 2, axis=1)
    p = O.Params(lattice=lat, tau=1.0, G=-5.5)
    z = np.zeros_like(rho)
    f = O.run(p, None, O.initial_populations(p, rho, z, z), 6000)
    r, ux, uy = O.macroscopic(p, None, f)
    rl, rv = r[32, 0], r[0, 0]
    th = lat.theta

    def pres(d):
        ps = 1.0 - math.exp(-d)
        return d * th + p.G * th * ps * ps / 2.0

    assert rl / rv > 10.0
    assert abs(pres(rl) - pres(rv)) / pres(rl) < 2e-3
    assert np.max(np.abs(uy)) < 1e-6


def test_paper_eos_flat_interface_density_ratio_d2q21():
    """Paper profile (D2Q21, Eq. EOS, G = -1/theta, projection on): a flat
    interface settles near rho_V = 0.1, rho_L = 1.0 (density ratio 10)."""
    lat = O.D2Q21
    pv = _golden.paper_values()
    ny = 80
    y = np.arange(ny, dtype=float)[:, None]
    rho = np.repeat(0.1 + 0.9 * 0.5 * (np.tanh((y - 20) / 3.0) - np.tanh((y - 60) / 3.0)), 1, axis=1)
    p = O.paper_profile(lat, tau=1.0)
    z = np.zeros_like(rho)
    f = O.run(p, None, O.initial_populations(p, rho, z, z), 4000)
    r, ux, uy = O.macroscopic(p, None, f)
    rl, rv = r[40, 0], r[0, 0]
    ratio, tol = pv["density_ratio"]
    assert abs(rl - pv["eos_rho_l"][0]) < 0.1
    assert abs(rv - pv["eos_rho_v"][0]) < 0.01
    assert abs(rl / rv - ratio) / ratio < tol


def _eos_drop(R, n=48, steps=1500):
    """Free drop of the paper fluid (D2Q21, Eq. EOS, G = -1/theta, projection
    on) of initial radius R on an n x n periodic lattice: its radius from the
    liquid area and p_in - p_out with p = p_EOS(rho)."""
    p = O.paper_profile(O.D2Q21, tau=1.0)
    rho = W.droplet_density(n, n, [(n / 2.0, n / 2.0)], [R], 1.0, 0.1, 2.0)
    z = np.zeros_like(rho)
    r, _, _ = O.macroscopic(p, None, O.run(p, None, O.initial_populations(p, rho, z, z), steps))
    frac = np.clip((r - r.min()) / (r.max() - r.min()), 0.0, 1.0)
    R_eq = math.sqrt(frac.sum() / math.pi)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    d = np.hypot(x - n / 2.0, y - n / 2.0)
    pr = O.p_eos(p, r)
    return R_eq, float(pr[d < R_eq - 4].mean() - pr[d > R_eq + 6].mean())


def test_paper_eos_surface_tension_from_laplace_law_d2q21():
    """Paper profile: the pressure jump across free drops (radii 7.5-14) is
    linear in 1/R (Laplace's law in 2-D, dp = gamma / R) with a negligible
    intercept, and the slope gamma is the printed surface tension of the
    Eq. EOS fluid, 0.09, within 10% (the oracle gives 0.084).  This pins the
    normalisation of the fluid-fluid force in magnitude (G = -1/theta with the
    paper's psi): with G = -1 the fluid would not be the printed one."""
    pv = _golden.paper_values()
    pts = [_eos_drop(R) for R in (8.0, 11.0, 14.0)]
    inv_r = np.array([1.0 / a for a, _ in pts])
    dp = np.array([b for _, b in pts])
    slope, icept = np.polyfit(inv_r, dp, 1)
    fit = slope * inv_r + icept
    r2 = 1.0 - np.sum((dp - fit) ** 2) / np.sum((dp - dp.mean()) ** 2)
    gamma, tol = pv["surface_tension"]
    assert r2 > 0.999, (r2, pts)
    assert abs(icept) < 0.05 * dp.min(), (icept, pts)
    assert abs(slope - gamma) < tol * gamma, (slope, pts)


# --------------------------------------------------------------------------
# Wall functions (Appendix)
# --------------------------------------------------------------------------

def test_wall_filter_bounds_monotone_and_hydrodynamic_boundary():
    pv = _golden.paper_values()
    lat = O.D2Q21
    ny, nx = 74, 10
    solid = np.zeros((ny, nx), bool)
    solid[0, :] = True
    its = WF.iterates(lat, solid, int(pv["n_att"][0]))
    for a, b in zip(its[:-1], its[1:]):
        assert np.all(b >= a - 1e-15)
        assert np.all((b >= 0.0) & (b <= 1.0 + 1e-15))
    phi, pr, pa = WF.wall_functions(lat, solid, int(pv["n_rep"][0]), int(pv["n_att"][0]))
    col = phi[:, 0]
    # first crossing of 0.01 above the bottom wall, linearly interpolated
    k = next(y for y in range(1, ny // 2) if col[y] <= 0.01)
    yw = (k - 1) + (col[k - 1] - 0.01) / (col[k - 1] - col[k])
    yw_paper, tol = pv["y_w"]
    assert abs(yw - yw_paper) <= tol
    # symmetric about the solid row (opposite wall across the periodic seam)
    np.testing.assert_allclose(col[1:], col[1:][::-1], rtol=1e-12)
    np.testing.assert_allclose(pa, phi - pr, rtol=0, atol=0)


def test_adsorbed_fraction_falls_with_repulsion_strength():
    """Sec. III: the vapour fraction adsorbed in the solid falls from about 0.03
    (G_R = 0.9) to about 0.001 (G_R = 3.0).  Pins the sign of the core term of
    psi_FS (a core that attracted fluid would raise it) and, through the ratio
    of the two printed values (30), the scaling of F_FS with G_R."""
    pv = _golden.paper_values()
    lat = O.D2Q21
    ny = 40
    solid = np.zeros((ny, 1), bool)
    solid[0, :] = True
    phi, pr, pa = WF.wall_functions(lat, solid)
    frac = {}
    for GR in (0.9, 3.0):
        p = O.paper_profile(lat, tau=1.0)
        wall = O.Wall(phi, pr, pa, GR, 0.0, 1.0)
        rho = np.full((ny, 1), 1.0)
        z = np.zeros_like(rho)
        f = O.run(p, wall, O.initial_populations(p, rho, z, z), 1500)
        r, _, _ = O.macroscopic(p, wall, f)
        frac[GR] = r[0, 0] / r[ny // 2, 0]
    assert frac[3.0] < frac[0.9]
    printed = pv["adsorbed_GR_0p9"][0] / pv["adsorbed_GR_3p0"][0]
    assert 0.5 * printed < frac[0.9] / frac[3.0] < 2.0 * printed
    assert frac[3.0] < 10 * pv["adsorbed_GR_3p0"][0]


def test_moving_wall_drives_linear_couette_profile():
    """Eq. wall_shift with U_wall != 0: two solid slabs, one at rest (y = 0) and
    one moving at U (y = ny/2).  At steady state the solid slabs move with
    their wall velocity and the fluid between them carries a linear shear
    profile, antisymmetric about the mid-plane, with zero mean stress jump."""
    ny, U = 60, 0.01
    y = np.arange(ny, dtype=float)
    d = np.minimum(np.minimum(y, ny - y), np.abs(y - ny // 2))[:, None]
    phi, pr, pa = W.wall_core_tail(d, 3.0)
    uw = np.zeros((2, ny, 1))
    uw[0, np.abs(y - ny // 2) < 8, 0] = U
    p = O.Params(lattice=O.D2Q9, tau=1.0, G=-5.5)
    wall = O.Wall(phi, pr, pa, 0.1, 0.05, 1.0, uw)
    rho = np.full((ny, 1), 2.0)
    z = np.zeros_like(rho)
    f = O.run(p, wall, O.initial_populations(p, rho, z, z), 5000)
    r, ux, uy = O.macroscopic(p, wall, f)
    u = ux[:, 0]
    assert abs(u[0]) < 0.02 * U
    assert abs(u[ny // 2] - U) < 0.02 * U
    # bulk band between the slabs: linear, rising from the resting to the moving wall
    band = (phi[:, 0] < 0.01) & (y < ny // 2)
    a1, a0 = np.polyfit(y[band], u[band], 1)
    resid = u[band] - (a1 * y[band] + a0)
    assert a1 > 0 and np.max(np.abs(resid)) < 0.02 * U
    # the other band mirrors it
    band2 = (phi[:, 0] < 0.01) & (y > ny // 2)
    b1, _ = np.polyfit(y[band2], u[band2], 1)
    assert abs(a1 + b1) < 0.02 * abs(a1)
