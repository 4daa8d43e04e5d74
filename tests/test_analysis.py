"""The host-side measurements recover known answers from synthetic fields."""
import math

import numpy as np
import pytest

from paper_1202_6130_gb300 import analysis as A
import workloads as W


@pytest.mark.parametrize("theta_deg", [40.0, 90.0, 120.0])
def test_contact_angle_of_an_exact_circular_cap(theta_deg):
    nx, ny = 400, 240
    dist = W.wall_distance_slab(nx, ny)
    phi, _, _ = W.wall_core_tail(dist, 3.0)
    yb = A.surface_line(phi[:, 0], 0.5)
    R = 60.0
    yc = yb - R * math.cos(math.radians(theta_deg))
    rho = W.droplet_density(nx, ny, [(200.0, yc)], [R], 2.0, 0.1, 2.0)
    ca = A.contact_angle(rho, phi, 2.0, 0.1)
    assert abs(ca.theta_deg - theta_deg) < 0.5, ca
    assert abs(ca.R - R) < 0.5


def test_slip_length_of_a_shifted_parabola():
    ny, nx = 120, 4
    dist = W.wall_distance_slab(nx, ny)
    phi, _, _ = W.wall_core_tail(dist, 3.0)
    yw = A.surface_line(phi[:, 0], 0.01)
    b_true = 2.5
    # u = A (y - y0)(y1 - y), zero at y_w - b and ny - y_w + b
    y0, y1 = yw - b_true, ny - yw + b_true
    y = np.arange(ny, dtype=float)[:, None]
    u = 1e-4 * (y - y0) * (y1 - y) * np.ones((1, nx))
    s = A.slip_length(u, phi)
    # Navier slip: u(y_w) / u'(y_w) of the exact parabola
    uw = 1e-4 * (yw - y0) * (y1 - yw)
    du = 1e-4 * ((y1 - yw) - (yw - y0))
    assert abs(s.slip_length - uw / du) < 1e-8
    assert abs(s.curvature + 2e-4) < 1e-12


def test_laplace_pressure_of_a_flat_state_is_zero():
    rho = np.full((64, 64), 1.3)
    assert abs(A.laplace_jump(rho, -5.5, (32, 32), 5, 20)) < 1e-15


def test_dynamic_angles_of_two_joined_circular_arcs():
    """A drop whose front is an arc of 70 deg and whose rear is an arc of 50
    deg (same apex height): the two-circle fit returns both angles, also when
    the drop straddles the periodic seam."""
    nx, ny = 600, 200
    dist = W.wall_distance_slab(nx, ny)
    phi, _, _ = W.wall_core_tail(dist, 3.0)
    yb = A.surface_line(phi[:, 0], 0.5)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    h = 40.0
    dens = np.full((ny, nx), 0.1)
    for th_deg, side in ((70.0, 1), (50.0, -1)):
        th = math.radians(th_deg)
        R = h / (1.0 - math.cos(th))
        yc = yb + h - R
        xa = 300.0
        r = np.sqrt((x - xa) ** 2 + (y - yc) ** 2)
        cap = 0.1 + 0.9 * 0.5 * (1.0 - np.tanh(2.0 * (r - R) / 2.0))
        half = (x - xa) * side >= 0
        dens = np.where(half, np.maximum(dens, cap), dens)
    for shift in (0, 320):
        d = A.dynamic_angles(np.roll(dens, shift, axis=1), phi, 1.0, 0.1)
        assert abs(d.theta_adv_deg - 70.0) < 1.0 and abs(d.theta_rec_deg - 50.0) < 1.0, d
        # the same arcs through the common apex: acos(1 - h/R) gives the same angles
        assert abs(d.theta_adv_hR_deg - 70.0) < 1.0 and abs(d.theta_rec_hR_deg - 50.0) < 1.0, d


def test_contact_angle_base_line_readings():
    """The three base lines of the static angle on a cap whose liquid ends in
    a sharp step at y = 4 (a stand-in for the liquid-vapour interface at the
    bottom of a drop): "surface" (phi_S = 0.5), "outer" (the row y = 0) and
    "interface" (the step), each acos((y_b - y_c) / R) of the same circle."""
    nx, ny = 400, 240
    phi, _, _ = W.wall_core_tail(W.wall_distance_slab(nx, ny), 3.0)
    R, yc = 60.0, -10.0
    rho = W.droplet_density(nx, ny, [(200.0, yc)], [R], 2.0, 0.1, 2.0)
    rho[:4, :] = 0.1
    rho[4, :] = np.where(rho[4, :] > 1.05, 1.05 + 0.5 * (rho[4, :] - 1.05), rho[4, :])
    ys = {"surface": A.surface_line(phi[:, 200], 0.5), "outer": 0.0}
    col = rho[:, 200] - 1.05
    k = int(np.nonzero(col[:-1] * col[1:] < 0)[0][0])
    ys["interface"] = k + col[k] / (col[k] - col[k + 1])
    for base, yb in ys.items():
        ca = A.contact_angle(rho, phi, 2.0, 0.1, base=base)
        want = math.degrees(math.acos((yb - yc) / R))
        assert abs(ca.theta_deg - want) < 0.3, (base, ca.theta_deg, want)
        assert abs(ca.y_base - yb) < 1e-12


def test_contact_angles_of_several_drops_across_the_seam():
    """Three caps of 50, 90 and 120 degrees, one straddling the periodic seam:
    each is found and fitted on its own columns."""
    nx, ny = 900, 200
    phi, _, _ = W.wall_core_tail(W.wall_distance_slab(nx, ny), 3.0)
    yb = A.surface_line(phi[:, 0], 0.5)
    rho = np.full((ny, nx), 0.1)
    want = []
    for xc, th, R in ((20.0, 50.0, 60.0), (330.0, 90.0, 40.0), (640.0, 120.0, 30.0)):
        yc = yb - R * math.cos(math.radians(th))
        for shift in (-nx, 0, nx):
            rho = np.maximum(rho, W.droplet_density(nx, ny, [(xc + shift, yc)], [R], 2.0, 0.1, 2.0))
        want.append((xc, th))
    got = A.contact_angles_of_drops(rho, phi, 2.0, 0.1, y_max=150)
    assert len(got) == 3, got
    for (xc, th), (gx, gth, _) in zip(sorted(want), got):
        assert abs(((gx - xc + nx / 2) % nx) - nx / 2) < 1.0 and abs(gth - th) < 0.5, (xc, th, gx, gth)


def test_contact_line_angles_at_the_ends_of_a_ridge():
    """A ridge made of two overlapping caps of 70 degrees: the angle at each of
    its two contact lines is that of the cap ending there."""
    nx, ny = 700, 200
    phi, _, _ = W.wall_core_tail(W.wall_distance_slab(nx, ny), 3.0)
    yb = A.surface_line(phi[:, 0], 0.5)
    R = 60.0
    yc = yb - R * math.cos(math.radians(70.0))
    rho = W.droplet_density(nx, ny, [(300.0, yc), (380.0, yc)], [R, R], 2.0, 0.1, 2.0)
    lines = A.contact_line_angles(rho, phi, 2.0, 0.1, y_max=150)
    assert [s for _, s, _ in lines] == [-1, 1], lines
    for _, _, th in lines:
        assert abs(th - 70.0) < 1.0, lines
