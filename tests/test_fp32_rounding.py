"""How FP32 rounding accumulates on the 128x64 drop over 1000 steps (CPU).

A float32 restatement of the FP32 step (tests/_f32_step.py) stays within the
1e-5 pointwise density bound of the FP64 oracle when 1/rho is correctly
rounded, and leaves it when the reciprocal is one unit too large: a one-sided
error in u = j/rho accumulates on the interface.  This is why the FP32
kernel takes the correctly rounded reciprocal.  An FP32-sized perturbation of
the initial state, by contrast, does not grow under the FP64 oracle: the
error is accumulated rounding, not amplification by the dynamics."""
import numpy as np
import pytest

import workloads as W
from oracle import lbm_oracle as O

from tests import _f32_step as F


@pytest.fixture(scope="module")
def drop():
    w = W.droplet_on_wall()
    p = O.Params(lattice=O.D2Q9, tau=w.tau, G=w.G, rho0=w.rho0)
    wall = O.Wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)
    f0 = O.initial_populations(p, w.rho, w.ux, w.uy, w.noise)
    return w, p, wall, f0, O.moments(p.lattice, O.run(p, wall, f0, 1000))[0]


def _err(p, f, rho_o):
    rho = O.moments(p.lattice, f.astype(np.float64))[0]
    return float(np.max(np.abs(rho - rho_o) / rho_o))


def test_float32_step_meets_1e5_with_a_correctly_rounded_reciprocal(drop):
    w, p, _, _, rho_o = drop
    e_rn = _err(p, F.run(w, 1000, rcp_bias=0), rho_o)
    e_up = _err(p, F.run(w, 1000, rcp_bias=+1), rho_o)
    assert e_rn <= 1e-5, e_rn
    assert e_up > 1e-5 and e_up > 1.5 * e_rn, (e_up, e_rn)


def test_fp32_sized_initial_perturbation_does_not_grow(drop):
    _, p, wall, f0, rho_o = drop
    rng = np.random.default_rng(5)
    f1 = f0 * (1.0 + rng.uniform(-2.0 ** -24, 2.0 ** -24, f0.shape))
    rho1 = O.moments(p.lattice, O.run(p, wall, f1, 1000))[0]
    assert float(np.max(np.abs(rho1 - rho_o) / rho_o)) < 2e-7
