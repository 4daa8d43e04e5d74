"""Stochastic rounding of the 16-bit population storage.

A uniform liquid (rho = 2, storage shift 1, so every stored deviation is
about w_i) is driven by a body force of 1e-6 per node.  Each step adds about
3e-7 to a population, far below the spacing of the stored 16-bit deviation
(6e-5 in FP16S, 5e-4 in BF16S): round-to-nearest discards every increment and
the liquid never moves, while stochastic rounding keeps them on average, so the
total momentum follows the FP64 run up to its rounding noise.  The noise of
the total x momentum after t steps is a random walk over the N nodes and t
steps: about sqrt(6 N t) * spacing / sqrt(6) (six populations carry x
momentum, each rounding error has variance spacing^2 / 6)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NY, STEPS, FORCE = 256, 128, 400, 1e-6


@pytest.fixture(scope="module")
def pkg():
    import torch
    torch.cuda.set_device(0)
    import paper_1202_6130_gb300 as p
    p.load()
    return p


def _drive(pkg, storage, rounding="stochastic"):
    """Totals after STEPS steps minus those of the encoded initial state (the
    16-bit encoding of the uniform start is itself rounded, identically at
    every node), and the final populations."""
    sim = pkg.Simulation(NX, NY, storage=storage, G=0.0, body_force=(FORCE, 0.0), shift_rho=1.0,
                         rounding=rounding)
    sim.set_equilibrium(np.full((NY, NX), 2.0))
    t0 = sim.totals()
    sim.step(STEPS)
    out = sim.totals() - t0, sim.populations()
    sim.close()
    return out


@pytest.fixture(scope="module")
def exact(pkg):
    (tot, _) = _drive(pkg, "fp64")
    # FP64 storage: the momentum grows by N * F per step; mass is conserved.
    assert tot[1] == pytest.approx(NX * NY * FORCE * STEPS, rel=1e-9)
    assert abs(tot[0]) < 1e-6
    return tot


@pytest.mark.parametrize("storage,spacing", [("fp16s", 2.0 ** -6 / 256.0), ("bf16s", 2.0 ** -11)])
def test_stochastic_rounding_keeps_sub_ulp_force_increments(pkg, exact, storage, spacing):
    tot, _ = _drive(pkg, storage)
    sigma = np.sqrt(NX * NY * STEPS) * spacing
    assert abs(tot[1] - exact[1]) < 6.0 * sigma, (tot[1], exact[1], sigma)
    assert abs(tot[1] - exact[1]) < 0.5 * exact[1]
    # mass: the rest population's spacing is at most 4x the largest moving one
    assert abs(tot[0] - exact[0]) < 6.0 * sigma * 4.0


def test_round_to_nearest_loses_them(pkg, exact):
    tot, _ = _drive(pkg, "fp16s", rounding="nearest")
    assert abs(tot[1]) < 0.05 * exact[1], (tot[1], exact[1])


def test_stochastic_rounding_is_reproducible(pkg):
    _, a = _drive(pkg, "bf16s")
    _, b = _drive(pkg, "bf16s")
    np.testing.assert_array_equal(a, b)


def _ulp(v, storage):
    """Spacing of the 16-bit number holding v (binary16 or bfloat16)."""
    a = np.abs(v)
    if storage == "fp16s":
        return 2.0 ** (np.floor(np.log2(np.maximum(a, 2.0 ** -14))) - 10)
    return 2.0 ** (np.floor(np.log2(np.maximum(a, 2.0 ** -126))) - 7)


@pytest.mark.parametrize("storage", ["fp16s", "bf16s"])
def test_16bit_codec_round_trip_within_half_an_ulp(pkg, storage):
    """set_populations stores each population's deviation from its shift,
    h = sigma (f - w_i rho_s) (sigma = 2^8 for FP16S, 1 for BF16S), formed in
    FP64 and rounded once to 16 bits (nearest-even); the read-back is
    h / sigma + w_i rho_s in FP64.  So each population comes back within half
    a unit in the last place of its stored deviation, plus FP64 rounding.
    Deviations of both signs, from about 1e-5 to the largest the lattice
    holds."""
    rng = np.random.default_rng(7)
    nx, ny = 64, 32
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho = rng.uniform(0.1, 2.5, (ny, nx))
    f = w[:, None, None] * rho[None] * rng.uniform(0.5, 1.5, (9, ny, nx))
    f[:, :4, :] = w[:, None, None] * (1.0 + rng.normal(0.0, 1e-6, (9, 4, nx)))  # tiny deviations
    sim = pkg.Simulation(nx, ny, storage=storage, shift_rho=1.0)
    sim.set_populations(f)
    g = sim.populations()
    sim.close()
    shift = w[:, None, None] * 1.0
    scale = 256.0 if storage == "fp16s" else 1.0
    dev = np.maximum(np.abs(f - shift), np.abs(g - shift)) * scale
    bound = 0.5 * _ulp(dev, storage) / scale + 4e-16 * np.abs(f)
    assert np.all(np.abs(g - f) <= bound), float(np.max(np.abs(g - f) / bound))
