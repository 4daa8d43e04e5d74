"""Checkpoint and resume: n steps, a checkpoint (populations and clock) saved
to disk, a new context restored from it and stepped m more times, equals n + m
steps of one context bit for bit, in every storage (16-bit values survive the
FP64 round trip of the checkpoint exactly, and the stochastic-rounding counter
is part of the clock)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16s", "bf16s"])
@pytest.mark.parametrize("lattice", [9, 21])
def test_resume_from_checkpoint_is_bit_exact(tmp_path, storage, lattice):
    import torch
    torch.cuda.set_device(0)
    import paper_1202_6130_gb300 as pkg
    w = W.droplet_on_wall(nx=70, ny=37, R=12.0, noise_amp=1e-5, lattice=lattice, tau=0.9)
    w.body_force = (1e-6, 0.0)
    ref = pkg.Simulation.from_workload(w, storage=storage)
    ref.step(23)
    path = str(tmp_path / "ckpt.npz")
    ref.save(path)
    assert ref.clock()[0] == 23
    ref.step(17)
    want = ref.populations()
    ref.close()

    sim = pkg.Simulation.from_checkpoint(path)
    sim.set_wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)
    assert sim.clock()[0] == 23
    sim.step(17)
    np.testing.assert_array_equal(sim.populations(), want)
    assert sim.clock()[0] == 40
    sim.close()
