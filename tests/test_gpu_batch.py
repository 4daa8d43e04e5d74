"""Batches: many lattices advanced by one fused launch per step.

Each member's node arithmetic is the same as when it runs alone, so a member's
populations after n batch steps must equal, bit for bit, those after n steps on
its own -- for every tiling, with persistent CTAs, across odd step counts (the
16- and 2-step graphs plus single launches) and when members are stepped on
their own or removed between batch steps."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    torch.cuda.set_device(0)
    import paper_1202_6130_gb300 as p
    p.load()
    return p


def _cases():
    out = []
    for k, (nx, ny) in enumerate([(64, 32), (200, 90), (131, 47), (300, 160), (8, 8), (257, 33)]):
        w = W.droplet_on_wall(nx=nx, ny=ny, R=min(nx, ny) / 3.0, seed=20 + k, noise_amp=1e-5,
                              tau=0.7 + 0.15 * k, G=-5.0 - 0.2 * k, G_A=0.02 * k, G_R=0.15 - 0.02 * k)
        if k % 2 == 1:
            uw = np.zeros((2, ny, nx))
            uw[0, ny // 2:, :] = 0.01
            w.u_wall = uw
        if k == 3:
            w.body_force = (2e-6, 0.0)
        out.append(w)
    return out


def _alone(pkg, w, storage, n, **kw):
    sim = pkg.Simulation.from_workload(w, storage=storage, **kw)
    sim.step(n)
    f = sim.populations()
    sim.close()
    return f


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16s", "bf16s"])
@pytest.mark.parametrize("tiling", [(0, 0), (8, 0), (16, 300), (5, 7)])
def test_batch_equals_members_alone_bitwise(pkg, storage, tiling):
    ws = _cases()
    n1, n2 = 7, 10  # odd then even: single launch, graph replays, phase carry-over
    want = [_alone(pkg, w, storage, n1 + n2) for w in ws]
    sims = [pkg.Simulation.from_workload(w, storage=storage) for w in ws]
    b = pkg.Batch()
    for s in sims:
        b.add(s)
    b.set_tiling(*tiling)
    b.step(n1)
    b.step(n2)
    for s, f in zip(sims, want):
        np.testing.assert_array_equal(s.populations(), f)
        assert s.steps_done() == n1 + n2
    b.close()


def test_members_stepped_alone_or_removed_between_batch_steps(pkg):
    ws = _cases()[:4]
    sims = [pkg.Simulation.from_workload(w, storage="fp64") for w in ws]
    b = pkg.Batch()
    for s in sims:
        b.add(s)
    b.step(3)
    sims[1].step(2)          # member advanced on its own
    b.step(4)
    b.remove(sims[2])        # sims[2] stays at 7 steps
    b.step(1)
    expect = {0: 8, 1: 10, 2: 7, 3: 8}
    for i, s in enumerate(sims):
        assert s.steps_done() == expect[i]
        np.testing.assert_array_equal(s.populations(), _alone(pkg, ws[i], "fp64", expect[i]))
    b.close()


def test_batch_rejects_mixed_kinds_and_autotunes(pkg):
    ws = _cases()[:3]
    a = pkg.Simulation.from_workload(ws[0], storage="fp32")
    c = pkg.Simulation.from_workload(ws[1], storage="fp64")
    b = pkg.Batch()
    b.add(a)
    with pytest.raises(pkg.LbmError):
        b.add(c)
    b.add(pkg.Simulation.from_workload(ws[2], storage="fp32"))
    best = b.autotune(steps_per_trial=4)
    assert best["tile_rows"] in (4, 8, 12, 16, 24, 32, 64) and best["ms_per_step"] > 0
    b.step(3)
    assert np.isfinite(a.moments()[0]).all()
    b.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16s"])
def test_long_graph_replays_equal_members_alone_bitwise(pkg, storage):
    """37 steps from parity 0 replay the 16-step graph twice, the 2-step graph
    twice and one single launch; 16 more from parity 1 start with a single
    launch and then replay the 16-step graph from the other parity's side.
    Drops of uneven sizes and a body-force-driven channel equal their solo
    runs bit for bit."""
    ws = [W.droplet_on_wall(nx=48 + 16 * k, ny=24 + 8 * k, R=6.0 + k, seed=500 + k,
                            noise_amp=1e-5, tau=0.8 + 0.1 * k) for k in range(3)]
    ws.append(W.poiseuille_channel(nx=32, ny=40, force=2e-6))
    sims = [pkg.Simulation.from_workload(w, storage=storage) for w in ws]
    b = pkg.Batch()
    for s_ in sims:
        b.add(s_)
    b.step(37)
    for s_, w in zip(sims, ws):
        assert s_.steps_done() == 37
        np.testing.assert_array_equal(s_.populations(), _alone(pkg, w, storage, 37))
    b.step(16)
    for s_, w in zip(sims, ws):
        np.testing.assert_array_equal(s_.populations(), _alone(pkg, w, storage, 53))
    b.close()


def test_tuned_tiling_is_kept_per_size_class(pkg):
    """autotune records its choice for the batch's (lattice, storage, size
    class); another batch of that class adopts it without stepping, one of
    another class (or storage) finds none; bits do not depend on the tiling."""
    ws = [W.droplet_on_wall(nx=40 + 8 * k, ny=24 + 4 * k, R=6.0, seed=300 + k, noise_amp=1e-5)
          for k in range(4)]
    tuned = pkg.Batch()
    for w in ws:
        tuned.add(pkg.Simulation.from_workload(w, storage="bf16s"))
    best = tuned.autotune(steps_per_trial=4)
    tuned.close()
    same = [pkg.Simulation.from_workload(w, storage="bf16s") for w in ws]
    b = pkg.Batch()
    for s in same:
        b.add(s)
    assert b.use_tuned()
    assert all(s.steps_done() == 0 for s in same)
    b.step(5)
    for s, w in zip(same, ws):
        np.testing.assert_array_equal(s.populations(), _alone(pkg, w, "bf16s", 5))
    b.close()
    big = pkg.Batch()
    big.add(pkg.Simulation.from_workload(W.droplet_on_wall(nx=256, ny=128, R=20.0), storage="bf16s"))
    assert not big.use_tuned()
    big.close()
    other = pkg.Batch()
    for w in ws:
        other.add(pkg.Simulation.from_workload(w, storage="fp16s"))
    assert not other.use_tuned()
    other.close()
    assert best["tile_rows"] > 0


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16s", "bf16s"])
def test_d2q21_paper_fluid_batch_equals_members_alone_bitwise(pkg, storage):
    """D2Q21 (one node per thread in FP64 and FP32, node pairs in 16-bit
    storage; plane groups as boxes of depth 1, 3 and 7) with the Eq. EOS
    pseudo-potential and the projection step; one member also has a body
    force."""
    th = 2.0 / 3.0
    kw = dict(eos=(0.25 * th, -0.25 * th, th, 0.222, 0.869), project=True)
    ws = []
    for k, (nx, ny) in enumerate([(96, 48), (131, 40)]):
        w = W.droplet_on_wall(nx=nx, ny=ny, R=14.0, lattice=21, seed=40 + k, noise_amp=1e-5,
                              tau=0.8 + 0.3 * k, G=-1.0 / th, G_A=0.3, G_R=1.33, rho_l=1.0,
                              rho_v=0.1)
        w.psi_kind = 1
        if k == 1:
            w.body_force = (2e-6, 0.0)
        ws.append(w)
    want = [_alone(pkg, w, storage, 9, **kw) for w in ws]
    sims = [pkg.Simulation.from_workload(w, storage=storage, **kw) for w in ws]
    b = pkg.Batch()
    for sm in sims:
        b.add(sm)
    b.step(4)
    b.step(5)
    for sm, f in zip(sims, want):
        np.testing.assert_array_equal(sm.populations(), f)
    b.close()


def test_member_reinitialised_between_batch_steps(pkg):
    """Setting a member's populations again (new 16-bit storage shift, step
    counter back to 0) makes the batch rebuild that member's step arguments."""
    ws = _cases()[:2]
    sims = [pkg.Simulation.from_workload(w, storage="fp16s") for w in ws]
    b = pkg.Batch()
    for s in sims:
        b.add(s)
    b.step(3)
    w2 = W.droplet_on_wall(nx=ws[1].nx, ny=ws[1].ny, R=10.0, seed=77, rho_l=1.2, rho_v=0.3)
    sims[1].set_equilibrium(w2.rho, w2.ux, w2.uy)
    b.step(4)
    ref = pkg.Simulation.from_workload(ws[1], storage="fp16s")
    ref.set_equilibrium(w2.rho, w2.ux, w2.uy)
    ref.step(4)
    np.testing.assert_array_equal(sims[1].populations(), ref.populations())
    np.testing.assert_array_equal(sims[0].populations(), _alone(pkg, ws[0], "fp16s", 7))
    b.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16s"])
def test_many_members_span_several_launch_chunks(pkg, storage):
    """140 lattices: three launch chunks of at most 64 members, each chunk on its
    own stream forked from and joined to the batch stream inside each graph
    replay.  Every member still equals its solo run bit for bit, across an odd
    step count."""
    ws = [W.droplet_on_wall(nx=24 + 4 * (k % 7), ny=16 + 2 * (k % 5), R=5.0, seed=100 + k,
                            noise_amp=1e-5, tau=0.7 + 0.005 * k, G_A=0.0005 * k) for k in range(140)]
    want = [_alone(pkg, w, storage, 5) for w in ws]
    sims = [pkg.Simulation.from_workload(w, storage=storage) for w in ws]
    b = pkg.Batch()
    for s in sims:
        b.add(s)
    assert b.launches_per_step() == 3
    b.step(2)
    b.step(3)
    for s, f in zip(sims, want):
        np.testing.assert_array_equal(s.populations(), f)
        assert s.steps_done() == 5
    b.set_tiling(8, 300)       # persistent CTAs shared out over the chunks
    b.step(2)
    ref = [pkg.Simulation.from_workload(w, storage=storage) for w in ws[:5]]
    for r in ref:
        r.step(7)
    for s, r in zip(sims[:5], ref):
        np.testing.assert_array_equal(s.populations(), r.populations())
    b.close()
