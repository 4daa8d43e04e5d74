"""Batches and the serving loop against the FP64 oracle.

The batch kernel and the server's shared launches are separate code paths
from a lattice stepped on its own; here their results are compared with the
oracle directly, not only with the solo CUDA path: FP64 storage, every member
or request element by element at 1e-12 relative (velocities relative to their
maximum), and the served contact angle or slip length equal to the one the
host analysis takes from the oracle's own moments.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lbm_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    torch.cuda.set_device(0)
    import paper_1202_6130_gb300 as p
    p.load()
    return p


def _oracle_params(w):
    if getattr(w, "psi_kind", 0) == 1:
        p = O.paper_profile(O.LATTICES[w.lattice], tau=w.tau, project_step=True)
        p.body_force = tuple(w.body_force)
        return p
    return O.Params(lattice=O.LATTICES[w.lattice], tau=w.tau, G=w.G, rho0=w.rho0,
                    body_force=tuple(w.body_force))


def _oracle_moments(w, steps):
    p = _oracle_params(w)
    wall = O.Wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)
    f = O.run(p, wall, O.initial_populations(p, w.rho, w.ux, w.uy, w.noise), steps)
    return O.macroscopic(p, wall, f)


def _errors(g, o):
    e_rho = float(np.max(np.abs(g[0] - o[0]) / np.abs(o[0])))
    umax = max(float(np.max(np.abs(o[1]))), float(np.max(np.abs(o[2]))), 1e-3)
    e_u = max(float(np.max(np.abs(g[1] - o[1]))), float(np.max(np.abs(g[2] - o[2])))) / umax
    return e_rho, e_u


def _sim(pkg, w):
    kw = {}
    G = w.G
    if getattr(w, "psi_kind", 0) == 1:
        th = O.LATTICES[w.lattice].theta
        kw = dict(eos=(0.25 * th, -0.25 * th, th, 0.222, 0.869), project=True)
        G = -1.0 / th
    s = pkg.Simulation(w.nx, w.ny, lattice=w.lattice, storage="fp64", tau=w.tau, G=G,
                       rho0=w.rho0, psi_kind=getattr(w, "psi_kind", 0),
                       body_force=tuple(w.body_force), **kw)
    s.set_wall(w.phi_s, w.psi_r, w.psi_a, w.G_R, w.G_A, w.epsilon, w.u_wall)
    s.set_equilibrium(w.rho, w.ux, w.uy, w.noise)
    return s


def _d2q9_members():
    """Uneven D2Q9 members: a drop, one with a moving upper wall, one driven by
    a body force, a ragged narrow one with its own tau, G and wall strengths."""
    a = W.droplet_on_wall(nx=96, ny=40, R=13.0, seed=31, noise_amp=1e-5)
    b = W.droplet_on_wall(nx=131, ny=29, R=9.0, seed=32, noise_amp=1e-5, tau=0.75, G=-5.2,
                          G_A=0.08, G_R=0.12)
    uw = np.zeros((2, b.ny, b.nx))
    uw[0, b.ny // 2:, :] = 0.01
    b.u_wall = uw
    c = W.droplet_on_wall(nx=70, ny=57, R=15.0, seed=33, noise_amp=1e-5, tau=1.3, G=-5.8)
    c.body_force = (3e-6, -1e-6)
    d = W.droplet_on_wall(nx=5, ny=33, R=2.0, seed=34, noise_amp=1e-4, tau=0.9, G_A=0.0)
    return [a, b, c, d]


def _d2q21_members():
    """D2Q21 members: the exponential fluid with a moving wall, and the
    paper's Eq. EOS fluid with the projection step and a body force."""
    a = W.droplet_on_wall(nx=67, ny=35, R=10.0, seed=41, noise_amp=1e-4, lattice=21, tau=0.8)
    uw = np.zeros((2, a.ny, a.nx))
    uw[0] = 0.005
    a.u_wall = uw
    b = W.droplet_on_wall(nx=61, ny=47, R=14.0, seed=42, noise_amp=0.0, lattice=21, tau=1.0)
    b.psi_kind = 1
    b.rho = 0.1 + 0.9 * (b.rho - 0.15) / 1.85
    b.G_R, b.G_A, b.epsilon = 1.33, 0.5, 1.3
    b.noise = None
    b.body_force = (2e-6, 0.0)
    return [a, b]


@pytest.mark.parametrize("which", ["d2q9", "d2q21"])
def test_batch_members_match_oracle(pkg, which):
    """Members of one batch (one fused launch per step for all of them, CUDA
    graph replays plus a single launch) against the oracle after 41 steps."""
    ws = _d2q9_members() if which == "d2q9" else _d2q21_members()
    sims = [_sim(pkg, w) for w in ws]
    b = pkg.Batch()
    for s in sims:
        b.add(s)
    b.set_tiling(5, 0)
    b.step(40)
    b.step(1)
    b.synchronize()
    for w, s in zip(ws, sims):
        e_rho, e_u = _errors(s.moments(), _oracle_moments(w, 41))
        assert e_rho <= 1e-12 and e_u <= 1e-12, (w.nx, w.ny, e_rho, e_u)
    b.close()
    for s in sims:
        s.close()


def test_served_results_match_oracle():
    """Four FP64 requests (drops and channels) served with a budget that holds
    about two at a time and a quantum shorter than every budget, so requests
    join and leave a running batch: each final state equals the oracle's after
    the same steps, and the returned angle or slip length equals the one the
    analysis takes from the oracle's moments."""
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import analysis as A
    from paper_1202_6130_gb300 import serve
    R = serve.Request
    reqs = [R(0, 0.0, "droplet", 64, 32, 180, G_A=0.03), R(1, 0.0, "channel", 8, 48, 260),
            R(2, 0.0, "droplet", 48, 40, 120, G_R=0.05, tau=0.9),
            R(3, 0.0, "channel", 8, 40, 200, epsilon=1.3)]
    budget = 2.2 * max(serve.footprint_bytes(r.nx, r.ny, "fp64") for r in reqs)
    srv = serve.Server(storage="fp64", hbm_budget=budget, quantum=50, keep_fields=True)
    out = {r.id: r for r in srv.run(reqs, realtime=False)}
    srv.close()
    assert sorted(out) == [0, 1, 2, 3]
    assert max(r.t_admit for r in out.values()) > min(r.t_admit for r in out.values())
    for req in reqs:
        w = serve.default_workload(req)
        mo = _oracle_moments(w, req.steps)
        got = out[req.id]
        e_rho, e_u = _errors((got.rho, got.ux, got.uy), mo)
        assert e_rho <= 1e-12 and e_u <= 1e-12, (req.id, e_rho, e_u)
        if req.kind == "droplet":
            want = A.contact_angle(mo[0], w.phi_s, w.meta["rho_l"], w.meta["rho_v"]).theta_deg
        else:
            want = A.slip_length(mo[1], w.phi_s).slip_length
        assert abs(got.value - want) <= 1e-8 * max(1.0, abs(want)), (req.id, got.value, want)
