"""Measurement studies on the GPU engine (host-side drivers; every time step
runs in the fused kernel, several lattices at once through a Batch).

  contact_angle_sweep  static contact angle of a 1024x512 drop (R = 160) for 8
                       tail strengths G_A in [0, 0.1] at G_R = 0.1, per storage
                       precision, with convergence history and spurious currents
  slip_study           slip length of a body-force-driven liquid channel, per
                       storage precision (x-invariant: a narrow periodic slice)
  large_precision      mass drift and density error of the 8192x4096 lattice in
                       FP32 / FP16S / BF16S storage against FP64 storage
  paper_theta_table    the paper's fluid (D2Q21, Eq. EOS, projection) with
                       Appendix wall functions: static angle vs G_A at G_R = 1.33,
                       next to the angles printed in Sec. III B
  dynamic_angles       the same drop driven along the wall by a uniform force:
                       droplet speed, capillary number, advancing and receding
                       angles (Sec. III C)

  python -m paper_1202_6130_gb300.studies sweep|slip|large|paper|dynamic [--steps N] ...
prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import analysis
from .sim import Batch, Simulation, wall_gaussian_filter

STORAGES = ("fp64", "fp32", "fp16s", "bf16s", "fp16s-rn", "bf16s-rn")


def storage_kw(label: str) -> dict:
    """Simulation keywords of a storage label: "fp16s" / "bf16s" round the
    stored deviations stochastically (the default), "fp16s-rn" / "bf16s-rn"
    to nearest-even."""
    if label.endswith("-rn"):
        return {"storage": label[:-3], "rounding": "nearest"}
    return {"storage": label}


def _run_batch(sims, steps: int, chunk: int, on_chunk=None):
    b = Batch()
    for s in sims:
        b.add(s)
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        b.step(n)
        done += n
        if on_chunk is not None:
            b.synchronize()
            on_chunk(done)
    b.synchronize()
    b.close()


def contact_angle_sweep(storages=STORAGES, steps: int = 50000, chunk: int = 10000,
                        n_tail: int = 8, nx: int = 1024, ny: int = 512, R: float = 160.0,
                        G_R: float = 0.1, G_A_max: float = 0.1):
    import workloads as W
    gas = [G_A_max * k / (n_tail - 1) for k in range(n_tail)]
    out = {"nx": nx, "ny": ny, "R": R, "G_R": G_R, "G_A": gas, "steps": steps, "storages": {}}
    for st in storages:
        ws = [W.droplet_on_wall(nx=nx, ny=ny, R=R, G_A=ga, G_R=G_R, noise_amp=1e-6, seed=0)
              for ga in gas]
        sims = [Simulation.from_workload(w, **storage_kw(st)) for w in ws]
        m0 = [s.totals()[0] for s in sims]
        hist = {i: [] for i in range(len(sims))}

        def record(done):
            for i, (s, w) in enumerate(zip(sims, ws)):
                rho, ux, uy = s.moments()
                try:
                    th = analysis.contact_angle(rho, w.phi_s, w.meta["rho_l"], w.meta["rho_v"]).theta_deg
                except Exception:
                    th = float("nan")
                hist[i].append((done, th, analysis.spurious_current(ux, uy)))

        t0 = time.perf_counter()
        _run_batch(sims, steps, chunk, record)
        wall = time.perf_counter() - t0
        m1 = [s.totals()[0] for s in sims]
        out["storages"][st] = {
            "theta_deg": [h[-1][1] for h in hist.values()],
            "theta_change_last_chunk_deg": [h[-1][1] - h[-2][1] if len(h) > 1 else float("nan")
                                            for h in hist.values()],
            "spurious_current": [h[-1][2] for h in hist.values()],
            "mass_drift_rel": [(b - a) / a for a, b in zip(m0, m1)],
            "history": {str(gas[i]): h for i, h in hist.items()},
            "wall_s": wall}
        for s in sims:
            s.close()
    if "fp64" in out["storages"]:
        ref = np.array(out["storages"]["fp64"]["theta_deg"])
        for st, d in out["storages"].items():
            d["theta_err_vs_fp64_deg"] = list(np.array(d["theta_deg"]) - ref)
    return out


def slip_study(storages=STORAGES, nx: int = 8, ny: int = 256, steps: int = 300000,
               chunk: int = 50000, force: float = 1e-6, epsilons=(1.0, 1.3)):
    import workloads as W
    out = {"nx": nx, "ny": ny, "force": force, "steps": steps, "storages": {}}
    for st in storages:
        res = {}
        for eps in epsilons:
            w = W.poiseuille_channel(nx=nx, ny=ny, force=force, epsilon=eps)
            sim = Simulation.from_workload(w, **storage_kw(st))
            hist = []

            def record(done):
                _, ux, _ = sim.moments()
                hist.append((done, analysis.slip_length(ux, w.phi_s).slip_length,
                             float(ux.max())))

            _run_batch([sim], steps, chunk, record)
            rho, ux, uy = sim.moments()
            s = analysis.slip_length(ux, w.phi_s)
            res[str(eps)] = {"slip_length": s.slip_length, "y_w": s.y_w, "u_max": float(ux.max()),
                             "curvature": s.curvature,
                             "curvature_expected": -force / (float(rho[ny // 2].mean()) * (1.0 / 3.0) * 0.5),
                             "history": hist}
            sim.close()
        out["storages"][st] = res
    if "fp64" in out["storages"]:
        for st, d in out["storages"].items():
            for eps, r in d.items():
                ref = out["storages"]["fp64"][eps]["slip_length"]
                r["slip_rel_err_vs_fp64"] = (r["slip_length"] - ref) / ref if ref else float("nan")
    return out


def _interface_height(rho, mid):
    """Height of the topmost liquid node per column (-1 where none)."""
    liquid = rho > mid
    ny = rho.shape[0]
    top = ny - 1 - np.argmax(liquid[::-1, :], axis=0)
    return np.where(liquid.any(axis=0), top, -1)


def large_precision(storages=("fp32", "fp16s", "bf16s", "fp16s-rn", "bf16s-rn"), steps: int = 20000):
    """8192x4096 multi-drop lattice: each storage precision against FP64 storage
    after `steps` steps: mass drift, density differences, the liquid height of
    every column, and the angle at every contact line (the 64 caps overlap from
    the start and merge into ridges, so the angles are those of the ridge ends,
    each from a circle fitted to the 40 columns next to the line), matched to
    the same line in FP64."""
    import workloads as W
    w = W.large_multi_droplet(noise_amp=0.0)
    rho_l, rho_v = w.meta["rho_l"], w.meta["rho_v"]
    mid = 0.5 * (rho_l + rho_v)
    ref = Simulation.from_workload(w, storage="fp64")
    m0 = ref.totals()[0]
    t0 = time.perf_counter()
    ref.step(steps)
    rho64 = ref.moments()[0]
    t64 = time.perf_counter() - t0
    lines64 = analysis.contact_line_angles(rho64, w.phi_s, rho_l, rho_v, y_max=400)
    h64 = _interface_height(rho64[:400], mid)
    out = {"steps": steps, "fp64": {"mass_drift_rel": (ref.totals()[0] - m0) / m0, "wall_s": t64,
                                    "contact_lines": lines64}}
    ref.close()
    for st in storages:
        sim = Simulation.from_workload(w, **storage_kw(st))
        a = sim.totals()[0]
        sim.step(steps)
        rho = sim.moments()[0]
        b = sim.totals()[0]
        d = np.abs(rho - rho64)
        try:
            lines = analysis.contact_line_angles(rho, w.phi_s, rho_l, rho_v, y_max=400)
        except ValueError:
            lines = []
        errs = []
        for xl, side, th in lines:
            for x64, s64, th64 in lines64:
                dx = abs(((xl - x64 + w.nx / 2) % w.nx) - w.nx / 2)
                if s64 == side and dx <= 5:
                    errs.append(th - th64)
                    break
        dh = np.abs(_interface_height(rho[:400], mid) - h64)
        out[st] = {"mass_drift_rel": (b - a) / a, "mass_vs_fp64_rel": (b - m0) / m0,
                   "rho_max_abs_err": float(d.max()), "rho_mean_abs_err": float(d.mean()),
                   "rho_rms_err": float(np.sqrt((d * d).mean())),
                   "contact_lines": lines, "contact_lines_matched": len(errs),
                   "theta_max_abs_err_vs_fp64_deg": float(np.max(np.abs(errs))) if errs else float("nan"),
                   "theta_err_vs_fp64_deg": errs,
                   "liquid_height_max_abs_diff": int(dh.max()),
                   "liquid_height_columns_differing": int((dh > 0).sum()),
                   "finite": bool(np.isfinite(rho).all())}
        sim.close()
    return out


# Angles printed in Sec. III B (Figs. 6-7 captions): G_R = 1.33, R0 = 50, 650 x 150.
PAPER_THETA = {0.0: 150.0, 0.2: 112.0, 0.5: 58.7, 0.7: 36.7, 0.8: 30.9, 0.9: 24.0}


BASES = ("surface", "outer", "interface")


def paper_wall_functions(solid, mode: str = "iterate", n_rep: int = 5, n_att: int = 22):
    """Wall functions of the Appendix for a solid mask, D2Q21.  "iterate": the
    reading the oracle and the library take, G^(n) = one filter pass of
    G^(n-1) reset to one on the solid, psi_R-bar = G^(5), psi_A-bar = G^(22) -
    G^(5), phi_S = G^(22).  "mean": the printed outer sum over passes read as
    the mean of the iterates G^(1) .. G^(N) (a sum would exceed one, which a
    wall probability cannot), each function then built from those means; every
    iterate comes from the library's filter."""
    if mode == "iterate":
        return wall_gaussian_filter(solid, lattice=21, n_rep=n_rep, n_att=n_att)
    if mode != "mean":
        raise ValueError(mode)
    its = [wall_gaussian_filter(solid, lattice=21, n_rep=n, n_att=n)[0] for n in range(1, n_att + 1)]
    g_r = np.mean(its[:n_rep], axis=0)
    g_a = np.mean(its, axis=0)
    return g_a, g_r, g_a - g_r


def paper_drops(cases, steps: int = 100000, chunk: int = 20000, storage: str = "fp32",
                nx: int = 650, ny: int = 150, G_R: float = 1.33, tau: float = 1.0,
                solid_rows: int = 1, filter_mode: str = "iterate"):
    """Sessile drops of the paper's fluid and walls, one per (R0, G_A) in
    ``cases``, advanced together in one batch: D2Q21, Eq. EOS (theta_V =
    theta/4, theta_U = -theta/4, theta_L = theta, rho_1 = 0.222, rho_2 =
    0.869) with G = -1/theta, projection on, wall functions from the Appendix
    filter of a solid slab (psi_R = G^(5), psi_A = G^(22) - G^(5), phi_S =
    G^(22), epsilon = 1).  A disc of area pi R0^2 starts tangent to the wall.
    Per case: the static angle on each base line of ``analysis.contact_angle``
    (the solid surface, the domain's outer boundary, the bottom liquid-vapour
    interface) and its history.  Readings (1/theta in the force, the sign of
    psi_FS) are the ones the oracle uses; filter_mode selects the reading of the
    Appendix filter (paper_wall_functions)."""
    import workloads as W
    th = 2.0 / 3.0
    solid = np.zeros((ny, nx), bool)
    solid[:solid_rows, :] = True
    phi, pr, pa = paper_wall_functions(solid, filter_mode)
    yb = analysis.surface_line(phi[:, 0], 0.5)
    rho_l, rho_v = 1.0, 0.1
    sims = []
    for R0, ga in cases:
        rho = W.droplet_density(nx, ny, [(nx / 2.0, yb + R0)], [R0], rho_l, rho_v, 3.0)
        s = Simulation(nx, ny, lattice=21, storage=storage, tau=tau, G=-1.0 / th, psi_kind=1,
                       project=True, eos=(0.25 * th, -0.25 * th, th, 0.222, 0.869))
        s.set_wall(phi, pr, pa, G_R, ga, 1.0)
        s.set_equilibrium(rho)
        sims.append(s)
    hist = [[] for _ in cases]

    def record(done):
        for k, s in enumerate(sims):
            rho, _, _ = s.moments()
            row = [done]
            for base in BASES:
                try:
                    row.append(analysis.contact_angle(rho, phi, rho_l, rho_v, y_max=ny - 10,
                                                      base=base).theta_deg)
                except Exception:
                    row.append(float("nan"))
            hist[k].append(tuple(row))

    t0 = time.perf_counter()
    _run_batch(sims, steps, chunk, record)
    wall = time.perf_counter() - t0
    rows = []
    for (R0, ga), h in zip(cases, hist):
        last, prev = h[-1], h[-2] if len(h) > 1 else h[-1]
        rows.append({"R0": R0, "G_A": ga,
                     "theta_deg": dict(zip(BASES, last[1:])),
                     "theta_change_last_chunk_deg": last[1] - prev[1], "history": h})
    for s in sims:
        s.close()
    return {"nx": nx, "ny": ny, "G_R": G_R, "steps": steps, "storage": storage,
            "filter_mode": filter_mode, "wall_s": wall, "y_surface": yb,
            "y_hydrodynamic": analysis.surface_line(phi[:, 0], 0.01), "rows": rows}


def paper_theta_table(steps: int = 100000, chunk: int = 20000, storage: str = "fp32",
                      nx: int = 650, ny: int = 150, R0: float = 50.0, G_R: float = 1.33,
                      tau: float = 1.0, solid_rows: int = 1, R0_others=(30.0, 65.0),
                      filter_mode: str = "iterate"):
    """The static angle against G_A at G_R = 1.33 (Sec. III B, Figs. 6-7) next
    to the printed angles, at R0 = ``R0``; and, for the angles the domain
    holds at every size (G_A = 0-0.7), at the drop sizes ``R0_others`` too
    (the paper reports no significant dependence on R0 = 30-80)."""
    cases = [(R0, ga) for ga in PAPER_THETA]
    cases += [(r, ga) for r in R0_others for ga in PAPER_THETA if ga <= 0.7]
    out = paper_drops(cases, steps=steps, chunk=chunk, storage=storage, nx=nx, ny=ny, G_R=G_R,
                      tau=tau, solid_rows=solid_rows, filter_mode=filter_mode)
    for r in out["rows"]:
        r["paper_theta_deg"] = PAPER_THETA[r["G_A"]]
        r["diff_deg"] = r["theta_deg"]["surface"] - PAPER_THETA[r["G_A"]]
    out["R0"] = R0
    return out


def _paper_sim(nx, ny, storage, tau, G_R, G_A, eps, phi, pr, pa, body=(0.0, 0.0)):
    th = 2.0 / 3.0
    s = Simulation(nx, ny, lattice=21, storage=storage, tau=tau, G=-1.0 / th, psi_kind=1,
                   project=True, eos=(0.25 * th, -0.25 * th, th, 0.222, 0.869), body_force=body)
    s.set_wall(phi, pr, pa, G_R, G_A, eps)
    return s


def dynamic_angles(steps_static: int = 60000, steps: int = 100000, chunk: int = 25000,
                   dps=(0.175e-4, 1.75e-4, 3.5e-4, 5.25e-4),
                   surfaces=((1.33, 0.5, 1.0), (0.9, 0.42, 1.0), (1.33, 0.57, 1.3)),
                   storage: str = "fp32", nx: int = 650, ny: int = 150, R0: float = 50.0,
                   tau: float = 1.0, gamma: float = 0.09, filter_mode: str = "iterate"):
    """Contact-angle dynamics of Sec. III C: each surface (G_R, G_A, epsilon)
    first relaxes a static drop; the relaxed populations then restart under a
    uniform force density dp / nx along +x (a pressure difference dp over the
    domain length).  Reported per run: droplet speed U (mass-weighted liquid
    velocity), Ca = U mu_L / gamma with mu_L = rho_L theta (tau - 1/2) and the
    paper's gamma = 0.09, and the advancing / receding angles from two circle
    fits, with their change over the last chunk."""
    import workloads as W
    th = 2.0 / 3.0
    solid = np.zeros((ny, nx), bool)
    solid[0, :] = True
    phi, pr, pa = paper_wall_functions(solid, filter_mode)
    yb = analysis.surface_line(phi[:, 0], 0.5)
    rho_l, rho_v = 1.0, 0.1
    mu_l = rho_l * th * (tau - 0.5)
    out = {"nx": nx, "ny": ny, "R0": R0, "tau": tau, "gamma": gamma, "storage": storage,
           "filter_mode": filter_mode, "steps_static": steps_static, "steps": steps, "runs": []}
    statics = []
    for (GR, GA, eps) in surfaces:
        s = _paper_sim(nx, ny, storage, tau, GR, GA, eps, phi, pr, pa)
        s.set_equilibrium(W.droplet_density(nx, ny, [(nx / 2.0, yb + R0)], [R0], rho_l, rho_v, 3.0))
        statics.append(s)
    _run_batch(statics, steps_static, steps_static)
    f0s = []
    for s, (GR, GA, eps) in zip(statics, surfaces):
        rho, _, _ = s.moments()
        c = analysis.contact_angle(rho, phi, rho_l, rho_v, y_max=ny - 10)
        f0s.append(s.populations())
        out["runs"].append({"G_R": GR, "G_A": GA, "epsilon": eps, "dp": 0.0,
                            "theta_static_deg": c.theta_deg})
        s.close()
    sims, meta = [], []
    for f0, (GR, GA, eps) in zip(f0s, surfaces):
        for dp in dps:
            s = _paper_sim(nx, ny, storage, tau, GR, GA, eps, phi, pr, pa, body=(dp / nx, 0.0))
            s.set_populations(f0)
            sims.append(s)
            meta.append((GR, GA, eps, dp))
    hist = {i: [] for i in range(len(sims))}

    def record(done):
        for i, s in enumerate(sims):
            rho, ux, uy = s.moments()
            try:
                d = analysis.dynamic_angles(rho, phi, rho_l, rho_v, y_max=ny - 10)
                U = analysis.drop_velocity(rho, ux, 0.5 * (rho_l + rho_v), phi)
                hist[i].append((done, d.theta_adv_deg, d.theta_rec_deg, U, d.theta_adv_hR_deg,
                                d.theta_rec_hR_deg))
            except Exception:
                hist[i].append((done,) + (float("nan"),) * 5)

    t0 = time.perf_counter()
    _run_batch(sims, steps, chunk, record)
    for i, (GR, GA, eps, dp) in enumerate(meta):
        h = hist[i]
        last, prev = h[-1], h[-2] if len(h) > 1 else h[-1]
        out["runs"].append({"G_R": GR, "G_A": GA, "epsilon": eps, "dp": dp, "U": last[3],
                            "Ca": last[3] * mu_l / gamma, "theta_adv_deg": last[1],
                            "theta_rec_deg": last[2], "theta_adv_hR_deg": last[4],
                            "theta_rec_hR_deg": last[5],
                            "theta_adv_change_last_chunk": last[1] - prev[1],
                            "theta_rec_change_last_chunk": last[2] - prev[2], "history": h})
        sims[i].close()
    out["wall_s"] = time.perf_counter() - t0
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["sweep", "slip", "large", "paper", "dynamic"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--storages", default=None, help="comma-separated storage modes")
    ap.add_argument("--size", default=None, help="lattice NXxNY (sweep, slip)")
    ap.add_argument("--filter", default=None, choices=["iterate", "mean"],
                    help="paper: reading of the Appendix filter")
    ap.add_argument("--surfaces", default=None,
                    help="dynamic: surfaces as 'G_R,G_A,eps;G_R,G_A,eps;...'")
    ap.add_argument("--out", default=None, help="also write the JSON object to this file")
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    kw = {}
    if args.steps is not None:
        kw["steps"] = args.steps
    if args.storages and args.which not in ("paper", "dynamic"):
        kw["storages"] = tuple(args.storages.split(","))
    if args.filter and args.which in ("paper", "dynamic"):
        kw["filter_mode"] = args.filter
    if args.surfaces and args.which == "dynamic":
        kw["surfaces"] = tuple(tuple(float(v) for v in t.split(","))
                               for t in args.surfaces.split(";"))
    if args.size and args.which in ("sweep", "slip"):
        kw["nx"], kw["ny"] = (int(v) for v in args.size.lower().split("x"))
    fn = {"sweep": contact_angle_sweep, "slip": slip_study, "large": large_precision,
          "paper": paper_theta_table, "dynamic": dynamic_angles}[args.which]
    res = fn(**kw)
    text = json.dumps(res, default=float)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
