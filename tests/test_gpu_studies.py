"""The study drivers run end to end at small sizes and return finite values
(their full-size results are in the design notes)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def studies():
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import studies as S
    return S


def test_contact_angle_sweep_small(studies):
    out = studies.contact_angle_sweep(storages=("fp64", "fp32", "fp16s-rn"), steps=400, chunk=200,
                                      n_tail=2, nx=128, ny=64, R=20.0)
    for st in ("fp64", "fp32", "fp16s-rn"):
        th = out["storages"][st]["theta_deg"]
        assert len(th) == 2 and all(0.0 < t < 180.0 for t in th), (st, th)
    assert max(abs(e) for e in out["storages"]["fp32"]["theta_err_vs_fp64_deg"]) < 0.5


def test_slip_study_small(studies):
    out = studies.slip_study(storages=("fp64", "bf16s"), ny=48, steps=2000, chunk=1000)
    for st, d in out["storages"].items():
        for eps, r in d.items():
            assert math.isfinite(r["slip_length"]) and r["u_max"] > 0.0, (st, eps, r)


def test_paper_profile_and_dynamic_angles_small(studies):
    t = studies.paper_theta_table(steps=600, chunk=300, nx=160, ny=60, R0=15.0, R0_others=())
    assert len(t["rows"]) == len(studies.PAPER_THETA)
    assert all(np.isfinite(r["theta_deg"]["surface"]) for r in t["rows"][:3])
    d = studies.dynamic_angles(steps_static=400, steps=400, chunk=200, dps=(3.5e-4,),
                               surfaces=((1.33, 0.5, 1.0),), nx=200, ny=60, R0=15.0)
    moving = [r for r in d["runs"] if r["dp"] > 0]
    assert len(moving) == 1 and moving[0]["U"] > 0.0 and np.isfinite(moving[0]["theta_adv_deg"])


def test_reduced_precision_keeps_angle_and_slip(studies):
    """The precision target: FP16S and BF16S storage (FP32 arithmetic) keep the
    static contact angle within 0.5 degrees and the slip length within 2% of
    FP64 storage (itself equal to the oracle to 1e-12).  Drops: 96x48, R = 15,
    three tail strengths, 12k steps (the angle moves < 0.02 degrees over the
    last 3k).  Channels: 1024x96, liquid-filled, body force 1e-6, epsilon 1 and
    1.3, 60k steps (the FP64 slip length moves < 0.1% over the last 15k); the
    profile is averaged over all 1024 columns, as in the full-width channel."""
    drops = studies.contact_angle_sweep(storages=("fp64", "fp16s", "bf16s"), steps=12000,
                                        chunk=3000, n_tail=3, nx=96, ny=48, R=15.0)
    for st in ("fp16s", "bf16s"):
        err = drops["storages"][st]["theta_err_vs_fp64_deg"]
        assert len(err) == 3 and max(abs(e) for e in err) < 0.5, (st, err)
    chg = drops["storages"]["fp64"]["theta_change_last_chunk_deg"]
    assert max(abs(c) for c in chg) < 0.1, chg
    slip = studies.slip_study(storages=("fp64", "fp16s", "bf16s"), nx=1024, ny=96, steps=60000,
                              chunk=15000)
    for eps, r in slip["storages"]["fp64"].items():
        h = [v[1] for v in r["history"]]
        assert abs(h[-1] - h[-2]) < 1e-3 * abs(h[-1]), (eps, h)
    for st in ("fp16s", "bf16s"):
        for eps, r in slip["storages"][st].items():
            assert abs(r["slip_rel_err_vs_fp64"]) < 0.02, (st, eps, r["slip_rel_err_vs_fp64"])


def test_paper_theta_table_trend_offset_and_drop_size(studies):
    """The paper's fluid and walls (D2Q21, Eq. EOS, projection, Appendix wall
    functions, G_R = 1.33, 650x150), 40k steps (the angles at G_A <= 0.7 are
    then within 0.1 degree of their 100k-step values).

    * Trend (Sec. III B): the static angle falls as G_A grows.
    * Magnitude: the adopted force readings give angles 8-35 degrees below the
      printed 150 / 112 / 58.7 / 36.7 degrees at G_A = 0-0.7, and none of the
      three base lines for the height h (solid surface, the domain's outer
      boundary, the bottom liquid-vapour interface) brings every angle within
      5 degrees of the table: parity with the printed magnitudes is unpinned,
      and this test records by how much.
    * Drop size (Sec. III B: no significant dependence on R0 = 30-80): at
      R0 = 30, 50 and 65 the angles agree within 7 degrees or 10%."""
    out = studies.paper_theta_table(steps=40000, chunk=20000)
    th = {(r["R0"], r["G_A"]): r["theta_deg"] for r in out["rows"]}
    paper = studies.PAPER_THETA
    low = (0.0, 0.2, 0.5, 0.7)
    main = [th[(50.0, ga)]["surface"] for ga in low]
    assert all(a > b for a, b in zip(main, main[1:])), main
    assert th[(50.0, 0.8)]["surface"] < main[-1] and th[(50.0, 0.9)]["surface"] < main[-1]
    for ga, t in zip(low, main):
        assert 8.0 <= paper[ga] - t <= 35.0, (ga, t, paper[ga])
    for base in studies.BASES:
        worst = max(abs(th[(50.0, ga)][base] - paper[ga]) for ga in low)
        assert worst > 5.0, (base, worst)
    for ga in low:
        v = [th[(r0, ga)]["surface"] for r0 in (30.0, 50.0, 65.0)]
        assert max(v) - min(v) <= max(7.0, 0.1 * float(np.mean(v))), (ga, v)


def test_printed_angles_lie_between_two_readings_of_the_wall_filter(studies):
    """The Appendix filter prints an outer sum over passes.  Read as one filter
    pass per iterate (the oracle's and the library's reading) the drops wet
    more than the paper reports; read as the mean of the iterates G^(1)..G^(N)
    they wet less: at every G_A of Sec. III B the printed angle lies strictly
    between the two (R0 = 50, 650x150, 40k steps)."""
    gas = (0.0, 0.2, 0.5, 0.7, 0.9)
    cases = [(50.0, ga) for ga in gas]
    it = studies.paper_drops(cases, steps=40000, chunk=20000, filter_mode="iterate")
    mn = studies.paper_drops(cases, steps=40000, chunk=20000, filter_mode="mean")
    for ga, a, b in zip(gas, it["rows"], mn["rows"]):
        lo, hi = a["theta_deg"]["surface"], b["theta_deg"]["surface"]
        assert lo < studies.PAPER_THETA[ga] < hi, (ga, lo, studies.PAPER_THETA[ga], hi)
    # the hydrodynamic boundary (phi_S = 0.01), printed as y_w = 8.5: 9.8 and 7.9
    assert it["y_hydrodynamic"] > 8.5 > mn["y_hydrodynamic"]
