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
    t = studies.paper_theta_table(steps=600, chunk=300, nx=160, ny=60, R0=15.0)
    assert len(t["rows"]) == len(studies.PAPER_THETA)
    assert all(np.isfinite(r["theta_deg"]) for r in t["rows"][:3])
    d = studies.dynamic_angles(steps_static=400, steps=400, chunk=200, dps=(3.5e-4,),
                               surfaces=((1.33, 0.5, 1.0),), nx=200, ny=60, R0=15.0)
    moving = [r for r in d["runs"] if r["dp"] > 0]
    assert len(moving) == 1 and moving[0]["U"] > 0.0 and np.isfinite(moving[0]["theta_adv_deg"])
