"""The continuous-batching server: results are the same, bit for bit, whether
a request runs alone or in the mix, and admission respects the HBM budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests(serve):
    R = serve.Request
    return [R(0, 0.0, "droplet", 96, 48, 300, G_A=0.02), R(1, 0.0, "channel", 40, 64, 450),
            R(2, 0.0, "droplet", 200, 100, 150, G_A=0.1, tau=0.8), R(3, 0.0, "channel", 16, 96, 600, epsilon=1.3),
            R(4, 0.0, "droplet", 130, 70, 520, G_R=0.05), R(5, 0.0, "droplet", 64, 32, 90)]


def test_results_equal_alone_and_in_the_mix():
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import serve
    reqs = _requests(serve)
    alone = {r.id: r for r in serve.run_sequential(reqs, storage="fp32", realtime=False,
                                                   keep_fields=True)}
    # budget for about three requests at a time: requests queue and join later
    budget = 3.2 * max(serve.footprint_bytes(r.nx, r.ny, "fp32") for r in reqs)
    srv = serve.Server(storage="fp32", hbm_budget=budget, quantum=70, keep_fields=True)
    mixed = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.id for r in mixed) == list(range(len(reqs)))
    admits = sorted(r.t_admit for r in mixed)
    assert admits[-1] > admits[0]            # some requests waited for memory
    for r in mixed:
        a = alone[r.id]
        np.testing.assert_array_equal(r.rho, a.rho)
        np.testing.assert_array_equal(r.ux, a.ux)
        assert (np.isnan(r.value) and np.isnan(a.value)) or r.value == a.value
        assert r.t_done >= r.t_admit >= r.t_arrival
