"""lbm_reduce3_noalloc, the reduction for callers that must not allocate
device memory while they run (fixed-budget real-time loops, code inside a
memory pool it does not own): its sums of rho and j + F/2 must equal those of
lbm_totals (the mass bit for bit: the same kernels and partition), on two
calls in a row that reuse its fixed scratch array.

Collected last on purpose, so that a run stopping at the first failure has
already run every other test."""
import ctypes
import math

import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _device_sums(pkg, lib, sim, torch):
    rho, ux, uy = sim.moments_device()
    px = (rho * ux).contiguous()
    py = (rho * uy).contiguous()
    out = torch.zeros(3, dtype=torch.float64, device=rho.device)
    stream = torch.cuda.current_stream()
    rc = lib.lbm_reduce3_noalloc(ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(px.data_ptr()),
                                 ctypes.c_void_p(py.data_ptr()), rho.numel(),
                                 ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.lbm_last_error(None)
    return out.cpu().numpy()


def test_noalloc_reduction_matches_lbm_totals_on_two_calls():
    import torch
    torch.cuda.set_device(0)
    import paper_1202_6130_gb300 as pkg
    from paper_1202_6130_gb300 import _lib
    lib = _lib.load()
    # 600 x 320 = 192000 nodes
    w = W.droplet_on_wall(nx=600, ny=320, R=60.0)
    sim = pkg.Simulation.from_workload(w, storage="fp64")
    sim.step(20)
    for _ in range(2):
        want = sim.totals()
        got = _device_sums(pkg, lib, sim, torch)
        # the same rho array through the same kernels and partition: the same bits
        assert got[0] == want[0]
        assert abs(got[1] - want[1]) <= 1e-10 and abs(got[2] - want[2]) <= 1e-10
        sim.step(15)
    sim.close()


def test_noalloc_reduction_rejects_a_negative_length_and_a_null_output():
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import _lib
    lib = _lib.load()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = lib.lbm_reduce3_noalloc(None, None, None, -1, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _lib.LBM_EINVAL
    assert b"negative length" in lib.lbm_last_error(None)
    rc = lib.lbm_reduce3_noalloc(None, None, None, 5, None, None)
    assert rc == _lib.LBM_EINVAL


def test_noalloc_reduction_null_arrays_and_empty_input():
    """A NULL array sums to zero and n = 0 writes zeros (the start-up call
    that loads the scratch array on a device)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import _lib
    lib = _lib.load()
    a = torch.linspace(0.5, 2.0, 70001, dtype=torch.float64, device="cuda")
    out = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    rc = lib.lbm_reduce3_noalloc(ctypes.c_void_p(a.data_ptr()), None, None, a.numel(),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0, lib.lbm_last_error(None)
    got = out.cpu().numpy()
    want = float(a.sum().item())
    assert abs(got[0] - want) <= 1e-13 * abs(want) and got[1] == 0.0 and got[2] == 0.0
    out.fill_(7.0)
    rc = lib.lbm_reduce3_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                 None, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0, lib.lbm_last_error(None)
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0]


def test_noalloc_reduction_captures_into_a_graph_and_replays():
    """After the start-up call, a call captured into a CUDA graph in global
    capture mode (where any device allocation during capture fails the
    capture) replays to the right sums: the entry point neither allocates nor
    synchronises once its scratch array is loaded."""
    import torch
    torch.cuda.set_device(0)
    from paper_1202_6130_gb300 import _lib
    lib = _lib.load()
    n = 150001
    a = torch.linspace(0.25, 3.0, n, dtype=torch.float64, device="cuda")
    b = torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device="cuda") ** 3
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = lib.lbm_reduce3_noalloc(None, None, None, 0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        rc = lib.lbm_reduce3_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                     None, n, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.lbm_last_error(None)
    for scale in (1.0, 2.0):
        a.mul_(scale)
        out.fill_(7.0)
        g.replay()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        wa = math.fsum(a.cpu().numpy().tolist())   # correctly rounded sums
        wb = math.fsum(b.cpu().numpy().tolist())
        assert abs(got[0] - wa) <= 1e-13 * abs(wa)
        assert abs(got[1] - wb) <= 1e-12
        assert got[2] == 0.0
