"""The C-ABI library: it builds, loads, exports every symbol include/lbm.h
declares, and its host-only paths (defaults, argument validation, the
closed-form wall helper) behave without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1202_6130_gb300 import build as b
    b.build()
    from paper_1202_6130_gb300 import _lib
    return _lib.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lbm_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1202_6130_gb300 import _lib
    declared = _declared()
    assert "lbm_step" in declared and "lbm_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_struct_sizes_match_header(lib):
    from paper_1202_6130_gb300 import _lib
    # 6 int32 + 8 doubles + 2 doubles + 1 double + 4 int32 -> 6*4 + 11*8 + 16 = 128 (aligned)
    assert ctypes.sizeof(_lib.lbm_params) == 128
    p = _lib.lbm_params()
    assert lib.lbm_params_default(ctypes.byref(p)) == 0
    assert p.nx == 128 and p.ny == 64 and p.lattice == 9 and p.storage == _lib.LBM_FP32
    assert p.rounding == _lib.LBM_ROUND_STOCHASTIC
    assert p.tau == 1.0 and p.G == -5.5 and p.eos_rho1 == 0.222 and p.eos_rho2 == 0.869


@pytest.mark.parametrize("field,value", [("tau", 0.5), ("nx", 0), ("lattice", 7), ("storage", 9),
                                         ("psi_kind", 3), ("rho0", 0.0), ("check_every", -1),
                                         ("rounding", 2)])
def test_create_rejects_invalid_parameters_without_touching_the_gpu(lib, field, value):
    from paper_1202_6130_gb300 import _lib
    p = _lib.lbm_params()
    lib.lbm_params_default(ctypes.byref(p))
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(p), None, None, ctypes.byref(ctx))
    assert rc == _lib.LBM_EINVAL
    assert not ctx.value
    assert lib.lbm_last_error(None)


def test_null_context_is_einval_and_destroy_null_is_ok(lib):
    from paper_1202_6130_gb300 import _lib
    assert lib.lbm_step(None, 1) == _lib.LBM_EINVAL
    assert lib.lbm_destroy(None) == _lib.LBM_OK
    assert lib.lbm_wall_gaussian_filter(0, 4, 9, None, 5, 22, None, None, None) == _lib.LBM_EINVAL


def test_core_tail_helper_matches_input_generator(lib):
    import paper_1202_6130_gb300 as pkg
    nx, ny = 37, 29
    d = W.wall_distance_slab(nx, ny)
    T = 3.0 + 1.5 * np.sin(2 * np.pi * 3 * np.arange(nx) / nx)
    a = pkg.wall_core_tail(d, T)
    b = W.wall_core_tail(d, T[None, :])
    for u, v in zip(a, b):
        # 1 - tanh(.) cancels: compare absolutely at the FP64 rounding level
        np.testing.assert_allclose(u, v, rtol=1e-14, atol=1e-15)


def test_allocator_failure_is_enomem(lib):
    """Failure injected through the allocator callback: the first request (a
    population buffer, made before the library touches a device) returns NULL;
    lbm_create reports LBM_ENOMEM, returns no context and holds no block."""
    fail_at = 1
    from paper_1202_6130_gb300 import _lib
    live, calls = set(), [0]

    def alloc(n, user):
        calls[0] += 1
        if calls[0] >= fail_at:
            return None
        p = 0x1000 * calls[0]          # a fake address; never dereferenced
        live.add(p)
        return p

    def free(p, user):
        live.discard(p)

    a = _lib.lbm_allocator(_lib.ALLOC_FN(alloc), _lib.FREE_FN(free), None)
    p = _lib.lbm_params()
    lib.lbm_params_default(ctypes.byref(p))
    ctx = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(p), ctypes.byref(a), None, ctypes.byref(ctx))
    assert rc == _lib.LBM_ENOMEM
    assert not ctx.value
    assert not live
    assert b"population buffer" in lib.lbm_last_error(None)
