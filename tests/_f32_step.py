"""A float32 restatement of the D2Q9 step, for a CPU test of how FP32 rounding
accumulates over many steps.

Test helper only (not the oracle and not the product): every quantity of the
step is held in float32 and every operation rounds to float32, in the order
the fused FP32 kernel evaluates it (pair form of the EDM-BGK collision, the
rest population from the mass balance, fused multiply-adds where the kernel
fuses).  A fused multiply-add is emulated exactly: the product of two float32
values is exact in float64, so float64 a*b + c rounded once to float32 differs
from a true fused operation only when the float64 sum itself rounds (rare,
and at 2^-53).  The reciprocal of rho can be biased by one unit in the last
place to show what a one-sided reciprocal does to the accumulated error.
"""
from __future__ import annotations

import numpy as np

from oracle import lbm_oracle as O

f32 = np.float32
CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
W = (4 / 9,) + (1 / 9,) * 4 + (1 / 36,) * 4


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * b + c).astype(f32)


def _nb(a, cx, cy):
    return np.roll(a, shift=(-cy, -cx), axis=(0, 1))


def run(w, steps: int, rcp_bias: int = 0) -> np.ndarray:
    """Populations after `steps` float32 steps of workload `w` (D2Q9,
    exponential psi, static wall).  rcp_bias: 0 for the correctly rounded
    1/rho, +1 for one unit above it, -1 for one unit below."""
    p = O.Params(lattice=O.D2Q9, tau=w.tau, G=w.G, rho0=w.rho0)
    f = O.initial_populations(p, w.rho, w.ux, w.uy, w.noise).astype(f32)
    psi_fs = w.G_A * w.psi_a - w.G_R * w.psi_r
    Sx = sum(W[i] * _nb(psi_fs, CX[i], CY[i]) * CX[i] for i in range(9)).astype(f32)
    Sy = sum(W[i] * _nb(psi_fs, CX[i], CY[i]) * CY[i] for i in range(9)).astype(f32)
    phie = (w.phi_s ** w.epsilon).astype(f32)
    nx = w.rho.shape[1]
    wallnode = (phie != 0) | (Sx != 0) | (Sy != 0)
    flag = np.zeros_like(wallnode)
    for c0 in range(0, nx, 32):                     # wall terms per 32-column chunk
        flag[:, c0:c0 + 32] = wallnode[:, c0:c0 + 32].any(axis=1)[:, None]
    g, om, G = f32(1 - 1 / w.tau), f32(1 / w.tau), f32(w.G)
    w1, w5 = f32(1 / 9), f32(1 / 36)
    for _ in range(steps):
        rho = f[0].copy()
        for i in range(1, 9):
            rho = (rho + f[i]).astype(f32)
        psi = (f32(1) - np.exp(-rho).astype(f32)).astype(f32)
        d57, d86 = f[5] - f[7], f[8] - f[6]
        jx = ((f[1] - f[3]) + d57) + d86
        jy = ((f[2] - f[4]) + d57) - d86
        inv = (f32(1) / rho).astype(f32)
        if rcp_bias:
            inv = np.nextafter(inv, f32(np.inf) if rcp_bias > 0 else f32(0))
        ux, uy = jx * inv, jy * inv
        sfx = np.zeros_like(rho)
        sfy = np.zeros_like(rho)
        for cy in (-1, 0, 1):
            pm, p0, pp = _nb(psi, -1, cy), _nb(psi, 0, cy), _nb(psi, 1, cy)
            if cy == 0:
                sfx = _fma(pp - pm, w1, sfx)
            else:
                sg = f32(cy)
                sfy = _fma(p0, sg * w1, sfy)
                sfy = _fma(pp + pm, sg * w5, sfy)
                sfx = _fma(pp - pm, w5, sfx)
        mg = -G * psi
        ffx, ffy = mg * sfx, mg * sfy
        rp = rho * phie
        Fxw = (ffx + rho * Sx) + rp * ((f32(0) - ux) - ffx * inv)
        Fyw = (ffy + rho * Sy) + rp * ((f32(0) - uy) - ffy * inv)
        Fx = np.where(flag, Fxw, _fma(mg, sfx, f32(0))).astype(f32)
        Fy = np.where(flag, Fyw, _fma(mg, sfy, f32(0))).astype(f32)
        usx, usy = _fma(Fx, inv, ux), _fma(Fy, inv, uy)
        ax3, ay3 = _fma(-g, ux, usx) * f32(3), _fma(-g, uy, usy) * f32(3)
        us2, u2 = _fma(usy, usy, usx * usx), _fma(uy, uy, ux * ux)
        wB = _fma(_fma(-g, u2, us2), f32(-1.5), om)
        out = np.empty_like(f)
        for i, j in ((1, 3), (2, 4), (5, 7), (6, 8)):
            def cd(a, b):
                if CX[i] and CY[i]:
                    return (CX[i] * a + CY[i] * b).astype(f32)
                return (CX[i] * a if CX[i] else CY[i] * b).astype(f32)
            cs, cu, ca = cd(usx, usy), cd(ux, uy), cd(ax3, ay3)
            wr = f32(W[i]) * rho
            t = _fma(-g, cu * cu, cs * cs)
            sb = _fma(t, f32(4.5), wB)
            out[i] = _fma(g, f[i], wr * (sb + ca))
            out[j] = _fma(g, f[j], wr * (sb - ca))
        moving = out[1].copy()
        for i in range(2, 9):
            moving = moving + out[i]
        out[0] = rho - moving
        for i in range(9):
            f[i] = np.roll(out[i], shift=(CY[i], CX[i]), axis=(0, 1))
    return f
