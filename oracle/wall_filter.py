"""Recursive Gaussian filter for the wall functions (Appendix, Eq. iteration).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading of the Appendix formula: the printed outer sum over n_s would make the
iterate grow past one, so each pass is a single application of the lattice
filter to the previous iterate,

    G^(n)(x) = sum_i w_i G^(n-1)(x + r_i),      G^(0) = H (1 on solid nodes),

after which the iterate is reset to one on the solid nodes (the outer boundary
of the domain is solid bulk).  The lattice is periodic; a wall "at the domain
boundary" is the solid row(s) of the mask.  The paper's choice is
psi_R-bar = G^(5), psi_A-bar = G^(22) - G^(5), phi_S = G^(22).
"""
from __future__ import annotations

import numpy as np

from .lbm_oracle import Lattice


def filter_pass(lat: Lattice, g: np.ndarray) -> np.ndarray:
    out = np.zeros_like(g)
    for i, (cx, cy) in enumerate(lat.c):
        out = out + lat.w[i] * np.roll(g, shift=(-cy, -cx), axis=(0, 1))
    return out


def iterates(lat: Lattice, solid: np.ndarray, n_max: int):
    """[G^(0), ..., G^(n_max)] for a boolean solid mask [ny, nx]."""
    g = solid.astype(np.float64)
    out = [g.copy()]
    for _ in range(n_max):
        g = filter_pass(lat, g)
        g[solid] = 1.0
        out.append(g.copy())
    return out


def wall_functions(lat: Lattice, solid: np.ndarray, n_rep: int = 5, n_att: int = 22):
    """(phi_S, psi_R-bar, psi_A-bar) = (G^(n_att), G^(n_rep), G^(n_att) - G^(n_rep))."""
    its = iterates(lat, solid, max(n_rep, n_att))
    g_r = its[n_rep]
    g_a = its[n_att]
    return g_a.copy(), g_r.copy(), g_a - g_r
