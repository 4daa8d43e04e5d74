"""FP64 CPU oracle for the pseudo-potential wetting lattice-Boltzmann update.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (no tables, no helpers, no headers).

Contents:
  lbm_oracle   -- the time step, restated from Sec. II (Eqs. BE-BGK, feqc, M0-M2,
                  f2, force_SC, force_SC_FS, EOS, pseudopotential, wall_shift)
  wall_filter  -- the recursive Gaussian filter for the wall functions (Appendix)
"""
