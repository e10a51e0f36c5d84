"""Plain FP64 CPU oracle for the worm-LBM time step (Hammer, Fritz, Bedoya-Martinez,
arXiv 1911.00180).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this code.  Only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may call it.  It shares no code, tables or constants with the CUDA path:
every quantity here is recomputed from the paper in numpy float64, slowly and plainly.

Modules
-------
lattice   directions, angular weights, worm paths, Lambda_corr, W_corr, TAS schedule
          (Sec. 2.3-2.5: Eqs. algorithm, W-correction, weight, worm-paths).
stepper   framed-grid state, boundary conditions (Sec. 2.6), the step (Eqs. lbm-energy
          and algorithm), moments (Eqs. pseudo-T and q_corr) and FP64 reductions.
transport effective conductivity (apparent and central-band), steady-state temperature
          residual, Fuchs-Sondheimer reference ratios (Sec. 4.5).
adjoint   the exact transpose of one step and its reverse sweep (derived from Eq.
          lbm-energy; the paper has no adjoint), plus central finite differences.

Parity pinning status of each function is stated in its module header.
"""
