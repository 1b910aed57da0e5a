"""FP64 CPU oracle for the half-range Gauss-Hermite lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (``paper_1708_03249_gb300/csrc``): quadratures, kernels
``K``, equilibria, grids and the time step are all re-derived here from the
paper (arXiv:1708.03249, "Implementation of the force term in half-range
lattice Boltzmann models"), plainly and slowly.

Modules
-------
quadrature  half-range Hermite polynomials and quadrature (Sec. IV.B.1, App. B,
            Eqs. (4.14)-(4.19) "eq:hh_quad", "eq:wk_half"), full-range
            Gauss-Hermite quadrature (Sec. IV.A.1, "eq:H_quad", "eq:H_wk");
            built in 80-digit ``decimal`` arithmetic.
model       the discrete force matrices K^h (Eq. "eq:hh_Kk_hh") and K^H
            (Eq. "eq:H_Kk"), the projected equilibria (Eqs. "eq:hh_gk",
            "eq:H_gk") and the direct-product velocity set (App. A).
highorder   the half-range quadrature and K^h at orders up to 200 (the
            HHLB(20;200) model of Sec. V) by the Golub-Welsch recurrence of the
            Cholesky-factorised Hankel matrix in mpmath (2.5 Q + 60 digits);
            order 200 stored to 40 digits (tests/golden), so that the oracle
            needs no mpmath for it; K^h from the stored recurrence in FP64.
ballistic   the free-streaming reference profiles of Sec. V and eps_max.
hydrodynamic  the Navier-Stokes (Chapman-Enskog) profiles of Sec. V
            (Eqs. "eq:NS_temp", "eq:NS_n", "eq:NS_q").
solver      grid (Eqs. "eq:x_eta", "eq:etai"), WENO-5 without epsilon
            (Sec. IV.C.2, Tab. "weno"), 2nd-order upwind, diffuse-reflection
            walls (Sec. IV.C.3), BGK with tau = Kn/n (Eq. "eq:tau"), the TVD
            RK-3 step (Eq. "eq:rk3") and the macroscopic moments
            (Eq. "eq:fmoms").

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute-force integrals, library routines, exact
identities of the paper); see ``tests/test_oracle_*.py``.
"""
