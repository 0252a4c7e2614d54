"""FP64 CPU oracle of the MRT finite-difference lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain restatement of
the paper's method (Chen, Xu, Zhang & Li, "Prandtl number effects in MRT
lattice Boltzmann models for shocked and unshocked compressible fluids",
arXiv:1106.0785) that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with ``paper_1106_0785_gb300`` and imports
nothing from it.

Modules
-------
d2v16        velocity set (Sec. II, Fig. 1) and moment matrix M (Sec. II)
equilibrium  equilibrium moments, Eqs. 14a-14i and versions 1-3 (Sec. II)
fdlb         the time step: boundaries, macroscopic recovery, collision with
             the modified energy-flux relaxation, Lax-Wendroff advection,
             forward-Euler update (Sec. II, Eq. 3; scheme read from the
             amplification matrix G of Sec. III)
riemann      exact Riemann solver and Rankine-Hugoniot states for gamma = 2
couette      closed-form thermal Couette temperature profile (Sec. IV A)
stability    the amplification matrix G(k) of Sec. III
cfdlb        the same time step as plain C loops (fdlb_c.c, built with gcc
             -O3) for the periodic, outflow and inflow sides, pinned against
             fdlb step by step; the bench's CPU legs time it

Every function works on numpy arrays of float64; the step also accepts
complex128 so that a complex-step derivative (Squire & Trapp 1998) gives the
exact tangent of the step.

Parity unpinned: the values of equilibrium version 2 (see ``equilibrium``);
every other function is pinned by the tests in ``tests/test_oracle_*.py``.
"""
