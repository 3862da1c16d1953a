"""Plain, slow FP64 CPU oracle for the GMG-preconditioned Krylov solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library may import, call
or link anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path: the only common module is the seeded
input generator ``workloads`` (leaf meshes, right-hand-side functions, random
vectors), which holds none of the method's arithmetic.

What it computes (paper: "An adaptive finite element multigrid solver using
GPU acceleration", arXiv:2405.05047):

* ``mesh``      Q1 node set, hanging-node matrix H_h (Sec. 2.2) and the global
                coarsening hierarchy (Sec. 2.2, Fig. "coarsening").
* ``fem``       Q1 element matrices by tensor Gauss quadrature (Sec. 2.1) for
                the Poisson, transport-diffusion (+SUPG), elasticity (Sec. 5.2)
                and Oseen (+LPS) forms, condensation H^T A H, Dirichlet rows.
* ``mg``        transfer matrices from the local embedding (Eq. "prolongation",
                Sec. 4.1.4), R = P^T, the (block-)Jacobi smoother
                x <- x + omega S (b - A x) (Sec. 4.1.4), the direct coarse solve
                and the V-cycle of Algorithm "Geometric multigrid solver".
* ``krylov``    CG, BiCGStab and restarted GMRES (Sec. 4.1.5, Saad 2003).
* ``timestep``  backward-Euler steps of the time-dependent transport-diffusion
                problem (Sec. 5.1; Algorithm "Nonstationary Linear Problem").

Every function states the passage it follows.  Pins (tests that tie this
code to facts other than itself) live in ``tests/test_oracle_*.py``.
Parity pinned for every function here except the contraction *value* of the
V-cycle (only its mesh independence is pinned) and iteration counts, which
the paper does not print ("parity unpinned" for those two quantities).
"""
