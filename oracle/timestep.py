"""Oracle: backward-Euler time stepping of the transport-diffusion problem.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 5.1 of the paper: d_t theta - lambda Laplace theta + (b.grad) theta = f
on (0, T] x Omega, theta = theta_b on the boundary, theta(0) = theta_0,
discretised by Q1 in space and the backward Euler method in time (step dt),
one linear system per step with the same matrix (Algorithm "Nonstationary
Linear Problem": matrices assembled once, right-hand side and solve per step).

Step n (t_n = n dt), with M the consistent mass matrix and A the stationary
operator (``problems.Problem`` with mass = 0):

    (M / dt + A) theta_n = M theta_{n-1} / dt + M I_h f(t_n),

hanging nodes eliminated by H (Sec. 2.2) and the Dirichlet data theta_b(t_n)
eliminated symmetrically.  Both right-hand-side terms are one load vector
b = H^T F (theta_{n-1} / dt + I_h f(t_n)) of the nodal field in brackets
(F = M, plus the SUPG load when stabilised), since theta_{n-1} is itself a
Q1 function given by its nodal values.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse.linalg as spl

from . import problems as PB


def step_problem(prob: PB.Problem, dt: float) -> PB.Problem:
    """The backward-Euler step's problem: mass coefficient 1/dt."""
    return dataclasses.replace(prob, mass=1.0 / dt)


def run(mesh, prob: PB.Problem, dt: float, theta0, f_of_t, g_of_t, n_steps: int, solve=None):
    """theta_n for n = 1..n_steps on the nodes of `mesh` (all nodes, hanging
    values filled by H).  theta0: nodal values at t = 0; f_of_t(t), g_of_t(t):
    nodal source values and Dirichlet data at time t (arrays over the nodes;
    g may be None for homogeneous data).  solve(A, b) -> x, default a sparse
    LU factorisation of the step matrix reused for every step."""
    sp_ = step_problem(prob, dt)
    sysm = PB.build_system(mesh, sp_)
    if solve is None:
        lu = spl.splu(sysm.A.tocsc())
        solve = lambda A, b: lu.solve(b)   # noqa: E731
    theta = np.asarray(theta0, dtype=np.float64).copy()
    out = []
    for n in range(1, n_steps + 1):
        t = n * dt
        fn = f_of_t(t)
        fbar = theta / dt + (0.0 if fn is None else np.asarray(fn, dtype=np.float64))
        b = sysm.rhs(fbar, g_of_t(t))
        theta = sysm.H @ solve(sysm.A, b)
        out.append(theta)
    return sysm, out
