"""Oracle: backward-Euler time stepping (transport-diffusion, Sec. 5.1;
elastodynamics as a first-order system, Sec. 5.2).

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


def run_first_order(mesh, prob: PB.Problem, dt: float, u0, v0, f_of_t, g_of_t, n_steps: int):
    """Backward Euler for d_t^2 u - div sigma(u) = f written, as in Sec. 5.2,
    as the first-order system d_t u - v = 0, d_t v - div sigma(u) = f in the
    unknowns (u, v).  Step n solves the coupled system on the free dofs
    (hanging dofs eliminated by H, Dirichlet dofs prescribed):

        M (u_n - u_{n-1}) / dt - M v_n = 0,
        M (v_n - v_{n-1}) / dt + K u_n = F_n,

    K the stiffness of `prob` (mass 0), M the consistent mass on every
    component, F_n the load of the nodal f(t_n).  On Dirichlet dofs
    u_n = g(t_n) and v_n = (g(t_n) - g(t_{n-1})) / dt, the first equation
    there.  Returns the system and [(u_n, v_n)] on all nodes (hanging values
    by H).  Sparse LU of the 2n x 2n block matrix, factored once."""
    import scipy.sparse as sp

    from . import fem
    S = PB.build_system(mesh, prob)
    nc = prob.nc
    H = S.H
    Mraw = fem.expand(S.F, nc)
    Kc = (H.T @ S.A_raw @ H).tocsr()
    Mc = (H.T @ Mraw @ H).tocsr()
    free = np.nonzero(~S.fixed)[0]
    dirl = np.nonzero(S.dirichlet)[0]
    Kff, Kfd = Kc[free][:, free], Kc[free][:, dirl]
    Mff, Mfd = Mc[free][:, free], Mc[free][:, dirl]
    big = sp.bmat([[Mff / dt, -Mff], [Kff, Mff / dt]]).tocsc()
    lu = spl.splu(big)
    nf = free.size
    u = np.asarray(u0, dtype=np.float64).ravel().copy()
    v = np.asarray(v0, dtype=np.float64).ravel().copy()
    g_prev = u[dirl].copy()
    vd_prev = v[dirl].copy()
    out = []
    for n in range(1, n_steps + 1):
        t = n * dt
        g = g_of_t(t)
        g = np.zeros(dirl.size) if g is None else np.asarray(g, dtype=np.float64).ravel()[dirl]
        vd = (g - g_prev) / dt
        fn = f_of_t(t)
        Fn = (H.T @ (Mraw @ np.asarray(fn, dtype=np.float64).ravel()))[free] if fn is not None else 0.0
        rhs = np.concatenate([Mff @ u[free] / dt,
                              Fn + Mff @ v[free] / dt - Mfd @ (vd - vd_prev) / dt - Kfd @ g])
        sol = lu.solve(rhs)
        ut = np.zeros(u.size)
        vt = np.zeros(v.size)
        ut[free], vt[free] = sol[:nf], sol[nf:]
        ut[dirl], vt[dirl] = g, vd
        u, v = H @ ut, H @ vt
        g_prev, vd_prev = g, vd
        out.append((u, v))
    return S, out
