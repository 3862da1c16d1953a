"""Pins of the backward-Euler transport-diffusion oracle (the paper's Sec. 5.1
problem) against facts other than itself: exactness on solutions that are
linear in space and time (hanging nodes, with and without SUPG), first-order
convergence in dt to the paper's manufactured solution, the mass term, and
the source term against finite differences of the exact solution."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mesh as M
from oracle import problems as PB
from oracle import timestep as TS


def q1mesh(lm):
    return M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)


@pytest.mark.parametrize("supg", [0.0, 0.5])
def test_backward_euler_exact_for_linear_space_time_solutions(supg):
    """theta = a + c.x + d t lies in the discrete space at every step and
    backward Euler differentiates it exactly in time, so the discrete
    solution equals it at every node after every step: f = d + beta.grad theta,
    Dirichlet data theta(t_n).  With SUPG the stabilisation must test the
    whole residual, the mass part included."""
    lm = W.td_adaptive(rounds=3, gamma=1.0, base_level=4)
    m = q1mesh(lm)
    assert m.hanging.sum() > 0
    beta = (1.0, 0.5)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=beta, supg_delta0=supg)
    a, c, d = 0.3, (1.2, -0.7), 0.9
    xy = m.coords
    lin = lambda t: a + c[0] * xy[:, 0] + c[1] * xy[:, 1] + d * t   # noqa: E731
    f = d + beta[0] * c[0] + beta[1] * c[1]
    dt = 0.1
    _, thetas = TS.run(m, prob, dt, lin(0.0), lambda t: np.full(m.n_nodes, f), lin, 5)
    for n, th in enumerate(thetas, 1):
        assert np.abs(th - lin(n * dt)).max() <= 1e-12


def test_time_stepping_converges_first_order_in_dt():
    """The paper's problem (lambda = 0.01, b = (0, -1)) against its exact
    solution at T = 0.16 on a 32 x 32 mesh: backward Euler is first order,
    so halving dt halves the error (the Q1 space error of this smooth
    solution, about 2e-5, stays far below the time error)."""
    m = q1mesh(W.td_uniform(32))
    xy = m.coords
    prob = PB.Problem(PB.TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B, supg_delta0=0.0)
    T = 0.16
    errs = []
    for dt in (0.04, 0.02, 0.01):
        _, th = TS.run(m, prob, dt, W.td_theta(0.0, xy), lambda t: W.td_source(t, xy),
                       lambda t: W.td_theta(t, xy), int(round(T / dt)))
        errs.append(np.abs(th[-1] - W.td_theta(T, xy)).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.15), (errs, ratios)


def test_source_term_matches_finite_differences():
    rng = np.random.default_rng(5)
    xy = rng.uniform(0.1, 0.9, size=(20, 2))
    e = 1e-4
    for t in (0.0, 0.37, 1.5):
        dth = (W.td_theta(t + e, xy) - W.td_theta(t - e, xy)) / (2 * e)
        gx = (W.td_theta(t, xy + [e, 0]) - W.td_theta(t, xy - [e, 0])) / (2 * e)
        gy = (W.td_theta(t, xy + [0, e]) - W.td_theta(t, xy - [0, e])) / (2 * e)
        lap = sum((W.td_theta(t, xy + s) - 2 * W.td_theta(t, xy) + W.td_theta(t, xy - s)) / e ** 2
                  for s in ([e, 0], [0, e]))
        f = dth - W.TD_LAMBDA * lap + W.TD_B[0] * gx + W.TD_B[1] * gy
        assert np.abs(f - W.td_source(t, xy)).max() <= 1e-6


def test_mass_term_adds_scaled_mass_matrix():
    """The step matrix minus the stationary one is s M (no SUPG), with M the
    pinned Q1 mass matrix: an interior row of s M has (s h^2 / 36) {16, 4, 1}."""
    m = q1mesh(W.td_uniform(8))
    s = 50.0
    p0 = PB.Problem(PB.TRANSPORT, eps=0.01, beta=(0.0, -1.0), supg_delta0=0.0)
    A0 = PB.build_system(m, p0, with_load=False).A_raw
    A1 = PB.build_system(m, TS.step_problem(p0, 1.0 / s), with_load=False).A_raw
    D = (A1 - A0).tocsr()
    h = 1.0 / 8
    i = int(np.nonzero((m.X[:, 0] == 4) & (m.X[:, 1] == 4))[0][0])
    row = D.getrow(i)
    for j, v in zip(row.indices, row.data):
        dist = int(np.abs(m.X[j] - m.X[i]).sum())
        assert v == pytest.approx(s * {0: 16, 1: 4, 2: 1}[dist] * h * h / 36, rel=1e-13)


# ---------------------------------------------------------------- elastodynamics (Sec. 5.2)
def _el_prob(dirichlet=(0x3F,)):
    return PB.Problem(PB.ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=dirichlet)


def test_first_order_elasticity_exact_for_linear_space_time_motion():
    """u = a + C x + d t (v = d) has a constant stress and no acceleration, so
    with f = 0 and Dirichlet data u(t_n) on every face the backward-Euler
    steps of the first-order system reproduce it at every node, hanging ones
    included, on the edge-refined mesh of Sec. 5.2."""
    m = q1mesh(W.elasticity_adaptive("edge", 2))
    assert m.hanging.sum() > 0
    xyz = m.coords
    a = np.array([0.1, -0.2, 0.05])
    C = np.array([[0.3, 0.1, -0.2], [0.0, -0.4, 0.25], [0.15, 0.2, 0.1]])
    d = np.array([0.7, -0.3, 0.4])
    lin = lambda t: (a + xyz @ C.T + d * t).ravel()   # noqa: E731
    dt = 0.025
    _, out = TS.run_first_order(m, _el_prob(), dt, lin(0.0), np.tile(d, m.n_nodes), lambda t: None, lin, 4)
    for n, (u, v) in enumerate(out, 1):
        assert np.abs(u - lin(n * dt)).max() <= 1e-11
        # v carries the rounding of the stiff block system (K ~ 1e4 h against M / dt ~ 40 h^3)
        assert np.abs(v - np.tile(d, m.n_nodes)).max() <= 1e-5


def test_first_order_elasticity_energy_decays():
    """f = 0, homogeneous data: backward Euler dissipates the energy
    (v, v)_M / 2 + (K u, u) / 2 in every step."""
    m = q1mesh(W.elasticity_adaptive("vertex", 2))
    prob = _el_prob()
    xyz = m.coords
    bump = np.prod(np.sin(np.pi * xyz), axis=1)
    u0 = np.stack([bump, 0.5 * bump, -bump], axis=1).ravel() * 1e-3
    S, out = TS.run_first_order(m, prob, W.EL_DT, u0, np.zeros_like(u0), lambda t: None, lambda t: None, 5)
    from oracle import fem
    M3 = fem.expand(S.F, 3)
    K = S.A_raw
    energy = [0.5 * u0 @ (K @ u0)] + [0.5 * v @ (M3 @ v) + 0.5 * u @ (K @ u) for u, v in out]
    assert all(b < a for a, b in zip(energy[:-1], energy[1:])), energy


def test_first_order_elasticity_tends_to_the_static_solution():
    """With a constant load the backward-Euler iteration is damped and its
    fixed point is the static problem K u = F: after many long steps u equals
    the static solution of the (pinned) elasticity operator."""
    m = q1mesh(W.elasticity_adaptive("vertex", 2))
    prob = _el_prob()
    f = np.tile(W.EL_F, m.n_nodes)
    S, out = TS.run_first_order(m, prob, 2.0, np.zeros(3 * m.n_nodes), np.zeros(3 * m.n_nodes),
                                lambda t: f, lambda t: None, 60)
    import scipy.sparse.linalg as spl
    ustat = S.H @ spl.spsolve(S.A.tocsc(), S.rhs(f))
    u = out[-1][0]
    assert np.abs(u - ustat).max() <= 1e-8 * np.abs(ustat).max()
