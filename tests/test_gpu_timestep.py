"""Backward-Euler time stepping on the device (mg_time_steps) against the
oracle's time loop (GB300 only).

The paper's Sec. 5.1 problem (lambda = 0.01, b = (0, -1), dt = 0.02, exact
solution theta_ex) on a 64 x 64 mesh: after every step the library's theta_n
matches the oracle's (sparse LU per step) to 1e-9 (FP64 V-cycle, rtol 1e-10)
or 1e-8 (FP32 V-cycle) in the relative lumped-mass L2 norm, and one call over
all steps gives the same bits as one call per step.  On an adaptive mesh with
SUPG the solutions that are linear in space and time are reproduced at every
node.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mesh as M
from oracle import problems as PB
from oracle import timestep as TS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def q1mesh(lm):
    return M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)


def paper_problem(dt):
    prob = PB.Problem(PB.TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B, supg_delta0=0.0)
    pb = B.make_problem(kind=B.MG_TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B, supg_delta0=0.0, mass=1.0 / dt)
    return prob, pb


@pytest.mark.parametrize("krylov", [B.MG_GMRES, B.MG_BICGSTAB])
@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_time_steps_match_oracle(ctx, prec, krylov):
    dt, steps = W.TD_DT, 8
    lm = W.td_uniform(64)
    prob, pb = paper_problem(dt)
    m = q1mesh(lm)
    xy = m.coords
    S, ref = TS.run(m, prob, dt, W.td_theta(0.0, xy), lambda t: W.td_source(t, xy),
                    lambda t: W.td_theta(t, xy), steps)
    w = np.asarray(S.F.sum(axis=1)).ravel()
    h = G.Hierarchy(ctx, lm, pb, B.make_opts(krylov=krylov))
    try:
        assert np.array_equal(h.coords(), xy)
        f = dev(np.stack([W.td_source((k + 1) * dt, xy) for k in range(steps)]))
        g = dev(np.stack([W.td_theta((k + 1) * dt, xy) for k in range(steps)]))
        th1 = dev(W.td_theta(0.0, xy))
        tol = 1e-9 if prec == B.MG_FP64 else 1e-8
        for k in range(steps):          # one call per step
            rc, sts = h.time_steps(th1, f[k], g[k], 1, rtol=1e-10, max_it=100, prec=prec)
            assert rc == 0 and sts[0].status == 0 and sts[0].iters > 0 and sts[0].rel_res <= 1e-10
            e = th1.cpu().numpy() - ref[k]
            rel = np.sqrt(np.sum(w * e * e) / np.sum(w * ref[k] ** 2))
            assert rel <= tol, (k, rel)
            assert np.array_equal(th1.cpu().numpy()[S.dirichlet], W.td_theta((k + 1) * dt, xy)[S.dirichlet])
        th = dev(W.td_theta(0.0, xy))   # one call for all steps
        rc, sts = h.time_steps(th, f, g, steps, rtol=1e-10, max_it=100, prec=prec)
        assert rc == 0 and len(sts) == steps and all(s.status == 0 for s in sts)
        assert torch.equal(th, th1)
    finally:
        h.free()


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_time_steps_linear_solution_exact_with_supg(ctx, prec):
    """theta = 0.3 + 1.2 x - 0.7 y + 0.9 t, SUPG (eps = 1e-3, beta = (1, 0.5))
    with its mass part, hanging nodes: every step reproduces theta(t_n)."""
    lm = W.td_adaptive(rounds=3, gamma=1.0, base_level=4)
    dt = 0.1
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5), mass=1.0 / dt))
    try:
        assert h.info.n_hanging > 0
        xy = h.coords()
        lin = lambda t: 0.3 + 1.2 * xy[:, 0] - 0.7 * xy[:, 1] + 0.9 * t   # noqa: E731
        steps = 5
        f = dev(np.full((steps, h.n_dofs), 0.9 + 1.2 - 0.35))
        g = dev(np.stack([lin((k + 1) * dt) for k in range(steps)]))
        th = dev(lin(0.0))
        rc, sts = h.time_steps(th, f, g, steps, rtol=1e-11, max_it=100, prec=prec)
        assert rc == 0 and all(s.iters > 0 for s in sts)
        assert np.abs(th.cpu().numpy() - lin(steps * dt)).max() <= 1e-8
    finally:
        h.free()


def test_time_steps_need_a_mass_term(ctx):
    h = G.Hierarchy(ctx, W.td_uniform(16), B.make_problem(kind=B.MG_TRANSPORT, eps=0.01, beta=(0.0, -1.0)))
    try:
        th = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        with pytest.raises(G.MGError) as e:
            h.time_steps(th, None, None, 1)
        assert e.value.code == -1
    finally:
        h.free()


def test_time_steps_zero_steps_and_homogeneous_data(ctx):
    """No steps leave theta untouched; with f = g = NULL (no source,
    homogeneous Dirichlet data) the solution decays in the consistent-mass
    norm: testing a step with theta_n gives ||theta_n||_M^2 / dt +
    lambda ||grad theta_n||^2 = (theta_{n-1}, theta_n)_M / dt, since the
    divergence-free transport term is skew on functions that vanish on the
    boundary."""
    lm = W.td_uniform(32)
    F = PB.build_system(q1mesh(lm), PB.Problem(PB.POISSON)).F
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B,
                                            supg_delta0=0.0, mass=50.0))
    try:
        xy = h.coords()
        th0 = np.sin(np.pi * xy[:, 0]) * np.sin(np.pi * xy[:, 1])
        th = dev(th0)
        rc, sts = h.time_steps(th, None, None, 0)
        assert rc == 0 and sts == [] and np.array_equal(th.cpu().numpy(), th0)
        mnorm = lambda v: float(np.sqrt(v @ (F @ v)))   # noqa: E731
        norms = [mnorm(th0)]
        for _ in range(4):
            rc, _ = h.time_steps(th, None, None, 1, rtol=1e-10)
            assert rc == 0
            norms.append(mnorm(th.cpu().numpy()))
        assert all(b < a * (1.0 - 1e-3) for a, b in zip(norms[:-1], norms[1:])), norms
    finally:
        h.free()


# ---------------------------------------------------------------- elastodynamics (Sec. 5.2)
def el_problem(dt, dirichlet=(0x3F,)):
    prob = PB.Problem(PB.ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=dirichlet)
    pb = B.make_problem(kind=B.MG_ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=dirichlet, mass=1.0 / dt ** 2)
    return prob, pb


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_time_steps2_match_first_order_oracle(ctx, prec):
    """Sec. 5.2 on the edge-refined mesh (level 3, 4129 nodes, hanging nodes):
    the library solves the step for u with the matrix M/dt^2 + K and recovers
    v; the oracle solves the coupled first-order system in (u, v).  Every
    step agrees in u and v (relative lumped-mass L2)."""
    dt, steps = W.EL_DT, 4
    lm = W.elasticity_adaptive("edge", 3)
    prob, pb = el_problem(dt)
    m = q1mesh(lm)
    nd = 3 * m.n_nodes
    f = np.tile(W.EL_F, m.n_nodes)
    S, ref = TS.run_first_order(m, prob, dt, np.zeros(nd), np.zeros(nd), lambda t: f, lambda t: None, steps)
    w = np.repeat(np.asarray(S.F.sum(axis=1)).ravel(), 3)
    h = G.Hierarchy(ctx, lm, pb, B.make_opts(krylov=B.MG_CG))
    try:
        assert np.array_equal(h.coords(), m.coords) and h.info.n_hanging > 0
        u = torch.zeros(nd, device="cuda", dtype=torch.float64)
        v = torch.zeros_like(u)
        fd = dev(np.tile(f, (steps, 1)))
        # v is the difference quotient (u_n - u_{n-1}) / dt: its error is
        # measured on the scale of u / dt, since u_n - u_{n-1} cancels
        tol = 1e-8 if prec == B.MG_FP64 else 1e-7
        mnorm = lambda a: np.sqrt(np.sum(w * a * a))   # noqa: E731
        for k in range(steps):
            rc, sts = h.time_steps2(u, v, fd[k], None, 1, dt, rtol=1e-11, max_it=200, prec=prec)
            assert rc == 0 and sts[0].iters > 0
            uref, vref = ref[k]
            eu = mnorm(u.cpu().numpy() - uref) / mnorm(uref)
            ev = mnorm(v.cpu().numpy() - vref) / (mnorm(uref) / dt)
            assert eu <= tol and ev <= 4 * tol, (k, eu, ev)
    finally:
        h.free()


def test_time_steps2_linear_motion_exact(ctx):
    """u = a + C x + d t, v = d, f = 0, Dirichlet data u(t_n) on every face,
    face-refined mesh with hanging nodes: reproduced at every node."""
    dt, steps = W.EL_DT, 3
    lm = W.elasticity_adaptive("face", 3)
    _, pb = el_problem(dt)
    h = G.Hierarchy(ctx, lm, pb, B.make_opts(krylov=B.MG_CG))
    try:
        xyz = h.coords()
        a = np.array([0.1, -0.2, 0.05])
        C = np.array([[0.3, 0.1, -0.2], [0.0, -0.4, 0.25], [0.15, 0.2, 0.1]])
        d = np.array([0.7, -0.3, 0.4])
        lin = lambda t: (a + xyz @ C.T + d * t).ravel()   # noqa: E731
        u = dev(lin(0.0))
        v = dev(np.tile(d, h.n_nodes))
        g = dev(np.stack([lin((k + 1) * dt) for k in range(steps)]))
        rc, sts = h.time_steps2(u, v, None, g, steps, dt, rtol=1e-12, max_it=300)
        assert rc == 0
        assert np.abs(u.cpu().numpy() - lin(steps * dt)).max() <= 1e-9
        assert np.abs(v.cpu().numpy() - np.tile(d, h.n_nodes)).max() <= 1e-6
    finally:
        h.free()


def test_time_steps2_need_the_matching_mass(ctx):
    _, pb = el_problem(0.05)
    h = G.Hierarchy(ctx, W.elasticity_adaptive("vertex", 2), pb)
    try:
        u = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        with pytest.raises(G.MGError) as e:
            h.time_steps2(u, torch.zeros_like(u), None, None, 1, 0.025)
        assert e.value.code == -1
        rc, _ = h.time_steps2(u, torch.zeros_like(u), None, None, 1, 0.05)
        assert rc == 0
    finally:
        h.free()
