"""Batched solves of many small problems in one launch (mg_solve_batch)
against the oracle's direct solves and the graph-driven mg_solve, through
the C ABI (GB300 only).

A thread block solves one problem with the Krylov method of mg_solve (the
same iteration formulas; its dot products are block sums in another order),
so a batched solution is held to the same bounds as mg_solve's:
* against the oracle's direct solve (sparse LU of the condensed system, then
  H for the hanging values): <= 1e-9 relative in the lumped-mass L2 norm
  for the FP64 V-cycle, <= 1e-8 for the FP32 one, at rtol 1e-10;
* against mg_solve on the same input: the difference of two solutions that
  both reach rtol 1e-10, <= 2e-8 relative;
* the true residual, recomputed by the oracle, <= 1.01 rtol.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import workloads as W
from oracle import mesh as M
from oracle import problems as PB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402

TR = dict(eps=1e-3, beta=(1.0, 0.5))
EL = dict(mu=1.0, lam=10.0, dirichlet=(0x1,))

# name -> (leaf mesh, oracle problem, library problem, library options)
CASES = {
    "poisson16": (lambda: W.uniform_leaves(2, (1, 1), 4), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "poisson24": (lambda: W.uniform_leaves(2, (3, 3), 3), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "poisson64": (lambda: W.poisson64(64), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "poisson80": (lambda: W.uniform_leaves(2, (5, 5), 4), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "td_adaptive2": (lambda: W.td_adaptive(rounds=2, gamma=1.0), PB.Problem(PB.TRANSPORT, **TR),
                     dict(kind=B.MG_TRANSPORT, **TR), {}),
    "td_uniform24": (lambda: W.uniform_leaves(2, (3, 3), 3), PB.Problem(PB.TRANSPORT, **TR),
                     dict(kind=B.MG_TRANSPORT, **TR), {}),
    "poisson3d_8": (lambda: W.uniform_leaves(3, (1, 1, 1), 3), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "poisson3d_12": (lambda: W.uniform_leaves(3, (3, 3, 3), 2), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "poisson3d_16": (lambda: W.uniform_leaves(3, (1, 1, 1), 4), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "elasticity8": (lambda: W.uniform_leaves(3, (1, 1, 1), 3), PB.Problem(PB.ELASTICITY, **EL),
                    dict(kind=B.MG_ELASTICITY, **EL), dict(omega=0.5)),
}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def load(name, coords, nc):
    if name.startswith("td"):
        return W.f_transport(coords, TR["eps"], TR["beta"])
    if name.startswith("poisson"):
        return W.f_poisson(coords) if coords.shape[1] == 2 else np.ones(coords.shape[0])
    return np.tile([0.0, 0.0, -1.0], (coords.shape[0], 1)).ravel()


class Case:
    """A hierarchy of the library, the oracle's condensed system on the same
    mesh and its direct solution for the case's load."""

    def __init__(self, ctx, name, opts=None):
        mk, prob, pkw, okw = CASES[name]
        lm = mk()
        self.name, self.prob = name, prob
        self.h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(**{**okw, **(opts or {})}))
        fm = M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
        self.s = PB.build_system(fm, prob)
        self.f = load(name, fm.coords, prob.nc)
        self.b = self.s.rhs(self.f, None)
        self.xstar = self.s.H @ spl.spsolve(self.s.A.tocsc(), self.b)
        self.w = np.repeat(np.asarray(self.s.F.sum(axis=1)).ravel(), prob.nc)

    def err(self, x):
        return math.sqrt(np.sum(self.w * (x - self.xstar) ** 2) / np.sum(self.w * self.xstar ** 2))

    def true_rel_res(self, x, b=None):
        b = self.b if b is None else b
        xr = x.copy()
        xr[self.s.hang] = 0.0
        return np.linalg.norm(b - self.s.A @ xr) / np.linalg.norm(b[~self.s.fixed])


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cases(ctx):
    cs = {name: Case(ctx, name, dict(store_bf16=1)) for name in CASES}
    yield cs
    for c in cs.values():
        c.h.free()


def graph_solve(c, b, rtol, prec, x0=None):
    x = torch.zeros(c.h.n_dofs, device="cuda", dtype=torch.float64) if x0 is None else x0.clone()
    st = c.h.solve(b, x, rtol=rtol, max_it=400, prec=prec)
    assert st.status == 0, st.as_dict()
    return st, x.cpu().numpy()


SMEM = 226 * 1024          # shared memory of the staged tail


def vec_bytes(c, prec):
    """Bytes of the V-cycle vectors of every level (4 per level) at prec."""
    es = 8 if prec == B.MG_FP64 else 4
    nc = c.prob.nc
    return sum(4 * ((n * nc * es + 15) // 16 * 16) for n in c.h.level_nodes())


def fitting(cases, prec):
    return [n for n, c in cases.items() if c.h.batch_fits(prec)]


def test_fit_rule(cases):
    """A problem fits exactly when its V-cycle vectors (plus the level
    headers, under 8 KiB) fit in the 226 KiB of the staged tail; every case
    fits with the FP32 V-cycle."""
    for c in cases.values():
        for prec in (B.MG_FP64, B.MG_MIXED_FP32, B.MG_MIXED_BF16):
            vb = vec_bytes(c, prec)
            if vb + 8192 <= SMEM:
                assert c.h.batch_fits(prec), (c.name, prec, B.load_library().mg_last_error())
            if vb > SMEM:
                assert not c.h.batch_fits(prec), (c.name, prec)
        assert c.h.batch_fits(B.MG_MIXED_FP32)


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32, B.MG_MIXED_BF16])
def test_uneven_batch_matches_direct_and_mg_solve(ctx, cases, prec):
    """All cases in one batch (2D and 3D, scalar and 3-component, CG and
    BiCGStab, hanging nodes): each solution against the oracle's direct solve
    and against mg_solve on the same right-hand side."""
    names = fitting(cases, prec)
    assert len(names) >= 8
    cs = [cases[n] for n in names]
    bs = [dev(c.b) for c in cs]
    xs = [torch.zeros(c.h.n_dofs, device="cuda", dtype=torch.float64) for c in cs]
    rc, stats = ctx.solve_batch([c.h for c in cs], bs, xs, rtol=1e-10, max_it=400, prec=prec)
    assert rc == 0
    for c, b, x, st in zip(cs, bs, xs, stats):
        assert st.status == 0 and st.iters > 0, (c.name, st.as_dict())
        assert st.rel_res <= 1e-10
        xb = x.cpu().numpy()
        tol = 1e-9 if prec == B.MG_FP64 else 1e-8
        assert c.err(xb) <= tol, (c.name, c.err(xb))
        assert c.true_rel_res(xb) <= 1.01e-10, c.name
        assert np.array_equal(xb[c.s.dirichlet], c.b[c.s.dirichlet])
        gst, xg = graph_solve(c, b, 1e-10, prec)
        assert abs(gst.iters - st.iters) <= 2, (c.name, gst.iters, st.iters)
        assert np.linalg.norm(xb - xg) <= 2e-8 * np.linalg.norm(xg), c.name


def test_repeated_hierarchy_and_initial_guess(ctx, cases):
    """The same hierarchy several times in one batch, with different
    right-hand sides and initial guesses (the guess's fixed entries come from
    b, as in mg_solve); each result equals the problem solved alone."""
    c = cases["td_adaptive2"]
    rng = np.random.default_rng(21)
    k = 12
    scales = 1.0 + rng.random(k)
    bs = [dev(c.b * s) for s in scales]
    x0 = [dev(rng.standard_normal(c.h.n_dofs)) for _ in range(k)]
    xs = [x.clone() for x in x0]
    rc, stats = ctx.solve_batch([c.h] * k, bs, xs, rtol=1e-10, max_it=400, prec=B.MG_MIXED_FP32)
    assert rc == 0
    for i in range(k):
        xb = xs[i].cpu().numpy()
        assert stats[i].status == 0
        assert c.err(xb / scales[i]) <= 1e-8
        _, xg = graph_solve(c, bs[i], 1e-10, B.MG_MIXED_FP32, x0=x0[i])
        assert np.linalg.norm(xb - xg) <= 2e-8 * np.linalg.norm(xg)
    # a batch of copies of one problem gives identical bits in every copy
    xs2 = [torch.zeros(c.h.n_dofs, device="cuda", dtype=torch.float64) for _ in range(k)]
    ctx.solve_batch([c.h] * k, [bs[0]] * k, xs2, rtol=1e-10, max_it=400, prec=B.MG_MIXED_FP32)
    ref = xs2[0].cpu().numpy()
    for x in xs2[1:]:
        assert np.array_equal(x.cpu().numpy(), ref)


def test_nonhomogeneous_dirichlet_and_hanging(ctx, cases):
    """Dirichlet data g lifted into b by mg_assemble_rhs, hanging values
    filled by H: the batched solution equals the oracle's direct solve."""
    c = cases["td_adaptive2"]
    xy = c.h.coords()
    assert c.h.info.n_hanging > 0
    g = 1.0 + xy[:, 0] ** 2 - 0.5 * xy[:, 1]
    b = torch.empty(c.h.n_dofs, device="cuda", dtype=torch.float64)
    c.h.assemble_rhs(dev(c.f), b, dev(g))
    ref = c.s.rhs(c.f, g)
    xstar = c.s.H @ spl.spsolve(c.s.A.tocsc(), ref)
    x = torch.zeros_like(b)
    rc, stats = ctx.solve_batch([c.h], [b], [x], rtol=1e-10, max_it=400, prec=B.MG_MIXED_FP32)
    assert rc == 0
    xb = x.cpu().numpy()
    assert np.abs(xb - xstar).max() <= 1e-8 * np.abs(xstar).max()
    assert np.array_equal(xb[c.s.dirichlet], g[c.s.dirichlet])
    hang = c.s.hang
    assert np.abs(xb[hang] - (c.s.H @ np.where(hang, 0.0, xb))[hang]).max() <= 1e-14 * np.abs(xb).max()


def test_not_converged_status_and_empty_batch(ctx, cases):
    c = cases["poisson64"]
    b = dev(c.b)
    x = torch.zeros(c.h.n_dofs, device="cuda", dtype=torch.float64)
    rc, stats = ctx.solve_batch([c.h], [b], [x], rtol=1e-14, max_it=2, prec=B.MG_MIXED_FP32)
    assert rc == B.MG_ERR_NOT_CONVERGED and stats[0].status == B.MG_ERR_NOT_CONVERGED
    assert stats[0].iters == 2 and stats[0].rel_res > 1e-14
    rc, stats = ctx.solve_batch([], [], [], rtol=1e-8, max_it=10)
    assert rc == 0 and stats == []


def test_refuses_what_does_not_fit(ctx, cases):
    """A hierarchy whose V-cycle vectors exceed shared memory, or a GMRES
    problem, is refused before anything runs; the other outputs stay as
    they were."""
    big = G.Hierarchy(ctx, W.poisson64(256), B.make_problem(kind=B.MG_POISSON))
    try:
        assert not big.batch_fits(B.MG_MIXED_FP32)
        c = cases["poisson16"]
        x = torch.full((c.h.n_dofs,), 7.0, device="cuda", dtype=torch.float64)
        xb = torch.zeros(big.n_dofs, device="cuda", dtype=torch.float64)
        bb = torch.ones(big.n_dofs, device="cuda", dtype=torch.float64)
        with pytest.raises(B.MGError):
            ctx.solve_batch([c.h, big], [dev(c.b), bb], [x, xb], rtol=1e-8, max_it=50)
        assert bool((x == 7.0).all())
    finally:
        big.free()
    gm = G.Hierarchy(ctx, W.uniform_leaves(2, (1, 1), 4), B.make_problem(kind=B.MG_POISSON),
                     B.make_opts(krylov=B.MG_GMRES))
    try:
        assert not gm.batch_fits(B.MG_MIXED_FP32)
    finally:
        gm.free()
