"""Degenerate inputs of the method through the C ABI (GB300).

* One-level hierarchies: the mesh is its own coarsest level, so the V-cycle
  is the coarse direct solve alone (Sec. 2.2 with L = 0) and the Krylov
  solve must reach the direct solution in a step or two, in every precision,
  through the graph-driven solve and the batched one.
* No free dof: every node carries Dirichlet data.  The right-hand side is g,
  the solve returns x = g bit for bit after zero iterations.
* An exact initial guess: the solve stops at once and keeps it.

Expected values are the oracle's direct solves on the same meshes.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import workloads as W
from oracle import mg
from oracle import problems as PB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402

ONE_LEVEL = {
    # 9 nodes, 1 free
    "poisson2d": (lambda: W.uniform_leaves(2, (1, 1), 1), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON)),
    # 27 nodes, 1 free
    "poisson3d": (lambda: W.uniform_leaves(3, (1, 1, 1), 1), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON)),
    # 25 nodes, 9 free, SUPG on
    "transport": (lambda: W.uniform_leaves(2, (2, 2), 1), PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                  dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))),
    # 81 dofs, 54 free, 3x3 blocks
    "elasticity": (lambda: W.uniform_leaves(3, (1, 1, 1), 1),
                   PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                   dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,))),
}

NO_FREE = {
    # one cell, 4 nodes, all on the boundary
    "poisson2d": (lambda: W.uniform_leaves(2, (1, 1), 0), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON)),
    # one hexahedron clamped on all six faces
    "elasticity": (lambda: W.uniform_leaves(3, (1, 1, 1), 0),
                   PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x3F,)),
                   dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x3F,))),
}

PRECS = [B.MG_FP64, B.MG_MIXED_FP32, B.MG_MIXED_BF16]


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def build(ctx, table, name):
    mk, prob, pkw = table[name]
    lm = mk()
    oh = mg.Hierarchy(lm, prob)
    s = PB.build_system(oh.fine.mesh, prob)
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(store_bf16=1, autotune=0))
    return lm, prob, oh, s, h


@pytest.mark.parametrize("name", list(ONE_LEVEL))
def test_one_level_hierarchy_is_the_coarse_solve(ctx, name):
    lm, prob, oh, s, h = build(ctx, ONE_LEVEL, name)
    try:
        assert h.levels == 1 == len(oh.levels)
        assert h.info.n_free == int((~s.fixed).sum()) > 0
        rng = np.random.default_rng(20)
        f = rng.standard_normal(h.n_dofs)
        g = rng.standard_normal(h.n_dofs)
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(dev(f), b, dev(g))
        bref = s.rhs(f, g)
        assert np.abs(b.cpu().numpy() - bref).max() <= 1e-13 * np.abs(bref).max()
        xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
        scale = np.abs(xstar).max()
        fits = []
        for prec in PRECS:
            x = torch.zeros_like(b)
            st = h.solve(b, x, rtol=1e-12, max_it=20, prec=prec)
            assert st.status == 0, (prec, st.as_dict())
            # the preconditioner is A^-1 (FP64) or A^-1 applied in FP32 / to
            # BF16-rounded data: a step or two, a few more for the roundings
            assert 1 <= st.iters <= (1 if prec == B.MG_FP64 else 6), (prec, st.iters)
            assert np.abs(x.cpu().numpy() - xstar).max() <= 1e-10 * scale, prec
            if h.batch_fits(prec):
                fits.append(prec)
                xb = torch.zeros_like(b)
                rc, stats = ctx.solve_batch([h], [b], [xb], rtol=1e-12, max_it=20, prec=prec)
                assert rc == 0 and stats[0].status == 0, (prec, stats[0].as_dict())
                assert np.abs(xb.cpu().numpy() - xstar).max() <= 1e-10 * scale, prec
        assert B.MG_MIXED_FP32 in fits
    finally:
        h.free()


@pytest.mark.parametrize("name", list(NO_FREE))
def test_no_free_dof_returns_the_dirichlet_data(ctx, name):
    lm, prob, oh, s, h = build(ctx, NO_FREE, name)
    try:
        assert h.info.n_free == 0 and s.fixed.all()
        rng = np.random.default_rng(21)
        f = rng.standard_normal(h.n_dofs)
        g = rng.standard_normal(h.n_dofs)
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(dev(f), b, dev(g))
        assert np.array_equal(b.cpu().numpy(), g)
        assert np.array_equal(s.rhs(f, g), g)
        for prec in PRECS:
            x = dev(rng.standard_normal(h.n_dofs))      # any initial guess
            st = h.solve(b, x, rtol=1e-10, max_it=20, prec=prec)
            assert st.status == 0 and st.iters == 0, (prec, st.as_dict())
            assert np.array_equal(x.cpu().numpy(), g), prec
            if h.batch_fits(prec):
                xb = dev(rng.standard_normal(h.n_dofs))
                rc, stats = ctx.solve_batch([h], [b], [xb], rtol=1e-10, max_it=20, prec=prec)
                assert rc == 0 and stats[0].iters == 0, (prec, stats[0].as_dict())
                assert np.array_equal(xb.cpu().numpy(), g), prec
    finally:
        h.free()


def test_exact_initial_guess_stops_at_once(ctx):
    """x0 = the FP64 direct solution: the first residual already meets the
    tolerance, so no iteration runs and x0 comes back unchanged (its hanging
    entries recomputed from their parents)."""
    lm = W.td_adaptive(rounds=3, gamma=1.0)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    oh = mg.Hierarchy(lm, prob)
    s = PB.build_system(oh.fine.mesh, prob)
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)))
    try:
        f = np.random.default_rng(22).standard_normal(h.n_dofs)
        bref = s.rhs(f)
        xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
        for prec in (B.MG_FP64, B.MG_MIXED_FP32):
            x = dev(xstar)
            st = h.solve(dev(bref), x, rtol=1e-8, max_it=50, prec=prec)
            assert st.status == 0 and st.iters == 0, (prec, st.as_dict())
            xg = x.cpu().numpy()
            free = ~s.fixed
            # free entries untouched; hanging ones re-interpolated from them
            assert np.array_equal(xg[free], xstar[free]), prec
            assert np.abs(xg - xstar).max() <= 1e-14 * np.abs(xstar).max(), prec
    finally:
        h.free()
