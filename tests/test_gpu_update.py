"""mg_update_problem: new coefficients on a resident hierarchy (GB300).

After the update, every solve path (the graph-driven solve in both
precisions, the batched solve, a serving request on a reserved slot) must
equal the same solve on a hierarchy set up from scratch with the new problem
bit for bit: the re-assembly rewrites the same values into the same layouts,
and stale copies (the small-level images, the damping carried by cached
graphs) would show up as differing bits.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mesh as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    c.close()


def rhs(h, seed):
    rng = np.random.default_rng(seed)
    f = torch.from_numpy(rng.standard_normal(h.n_dofs)).cuda()
    b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
    h.assemble_rhs(f, b)
    return b


def solve(h, b, prec, rtol=1e-10):
    x = torch.zeros_like(b)
    st = h.solve(b, x, rtol=rtol, max_it=400, prec=prec)
    assert st.status == 0
    return st.iters, x


def oseen_case():
    lm = W.oseen_channel(1, 2)
    fm = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    kw = dict(dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01)
    return lm, [B.make_problem(kind=B.MG_OSEEN, conv=W.oseen_beta(fm.coords, seed=s), **kw) for s in (1, 2)], {}


CASES = {
    "transport": lambda: (W.td_adaptive(rounds=4, gamma=1.0),
                          [B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                           B.make_problem(kind=B.MG_TRANSPORT, eps=2e-2, beta=(-0.3, 1.0), supg_delta0=0.3)], {}),
    "poisson_step": lambda: (W.poisson64(64), [B.make_problem(kind=B.MG_POISSON, mass=10.0),
                                               B.make_problem(kind=B.MG_POISSON, mass=500.0)], {}),
    "elasticity": lambda: (W.uniform_leaves(3, (1, 1, 1), 4),
                           [B.make_problem(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                            B.make_problem(kind=B.MG_ELASTICITY, mu=2.0, lam=100.0, dirichlet=(0x1,))], {}),
    "oseen_vanka": lambda: (*oseen_case()[:2], dict(smoother=B.MG_SMOOTHER_VANKA)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_update_equals_fresh_setup(ctx, name):
    lm, (p1, p2), okw = CASES[name]()
    opts = B.make_opts(autotune=0, store_bf16=1, **okw)
    h = G.Hierarchy(ctx, lm, p1, opts)
    fresh = G.Hierarchy(ctx, lm, p2, opts)
    try:
        precs = (B.MG_FP64, B.MG_MIXED_FP32, B.MG_MIXED_BF16)
        b1 = rhs(h, 1)
        for prec in precs:            # solve graphs of the old problem are cached now
            solve(h, b1, prec)
        h.update_problem(p2)
        assert h.info.n_free == fresh.info.n_free
        assert list(h.info.level_omega[:h.levels]) == list(fresh.info.level_omega[:fresh.levels])
        b2, b2f = rhs(h, 2), rhs(fresh, 2)
        assert torch.equal(b2, b2f)   # the load matrix was re-assembled too
        for prec in precs:
            it, x = solve(h, b2, prec)
            itf, xf = solve(fresh, b2f, prec)
            assert it == itf and torch.equal(x, xf), (name, prec)
        if h.batch_fits(B.MG_MIXED_FP32):
            xa, xb = torch.zeros_like(b2), torch.zeros_like(b2)
            ctx.solve_batch([h], [b2], [xa], rtol=1e-10, max_it=400)
            ctx.solve_batch([fresh], [b2f], [xb], rtol=1e-10, max_it=400)
            assert torch.equal(xa, xb)
    finally:
        h.free()
        fresh.free()


def test_update_keeps_serving_reservations(ctx):
    lm = W.td_adaptive(rounds=3, gamma=1.0)
    p1 = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    p2 = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-1, beta=(1.0, 0.5))
    h = G.Hierarchy(ctx, lm, p1)
    fresh = G.Hierarchy(ctx, lm, p2)
    try:
        ctx.serve_reserve(h, 2, B.MG_MIXED_FP32)
        h.update_problem(p2)
        b = rhs(h, 3)
        xs = [torch.zeros_like(b) for _ in range(4)]
        torch.cuda.synchronize()
        ts = [ctx.submit(h, b, x, rtol=1e-9, max_it=300) for x in xs]
        done = {}
        while len(done) < len(ts):
            for t in ts:
                if t not in done:
                    rc, st = ctx.poll(t)
                    if rc != B.MG_PENDING:
                        done[t] = rc
        assert all(rc == 0 for rc in done.values())
        _, xf = solve(fresh, rhs(fresh, 3), B.MG_MIXED_FP32, rtol=1e-9)
        for x in xs:
            assert torch.equal(x, xf)
    finally:
        h.free()
        fresh.free()


def test_update_refuses_structural_changes(ctx):
    h = G.Hierarchy(ctx, W.poisson64(64), B.make_problem(kind=B.MG_POISSON))
    try:
        with pytest.raises(B.MGError):
            h.update_problem(B.make_problem(kind=B.MG_TRANSPORT, eps=1.0))
        with pytest.raises(B.MGError):
            h.update_problem(B.make_problem(kind=B.MG_POISSON, dirichlet=(0x1,)))
        # still usable, unchanged
        b = rhs(h, 4)
        solve(h, b, B.MG_MIXED_FP32)
    finally:
        h.free()
