"""Serving: continuous batching of solves on resident hierarchies (GB300).

Requests of different problems and sizes are submitted while others run;
every result must be bitwise identical to the same solve run alone (fixed
reduction orders, no shared state between workspaces), the budget refuses
requests whose workspace can never fit, and queued requests can be cancelled.
"""
import time

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402


def rhs_of(h, seed):
    rng = np.random.default_rng(seed)
    f = torch.from_numpy(rng.standard_normal(h.n_dofs)).cuda()
    b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
    h.assemble_rhs(f, b)
    return b


def make_hiers(ctx):
    return [
        G.Hierarchy(ctx, W.poisson64(64), B.make_problem(kind=B.MG_POISSON)),
        G.Hierarchy(ctx, W.uniform_leaves(2, (1, 1), 5),
                    B.make_problem(kind=B.MG_TRANSPORT, eps=1e-2, beta=(1.0, 0.5))),
        G.Hierarchy(ctx, W.td_adaptive(rounds=4, gamma=1.0),
                    B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                    B.make_opts(krylov=B.MG_GMRES)),
        G.Hierarchy(ctx, W.uniform_leaves(3, (1, 1, 1), 3),
                    B.make_problem(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                    B.make_opts(omega=0.5)),
    ]


def wait(ctx, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            rc, st = ctx.poll(t)
            if rc != B.MG_PENDING:
                out[t] = (rc, st)
        assert time.time() - t0 < timeout, "serving requests did not finish"
        time.sleep(0.0005)
    return out


@pytest.mark.parametrize("prec", [B.MG_MIXED_FP32, B.MG_FP64])
def test_results_identical_alone_and_in_the_mix(prec):
    ctx = G.Context(0)
    hs = make_hiers(ctx)
    reqs = []
    for k in range(12):
        h = hs[k % len(hs)]
        reqs.append((h, rhs_of(h, 100 + k)))
    # alone: one synchronous solve each
    alone = []
    for h, b in reqs:
        x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        st = h.solve(b, x, rtol=1e-9, max_it=300, prec=prec)
        assert st.status == 0
        alone.append((x.cpu().numpy(), st.iters))
    # in the mix: all submitted at once, several in flight per hierarchy
    xs = [torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64) for h, _ in reqs]
    torch.cuda.synchronize()
    tickets = [ctx.submit(h, b, x, rtol=1e-9, max_it=300, prec=prec) for (h, b), x in zip(reqs, xs)]
    res = wait(ctx, tickets)
    for t, x, (xa, ita) in zip(tickets, xs, alone):
        rc, st = res[t]
        assert rc == 0 and st.iters == ita
        assert np.array_equal(x.cpu().numpy(), xa)
    for h in hs:
        h.free()
    ctx.close()


def test_admission_refuses_a_request_that_never_fits():
    probe = G.Context(0)
    h0 = G.Hierarchy(probe, W.poisson64(64), B.make_problem(kind=B.MG_POISSON))
    need, ws = h0.info.bytes_device, h0.info.bytes_workspace
    h0.free()
    probe.close()
    # budget: the hierarchy with its default workspace fits, a second workspace does not
    ctx = G.Context(0, hbm_budget_bytes=int(need + ws // 2))
    h = G.Hierarchy(ctx, W.poisson64(64), B.make_problem(kind=B.MG_POISSON))
    b = rhs_of(h, 1)
    x = torch.zeros_like(b)
    with pytest.raises(G.MGError) as e:
        ctx.submit(h, b, x)
    assert e.value.code == -3
    # the synchronous path still works on the resident workspace
    st = h.solve(b, x, rtol=1e-9)
    assert st.status == 0
    h.free()
    ctx.close()


def test_hierarchy_over_budget_is_refused():
    ctx = G.Context(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(G.MGError) as e:
        G.Hierarchy(ctx, W.poisson64(64), B.make_problem(kind=B.MG_POISSON))
    assert e.value.code == -3
    ctx.close()


def test_cancel_queued_request():
    ctx = G.Context(0)
    ctx.serve_config(1)
    h = G.Hierarchy(ctx, W.td_adaptive(rounds=5, gamma=1.0),
                    B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)))
    b = rhs_of(h, 3)
    xs = [torch.zeros_like(b) for _ in range(6)]
    tickets = [ctx.submit(h, b, x, rtol=1e-10) for x in xs]
    rc = ctx.cancel(tickets[-1])
    res = wait(ctx, tickets[:-1])
    assert all(r[0] == 0 for r in res.values())
    if rc == 0:
        rc2, _ = ctx.poll(tickets[-1])
        assert rc2 == B.MG_ERR_CANCELLED if hasattr(B, "MG_ERR_CANCELLED") else rc2 == -9
    with pytest.raises(G.MGError):
        G.binding._check(G.binding.load_library().mg_poll(ctx.handle, 987654321, None))
    h.free()
    ctx.close()


def test_mixed_solve_without_fp64_level_copies():
    """A hierarchy built with store_fp64 = 0 (no FP64 V-cycle) still keeps
    the finest FP64 operator, which the outer Krylov residual uses in every
    precision mode: its mixed solves equal the default hierarchy's bit for
    bit, synchronously and through mg_submit / mg_poll, and really iterate.
    An FP64 solve on it is refused."""
    ctx = G.Context(0)
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    hd = G.Hierarchy(ctx, lm, pb)
    hn = G.Hierarchy(ctx, lm, pb, B.make_opts(store_fp64=0))
    b = rhs_of(hd, 11)
    xd = torch.zeros_like(b)
    sd = hd.solve(b, xd, rtol=1e-9, max_it=300, prec=B.MG_MIXED_FP32)
    assert sd.status == 0 and sd.iters > 0 and sd.rel_res <= 1e-9
    xn = torch.zeros_like(b)
    sn = hn.solve(b, xn, rtol=1e-9, max_it=300, prec=B.MG_MIXED_FP32)
    assert sn.status == 0 and sn.iters == sd.iters and sn.rel_res == sd.rel_res
    assert torch.equal(xn, xd)
    xs = [torch.zeros_like(b) for _ in range(3)]
    torch.cuda.synchronize()
    tickets = [ctx.submit(hn, b, x, rtol=1e-9, max_it=300, prec=B.MG_MIXED_FP32) for x in xs]
    res = wait(ctx, tickets)
    for t, x in zip(tickets, xs):
        rc, st = res[t]
        assert rc == 0 and st.iters == sd.iters
        assert torch.equal(x, xd)
    with pytest.raises(G.MGError) as e:
        hn.solve(b, torch.zeros_like(b), prec=B.MG_FP64)
    assert e.value.code == -1
    hd.free()
    hn.free()
    ctx.close()


def test_reserved_slots_bound_the_workspaces():
    """mg_serve_reserve allocates the slots and builds their graphs up front;
    with 2 reserved slots 8 requests on one hierarchy still all finish (they
    wait for a free slot instead of allocating), bitwise equal to the solve
    alone."""
    ctx = G.Context(0)
    h = G.Hierarchy(ctx, W.td_adaptive(rounds=4, gamma=1.0),
                    B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)))
    ctx.serve_reserve(h, 2, B.MG_MIXED_FP32)
    b = rhs_of(h, 21)
    xa = torch.zeros_like(b)
    st = h.solve(b, xa, rtol=1e-9, max_it=300, prec=B.MG_MIXED_FP32)
    assert st.status == 0
    xs = [torch.zeros_like(b) for _ in range(8)]
    torch.cuda.synchronize()
    tickets = [ctx.submit(h, b, x, rtol=1e-9, max_it=300, prec=B.MG_MIXED_FP32) for x in xs]
    res = wait(ctx, tickets)
    for t, x in zip(tickets, xs):
        assert res[t][0] == 0 and torch.equal(x, xa)
    with pytest.raises(G.MGError):
        ctx.serve_reserve(h, 0)
    h.free()
    ctx.close()


@pytest.mark.parametrize("prec", [B.MG_MIXED_FP32, B.MG_FP64])
def test_batched_serving_equals_batch_alone(prec):
    """With batching on (every fitting request batched), a served request's
    result equals mg_solve_batch of that request alone bit for bit, whatever
    else was in its launch; requests that do not fit (GMRES) take the graph
    path and equal mg_solve."""
    ctx = G.Context(0)
    hs = make_hiers(ctx)
    fits = [h.batch_fits(prec) for h in hs]
    assert fits == [True, True, False, True]
    reqs = []
    for k in range(16):
        h = hs[k % len(hs)]
        reqs.append((h, rhs_of(h, 200 + k)))
    alone = []
    for h, b in reqs:
        x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        if h.batch_fits(prec):
            rc, (st,) = ctx.solve_batch([h], [b], [x], rtol=1e-9, max_it=300, prec=prec)
        else:
            st = h.solve(b, x, rtol=1e-9, max_it=300, prec=prec)
        assert st.status == 0
        alone.append((x.cpu().numpy(), st.iters))
    ctx.serve_batching(256, 1)
    xs = [torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64) for h, _ in reqs]
    torch.cuda.synchronize()
    tickets = [ctx.submit(h, b, x, rtol=1e-9, max_it=300, prec=prec) for (h, b), x in zip(reqs, xs)]
    res = wait(ctx, tickets)
    for t, x, (xa, ita) in zip(tickets, xs, alone):
        rc, st = res[t]
        assert rc == 0 and st.iters == ita
        assert np.array_equal(x.cpu().numpy(), xa)
    # a lone fitting request below min_batch takes the graph path
    ctx.serve_batching(256, 4)
    h, b = reqs[0]
    xg = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(b, xg, rtol=1e-9, max_it=300, prec=prec)
    x = torch.zeros_like(xg)
    t = ctx.submit(h, b, x, rtol=1e-9, max_it=300, prec=prec)
    rc, st2 = wait(ctx, [t])[t]
    assert rc == 0 and torch.equal(x, xg) and st2.iters == st.iters
    with pytest.raises(G.MGError):
        ctx.serve_batching(-1, 1)
    for h in hs:
        h.free()
    ctx.close()


def test_first_batched_use_inside_the_scheduler():
    """Fresh hierarchies whose batched-kernel data (the staged image of every
    level) is first built by the scheduler and read by a launch on one of its
    non-blocking streams: the image is complete before the launch, so every
    request converges and equals the same request solved alone afterwards."""
    ctx = G.Context(0)
    hs = [G.Hierarchy(ctx, W.uniform_leaves(2, (m, m), 3), B.make_problem(kind=B.MG_POISSON))
          for m in (1, 3, 5, 7, 9)]
    hs += [G.Hierarchy(ctx, W.uniform_leaves(3, (m, m, m), 2), B.make_problem(kind=B.MG_POISSON))
           for m in (1, 3, 5)]
    ctx.serve_batching(256, 1)
    reqs = [(h, rhs_of(h, 300 + k)) for k, h in enumerate(hs * 4)]
    xs = [torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64) for h, _ in reqs]
    torch.cuda.synchronize()
    tickets = [ctx.submit(h, b, x, rtol=1e-9, max_it=300) for (h, b), x in zip(reqs, xs)]
    res = wait(ctx, tickets)
    ctx.serve_batching(0, 1)
    for t, (h, b), x in zip(tickets, reqs, xs):
        rc, st = res[t]
        assert rc == 0 and st.iters > 0 and st.launches <= 2, st.as_dict()
        xa = torch.zeros_like(x)
        rc2, (st2,) = ctx.solve_batch([h], [b], [xa], rtol=1e-9, max_it=300)
        assert st2.iters == st.iters and torch.equal(xa, x)
    for h in hs:
        h.free()
    ctx.close()
