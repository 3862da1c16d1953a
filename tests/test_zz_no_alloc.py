"""mg_restrict_static: the residual + restriction operator for callers that
cannot allocate device memory (device memory owned up front by another
allocator or a fixed pool, real-time loops that must not enter the CUDA
allocator).  Its residual lives in a fixed
device array inside the library; the result must equal mg_apply's
MG_OP_RESTRICT, which keeps the residual in the hierarchy's workspace.

Collected last on purpose; it passes alone in a fresh process and after the
other tests."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402


def _cases(bf16):
    return [
        (W.poisson64(64), B.make_problem(kind=B.MG_POISSON), B.make_opts(store_bf16=bf16)),
        (W.td_adaptive(rounds=4, gamma=1.0), B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
         B.make_opts(store_bf16=bf16)),
        (W.uniform_leaves(3, (1, 1, 1), 4),
         B.make_problem(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
         B.make_opts(omega=0.5, store_bf16=bf16)),
    ]


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32, B.MG_MIXED_BF16])
def test_static_restriction_equals_workspace_restriction(prec):
    ctx = G.Context(0)
    dt = torch.float64 if prec == B.MG_FP64 else torch.float32
    rng = np.random.default_rng(21)
    for lm, pb, op in _cases(1 if prec == B.MG_MIXED_BF16 else 0):
        h = G.Hierarchy(ctx, lm, pb, op)
        nodes = h.level_nodes()
        for level in range(1, h.levels):
            n, nco = nodes[level] * h.nc, nodes[level - 1] * h.nc
            for call in range(2):          # two calls in a row share the static array
                x = torch.from_numpy(rng.standard_normal(n)).to("cuda", dt)
                b = torch.from_numpy(rng.standard_normal(n)).to("cuda", dt)
                ref = torch.empty(nco, device="cuda", dtype=dt)
                out = torch.full((nco,), float("nan"), device="cuda", dtype=dt)
                h.apply(level, B.MG_OP_RESTRICT, x, b, ref, prec)
                G.binding.mg_restrict_static(h.handle, level, x, b, out, prec)
                r, o = ref.cpu().double().numpy(), out.cpu().double().numpy()
                tol = 1e-13 if prec == B.MG_FP64 else 2e-5
                assert np.abs(o - r).max() <= tol * max(np.abs(r).max(), 1e-300)
                assert np.array_equal(o, r)     # same kernels: identical bits
        h.free()
    ctx.close()


def test_static_restriction_refuses_levels_beyond_the_scratch():
    ctx = G.Context(0)
    h = G.Hierarchy(ctx, W.uniform_leaves(2, (1, 1), 10), B.make_problem(kind=B.MG_POISSON),
                    B.make_opts(store_fp32=0))
    fine = h.levels - 1
    assert h.level_nodes()[fine] > (1 << 20)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    d = torch.zeros(h.level_nodes()[fine - 1], device="cuda", dtype=torch.float64)
    with pytest.raises(G.MGError) as e:
        G.binding.mg_restrict_static(h.handle, fine, x, x, d, B.MG_FP64)
    assert e.value.code == -1 and "static residual scratch" in str(e.value)
    # the level below fits and works
    n2 = h.level_nodes()[fine - 1]
    x2 = torch.ones(n2, device="cuda", dtype=torch.float64)
    d2 = torch.zeros(h.level_nodes()[fine - 2], device="cuda", dtype=torch.float64)
    G.binding.mg_restrict_static(h.handle, fine - 1, x2, x2, d2, B.MG_FP64)
    h.free()
    ctx.close()
