"""Explicit Navier-Stokes pressure correction (Sec. 5.3) through the C ABI
against the oracle (GB300 only): the same seeded state advanced a few steps
on both sides, compared entry by entry.

Tolerances: Steps 1 and 3 are explicit FP64 stencils summed in another order
than the oracle's sparse products (a few ulps); Step 2 is an iterative solve
to the relative residual rtol against the oracle's sparse LU, so the pressure
increment carries about rtol x cond(K_p) of relative error, and the pressure
and (through it) the velocity inherit it.  FP64 multigrid at rtol 1e-12:
1e-8 relative on p and q, 1e-11 on u; FP32 multigrid inside FP64 GMRES at
rtol 1e-10: 1e-6 and 1e-9.
"""
import numpy as np
import pytest

from oracle import ns as ONS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    c.close()


def seeded_state(S, seed):
    """Random interior velocity with the cavity's boundary values, random
    pressure and increment of mean zero (the space Q)."""
    rng = np.random.default_rng(seed)
    u = 0.2 * rng.standard_normal((S.vm.n_nodes, 3))
    u[S.fixed] = S.g[S.fixed]
    p = rng.standard_normal(S.pm.n_nodes)
    q = 0.1 * rng.standard_normal(S.pm.n_nodes)
    p -= (S.mp @ p) / S.mp.sum()
    q -= (S.mp @ q) / S.mp.sum()
    return u, p, q


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("shape,graded,prec,rtol,krylov", [
    ((4, 4, 8), 1, B.MG_FP64, 1e-12, B.MG_GMRES),
    ((8, 8, 16), 1, B.MG_FP64, 1e-12, B.MG_GMRES),
    ((8, 8, 16), 1, B.MG_MIXED_FP32, 1e-10, B.MG_GMRES),
    ((6, 4, 10), 0, B.MG_FP64, 1e-12, B.MG_CG),
])
def test_steps_match_oracle(ctx, shape, graded, prec, rtol, krylov):
    nx, ny, nz = shape
    S = ONS.cavity(nx, ny, nz, re=1000.0, dt=1e-4, graded=bool(graded))
    sim = B.NavierStokes(ctx, nx=nx, ny=ny, nz=nz, graded=graded, re=1000.0, dt=1e-4, prec=prec, rtol=rtol,
                         krylov=krylov, max_it=400)
    try:
        assert sim.n_vel == S.vm.n and sim.n_pres == S.pm.n
        u0, p0, q0 = seeded_state(S, 11)
        sim.set_state(torch.from_numpy(u0).cuda(), torch.from_numpy(p0).cuda(), torch.from_numpy(q0).cuda())
        u, p, q = u0, p0, q0
        tp, tu = (1e-8, 1e-11) if prec == B.MG_FP64 else (1e-6, 1e-9)
        for k in range(3):
            st = sim.steps(1)
            assert st.status == 0 and st.steps == 1 and st.iters > 0 and st.rel_res_max <= rtol
            u, p, q, _ = ONS.step(S, u, p, q)
            ug, pg, qg = (t.cpu().numpy() for t in sim.get_state())
            assert rel(ug, u) <= tu, (k, rel(ug, u))
            assert rel(qg, q) <= tp, (k, rel(qg, q))
            assert rel(pg, p) <= tp, (k, rel(pg, p))
            assert np.array_equal(ug[S.fixed], S.g[S.fixed])
            assert abs(S.mp @ qg) <= 1e-12 * (S.mp @ np.abs(qg))
    finally:
        sim.free()


def test_cavity_from_rest(ctx):
    """The lid drives the fluid from rest: 20 steps on the graded 8x8x16
    cavity against the oracle, and the phase timings are reported."""
    S = ONS.cavity(8, 8, 16)
    sim = B.NavierStokes(ctx, nx=8, ny=8, nz=16, prec=B.MG_FP64, rtol=1e-12, max_it=400)
    try:
        st = sim.steps(20)
        assert st.status == 0 and st.steps == 20
        assert st.ms_momentum > 0 and st.ms_pres_rhs > 0 and st.ms_pres_solve > 0 and st.ms_pres_up > 0
        u, p, q = ONS.run(S, 20)
        ug, pg, qg = (t.cpu().numpy() for t in sim.get_state())
        assert rel(ug, u) <= 1e-10 and rel(pg, p) <= 1e-7
        assert 0 < np.abs(ug[~S.fixed]).max() < 1.0
        info = sim.pressure_info()
        assert info.n_free == S.pm.n_nodes              # pure Neumann: no prescribed node
    finally:
        sim.free()


def test_rejects_bad_parameters(ctx):
    with pytest.raises(B.MGError):
        B.NavierStokes(ctx, nx=1)
    with pytest.raises(B.MGError):
        B.NavierStokes(ctx, nx=4, ny=4, nz=8, dt=-1.0)
