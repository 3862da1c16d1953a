"""CUDA path against the CPU oracle, through the C ABI (GB300 only).

Every level operator (SpMV, fused smoother sweep, residual + restriction,
prolongation + correction, coarse solve), one V-cycle, the right-hand-side
assembly and the full Krylov solves are compared element by element with the
oracle on the same seeded inputs.  Sizes span many SELL slices with a ragged
tail (4225 = 132*32 + 1 nodes on the 64x64 mesh).

Tolerances (derived from the arithmetic):
* FP64 operators: |gpu - oracle| <= 1e-13 * (|A| |x| + |b|)_max  -- a few ulps
  of the summed magnitudes (summation order differs).
* FP32 operators: the same bound with 1e-5 (FP32 unit round-off 6e-8 times
  row lengths <= 27 and FP32 rounding of the stored values).
* Solves: FP64 solution vs the oracle's direct solve <= 1e-9 relative
  (lumped-mass weighted L2) at rtol 1e-10; mixed precision reaches the same
  residual with <= 1e-8 relative error.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import workloads as W
from oracle import mesh as M
from oracle import mg
from oracle import problems as PB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2405_05047_gb300 as G  # noqa: E402
from paper_2405_05047_gb300 import binding as B  # noqa: E402

CASES = {
    "poisson64": (lambda: W.poisson64(64), PB.Problem(PB.POISSON), dict(kind=B.MG_POISSON), {}),
    "td_adaptive": (lambda: W.td_adaptive(rounds=4, gamma=1.0),
                    PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                    dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)), {}),
    "elasticity16": (lambda: W.uniform_leaves(3, (1, 1, 1), 4),
                     PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                     dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)), dict(omega=0.5)),
    "elasticity_adaptive": (lambda: W.refine(W.uniform_leaves(3, (1, 1, 1), 3),
                                             W._cell_box(W.uniform_leaves(3, (1, 1, 1), 3))[1][:, 0] <= 0.25 + 1e-12),
                            PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                            dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)), {}),
}


def _oseen_entry(rounds=3):
    """Oseen + LPS on the channel patch mesh: GMRES(30), point-block smoother."""
    lm = W.oseen_channel(1, rounds)
    fm = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    beta = W.oseen_beta(fm.coords)
    kw = dict(dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01)
    return (lambda: lm, PB.Problem(PB.OSEEN, conv=beta, **kw), dict(kind=B.MG_OSEEN, conv=beta, **kw), {})


CASES["oseen"] = _oseen_entry()
# the cell-patch Vanka smoother: on every level >= 1 of the Oseen channel, and
# on the levels of >= 2000 rows of the adaptive transport problem (Jacobi and
# the small-level kernel below)
_mk, _prob, _pkw, _ = CASES["oseen"]
CASES["oseen_vanka"] = (_mk, _prob, _pkw, dict(smoother=B.MG_SMOOTHER_VANKA))
_mk, _prob, _pkw, _ = CASES["td_adaptive"]
CASES["td_vanka"] = (_mk, _prob, _pkw, dict(smoother=B.MG_SMOOTHER_VANKA, vanka_rows=2000))


def system_for(oh, prob):
    return PB.build_system(oh.fine.mesh, prob, beta=prob.conv)


def g_for(name, coords):
    """Nodal Dirichlet data: the parabolic inflow for the channel, else none."""
    return W.oseen_inflow(coords).ravel() if name.startswith("oseen") else None


@pytest.fixture(scope="module")
def ctx():
    c = G.Context(0)
    yield c
    _cache.clear()
    c.close()


_cache = {}


def setup_case(ctx, name):
    if name in _cache:
        return _cache[name]
    mk, prob, pkw, okw = CASES[name]
    lm = mk()
    ov = {}
    if okw.get("smoother") == B.MG_SMOOTHER_VANKA:
        ov = dict(smoother="vanka", vanka_rows=okw.get("vanka_rows", 0))
    oh = mg.Hierarchy(lm, prob, omega=okw.get("omega"), **ov)
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(**okw))
    _cache[name] = (lm, prob, oh, h)
    return _cache[name]


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def bound(A, x, b=None):
    s = abs(A) @ np.abs(x)
    if b is not None:
        s = s + np.abs(b)
    return max(float(s.max()), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_structure_and_coords(ctx, name):
    lm, prob, oh, h = setup_case(ctx, name)
    assert h.levels == len(oh.levels)
    assert h.level_nodes() == [lv.mesh.n_nodes for lv in oh.levels]
    assert np.array_equal(h.coords(), oh.fine.mesh.coords)
    assert h.info.n_hanging == int(oh.fine.mesh.hanging.sum())
    # storage per block: the Oseen blocks [[a, 0, g1], [0, a, g2], [d1, d2, c]]
    # (the oracle's matrices have that pattern on every level) keep 6 values
    vals = [h.info.level_block_values[l] for l in range(h.levels)]
    sm = [h.info.level_smoother[l] for l in range(h.levels)]
    assert sm == [int(getattr(lv, "vanka", False)) for lv in oh.levels]
    if any(sm):       # the small-level kernel stays below the first Vanka level
        assert h.info.tail_levels <= sm.index(1)
    if name.startswith("oseen"):
        for lv in oh.levels:
            C = lv.A.tocoo()
            ru, cu = C.row % 3, C.col % 3
            assert not np.any(C.data[(ru == 0) & (cu == 1)]) and not np.any(C.data[(ru == 1) & (cu == 0)])
        assert vals == [6] * h.levels
    else:
        assert vals == [prob.nc * prob.nc] * h.levels


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
@pytest.mark.parametrize("name", list(CASES))
def test_level_operators(ctx, name, prec):
    lm, prob, oh, h = setup_case(ctx, name)
    nc = prob.nc
    tdt = torch.float64 if prec == B.MG_FP64 else torch.float32
    tol = 1e-13 if prec == B.MG_FP64 else 2e-5
    rng = np.random.default_rng(11)
    for l, lv in enumerate(oh.levels):
        n = lv.A.shape[0]
        x = rng.standard_normal(n)
        bvec = rng.standard_normal(n)
        x[lv.sys.fixed] = 0.0
        bvec[lv.sys.fixed] = 0.0
        if prec != B.MG_FP64:      # compare with FP64 evaluation of the FP32-rounded inputs
            x = x.astype(np.float32).astype(np.float64)
            bvec = bvec.astype(np.float32).astype(np.float64)
        out = torch.empty(n, device="cuda", dtype=tdt)
        h.apply(l, B.MG_OP_MATVEC, dev(x, tdt), None, out, prec)
        ref = lv.A @ x
        assert np.abs(out.cpu().double().numpy() - ref).max() <= tol * bound(lv.A, x), f"matvec level {l}"
        h.apply(l, B.MG_OP_SMOOTH, dev(x, tdt), dev(bvec, tdt), out, prec)
        assert h.info.level_omega[l] == pytest.approx(lv.omega, rel=1e-12)
        ref = x + lv.omega * (lv.S @ (bvec - lv.A @ x))
        sc = bound(abs(lv.S) @ abs(lv.A), x) + float((abs(lv.S) @ np.abs(bvec)).max()) + np.abs(x).max()
        assert np.abs(out.cpu().double().numpy() - ref).max() <= tol * sc, f"smooth level {l}"
        if l > 0:
            nco = oh.levels[l - 1].A.shape[0]
            d = torch.empty(nco, device="cuda", dtype=tdt)
            h.apply(l, B.MG_OP_RESTRICT, dev(x, tdt), dev(bvec, tdt), d, prec)
            ref = lv.R @ (bvec - lv.A @ x)
            sc = float((abs(lv.R) @ (abs(lv.A) @ np.abs(x) + np.abs(bvec))).max())
            assert np.abs(d.cpu().double().numpy() - ref).max() <= tol * sc, f"restrict level {l}"
            y = rng.standard_normal(nco)
            y[oh.levels[l - 1].sys.fixed] = 0.0
            if prec != B.MG_FP64:
                y = y.astype(np.float32).astype(np.float64)
            h.apply(l, B.MG_OP_PROLONG_ADD, dev(y, tdt), dev(x, tdt), out, prec)
            ref = x + lv.P @ y
            sc = float((abs(lv.P) @ np.abs(y) + np.abs(x)).max())
            assert np.abs(out.cpu().double().numpy() - ref).max() <= tol * sc, f"prolong level {l}"
    # coarse direct solve
    lv0 = oh.levels[0]
    d0 = rng.standard_normal(lv0.A.shape[0])
    if prec != B.MG_FP64:
        d0 = d0.astype(np.float32).astype(np.float64)
    z0 = torch.empty(lv0.A.shape[0], device="cuda", dtype=tdt)
    h.apply(0, B.MG_OP_COARSE, dev(d0, tdt), None, z0, prec)
    ref = np.linalg.solve(lv0.A.toarray(), d0)
    ctol = 1e-11 if prec == B.MG_FP64 else 1e-6
    assert np.abs(z0.cpu().double().numpy() - ref).max() <= ctol * max(np.abs(ref).max(), 1.0)


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_fp64(ctx, name):
    lm, prob, oh, h = setup_case(ctx, name)
    rng = np.random.default_rng(5)
    n = oh.fine.A.shape[0]
    r = rng.standard_normal(n)
    r[oh.fine.sys.fixed] = 0.0
    z = torch.empty(n, device="cuda", dtype=torch.float64)
    h.vcycle(dev(r), z, B.MG_FP64)
    ref = oh.precondition(r)
    assert np.abs(z.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def test_vcycle_and_solve_with_five_sweeps(ctx):
    """The V(5,5) cycle of the transport-diffusion bench: the FP64 V-cycle
    equals the oracle's V(5,5) cycle, and the mixed-precision BiCGStab solve
    matches the oracle's direct solve."""
    mk, prob, pkw, okw = CASES["td_adaptive"]
    lm = mk()
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(krylov=B.MG_BICGSTAB, nu1=5, nu2=5))
    oh = mg.Hierarchy(lm, prob, nu1=5, nu2=5)
    rng = np.random.default_rng(15)
    n = oh.fine.A.shape[0]
    r = rng.standard_normal(n)
    r[oh.fine.sys.fixed] = 0.0
    z = torch.empty(n, device="cuda", dtype=torch.float64)
    h.vcycle(dev(r), z, B.MG_FP64)
    ref = oh.precondition(r)
    assert np.abs(z.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    s = system_for(oh, prob)
    bref = s.rhs(rhs_for("td_adaptive", oh.fine.mesh.coords, 1))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-10, max_it=200, prec=B.MG_MIXED_FP32)
    assert st.status == 0 and st.rel_res <= 1e-10, st.as_dict()
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= 1e-8
    h.free()


def test_vcycle_fp32_close_to_fp64(ctx):
    lm, prob, oh, h = setup_case(ctx, "poisson64")
    rng = np.random.default_rng(6)
    n = oh.fine.A.shape[0]
    r = rng.standard_normal(n)
    r[oh.fine.sys.fixed] = 0.0
    r32 = r.astype(np.float32)
    z = torch.empty(n, device="cuda", dtype=torch.float32)
    h.vcycle(dev(r32, torch.float32), z, B.MG_MIXED_FP32)
    ref = oh.precondition(r32.astype(np.float64))
    assert np.abs(z.cpu().double().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def rhs_for(name, coords, nc):
    if name.startswith("oseen"):
        return np.zeros(coords.shape[0] * 3)
    if name.startswith("poisson"):
        return W.f_poisson(coords)
    if name.startswith("td"):
        return W.f_transport(coords, 1e-3, (1.0, 0.5))
    return np.tile([0.0, 0.0, -1.0], (coords.shape[0], 1)).ravel()


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_assembly(ctx, name):
    lm, prob, oh, h = setup_case(ctx, name)
    s = system_for(oh, prob)
    f = rhs_for(name, oh.fine.mesh.coords, prob.nc)
    g = g_for(name, oh.fine.mesh.coords)
    b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
    h.assemble_rhs(dev(f), b, dev(g) if g is not None else None)
    ref = s.rhs(f, g)
    assert np.abs(b.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_rhs_lifting_with_dirichlet_data(ctx):
    """Nonhomogeneous Dirichlet data on a scalar problem: b = g on Dirichlet
    rows, the couplings lifted into the free rows."""
    lm, prob, oh, h = setup_case(ctx, "td_adaptive")
    s = system_for(oh, prob)
    xy = oh.fine.mesh.coords
    f = rhs_for("td", xy, 1)
    g = 1.0 + xy[:, 0] ** 2 - 0.5 * xy[:, 1]
    b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
    h.assemble_rhs(dev(f), b, dev(g))
    ref = s.rhs(f, g)
    assert np.abs(b.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(b, x, rtol=1e-10, max_it=200)
    xstar = s.H @ spl.spsolve(s.A.tocsc(), ref)
    assert st.status == 0
    assert np.abs(x.cpu().numpy() - xstar).max() <= 1e-8 * np.abs(xstar).max()
    assert np.array_equal(x.cpu().numpy()[s.dirichlet], g[s.dirichlet])


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_supg_linear_solution_exact(ctx, prec):
    """SUPG is consistent: with eps = 1e-3, beta = (1, 0.5), the linear exact
    solution u = 0.3 + 1.2 x - 0.7 y, f = beta.grad u and Dirichlet data g = u
    on an adaptive mesh with hanging nodes, the discrete solution is u at
    every node.  The right-hand side (Galerkin and SUPG load, lifting) equals
    the oracle's, and the solve through the C ABI reproduces u to the solver
    tolerance in both precisions."""
    lm = W.td_adaptive(rounds=3, gamma=1.0)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    fm = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    s = PB.build_system(fm, prob)
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)))
    try:
        assert h.info.n_hanging > 0
        xy = h.coords()
        assert np.array_equal(xy, fm.coords)
        u = 0.3 + 1.2 * xy[:, 0] - 0.7 * xy[:, 1]
        f = np.full(h.n_dofs, 1.2 - 0.35)
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(dev(f), b, dev(u))
        ref = s.rhs(f, u)
        assert np.abs(b.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
        x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        st = h.solve(b, x, rtol=1e-10, max_it=200, prec=prec)
        assert st.status == 0 and st.iters > 0, st.as_dict()
        assert np.abs(x.cpu().numpy() - u).max() <= 1e-8
    finally:
        h.free()


def lumped_weights(oh, prob):
    s = system_for(oh, prob)
    m = np.asarray(s.F.sum(axis=1)).ravel()
    return np.repeat(m, prob.nc)


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
@pytest.mark.parametrize("name", list(CASES))
def test_solve_matches_direct(ctx, name, prec):
    lm, prob, oh, h = setup_case(ctx, name)
    s = system_for(oh, prob)
    f = rhs_for(name, oh.fine.mesh.coords, prob.nc)
    bref = s.rhs(f, g_for(name, oh.fine.mesh.coords))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    b = dev(bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(b, x, rtol=1e-10, max_it=600, prec=prec)
    assert st.status == 0, st.as_dict()
    assert st.rel_res <= 1e-10
    xg = x.cpu().numpy()
    w = lumped_weights(oh, prob)
    err = math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2))
    assert err <= (1e-9 if prec == B.MG_FP64 else 1e-8), err
    # the true residual of the returned solution, recomputed by the oracle
    xr = xg.copy()
    xr[s.hang] = 0.0
    assert np.linalg.norm(bref - oh.fine.A @ xr) <= 1.01e-10 * np.linalg.norm(bref[~s.fixed])


@pytest.mark.parametrize("name", ["poisson64", "elasticity16", "oseen"])
def test_defect_correction_rounds(ctx, name):
    """Defect correction (inner_rtol): rounds of the mixed-precision Krylov
    solve, each on the recomputed FP64 defect, reach the outer tolerance and
    the direct solution."""
    lm, prob, oh, h0 = setup_case(ctx, name)
    mk, _, pkw, okw = CASES[name]
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(inner_rtol=1e-2, autotune=0, **okw))
    s = system_for(oh, prob)
    bref = s.rhs(rhs_for(name, oh.fine.mesh.coords, prob.nc), g_for(name, oh.fine.mesh.coords))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-10, max_it=2000, prec=B.MG_MIXED_FP32)
    assert st.status == 0 and st.rel_res <= 1e-10, st.as_dict()
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= 1e-8
    h.free()


@pytest.mark.parametrize("name", ["poisson64", "td_adaptive", "oseen", "oseen_vanka"])
def test_zero_and_nan_right_hand_sides(ctx, name):
    """b = 0 returns x = 0 at once (the tolerance is absolute when b_free = 0);
    a NaN in b ends the device loop with MG_ERR_NAN instead of iterating on."""
    lm, prob, oh, h = setup_case(ctx, name)
    n = h.n_dofs
    x = torch.zeros(n, device="cuda", dtype=torch.float64)
    st = h.solve(torch.zeros(n, device="cuda", dtype=torch.float64), x, rtol=1e-10, max_it=50,
                 prec=B.MG_MIXED_FP32)
    assert st.status == 0 and st.iters == 0 and not x.any()
    b = np.zeros(n)
    free = np.nonzero(~oh.fine.sys.fixed)[0]
    b[free[len(free) // 2]] = np.nan
    x.zero_()
    st = h.solve(dev(b), x, rtol=1e-10, max_it=50, prec=B.MG_MIXED_FP32)
    assert st.status == B.MG_ERR_NAN, st.as_dict()


def test_solve_host_equals_device(ctx):
    lm, prob, oh, h = setup_case(ctx, "td_adaptive")
    s = PB.build_system(oh.fine.mesh, prob)
    bref = s.rhs(rhs_for("td", oh.fine.mesh.coords, 1))
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st1 = h.solve(dev(bref), x, rtol=1e-10, max_it=200)
    xh = np.zeros(h.n_dofs)
    st2 = h.solve_host(bref.copy(), xh, rtol=1e-10, max_it=200)
    assert st1.iters == st2.iters
    assert np.array_equal(x.cpu().numpy(), xh)


def test_deterministic_repeat(ctx):
    """Fixed-order reductions: two solves give bitwise identical results."""
    lm, prob, oh, h = setup_case(ctx, "poisson64")
    s = PB.build_system(oh.fine.mesh, prob)
    b = dev(s.rhs(W.f_poisson(oh.fine.mesh.coords)))
    xs = []
    for _ in range(2):
        x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        h.solve(b, x, rtol=1e-10, max_it=100, prec=B.MG_MIXED_FP32)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


def test_not_converged_status(ctx):
    lm, prob, oh, h = setup_case(ctx, "poisson64")
    s = PB.build_system(oh.fine.mesh, prob)
    b = dev(s.rhs(W.f_poisson(oh.fine.mesh.coords)))
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(b, x, rtol=1e-14, max_it=2)
    assert st.status == B.MG_ERR_NOT_CONVERGED and st.iters == 2


@pytest.mark.parametrize("name,nu", [("td_adaptive", 2), ("elasticity16", 2), ("td_adaptive", 5)])
def test_tail_kernel_bitwise_equals_level_kernels(ctx, name, nu):
    """The tail V-cycle runs the same row steps as the grid kernels: identical
    bits without it, with it on a cluster of 1, 2, 4, 8 or 16 CTAs (16 where
    the GPU schedules it), and on one CTA
    working in shared memory (cluster 0: all vectors staged, matrices staged
    coarsest first while they fit), in FP64, FP32 and with BF16 values; with
    V(2,2) and with the V(5,5) cycle of the transport-diffusion bench."""
    mk, prob, pkw, okw = CASES[name]
    lm = mk()
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(autotune=0, store_bf16=1, nu1=nu, nu2=nu, **okw))
    n = h.n_dofs
    rng = np.random.default_rng(9)
    r = rng.standard_normal(n)
    oh = mg.Hierarchy(lm, prob, omega=okw.get("omega"))
    r[oh.fine.sys.fixed] = 0.0
    shapes = ((0, 1), (1 << 20, 1), (1 << 20, 2), (1 << 20, 4), (1 << 20, 8), (1024, 4),
              (1 << 20, 0), (4096, 0), (256, 0), (1 << 20, 16), (4096, 16))
    for prec, dt in ((B.MG_FP64, torch.float64), (B.MG_MIXED_FP32, torch.float32),
                     (B.MG_MIXED_BF16, torch.float32)):
        outs, staged_levels = [], []
        for rows, cl in shapes:
            try:
                h.tune(prec, rows, cl)
            except G.MGError:
                assert cl > 8            # only the non-portable cluster size may be refused
                continue
            if cl == 0:
                staged_levels.append(h.info.tail_levels)
            z = torch.empty(n, device="cuda", dtype=dt)
            h.vcycle(dev(r, dt), z, prec)
            outs.append(z.cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(outs[0], o)
        assert max(staged_levels) >= 2      # the shared-memory tail really ran
    # the autotuner picks one of these shapes and the solve still matches
    h.tune(B.MG_MIXED_FP32, -1)
    assert -16 <= h.info.tail_cluster <= 16
    h.free()


@pytest.mark.parametrize("name", ["td_adaptive", "poisson64"])
def test_cluster_resident_tail_bitwise(ctx, name):
    """The cluster-resident tail (every level cut into power-of-two row chunks,
    one per CTA, vectors gathered across the cluster through distributed
    shared memory) runs the same row steps: V-cycles in FP64, FP32 and with
    BF16 values equal the grid kernels' bit for bit for every cluster size and
    threshold that fits, and so does a whole solve."""
    mk, prob, pkw, okw = CASES[name]
    lm = mk()
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(autotune=0, store_bf16=1, **okw))
    n = h.n_dofs
    rng = np.random.default_rng(19)
    r = rng.standard_normal(n)
    oh = mg.Hierarchy(lm, prob, omega=okw.get("omega"))
    r[oh.fine.sys.fixed] = 0.0
    shapes = ((0, 1), (512, -2), (1024, -4), (4096, -8), (1 << 20, -8), (4096, -16), (1 << 20, -16))
    ran = []
    for prec, dt in ((B.MG_FP64, torch.float64), (B.MG_MIXED_FP32, torch.float32),
                     (B.MG_MIXED_BF16, torch.float32)):
        outs = []
        for rows, cl in shapes:
            try:
                h.tune(prec, rows, cl)
            except G.MGError:
                assert cl < 0            # a cluster-resident tail may not fit or not be schedulable
                continue
            if cl < 0:
                assert h.info.tail_cluster == cl or h.info.tail_levels == 0
                ran.append(h.info.tail_levels)
            z = torch.empty(n, device="cuda", dtype=dt)
            h.vcycle(dev(r, dt), z, prec)
            outs.append(z.cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(outs[0], o)
    assert max(ran) >= 3                 # the cluster-resident tail really ran
    b = torch.empty(n, device="cuda", dtype=torch.float64)
    h.assemble_rhs(dev(rhs_for(name, h.coords(), 1)), b)
    sols = []
    for rows, cl in ((0, 1), (4096, -8)):
        try:
            h.tune(B.MG_MIXED_FP32, rows, cl)
        except G.MGError:
            continue
        x = torch.zeros_like(b)
        st = h.solve(b, x, rtol=1e-10, max_it=200, prec=B.MG_MIXED_FP32)
        assert st.status == 0
        sols.append((st.iters, x.cpu().numpy()))
    for sv in sols[1:]:
        assert sv[0] == sols[0][0] and np.array_equal(sv[1], sols[0][1])
    h.free()


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_shared_memory_tail_solve_identical(ctx, prec):
    """A whole solve (CUDA-graph while loop) with the shared-memory tail gives
    the same iterates, bit for bit, as the multi-kernel V-cycle."""
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)), B.make_opts(autotune=0))
    f = dev(W.f_transport(h.coords(), 1e-3, (1.0, 0.5)))
    b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
    h.assemble_rhs(f, b)
    xs, its = [], []
    for rows, cl in ((0, 1), (1 << 20, 0)):
        h.tune(prec, rows, cl)
        x = torch.zeros_like(b)
        st = h.solve(b, x, rtol=1e-10, max_it=100, prec=prec)
        assert st.status == B.MG_OK
        xs.append(x.cpu().numpy())
        its.append(st.iters)
    assert its[0] == its[1] and np.array_equal(xs[0], xs[1])
    h.free()


@pytest.mark.parametrize("name", ["td_adaptive", "oseen", "elasticity16"])
def test_sell_sigma_sorting_is_bitwise_neutral(ctx, name):
    """Rows sorted by length within windows (SELL-C-sigma) with 16-bit column
    offsets give the same V-cycle bits as rows in node order with 32-bit
    columns (each row's sum keeps its order), and a solve with that layout
    still matches the direct solution."""
    lm, prob, oh, _ = setup_case(ctx, name)
    mk, _, pkw, okw = CASES[name]
    hs = [G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(sell_sigma=sg, col16=c16, autotune=0, **okw))
          for sg, c16 in ((0, 0), (256, 1))]
    rng = np.random.default_rng(8)
    n = oh.fine.A.shape[0]
    r = rng.standard_normal(n)
    r[oh.fine.sys.fixed] = 0.0
    for prec, dt in ((B.MG_FP64, torch.float64), (B.MG_MIXED_FP32, torch.float32)):
        outs = []
        for hh in hs:
            hh.tune(prec, 0, 1)
            z = torch.empty(n, device="cuda", dtype=dt)
            hh.vcycle(dev(r, dt), z, prec)
            outs.append(z.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
    s = system_for(oh, prob)
    bref = s.rhs(rhs_for(name, oh.fine.mesh.coords, prob.nc), g_for(name, oh.fine.mesh.coords))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(n, device="cuda", dtype=torch.float64)
    st = hs[1].solve(dev(bref), x, rtol=1e-10, max_it=600, prec=B.MG_MIXED_FP32)
    assert st.status == 0
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= 1e-8
    for hh in hs:
        hh.free()


@pytest.mark.slow
def test_col16_fallback_slices_bitwise(ctx):
    """On the 1.2 M-node adaptive mesh some slices have column offsets outside
    int16 and keep 32-bit columns; V-cycles with the mixed layout equal the
    plain 32-bit layout bit for bit (FP32 and BF16 values)."""
    lm = W.td_adaptive(rounds=8, gamma=0.18)
    pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    h0 = G.Hierarchy(ctx, lm, pb, B.make_opts(col16=0, sell_sigma=0, autotune=0, store_fp64=0, store_bf16=1))
    h1 = G.Hierarchy(ctx, lm, pb, B.make_opts(col16=-1, sell_sigma=-1, autotune=0, store_fp64=0, store_bf16=1))
    assert h1.info.col16_slices > 0 and h1.info.col32_slices > 0 and h0.info.col16_slices == 0
    rng = np.random.default_rng(12)
    r = rng.standard_normal(h0.n_dofs).astype(np.float32)
    for prec in (B.MG_MIXED_FP32, B.MG_MIXED_BF16):
        outs = []
        for hh in (h0, h1):
            hh.tune(prec, 0, 1)
            z = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float32)
            hh.vcycle(dev(r, torch.float32), z, prec)
            outs.append(z.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
    h0.free()
    h1.free()


def test_layout_choices_bitwise_and_tuned(ctx):
    """Every layout the setup autotuner may pick for a level operator (SELL
    window 0 / 256 / 1024, 16-bit columns off / on) gives the same V-cycle
    bits in FP32 and FP64; the tuned hierarchy (choices per level reported in
    level_sigma / level_col16) equals them, and its solves equal those of the
    untuned hierarchy bit for bit (the FP64 outer operator keeps the size
    rule in both)."""
    lm = W.td_adaptive(rounds=5, gamma=1.0)
    pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    hs = [G.Hierarchy(ctx, lm, pb, B.make_opts(sell_sigma=sg, col16=c, autotune=0))
          for sg in (0, 256, 1024) for c in (0, 1)]
    hs.append(G.Hierarchy(ctx, lm, pb, B.make_opts(autotune=0)))
    hs.append(G.Hierarchy(ctx, lm, pb, B.make_opts(autotune=1)))
    tuned = hs[-1].info
    for l in range(tuned.levels):
        assert tuned.level_sigma[l] in (0, 256, 1024) and tuned.level_col16[l] in (0, 1)
    rng = np.random.default_rng(14)
    r = rng.standard_normal(hs[0].n_dofs)
    f = dev(W.f_transport(hs[0].coords(), 1e-3, (1.0, 0.5)))
    for prec, dt in ((B.MG_MIXED_FP32, torch.float32), (B.MG_FP64, torch.float64)):
        outs, sols = [], []
        for hh in hs:
            hh.tune(prec, 0, 1)
            z = torch.empty(hh.n_dofs, device="cuda", dtype=dt)
            hh.vcycle(dev(r, dt), z, prec)
            outs.append(z.cpu().numpy())
            b = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float64)
            hh.assemble_rhs(f, b)
            x = torch.zeros_like(b)
            st = hh.solve(b, x, rtol=1e-10, max_it=100, prec=prec)
            assert st.status == 0
            sols.append((st.iters, x.cpu().numpy()))
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        assert sols[-1][0] == sols[-2][0] and np.array_equal(sols[-1][1], sols[-2][1])
    for hh in hs:
        hh.free()


@pytest.mark.parametrize("case", ["transport2d", "poisson3d"])
def test_row_lanes_reported_and_equivalent(ctx, case):
    """level_lanes reports the lane-count rule (one lane per row everywhere
    with row_lanes = 1; four on the scalar levels of 1024..32767 rows
    otherwise).  The lane count changes the row sums' order, so one- and
    four-lane solves agree to the solver tolerance, not bit for bit."""
    if case == "transport2d":
        lm = W.td_adaptive(rounds=5, gamma=1.0)
        pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    else:
        lm = W.uniform_leaves(3, (1, 1, 1), 5)
        pb = B.make_problem(kind=B.MG_POISSON)
    hs = [G.Hierarchy(ctx, lm, pb, B.make_opts(row_lanes=1, store_bf16=1)),
          G.Hierarchy(ctx, lm, pb, B.make_opts(store_bf16=1))]
    info = hs[1].info
    lanes = [list(hh.info.level_lanes[:hh.info.levels]) for hh in hs]
    assert set(lanes[0]) == {1}
    assert lanes[1] == [4 if 1024 <= info.level_nodes[l] < 32768 else 1 for l in range(info.levels)]
    assert 4 in lanes[1]
    if case == "transport2d":
        f = dev(W.f_transport(hs[0].coords(), 1e-3, (1.0, 0.5)))
    else:
        f = dev(np.ones(hs[0].n_dofs))
    for prec in (B.MG_MIXED_FP32, B.MG_MIXED_BF16):
        sols = []
        for hh in hs:
            b = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float64)
            hh.assemble_rhs(f, b)
            x = torch.zeros_like(b)
            st = hh.solve(b, x, rtol=1e-10, max_it=100, prec=prec)
            assert st.status == 0
            sols.append((st.iters, x.cpu().numpy()))
        assert abs(sols[0][0] - sols[1][0]) <= 1
        assert np.linalg.norm(sols[0][1] - sols[1][1]) <= 1e-8 * np.linalg.norm(sols[0][1])
    for hh in hs:
        hh.free()


@pytest.mark.parametrize("case", ["transport2d", "poisson3d"])
def test_staged_sweep_bitwise(ctx, case):
    """The sweep that gathers x from a shared-memory copy of each window's
    column range (stage_x) gives the same V-cycle and solve bits as the one
    that gathers from device memory, in FP32 and with BF16-stored values;
    3D windows span too many columns to be staged and take the fallback."""
    if case == "transport2d":
        lm = W.td_adaptive(rounds=5, gamma=1.0)
        pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    else:
        lm = W.uniform_leaves(3, (1, 1, 1), 5)
        pb = B.make_problem(kind=B.MG_POISSON)
    hs = [G.Hierarchy(ctx, lm, pb, B.make_opts(stage_x=v, autotune=0, store_bf16=1)) for v in (0, 1, -1)]
    rng = np.random.default_rng(16)
    r = rng.standard_normal(hs[0].n_dofs)
    f = dev(np.ones(hs[0].n_dofs))
    for prec in (B.MG_MIXED_FP32, B.MG_MIXED_BF16):
        outs, sols = [], []
        for hh in hs:
            z = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float32)
            hh.vcycle(dev(r, torch.float32), z, prec)
            outs.append(z.cpu().numpy())
            b = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float64)
            hh.assemble_rhs(f, b)
            x = torch.zeros_like(b)
            st = hh.solve(b, x, rtol=1e-10, max_it=200, prec=prec)
            assert st.status == 0
            sols.append((st.iters, x.cpu().numpy()))
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        for it, x in sols[1:]:
            assert it == sols[0][0] and np.array_equal(x, sols[0][1])
        # the level operator alone, on every level
        for l in range(hs[0].levels):
            n = hs[0].info.level_nodes[l]
            xin = dev(rng.standard_normal(n), torch.float32)
            bb = dev(rng.standard_normal(n), torch.float32)
            res = []
            for hh in hs[:2]:
                out = torch.empty(n, device="cuda", dtype=torch.float32)
                hh.apply(l, B.MG_OP_SMOOTH, xin, bb, out, prec)
                res.append(out.cpu().numpy())
            assert np.array_equal(res[0], res[1]), l
    for hh in hs:
        hh.free()


def test_direct_launch_mode_equals_graph(ctx):
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    pk = dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    hs = [G.Hierarchy(ctx, lm, B.make_problem(**pk), B.make_opts(launch_mode=m)) for m in (0, 1)]
    coords = hs[0].coords()
    f = dev(W.f_transport(coords, 1e-3, (1.0, 0.5)))
    xs, its = [], []
    for hh in hs:
        b = torch.empty(hh.n_dofs, device="cuda", dtype=torch.float64)
        hh.assemble_rhs(f, b)
        x = torch.zeros_like(b)
        st = hh.solve(b, x, rtol=1e-10, max_it=100, prec=B.MG_MIXED_FP32)
        xs.append(x.cpu().numpy())
        its.append(st.iters)
    assert its[0] == its[1] and np.array_equal(xs[0], xs[1])
    for hh in hs:
        hh.free()


@pytest.mark.parametrize("name", ["td_adaptive", "oseen", "td_vanka"])
def test_profiled_solve_equals_solve(ctx, name):
    """mg_solve_profiled runs the kernels of mg_solve in the same order (one
    graph per iteration, event nodes between runs of the same kernel): the same bits and
    iterations; every launch of the solve is in its table, and the finest
    level's sweeps appear with three launches per V-cycle (V(2,2), the first
    sweep from zero being a kernel of its own)."""
    lm, prob, oh, h = setup_case(ctx, name)
    b = dev(system_for(oh, prob).rhs(rhs_for(name, oh.fine.mesh.coords, prob.nc),
                                     g_for(name, oh.fine.mesh.coords)))
    x0 = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st0 = h.solve(b, x0, rtol=1e-10, max_it=500, prec=B.MG_MIXED_FP32)
    x1 = torch.zeros_like(x0)
    st1, ents = h.solve_profiled(b, x1, rtol=1e-10, max_it=500, prec=B.MG_MIXED_FP32)
    assert st0.status == 0 and st1.status == 0
    assert st1.iters == st0.iters and st1.vcycles == st0.vcycles and torch.equal(x0, x1)
    assert all(e["launches"] > 0 and e["ms"] > 0 for e in ents)
    assert sum(e["launches"] for e in ents if e["level"] != -2) == st1.launches
    floor = [e for e in ents if e["level"] == -2]
    assert len(floor) == 1 and floor[0]["kernel"] == "k_prof_empty"
    assert [e["ms"] for e in ents] == sorted((e["ms"] for e in ents), reverse=True)
    fine = h.levels - 1
    if h.info.level_smoother[fine] == B.MG_SMOOTHER_VANKA:
        # V(2,2) with Vanka: four updates per cycle (the first from zero), three after a residual
        vk = [e for e in ents if e["kernel"].startswith("k_vanka<float") and e["level"] == fine]
        assert len(vk) == 1 and vk[0]["launches"] == 4 * st1.vcycles, [e["kernel"] for e in ents]
        return
    sweeps = [e for e in ents if e["kernel"].startswith("k_smooth<float") and ", false," in e["kernel"]
              and e["level"] == fine]
    if h.info.tail_levels < h.levels:        # the finest level is not inside the small-level kernel
        assert len(sweeps) == 1, [e["kernel"] for e in ents]
        assert sweeps[0]["launches"] % 3 == 0 and sweeps[0]["launches"] >= 3 * st1.vcycles
    else:
        assert any(e["kernel"].startswith("k_tail") for e in ents)


@pytest.mark.parametrize("restart", [30, 4])
@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_gmres_matches_direct(ctx, prec, restart):
    """Device GMRES(m) (flexible, CGS2, Givens on the device), including
    restarts (m = 4), against the oracle's direct solve."""
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    h = G.Hierarchy(ctx, lm, B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                    B.make_opts(krylov=B.MG_GMRES, restart=restart))
    oh = mg.Hierarchy(lm, prob)
    s = PB.build_system(oh.fine.mesh, prob)
    bref = s.rhs(W.f_transport(oh.fine.mesh.coords, 1e-3, (1.0, 0.5)))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-10, max_it=300, prec=prec)
    assert st.status == 0 and st.rel_res <= 1e-10, st.as_dict()
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    err = math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2))
    assert err <= (1e-9 if prec == B.MG_FP64 else 1e-8), err
    # the oracle's GMRES with the same restart needs a comparable number of steps
    _, info = __import__("oracle.krylov", fromlist=["gmres"]).gmres(oh.fine.A, bref, oh.precondition, rtol=1e-10,
                                                                    restart=restart, maxit=300)
    assert abs(info["iters"] - st.iters) <= max(3, info["iters"] // 3), (info["iters"], st.iters)
    h.free()


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
def test_gmres_long_cycle_two_chunks(ctx, prec):
    """GMRES(40) on the Oseen channel with a weak smoother (V(1,1)): more
    than 32 Arnoldi steps in one cycle, so the orthogonalisation kernels run
    their second chunk of 32 basis vectors; the solution matches the direct
    solve."""
    lm, prob, oh, _ = setup_case(ctx, "oseen")
    _, _, pkw, _ = CASES["oseen"]
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(krylov=B.MG_GMRES, restart=40, nu1=1, nu2=1))
    s = system_for(oh, prob)
    bref = s.rhs(rhs_for("oseen", oh.fine.mesh.coords, prob.nc), g_for("oseen", oh.fine.mesh.coords))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-11, max_it=400, prec=prec)
    assert st.status == 0 and st.rel_res <= 1e-11, st.as_dict()
    assert st.iters > 32, st.iters
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= 1e-8
    h.free()


def _bf16_round(a):
    """Round-to-nearest-even of FP64 values to BF16 through FP32 (the
    library's stored-value rounding), returned as FP64."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name", ["poisson64", "elasticity16"])
def test_bf16_values_smoother_parity(ctx, name):
    """BF16-stored values (ablation): one smoothing sweep equals an FP64
    evaluation with the BF16-rounded operator, FP32 vectors."""
    mk, prob, pkw, okw = CASES[name]
    lm = mk()
    ov = {}
    if okw.get("smoother") == B.MG_SMOOTHER_VANKA:
        ov = dict(smoother="vanka", vanka_rows=okw.get("vanka_rows", 0))
    oh = mg.Hierarchy(lm, prob, omega=okw.get("omega"), **ov)
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(store_bf16=1, **okw))
    lv = oh.fine
    A16 = lv.A.copy()
    A16.data = _bf16_round(A16.data)
    rng = np.random.default_rng(13)
    n = lv.A.shape[0]
    x = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    bvec = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    x[lv.sys.fixed] = 0.0
    bvec[lv.sys.fixed] = 0.0
    out = torch.empty(n, device="cuda", dtype=torch.float32)
    h.apply(h.levels - 1, B.MG_OP_MATVEC, dev(x, torch.float32), None, out, B.MG_MIXED_BF16)
    ref = A16 @ x
    assert np.abs(out.cpu().double().numpy() - ref).max() <= 2e-5 * bound(A16, x)
    h.free()


@pytest.mark.parametrize("name", ["td_adaptive", "elasticity16"])
def test_bf16_values_solve_reaches_tolerance(ctx, name):
    lm, prob, oh, _ = setup_case(ctx, name)
    mk, prob, pkw, okw = CASES[name]
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(store_bf16=1, **okw))
    s = PB.build_system(oh.fine.mesh, prob)
    bref = s.rhs(rhs_for(name, oh.fine.mesh.coords, prob.nc))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-10, max_it=300, prec=B.MG_MIXED_BF16)
    assert st.status == 0 and st.rel_res <= 1e-10
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= 1e-8
    h.free()


@pytest.mark.parametrize("prec", [B.MG_FP64, B.MG_MIXED_FP32])
@pytest.mark.parametrize("name", ["poisson64", "elasticity16"])
def test_multigrid_iteration_solver(ctx, name, prec):
    """The V-cycle iterated as the solver (Algorithm "Geometric multigrid
    solver"), defect b - A x in FP64: reaches the tolerance, equals the
    direct solve, and contracts at least as fast as the oracle's iteration."""
    lm, prob, oh, _ = setup_case(ctx, name)
    mk, prob, pkw, okw = CASES[name]
    h = G.Hierarchy(ctx, lm, B.make_problem(**pkw), B.make_opts(krylov=B.MG_MGITER, **okw))
    s = PB.build_system(oh.fine.mesh, prob)
    bref = s.rhs(rhs_for(name, oh.fine.mesh.coords, prob.nc))
    xstar = s.H @ spl.spsolve(oh.fine.A.tocsc(), bref)
    x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
    st = h.solve(dev(bref), x, rtol=1e-10, max_it=300, prec=prec)
    assert st.status == 0 and st.rel_res <= 1e-10, st.as_dict()
    w = lumped_weights(oh, prob)
    xg = x.cpu().numpy()
    assert math.sqrt(np.sum(w * (xg - xstar) ** 2) / np.sum(w * xstar ** 2)) <= (1e-9 if prec == B.MG_FP64 else 1e-8)
    # the oracle's multigrid iteration needs the same number of cycles (FP64)
    xo = np.zeros_like(bref)
    its = 0
    nb = np.linalg.norm(bref[~s.fixed])
    while np.linalg.norm(bref - oh.fine.A @ xo) > 1e-10 * nb and its < 300:
        xo = xo + oh.precondition(bref - oh.fine.A @ xo)
        its += 1
    if prec == B.MG_FP64:
        assert st.iters == its
    else:
        assert abs(st.iters - its) <= 2
    h.free()


def test_vanka_reduces_gmres_iterations_on_the_channel(ctx):
    """The cell-patch Vanka smoother cuts the GMRES iterations of the Oseen
    channel at least in half against the point-block smoother, with the same
    solution (both to rtol 1e-10, both against the direct solve)."""
    its = {}
    for name in ("oseen", "oseen_vanka"):
        lm, prob, oh, h = setup_case(ctx, name)
        s = system_for(oh, prob)
        bref = s.rhs(rhs_for(name, oh.fine.mesh.coords, 3), g_for(name, oh.fine.mesh.coords))
        x = torch.zeros(h.n_dofs, device="cuda", dtype=torch.float64)
        st = h.solve(dev(bref), x, rtol=1e-10, max_it=500, prec=B.MG_MIXED_FP32)
        assert st.status == 0
        its[name] = st.iters
    assert 2 * its["oseen_vanka"] <= its["oseen"], its
