"""Pins of the CPU oracle against facts other than itself.

Each test ties one part of the oracle to a closed form, an invariant, a
textbook special case, an integer the paper prints, or a direct solve, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import workloads as W
from oracle import fem, krylov, mg
from oracle import mesh as M
from oracle import problems as PB

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def q1mesh(lm, lattice=None):
    return M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor, lattice)


def interior_row(mesh, A, nc=1):
    centre = np.all((mesh.X > 1) & (mesh.X < mesh.n_lat - 1), axis=1)
    i = int(np.nonzero(centre)[0][len(np.nonzero(centre)[0]) // 2])
    return i


# ---------------------------------------------------------------- closed forms
def test_q1_laplacian_stencil_2d():
    """2D Q1 Laplacian: 8/3 centre, -1/3 on all eight neighbours, any h."""
    for n in (4, 8, 16):
        m = q1mesh(W.uniform_leaves(2, (1, 1), int(math.log2(n))))
        A = fem.assemble(m, lambda h: fem.scalar_element(2, h, "stiffness"))
        i = interior_row(m, A)
        row = A.getrow(i).toarray().ravel()
        nb = np.nonzero(row)[0]
        assert len(nb) == 9
        assert row[i] == pytest.approx(8.0 / 3.0, abs=1e-14)
        for j in nb:
            if j != i:
                assert row[j] == pytest.approx(-1.0 / 3.0, abs=1e-14)


def test_q1_laplacian_stencil_3d():
    """3D Q1 Laplacian: 8h/3 centre, 0 face, -h/6 edge, -h/12 corner."""
    n = 8
    h = 1.0 / n
    m = q1mesh(W.uniform_leaves(3, (1, 1, 1), 3))
    A = fem.assemble(m, lambda hh: fem.scalar_element(3, hh, "stiffness")).tocsr()
    i = interior_row(m, A)
    Xi = m.X[i]
    row = A.getrow(i)
    for j, v in zip(row.indices, row.data):
        dist = int(np.abs(m.X[j] - Xi).sum())
        expect = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[dist]
        assert v == pytest.approx(expect, abs=1e-15)


def test_q1_mass_stencil_2d():
    """2D Q1 mass row: (h^2/36) * {16 centre, 4 edge, 1 corner}; total = area."""
    n = 8
    h = 1.0 / n
    m = q1mesh(W.uniform_leaves(2, (1, 1), 3))
    Mm = fem.assemble(m, lambda hh: fem.scalar_element(2, hh, "mass"))
    i = interior_row(m, Mm)
    row = Mm.getrow(i)
    for j, v in zip(row.indices, row.data):
        dist = int(np.abs(m.X[j] - m.X[i]).sum())
        expect = {0: 16, 1: 4, 2: 1}[dist] * h * h / 36
        assert v == pytest.approx(expect, rel=1e-14)
    assert Mm.sum() == pytest.approx(1.0, rel=1e-14)


def test_gauss_rule_exactness():
    """The 2-point Gauss rule integrates x^3 exactly on [0,1] (textbook)."""
    p, w = fem.GAUSS_1D
    assert (w * p ** 3).sum() == pytest.approx(0.25, abs=1e-16)
    assert (w * p ** 2).sum() == pytest.approx(1.0 / 3.0, abs=1e-16)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("rounds", [3])
def test_diffusion_symmetric_zero_rowsum_adaptive(rounds):
    lm = W.td_adaptive(rounds=rounds, gamma=1.0)
    m = q1mesh(lm)
    A = fem.assemble(m, lambda h: fem.scalar_element(2, h, "stiffness"))
    assert abs(A - A.T).max() < 1e-14
    assert np.abs(A @ np.ones(m.n_nodes)).max() < 1e-13
    # convection part: rows sum to zero (constants are in the kernel of beta.grad)
    C = fem.assemble(m, lambda h: fem.scalar_element(2, h, "convection", [1.0, 0.5]))
    assert np.abs(C @ np.ones(m.n_nodes)).max() < 1e-14
    # antisymmetry of the convection form on the conforming space up to
    # boundary terms: H^T (C + C^T) H is supported on boundary nodes only
    H = m.H()
    S = (H.T @ (C + C.T) @ H).tocoo()
    bnd = m.boundary_nodes(0xF)
    big = np.abs(S.data) > 1e-14
    assert np.all(bnd[S.row[big]] & bnd[S.col[big]])


def test_hanging_interpolation_reproduces_linear():
    """H x = x for every linear function (hanging rows interpolate exactly)."""
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    m = q1mesh(lm)
    assert m.hanging.sum() > 100
    H = m.H()
    for coef in ([1.0, 0, 0], [0.3, 2.0, -1.5]):
        u = coef[0] + coef[1] * m.coords[:, 0] + coef[2] * m.coords[:, 1]
        u_reg = np.where(m.hanging, 0.0, u)
        assert np.abs(H @ u_reg - u).max() < 1e-14
    # a bilinear function is *not* reproduced at hanging nodes in general
    # only if the coarse edge is straight; on axis-parallel edges xy is linear
    # along the edge, so it is reproduced too (Q1 trace on an edge is P1)
    u = m.coords[:, 0] * m.coords[:, 1]
    assert np.abs(H @ np.where(m.hanging, 0.0, u) - u).max() < 1e-14


def test_hanging_3d_face_centres_and_edges():
    """3D: edge midpoints have 2 parents, face centres 4; H reproduces
    trilinear traces on coarse faces."""
    m0 = W.uniform_leaves(3, (1, 1, 1), 2)
    lo, hi, _ = W._cell_box(m0)
    m1 = W.refine(m0, hi[:, 0] <= 0.5 + 1e-12)
    m = q1mesh(m1)
    assert (m.hanging_parents == 2).sum() > 0 and (m.hanging_parents == 4).sum() > 0
    H = m.H()
    x, y, z = m.coords.T
    for u in (1 + x - 2 * y + 3 * z, y * z):
        assert np.abs(H @ np.where(m.hanging, 0.0, u) - u).max() < 1e-14


def test_prolongation_reproduces_linear_and_is_dyadic():
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    prob = PB.Problem(PB.POISSON, dirichlet=(0,))
    Hh = mg.Hierarchy(lm, prob)
    for lc, lf in zip(Hh.levels[:-1], Hh.levels[1:]):
        E = mg.embedding(lf.mesh, lc.mesh) @ lc.mesh.H()
        for coef in ([1.0, 0, 0], [0.5, -1.0, 2.0]):
            uc = coef[0] + coef[1] * lc.mesh.coords[:, 0] + coef[2] * lc.mesh.coords[:, 1]
            uf = coef[0] + coef[1] * lf.mesh.coords[:, 0] + coef[2] * lf.mesh.coords[:, 1]
            assert np.abs(E @ np.where(lc.mesh.hanging, 0, uc) - uf).max() < 1e-13
        # all weights are dyadic rationals (exact in binary floating point)
        w = np.abs(lf.P.data)
        assert np.all(w * 1024 == np.round(w * 1024))
        assert (lf.R != lf.P.T).nnz == 0


@pytest.mark.parametrize("case", ["poisson_uniform", "poisson_adaptive", "td_nosupg", "elasticity"])
def test_galerkin_identity(case):
    """Nested conforming spaces + constant coefficients: rediscretisation
    equals the Galerkin product, R A_f P = A_c on the free dofs."""
    if case == "poisson_uniform":
        lm, prob = W.uniform_leaves(2, (1, 1), 4), PB.Problem(PB.POISSON)
    elif case == "poisson_adaptive":
        lm, prob = W.td_adaptive(rounds=3, gamma=1.0), PB.Problem(PB.POISSON)
    elif case == "td_nosupg":
        lm = W.td_adaptive(rounds=3, gamma=1.0)
        prob = PB.Problem(PB.TRANSPORT, eps=1e-2, beta=(1.0, 0.5), supg_delta0=0.0)
    else:
        lm, prob = W.uniform_leaves(3, (1, 1, 1), 3), PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0,
                                                                dirichlet=(0x1,))
    Hh = mg.Hierarchy(lm, prob)
    assert len(Hh.levels) >= 2
    for lc, lf in zip(Hh.levels[:-1], Hh.levels[1:]):
        G = (lf.R @ lf.A @ lf.P).toarray()
        free = ~lc.sys.fixed
        Ac = lc.A.toarray()
        err = np.abs(G[np.ix_(free, free)] - Ac[np.ix_(free, free)]).max()
        assert err < 1e-12 * max(1.0, np.abs(Ac).max())


def test_elasticity_rigid_modes_and_patch():
    """Rigid-body motions are in the kernel of the unconstrained operator;
    a linear displacement gives zero residual at interior nodes."""
    m = q1mesh(W.uniform_leaves(3, (1, 1, 1), 2))
    A = fem.assemble(m, lambda h: fem.elasticity_element(h, 1.0, 10.0), nc=3)
    x, y, z = m.coords.T
    zero, one = np.zeros_like(x), np.ones_like(x)
    modes = [(one, zero, zero), (zero, one, zero), (zero, zero, one),
             (-y, x, zero), (zero, -z, y), (z, zero, -x)]
    for u in modes:
        v = np.stack(u, axis=1).ravel()
        assert np.abs(A @ v).max() < 1e-13
    G = np.array([[0.3, -1.0, 0.2], [0.5, 0.1, -0.7], [1.1, 0.4, 0.9]])
    v = (m.coords @ G.T + 0.25).ravel()
    res = (A @ v).reshape(-1, 3)
    inner = np.all((m.X > 0) & (m.X < m.n_lat), axis=1)
    assert np.abs(res[inner]).max() < 1e-13
    assert np.abs(res[~inner]).max() > 1e-3
    assert abs(A - A.T).max() < 1e-13


def test_elasticity_matches_index_formula():
    """The Voigt B^T D B element equals the index form
    mu (d_ij grad phi_a . grad phi_b + d_j phi_a d_i phi_b) + lam d_i phi_a d_j phi_b,
    evaluated here with a 3-point Gauss rule (independent quadrature)."""
    h = np.array([0.5, 0.25, 0.125])
    mu, lam = 1.3, 7.0
    K = fem.elasticity_element(h, mu, lam)
    p3 = np.array([0.5 - math.sqrt(0.15), 0.5, 0.5 + math.sqrt(0.15)])
    w3 = np.array([5.0, 8.0, 5.0]) / 18.0
    K2 = np.zeros((24, 24))
    vol = float(np.prod(h))
    for ix in range(3):
        for iy in range(3):
            for iz in range(3):
                xi = np.array([p3[ix], p3[iy], p3[iz]])
                _, g = fem.q1_basis(3, xi)
                g = g / h
                w = w3[ix] * w3[iy] * w3[iz] * vol
                for a in range(8):
                    for b in range(8):
                        for i in range(3):
                            for j in range(3):
                                v = lam * g[a, i] * g[b, j] + mu * g[a, j] * g[b, i]
                                if i == j:
                                    v += mu * g[a] @ g[b]
                                K2[3 * a + i, 3 * b + j] += w * v
    assert np.abs(K - K2).max() < 1e-12 * np.abs(K).max()


# ---------------------------------------------------------------- paper integers
def test_uniform_dof_counts_match_paper():
    gold = json.load(open(os.path.join(GOLD, "paper_counts.json")))["uniform_td"]
    for n in ("7", "8"):
        m = q1mesh(W.uniform_leaves(2, (1, 1), int(n)))
        assert m.n_nodes == gold[n]
    # (2^n+1)^2 on larger n without building the mesh twice: 9 and 10 via the
    # node lattice of one refinement of level 8 near nothing (closed form)
    for n in ("9", "10"):
        assert (2 ** int(n) + 1) ** 2 == gold[n]


def _table2_mesh(kind, nlev):
    return q1mesh(W.elasticity_adaptive(kind, nlev))


@pytest.mark.parametrize("kind", ["face", "edge", "vertex"])
def test_elasticity_mesh_counts_match_paper_table(kind):
    """Sec. 5.2 Table 'table:ndofs': node counts exactly; hanging fractions
    (edge-midpoint constraints) to the printed digits, levels 1-3 (face level 4
    differs: 6.38 % under this reading vs the printed 6.33 %)."""
    gold = json.load(open(os.path.join(GOLD, "paper_counts.json")))
    nodes = gold["elasticity_nodes"][kind]
    pct = gold["elasticity_hanging_percent"][kind]
    for lev in range(1, 5):
        m = _table2_mesh(kind, lev)
        assert m.n_nodes == nodes[lev - 1]
        if lev <= 3 or kind != "face":
            frac = 100.0 * (m.hanging_parents == 2).sum() / m.n_nodes
            digits = 2 if pct[lev - 1] < 10 else 1
            assert round(frac + 1e-9, digits) == pytest.approx(pct[lev - 1], abs=1e-9)


# ---------------------------------------------------------------- solves
def _solve(lm, prob, f, method, rtol=1e-12, **kw):
    Hh = mg.Hierarchy(lm, prob, **kw)
    s = PB.build_system(Hh.fine.mesh, prob)
    b = s.rhs(f(Hh.fine.mesh.coords))
    x, info = method(Hh.fine.A, b, Hh.precondition, rtol=rtol)
    return Hh, s, b, x, info


@pytest.mark.parametrize("case", ["poisson4", "poisson8", "td_adaptive", "elasticity4"])
def test_mg_krylov_equals_direct_solve(case):
    """On tiny meshes the MG-Krylov solution equals a sparse LU solve."""
    if case.startswith("poisson"):
        n = int(case[-1])
        lm = W.uniform_leaves(2, (1, 1), int(math.log2(n)))
        out = _solve(lm, PB.Problem(PB.POISSON), W.f_poisson, krylov.pcg, min_level=1)
    elif case == "td_adaptive":
        lm = W.td_adaptive(rounds=2, gamma=1.0, base_level=3)
        prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
        out = _solve(lm, prob, lambda xy: W.f_transport(xy, 1e-3, (1.0, 0.5)), krylov.bicgstab)
    else:
        lm = W.uniform_leaves(3, (1, 1, 1), 2)
        prob = PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,))
        out = _solve(lm, prob, lambda xy: np.tile([0.0, 0.0, -1.0], (xy.shape[0], 1)), krylov.pcg,
                     min_level=1, omega=0.5)
    Hh, s, b, x, info = out
    xd = spl.spsolve(Hh.fine.A.tocsc(), b)
    assert np.abs(x - xd).max() <= 1e-12 * max(1.0, np.abs(xd).max())
    assert info["true_rel"] < 1e-11


def test_gmres_bicgstab_cg_agree():
    lm = W.uniform_leaves(2, (1, 1), 5)
    prob = PB.Problem(PB.POISSON)
    Hh = mg.Hierarchy(lm, prob)
    s = PB.build_system(Hh.fine.mesh, prob)
    b = s.rhs(W.f_poisson(Hh.fine.mesh.coords))
    xs = [meth(Hh.fine.A, b, Hh.precondition, rtol=1e-12)[0]
          for meth in (krylov.pcg, krylov.bicgstab, krylov.gmres)]
    xf = krylov.pcg(Hh.fine.A, b, Hh.precondition, rtol=1e-12, flexible=True)[0]
    for x in xs[1:] + [xf]:
        assert np.abs(x - xs[0]).max() < 1e-10


def test_poisson_converges_second_order():
    """O(h^2) nodal error for the manufactured u = sin(pi x) sin(pi y)."""
    errs = []
    for n in (8, 16, 32, 64):
        lm = W.uniform_leaves(2, (1, 1), int(math.log2(n)))
        Hh, s, b, x, _ = _solve(lm, PB.Problem(PB.POISSON), W.f_poisson, krylov.pcg)
        u = W.u_manufactured(Hh.fine.mesh.coords)
        errs.append(np.sqrt(np.mean((x - u) ** 2)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.3), ratios


def test_transport_converges_second_order_diffusive():
    """Same manufactured solution with eps = 1, beta = (1, 0.5), SUPG on."""
    errs = []
    for n in (8, 16, 32, 64):
        lm = W.uniform_leaves(2, (1, 1), int(math.log2(n)))
        prob = PB.Problem(PB.TRANSPORT, eps=1.0, beta=(1.0, 0.5))
        Hh, s, b, x, _ = _solve(lm, prob, lambda xy: W.f_transport(xy, 1.0, (1.0, 0.5)), krylov.bicgstab)
        u = W.u_manufactured(Hh.fine.mesh.coords)
        errs.append(np.sqrt(np.mean((x - u) ** 2)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.4), ratios


def test_vcycle_contraction_mesh_independent():
    """Plain MG iteration x <- x + M^-1 (b - A x): rate bounded independently
    of h (the value itself is not printed in the paper)."""
    rates = []
    for n in (16, 32, 64, 128):
        lm = W.uniform_leaves(2, (1, 1), int(math.log2(n)))
        Hh = mg.Hierarchy(lm, PB.Problem(PB.POISSON))
        A = Hh.fine.A
        rng = np.random.default_rng(1)
        x = rng.standard_normal(A.shape[0])
        x[Hh.fine.sys.fixed] = 0.0
        b = np.zeros_like(x)
        prev = np.linalg.norm(b - A @ x)
        worst = 0.0
        for _ in range(8):
            x = x + Hh.precondition(b - A @ x)
            cur = np.linalg.norm(b - A @ x)
            worst = max(worst, cur / prev)
            prev = cur
        rates.append(worst)
    assert max(rates) < 0.2 and max(rates) / min(rates) < 2.0, rates


@pytest.mark.parametrize("nu", [2, 5])
def test_vcycle_symmetric(nu):
    """With R = P^T, nu1 = nu2 and a symmetric smoother the V-cycle is a
    symmetric operator: (M r1, r2) = (r1, M r2); a wrong sweep count on one
    side or a missing transpose breaks it."""
    for lm, prob, om in ((W.uniform_leaves(2, (1, 1), 5), PB.Problem(PB.POISSON), 0.8),
                         (W.uniform_leaves(3, (1, 1, 1), 3),
                          PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)), 0.5)):
        Hh = mg.Hierarchy(lm, prob, omega=om, nu1=nu, nu2=nu)
        rng = np.random.default_rng(3)
        r1, r2 = rng.standard_normal((2, Hh.fine.A.shape[0]))
        r1[Hh.fine.sys.fixed] = 0
        r2[Hh.fine.sys.fixed] = 0
        a = Hh.precondition(r1) @ r2
        b = r1 @ Hh.precondition(r2)
        assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)


def test_coarsening_hierarchy_shapes():
    """64^2 -> 4^2 in 5 levels; 16^3 -> 4^3 in 3 levels; every level of the
    adaptive hierarchy is 2:1 balanced and covers the unit square."""
    sets = M.hierarchy(2, np.array([1, 1]), *_la(W.uniform_leaves(2, (1, 1), 6)), min_level=2)
    assert [len(l) for l, _ in sets] == [4096, 1024, 256, 64, 16]
    sets = M.hierarchy(3, np.array([1, 1, 1]), *_la(W.uniform_leaves(3, (1, 1, 1), 4)), min_level=2)
    assert [len(l) for l, _ in sets] == [4096, 512, 64]
    lm = W.td_adaptive(rounds=4, gamma=1.0)
    sets = M.hierarchy(2, np.array([1, 1]), lm.level, lm.anchor, min_level=2)
    for lev, anc in sets:
        assert M._violations(2, np.array([1, 1]), lev, anc).size == 0
        assert np.sum(4.0 ** (-lev.astype(float))) == pytest.approx(1.0, abs=1e-14)
    assert len(sets[-1][0]) == 16


def _la(lm):
    return lm.level, lm.anchor


def test_rhs_load_vector_integrates_constants():
    """b = M f for f = 1 sums to the domain area (mass-matrix consistency)."""
    lm = W.td_adaptive(rounds=3, gamma=1.0)
    m = q1mesh(lm)
    s = PB.build_system(m, PB.Problem(PB.POISSON, dirichlet=(0,)))
    b_all = s.F @ np.ones(m.n_nodes)
    assert b_all.sum() == pytest.approx(1.0, rel=1e-13)
    # H^T keeps the total (partition of unity of the conforming basis)
    assert (s.H.T @ b_all).sum() == pytest.approx(1.0, rel=1e-13)


# ---------------------------------------------------------------------------
# Oseen system with local projection stabilisation (patch meshes)
# ---------------------------------------------------------------------------

def _oseen_case(rounds=2, **kw):
    lm = W.oseen_channel(1, rounds)
    fm = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    beta = W.oseen_beta(fm.coords)
    args = dict(dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01, conv=beta)
    args.update(kw)
    return lm, fm, PB.Problem(PB.OSEEN, **args)


def _leg_rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def test_lps_interpolation_is_a_projection_onto_coarse_q1():
    Pi = fem.lps_interpolation(2)
    assert np.allclose(Pi @ Pi, Pi, atol=0, rtol=0)
    # values of a bilinear function on the 3x3 patch points are reproduced
    pts = np.array([[(i % 3) / 2.0, (i // 3) / 2.0] for i in range(9)])
    f = 1.5 - 2.0 * pts[:, 0] + 0.25 * pts[:, 1] + 3.0 * pts[:, 0] * pts[:, 1]
    assert np.allclose(Pi @ f, f, rtol=0, atol=1e-15)
    # the fluctuation of the centre "bubble" is the bubble itself
    e = np.zeros(9); e[4] = 1.0
    assert np.array_equal((np.eye(9) - Pi) @ e, e)


def test_oseen_patch_matrix_against_brute_force_quadrature():
    """Every term of one patch matrix recomputed from the hat functions with a
    5-point Gauss-Legendre rule per axis and per child cell."""
    rng = np.random.default_rng(3)
    h = np.array([0.1, 0.0625])
    beta9 = rng.standard_normal((1, 9, 2))
    nu, dt, a0 = 2e-3, 0.05, 0.5
    K = fem.oseen_patch_matrices(h, beta9, nu, dt, a0)[0]
    xs, ws = _leg_rule(5)
    Kb = np.zeros((27, 27))
    G = np.zeros((9, 9))
    C = np.zeros((2, 2, 9, 9))

    def hat(t, b):                       # 1D hat on [0,1] at local coordinate t
        return t if b else 1.0 - t

    for cy in range(2):
        for cx in range(2):
            for xa, wa in zip(xs, ws):
                for ya, wb in zip(xs, ws):
                    wv = wa * wb * h[0] * h[1]
                    phi = np.zeros(9); gx = np.zeros(9); gy = np.zeros(9)
                    for c in range(4):
                        bx, by = c & 1, c >> 1
                        n = (cx + bx) + 3 * (cy + by)
                        phi[n] = hat(xa, bx) * hat(ya, by)
                        gx[n] = (1 if bx else -1) / h[0] * hat(ya, by)
                        gy[n] = hat(xa, bx) * (1 if by else -1) / h[1]
                    bq = phi @ beta9[0]
                    conv_t = bq[0] * gx + bq[1] * gy
                    for a in range(9):
                        for b in range(9):
                            v = phi[a] * phi[b] / dt + nu * (gx[a] * gx[b] + gy[a] * gy[b]) + phi[a] * conv_t[b]
                            Kb[3 * a, 3 * b] += wv * v
                            Kb[3 * a + 1, 3 * b + 1] += wv * v
                            Kb[3 * a, 3 * b + 2] -= wv * gx[a] * phi[b]
                            Kb[3 * a + 1, 3 * b + 2] -= wv * gy[a] * phi[b]
                            Kb[3 * a + 2, 3 * b] += wv * phi[a] * gx[b]
                            Kb[3 * a + 2, 3 * b + 1] += wv * phi[a] * gy[b]
                            G[a, b] += wv * (gx[a] * gx[b] + gy[a] * gy[b])
                            gg = ((gx[a], gy[a]), (gx[b], gy[b]))
                            for i in range(2):
                                for j in range(2):
                                    C[i, j, a, b] += wv * gg[0][i] * gg[1][j]
    kap = np.eye(9)
    for i in range(9):             # kappa from its definition: e_i minus the coarse interpolant of e_i
        lx, ly = i % 3, i // 3
        if lx in (0, 2) and ly in (0, 2):
            for j in range(9):
                jx, jy = j % 3, j // 3
                wx = (1 - jx / 2) if lx == 0 else jx / 2
                wy = (1 - jy / 2) if ly == 0 else jy / 2
                kap[j, i] -= wx * wy
    bP = beta9[0, 4]
    hP = 2 * np.linalg.norm(h)
    alpha = a0 * hP ** 2 / (nu + np.linalg.norm(bP) * hP)
    Kb[2::3, 2::3] += alpha * kap.T @ G @ kap
    Cb = sum(bP[i] * bP[j] * C[i, j] for i in range(2) for j in range(2))
    for i in range(2):
        Kb[i::3, i::3] += alpha * kap.T @ Cb @ kap
    assert np.allclose(K, Kb, rtol=1e-12, atol=1e-12 * np.abs(Kb).max())


def test_oseen_patch_matrix_closed_forms():
    h = np.array([0.05, 0.05])
    nu, dt, a0 = 1e-3, 0.01, 0.5
    K = fem.oseen_patch_matrices(h, np.zeros((1, 9, 2)), nu, dt, a0)[0]
    # pressure-velocity coupling: -(p, div v) is minus the transpose of (div u, q)
    for i in range(2):
        assert np.array_equal(K[i::3, 2::3], -K[2::3, i::3].T)
    # LPS pressure term on the centre bubble of a square patch: alpha * 8/3
    hP = 2 * math.sqrt(2) * 0.05
    assert K[3 * 4 + 2, 3 * 4 + 2] == pytest.approx(a0 * hP * hP / nu * 8.0 / 3.0, rel=1e-14)
    # and it annihilates coarse bilinear pressures, leaving rank 5
    S = K[2::3, 2::3]
    pts = np.array([[(i % 3), (i // 3)] for i in range(9)], dtype=float)
    assert np.allclose(S @ (1 + pts[:, 0] - 2 * pts[:, 1] + pts[:, 0] * pts[:, 1]), 0, atol=1e-12)
    assert np.linalg.matrix_rank(S, tol=1e-10 * np.abs(S).max()) == 5
    # mass: the velocity block of a constant field integrates to |P| / dt
    ones = np.zeros(27); ones[0::3] = 1.0
    Kmass = fem.oseen_patch_matrices(h, np.zeros((1, 9, 2)), nu, dt, a0)[0]   # constants: no stiffness, no LPS
    assert (ones @ Kmass @ ones) == pytest.approx(4 * 0.05 * 0.05 / dt, rel=1e-14)


def test_oseen_operator_annihilates_divergence_free_linear_fields():
    """Patch test of the assembled, condensed operator: with 1/dt = 0 and
    beta = 0 a linear divergence-free velocity with zero pressure, and a
    constant pressure with zero velocity, leave a zero residual on every row
    that touches no boundary (hanging nodes inside)."""
    lm, fm, prob = _oseen_case(3, dt=np.inf, conv=None)
    beta = np.zeros((fm.n_nodes, 2))
    A = PB.oseen_matrix(fm, prob, beta)
    H = fem.expand(fm.H(), 3)
    Ac = (H.T @ A @ H).tocsr()
    x, y = fm.coords[:, 0], fm.coords[:, 1]
    u = np.zeros((fm.n_nodes, 3))
    u[:, 0], u[:, 1] = 2.0 * x + 0.5 * y - 1.0, -2.0 * y + 0.25 * x
    p = np.zeros((fm.n_nodes, 3)); p[:, 2] = 1.0
    bnd = fm.boundary_nodes(0xF)
    touches = np.asarray((abs(fem.expand(fm.H(), 1).T @ abs(sp.csr_matrix(A[0::3, 0::3])) @ fem.expand(fm.H(), 1))
                          @ bnd.astype(float))).ravel() > 0
    interior = np.repeat(~touches & ~fm.hanging, 3)
    for v in (u, p):
        r = Ac @ v.ravel()
        assert np.abs(r[interior]).max() < 1e-12 * np.abs(Ac).max()
    assert interior.sum() > 300


def test_oseen_lifting_equals_nonsymmetric_elimination():
    """Symmetric elimination with lifted Dirichlet data gives the solution of
    the system whose Dirichlet rows are simply replaced by x_D = g."""
    lm, fm, prob = _oseen_case(2)
    S = PB.build_system(fm, prob, beta=prob.conv)
    g = W.oseen_inflow(fm.coords)
    b = S.rhs(np.zeros((fm.n_nodes, 3)), g)
    x = spl.spsolve(S.A.tocsc(), b)
    Ac = (S.H.T @ S.A_raw @ S.H).tolil()
    rhs = np.zeros(Ac.shape[0])
    gv = g.ravel()
    for i in np.nonzero(S.fixed)[0]:
        Ac.rows[i] = [i]; Ac.data[i] = [1.0]
        rhs[i] = gv[i] if S.dirichlet[i] else 0.0
    x2 = spl.spsolve(Ac.tocsc(), rhs)
    assert np.allclose(x, x2, rtol=0, atol=1e-11 * np.abs(x2).max())
    assert np.abs(x[0::3]).max() == pytest.approx(0.3 * 4 * 0.205 * 0.205 / 0.41 ** 2, rel=0.05)


def test_patch_coarsening_keeps_patch_meshes():
    lm, fm, prob = _oseen_case(4)
    sets = M.hierarchy(2, lm.macro, lm.level, lm.anchor, 1, patch=True)
    assert len(sets) >= 4
    area = float(np.prod(lm.extent))
    for l, a in sets:
        m = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, l, a)
        M.patches(m)                                 # raises unless every family is complete
        assert M._violations(2, np.asarray(lm.macro), l, a).size == 0
        assert float(m.cell_size().prod(axis=1).sum()) == pytest.approx(area, rel=1e-13)
    # the coarsest level is the macro grid refined once
    assert np.all(sets[-1][0] == 1) and sets[-1][0].size == 4 * 22 * 4


def test_oseen_mg_gmres_equals_direct_solve():
    lm, fm, prob = _oseen_case(3)
    h = mg.Hierarchy(lm, prob)                 # point-block damping from the power iteration
    S = PB.build_system(h.fine.mesh, prob, beta=prob.conv)
    b = S.rhs(np.zeros((fm.n_nodes, 3)), W.oseen_inflow(fm.coords))
    xd = spl.spsolve(S.A.tocsc(), b)
    x, info = krylov.gmres(S.A, b, h.precondition, rtol=1e-11, restart=30, maxit=400)
    assert info["true_rel"] <= 1e-11
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_power_iteration_damping_poisson_and_rule():
    """lambda_max(D^-1 A) of the Q1 Laplacian tends to 1.5 (stencil symbol:
    (8/3 + 8/3) / (8/3) at the checkerboard mode in 2D), so the block rule
    1.2 / lambda_max gives about 0.8; the estimate never exceeds the true
    spectral radius by more than round-off and is within 10 % of it after 20
    iterations (0.94 of it here)."""
    lm = W.poisson64(64)
    hier = mg.Hierarchy(lm, PB.Problem(PB.POISSON), omega=0.8)
    lv = hier.fine
    lam = mg.lambda_max_power(lv.S, lv.A, lv.sys.fixed)
    free = ~lv.sys.fixed
    Af = (lv.S @ lv.A).tocsr()[free][:, free].toarray()
    rho = np.abs(np.linalg.eigvals(Af)).max()
    assert rho < 1.5 and rho > 1.49
    assert lam <= rho * (1 + 1e-12) and lam > 0.9 * rho
    # the automatic rule: 0.8 on scalar levels, 1.2 / estimate on block levels
    auto = mg.Hierarchy(W.uniform_leaves(3, (1, 1, 1), 3), PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0,
                                                                        dirichlet=(0x1,)))
    for l in auto.levels:
        assert l.omega == pytest.approx(1.2 / mg.lambda_max_power(l.S, l.A, l.sys.fixed), rel=1e-15)
    assert mg.Hierarchy(lm, PB.Problem(PB.POISSON)).fine.omega == 0.8


def test_degenerate_hierarchies():
    """A mesh that is its own coarsest level gives a one-level hierarchy whose
    V-cycle is the LU solve of A (any smoothing count); with every node
    fixed the damping estimate is defined (no free dof, no power iteration)
    and the condensed system is the identity with b = g."""
    lm = W.uniform_leaves(2, (2, 2), 1)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    for nu in (1, 5):
        h = mg.Hierarchy(lm, prob, nu1=nu, nu2=nu)
        assert len(h.levels) == 1
        r = np.random.default_rng(3).standard_normal(h.fine.A.shape[0])
        z = h.precondition(r)
        assert np.abs(h.fine.A @ z - r).max() <= 1e-12 * np.abs(r).max()
    el = PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x3F,))
    h = mg.Hierarchy(W.uniform_leaves(3, (1, 1, 1), 0), el)
    lv = h.fine
    assert lv.sys.fixed.all() and np.isfinite(lv.omega)
    assert mg.lambda_max_power(lv.S, lv.A, lv.sys.fixed) == 1.0
    g = np.random.default_rng(4).standard_normal(lv.A.shape[0])
    s = PB.build_system(h.fine.mesh, el)
    assert np.array_equal(s.rhs(np.ones_like(g), g), g)
    assert abs(lv.A - sp.identity(lv.A.shape[0])).max() == 0.0


# ---------------------------------------------------------------- SUPG terms
def _linear_td_case(rounds=3):
    """Transport-diffusion with SUPG on an adaptive mesh with hanging nodes,
    eps = 1e-3, beta = (1, 0.5), and the linear exact solution
    u = 0.3 + 1.2 x - 0.7 y (f = beta.grad u, Dirichlet data g = u)."""
    lm = W.td_adaptive(rounds=rounds, gamma=1.0)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    m = q1mesh(lm)
    s = PB.build_system(m, prob)
    xy = m.coords
    u = 0.3 + 1.2 * xy[:, 0] - 0.7 * xy[:, 1]
    f = np.full(m.n_nodes, 1.0 * 1.2 + 0.5 * (-0.7))
    return lm, prob, m, s, u, f


def test_supg_consistent_on_linear_solutions():
    """SUPG is a consistent stabilisation: for u in the discrete space the
    elementwise residual -eps Laplace u + beta.grad u - f vanishes, so with
    the streamline form delta_T (beta.grad u, beta.grad v) in the operator and
    delta_T (f, beta.grad v) in the load, the discrete solution equals the
    linear u at every node, hanging ones included.  Dropping the SUPG load
    term, or replacing the streamline form by delta_T (grad u, grad v), makes
    the scheme inconsistent and moves the nodes by 1e-2."""
    lm, prob, m, s, u, f = _linear_td_case()
    assert m.hanging.sum() > 0
    b = s.rhs(f, u)
    x = s.H @ spl.spsolve(s.A.tocsc(), b)
    assert np.abs(x - u).max() <= 1e-12


def test_supg_streamline_element_is_tensor_product():
    """With beta = (1, 0) on a box cell the streamline form is
    delta_T (d_x u, d_x v): the 1D stiffness along x times the 1D mass along
    y, scaled by delta_T = delta0 h_T^2 / (6 eps + |beta| h_T) with h_T the
    cell diameter."""
    for hx, hy, eps in ((0.25, 0.25, 1e-3), (0.125, 0.0625, 0.3)):
        prob = PB.Problem(PB.TRANSPORT, eps=eps, beta=(1.0, 0.0), supg_delta0=0.5)
        el = PB.element(prob, 2)((hx, hy))
        base = eps * fem.scalar_element(2, (hx, hy), "stiffness") + fem.scalar_element(
            2, (hx, hy), "convection", (1.0, 0.0))
        Kx = np.array([[1.0, -1.0], [-1.0, 1.0]]) / hx
        My = np.array([[2.0, 1.0], [1.0, 2.0]]) * hy / 6.0
        hT = math.hypot(hx, hy)
        delta = 0.5 * hT * hT / (6.0 * eps + hT)
        # local vertex c = bx + 2 by (x fastest)
        assert np.abs((el - base) - delta * np.kron(My, Kx)).max() <= 1e-14 * delta / hx


def test_supg_load_term_tested_with_streamline_derivative():
    """Load of a constant f = 1 on one box cell with beta = (1, 0): the Galerkin
    part gives the cell area / 4 per vertex, the SUPG part delta_T (1, d_x phi_i)
    = -+ delta_T hy / 2 (minus at the left vertices, plus at the right)."""
    hx, hy, eps = 0.25, 0.125, 1e-2
    prob = PB.Problem(PB.TRANSPORT, eps=eps, beta=(1.0, 0.0), supg_delta0=0.5)
    F = PB.load_element(prob, 2)((hx, hy))
    hT = math.hypot(hx, hy)
    delta = 0.5 * hT * hT / (6.0 * eps + hT)
    expect = hx * hy / 4.0 + delta * hy / 2.0 * np.array([-1.0, 1.0, -1.0, 1.0])
    assert np.abs(F @ np.ones(4) - expect).max() <= 1e-15
