"""The library's host-built hierarchy against the oracle (CPU, no GPU).

Level operators, transfers, smoother blocks, the coarse inverse and the
right-hand-side load matrix that ``mg_setup`` would upload are compared entry
by entry with the oracle's independently assembled matrices; the integer
structure (levels, node counts, fixed-dof masks) must agree exactly.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import mesh as M
from oracle import mg
from oracle import problems as PB
from paper_2405_05047_gb300 import binding as B
from paper_2405_05047_gb300 import hostview as HV

CASES = {
    "poisson16": (lambda: W.uniform_leaves(2, (1, 1), 4), PB.Problem(PB.POISSON),
                  dict(kind=B.MG_POISSON)),
    "td_adaptive": (lambda: W.td_adaptive(rounds=3, gamma=1.0),
                    PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5)),
                    dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))),
    "elasticity8": (lambda: W.uniform_leaves(3, (1, 1, 1), 3),
                    PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                    dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,))),
    "elasticity_adaptive": (lambda: W.refine(W.uniform_leaves(3, (1, 1, 1), 2),
                                             W._cell_box(W.uniform_leaves(3, (1, 1, 1), 2))[1][:, 0] <= 0.5 + 1e-12),
                            PB.Problem(PB.ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                            dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,))),
    # backward-Euler step matrices of the time-dependent problem (mass 1/dt)
    "td_step": (lambda: W.td_uniform(32),
                PB.Problem(PB.TRANSPORT, eps=0.01, beta=(0.0, -1.0), supg_delta0=0.0, mass=50.0),
                dict(kind=B.MG_TRANSPORT, eps=0.01, beta=(0.0, -1.0), supg_delta0=0.0, mass=50.0)),
    "td_step_supg_adaptive": (lambda: W.td_adaptive(rounds=3, gamma=1.0),
                              PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5), mass=10.0),
                              dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5), mass=10.0)),
    "elasticity_step_edge": (lambda: W.elasticity_adaptive("edge", 2),
                             PB.Problem(PB.ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=(0x3F,),
                                        mass=1.0 / W.EL_DT ** 2),
                             dict(kind=B.MG_ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=(0x3F,),
                                  mass=1.0 / W.EL_DT ** 2)),
    "poisson_mass": (lambda: W.uniform_leaves(2, (1, 1), 4), PB.Problem(PB.POISSON, mass=3.0),
                     dict(kind=B.MG_POISSON, mass=3.0)),
    # graded box of the driven cavity: per-cell element matrices, pure
    # Neumann problem with the origin node pinned
    "ns_pressure_graded": (lambda: W.ns_cavity_mesh(8, 8, 16),
                           PB.Problem(PB.POISSON, dirichlet=(0,), pin_origin=True),
                           dict(kind=B.MG_POISSON, dirichlet=(0,), pin_origin=1)),
    "graded_transport2d": (lambda: _graded2d(),
                           PB.Problem(PB.TRANSPORT, eps=1e-2, beta=(1.0, 0.5)),
                           dict(kind=B.MG_TRANSPORT, eps=1e-2, beta=(1.0, 0.5))),
    "channel": (lambda: W.oseen_channel(uniform=1, rounds=3),
                PB.Problem(PB.TRANSPORT, eps=1e-2, beta=(1.0, 0.3), dirichlet=(0b1101,)),
                dict(kind=B.MG_TRANSPORT, eps=1e-2, beta=(1.0, 0.3), dirichlet=(0b1101,))),
}


def _graded2d():
    m = W.uniform_leaves(2, (3, 1), 3)
    n = [3 * 8 + 1, 8 + 1]
    m.axis = tuple(np.sort(np.concatenate([[0.0, 1.0], np.random.default_rng(7 + d).random(k - 2)]))
                   for d, k in enumerate(n))
    return m


def close(a, b, tol=1e-13):
    a, b = sp.csr_matrix(a), sp.csr_matrix(b)
    d = (a - b).tocsr()
    scale = max(abs(b).max(), 1e-300)
    return abs(d).max() <= tol * scale if d.nnz else True


@pytest.mark.parametrize("name", list(CASES))
def test_host_hierarchy_matches_oracle(name):
    mk, prob, pkw = CASES[name]
    lm = mk()
    oh = mg.Hierarchy(lm, prob)
    hh = HV.HostHierarchy(lm, B.make_problem(**pkw))
    _compare(oh, hh, prob)


@pytest.mark.parametrize("rounds", [2, 4])
def test_host_hierarchy_oseen_matches_oracle(rounds):
    """Oseen + LPS on a patch mesh: per-level operators (patch-preserving
    coarsening, injected convection field), transfers, 3x3 point blocks, the
    load matrix and the lifting couplings of the Dirichlet data."""
    lm = W.oseen_channel(1, rounds)
    xy = B.mg_mesh_nodes(lm)
    fm = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    assert np.array_equal(xy, fm.coords)
    beta = W.oseen_beta(xy)
    kw = dict(dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01)
    prob = PB.Problem(PB.OSEEN, conv=beta, **kw)
    oh = mg.Hierarchy(lm, prob)
    hh = HV.HostHierarchy(lm, B.make_problem(kind=B.MG_OSEEN, conv=beta, **kw))
    _compare(oh, hh, prob, tol=1e-12)
    # lifting: the free-row x Dirichlet-column part of H^T A H
    S = PB.build_system(oh.fine.mesh, prob, beta=beta)
    Ac = (S.H.T @ S.A_raw @ S.H).tocsr()
    free = (~S.fixed).astype(float)
    Lo = sp.diags(free) @ Ac @ sp.diags(S.dirichlet.astype(float))
    assert close(hh.matrix(hh.levels - 1, HV.LIFT), Lo, 1e-12)


@pytest.mark.parametrize("rounds", [2, 6])
def test_oseen_level_blocks_have_velocity_pressure_pattern(rounds):
    """Every 3x3 block of every Oseen level operator the setup builds is
    [[a, 0, g1], [0, a, g2], [d1, d2, c]] exactly (the two velocity
    components share one operator and do not couple): the condition under
    which the library stores 6 values per block.  Elasticity blocks are not."""
    lm = W.oseen_channel(1, rounds)
    beta = W.oseen_beta(B.mg_mesh_nodes(lm))
    hh = HV.HostHierarchy(lm, B.make_problem(kind=B.MG_OSEEN, conv=beta, dirichlet=(0xD, 0xD, 0x0), nu=1e-3,
                                             dt=0.01))
    for l in range(hh.levels):
        A = hh.matrix(l, HV.A).tocsr()
        C = A.tocoo()
        ru, cu = C.row % 3, C.col % 3
        assert not np.any(C.data[(ru == 0) & (cu == 1)]) and not np.any(C.data[(ru == 1) & (cu == 0)])
        assert (A[0::3, 0::3] != A[1::3, 1::3]).nnz == 0
    he = HV.HostHierarchy(W.uniform_leaves(3, (1, 1, 1), 2),
                          B.make_problem(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)))
    C = he.matrix(he.levels - 1, HV.A).tocoo()
    assert np.any(C.data[(C.row % 3 == 0) & (C.col % 3 == 1)])


def test_oseen_rejects_non_patch_mesh():
    lm = W.oseen_channel(1, 0)
    lm = W.refine(lm, np.arange(lm.n_leaves) == 5)       # one leaf refined alone: its family is incomplete
    beta = np.zeros((B.mg_mesh_nodes(lm).shape[0], 2))
    with pytest.raises(B.MGError, match="patch mesh"):
        HV.HostHierarchy(lm, B.make_problem(kind=B.MG_OSEEN, conv=beta, dirichlet=(0xD, 0xD, 0)))


def _compare(oh, hh, prob, tol=1e-13):
    assert hh.levels == len(oh.levels)
    nc = prob.nc
    for l, lv in enumerate(oh.levels):
        A = hh.matrix(l, HV.A)
        assert A.shape == lv.A.shape
        assert close(A, lv.A, tol), f"A level {l}"
        fm = hh.fixmask(l)
        fixed = np.zeros(lv.mesh.n_nodes * nc, dtype=bool)
        for c in range(nc):
            fixed[c::nc] = (fm >> c) & 1
        assert np.array_equal(fixed, lv.sys.fixed)
        assert hh.omega(l) == pytest.approx(lv.omega, rel=1e-12), f"omega level {l}"
        S = hh.matrix(l, HV.SMOOTHER)
        assert close(S, lv.S, max(tol, 1e-12)), f"smoother level {l}"
        if l > 0:
            # the library's scalar P, with the per-component rows of partly
            # fixed nodes masked (as its kernels do), is each component block
            # of the oracle's P_eff
            Pl = hh.matrix(l, HV.P)
            fc = hh.fixmask(l - 1)
            for c in range(nc):
                keep_f = sp.diags(((fm >> c) & 1 == 0).astype(float))
                keep_c = sp.diags(((fc >> c) & 1 == 0).astype(float))
                assert close(keep_f @ Pl @ keep_c, lv.P[c::nc, c::nc], 0.0), f"P level {l} comp {c}"
            Rl = hh.matrix(l, HV.R)
            assert (abs(Rl - Pl.T) > 0).nnz == 0
    inv = hh.coarse_inverse()
    A0 = oh.levels[0].A.toarray()
    assert np.abs(inv @ A0 - np.eye(A0.shape[0])).max() < 1e-11
    # load matrix: b = H^T F f on the finest level
    sysf = PB.build_system(oh.fine.mesh, prob, beta=prob.conv)
    F = hh.matrix(hh.levels - 1, HV.LOAD)
    Fo = (oh.fine.mesh.H().T @ sysf.F).tocsr()
    hang = oh.fine.mesh.hanging
    Fo = sp.diags((~hang).astype(float)) @ Fo
    Fl = sp.diags((~hang).astype(float)) @ F
    assert close(Fl, Fo), "load matrix"


@pytest.mark.parametrize("case", ["oseen", "td_adaptive", "elasticity_adaptive"])
def test_host_vanka_matrices_match_oracle(case):
    """The cell-patch Vanka matrix of every level that uses it equals the
    oracle's W sum_T P_T A_T^-1 P_T^T (local inverses formed independently:
    Gauss-Jordan in the library, LAPACK in the oracle); the levels below
    vanka_rows keep the Jacobi smoother in both."""
    if case == "oseen":
        lm = W.oseen_channel(1, 3)
        xy = B.mg_mesh_nodes(lm)
        beta = W.oseen_beta(xy)
        kw = dict(dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01)
        prob = PB.Problem(PB.OSEEN, conv=beta, **kw)
        pb = B.make_problem(kind=B.MG_OSEEN, conv=beta, **kw)
        rows = 3000
    elif case == "td_adaptive":
        lm = W.td_adaptive(rounds=3, gamma=1.0)
        prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
        pb = B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
        rows = 0
    else:
        mk, prob, pkw = CASES["elasticity_adaptive"]
        lm, pb, rows = mk(), B.make_problem(**pkw), 0
    oh = mg.Hierarchy(lm, prob, smoother="vanka", vanka_rows=rows)
    hh = HV.HostHierarchy(lm, pb, B.make_opts(smoother=B.MG_SMOOTHER_VANKA, vanka_rows=rows))
    assert hh.levels == len(oh.levels)
    for l, lv in enumerate(oh.levels):
        S = hh.matrix(l, 7)
        if not lv.vanka:
            assert S.shape[0] == 0
            continue
        assert close(S, lv.S, 1e-11)
        assert hh.omega(l) == 1.0


def test_graded_coordinates_and_pin():
    """Node coordinates of a graded mesh come from the axis arrays (library
    and oracle); the pinned node is the origin corner on every level, and a
    graded mesh with mixed leaf levels is refused."""
    lm = W.ns_cavity_mesh(4, 4, 8)
    xyz = B.mg_mesh_nodes(lm)
    from oracle import mesh as M, ns
    fm = M.Q1Mesh(3, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor, axis=lm.axis)
    assert np.array_equal(xyz, fm.coords)
    ax = ns.graded_axes(4, 4, 8)
    assert all(np.allclose(a, b, atol=1e-15) for a, b in zip(ax, lm.axis))
    hh = HV.HostHierarchy(lm, B.make_problem(kind=B.MG_POISSON, dirichlet=(0,), pin_origin=1))
    for l in range(hh.levels):
        fm_l = hh.fixmask(l)
        assert fm_l[0] == 1 and fm_l[1:].sum() == 0
    bad = W.refine(W.uniform_leaves(2, (1, 1), 2), np.arange(16) == 0)
    bad.axis = (np.linspace(0, 1, 9) ** 2, np.linspace(0, 1, 9))
    with pytest.raises(B.MGError):
        B.mg_mesh_nodes(bad)


def test_oracle_graded_stiffness_equals_tensor_assembly():
    """Two oracle paths on the graded cavity mesh agree: the generic Q1
    assembly over Q1Mesh cells (per-cell edge lengths) and the tensor-grid
    assembly of the Navier-Stokes module."""
    from oracle import mesh as M, ns
    lm = W.ns_cavity_mesh(4, 4, 8)
    fm = M.Q1Mesh(3, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor, axis=lm.axis)
    A = PB.build_system(fm, PB.Problem(PB.POISSON, dirichlet=(0,))).A_raw
    _, K, _ = ns.assemble(ns.Grid(lm.axis))
    assert close(A, K, 1e-13)


def test_pure_neumann_coarse_pseudo_inverse():
    """A Poisson problem with no prescribed dof: the coarse solve applies the
    pseudo-inverse, so for a compatible right-hand side (sum b = 0) it returns
    the solution of A_0 x = b orthogonal to the constants."""
    lm = W.ns_cavity_mesh(4, 4, 8)
    hh = HV.HostHierarchy(lm, B.make_problem(kind=B.MG_POISSON, dirichlet=(0,)))
    A0 = hh.matrix(0, HV.A).toarray()
    assert np.abs(A0 @ np.ones(A0.shape[0])).max() < 1e-13 * np.abs(A0).max()
    inv = hh.coarse_inverse()
    b = np.random.default_rng(9).standard_normal(A0.shape[0])
    b -= b.mean()
    x = inv @ b
    assert np.abs(A0 @ x - b).max() < 1e-10 * np.abs(b).max()
    assert abs(x.sum()) < 1e-10 * np.abs(x).sum()
