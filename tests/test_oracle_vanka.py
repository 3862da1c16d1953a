"""Pins of the oracle's cell-patch Vanka smoother (the paper's Sec. 6 names
Vanka smoothers as the next step for saddle-point problems): closed forms on
the uniform Q1 Laplacian, exactness on a one-cell mesh, and its use as a
multigrid smoother on the Oseen channel (direct-solve equality, fewer GMRES
iterations than the point-block smoother)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import workloads as W
from oracle import krylov, mg
from oracle import mesh as M
from oracle import problems as PB


def q1mesh(lm):
    return M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)


def test_vanka_interior_row_closed_form_on_the_laplacian():
    """Uniform 2D Q1 Laplacian: the four vertices of a cell are mutual
    neighbours, so A_T = 3 I - J/3 (J all ones) and A_T^{-1} = (I + J/5)/3.
    An interior node lies in 4 cells (W = 1/4): S_ii = 4/4 (1/3)(6/5) = 2/5,
    an edge neighbour shares 2 cells: 2/4 (1/15) = 1/30, a diagonal one 1:
    1/60."""
    m = q1mesh(W.uniform_leaves(2, (1, 1), 3))
    S_sys = PB.build_system(m, PB.Problem(PB.POISSON, dirichlet=(0,)), with_load=False)
    S = mg.vanka_matrix(m, S_sys.A_raw, 1)
    i = int(np.nonzero((m.X[:, 0] == 4) & (m.X[:, 1] == 4))[0][0])
    row = S.getrow(i)
    assert row.nnz == 9
    for j, v in zip(row.indices, row.data):
        dist = int(np.abs(m.X[j] - m.X[i]).sum())
        assert v == pytest.approx({0: 0.4, 1: 1.0 / 30, 2: 1.0 / 60}[dist], rel=1e-13)


def test_vanka_on_one_cell_is_the_inverse():
    """One cell: a single local problem with m_i = 1, so S = A^{-1} and one
    sweep with omega = 1 solves the system (Oseen-type 3-component operator:
    mass, diffusion and a pressure coupling)."""
    m = q1mesh(W.uniform_leaves(2, (1, 1), 0))
    assert m.n_nodes == 4
    prob = PB.Problem(PB.TRANSPORT, eps=0.3, beta=(1.0, -0.5), mass=7.0, dirichlet=(0,))
    A = PB.build_system(m, prob, with_load=False).A_raw
    S = mg.vanka_matrix(m, A, 1)
    assert np.abs(S.toarray() @ A.toarray() - np.eye(4)).max() <= 1e-13


def _oseen(rounds):
    lm = W.oseen_channel(1, rounds)
    fm = q1mesh(lm)
    beta = W.oseen_beta(fm.coords)
    prob = PB.Problem(PB.OSEEN, conv=beta, dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01)
    S = PB.build_system(fm, prob, beta=beta)
    b = S.rhs(np.zeros(fm.n_nodes * 3), W.oseen_inflow(fm.coords).ravel())
    return lm, prob, S, b


def test_vanka_mg_gmres_equals_direct_solve_with_fewer_iterations():
    lm, prob, S, b = _oseen(3)
    xd = spl.spsolve(S.A.tocsc(), b)
    its = {}
    for sm in ("jacobi", "vanka"):
        Hh = mg.Hierarchy(lm, prob, smoother=sm)
        x, info = krylov.gmres(Hh.fine.A, b, Hh.precondition, rtol=1e-12, restart=30, maxit=500)
        assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
        its[sm] = info["iters"]
        if sm == "vanka":
            assert all(lv.vanka for lv in Hh.levels[1:]) and not Hh.levels[0].vanka
    assert its["vanka"] * 2 <= its["jacobi"], its


def test_vanka_rows_threshold_selects_levels():
    lm, prob, S, b = _oseen(3)
    Hh = mg.Hierarchy(lm, prob, smoother="vanka", vanka_rows=3000)
    for lv in Hh.levels[1:]:
        assert lv.vanka == (lv.A.shape[0] >= 3000)
        assert lv.omega == 1.0 if lv.vanka else lv.omega < 1.0
