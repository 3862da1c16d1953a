"""Pins of the oracle's explicit Navier-Stokes pressure correction (Sec. 5.3)
against facts that do not come from the oracle itself: integration by
parts, partitions of unity, exact interpolation of trilinear functions, the
volume of the box, the symmetry of the graded coordinates, and the
compatibility of the pure Neumann pressure problem.  Each pin is chosen so
that a plausible slip (a transposed C, a swapped product index, a sign, a
wrong grading) breaks it."""
import numpy as np
import pytest

from oracle import ns


@pytest.fixture(scope="module")
def S():
    return ns.cavity(4, 4, 8)


def test_graded_axes():
    x, y, z = ns.graded_axes(8, 8, 16)
    assert x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-15 and abs(z[-1] - 2.0) < 1e-15 and z[0] == 0.0
    assert np.all(np.diff(x) > 0) and np.all(np.diff(z) > 0)
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15) and np.allclose(z + z[::-1], 2.0, atol=1e-15)
    # cosine grading: the cells next to the walls are the smallest, the
    # middle ones the largest; the first one is (1 - cos(pi / n)) / 2
    hx = np.diff(x)
    assert np.argmin(hx) in (0, hx.size - 1) and abs(hx[0] - 0.5 * (1 - np.cos(np.pi / 8))) < 1e-16
    r = ns.refine_axis(x)
    assert np.array_equal(r[0::2], x) and np.allclose(r[1::2], 0.5 * (x[:-1] + x[1:]))


def test_masses_sum_to_the_volume(S):
    assert abs(S.mv.sum() - 2.0) < 1e-13 and abs(S.mp.sum() - 2.0) < 1e-13
    assert np.all(S.mv > 0) and np.all(S.mp > 0)


def test_stiffness_kills_linear_functions(S):
    inner = ~S.fixed
    for d in range(3):
        lin = S.vm.coords[:, d]
        assert np.abs((S.K @ lin)[inner]).max() < 1e-13
    assert np.abs(S.K @ np.ones(S.vm.n_nodes)).max() < 1e-13


def test_c_integration_by_parts(S):
    """(x_d, d_d phi_i) = -(1, phi_i) = -m_i at interior nodes, and
    (x_e, d_d phi_i) = 0 for e != d: pins the sign and which index of C is
    differentiated."""
    inner = ~S.fixed
    for d in range(3):
        for e in range(3):
            r = S.C[d] @ S.vm.coords[:, e]
            want = -S.mv if d == e else np.zeros_like(S.mv)
            assert np.abs((r - want)[inner]).max() < 1e-13, (d, e)
        assert np.abs((S.C[d] @ np.ones(S.vm.n_nodes))[inner]).max() < 1e-14
        # partition of unity in the differentiated index: columns sum to 0
        assert np.abs(np.asarray(S.C[d].sum(axis=0)).ravel()).max() < 1e-14


def test_convection_of_a_shear_field(S):
    """u = (1, x, 0): u.grad u = (0, 1, 0), so the interpolated convective
    term equals -(u.grad u, phi_i) = (0, -m_i, 0) at interior nodes (every
    product u_b u_c is trilinear or a function of x alone, so the nodal
    interpolation is exact where it matters)."""
    x = S.vm.coords
    u = np.stack([np.ones(len(x)), x[:, 0], np.zeros(len(x))], axis=1)
    N = ns.convection(S.C, u)
    inner = ~S.fixed
    want = np.stack([0 * S.mv, -S.mv, 0 * S.mv], axis=1)
    assert np.abs((N - want)[inner]).max() < 1e-13
    # swapping the roles of b and c would give (x-part) -(u_c d_b u_b) != 0
    u2 = np.stack([x[:, 1], np.ones(len(x)), np.zeros(len(x))], axis=1)   # u.grad u = (1, 0, 0)
    N2 = ns.convection(S.C, u2)
    assert np.abs((N2 - np.stack([-S.mv, 0 * S.mv, 0 * S.mv], axis=1))[inner]).max() < 1e-13


def test_interpolation_is_exact_for_trilinear_functions(S):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(8)

    def f(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * y * z + a[6] * x * z + a[7] * x * y * z

    assert np.abs(S.P @ f(S.pm.coords) - f(S.vm.coords)).max() < 1e-13
    assert np.allclose(np.asarray(S.P.sum(axis=1)).ravel(), 1.0)


def test_divergence_tested_with_the_pressure_basis(S):
    """(div u, psi_j) for u = (x, 2y, -z): div u = 2, so d = 2 m^p at every
    pressure node (no integration by parts involved)."""
    X = S.vm.coords
    u = np.stack([X[:, 0], 2 * X[:, 1], -X[:, 2]], axis=1)
    assert np.abs(ns.divergence(S, u) - 2.0 * S.mp).max() < 1e-13


def test_pressure_increment_solves_the_singular_system(S):
    """The increment satisfies every equation of the pure Neumann system (the
    row of the node held during the direct solve included) when the data are
    compatible (u.n = 0 on the boundary: here any field with the cavity's
    Dirichlet values), and has mean zero."""
    rng = np.random.default_rng(4)
    u = rng.standard_normal((S.vm.n_nodes, 3))
    u[S.fixed] = S.g[S.fixed]
    d = ns.divergence(S, u)
    assert abs(d.sum()) < 1e-12 * np.abs(d).sum()
    q = ns.pressure_increment(S, d)
    assert abs(S.mp @ q) < 1e-12 * (S.mp @ np.abs(q))
    assert np.abs(S.Kp @ q + d / S.dt).max() < 1e-9 * np.abs(d / S.dt).max()


def test_step_invariants(S):
    """At rest with the lid still nothing moves; a constant added to the
    pressure changes no velocity (C_c P 1 = 0 at interior nodes)."""
    import copy
    S0 = copy.copy(S)
    S0.g = np.zeros_like(S.g)
    u, p, q = ns.run(S0, 2)
    assert np.abs(u).max() == 0.0 and np.abs(p).max() == 0.0 and np.abs(q).max() == 0.0
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((S.vm.n_nodes, 3)) * 0.1
    u0[S.fixed] = S.g[S.fixed]
    p0 = rng.standard_normal(S.pm.n_nodes)
    a = ns.momentum(S, u0, p0, 0 * p0)
    b = ns.momentum(S, u0, p0 + 3.0, 0 * p0)
    assert np.abs(a - b).max() < 1e-12


def test_lid_drives_the_flow(S):
    """After a few steps from rest the interior velocity, set in motion by the
    lid alone, is nonzero and stays below the lid speed."""
    u, p, q = ns.run(S, 5)
    assert 0 < np.abs(u[~S.fixed]).max() < 1.0
    assert np.isfinite(p).all() and np.isfinite(q).all()
