"""Explicit Navier-Stokes pressure correction: the 3D driven cavity of Sec. 5.3.

Test infrastructure (CPU, FP64, plain numpy / scipy): only tests, smoke and
the bench's CPU legs use it.  It restates the fully discrete procedure of
Sec. 5.3 (Algorithm "The fully discrete solution procedure for the
Navier-Stokes equations") directly:

* spaces: pressure Q_h / S_h = Q1 on the mesh Omega_h, velocity V_h = Q1 on its
  equidistant refinement Omega_{h/2} (the Q1-iso-Q2/Q1 pair); the pressure
  mesh is the graded box of Sec. 5.3 (cosine grading of the node coordinates);
* lumped masses m_i = sum_j (phi_j, phi_i) (Eq. "mass_lumping");
* the convective term through the nodal interpolant of u (x) u and the
  matrices C_d[i, j] = (phi_j, d_d phi_i), d = x, y, z (Eqs.
  "conv_mass_lumping", "tp", "multC"): component c of node i receives
  sum_b sum_j C_b[i, j] u_{j,b} u_{j,c};
* Step 1 (explicit momentum): for every free velocity node
    m_i (u^m - u^{m-1})_i / k = - nu (K u^{m-1})_i + N(u^{m-1})_i
                                + (C_c P (p^{m-1} + q^{m-1}))_i
  with K the Q1 stiffness on Omega_{h/2}, P the nodal interpolation from
  Omega_h to Omega_{h/2}, Dirichlet data on the boundary (lid: u = (0, 1, 0)
  on x = 1);
* Step 2 (pressure increment): K_p q^m = -(1/k) d^m, d^m = P^T sum_c C_c^T u^m_c
  = ((div u^m, psi_j))_j, K_p the Q1 stiffness on Omega_h (pure Neumann, a
  compatible singular system); the solution of mean zero, sum_j m^p_j q_j = 0
  (the space Q of Sec. 5.3, with the lumped mass as the inner product);
* Step 3 (pressure update): p^m = p^{m-1} + q^m - nu d^m / m^p.

Readings of the paper (where it is garbled or silent; the same list is in the
design notes): the sign of the viscous term in the form A of Sec. 5.3 is taken
as + nu (grad u, grad chi) (the stated one would be anti-diffusive); the three
matrices of Eq. "multC" are C_x, C_y, C_z (the text repeats C_x); the z
coordinates are z_k = 1 - cos(k pi / N_z), i.e. 1 + sin((2k - N_z) pi / (2 N_z)),
which spans the domain's (0, 2) (the printed 1 + sin((k - N_z) pi / (2 N_z))
spans (0, 1) only); x and y are ordered increasingly, x_i = (1 - cos(i pi / N_x)) / 2.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import fem


def graded_axes(nx, ny, nz):
    """Node coordinates of the pressure mesh along x, y, z (Sec. 5.3)."""
    x = 0.5 * (1.0 - np.cos(np.arange(nx + 1) * np.pi / nx))
    y = 0.5 * (1.0 - np.cos(np.arange(ny + 1) * np.pi / ny))
    z = 1.0 - np.cos(np.arange(nz + 1) * np.pi / nz)
    return x, y, z


def refine_axis(a):
    """Coordinates of the equidistant refinement: every cell halved."""
    out = np.empty(2 * a.size - 1)
    out[0::2] = a
    out[1::2] = 0.5 * (a[:-1] + a[1:])
    return out


class Grid:
    """Tensor-product Q1 mesh of a box: nodes (i, j, k) numbered x fastest."""

    def __init__(self, axes):
        self.axes = [np.asarray(a, dtype=np.float64) for a in axes]
        self.n = tuple(a.size for a in self.axes)             # nodes per axis
        self.n_nodes = int(np.prod(self.n))
        idx = np.indices(self.n[::-1]).reshape(3, -1)[::-1].T   # (n_nodes, 3): i fastest
        self.X = idx
        self.coords = np.stack([self.axes[d][idx[:, d]] for d in range(3)], axis=1)

    def node(self, i, j, k):
        return i + self.n[0] * (j + self.n[1] * k)

    def cells(self):
        """(n_cells, 8) corner nodes (x fastest) and (n_cells, 3) edge lengths."""
        ci = np.indices((self.n[2] - 1, self.n[1] - 1, self.n[0] - 1)).reshape(3, -1)[::-1].T
        corners = []
        for c in range(8):
            o = np.array([(c >> d) & 1 for d in range(3)])
            X = ci + o
            corners.append(self.node(X[:, 0], X[:, 1], X[:, 2]))
        h = np.stack([self.axes[d][ci[:, d] + 1] - self.axes[d][ci[:, d]] for d in range(3)], axis=1)
        return np.stack(corners, axis=1), h

    def boundary(self):
        on = np.zeros(self.n_nodes, dtype=bool)
        for d in range(3):
            on |= (self.X[:, d] == 0) | (self.X[:, d] == self.n[d] - 1)
        return on


def element_forms(h):
    """Q1 element matrices of a box with edge lengths h, by tensor Gauss
    quadrature (exact: every integrand has degree <= 2 per axis):
    mass M[a, b] = (phi_b, phi_a), stiffness K[a, b] = (grad phi_b, grad phi_a),
    C_d[a, b] = (phi_b, d_d phi_a)."""
    pts, wts = fem.quadrature(3)
    h = np.asarray(h, dtype=np.float64)
    vol = float(np.prod(h))
    M = np.zeros((8, 8))
    K = np.zeros((8, 8))
    C = np.zeros((3, 8, 8))
    for xi, w in zip(pts, wts):
        val, grad = fem.q1_basis(3, xi)
        g = grad / h[None, :]                  # physical gradients
        M += w * vol * np.outer(val, val)
        K += w * vol * g @ g.T
        for d in range(3):
            C[d] += w * vol * np.outer(g[:, d], val)   # row a: d_d phi_a, column b: phi_b
    return M, K, C


def assemble(grid):
    """Global lumped mass (vector), stiffness K and C_x, C_y, C_z (CSR)."""
    cn, h = grid.cells()
    _, group = np.unique(h, axis=0, return_inverse=True)
    group = np.asarray(group).ravel()
    n = grid.n_nodes
    rows = np.repeat(cn, 8, axis=1).ravel()
    cols = np.tile(cn, (1, 8)).ravel()
    mv, kv = np.empty((cn.shape[0], 64)), np.empty((cn.shape[0], 64))
    cv = np.empty((3, cn.shape[0], 64))
    for g in np.unique(group):
        sel = group == g
        Me, Ke, Ce = element_forms(h[np.nonzero(sel)[0][0]])
        mv[sel] = Me.ravel()
        kv[sel] = Ke.ravel()
        for d in range(3):
            cv[d, sel] = Ce[d].ravel()
    mk = lambda v: sp.coo_matrix((v.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    m = np.asarray(mk(mv).sum(axis=1)).ravel()
    return m, mk(kv), [mk(cv[d]) for d in range(3)]


def interpolation(coarse, fine):
    """Nodal interpolation from the Q1 space of `coarse` to that of its
    equidistant refinement `fine` (exact: Q1(Omega_h) is a subspace)."""
    rows, cols, vals = [], [], []
    I = [fine.X[:, d] for d in range(3)]
    parts = []
    for d in range(3):
        even = I[d] % 2 == 0
        lo = I[d] // 2
        parts.append([(lo, np.where(even, 1.0, 0.5)), (np.where(even, lo, lo + 1), np.where(even, 0.0, 0.5))])
    for a, b, c in itertools.product(range(2), repeat=3):
        (ix, wx), (iy, wy), (iz, wz) = parts[0][a], parts[1][b], parts[2][c]
        w = wx * wy * wz
        keep = w != 0.0
        rows.append(np.nonzero(keep)[0])
        cols.append(coarse.node(ix[keep], iy[keep], iz[keep]))
        vals.append(w[keep])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.n_nodes, coarse.n_nodes)).tocsr()


@dataclass
class Cavity:
    """The driven-cavity problem: meshes, operators, boundary data."""
    pm: Grid                  # pressure mesh Omega_h
    vm: Grid                  # velocity mesh Omega_{h/2}
    mv: np.ndarray            # lumped velocity masses
    K: sp.csr_matrix          # velocity stiffness
    C: list                   # C_x, C_y, C_z on the velocity mesh
    P: sp.csr_matrix          # interpolation pressure -> velocity mesh
    mp: np.ndarray            # lumped pressure masses
    Kp: sp.csr_matrix         # pressure stiffness (pure Neumann)
    fixed: np.ndarray         # velocity nodes with Dirichlet data (the whole boundary)
    g: np.ndarray             # (n_v, 3) Dirichlet values
    nu: float
    dt: float
    pin: int = 0              # node held at 0 in the direct solve of Step 2 (before the mean shift)


def cavity(nx, ny, nz, re=1e3, dt=1e-4, lid=1.0, graded=True):
    """Sec. 5.3's driven cavity on an nx x ny x nz pressure mesh of the box
    (0, 1) x (0, 1) x (0, 2); the lid x = 1 moves with (0, lid, 0)."""
    if graded:
        ax = graded_axes(nx, ny, nz)
    else:
        ax = (np.linspace(0, 1, nx + 1), np.linspace(0, 1, ny + 1), np.linspace(0, 2, nz + 1))
    pm = Grid(ax)
    vm = Grid([refine_axis(a) for a in ax])
    mv, K, C = assemble(vm)
    mp, Kp, _ = assemble(pm)
    P = interpolation(pm, vm)
    fixed = vm.boundary()
    g = np.zeros((vm.n_nodes, 3))
    g[vm.X[:, 0] == vm.n[0] - 1, 1] = lid
    return Cavity(pm, vm, mv, K, C, P, mp, Kp, fixed, g, 1.0 / re, dt)


def convection(C, u):
    """N(u)_{i,c} = sum_b sum_j C_b[i, j] u_{j,b} u_{j,c} (Eqs. "tp", "multC")."""
    out = np.zeros_like(u)
    for b in range(3):
        out += C[b] @ (u[:, [b]] * u)
    return out


def divergence(S, u):
    """d_j = (div u, psi_j) for the pressure basis psi_j = sum_i P[i, j] phi_i:
    d = P^T sum_c C_c^T u_c."""
    dv = sum(S.C[c].T @ u[:, c] for c in range(3))
    return S.P.T @ dv


def momentum(S, u, p, q):
    """Step 1: the explicit lumped-mass momentum update."""
    pt = S.P @ (p + q)
    r = -S.nu * (S.K @ u) + convection(S.C, u)
    for c in range(3):
        r[:, c] += S.C[c] @ pt
    un = u + S.dt * r / S.mv[:, None]
    un[S.fixed] = S.g[S.fixed]
    return un


def pressure_increment(S, d):
    """Step 2: K_p q = -d / k, the solution of mean zero.  One solution of the
    compatible pure Neumann system by a sparse direct solve with the node
    S.pin held at 0, then the constant that makes sum_j m^p_j q_j = 0."""
    n = S.pm.n_nodes
    keep = np.ones(n, dtype=bool)
    keep[S.pin] = False
    A = S.Kp[keep][:, keep].tocsc()
    q = np.zeros(n)
    q[keep] = spl.spsolve(A, -d[keep] / S.dt)
    return q - (S.mp @ q) / S.mp.sum()


def step(S, u, p, q):
    """One time step of the procedure: (u^m, p^m, q^m) from (u^{m-1}, p^{m-1}, q^{m-1})."""
    un = momentum(S, u, p, q)
    d = divergence(S, un)
    qn = pressure_increment(S, d)
    pn = p + qn - S.nu * d / S.mp
    return un, pn, qn, d


def run(S, steps, u=None, p=None, q=None):
    u = np.zeros((S.vm.n_nodes, 3)) if u is None else u.copy()
    p = np.zeros(S.pm.n_nodes) if p is None else p.copy()
    q = np.zeros(S.pm.n_nodes) if q is None else q.copy()
    for _ in range(steps):
        u, p, q, _ = step(S, u, p, q)
    return u, p, q
