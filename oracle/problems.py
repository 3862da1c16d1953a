"""Oracle: the four PDE systems and their condensed linear systems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Poisson (-Laplace u = f) and transport-diffusion (-eps Laplace u + beta.grad u
= f) are the scalar problems; the paper's transport-diffusion example is
Sec. 5.1 (there with a time derivative and without stabilisation).  Linear
elasticity, -div sigma(u) = f with sigma = lambda tr(eps(u)) I + 2 mu eps(u),
is Sec. 5.2 (here the static operator).  The Oseen system (one linearised
backward-Euler step of the incompressible Navier-Stokes equations, equal-order
Q1 velocity and pressure with local projection stabilisation, the form in
``fem.oseen_patch_matrices``) is the saddle-point problem of Sec. 5.3's flow
example.  Right-hand side: b = H^T (M I_h f) with the consistent mass matrix M
and the nodal interpolant I_h f, plus the SUPG load term for
transport-diffusion; Dirichlet data g are eliminated symmetrically (lifted
into the free rows).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fem
from . import mesh as M

POISSON, TRANSPORT, ELASTICITY, OSEEN = "poisson", "transport", "elasticity", "oseen"


@dataclass
class Problem:
    kind: str = POISSON
    eps: float = 1.0
    beta: tuple = (0.0, 0.0, 0.0)
    mu: float = 1.0
    lam: float = 1.0
    supg_delta0: float = 0.5
    dirichlet: tuple = (0xFF,)          # face mask per component
    nu: float = 1e-3                    # Oseen: viscosity
    dt: float = 0.01                    # Oseen: time step of the mass term
    lps_alpha0: float = 0.5             # Oseen: LPS parameter
    conv: object = None                 # Oseen: nodal beta (n_nodes, 2) on the finest mesh
    mass: float = 0.0                   # Poisson/transport: coefficient s of s (u, v)
    pin_origin: bool = False            # also prescribe the node at the origin corner

    @property
    def nc(self):
        return 3 if self.kind in (ELASTICITY, OSEEN) else 1

    def masks(self):
        m = tuple(self.dirichlet)
        return m if len(m) == self.nc else m * self.nc


def element(prob: Problem, dim: int):
    """Function h -> element matrix of the problem's bilinear form.

    A mass coefficient s = prob.mass > 0 adds s (u, v): with s = 1/dt this is
    the matrix of one backward-Euler step of the time-dependent problem
    (Sec. 5.1, Eq. "condif_a").  With SUPG the stabilisation tests the whole
    residual, so the mass part also enters it: delta_T s (u, beta.grad v)_T."""
    s = float(prob.mass)
    if prob.kind == POISSON:
        if s == 0.0:
            return lambda h: fem.scalar_element(dim, h, "stiffness")
        return lambda h: fem.scalar_element(dim, h, "stiffness") + s * fem.scalar_element(dim, h, "mass")
    if prob.kind == TRANSPORT:
        beta = np.asarray(prob.beta[:dim], dtype=np.float64)

        def el(h):
            d = fem.supg_delta(h, prob.eps, beta, prob.supg_delta0)
            K = (prob.eps * fem.scalar_element(dim, h, "stiffness")
                 + fem.scalar_element(dim, h, "convection", beta)
                 + d * fem.scalar_element(dim, h, "streamline", beta))
            if s != 0.0:
                K = K + s * (fem.scalar_element(dim, h, "mass")
                             + d * fem.scalar_element(dim, h, "convection", beta).T)
            return K
        return el
    if prob.kind == ELASTICITY:
        assert dim == 3
        if s == 0.0:
            return lambda h: fem.elasticity_element(h, prob.mu, prob.lam)
        # s (u, v) for vector fields: the scalar mass matrix on every component
        return lambda h: (fem.elasticity_element(h, prob.mu, prob.lam)
                          + s * np.kron(fem.scalar_element(3, h, "mass"), np.eye(3)))
    raise ValueError(prob.kind)


def load_element(prob: Problem, dim: int):
    """Function h -> element matrix F with b_T = F f_T for nodal f:
    F_ij = (phi_j, phi_i) (+ delta_T (phi_j, beta.grad phi_i) for SUPG)."""
    if prob.kind == TRANSPORT:
        beta = np.asarray(prob.beta[:dim], dtype=np.float64)

        def el(h):
            d = fem.supg_delta(h, prob.eps, beta, prob.supg_delta0)
            return fem.scalar_element(dim, h, "mass") + d * fem.scalar_element(dim, h, "convection", beta).T
        return el
    return lambda h: fem.scalar_element(dim, h, "mass")


@dataclass
class System:
    mesh: object
    prob: Problem
    A_raw: sp.csr_matrix        # assembled on all nodes, before condensation
    H: sp.csr_matrix            # H_h expanded to dofs
    hang: np.ndarray
    dirichlet: np.ndarray
    A: sp.csr_matrix            # condensed system matrix
    F: sp.csr_matrix = field(default=None)   # scalar load matrix (nodes x nodes)

    @property
    def fixed(self):
        return self.hang | self.dirichlet

    def rhs(self, f_nodal, g_nodal=None):
        """b_c for nodal source values f (n_nodes x nc or n_nodes) and
        optional nodal Dirichlet data g (same shape; used on Dirichlet dofs)."""
        f = np.asarray(f_nodal, dtype=np.float64).reshape(self.mesh.n_nodes, -1)
        b_all = (self.F @ f).ravel()
        g = None if g_nodal is None else np.asarray(g_nodal, dtype=np.float64).ravel()
        return fem.condense_rhs(b_all, self.H, self.hang, self.dirichlet, g, self.A_raw)


def inject(fine_mesh, values, mesh):
    """Values of a nodal field of fine_mesh at the nodes of a coarser mesh of
    the same hierarchy (every coarse node is a fine node)."""
    X = np.asarray(mesh.X, dtype=np.int64) << (fine_mesh.L - mesh.L)
    idx = fine_mesh.lookup(fine_mesh.key(X))
    assert np.all(idx >= 0)
    return np.asarray(values)[idx]


def oseen_matrix(mesh, prob: Problem, beta):
    """Oseen + LPS operator assembled patch by patch (before condensation)."""
    nodes, lev = M.patches(mesh)
    beta = np.asarray(beta, dtype=np.float64)
    A = None
    for l in np.unique(lev):
        sel = np.nonzero(lev == l)[0]
        assert mesh.axis is None, "graded meshes are not available for Oseen"
        h = mesh.extent / (mesh.macro * 2.0 ** int(l))
        Kp = fem.oseen_patch_matrices(h, beta[nodes[sel]], prob.nu, prob.dt, prob.lps_alpha0)
        Al = fem.assemble_patches(mesh, nodes[sel], Kp, 3)
        A = Al if A is None else A + Al
    return A.tocsr()


def build_system(mesh, prob: Problem, with_load=True, beta=None) -> System:
    """beta: nodal convection field of this mesh (Oseen only)."""
    nc = prob.nc
    if prob.kind == OSEEN:
        A_raw = oseen_matrix(mesh, prob, beta)
    else:
        A_raw = fem.assemble(mesh, element(prob, mesh.dim), nc)
    H = fem.expand(mesh.H(), nc)
    hang, dirichlet = fem.constrained_dofs(mesh, prob.masks(), nc)
    if prob.pin_origin:               # one solution of a pure Neumann problem: fix the origin node
        origin = np.nonzero(np.all(mesh.X == 0, axis=1))[0]
        for c in range(nc):
            dirichlet[origin * nc + c] = True
    A = fem.condense(A_raw, H, hang, dirichlet)
    F = fem.assemble(mesh, load_element(prob, mesh.dim), 1) if with_load else None
    return System(mesh, prob, A_raw, H, hang, dirichlet, A, F)


def fill_constrained(system: System, x):
    """x_all = H x: hanging values from their parents (Sec. 2.2)."""
    return system.H @ x
