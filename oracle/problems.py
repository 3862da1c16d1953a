"""Oracle: the four PDE systems and their condensed linear systems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Poisson (-Laplace u = f) and transport-diffusion (-eps Laplace u + beta.grad u
= f) are the scalar problems; the paper's transport-diffusion example is
Sec. 5.1 (there with a time derivative and without stabilisation).  Linear
elasticity, -div sigma(u) = f with sigma = lambda tr(eps(u)) I + 2 mu eps(u),
is Sec. 5.2 (here the static operator).  Right-hand side: b = H^T (M I_h f)
with the consistent mass matrix M and the nodal interpolant I_h f, plus the
SUPG load term for transport-diffusion; Dirichlet data are homogeneous.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fem

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

    @property
    def nc(self):
        return 3 if self.kind in (ELASTICITY, OSEEN) else 1

    def masks(self):
        m = tuple(self.dirichlet)
        return m if len(m) == self.nc else m * self.nc


def element(prob: Problem, dim: int):
    """Function h -> element matrix of the problem's bilinear form."""
    if prob.kind == POISSON:
        return lambda h: fem.scalar_element(dim, h, "stiffness")
    if prob.kind == TRANSPORT:
        beta = np.asarray(prob.beta[:dim], dtype=np.float64)

        def el(h):
            d = fem.supg_delta(h, prob.eps, beta, prob.supg_delta0)
            return (prob.eps * fem.scalar_element(dim, h, "stiffness")
                    + fem.scalar_element(dim, h, "convection", beta)
                    + d * fem.scalar_element(dim, h, "streamline", beta))
        return el
    if prob.kind == ELASTICITY:
        assert dim == 3
        return lambda h: fem.elasticity_element(h, prob.mu, prob.lam)
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

    def rhs(self, f_nodal):
        """b_c for nodal source values f (n_nodes x nc or n_nodes)."""
        f = np.asarray(f_nodal, dtype=np.float64).reshape(self.mesh.n_nodes, -1)
        b_all = (self.F @ f).ravel()
        return fem.condense_rhs(b_all, self.H, self.hang, self.dirichlet)


def build_system(mesh, prob: Problem, with_load=True) -> System:
    nc = prob.nc
    A_raw = fem.assemble(mesh, element(prob, mesh.dim), nc)
    H = fem.expand(mesh.H(), nc)
    hang, dirichlet = fem.constrained_dofs(mesh, prob.masks(), nc)
    A = fem.condense(A_raw, H, hang, dirichlet)
    F = fem.assemble(mesh, load_element(prob, mesh.dim), 1) if with_load else None
    return System(mesh, prob, A_raw, H, hang, dirichlet, A, F)


def fill_constrained(system: System, x):
    """x_all = H x: hanging values from their parents (Sec. 2.2)."""
    return system.H @ x
