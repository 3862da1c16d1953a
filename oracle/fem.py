"""Oracle: Q1 element matrices, global assembly, condensation, Dirichlet rows.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1 of the paper: V_h = continuous functions that are Q^r on every cell
(here r = 1 on axis-parallel boxes); systems use equal-order components and a
node-major ("block") layout x_{i,c}, each matrix entry A_ij an n_c x n_c
block.  Sec. 2.2: assembled residuals and right-hand sides are multiplied by
H^T, the solution by H.

Quadrature: tensor 2-point Gauss, exact for every bilinear form below on
axis-parallel boxes (the integrands are polynomials of degree <= 3 per axis;
degree 3 only for the Oseen convection term with its cell-wise bilinear beta).

Bilinear forms (row = test function, column = trial function):
  Poisson            (grad u, grad v)
  transport-diff.    eps (grad u, grad v) + (beta.grad u, v)
                     + sum_T delta_T (beta.grad u, beta.grad v)_T      (SUPG)
  elasticity (3D)    2 mu (eps(u), eps(v)) + lambda (div u, div v)     (Sec. 5.2)
                     written with the Voigt strain-displacement matrix B.
  Oseen (2D, u,v,p)  see ``oseen_patch_matrices`` (assembled per patch).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

GAUSS_1D = (np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)]), np.array([0.5, 0.5]))


def quadrature(dim):
    """Tensor Gauss points on the unit cell and their weights."""
    p1, w1 = GAUSS_1D
    pts = np.array(list(itertools.product(p1, repeat=dim)))[:, ::-1]   # x fastest
    wts = np.array([np.prod(w) for w in itertools.product(w1, repeat=dim)])
    return pts, wts


def q1_basis(dim, xi):
    """Values (2^d,) and reference gradients (2^d, d) of the Q1 basis at xi;
    local vertex c has offsets ((c>>0)&1, (c>>1)&1, ...)."""
    n = 1 << dim
    val = np.ones(n)
    grad = np.ones((n, dim))
    for c in range(n):
        for d in range(dim):
            b = (c >> d) & 1
            f = xi[d] if b else 1.0 - xi[d]
            df = 1.0 if b else -1.0
            val[c] *= f
            for e in range(dim):
                grad[c, e] *= df if e == d else f
    return val, grad


def scalar_element(dim, h, kind, coef=None):
    """Element matrix of a scalar form on a box with edge lengths h."""
    h = np.asarray(h, dtype=np.float64)
    vol = float(np.prod(h))
    n = 1 << dim
    K = np.zeros((n, n))
    pts, wts = quadrature(dim)
    for xi, w in zip(pts, wts):
        phi, dref = q1_basis(dim, xi)
        g = dref / h[None, :]                       # physical gradients
        if kind == "stiffness":
            K += w * vol * (g @ g.T)
        elif kind == "mass":
            K += w * vol * np.outer(phi, phi)
        elif kind == "convection":                  # (beta.grad u, v)
            bg = g @ np.asarray(coef, dtype=np.float64)
            K += w * vol * np.outer(phi, bg)
        elif kind == "streamline":                  # (beta.grad u, beta.grad v)
            bg = g @ np.asarray(coef, dtype=np.float64)
            K += w * vol * np.outer(bg, bg)
        else:
            raise ValueError(kind)
    return K


def elasticity_element(h, mu, lam):
    """3D Q1 elasticity element (24x24, node-major: row 3a+i).
    a(u,v) = int eps(v)^T D eps(u), Voigt engineering strains
    (xx, yy, zz, 2xy, 2yz, 2xz), D the isotropic material matrix."""
    h = np.asarray(h, dtype=np.float64)
    vol = float(np.prod(h))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    K = np.zeros((24, 24))
    pts, wts = quadrature(3)
    for xi, w in zip(pts, wts):
        _, dref = q1_basis(3, xi)
        g = dref / h[None, :]
        B = np.zeros((6, 24))
        for a in range(8):
            gx, gy, gz = g[a]
            B[0, 3 * a + 0] = gx
            B[1, 3 * a + 1] = gy
            B[2, 3 * a + 2] = gz
            B[3, 3 * a + 0] = gy; B[3, 3 * a + 1] = gx
            B[4, 3 * a + 1] = gz; B[4, 3 * a + 2] = gy
            B[5, 3 * a + 0] = gz; B[5, 3 * a + 2] = gx
        K += w * vol * (B.T @ D @ B)
    return K


def supg_delta(h, eps, beta, delta0=0.5):
    """delta_T = delta0 h_T^2 / (6 eps + |beta| h_T), h_T the cell diameter."""
    hT = float(np.linalg.norm(h))
    return delta0 * hT * hT / (6.0 * eps + float(np.linalg.norm(beta)) * hT)


def lps_interpolation(dim=2):
    """Pi (3^d x 3^d): values at the 3^d patch lattice points of the coarse Q1
    interpolant i_2h built from the patch's 2^d corner values (corners
    weight 1, edge midpoints 1/2 each, centre 1/4 each)."""
    n = 3 ** dim
    Pi = np.zeros((n, n))
    for i in range(n):
        loc = [(i // 3 ** d) % 3 for d in range(dim)]
        for c in range(1 << dim):
            w = 1.0
            j = 0
            for d in range(dim):
                b = (c >> d) & 1
                w *= (loc[d] / 2.0) if b else (1.0 - loc[d] / 2.0)
                j += (2 * b) * 3 ** d
            Pi[i, j] += w
    return Pi


def oseen_patch_matrices(h, beta9, nu, dt, alpha0):
    """Patch matrices (n_p, 27, 27) of the 2D Oseen system with local
    projection stabilisation, node-major (row 3a+i, i = u, v, p):

      (1/dt)(u, v) + nu (grad u, grad v) + ((beta_h . grad) u, v)
      - (p, div v) + (div u, q)
      + alpha_P (grad kappa p, grad kappa q)_P
      + alpha_P (beta_P . grad kappa u, beta_P . grad kappa v)_P   (u, v comps)

    over a patch P of four child cells with edge lengths h.  beta_h is the
    cell-wise Q1 interpolant of the nodal field beta9 (n_p, 9, 2); beta_P its
    value at the patch centre; kappa = id - i_2h (fluctuation with respect to
    the patch's coarse Q1 interpolant); alpha_P = alpha0 h_P^2 / (nu +
    |beta_P| h_P) with h_P the patch diameter.  Two-point Gauss rules are
    exact for every integrand (degree <= 3 per axis)."""
    h = np.asarray(h, dtype=np.float64)
    beta9 = np.asarray(beta9, dtype=np.float64)
    n_p = beta9.shape[0]
    vol = float(np.prod(h))
    pts, wts = quadrature(2)
    K = np.zeros((n_p, 27, 27))
    G9 = np.zeros((9, 9))                       # patch stiffness (grad, grad)
    Gij = np.zeros((2, 2, 9, 9))                # int d_i phi_A d_j phi_B over the patch
    for cy in range(2):
        for cx in range(2):
            loc = np.array([(cx + (c & 1)) + 3 * (cy + (c >> 1)) for c in range(4)])
            bc = beta9[:, loc, :]                                  # (n_p, 4, 2)
            for xi, w in zip(pts, wts):
                phi, dref = q1_basis(2, xi)
                g = dref / h[None, :]
                wv = w * vol
                bq = np.einsum("c,pcd->pd", phi, bc)               # beta_h at the point
                conv = wv * np.einsum("a,pb->pab", phi, bq @ g.T)  # (beta.grad phi_B) phi_A
                mass = wv * np.outer(phi, phi) / dt
                diff = wv * nu * (g @ g.T)
                for i in range(2):
                    K[:, 3 * loc[:, None] + i, 3 * loc[None, :] + i] += mass + diff + conv
                    # -(p, div v): row velocity comp i (test phi_A), column p (phi_B)
                    K[:, 3 * loc[:, None] + i, 3 * loc[None, :] + 2] -= wv * np.outer(g[:, i], phi)
                    # (div u, q): row p (test phi_A), column velocity comp i
                    K[:, 3 * loc[:, None] + 2, 3 * loc[None, :] + i] += wv * np.outer(phi, g[:, i])
                G9[np.ix_(loc, loc)] += wv * (g @ g.T)
                for i in range(2):
                    for j in range(2):
                        Gij[i, j][np.ix_(loc, loc)] += wv * np.outer(g[:, i], g[:, j])
    kap = np.eye(9) - lps_interpolation(2)
    bP = beta9[:, 4, :]                                            # patch centre
    hP = 2.0 * float(np.linalg.norm(h))
    alpha = alpha0 * hP * hP / (nu + np.linalg.norm(bP, axis=1) * hP)
    Sp = kap.T @ G9 @ kap
    Cb = np.einsum("pi,pj,ijab->pab", bP, bP, Gij)
    Sc = np.einsum("ka,pkl,lb->pab", kap, Cb, kap)
    K[:, 2::3, 2::3] += alpha[:, None, None] * Sp[None, :, :]
    for i in range(2):
        K[:, i::3, i::3] += alpha[:, None, None] * Sc
    return K


def assemble_patches(mesh, patch_nodes, Kp, nc):
    """Sum patch matrices Kp (n_p, (3^d nc)^2) over the patches' nodes."""
    m = patch_nodes.shape[1] * nc
    dofs = (patch_nodes[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(-1, m)
    rows = np.repeat(dofs, m, axis=1).ravel()
    cols = np.tile(dofs, (1, m)).ravel()
    n = mesh.n_nodes * nc
    return sp.coo_matrix((Kp.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()


def assemble(mesh, element_of_size, nc=1):
    """Sum element matrices into a global (n_nodes*nc)^2 CSR matrix.
    element_of_size(h) returns the (2^d nc)^2 element matrix for a cell with
    edge lengths h (all our forms depend on the cell only through h)."""
    hs = mesh.cell_size()
    # cells with the same edge lengths share one element matrix (one group
    # per level on a uniform mesh, one per distinct box on a graded one)
    _, group = np.unique(hs, axis=0, return_inverse=True)
    group = np.asarray(group).ravel()
    rows, cols, vals = [], [], []
    nv = 1 << mesh.dim
    for g in np.unique(group):
        sel = np.nonzero(group == g)[0]
        Ke = element_of_size(hs[sel[0]])
        dofs = (mesh.cell_nodes[sel][:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(sel.size, nv * nc)
        rows.append(np.repeat(dofs, nv * nc, axis=1).ravel())
        cols.append(np.tile(dofs, (1, nv * nc)).ravel())
        vals.append(np.broadcast_to(Ke.ravel()[None, :], (sel.size, Ke.size)).ravel())
    n = mesh.n_nodes * nc
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


def expand(M, nc):
    """Scalar node operator -> node-major block operator (M kron I_nc)."""
    return sp.kron(M, sp.identity(nc), format="csr") if nc > 1 else M.tocsr()


def constrained_dofs(mesh, dirichlet_masks, nc=1):
    """Boolean masks over the dofs: hanging (all components) and Dirichlet
    (component c on the faces in dirichlet_masks[c])."""
    hang = np.repeat(mesh.hanging, nc)
    dir_ = np.zeros(mesh.n_nodes * nc, dtype=bool)
    for c in range(nc):
        dir_[c::nc] = mesh.boundary_nodes(dirichlet_masks[c])
    dir_ &= ~hang
    return hang, dir_


def condense(A, H, hang, dirichlet):
    """A_c = H^T A H (Sec. 2.2) with identity rows/columns for hanging and
    Dirichlet dofs (symmetric elimination)."""
    Ac = (H.T @ A @ H).tocsr()
    fixed = hang | dirichlet
    keep = sp.diags((~fixed).astype(np.float64))
    Ac = (keep @ Ac @ keep + sp.diags(fixed.astype(np.float64))).tocsr()
    Ac.eliminate_zeros()
    return Ac


def condense_rhs(b_all, H, hang, dirichlet, g=None, A_raw=None):
    """b_c = H^T b (Sec. 2.2), zero on hanging rows, g on Dirichlet rows.
    With Dirichlet data g (a dof vector; only its Dirichlet entries are used)
    the free rows are lifted: b_c -= (H^T A H)[:, D] g_D (symmetric
    elimination of the prescribed values)."""
    b = H.T @ b_all
    if g is not None:
        gd = np.where(dirichlet, np.asarray(g, dtype=np.float64), 0.0)
        b = b - H.T @ (A_raw @ (H @ gd))
    b[hang] = 0.0
    b[dirichlet] = 0.0 if g is None else np.asarray(g, dtype=np.float64)[dirichlet]
    return b
