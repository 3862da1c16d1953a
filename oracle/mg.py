"""Oracle: multigrid hierarchy, transfers, smoother, coarse solve, V-cycle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Transfers (Sec. 4.1.4, Eq. "prolongation"): the prolongation is the natural
  embedding of the coarse Q1 space into the fine one, u_fine(x_i) =
  sum_j chi_ij u_coarse_j, written as one sparse matrix P_l; the restriction
  is its transpose R = P^T.  With hanging nodes the coarse vertex values are
  first completed by H (Sec. 2.2), and rows/columns of constrained dofs are
  zero: P_eff = Z_f E H_c Z_c.
* Smoother (Sec. 4.1.4): x <- x + omega S (b - A x), S = D^{-1} (Jacobi) or
  the inverse of the n_c x n_c nodal diagonal blocks (block Jacobi), or the
  additive cell-patch Vanka matrix (``vanka_matrix``; Sec. 6 names Vanka
  smoothers as the next step) on the levels with >= vanka_rows unknowns.
* Coarse problem: a direct solve A_0^{-1} b_0 (the coarse-mesh problem of the
  multigrid cycle, Sec. 2.2), here LU with partial pivoting in FP64.
* Level operators: rediscretisation of the same form on every level of the
  global hierarchy (Sec. 2.2: "an approximation of the entire problem can be
  created on each grid level").
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import mesh as M
from . import problems as PB


def embedding(fine: M.Q1Mesh, coarse: M.Q1Mesh):
    """E (n_fine x n_coarse): value of the coarse Q1 function (given on all
    coarse vertices) at each fine node, by Q1 interpolation in the coarse
    leaf that contains the node."""
    dim = fine.dim
    Lf = fine.L
    X = fine.X                                         # fine lattice coords
    n = fine.n_nodes
    found = np.zeros(n, dtype=bool)
    rows, cols, vals = [], [], []
    ckeys = M._cell_keys(dim, coarse.level, coarse.anchor)
    order = np.argsort(ckeys)
    ckeys_sorted = ckeys[order]
    off = coarse.corners_offsets()
    for l in np.unique(coarse.level):
        s = 1 << (Lf - int(l))
        ncell = fine.macro << int(l)
        a = np.minimum(X >> (Lf - int(l)), ncell[None, :] - 1)
        k = M._cell_keys(dim, np.full(n, l), a)
        pos = np.minimum(np.searchsorted(ckeys_sorted, k), ckeys_sorted.size - 1)
        hit = (ckeys_sorted[pos] == k) & ~found
        idx = np.nonzero(hit)[0]
        if idx.size == 0:
            continue
        found[idx] = True
        t = (X[idx] - a[idx] * s) / float(s)           # local coordinates in [0,1]
        if fine.axis is not None:
            # graded boxes: the physical position inside the coarse cell (the
            # coarse Q1 function is linear along each axis of its box)
            sh = fine.axis_level - Lf
            t = np.stack([(fine.axis[d][X[idx, d] << sh] - fine.axis[d][(a[idx, d] * s) << sh])
                          / (fine.axis[d][((a[idx, d] + 1) * s) << sh] - fine.axis[d][(a[idx, d] * s) << sh])
                          for d in range(dim)], axis=1)
        for c in range(1 << dim):
            w = np.ones(idx.size)
            for d in range(dim):
                w *= t[:, d] if off[c, d] else 1.0 - t[:, d]
            corner = (a[idx] + off[c][None, :]) << (coarse.L - int(l))
            cn = coarse.lookup(coarse.key(corner))
            assert np.all(cn >= 0)
            nz = w != 0.0
            rows.append(idx[nz]); cols.append(cn[nz]); vals.append(w[nz])
    assert found.all(), "fine node outside the coarse mesh"
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, coarse.n_nodes))


class Level:
    def __init__(self, leaf_level, leaf_anchor, leafmesh, prob, lattice_level=None, fine_mesh=None):
        axis = getattr(leafmesh, "axis", None)
        self.mesh = M.Q1Mesh(leafmesh.dim, leafmesh.origin, leafmesh.extent, leafmesh.macro,
                             leaf_level, leaf_anchor, lattice_level, axis=axis,
                             axis_level=None if axis is None else int(np.max(leafmesh.level)))
        beta = None
        if prob.kind == PB.OSEEN:      # nodal convection field, injected from the finest mesh
            beta = PB.inject(fine_mesh, prob.conv, self.mesh) if fine_mesh is not None else prob.conv
        self.sys = PB.build_system(self.mesh, prob, with_load=False, beta=beta)
        self.A = self.sys.A
        self.nc = prob.nc
        self.P = None          # prolongation from the next coarser level
        self.R = None

    def smoother_matrix(self):
        """S of the smoothing step: D^-1 (nc=1) or block-diagonal inverse."""
        nc = self.nc
        if nc == 1:
            return sp.diags(1.0 / self.A.diagonal())
        n = self.A.shape[0] // nc
        blocks = []
        Ad = self.A.tocsr()
        for i in range(n):
            B = Ad[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc].toarray()
            blocks.append(np.linalg.inv(B))
        return sp.bsr_matrix((np.array(blocks), np.arange(n), np.arange(n + 1)),
                             shape=self.A.shape).tocsr()


def vanka_matrix(mesh, A, nc):
    """The additive cell-patch Vanka smoother as a matrix:
    S = W sum_T P_T A_T^{-1} P_T^T, with A_T = A restricted to the 2^d nc
    unknowns of the vertices of cell T (every component; constrained rows and
    columns of A are identity rows, so fixed unknowns stay decoupled) and
    W = diag(1 / m_i), m_i the number of cells that contain node i.  The
    paper names Vanka smoothers as the next step for saddle-point problems
    (Sec. 6); one cell's vertices form one local problem."""
    A = A.tocsr()
    cn = np.asarray(mesh.cell_nodes)                  # (n_cells, 2^d), x fastest
    ncell, nv = cn.shape
    k = nv * nc
    dofs = (cn[:, :, None] * nc + np.arange(nc)[None, None, :]).reshape(ncell, k)
    AT = np.zeros((ncell, k, k))
    idx = np.arange(ncell)
    for a in range(k):
        rows = A[dofs[:, a]]
        for b in range(k):
            AT[:, a, b] = np.asarray(rows[idx, dofs[:, b]]).ravel()
    inv = np.linalg.inv(AT)
    m = np.bincount(cn.ravel(), minlength=mesh.n_nodes).astype(np.float64)
    R = np.repeat(dofs, k, axis=1).ravel()
    C = np.tile(dofs, (1, k)).ravel()
    S = sp.csr_matrix((inv.ravel(), (R, C)), shape=A.shape)
    return (sp.diags(np.repeat(1.0 / m, nc)) @ S).tocsr()


def lambda_max_power(S, A, fixed, iters=20):
    """Largest eigenvalue magnitude of S A by `iters` power iterations
    w = S A v, lambda = |w| / |v|, v = w / |w|, from the start vector
    v_i = frac(i * 2654435761 / 2^32) - 1/2 on free dofs, 0 on fixed ones."""
    n = A.shape[0]
    v = ((np.arange(n, dtype=np.uint64) * np.uint64(2654435761)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5
    v[fixed] = 0.0
    if not np.any(v):
        return 1.0          # no free dof: the level is never smoothed, any damping does
    lam = 0.0
    for _ in range(iters):
        w = S @ (A @ v)
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return lam


class Hierarchy:
    """Levels 0 (coarsest) .. L (finest) of the global coarsening.

    omega: smoother damping on every level; None: 0.8 for scalar problems and
    1.2 / lambda_max(S_l A_l) per level for point-block smoothers (20 power
    iterations; lambda_max(D^-1 A) = 1.5 for the Q1 Laplacian, where this
    rule gives 0.8 as well)."""

    def __init__(self, leafmesh, prob, min_level=None, max_levels=0, omega=None, nu1=2, nu2=2,
                 smoother="jacobi", vanka_rows=0, vanka_omega=1.0):
        patch = prob.kind == PB.OSEEN   # LPS patches: keep every level a patch mesh
        if min_level is None:
            min_level = max(M.default_min_level(leafmesh.macro), 1 if patch else 0)
        sets = M.hierarchy(leafmesh.dim, leafmesh.macro, leafmesh.level, leafmesh.anchor,
                           min_level, max_levels, patch)[::-1]
        fine_mesh = None
        if patch:
            fine_mesh = M.Q1Mesh(leafmesh.dim, leafmesh.origin, leafmesh.extent, leafmesh.macro,
                                 sets[-1][0], sets[-1][1])
        self.levels = [Level(l, a, leafmesh, prob, fine_mesh=fine_mesh) for (l, a) in sets]
        self.prob = prob
        self.nu1, self.nu2 = nu1, nu2
        nc = prob.nc
        for lc, lf in zip(self.levels[:-1], self.levels[1:]):
            E = mesh_E = embedding(lf.mesh, lc.mesh)
            Hc = lc.mesh.H()
            P = fem_expand(mesh_E @ Hc, nc)
            zf = sp.diags((~lf.sys.fixed).astype(np.float64))
            zc = sp.diags((~lc.sys.fixed).astype(np.float64))
            lf.P = (zf @ P @ zc).tocsr()
            lf.P.eliminate_zeros()
            lf.R = lf.P.T.tocsr()
            del E
        for i, lv in enumerate(self.levels):
            lv.vanka = smoother == "vanka" and i > 0 and lv.A.shape[0] >= vanka_rows
            if lv.vanka:          # cell-patch Vanka, damping vanka_omega
                lv.S = vanka_matrix(lv.mesh, lv.A, nc)
                lv.omega = float(vanka_omega)
                continue
            lv.S = lv.smoother_matrix()
            if omega is not None:
                lv.omega = float(omega)
            elif nc == 1 and lv.mesh.axis is None:
                lv.omega = 0.8
            # graded boxes: anisotropic cells push lambda_max(D^-1 A) of the
            # scalar Q1 operator well above its value on cubes, where 0.8
            # diverges; the damping then comes from the estimate too
            else:
                lv.omega = 1.2 / lambda_max_power(lv.S, lv.A, lv.sys.fixed)
        A0 = self.levels[0].A.toarray()
        self.coarse_lu = sla.lu_factor(A0)

    @property
    def fine(self):
        return self.levels[-1]

    @property
    def omega(self):
        """Damping of the finest level."""
        return self.levels[-1].omega

    def smooth(self, l, x, b, sweeps):
        lv = self.levels[l]
        for _ in range(sweeps):
            x = x + lv.omega * (lv.S @ (b - lv.A @ x))
        return x

    def gmg(self, l, x, b):
        """The recursive multigrid cycle GMG(l, x, b) of Sec. 2.2."""
        if l == 0:
            return sla.lu_solve(self.coarse_lu, b)                 # coarse mesh problem
        lv = self.levels[l]
        x = self.smooth(l, x, b, self.nu1)                         # pre-smooth
        d = lv.R @ (b - lv.A @ x)                                  # restrict residual
        y = self.gmg(l - 1, np.zeros_like(d), d)                   # coarse correction
        x = x + lv.P @ y                                           # prolongate update
        return self.smooth(l, x, b, self.nu2)                      # post-smooth

    def precondition(self, r):
        """One V-cycle with zero initial guess: z = M^-1 r."""
        return self.gmg(len(self.levels) - 1, np.zeros_like(r), r)


def fem_expand(Msc, nc):
    return sp.kron(Msc, sp.identity(nc), format="csr") if nc > 1 else Msc.tocsr()
