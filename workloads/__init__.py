"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no part of the solver's arithmetic.  It only produces the
*inputs* of a solve: leaf meshes (levels and integer anchors of the cells of a
1-irregular quadtree/octree over a box), coefficient sets, right-hand-side
functions and request streams.  Both the CPU oracle and the GPU library derive
nodes, hanging-node constraints, matrices and the multigrid hierarchy from the
leaf list on their own.

Mesh convention (the one the C-ABI's ``mg_mesh`` uses as well): the domain is
the box ``origin + [0, extent]``; level 0 is a ``macro[0] x macro[1] (x
macro[2])`` grid of cells; a cell of level ``l`` has integer anchor ``a`` with
``0 <= a[d] < macro[d] * 2**l`` and covers
``origin + extent/(macro*2**l) * [a, a+1]``.

Workloads (Sec. 5 of the paper motivates the problem classes; sizes follow
the benchmark configurations restated in the repository design notes):

* ``poisson64``      2D uniform 64x64 Q1 mesh on the unit square.
* ``td_adaptive``    2D mesh refined around 16 seeded points (1-irregular).
* ``elasticity3d``   3D uniform n^3 hexahedral mesh on the unit cube.
* ``oseen_channel``  2D channel [0,2.2]x[0,0.41] refined towards a circle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 20240508


@dataclass
class LeafMesh:
    """A leaf set of a 1-irregular quadtree (dim=2) or octree (dim=3)."""

    dim: int
    origin: tuple
    extent: tuple
    macro: tuple
    level: np.ndarray          # (n,) int32
    anchor: np.ndarray         # (n, dim) int32
    meta: dict = field(default_factory=dict)
    # graded tensor-product geometry: per axis the node coordinates of the
    # finest lattice ((macro[d] << max level) + 1 increasing values), or None
    axis: tuple | None = None

    @property
    def n_leaves(self) -> int:
        return int(self.level.shape[0])


# ---------------------------------------------------------------------------
# leaf-set helpers (pure integer bookkeeping)
# ---------------------------------------------------------------------------

_SHIFT = {2: (56, 28), 3: (58, 19)}


def _keys(dim, level, anchor):
    lshift, bits = _SHIFT[dim]
    k = level.astype(np.int64) << lshift
    for d in range(dim):
        k |= anchor[:, d].astype(np.int64) << (bits * (dim - 1 - d))
    return k


def uniform_leaves(dim, macro, level, origin=None, extent=None) -> LeafMesh:
    """All cells of one level of the macro grid."""
    macro = tuple(int(m) for m in macro)
    n = [m << level for m in macro]
    grids = np.meshgrid(*[np.arange(k, dtype=np.int32) for k in n], indexing="ij")
    anchor = np.stack([g.ravel() for g in grids], axis=1).astype(np.int32)
    lev = np.full(anchor.shape[0], level, dtype=np.int32)
    origin = tuple(origin) if origin is not None else (0.0,) * dim
    extent = tuple(extent) if extent is not None else (1.0,) * dim
    return LeafMesh(dim, origin, extent, macro, lev, anchor)


def family_mask(mesh: LeafMesh, mask: np.ndarray) -> np.ndarray:
    """Extend a leaf mask to every sibling of a marked leaf (same parent)."""
    dim = mesh.dim
    sel = mesh.level >= 1
    pk = np.full(mesh.n_leaves, -1, dtype=np.int64)
    pk[sel] = _keys(dim, mesh.level[sel] - 1, mesh.anchor[sel] >> 1)
    marked = np.unique(pk[mask & sel])
    return mask | (sel & np.isin(pk, marked))


def refine(mesh: LeafMesh, mask: np.ndarray, families: bool = False) -> LeafMesh:
    """Replace every marked leaf by its 2**dim children.  With families=True
    every sibling of a marked leaf is refined too, so a mesh whose leaves all
    come in complete sibling families (a patch mesh) stays one."""
    dim = mesh.dim
    if families:
        mask = family_mask(mesh, mask)
    keep_l, keep_a = mesh.level[~mask], mesh.anchor[~mask]
    par_l, par_a = mesh.level[mask], mesh.anchor[mask]
    kids_l, kids_a = [], []
    for c in range(1 << dim):
        off = np.array([(c >> d) & 1 for d in range(dim)], dtype=np.int32)
        kids_l.append(par_l + 1)
        kids_a.append(2 * par_a + off)
    level = np.concatenate([keep_l] + kids_l).astype(np.int32)
    anchor = np.concatenate([keep_a] + kids_a).astype(np.int32)
    return LeafMesh(dim, mesh.origin, mesh.extent, mesh.macro, level, anchor, dict(mesh.meta))


def balance_2to1(mesh: LeafMesh, families: bool = False) -> LeafMesh:
    """Refine until face-neighbouring leaves differ by at most one level
    (refining whole sibling families when families=True)."""
    dim = mesh.dim
    while True:
        lev, anc = mesh.level, mesh.anchor
        # every existing cell: leaves and all their ancestors
        exist = []
        for up in range(int(lev.max()) + 1):
            ok = lev >= up
            exist.append(_keys(dim, lev[ok] - up, anc[ok] >> up))
        exist = np.unique(np.concatenate(exist))
        leaf_keys = np.sort(_keys(dim, lev, anc))
        mark = np.zeros(lev.shape[0], dtype=bool)
        for d in range(dim):
            for s in (-1, 1):
                sel = lev >= 1
                nl = lev[sel]
                na = anc[sel].copy()
                na[:, d] += s
                size = np.array(mesh.macro, dtype=np.int64)[None, :] << nl[:, None].astype(np.int64)
                inside = np.all((na >= 0) & (na < size), axis=1)
                nl, na = nl[inside], na[inside]
                cl, ca = nl - 1, na >> 1
                missing = ~np.isin(_keys(dim, cl, ca), exist)
                cl, ca = cl[missing], ca[missing]
                # walk up from the missing cell to the leaf that contains it
                for up in range(1, int(lev.max()) + 1):
                    if cl.size == 0:
                        break
                    pl, pa = cl - up, ca >> up
                    valid = pl >= 0
                    k = _keys(dim, np.where(valid, pl, 0), np.where(valid[:, None], pa, 0))
                    hit = valid & np.isin(k, leaf_keys)
                    if hit.any():
                        idx = np.searchsorted(leaf_keys, k[hit])
                        mark_keys = leaf_keys[idx]
                        mark |= np.isin(_keys(dim, lev, anc), mark_keys)
                    cl, ca = cl[~hit], ca[~hit]
        if not mark.any():
            return mesh
        mesh = refine(mesh, mark, families)


def _cell_box(mesh: LeafMesh):
    ext = np.array(mesh.extent, dtype=np.float64)
    org = np.array(mesh.origin, dtype=np.float64)
    h = ext[None, :] / (np.array(mesh.macro, dtype=np.float64)[None, :] * (2.0 ** mesh.level[:, None]))
    lo = org[None, :] + mesh.anchor * h
    return lo, lo + h, h


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def poisson64(n: int = 64) -> LeafMesh:
    """Uniform n x n mesh on the unit square (n a power of two)."""
    lvl = int(round(math.log2(n)))
    assert 1 << lvl == n
    m = uniform_leaves(2, (1, 1), lvl)
    m.meta.update(workload=f"poisson2d_{n}x{n}")
    return m


def td_points(seed: int = MASTER_SEED, n_points: int = 16) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, size=(n_points, 2))


def td_adaptive(rounds: int = 8, gamma: float = 0.0, base_level: int = 5, r0: float = 0.05,
                seed: int = MASTER_SEED, n_points: int = 16) -> LeafMesh:
    """Adaptive 2D mesh around seeded points.

    Start from the uniform 2**base_level grid of the unit square; in round
    k = 1..rounds refine every leaf whose closed cell lies within distance
    r_k = r0 * 2**(-gamma*k) of one of the points, then restore 2:1 balance.
    gamma = 1 is the literal radius rule r_k = r0 * 2**-k.
    """
    pts = td_points(seed, n_points)
    m = uniform_leaves(2, (1, 1), base_level)
    for k in range(1, rounds + 1):
        r = r0 * 2.0 ** (-gamma * k)
        lo, hi, _ = _cell_box(m)
        mark = np.zeros(m.n_leaves, dtype=bool)
        for p in pts:
            dx = np.maximum(np.maximum(lo[:, 0] - p[0], 0.0), p[0] - hi[:, 0])
            dy = np.maximum(np.maximum(lo[:, 1] - p[1], 0.0), p[1] - hi[:, 1])
            mark |= dx * dx + dy * dy <= r * r
        m = balance_2to1(refine(m, mark))
    m.meta.update(workload=f"td_adaptive_r{rounds}_g{gamma:g}", points=pts, gamma=gamma)
    return m


def elasticity3d(n: int = 128) -> LeafMesh:
    lvl = int(round(math.log2(n)))
    assert 1 << lvl == n
    m = uniform_leaves(3, (1, 1, 1), lvl)
    m.meta.update(workload=f"elasticity3d_{n}^3")
    return m


def oseen_channel(uniform: int = 1, rounds: int = 0, band: float = 2.0) -> LeafMesh:
    """Channel [0,2.2]x[0,0.41] on a 22x4 macro grid, refined `uniform` (>= 1)
    times everywhere, then `rounds` times in the cells within band*h of the
    circle |x - (0.2, 0.2)| = 0.05 (h the cell's diameter), 2:1 balanced.
    Refinement is by whole sibling families, so every leaf belongs to a
    complete family (the patches of the local projection stabilisation)."""
    m = uniform_leaves(2, (22, 4), uniform, origin=(0.0, 0.0), extent=(2.2, 0.41))
    c, rad = np.array([0.2, 0.2]), 0.05
    for _ in range(rounds):
        lo, hi, h = _cell_box(m)
        near = np.clip(c[None, :], lo, hi)
        far = np.where(np.abs(lo - c) > np.abs(hi - c), lo, hi)
        dmin = np.linalg.norm(near - c, axis=1)
        dmax = np.linalg.norm(far - c, axis=1)
        diam = np.linalg.norm(h, axis=1)
        dist = np.where((dmin <= rad) & (dmax >= rad), 0.0, np.minimum(np.abs(dmin - rad), np.abs(dmax - rad)))
        m = balance_2to1(refine(m, dist <= band * diam, families=True), families=True)
    m.meta.update(workload=f"oseen_channel_u{uniform}_r{rounds}")
    return m


def oseen_beta(xy: np.ndarray, seed: int = MASTER_SEED, modes: int = 4) -> np.ndarray:
    """Divergence-free convection field beta = (d psi/dy, -d psi/dx) of the
    seeded stream function psi = sum a_mn sin(m pi x/2.2) sin(n pi y/0.41)
    / (m^2 + n^2), scaled so that max |beta| over the given points is 1."""
    a = stream_coeffs(seed, modes)
    x, y = xy[:, 0], xy[:, 1]
    bx = np.zeros_like(x)
    by = np.zeros_like(x)
    for m in range(1, modes + 1):
        for n in range(1, modes + 1):
            km, kn = m * math.pi / 2.2, n * math.pi / 0.41
            c = a[m - 1, n - 1] / (m * m + n * n)
            bx += c * np.sin(km * x) * kn * np.cos(kn * y)
            by -= c * km * np.cos(km * x) * np.sin(kn * y)
    beta = np.stack([bx, by], axis=1)
    return beta / np.max(np.linalg.norm(beta, axis=1))


def oseen_inflow(xy: np.ndarray, um: float = 0.3) -> np.ndarray:
    """Nodal Dirichlet data (u, v, p): parabolic inflow u = 4 um y (H - y)/H^2
    at x = 0 (H = 0.41), zero elsewhere (walls); p entries are unused."""
    g = np.zeros((xy.shape[0], 3))
    H = 0.41
    at_in = xy[:, 0] == 0.0
    g[at_in, 0] = 4.0 * um * xy[at_in, 1] * (H - xy[at_in, 1]) / (H * H)
    return g


# ---------------------------------------------------------------------------
# right-hand sides and coefficient streams (the data the paper's tests use)
# ---------------------------------------------------------------------------

def f_poisson(xy: np.ndarray) -> np.ndarray:
    """f = 2 pi^2 sin(pi x) sin(pi y): -Laplace of u = sin(pi x) sin(pi y)."""
    return 2.0 * math.pi ** 2 * np.sin(math.pi * xy[:, 0]) * np.sin(math.pi * xy[:, 1])


def u_manufactured(xy: np.ndarray) -> np.ndarray:
    return np.sin(math.pi * xy[:, 0]) * np.sin(math.pi * xy[:, 1])


def f_transport(xy: np.ndarray, eps: float, beta) -> np.ndarray:
    """f = -eps Laplace u + beta . grad u for u = sin(pi x) sin(pi y)."""
    x, y = xy[:, 0], xy[:, 1]
    pi = math.pi
    return (eps * 2.0 * pi ** 2 * np.sin(pi * x) * np.sin(pi * y)
            + beta[0] * pi * np.cos(pi * x) * np.sin(pi * y)
            + beta[1] * pi * np.sin(pi * x) * np.cos(pi * y))


def random_nodal(n: int, ncomp: int = 1, seed: int = MASTER_SEED, stream: int = 0) -> np.ndarray:
    """Seeded N(0,1) vectors for operator-level parity tests."""
    rng = np.random.Generator(np.random.PCG64([seed, stream]))
    return rng.standard_normal((n, ncomp)) if ncomp > 1 else rng.standard_normal(n)


def stream_coeffs(seed: int = MASTER_SEED, modes: int = 4) -> np.ndarray:
    """a_mn ~ N(0,1), m,n = 1..modes, for the seeded stream function."""
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    return rng.standard_normal((modes, modes))


# ---------------------------------------------------------------------------
# time-dependent transport-diffusion (the paper's Sec. 5.1 example)
# ---------------------------------------------------------------------------
TD_LAMBDA = 0.01            # diffusion
TD_B = (0.0, -1.0)          # transport direction
TD_DT = 0.02                # backward-Euler step
TD_STEPS = 100              # T = 2


def td_m(t: float, z: np.ndarray) -> np.ndarray:
    return 0.5 + 0.25 * math.cos(0.5 * math.pi * t) - z


def td_theta(t: float, xy: np.ndarray) -> np.ndarray:
    """theta_ex(t, x, y) = exp(-(m(t,x)^2 + m(t,y)^2) / 4)."""
    mx, my = td_m(t, xy[:, 0]), td_m(t, xy[:, 1])
    return np.exp(-0.25 * (mx * mx + my * my))


def td_source(t: float, xy: np.ndarray, lam: float = TD_LAMBDA, b=TD_B) -> np.ndarray:
    """f = d_t theta - lam Laplace theta + b.grad theta for theta_ex: with
    Q = m_x^2 + m_y^2, d_z m = -1 and d_t m = -(pi/8) sin(pi t / 2),
    d_t theta = -theta (m_x + m_y) d_t m / 2, grad theta = theta (m_x, m_y) / 2,
    Laplace theta = theta (Q / 4 - 1)."""
    mx, my = td_m(t, xy[:, 0]), td_m(t, xy[:, 1])
    th = np.exp(-0.25 * (mx * mx + my * my))
    mdot = -0.125 * math.pi * math.sin(0.5 * math.pi * t)
    q = mx * mx + my * my
    return th * (-0.5 * (mx + my) * mdot - lam * (0.25 * q - 1.0) + 0.5 * (b[0] * mx + b[1] * my))


def td_uniform(n: int) -> LeafMesh:
    """Uniform n x n mesh of the unit square for the time-dependent problem
    (n = 2^7 .. 2^10 in the paper's study: 16,641 .. 1,050,625 DoFs)."""
    m = uniform_leaves(2, (1, 1), int(round(math.log2(n))))
    m.meta.update(workload=f"td_timedep_{n}x{n}")
    return m


# ---------------------------------------------------------------------------
# time-dependent linear elasticity on adaptive hex meshes (the paper's Sec. 5.2)
# ---------------------------------------------------------------------------
EL_LAMBDA = 8.0e4           # Lame parameters
EL_MU = 2.0e4
EL_F = (0.0, -1.0, 0.0)     # body force
EL_DT = 0.025               # backward-Euler step
EL_STEPS = 100              # T = 2.5


def elasticity_adaptive(kind: str, levels: int) -> LeafMesh:
    """Sec. 5.2 meshes: the uniform 8^3 grid of the unit cube (mesh level 1),
    then levels-1 rounds that refine every finest cell lying within 2^-r of
    the face x = 0 ("face"), the edge x = y = 0 ("edge") or the vertex 0
    ("vertex").  Node counts match Table "table:ndofs"."""
    m = uniform_leaves(3, (1, 1, 1), 3)
    ax = {"face": [0], "edge": [0, 1], "vertex": [0, 1, 2]}[kind]
    for r in range(1, levels):
        _, hi, _ = _cell_box(m)
        mark = (m.level == m.level.max()) & np.all(hi[:, ax] <= 2.0 ** -r + 1e-12, axis=1)
        m = refine(m, mark)
    m.meta.update(workload=f"elasticity_{kind}_l{levels}")
    return m


def ns_cavity_mesh(nx: int = 32, ny: int = 32, nz: int = 64, graded: bool = True) -> LeafMesh:
    """Pressure mesh of the 3D driven cavity (Sec. 5.3): nx x ny x nz cells of
    the box (0, 1) x (0, 1) x (0, 2), as a uniform leaf set of level L (the
    largest with nx, ny, nz divisible by 2^L) on the macro grid (n >> L), with
    the cosine-graded node coordinates x_i = (1 - cos(i pi / nx)) / 2 (y
    alike) and z_k = 1 - cos(k pi / nz) when graded, equidistant otherwise."""
    L = 0
    while all(n % (2 << L) == 0 for n in (nx, ny, nz)):
        L += 1
    m = uniform_leaves(3, (nx >> L, ny >> L, nz >> L), L, origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 2.0))
    if graded:
        ax = (0.5 * (1.0 - np.cos(np.arange(nx + 1) * np.pi / nx)),
              0.5 * (1.0 - np.cos(np.arange(ny + 1) * np.pi / ny)),
              1.0 - np.cos(np.arange(nz + 1) * np.pi / nz))
    else:
        ax = (np.linspace(0.0, 1.0, nx + 1), np.linspace(0.0, 1.0, ny + 1), np.linspace(0.0, 2.0, nz + 1))
    m.axis = ax
    m.meta.update(workload=f"ns_cavity_{nx}x{ny}x{nz}" + ("_graded" if graded else ""))
    return m
