"""Oracle: Q1 node set, hanging-node matrix and global coarsening.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2 of the paper: a refined cell is replaced by 2^d children, the level
jump between neighbours is at most one, nodes that are vertices of the fine
side of such a face but not of the coarse side are *hanging* and are replaced
by interpolation of their neighbours through the matrix H_h (identity on
regular nodes, interpolation weights on hanging rows).  The multigrid
hierarchy is built by *global coarsening*: starting from the finest mesh, each
step takes back every family of 2^d sibling leaves, and every level covers
the whole domain.

Node numbering (shared *convention* with the library's external order, not
code): integer coordinates on the lattice of the finest level L, sorted
lexicographically with x fastest, then y, then z.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Q1Mesh:
    """Nodes, cell->node map, hanging constraints of a 1-irregular leaf set."""

    def __init__(self, dim, origin, extent, macro, level, anchor, lattice_level=None, axis=None, axis_level=None):
        """axis (optional, graded tensor-product geometry): per dimension the
        node coordinates of the lattice of level axis_level (default: this
        mesh's own lattice); a node at lattice index i of this mesh sits at
        axis[d][i * 2^(axis_level - L)] and every cell is an axis-aligned box
        with its own edge lengths."""
        self.dim = dim
        self.origin = np.asarray(origin, dtype=np.float64)
        self.extent = np.asarray(extent, dtype=np.float64)
        self.axis = None if axis is None else [np.asarray(a, dtype=np.float64) for a in axis[:dim]]
        self.macro = np.asarray(macro, dtype=np.int64)
        self.level = np.asarray(level, dtype=np.int64)
        self.anchor = np.asarray(anchor, dtype=np.int64)
        # lattice: the finest level present, unless a finer one is requested
        self.L = int(self.level.max()) if lattice_level is None else int(lattice_level)
        self.n_lat = self.macro << self.L          # cells per axis on the lattice
        if self.axis is not None:
            # hanging-node weights of 1/2 put a hanging node at its edge's
            # middle, which graded coordinates do not: uniform leaf sets only
            assert np.all(self.level == self.level[0]), "graded meshes must be uniform"
            self.axis_level = self.L if axis_level is None else int(axis_level)
            assert self.axis_level >= self.L
            for d in range(dim):
                assert self.axis[d].size == (int(self.macro[d]) << self.axis_level) + 1
                assert np.all(np.diff(self.axis[d]) > 0)
            self.origin = np.array([a[0] for a in self.axis])
            self.extent = np.array([a[-1] - a[0] for a in self.axis])
        self.stride = np.ones(dim, dtype=np.int64)
        for d in range(1, dim):
            self.stride[d] = self.stride[d - 1] * (self.n_lat[d - 1] + 1)
        self._build_nodes()
        self._build_hanging()

    # -- lattice keys -------------------------------------------------------
    def key(self, X):
        return (np.asarray(X, dtype=np.int64) * self.stride).sum(axis=-1)

    def corners_offsets(self):
        return np.array([[(c >> d) & 1 for d in range(self.dim)] for c in range(1 << self.dim)],
                        dtype=np.int64)

    def _build_nodes(self):
        s = (1 << (self.L - self.level))[:, None]               # cell size on the lattice
        off = self.corners_offsets()                           # (2^d, d), x fastest
        X = (self.anchor[:, None, :] + off[None, :, :]) * s[:, None, :]
        keys = self.key(X)                                     # (n_cells, 2^d)
        self.node_keys, inv = np.unique(keys.ravel(), return_inverse=True)
        self.cell_nodes = inv.reshape(keys.shape)
        self.n_nodes = self.node_keys.size
        Xn = np.empty((self.n_nodes, self.dim), dtype=np.int64)
        rem = self.node_keys.copy()
        for d in reversed(range(self.dim)):
            Xn[:, d] = rem // self.stride[d]
            rem = rem - Xn[:, d] * self.stride[d]
        self.X = Xn                                            # integer lattice coordinates
        self.h_lat = self.extent / self.n_lat                  # lattice spacing per axis (uniform)
        if self.axis is None:
            self.coords = self.origin + Xn * self.h_lat
        else:
            sh = self.axis_level - self.L
            self.coords = np.stack([self.axis[d][Xn[:, d] << sh] for d in range(self.dim)], axis=1)

    def lookup(self, keys):
        """Node index of each lattice key, -1 where the key is not a node."""
        keys = np.asarray(keys)
        idx = np.searchsorted(self.node_keys, keys)
        idx = np.minimum(idx, self.n_nodes - 1)
        return np.where(self.node_keys[idx] == keys, idx, -1)

    def _build_hanging(self):
        """Edge midpoints (and in 3D face centres) of a cell that are nodes of
        the mesh are hanging; their value is the mean of the edge's 2 (face's
        4) vertices.  Chains are resolved so that H maps onto regular nodes."""
        dim = self.dim
        s = (1 << (self.L - self.level))
        cand = []   # (hanging key, parent key list)
        fine = s >= 2
        A = self.anchor[fine] * s[fine, None]
        sf = s[fine]
        half = sf // 2
        off = self.corners_offsets()
        # sub-entities of the unit cell: points with coordinates in {0, 1/2, 1}
        # with exactly one (edges) or two (faces, 3D) coordinates equal to 1/2
        for pattern in np.ndindex(*(3,) * dim):
            pattern = np.array(pattern)
            nhalf = int((pattern == 1).sum())
            if nhalf == 0 or nhalf == dim:
                continue
            P = A + (pattern[None, :] * half[:, None])
            # the vertices of the sub-entity: replace each 1/2 coordinate by 0 or 1
            free = np.nonzero(pattern == 1)[0]
            parents = []
            for c in range(1 << nhalf):
                q = pattern.copy()
                for k, d in enumerate(free):
                    q[d] = 2 * ((c >> k) & 1)
                parents.append(A + q[None, :] * half[:, None])
            cand.append((self.key(P), [self.key(Q) for Q in parents]))
        rows = {}
        kinds = {}
        for hk, pks in cand:
            hn = self.lookup(hk)
            hit = hn >= 0
            for j in np.nonzero(hit)[0]:
                h = int(hn[j])
                ps = tuple(int(self.lookup(pk[j])) for pk in pks)
                w = 1.0 / len(ps)
                if h not in rows:
                    rows[h] = {p: w for p in ps}
                    kinds[h] = len(ps)
        self.hanging = np.zeros(self.n_nodes, dtype=bool)
        self.hanging[list(rows.keys())] = True
        # resolve chains: substitute hanging parents until only regular nodes remain
        changed = True
        while changed:
            changed = False
            for h, dep in rows.items():
                if any(self.hanging[p] for p in dep):
                    new = {}
                    for p, w in dep.items():
                        if self.hanging[p]:
                            for q, v in rows[p].items():
                                new[q] = new.get(q, 0.0) + w * v
                        else:
                            new[p] = new.get(p, 0.0) + w
                    rows[h] = new
                    changed = True
        self.hanging_rows = rows
        # number of vertices each hanging node interpolates before chains are
        # resolved: 2 for edge midpoints, 4 for face centres (3D)
        self.hanging_parents = np.zeros(self.n_nodes, dtype=np.int64)
        for h, k in kinds.items():
            self.hanging_parents[h] = k

    # -- H_h (Sec. 2.2): identity on regular nodes, weights on hanging rows ---
    def H(self):
        r, c, v = [], [], []
        for i in range(self.n_nodes):
            if not self.hanging[i]:
                r.append(i); c.append(i); v.append(1.0)
        for h, dep in self.hanging_rows.items():
            for p, w in dep.items():
                r.append(h); c.append(p); v.append(w)
        return sp.csr_matrix((v, (r, c)), shape=(self.n_nodes, self.n_nodes))

    def boundary_nodes(self, face_mask):
        """Nodes on the domain faces selected by bits of face_mask:
        bit 2d = face x_d = min, bit 2d+1 = face x_d = max."""
        on = np.zeros(self.n_nodes, dtype=bool)
        for d in range(self.dim):
            if face_mask >> (2 * d) & 1:
                on |= self.X[:, d] == 0
            if face_mask >> (2 * d + 1) & 1:
                on |= self.X[:, d] == self.n_lat[d]
        return on

    def cell_size(self):
        """Edge lengths of every cell, (n_cells, dim)."""
        if self.axis is None:
            return self.extent[None, :] / (self.macro[None, :] * (2.0 ** self.level[:, None]))
        s = (1 << (self.axis_level - self.level))[:, None]     # cell size on the axis lattice
        lo = self.anchor * s
        return np.stack([self.axis[d][lo[:, d] + s[:, 0]] - self.axis[d][lo[:, d]] for d in range(self.dim)],
                        axis=1)


# ---------------------------------------------------------------------------
# global coarsening (Sec. 2.2): take back every complete sibling family, keep
# the 2:1 rule, every level spans the whole domain
# ---------------------------------------------------------------------------

def _cell_keys(dim, level, anchor):
    k = level.astype(np.int64) << 58
    for d in range(dim):
        k |= anchor[:, d].astype(np.int64) << (19 * (dim - 1 - d))
    return k


def _violations(dim, macro, level, anchor):
    """Leaves whose face neighbour is two or more levels finer: returns the
    keys of the too-coarse leaves."""
    lev, anc = level, anchor
    exist = np.unique(np.concatenate(
        [_cell_keys(dim, lev[lev >= u] - u, anc[lev >= u] >> u) for u in range(int(lev.max()) + 1)]))
    leaves = np.sort(_cell_keys(dim, lev, anc))
    bad = []
    for d in range(dim):
        for sgn in (-1, 1):
            sel = lev >= 1
            nl, na = lev[sel], anc[sel].copy()
            na[:, d] += sgn
            size = macro[None, :] << nl[:, None]
            ok = np.all((na >= 0) & (na < size), axis=1)
            nl, na = nl[ok] - 1, na[ok] >> 1
            miss = ~np.isin(_cell_keys(dim, nl, na), exist)
            nl, na = nl[miss], na[miss]
            for up in range(1, int(lev.max()) + 1):
                if nl.size == 0:
                    break
                pl = nl - up
                valid = pl >= 0
                k = _cell_keys(dim, np.where(valid, pl, 0), np.where(valid[:, None], na >> up, 0))
                hit = valid & np.isin(k, leaves)
                bad.append(k[hit])
                nl, na = nl[~hit], na[~hit]
    return np.unique(np.concatenate(bad)) if bad else np.zeros(0, dtype=np.int64)


def coarsen_once(dim, macro, level, anchor, min_level, patch=False):
    """One global coarsening step.  Returns (level, anchor) of the coarser
    leaf set, or None if nothing can be taken back.

    patch=False: the unit taken back is a family of 2^d sibling leaves.
    patch=True (patch meshes, where every leaf belongs to a complete family):
    the unit is the 4^d grandchildren of one cell, all leaves, which become
    that cell's 2^d children, so the coarser mesh is a patch mesh again."""
    macro = np.asarray(macro, dtype=np.int64)
    level = np.asarray(level, dtype=np.int64)
    anchor = np.asarray(anchor, dtype=np.int64)
    up = 2 if patch else 1
    cand = (level > min_level) & (level >= up)
    uk = np.full(level.shape[0], -1, dtype=np.int64)          # key of the unit's root cell
    uk[cand] = _cell_keys(dim, level[cand] - up, anchor[cand] >> up)
    uniq, counts = np.unique(uk[cand], return_counts=True)
    units = set(uniq[counts == (1 << (dim * up))].tolist())
    while True:
        take = np.array([k in units for k in uk.tolist()], dtype=bool)
        if not take.any():
            return None
        keep_l, keep_a = level[~take], anchor[~take]
        par_l = level[take] - 1
        par_a = anchor[take] >> 1
        pkeys, first = np.unique(_cell_keys(dim, par_l, par_a), return_index=True)
        new_l = np.concatenate([keep_l, par_l[first]])
        new_a = np.concatenate([keep_a, par_a[first]])
        bad = _violations(dim, macro, new_l, new_a)
        # a too-coarse new leaf reverts the unit it came from
        bad_units = set()
        if bad.size:
            nk = _cell_keys(dim, par_l[first], par_a[first])
            hit = np.isin(nk, bad)
            if hit.any():
                root = _cell_keys(dim, par_l[first][hit] - (up - 1), par_a[first][hit] >> (up - 1))
                bad_units = set(root.tolist())
        revert = units & bad_units
        if not revert:
            return new_l, new_a
        units -= revert


def hierarchy(dim, macro, level, anchor, min_level, max_levels=0, patch=False):
    """Leaf sets from finest (index 0) to coarsest."""
    out = [(np.asarray(level, dtype=np.int64), np.asarray(anchor, dtype=np.int64))]
    while max_levels <= 0 or len(out) < max_levels:
        nxt = coarsen_once(dim, macro, out[-1][0], out[-1][1], min_level, patch)
        if nxt is None:
            break
        out.append(nxt)
    return out


def patches(mesh):
    """Patches of a patch mesh: the parents of the sibling families.  Returns
    (nodes (n_p, 3^d) in lexicographic order of the patch's 3^d lattice
    points, x fastest; level of the children (n_p,)).  Raises if a leaf is
    not part of a complete family."""
    dim = mesh.dim
    if np.any(mesh.level < 1):
        raise ValueError("patch mesh: a leaf on level 0 has no family")
    pk = _cell_keys(dim, mesh.level - 1, mesh.anchor >> 1)
    uniq, inv, counts = np.unique(pk, return_inverse=True, return_counts=True)
    if np.any(counts != (1 << dim)):
        raise ValueError("not a patch mesh: incomplete sibling family")
    n_p = uniq.size
    nodes = np.full((n_p, 3 ** dim), -1, dtype=np.int64)
    lev = np.zeros(n_p, dtype=np.int64)
    off = mesh.corners_offsets()
    child = mesh.anchor & 1                                   # position of each leaf in its family
    for c in range(1 << dim):
        loc = child + off[c][None, :]                         # patch lattice point, entries in {0,1,2}
        li = np.zeros(mesh.level.shape[0], dtype=np.int64)
        for d in reversed(range(dim)):
            li = li * 3 + loc[:, d]
        nodes[inv, li] = mesh.cell_nodes[:, c]
    lev[inv] = mesh.level
    assert np.all(nodes >= 0)
    return nodes, lev


def default_min_level(macro):
    """Coarsest level: the macro grid refined until it has >= 4 cells along
    its longest axis (4x4 for the unit square, the macro grid itself when it
    already has 4 or more)."""
    m = int(max(macro))
    lvl = 0
    while (m << lvl) < 4:
        lvl += 1
    return lvl
