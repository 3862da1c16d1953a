// Host-side hierarchy setup: leaf mesh -> global coarsening -> per level node
// topology with hanging-node constraints, condensed Q1 operators, transfers,
// smoother blocks, coarse inverse and the right-hand-side load matrix.
//
// Paper (arXiv:2405.05047): Sec. 2.1 (Q1 spaces, node-major block layout),
// Sec. 2.2 (1-irregular meshes, hanging-node matrix H_h, global coarsening),
// Sec. 4.1.4 (smoother x <- x + omega S (b - A x), transfers P_l from the local
// embedding, Eq. "prolongation", R_l = P_l^T).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace mgi {

// ------------------------------------------------------------------ helpers
namespace {

// Packed cell key: level in the top 6 bits, anchors below.
inline uint64_t cell_key(int dim, int lev, const int64_t* a) {
  if (dim == 2) return ((uint64_t)lev << 58) | ((uint64_t)a[0] << 29) | (uint64_t)a[1];
  return ((uint64_t)lev << 58) | ((uint64_t)a[0] << 38) | ((uint64_t)a[1] << 19) | (uint64_t)a[2];
}

// Open-addressing hash set/map of 64-bit keys (value = int64 payload).
class KeyMap {
 public:
  explicit KeyMap(size_t expected = 16) {
    size_t cap = 16;
    while (cap < expected * 2 + 16) cap <<= 1;
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, -1);
    mask_ = cap - 1;
  }
  void insert(uint64_t k, int64_t v) {
    size_t i = hash(k) & mask_;
    while (keys_[i] != kEmpty && keys_[i] != k) i = (i + 1) & mask_;
    if (keys_[i] == kEmpty) {
      keys_[i] = k;
      vals_[i] = v;
      if (++count_ * 2 > keys_.size()) grow();
    }
  }
  int64_t get(uint64_t k) const {
    size_t i = hash(k) & mask_;
    while (keys_[i] != kEmpty) {
      if (keys_[i] == k) return vals_[i];
      i = (i + 1) & mask_;
    }
    return -1;
  }
  bool has(uint64_t k) const { return get(k) >= 0; }

 private:
  static constexpr uint64_t kEmpty = ~0ull;
  static size_t hash(uint64_t k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
    return (size_t)k;
  }
  void grow() {
    std::vector<uint64_t> ok = std::move(keys_);
    std::vector<int64_t> ov = std::move(vals_);
    keys_.assign(ok.size() * 2, kEmpty);
    vals_.assign(ok.size() * 2, -1);
    mask_ = keys_.size() - 1;
    count_ = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty) insert(ok[i], ov[i]);
  }
  std::vector<uint64_t> keys_;
  std::vector<int64_t> vals_;
  size_t mask_ = 0, count_ = 0;
};

// Leaves plus every ancestor (the cells that exist in the tree).
KeyMap existing_cells(const LeafSet& s) {
  KeyMap ex(s.size() * 2);
  int64_t a[3];
  for (size_t k = 0; k < s.size(); ++k) {
    int lev = s.lev[k];
    for (int d = 0; d < s.dim; ++d) a[d] = s.anc[k * s.dim + d];
    while (lev >= 0) {
      uint64_t key = cell_key(s.dim, lev, a);
      if (ex.has(key)) break;
      ex.insert(key, 1);
      --lev;
      for (int d = 0; d < s.dim; ++d) a[d] >>= 1;
    }
  }
  return ex;
}

KeyMap leaf_map(const LeafSet& s) {
  KeyMap m(s.size());
  int64_t a[3];
  for (size_t k = 0; k < s.size(); ++k) {
    for (int d = 0; d < s.dim; ++d) a[d] = s.anc[k * s.dim + d];
    m.insert(cell_key(s.dim, s.lev[k], a), (int64_t)k);
  }
  return m;
}

// For every leaf and face direction: if the face neighbour region holds leaves
// two or more levels finer, return the index of the too-coarse leaf.  The
// check is done from the fine side: leaf X (level m), neighbour cell N (level
// m), its parent C (level m-1) must exist; otherwise the leaf covering C is
// coarser than m-1.
std::vector<int64_t> too_coarse_leaves(const LeafSet& s) {
  KeyMap ex = existing_cells(s);
  KeyMap lm = leaf_map(s);
  std::vector<int64_t> out;
  int64_t a[3], c[3];
  for (size_t k = 0; k < s.size(); ++k) {
    int m = s.lev[k];
    if (m < 1) continue;
    for (int d = 0; d < s.dim; ++d) {
      for (int sg = -1; sg <= 1; sg += 2) {
        bool inside = true;
        for (int e = 0; e < s.dim; ++e) {
          a[e] = s.anc[k * s.dim + e] + (e == d ? sg : 0);
          if (a[e] < 0 || a[e] >= ((int64_t)s.macro[e] << m)) inside = false;
        }
        if (!inside) continue;
        for (int e = 0; e < s.dim; ++e) c[e] = a[e] >> 1;
        if (ex.has(cell_key(s.dim, m - 1, c))) continue;
        for (int up = m - 2; up >= 0; --up) {
          for (int e = 0; e < s.dim; ++e) c[e] >>= 1;
          int64_t idx = lm.get(cell_key(s.dim, up, c));
          if (idx >= 0) { out.push_back(idx); break; }
        }
      }
    }
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

}  // namespace

int LeafSet::max_level() const {
  int m = 0;
  for (int32_t l : lev) m = std::max(m, (int)l);
  return m;
}

int default_min_level(const int macro[3], int dim) {
  int mx = 0;
  for (int d = 0; d < dim; ++d) mx = std::max(mx, macro[d]);
  int lvl = 0;
  while (((int64_t)mx << lvl) < 4) ++lvl;
  return lvl;
}

// ------------------------------------------------------------------ validation
Status validate_mesh(const mg_mesh& mesh, LeafSet* out) {
  if (mesh.dim != 2 && mesh.dim != 3) return Status::err(MG_ERR_INVALID, "mesh.dim must be 2 or 3");
  if (mesh.n_leaves <= 0 || !mesh.leaf_level || !mesh.leaf_anchor)
    return Status::err(MG_ERR_INVALID, "empty leaf list");
  LeafSet s;
  s.dim = mesh.dim;
  for (int d = 0; d < 3; ++d) s.macro[d] = d < mesh.dim ? mesh.macro[d] : 1;
  const int maxbits = mesh.dim == 2 ? 29 : 19;
  for (int d = 0; d < mesh.dim; ++d) {
    if (mesh.macro[d] < 1) return Status::err(MG_ERR_INVALID, "macro grid must be >= 1 per axis");
    if (!(mesh.extent[d] > 0.0)) return Status::err(MG_ERR_INVALID, "extent must be positive");
  }
  s.lev.assign(mesh.leaf_level, mesh.leaf_level + mesh.n_leaves);
  s.anc.assign(mesh.leaf_anchor, mesh.leaf_anchor + mesh.n_leaves * mesh.dim);
  int L = 0;
  for (int64_t k = 0; k < mesh.n_leaves; ++k) {
    int l = s.lev[k];
    if (l < 0 || l > 24) return Status::err(MG_ERR_INVALID, "leaf level out of range [0,24]");
    L = std::max(L, l);
    for (int d = 0; d < mesh.dim; ++d) {
      int64_t a = s.anc[k * mesh.dim + d];
      if (a < 0 || a >= ((int64_t)mesh.macro[d] << l)) return Status::err(MG_ERR_INVALID, "leaf anchor outside the domain");
    }
  }
  for (int d = 0; d < mesh.dim; ++d)
    if (((int64_t)mesh.macro[d] << L) >= ((int64_t)1 << maxbits))
      return Status::err(MG_ERR_INVALID, "mesh too fine for the key width");
  // no leaf may be an ancestor of (or equal to) another one
  KeyMap lm = leaf_map(s);
  int64_t a[3];
  long double vol = 0;
  for (int64_t k = 0; k < mesh.n_leaves; ++k) {
    for (int d = 0; d < mesh.dim; ++d) a[d] = s.anc[k * mesh.dim + d];
    if (lm.get(cell_key(mesh.dim, s.lev[k], a)) != k) return Status::err(MG_ERR_INVALID, "duplicate leaf");
    for (int up = s.lev[k] - 1; up >= 0; --up) {
      for (int d = 0; d < mesh.dim; ++d) a[d] >>= 1;
      if (lm.has(cell_key(mesh.dim, up, a))) return Status::err(MG_ERR_INVALID, "overlapping leaves");
    }
    vol += std::ldexp((long double)1, -mesh.dim * s.lev[k]);
  }
  long double full = 1;
  for (int d = 0; d < mesh.dim; ++d) full *= mesh.macro[d];
  if (std::fabs((double)(vol - full)) > 1e-9) return Status::err(MG_ERR_INVALID, "leaves do not tile the domain");
  if (!too_coarse_leaves(s).empty()) return Status::err(MG_ERR_INVALID, "mesh violates the 2:1 rule");
  *out = std::move(s);
  return Status::ok();
}

// ------------------------------------------------------------------ coarsening
// Sec. 2.2: take back every family of 2^d sibling leaves (above min_level);
// families whose parent would be two levels coarser than a face neighbour are
// kept refined; repeat that check until the coarser mesh is 1-irregular.
// patch = true (patch meshes of the LPS-stabilised Oseen problem): the unit
// taken back is all 4^d grandchildren of one cell, which become its 2^d
// children, so every coarser level is again a patch mesh.
bool coarsen_once(const LeafSet& fine, int min_level, bool patch, LeafSet* coarse) {
  const int dim = fine.dim, up = patch ? 2 : 1, nunit = 1 << (dim * up);
  std::vector<uint64_t> ukey(fine.size(), ~0ull);
  std::vector<uint64_t> units;
  int64_t a[3];
  {
    // count leaves per unit root (parent, or grandparent for patch meshes)
    std::vector<std::pair<uint64_t, int>> tally;
    KeyMap slot(fine.size());
    for (size_t k = 0; k < fine.size(); ++k) {
      if (fine.lev[k] <= min_level || fine.lev[k] < up) continue;
      for (int d = 0; d < dim; ++d) a[d] = fine.anc[k * dim + d] >> up;
      uint64_t uk = cell_key(dim, fine.lev[k] - up, a);
      ukey[k] = uk;
      int64_t s = slot.get(uk);
      if (s < 0) { slot.insert(uk, (int64_t)tally.size()); tally.push_back({uk, 1}); }
      else tally[s].second++;
    }
    for (auto& t : tally)
      if (t.second == nunit) units.push_back(t.first);
  }
  if (units.empty()) return false;
  std::sort(units.begin(), units.end());
  std::vector<char> active(units.size(), 1);
  auto unit_index = [&](uint64_t k) -> int64_t {
    auto it = std::lower_bound(units.begin(), units.end(), k);
    return (it != units.end() && *it == k) ? (int64_t)(it - units.begin()) : -1;
  };
  while (true) {
    LeafSet c;
    c.dim = dim;
    std::copy(fine.macro, fine.macro + 3, c.macro);
    KeyMap made(units.size() * 4 + 16);       // new leaves already emitted
    std::vector<int64_t> unit_of_leaf;        // unit a new (coarsened) leaf came from, -1 otherwise
    for (size_t k = 0; k < fine.size(); ++k) {
      int64_t u = ukey[k] == ~0ull ? -1 : unit_index(ukey[k]);
      if (u >= 0 && active[u]) {
        for (int d = 0; d < dim; ++d) a[d] = fine.anc[k * dim + d] >> 1;
        uint64_t pk = cell_key(dim, fine.lev[k] - 1, a);
        if (made.has(pk)) continue;
        made.insert(pk, 1);
        c.lev.push_back(fine.lev[k] - 1);
        for (int d = 0; d < dim; ++d) c.anc.push_back((int32_t)a[d]);
        unit_of_leaf.push_back(u);
      } else {
        c.lev.push_back(fine.lev[k]);
        for (int d = 0; d < dim; ++d) c.anc.push_back(fine.anc[k * dim + d]);
        unit_of_leaf.push_back(-1);
      }
    }
    std::vector<int64_t> bad = too_coarse_leaves(c);
    bool reverted = false;
    for (int64_t b : bad)
      if (unit_of_leaf[b] >= 0) { active[unit_of_leaf[b]] = 0; reverted = true; }
    if (!reverted) {
      bool any = false;
      for (char x : active) any |= (x != 0);
      if (!any) return false;
      *coarse = std::move(c);
      return true;
    }
  }
}

// Patches of a patch mesh: the parents of its sibling families, each with
// its 3^d lattice points (x fastest) as node indices of T.  Fails when a leaf
// lies on level 0 or its family is incomplete.
Status mesh_patches(const LeafSet& s, const Topology& T, std::vector<int64_t>* nodes, std::vector<int32_t>* clev) {
  const int dim = s.dim, nv = 1 << dim, np3 = dim == 2 ? 9 : 27;
  KeyMap pidx(s.size() / nv + 16);
  std::vector<int> count;
  int64_t a[3];
  for (size_t k = 0; k < s.size(); ++k) {
    if (s.lev[k] < 1) return Status::err(MG_ERR_INVALID, "patch mesh: a leaf on level 0 has no sibling family");
    for (int d = 0; d < dim; ++d) a[d] = s.anc[k * dim + d] >> 1;
    uint64_t pk = cell_key(dim, s.lev[k] - 1, a);
    int64_t p = pidx.get(pk);
    if (p < 0) {
      p = (int64_t)count.size();
      pidx.insert(pk, p);
      count.push_back(0);
      clev->push_back(s.lev[k]);
      nodes->insert(nodes->end(), np3, -1);
    }
    count[p]++;
    for (int c = 0; c < nv; ++c) {
      int li = 0, m = 1;
      for (int d = 0; d < dim; ++d) {
        li += (int)(((s.anc[k * dim + d] & 1) + ((c >> d) & 1)) * m);
        m *= 3;
      }
      (*nodes)[p * np3 + li] = T.cell_node[k * nv + c];
    }
  }
  for (int c : count)
    if (c != nv) return Status::err(MG_ERR_INVALID, "not a patch mesh: a sibling family is incomplete");
  return Status::ok();
}

// ------------------------------------------------------------------ topology
int64_t Topology::find(int64_t k) const {
  auto it = std::lower_bound(key.begin(), key.end(), k);
  return (it != key.end() && *it == k) ? (int64_t)(it - key.begin()) : -1;
}

void Topology::lattice_coords(int64_t node, int64_t X[3]) const {
  int64_t k = key[node];
  for (int d = 0; d < dim; ++d) {
    X[d] = k % (ncell[d] + 1);
    k /= (ncell[d] + 1);
  }
}

void build_topology(const LeafSet& s, Topology* T) {
  const int dim = s.dim, nv = 1 << dim;
  T->dim = dim;
  T->L = s.max_level();
  for (int d = 0; d < 3; ++d) T->ncell[d] = d < dim ? ((int64_t)s.macro[d] << T->L) : 0;
  auto lat_key = [&](const int64_t* X) {
    int64_t k = 0, m = 1;
    for (int d = 0; d < dim; ++d) { k += X[d] * m; m *= (T->ncell[d] + 1); }
    return k;
  };
  const int64_t n = (int64_t)s.size();
  std::vector<int64_t> corner(n * nv);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    int64_t sz = (int64_t)1 << (T->L - s.lev[k]);
    int64_t X[3];
    for (int c = 0; c < nv; ++c) {
      for (int d = 0; d < dim; ++d) X[d] = (s.anc[k * dim + d] + ((c >> d) & 1)) * sz;
      corner[k * nv + c] = lat_key(X);
    }
  }
  T->key = corner;
  std::sort(T->key.begin(), T->key.end());
  T->key.erase(std::unique(T->key.begin(), T->key.end()), T->key.end());
  T->n_nodes = (int64_t)T->key.size();
  T->cell_node.resize(n * nv);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n * nv; ++i) T->cell_node[i] = T->find(corner[i]);

  // hanging nodes: midpoints of cell edges (and centres of cell faces in 3D)
  // that are nodes of the mesh; value = mean of the edge's/face's vertices.
  T->hanging.assign(T->n_nodes, 0);
  T->hang_kind.assign(T->n_nodes, 0);
  std::vector<std::vector<int64_t>> parents(T->n_nodes);
  for (int64_t k = 0; k < n; ++k) {
    if (s.lev[k] >= T->L) continue;
    int64_t sz = (int64_t)1 << (T->L - s.lev[k]);
    int64_t half = sz / 2;
    int pat[3];
    int npat = 1;
    for (int d = 0; d < dim; ++d) npat *= 3;
    for (int p = 0; p < npat; ++p) {
      int q = p, nh = 0;
      for (int d = 0; d < dim; ++d) { pat[d] = q % 3; q /= 3; nh += pat[d] == 1; }
      if (nh == 0 || nh == dim) continue;             // vertices and the cell centre
      int64_t X[3];
      for (int d = 0; d < dim; ++d) X[d] = s.anc[k * dim + d] * sz + pat[d] * half;
      int64_t h = T->find(lat_key(X));
      if (h < 0 || T->hanging[h]) continue;
      T->hanging[h] = 1;
      T->hang_kind[h] = (uint8_t)(1 << nh);
      for (int c = 0; c < (1 << nh); ++c) {
        int64_t Y[3];
        int bit = 0;
        for (int d = 0; d < dim; ++d) {
          if (pat[d] == 1) Y[d] = s.anc[k * dim + d] * sz + (((c >> bit++) & 1) ? sz : 0);
          else Y[d] = X[d];
        }
        parents[h].push_back(T->find(lat_key(Y)));
      }
    }
  }
  // constraints, chains resolved so that every entry is a regular node
  T->con_ptr.assign(T->n_nodes + 1, 0);
  std::vector<std::vector<std::pair<int64_t, double>>> res(T->n_nodes);
  std::function<void(int64_t)> resolve;
  std::vector<char> state(T->n_nodes, 0);
  resolve = [&](int64_t h) {
    if (state[h] == 2) return;
    state[h] = 1;
    std::vector<std::pair<int64_t, double>> acc;
    double w = 1.0 / (double)parents[h].size();
    for (int64_t p : parents[h]) {
      if (T->hanging[p]) {
        resolve(p);
        for (auto& e : res[p]) acc.push_back({e.first, w * e.second});
      } else {
        acc.push_back({p, w});
      }
    }
    std::sort(acc.begin(), acc.end());
    std::vector<std::pair<int64_t, double>> merged;
    for (auto& e : acc) {
      if (!merged.empty() && merged.back().first == e.first) merged.back().second += e.second;
      else merged.push_back(e);
    }
    res[h] = std::move(merged);
    state[h] = 2;
  };
  for (int64_t i = 0; i < T->n_nodes; ++i)
    if (T->hanging[i]) resolve(i);
  for (int64_t i = 0; i < T->n_nodes; ++i) T->con_ptr[i + 1] = T->con_ptr[i] + (T->hanging[i] ? (int64_t)res[i].size() : 1);
  T->con_node.resize(T->con_ptr[T->n_nodes]);
  T->con_w.resize(T->con_ptr[T->n_nodes]);
  for (int64_t i = 0; i < T->n_nodes; ++i) {
    int64_t o = T->con_ptr[i];
    if (!T->hanging[i]) { T->con_node[o] = i; T->con_w[o] = 1.0; continue; }
    for (auto& e : res[i]) { T->con_node[o] = e.first; T->con_w[o] = e.second; ++o; }
  }
}

// ------------------------------------------------------------------ elements
namespace {

// 1D integrals over [0, h] of products of the two linear hat functions,
// with or without derivative on the test (row) and trial (column) function.
struct Line {
  double v[2][2][2][2];   // [test deriv][trial deriv][a][b]
  explicit Line(double h) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double sa = a ? 1.0 : -1.0, sb = b ? 1.0 : -1.0;
        v[0][0][a][b] = h / 6.0 * (a == b ? 2.0 : 1.0);   // int phi_a phi_b
        v[1][1][a][b] = sa * sb / h;                      // int phi_a' phi_b'
        v[0][1][a][b] = 0.5 * sb;                         // int phi_a phi_b'
        v[1][0][a][b] = 0.5 * sa;                         // int phi_a' phi_b
      }
  }
};

// G(i, j)[A][B] = int D_i phi_A D_j phi_B over the box, D_-1 = value,
// D_d = d/dx_d.  Tensor product of the 1D integrals.
struct BoxIntegrals {
  int dim, nv;
  std::vector<Line> lines;
  BoxIntegrals(int dim_, const double* h) : dim(dim_), nv(1 << dim_) {
    for (int d = 0; d < dim; ++d) lines.emplace_back(h[d]);
  }
  double G(int i, int j, int A, int B) const {
    double r = 1.0;
    for (int e = 0; e < dim; ++e) r *= lines[e].v[i == e][j == e][(A >> e) & 1][(B >> e) & 1];
    return r;
  }
};

// Element matrix in node-major block order: K[(A*nc + i)*(nv*nc) + B*nc + j].
std::vector<double> element_matrix(const mg_problem& P, int dim, const double* h) {
  BoxIntegrals I(dim, h);
  const int nv = 1 << dim;
  if (P.kind == MG_ELASTICITY) {
    const int nc = 3, w = nv * nc;
    std::vector<double> K(w * w, 0.0);
    for (int A = 0; A < nv; ++A)
      for (int B = 0; B < nv; ++B) {
        double lap = 0;
        for (int e = 0; e < dim; ++e) lap += I.G(e, e, A, B);
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j)
            K[(A * nc + i) * w + B * nc + j] =
                P.mu * ((i == j ? lap : 0.0) + I.G(j, i, A, B)) + P.lambda * I.G(i, j, A, B) +
                (i == j ? P.mass * I.G(-1, -1, A, B) : 0.0);   // s (u, v) per component
      }
    return K;
  }
  std::vector<double> K(nv * nv, 0.0);
  double diff = P.kind == MG_TRANSPORT ? P.eps : 1.0;
  double delta = 0.0, bn = 0.0, hT = 0.0;
  if (P.kind == MG_TRANSPORT) {
    for (int d = 0; d < dim; ++d) { bn += P.beta[d] * P.beta[d]; hT += h[d] * h[d]; }
    bn = std::sqrt(bn);
    hT = std::sqrt(hT);
    delta = P.supg_delta0 * hT * hT / (6.0 * P.eps + bn * hT);
  }
  for (int A = 0; A < nv; ++A)
    for (int B = 0; B < nv; ++B) {
      double v = 0;
      for (int e = 0; e < dim; ++e) v += diff * I.G(e, e, A, B);
      if (P.kind == MG_TRANSPORT) {
        for (int j = 0; j < dim; ++j) v += P.beta[j] * I.G(-1, j, A, B);
        for (int i = 0; i < dim; ++i)
          for (int j = 0; j < dim; ++j) v += delta * P.beta[i] * P.beta[j] * I.G(i, j, A, B);
      }
      if (P.mass != 0.0) {
        // s (u, v), and its SUPG test delta_T s (u, beta.grad v)
        double m = I.G(-1, -1, A, B);
        if (P.kind == MG_TRANSPORT)
          for (int i = 0; i < dim; ++i) m += delta * P.beta[i] * I.G(i, -1, A, B);
        v += P.mass * m;
      }
      K[A * nv + B] = v;
    }
  return K;
}

// Triple 1D integrals over [0, h] for the cell-wise bilinear convection field:
// t[0][c][a][b] = int phi_c phi_a phi_b, t[1][c][a][b] = int phi_c phi_a phi_b'.
struct Line3 {
  double t[2][2][2][2];
  explicit Line3(double h) {
    for (int c = 0; c < 2; ++c)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double sb = b ? 1.0 : -1.0;
          t[0][c][a][b] = h / 12.0 * ((a == b && b == c) ? 3.0 : 1.0);
          t[1][c][a][b] = sb / 6.0 * (c == a ? 2.0 : 1.0);
        }
  }
};

// Patch matrix (27 x 27, node-major (A*3 + i)*27 + B*3 + j, i = u, v, p) of
// the 2D Oseen form with local projection stabilisation on a patch of four
// child cells of edge lengths h; beta9: nodal convection at the patch's 3x3
// lattice points (x fastest), 9 x 2.  Integrals are exact tensor products of
// 1D integrals (the convection field is bilinear on every child).
void oseen_patch_matrix(const mg_problem& P, const double* h, const double* beta9, double* K) {
  std::fill(K, K + 27 * 27, 0.0);
  BoxIntegrals I(2, h);
  Line3 L3x(h[0]), L3y(h[1]);
  const double inv_dt = std::isinf(P.dt) ? 0.0 : 1.0 / P.dt;
  double G9[9][9] = {}, Gij[2][2][9][9] = {};
  for (int cy = 0; cy < 2; ++cy)
    for (int cx = 0; cx < 2; ++cx) {
      int loc[4];
      for (int c = 0; c < 4; ++c) loc[c] = (cx + (c & 1)) + 3 * (cy + (c >> 1));
      for (int A = 0; A < 4; ++A)
        for (int B = 0; B < 4; ++B) {
          const int ax = A & 1, ay = A >> 1, bx = B & 1, by = B >> 1;
          const double mass = I.G(-1, -1, A, B);
          const double lap = I.G(0, 0, A, B) + I.G(1, 1, A, B);
          double conv = 0.0;    // int phi_A (beta_h . grad phi_B)
          for (int C = 0; C < 4; ++C) {
            const int cxx = C & 1, cyy = C >> 1;
            const double* bC = beta9 + 2 * loc[C];
            conv += bC[0] * L3x.t[1][cxx][ax][bx] * L3y.t[0][cyy][ay][by];
            conv += bC[1] * L3x.t[0][cxx][ax][bx] * L3y.t[1][cyy][ay][by];
          }
          const double vv = inv_dt * mass + P.nu * lap + conv;
          const int r = loc[A], c = loc[B];
          for (int i = 0; i < 2; ++i) {
            K[(r * 3 + i) * 27 + c * 3 + i] += vv;
            K[(r * 3 + i) * 27 + c * 3 + 2] -= I.G(i, -1, A, B);   // -(p, div v)
            K[(r * 3 + 2) * 27 + c * 3 + i] += I.G(-1, i, A, B);   // (div u, q)
          }
          G9[r][c] += lap;
          for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) Gij[i][j][r][c] += I.G(i, j, A, B);
        }
    }
  // kappa = id - Pi, Pi the coarse Q1 interpolant from the patch corners
  double kap[9][9];
  for (int n = 0; n < 9; ++n)
    for (int m = 0; m < 9; ++m) {
      double pi = 0.0;
      const int mx = m % 3, my = m / 3;
      if ((mx == 0 || mx == 2) && (my == 0 || my == 2)) {
        const double tx = (n % 3) / 2.0, ty = (n / 3) / 2.0;
        pi = (mx ? tx : 1.0 - tx) * (my ? ty : 1.0 - ty);
      }
      kap[n][m] = (n == m ? 1.0 : 0.0) - pi;
    }
  const double* bP = beta9 + 2 * 4;
  const double hP = 2.0 * std::sqrt(h[0] * h[0] + h[1] * h[1]);
  const double alpha = P.lps_alpha0 * hP * hP / (P.nu + std::sqrt(bP[0] * bP[0] + bP[1] * bP[1]) * hP);
  double Cb[9][9];
  for (int a = 0; a < 9; ++a)
    for (int b = 0; b < 9; ++b) {
      double v = 0.0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) v += bP[i] * bP[j] * Gij[i][j][a][b];
      Cb[a][b] = v;
    }
  // S = kappa^T M kappa for M = G9 (pressure) and Cb (velocity components)
  for (int which = 0; which < 2; ++which) {
    double (*M)[9] = which == 0 ? G9 : Cb;
    double Mk[9][9];
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 9; ++b) {
        double v = 0.0;
        for (int k = 0; k < 9; ++k) v += M[a][k] * kap[k][b];
        Mk[a][b] = v;
      }
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 9; ++b) {
        double v = 0.0;
        for (int k = 0; k < 9; ++k) v += kap[k][a] * Mk[k][b];
        v *= alpha;
        if (which == 0) K[(a * 3 + 2) * 27 + b * 3 + 2] += v;
        else
          for (int i = 0; i < 2; ++i) K[(a * 3 + i) * 27 + b * 3 + i] += v;
      }
  }
}

// Load element F[A][B]: b_A = sum_B F[A][B] f_B for nodal f (mass matrix,
// plus the SUPG term delta_T (f_h, beta.grad phi_A) for transport).
std::vector<double> load_element(const mg_problem& P, int dim, const double* h) {
  BoxIntegrals I(dim, h);
  const int nv = 1 << dim;
  std::vector<double> F(nv * nv);
  double delta = 0.0;
  if (P.kind == MG_TRANSPORT) {
    double bn = 0, hT = 0;
    for (int d = 0; d < dim; ++d) { bn += P.beta[d] * P.beta[d]; hT += h[d] * h[d]; }
    bn = std::sqrt(bn); hT = std::sqrt(hT);
    delta = P.supg_delta0 * hT * hT / (6.0 * P.eps + bn * hT);
  }
  for (int A = 0; A < nv; ++A)
    for (int B = 0; B < nv; ++B) {
      double v = I.G(-1, -1, A, B);
      if (delta != 0.0)
        for (int d = 0; d < dim; ++d) v += delta * P.beta[d] * I.G(d, -1, A, B);
      F[A * nv + B] = v;
    }
  return F;
}

void cell_size(const HostHierarchy& H, int lev, double* h) {
  for (int d = 0; d < H.dim; ++d) h[d] = H.extent[d] / ((double)H.macro[d] * std::ldexp(1.0, lev));
}
// Sizes of cell k of topology T on a graded mesh: its lowest and highest
// corners (corner 0 and corner 2^dim - 1, x fastest) looked up in the axis
// coordinates of the finest lattice.
void cell_size_graded(const HostHierarchy& H, const Topology& T, int64_t k, double* h) {
  const int nv = 1 << H.dim;
  int64_t X0[3], X1[3];
  T.lattice_coords(T.cell_node[k * nv], X0);
  T.lattice_coords(T.cell_node[k * nv + nv - 1], X1);
  const int sh = H.axis_L - T.L;
  for (int d = 0; d < H.dim; ++d) h[d] = H.axis[d][X1[d] << sh] - H.axis[d][X0[d] << sh];
}

// node -> list of (element, local node) incidences through the constraints:
// entry for every regular node p that receives a share of local node A of
// element k.  Elements are cells (m = 2^d corners) or LPS patches (m = 3^d).
struct Incidence {
  std::vector<int64_t> ptr, cell;
  std::vector<int8_t> corner;
  std::vector<double> w;
};

Incidence expanded_incidence(int64_t n_elem, int m, const std::vector<int64_t>& elem_node, const Topology& T) {
  Incidence inc;
  inc.ptr.assign(T.n_nodes + 1, 0);
  for (int64_t k = 0; k < n_elem; ++k)
    for (int A = 0; A < m; ++A) {
      int64_t v = elem_node[k * m + A];
      for (int64_t o = T.con_ptr[v]; o < T.con_ptr[v + 1]; ++o) inc.ptr[T.con_node[o] + 1]++;
    }
  for (int64_t i = 0; i < T.n_nodes; ++i) inc.ptr[i + 1] += inc.ptr[i];
  inc.cell.resize(inc.ptr.back());
  inc.corner.resize(inc.ptr.back());
  inc.w.resize(inc.ptr.back());
  std::vector<int64_t> fill(inc.ptr.begin(), inc.ptr.end() - 1);
  for (int64_t k = 0; k < n_elem; ++k)
    for (int A = 0; A < m; ++A) {
      int64_t v = elem_node[k * m + A];
      for (int64_t o = T.con_ptr[v]; o < T.con_ptr[v + 1]; ++o) {
        int64_t p = T.con_node[o];
        int64_t at = fill[p]++;
        inc.cell[at] = k;
        inc.corner[at] = (int8_t)A;
        inc.w[at] = T.con_w[o];
      }
    }
  return inc;
}

Incidence expanded_incidence(const LeafSet& s, const Topology& T) {
  return expanded_incidence((int64_t)s.size(), 1 << s.dim, T.cell_node, T);
}

uint8_t dirichlet_bits(const HostHierarchy& H, const Topology& T, int64_t node) {
  int64_t X[3];
  T.lattice_coords(node, X);
  uint8_t bits = 0;
  for (int c = 0; c < H.nc; ++c) {
    uint32_t m = H.prob.dirichlet_mask[c];
    for (int d = 0; d < H.dim; ++d) {
      if (((m >> (2 * d)) & 1) && X[d] == 0) bits |= (uint8_t)(1 << c);
      if (((m >> (2 * d + 1)) & 1) && X[d] == T.ncell[d]) bits |= (uint8_t)(1 << c);
    }
  }
  if (H.prob.pin_origin) {
    bool origin = true;
    for (int d = 0; d < H.dim; ++d) origin = origin && X[d] == 0;
    if (origin) bits |= (uint8_t)((1u << H.nc) - 1u);
  }
  return bits;
}

// Condensed operator H^T A H with identity rows/columns on fixed dofs,
// assembled row by row (each row gathers the elements whose constrained node
// shares reach it).  Elements have m nodes (elem_node[k*m + a]); Kof(k)
// returns element k's (m nc)^2 matrix, node-major.  With lift != nullptr the
// entries of H^T A H that couple free dofs (rows) to Dirichlet dofs (columns)
// are also kept there before the elimination (lifting of Dirichlet data).
void assemble_condensed(const HostHierarchy& H, HostLevel& lv, int64_t n_elem, int m,
                        const std::vector<int64_t>& elem_node, const std::function<const double*(int64_t)>& Kof,
                        BlockCSR* lift) {
  const Topology& T = lv.topo;
  const int nc = H.nc, nb = nc * nc;
  const uint8_t all = (uint8_t)((1 << nc) - 1);
  lv.fixmask.assign(T.n_nodes, 0);
  for (int64_t i = 0; i < T.n_nodes; ++i) lv.fixmask[i] = T.hanging[i] ? all : dirichlet_bits(H, T, i);
  Incidence inc = expanded_incidence(n_elem, m, elem_node, T);
  BlockCSR& A = lv.A;
  A.n = A.m = T.n_nodes;
  A.nc = nc;
  A.ptr.assign(T.n_nodes + 1, 0);
  auto row_cols = [&](int64_t p, std::vector<int64_t>& cols) {
    cols.clear();
    cols.push_back(p);
    if (T.hanging[p]) return;
    for (int64_t o = inc.ptr[p]; o < inc.ptr[p + 1]; ++o) {
      int64_t k = inc.cell[o];
      for (int B = 0; B < m; ++B) {
        int64_t v = elem_node[k * m + B];
        for (int64_t q = T.con_ptr[v]; q < T.con_ptr[v + 1]; ++q) cols.push_back(T.con_node[q]);
      }
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  };
#pragma omp parallel
  {
    std::vector<int64_t> cols;
#pragma omp for schedule(dynamic, 4096)
    for (int64_t p = 0; p < T.n_nodes; ++p) { row_cols(p, cols); A.ptr[p + 1] = (int64_t)cols.size(); }
  }
  for (int64_t p = 0; p < T.n_nodes; ++p) A.ptr[p + 1] += A.ptr[p];
  A.col.resize(A.ptr.back());
  A.val.assign(A.ptr.back() * nb, 0.0);
  std::vector<std::vector<int64_t>> lcol(lift ? T.n_nodes : 0);
  std::vector<std::vector<double>> lval(lift ? T.n_nodes : 0);
  const int w = m * nc;
#pragma omp parallel
  {
    std::vector<int64_t> cols;
#pragma omp for schedule(dynamic, 4096)
    for (int64_t p = 0; p < T.n_nodes; ++p) {
      row_cols(p, cols);
      int64_t base = A.ptr[p];
      std::copy(cols.begin(), cols.end(), A.col.begin() + base);
      double* rv = &A.val[base * nb];
      const int64_t len = (int64_t)cols.size();
      if (!T.hanging[p]) {
        for (int64_t o = inc.ptr[p]; o < inc.ptr[p + 1]; ++o) {
          int64_t k = inc.cell[o];
          int Acorner = inc.corner[o];
          double wa = inc.w[o];
          const double* K = Kof(k);
          for (int B = 0; B < m; ++B) {
            int64_t v = elem_node[k * m + B];
            for (int64_t q = T.con_ptr[v]; q < T.con_ptr[v + 1]; ++q) {
              int64_t c = T.con_node[q];
              double wq = wa * T.con_w[q];
              int64_t pos = std::lower_bound(cols.begin(), cols.end(), c) - cols.begin();
              double* blk = rv + pos * nb;
              for (int i = 0; i < nc; ++i)
                for (int j = 0; j < nc; ++j) blk[i * nc + j] += wq * K[(Acorner * nc + i) * w + B * nc + j];
            }
          }
        }
      }
      uint8_t fp = lv.fixmask[p];
      if (lift && fp != all)
        for (int64_t e = 0; e < len; ++e) {
          uint8_t fq = lv.fixmask[cols[e]];     // columns are regular nodes: Dirichlet bits only
          if (!fq) continue;
          std::vector<double> blk(nb, 0.0);
          bool any = false;
          for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j)
              if (!((fp >> i) & 1) && ((fq >> j) & 1)) { blk[i * nc + j] = rv[e * nb + i * nc + j]; any = true; }
          if (any) { lcol[p].push_back(cols[e]); lval[p].insert(lval[p].end(), blk.begin(), blk.end()); }
        }
      // symmetric elimination of fixed dofs: zero their rows and columns,
      // identity on their diagonal
      for (int64_t e = 0; e < len; ++e) {
        uint8_t fq = lv.fixmask[cols[e]];
        double* blk = rv + e * nb;
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j)
            if (((fp >> i) & 1) || ((fq >> j) & 1)) blk[i * nc + j] = 0.0;
        if (cols[e] == p)
          for (int i = 0; i < nc; ++i)
            if ((fp >> i) & 1) blk[i * nc + i] = 1.0;
      }
    }
  }
  if (lift) {
    lift->n = lift->m = T.n_nodes;
    lift->nc = nc;
    lift->ptr.assign(T.n_nodes + 1, 0);
    for (int64_t p = 0; p < T.n_nodes; ++p) lift->ptr[p + 1] = lift->ptr[p] + (int64_t)lcol[p].size();
    lift->col.clear();
    lift->val.clear();
    for (int64_t p = 0; p < T.n_nodes; ++p) {
      lift->col.insert(lift->col.end(), lcol[p].begin(), lcol[p].end());
      lift->val.insert(lift->val.end(), lval[p].begin(), lval[p].end());
    }
  }
}

// Level operator by rediscretisation: cell element matrices (constant
// coefficients, one matrix per cell level), or for OSEEN the patch matrices
// with the level's nodal convection field beta (n_nodes x 2).
Status assemble_level(const HostHierarchy& H, HostLevel& lv, const std::vector<double>& beta, BlockCSR* lift) {
  const LeafSet& s = lv.leaves;
  const Topology& T = lv.topo;
  const int dim = s.dim, nv = 1 << dim;
  if (H.prob.kind == MG_OSEEN) {
    std::vector<int64_t> pn;
    std::vector<int32_t> clev;
    Status st = mesh_patches(s, T, &pn, &clev);
    if (!st.good()) return st;
    const int64_t np = (int64_t)clev.size();
    std::vector<double> Kp((size_t)np * 27 * 27);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < np; ++k) {
      double h[3], b9[18];
      cell_size(H, clev[k], h);
      for (int a = 0; a < 9; ++a)
        for (int d = 0; d < 2; ++d) b9[2 * a + d] = beta[2 * pn[k * 9 + a] + d];
      oseen_patch_matrix(H.prob, h, b9, &Kp[(size_t)k * 729]);
    }
    assemble_condensed(H, lv, np, 9, pn, [&](int64_t k) { return &Kp[(size_t)k * 729]; }, lift);
    return Status::ok();
  }
  if (!H.axis[0].empty()) {
    // graded mesh: one element matrix per cell
    const size_t m = (size_t)nv * H.nc * nv * H.nc;
    std::vector<double> Kc(s.size() * m);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)s.size(); ++k) {
      double h[3];
      cell_size_graded(H, T, k, h);
      std::vector<double> e = element_matrix(H.prob, dim, h);
      std::copy(e.begin(), e.end(), Kc.begin() + (size_t)k * m);
    }
    assemble_condensed(H, lv, (int64_t)s.size(), nv, T.cell_node, [&](int64_t k) { return &Kc[(size_t)k * m]; },
                       lift);
    return Status::ok();
  }
  std::vector<std::vector<double>> Ke(32);
  for (size_t k = 0; k < s.size(); ++k) {
    int l = s.lev[k];
    if (Ke[l].empty()) { double h[3]; cell_size(H, l, h); Ke[l] = element_matrix(H.prob, dim, h); }
  }
  assemble_condensed(H, lv, (int64_t)s.size(), nv, T.cell_node, [&](int64_t k) { return Ke[s.lev[k]].data(); },
                     lift);
  return Status::ok();
}

// b = H^T (F f): rows are the nodes receiving constrained shares, columns are
// all nodes (f is given at every node, hanging ones included).
void assemble_load(const HostHierarchy& H, const HostLevel& lv, BlockCSR* F) {
  const LeafSet& s = lv.leaves;
  const Topology& T = lv.topo;
  const int dim = s.dim, nv = 1 << dim;
  std::vector<std::vector<double>> Fe(H.axis[0].empty() ? 32 : s.size());
  if (!H.axis[0].empty()) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)s.size(); ++k) {
      double h[3];
      cell_size_graded(H, T, k, h);
      Fe[k] = load_element(H.prob, dim, h);
    }
  } else {
    for (size_t k = 0; k < s.size(); ++k) {
      int l = s.lev[k];
      if (Fe[l].empty()) { double h[3]; cell_size(H, l, h); Fe[l] = load_element(H.prob, dim, h); }
    }
  }
  const bool graded = !H.axis[0].empty();
  Incidence inc = expanded_incidence(s, T);
  F->n = F->m = T.n_nodes;
  F->nc = 1;
  F->ptr.assign(T.n_nodes + 1, 0);
  std::vector<std::vector<int64_t>> rows(T.n_nodes);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t p = 0; p < T.n_nodes; ++p) {
    std::vector<int64_t>& cols = rows[p];
    cols.push_back(p);
    for (int64_t o = inc.ptr[p]; o < inc.ptr[p + 1]; ++o)
      for (int B = 0; B < nv; ++B) cols.push_back(T.cell_node[inc.cell[o] * nv + B]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
  }
  for (int64_t p = 0; p < T.n_nodes; ++p) F->ptr[p + 1] = F->ptr[p] + (int64_t)rows[p].size();
  F->col.resize(F->ptr.back());
  F->val.assign(F->ptr.back(), 0.0);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t p = 0; p < T.n_nodes; ++p) {
    const std::vector<int64_t>& cols = rows[p];
    std::copy(cols.begin(), cols.end(), F->col.begin() + F->ptr[p]);
    for (int64_t o = inc.ptr[p]; o < inc.ptr[p + 1]; ++o) {
      int64_t k = inc.cell[o];
      const std::vector<double>& Fk = Fe[graded ? (size_t)k : (size_t)s.lev[k]];
      for (int B = 0; B < nv; ++B) {
        int64_t c = T.cell_node[k * nv + B];
        int64_t pos = std::lower_bound(cols.begin(), cols.end(), c) - cols.begin();
        F->val[F->ptr[p] + pos] += inc.w[o] * Fk[inc.corner[o] * nv + B];
      }
    }
  }
}

// Prolongation fine <- coarse (Eq. "prolongation"): value of the coarse Q1
// function at each fine node, read from the coarse leaf that contains the
// node, with the coarse vertex values completed by the coarse constraints.
// Rows of fully fixed fine nodes and columns of fully fixed coarse nodes are
// zero.
void build_transfer(const HostHierarchy& H, const HostLevel& coarse, HostLevel& fine) {
  const int dim = H.dim, nv = 1 << dim;
  const Topology& Tf = fine.topo;
  const Topology& Tc = coarse.topo;
  const uint8_t all = (uint8_t)((1 << H.nc) - 1);
  KeyMap cl = leaf_map(coarse.leaves);
  int minl = 99, maxl = 0;
  for (int32_t l : coarse.leaves.lev) { minl = std::min(minl, (int)l); maxl = std::max(maxl, (int)l); }
  const int Lf = Tf.L, Lc = Tc.L;
  BlockCSR& P = fine.P;
  P.n = Tf.n_nodes;
  P.m = Tc.n_nodes;
  P.nc = 1;
  std::vector<std::vector<std::pair<int64_t, double>>> rows(Tf.n_nodes);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < Tf.n_nodes; ++i) {
    if (fine.fixmask[i] == all) continue;
    int64_t X[3], a[3];
    Tf.lattice_coords(i, X);
    int lev = -1;
    for (int l = minl; l <= maxl; ++l) {
      for (int d = 0; d < dim; ++d)
        a[d] = std::min(X[d] >> (Lf - l), ((int64_t)H.macro[d] << l) - 1);
      if (cl.has(cell_key(dim, l, a))) { lev = l; break; }
    }
    std::vector<std::pair<int64_t, double>> acc;
    const int64_t s = (int64_t)1 << (Lf - lev);
    for (int c = 0; c < nv; ++c) {
      double w = 1.0;
      int64_t Y[3];
      for (int d = 0; d < dim; ++d) {
        // position in the coarse cell: lattice fraction, or on a graded mesh
        // the physical one (the coarse Q1 function is linear along each axis
        // of its box, so this is its exact value at the fine node)
        double t = (double)(X[d] - a[d] * s) / (double)s;
        if (H.axis_L >= 0) {
          const int sh = H.axis_L - Lf;
          const double x0 = H.axis[d][(a[d] * s) << sh], x1 = H.axis[d][((a[d] + 1) * s) << sh];
          t = (H.axis[d][X[d] << sh] - x0) / (x1 - x0);
        }
        int b = (c >> d) & 1;
        w *= b ? t : 1.0 - t;
        Y[d] = (a[d] + b) << (Lc - lev);
      }
      if (w == 0.0) continue;
      int64_t k = 0, m = 1;
      for (int d = 0; d < dim; ++d) { k += Y[d] * m; m *= (Tc.ncell[d] + 1); }
      int64_t v = Tc.find(k);
      for (int64_t o = Tc.con_ptr[v]; o < Tc.con_ptr[v + 1]; ++o) {
        int64_t q = Tc.con_node[o];
        if (coarse.fixmask[q] == all) continue;
        acc.push_back({q, w * Tc.con_w[o]});
      }
    }
    std::sort(acc.begin(), acc.end());
    auto& out = rows[i];
    for (auto& e : acc) {
      if (!out.empty() && out.back().first == e.first) out.back().second += e.second;
      else out.push_back(e);
    }
  }
  P.ptr.assign(P.n + 1, 0);
  for (int64_t i = 0; i < P.n; ++i) P.ptr[i + 1] = P.ptr[i] + (int64_t)rows[i].size();
  P.col.resize(P.ptr.back());
  P.val.resize(P.ptr.back());
  for (int64_t i = 0; i < P.n; ++i)
    for (size_t e = 0; e < rows[i].size(); ++e) {
      P.col[P.ptr[i] + e] = rows[i][e].first;
      P.val[P.ptr[i] + e] = rows[i][e].second;
    }
  // R = P^T, stored as its own gather matrix (rows: coarse nodes)
  BlockCSR& R = fine.R;
  R.n = P.m; R.m = P.n; R.nc = 1;
  R.ptr.assign(R.n + 1, 0);
  for (int64_t c : P.col) R.ptr[c + 1]++;
  for (int64_t j = 0; j < R.n; ++j) R.ptr[j + 1] += R.ptr[j];
  R.col.resize(P.col.size());
  R.val.resize(P.col.size());
  std::vector<int64_t> fill(R.ptr.begin(), R.ptr.end() - 1);
  for (int64_t i = 0; i < P.n; ++i)
    for (int64_t e = P.ptr[i]; e < P.ptr[i + 1]; ++e) {
      int64_t at = fill[P.col[e]]++;
      R.col[at] = i;
      R.val[at] = P.val[e];
    }
}

// Inverse of a small dense matrix by Gauss-Jordan elimination with partial
// pivoting (row-major, n x n).  Returns false for a singular matrix.
bool invert_dense(int64_t n, std::vector<double>& M, std::vector<double>& Inv) {
  Inv.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) Inv[i * n + i] = 1.0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    double best = std::fabs(M[c * n + c]);
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > best) { best = std::fabs(M[r * n + c]); piv = r; }
    if (best == 0.0) return false;
    if (piv != c) {
      for (int64_t j = 0; j < n; ++j) { std::swap(M[c * n + j], M[piv * n + j]); std::swap(Inv[c * n + j], Inv[piv * n + j]); }
    }
    double d = 1.0 / M[c * n + c];
    for (int64_t j = 0; j < n; ++j) { M[c * n + j] *= d; Inv[c * n + j] *= d; }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < n; ++j) { M[r * n + j] -= f * M[c * n + j]; Inv[r * n + j] -= f * Inv[c * n + j]; }
    }
  }
  return true;
}

// Additive cell-patch Vanka smoother of a level as a block matrix:
// S = W sum_T P_T A_T^{-1} P_T^T over the level's cells T, with A_T the
// condensed operator restricted to the 2^dim nc unknowns of T's vertices
// (constrained rows and columns are identity rows, so fixed unknowns stay
// decoupled) and W = diag(1 / m_i), m_i the number of cells containing node
// i.  Row pattern: the nodes sharing a cell with the row's node.  Local
// inverses are formed in parallel in chunks of cells, then accumulated.
Status build_vanka(HostLevel& lv, int dim, int nc) {
  const Topology& T = lv.topo;
  const int nv = 1 << dim, k = nv * nc, nb = nc * nc;
  const int64_t n = T.n_nodes, ncell = (int64_t)T.cell_node.size() / nv;
  std::vector<int64_t> m(n, 0);
  for (int64_t q : T.cell_node) m[q]++;
  std::vector<std::vector<int64_t>> nbr(n);
  for (int64_t c = 0; c < ncell; ++c)
    for (int a = 0; a < nv; ++a)
      for (int b = 0; b < nv; ++b) nbr[T.cell_node[c * nv + a]].push_back(T.cell_node[c * nv + b]);
  BlockCSR& S = lv.Sv;
  S = BlockCSR();
  S.n = S.m = n;
  S.nc = nc;
  S.ptr.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    std::sort(nbr[i].begin(), nbr[i].end());
    nbr[i].erase(std::unique(nbr[i].begin(), nbr[i].end()), nbr[i].end());
    S.ptr[i + 1] = S.ptr[i] + (int64_t)nbr[i].size();
  }
  S.col.resize(S.ptr[n]);
  for (int64_t i = 0; i < n; ++i) std::copy(nbr[i].begin(), nbr[i].end(), S.col.begin() + S.ptr[i]);
  std::vector<std::vector<int64_t>>().swap(nbr);
  S.val.assign(S.col.size() * nb, 0.0);
  auto find = [](const BlockCSR& M, int64_t r, int64_t c) -> int64_t {
    for (int64_t e = M.ptr[r]; e < M.ptr[r + 1]; ++e)
      if (M.col[e] == c) return e;
    return -1;
  };
  const int64_t chunk = 16384;
  std::vector<double> inv(chunk * k * k);
  for (int64_t c0 = 0; c0 < ncell; c0 += chunk) {
    const int64_t c1 = std::min(ncell, c0 + chunk);
    bool singular = false;
#pragma omp parallel for schedule(static) reduction(|| : singular)
    for (int64_t c = c0; c < c1; ++c) {
      std::vector<double> M(k * k, 0.0), I;
      for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
          const int64_t e = find(lv.A, T.cell_node[c * nv + a], T.cell_node[c * nv + b]);
          if (e < 0) continue;
          for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j) M[(a * nc + i) * k + b * nc + j] = lv.A.val[e * nb + i * nc + j];
        }
      if (!invert_dense(k, M, I)) singular = true;
      else std::copy(I.begin(), I.end(), inv.begin() + (c - c0) * k * k);
    }
    if (singular) return Status::err(MG_ERR_INVALID, "singular cell block in the Vanka smoother");
    for (int64_t c = c0; c < c1; ++c) {
      const double* I = &inv[(c - c0) * k * k];
      for (int a = 0; a < nv; ++a) {
        const int64_t na = T.cell_node[c * nv + a];
        const double w = 1.0 / (double)m[na];
        for (int b = 0; b < nv; ++b) {
          const int64_t e = find(S, na, T.cell_node[c * nv + b]);
          for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j) S.val[e * nb + i * nc + j] += w * I[(a * nc + i) * k + b * nc + j];
        }
      }
    }
  }
  return Status::ok();
}

// Largest eigenvalue magnitude of S A (S the smoother blocks) by `iters`
// power iterations: w = S A v, lambda = |w| / |v|, v = w / |w|.  Start vector:
// v_i = frac(i * 2654435761 / 2^32) - 1/2 on the free dofs (a fixed
// integer hash, so every implementation starts from the same vector), 0 on
// the fixed ones.
double smoothed_operator_lambda_max(const HostLevel& lv, int nc, int iters) {
  const int nb = nc * nc;
  const int64_t nn = lv.topo.n_nodes, n = nn * nc;
  std::vector<double> v(n), w(n);
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t hsh = ((uint64_t)i * 2654435761ull) & 0xffffffffull;
    const bool fixed = (lv.fixmask[i / nc] >> (i % nc)) & 1;
    v[i] = fixed ? 0.0 : (double)hsh / 4294967296.0 - 0.5;
  }
  auto norm = [&](const std::vector<double>& x) {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) s2 += x[i] * x[i];
    return std::sqrt(s2);
  };
  double lam = 0.0, nv = norm(v);
  for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < nn; ++p) {
      double acc[3] = {0.0, 0.0, 0.0};
      for (int64_t e = lv.A.ptr[p]; e < lv.A.ptr[p + 1]; ++e) {
        const int64_t q = lv.A.col[e];
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j) acc[i] += lv.A.val[e * nb + i * nc + j] * v[q * nc + j];
      }
      for (int i = 0; i < nc; ++i) {
        double t = 0.0;
        for (int j = 0; j < nc; ++j) t += lv.Sinv[p * nb + i * nc + j] * acc[j];
        w[p * nc + i] = t;
      }
    }
    const double nw = norm(w);
    if (!(nw > 0.0) || !(nv > 0.0)) return 1.0;
    lam = nw / nv;
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
    nv = 1.0;
  }
  return lam;
}

}  // namespace

Status read_axes(const mg_mesh& mesh, const LeafSet& s, std::vector<double> axis[3], int* L) {
  for (int d = 0; d < 3; ++d) axis[d].clear();
  *L = -1;
  bool any = false, all = true;
  for (int d = 0; d < mesh.dim; ++d) {
    any = any || mesh.axis[d] != nullptr;
    all = all && mesh.axis[d] != nullptr;
  }
  if (!any) return Status::ok();
  if (!all) return Status::err(MG_ERR_INVALID, "graded mesh: give the axis coordinates of every dimension");
  const int lmax = s.max_level();
  // a hanging node's weights (1/2 per parent) place it at the middle of its
  // edge, which graded lattice coordinates do not: graded meshes are uniform
  for (int32_t l : s.lev)
    if (l != lmax) return Status::err(MG_ERR_INVALID, "graded mesh: every leaf must have the same level");
  for (int d = 0; d < mesh.dim; ++d) {
    const int64_t n = ((int64_t)mesh.macro[d] << lmax) + 1;
    axis[d].assign(mesh.axis[d], mesh.axis[d] + n);
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(axis[d][i]) || (i > 0 && !(axis[d][i] > axis[d][i - 1])))
        return Status::err(MG_ERR_INVALID, "graded mesh: axis coordinates must be finite and strictly increasing");
  }
  *L = lmax;
  return Status::ok();
}

Status build_hierarchy(const mg_mesh& mesh, const mg_problem& prob, const mg_opts& opts, HostHierarchy* H) {
  LeafSet fine;
  Status st = validate_mesh(mesh, &fine);
  if (!st.good()) return st;
  st = read_axes(mesh, fine, H->axis, &H->axis_L);
  if (!st.good()) return st;
  if (H->axis_L >= 0 && prob.kind == MG_OSEEN)
    return Status::err(MG_ERR_INVALID, "graded meshes are not available for OSEEN");
  if (prob.kind < MG_POISSON || prob.kind > MG_OSEEN) return Status::err(MG_ERR_INVALID, "unknown problem kind");
  if (prob.kind == MG_ELASTICITY && mesh.dim != 3) return Status::err(MG_ERR_INVALID, "elasticity needs dim = 3");
  if (prob.kind == MG_TRANSPORT && !(prob.eps > 0)) return Status::err(MG_ERR_INVALID, "transport needs eps > 0");
  if (!(prob.mass >= 0.0) || !std::isfinite(prob.mass)) return Status::err(MG_ERR_INVALID, "mass must be finite and >= 0");
  if (prob.mass != 0.0 && prob.kind == MG_OSEEN)
    return Status::err(MG_ERR_INVALID, "OSEEN takes its mass term from dt, not from mass");
  const bool oseen = prob.kind == MG_OSEEN;
  if (oseen) {
    if (mesh.dim != 2) return Status::err(MG_ERR_INVALID, "oseen needs dim = 2");
    if (!prob.conv) return Status::err(MG_ERR_INVALID, "oseen needs the nodal convection field conv");
    if (!(prob.nu > 0) || !(prob.dt > 0) || !(prob.lps_alpha0 >= 0))
      return Status::err(MG_ERR_INVALID, "oseen needs nu > 0, dt > 0, lps_alpha0 >= 0");
  }
  H->dim = mesh.dim;
  H->nc = (prob.kind == MG_ELASTICITY || oseen) ? 3 : 1;
  for (int d = 0; d < 3; ++d) {
    H->origin[d] = d < mesh.dim ? mesh.origin[d] : 0.0;
    H->extent[d] = d < mesh.dim ? mesh.extent[d] : 1.0;
    H->macro[d] = d < mesh.dim ? mesh.macro[d] : 1;
    if (d < mesh.dim && H->axis_L >= 0) {
      H->origin[d] = H->axis[d].front();
      H->extent[d] = H->axis[d].back() - H->axis[d].front();
    }
  }
  H->prob = prob;
  H->opts = opts;
  int min_level = opts.min_level >= 0 ? opts.min_level : default_min_level(H->macro, H->dim);
  if (oseen) min_level = std::max(min_level, 1);   // patches need a parent cell
  // leaf sets from fine to coarse, then reversed so that [0] is the coarsest
  std::vector<LeafSet> sets;
  sets.push_back(std::move(fine));
  while (opts.max_levels <= 0 || (int)sets.size() < opts.max_levels) {
    LeafSet c;
    if (!coarsen_once(sets.back(), min_level, oseen, &c)) break;
    sets.push_back(std::move(c));
    if ((int)sets.size() >= kMaxLevels) break;
  }
  std::reverse(sets.begin(), sets.end());
  const int nlev = (int)sets.size();
  H->levels.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    HostLevel& lv = H->levels[l];
    lv.leaves = std::move(sets[l]);
    build_topology(lv.leaves, &lv.topo);
  }
  for (int l = nlev - 1; l >= 0; --l) {
    HostLevel& lv = H->levels[l];
    std::vector<double> beta;
    if (oseen) {
      // nodal convection field of this level: injected from the finest nodes
      const Topology& Tf = H->levels[nlev - 1].topo;
      const Topology& T = lv.topo;
      beta.resize(T.n_nodes * 2);
      for (int64_t i = 0; i < T.n_nodes; ++i) {
        int64_t X[3];
        T.lattice_coords(i, X);
        const int64_t k = (X[0] << (Tf.L - T.L)) + (X[1] << (Tf.L - T.L)) * (Tf.ncell[0] + 1);
        const int64_t f = Tf.find(k);
        if (f < 0) return Status::err(MG_ERR_INVALID, "internal: coarse node missing on the finest level");
        beta[2 * i] = prob.conv[2 * f];
        beta[2 * i + 1] = prob.conv[2 * f + 1];
      }
    }
    Status st = assemble_level(*H, lv, beta, l == nlev - 1 ? &H->lift : nullptr);
    if (!st.good()) return st;
  }
  for (size_t l = 1; l < H->levels.size(); ++l) build_transfer(*H, H->levels[l - 1], H->levels[l]);
  // smoother: inverse of the nc x nc diagonal block of every node
  const int nc = H->nc, nb = nc * nc;
  for (HostLevel& lv : H->levels) {
    lv.Sinv.assign(lv.topo.n_nodes * nb, 0.0);
    for (int64_t p = 0; p < lv.topo.n_nodes; ++p) {
      int64_t pos = -1;
      for (int64_t e = lv.A.ptr[p]; e < lv.A.ptr[p + 1]; ++e)
        if (lv.A.col[e] == p) { pos = e; break; }
      std::vector<double> blk(lv.A.val.begin() + pos * nb, lv.A.val.begin() + (pos + 1) * nb), inv;
      if (!invert_dense(nc, blk, inv)) return Status::err(MG_ERR_INVALID, "singular diagonal block");
      std::copy(inv.begin(), inv.end(), lv.Sinv.begin() + p * nb);
    }
  }
  // cell-patch Vanka on the levels >= 1 with at least vanka_rows unknowns
  if (opts.smoother == MG_SMOOTHER_VANKA)
    for (size_t l = 1; l < H->levels.size(); ++l) {
      HostLevel& lv = H->levels[l];
      if (lv.topo.n_nodes * nc < opts.vanka_rows) continue;
      Status sv = build_vanka(lv, H->dim, nc);
      if (!sv.good()) return sv;
      lv.vanka = true;
      lv.omega = opts.vanka_omega;
    }
  // damping per level: opts.omega when positive; otherwise 0.8 for scalar
  // problems and 1.2 / lambda_max(S_l A_l) for the point-block smoothers
  for (HostLevel& lv : H->levels) {
    if (lv.vanka) continue;
    if (opts.omega > 0) lv.omega = opts.omega;
    else if (nc == 1 && H->axis_L < 0) lv.omega = 0.8;
    // point-block smoothers, and scalar levels of graded meshes (anisotropic
    // boxes push lambda_max(D^-1 A) far above its value on cubes, where the
    // fixed 0.8 diverges): from the estimate
    else lv.omega = 1.2 / smoothed_operator_lambda_max(lv, nc, 20);
    if (!(lv.omega > 0) || !std::isfinite(lv.omega)) return Status::err(MG_ERR_INVALID, "smoother damping estimate failed");
  }
  // coarse level: explicit inverse of A_0 (LU / Gauss-Jordan with pivoting)
  {
    const HostLevel& c = H->levels[0];
    const int64_t n = c.topo.n_nodes * nc;
    if (n > 8192) return Status::err(MG_ERR_INVALID, "coarse level too large for the dense solve");
    std::vector<double> M(n * n, 0.0);
    for (int64_t p = 0; p < c.topo.n_nodes; ++p)
      for (int64_t e = c.A.ptr[p]; e < c.A.ptr[p + 1]; ++e)
        for (int i = 0; i < nc; ++i)
          for (int j = 0; j < nc; ++j) M[(p * nc + i) * n + c.A.col[e] * nc + j] = c.A.val[e * nb + i * nc + j];
    // pure Neumann Poisson problem (no prescribed dof, no mass term): A_0 is
    // singular with the constants as its null space.  For a compatible
    // right-hand side (orthogonal to the constants, as every restricted
    // residual of a compatible problem is: P reproduces constants) the
    // inverse of A_0 + a 1 1^T (any a > 0) returns the solution orthogonal to
    // the constants, the pseudo-inverse solution.
    bool neumann = H->prob.kind == MG_POISSON && H->prob.mass == 0.0;
    for (uint8_t f : c.fixmask) neumann = neumann && f == 0;
    if (neumann) {
      double tr = 0.0;
      for (int64_t i = 0; i < n; ++i) tr += M[i * n + i];
      const double a = tr / ((double)n * (double)n);
      for (auto& v : M) v += a;
    }
    if (!invert_dense(n, M, H->coarse_inv)) return Status::err(MG_ERR_INVALID, "singular coarse matrix");
  }
  assemble_load(*H, H->levels.back(), &H->load);
  const HostLevel& f = H->levels.back();
  H->n_free = 0;
  for (int64_t p = 0; p < f.topo.n_nodes; ++p)
    for (int c = 0; c < nc; ++c) H->n_free += ((f.fixmask[p] >> c) & 1) ? 0 : 1;
  return Status::ok();
}

}  // namespace mgi
