// Internal structures of the GB300 multigrid library (host setup + device).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mg.h"

namespace mgi {

constexpr int kSlice = 32;          // SELL slice height (rows per warp)
constexpr int kMaxLevels = 32;

struct Status {
  int code = MG_OK;
  std::string msg;
  static Status ok() { return {}; }
  static Status err(int c, std::string m) { return {c, std::move(m)}; }
  bool good() const { return code == MG_OK; }
};

// ----------------------------------------------------------------- host side
struct LeafSet {
  int dim = 2;
  int macro[3] = {1, 1, 1};
  std::vector<int32_t> lev;   // n
  std::vector<int32_t> anc;   // n * dim
  size_t size() const { return lev.size(); }
  int max_level() const;
};

// Node set of one leaf set: lexicographic lattice numbering, hanging constraints.
struct Topology {
  int dim = 2;
  int L = 0;                        // lattice level (finest leaf level)
  int64_t ncell[3] = {1, 1, 1};     // lattice cells per axis
  int64_t n_nodes = 0;
  std::vector<int64_t> key;         // sorted lexicographic lattice keys
  std::vector<int64_t> cell_node;   // n_cells * 2^dim (x fastest)
  std::vector<uint8_t> hanging;     // 1 = hanging node
  std::vector<uint8_t> hang_kind;   // parents before chain resolution (2 or 4)
  // constraint of every node: regular -> (self, 1); hanging -> parents, weights
  std::vector<int64_t> con_ptr;
  std::vector<int64_t> con_node;
  std::vector<double> con_w;
  void lattice_coords(int64_t node, int64_t X[3]) const;
  int64_t find(int64_t k) const;    // node index of a lattice key or -1
};

// Block CSR on nodes (nc x nc dense blocks, row-major inside a block).
struct BlockCSR {
  int64_t n = 0;                    // block rows
  int64_t m = 0;                    // block columns
  int nc = 1;
  std::vector<int64_t> ptr;
  std::vector<int64_t> col;
  std::vector<double> val;          // nnzb * nc * nc
  int64_t nnzb() const { return (int64_t)col.size(); }
};

struct HostLevel {
  LeafSet leaves;
  Topology topo;
  BlockCSR A;                       // condensed level operator
  std::vector<uint8_t> fixmask;     // per node: bit c = dof c fixed (hanging or Dirichlet)
  BlockCSR P;                       // scalar (nc=1): prolongation from level-1 (rows: this level)
  BlockCSR R;                       // scalar: restriction to level-1 (rows: coarse nodes)
  std::vector<double> Sinv;         // n * nc * nc smoother blocks (inverse diagonal blocks)
  double omega = 0.8;               // damping of the smoother on this level
  bool vanka = false;               // cell-patch Vanka smoother (Sv) instead of Jacobi
  BlockCSR Sv;                      // Vanka matrix W sum_T P_T A_T^-1 P_T^T
};

struct HostHierarchy {
  int dim = 2, nc = 1;
  double origin[3] = {0, 0, 0}, extent[3] = {1, 1, 1};
  int macro[3] = {1, 1, 1};
  // graded geometry (mg_mesh.axis): node coordinates along each axis at the
  // finest lattice level axis_L; empty: uniform boxes
  std::vector<double> axis[3];
  int axis_L = -1;
  mg_problem prob{};
  mg_opts opts{};
  std::vector<HostLevel> levels;    // [0] = coarsest
  BlockCSR load;                    // finest: b = load * f  (scalar, rows regular nodes)
  BlockCSR lift;                    // finest: (H^T A H)[free rows, Dirichlet columns]
  std::vector<double> coarse_inv;   // dense (n0 nc)^2 inverse of A_0, row-major
  int64_t n_free = 0;
};

Status validate_mesh(const mg_mesh& mesh, LeafSet* out);
// Graded geometry of a mesh (mg_mesh.axis) at the finest leaf level *L
// (-1 and empty arrays for a uniform mesh).
Status read_axes(const mg_mesh& mesh, const LeafSet& s, std::vector<double> axis[3], int* L);
Status build_hierarchy(const mg_mesh& mesh, const mg_problem& prob, const mg_opts& opts, HostHierarchy* H);
void build_topology(const LeafSet& leaves, Topology* T);
bool coarsen_once(const LeafSet& fine, int min_level, bool patch, LeafSet* coarse);
Status mesh_patches(const LeafSet& s, const Topology& T, std::vector<int64_t>* nodes, std::vector<int32_t>* clev);
int default_min_level(const int macro[3], int dim);

}  // namespace mgi
