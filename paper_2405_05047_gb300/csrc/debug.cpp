// Host-only inspection entry points (include/mg_debug.h): build the same host
// hierarchy as mg_setup and expose its matrices without any GPU.
#include <cstring>
#include <memory>

#include "../../include/mg_debug.h"
#include "device.h"

using namespace mgi;

struct mg_host_hier {
  HostHierarchy H;
  std::vector<BlockCSR> sinv;   // smoother blocks as block-diagonal matrices
  std::vector<BlockCSR> hmat;   // H per level
};

extern "C" {

int mg_host_build(const mg_mesh* mesh, const mg_problem* prob, const mg_opts* opts_in, mg_host_hier** out) {
  if (!mesh || !prob || !out) return MG_ERR_INVALID;
  mg_opts opts;
  if (opts_in) opts = *opts_in;
  else mg_default_opts(&opts);
  auto h = std::make_unique<mg_host_hier>();
  Status st = build_hierarchy(*mesh, *prob, opts, &h->H);
  if (!st.good()) return fail(st.code, st.msg);
  const int nc = h->H.nc, nb = nc * nc;
  for (const HostLevel& lv : h->H.levels) {
    BlockCSR S;
    S.n = S.m = lv.topo.n_nodes;
    S.nc = nc;
    S.ptr.resize(S.n + 1);
    S.col.resize(S.n);
    for (int64_t i = 0; i <= S.n; ++i) S.ptr[i] = i;
    for (int64_t i = 0; i < S.n; ++i) S.col[i] = i;
    S.val = lv.Sinv;
    h->sinv.push_back(std::move(S));
    BlockCSR Hm;
    Hm.n = Hm.m = lv.topo.n_nodes;
    Hm.nc = 1;
    Hm.ptr = lv.topo.con_ptr;
    Hm.col = lv.topo.con_node;
    Hm.val = lv.topo.con_w;
    h->hmat.push_back(std::move(Hm));
  }
  (void)nb;
  *out = h.release();
  return MG_OK;
}

int mg_host_levels(const mg_host_hier* h) { return h ? (int)h->H.levels.size() : MG_ERR_INVALID; }

int mg_host_level(const mg_host_hier* h, int level, int which, int64_t* n, int64_t* m, int* nc, int64_t* nnzb,
                  const int64_t** ptr, const int64_t** col, const double** val) {
  if (!h || level < 0 || level >= (int)h->H.levels.size()) return MG_ERR_INVALID;
  const HostLevel& lv = h->H.levels[level];
  const BlockCSR* M = nullptr;
  switch (which) {
    case 0: M = &lv.A; break;
    case 1: M = &lv.P; break;
    case 2: M = &lv.R; break;
    case 3: M = &h->H.load; break;
    case 4: M = &h->sinv[level]; break;
    case 5: M = &h->hmat[level]; break;
    case 6: M = &h->H.lift; break;
    case 7: M = &lv.Sv; break;
    default: return MG_ERR_INVALID;
  }
  *n = M->n; *m = M->m; *nc = M->nc; *nnzb = M->nnzb();
  *ptr = M->ptr.data(); *col = M->col.data(); *val = M->val.data();
  return MG_OK;
}

int mg_host_nodes(const mg_host_hier* h, int level, const uint8_t** fixmask, int64_t* n_nodes) {
  if (!h || level < 0 || level >= (int)h->H.levels.size()) return MG_ERR_INVALID;
  *fixmask = h->H.levels[level].fixmask.data();
  *n_nodes = h->H.levels[level].topo.n_nodes;
  return MG_OK;
}

int mg_host_omega(const mg_host_hier* h, int level, double* omega) {
  if (!h || !omega || level < 0 || level >= (int)h->H.levels.size()) return MG_ERR_INVALID;
  *omega = h->H.levels[level].omega;
  return MG_OK;
}

int mg_host_coarse_inverse(const mg_host_hier* h, int64_t* n, const double** inv) {
  if (!h) return MG_ERR_INVALID;
  *n = h->H.levels[0].topo.n_nodes * h->H.nc;
  *inv = h->H.coarse_inv.data();
  return MG_OK;
}

int mg_host_free(mg_host_hier* h) {
  delete h;
  return MG_OK;
}

}  // extern "C"
