// C-ABI entry points (include/mg.h) and the serving scheduler.
//
// Serving: requests are solves on resident hierarchies.  A scheduler thread
// keeps up to `max_slots` solves in flight, each on its own CUDA stream with
// its own workspace, so requests that arrive while others run are admitted as
// soon as a slot and HBM budget for a workspace are free, and their work
// overlaps on the device (continuous batching).  Workspaces are pooled per
// hierarchy; the budget counts every device byte of the context.  Every solve
// is deterministic (fixed-order reductions, fixed grids), so a request's
// result does not depend on what else runs.
#include <cxxabi.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "device.h"

using namespace mgi;

#define CU(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct ServeRequest {
  uint64_t ticket = 0;
  mg_hier* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 1e-8;
  int max_it = 100;
  int prec = MG_MIXED_FP32;
  int state = 0;            // 0 queued, 1 running, 2 finished
  int status = MG_PENDING;
  mg_stats stats{};
  Workspace* ws = nullptr;
  cudaStream_t stream = nullptr;
  int batchable = -1;       // -1 unknown, 0 solved alone, 1 solved in a batched launch
  std::chrono::steady_clock::time_point t_submit, t_start, t_end;
};

// Requests solved by one batched launch on a stream of its own.
struct ServeBatch {
  BatchRun* run = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<std::shared_ptr<ServeRequest>> reqs;
};

namespace {

// A workspace for a serving request: an idle pooled one, or a new one if the
// budget allows (nullptr otherwise).
Workspace* acquire_ws(mg_hier* h, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lk(h->pool_mu);
    if (!h->pool.empty()) {
      Workspace* w = h->pool.back();
      h->pool.pop_back();
      return w;
    }
  }
  mg_ctx* c = h->ctx;
  if (c->budget && c->used + h->ws_bytes > c->budget) return nullptr;
  {
    std::lock_guard<std::mutex> lk(h->pool_mu);
    if (h->serve_cap > 0 && (int)h->all_ws.size() >= h->serve_cap) return nullptr;   // wait for a reserved one
  }
  Workspace* w = nullptr;
  if (ws_create(h, false, s, &w) != MG_OK) return nullptr;
  std::lock_guard<std::mutex> lk(h->pool_mu);
  h->all_ws.push_back(w);
  return w;
}

void release_ws(mg_hier* h, Workspace* w) {
  std::lock_guard<std::mutex> lk(h->pool_mu);
  h->pool.push_back(w);
}

void finish(mg_ctx* c, const std::shared_ptr<ServeRequest>& r, int status) {
  r->t_end = std::chrono::steady_clock::now();
  r->stats.setup_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
  r->status = status;
  r->state = 2;
  if (r->ws) release_ws(r->h, r->ws);
  r->ws = nullptr;
  if (r->stream) c->free_streams.push_back(r->stream);
  r->stream = nullptr;
}

void serve_worker(mg_ctx* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (!c->stop) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < c->running.size();) {
      auto r = c->running[i];
      const cudaError_t q = cudaEventQuery(r->ws->ev1);
      if (q != cudaSuccess && q != cudaErrorNotReady) {   // the device reported an error: never completes
        cudaGetLastError();
        fail(MG_ERR_CUDA, std::string("serving solve: ") + cudaGetErrorString(q));
        finish(c, r, MG_ERR_CUDA);
        c->running.erase(c->running.begin() + i);
        progress = true;
        continue;
      }
      if (q == cudaSuccess) {
        int rc = solve_check(r->h, *r->ws, r->stream, &r->stats);
        if (rc == MG_PENDING) { ++i; continue; }
        finish(c, r, rc);
        c->running.erase(c->running.begin() + i);
        progress = true;
      } else {
        ++i;
      }
    }
    // batched launches that completed
    for (size_t i = 0; i < c->batches.size();) {
      auto B = c->batches[i];
      const cudaError_t q = cudaEventQuery(B->run->done);
      if (q == cudaErrorNotReady) { ++i; continue; }
      std::vector<mg_stats> st(B->reqs.size());
      if (q == cudaSuccess) {
        batch_collect(*B->run, st.data());
      } else {                                            // the device reported an error
        cudaGetLastError();
        fail(MG_ERR_CUDA, std::string("serving batch: ") + cudaGetErrorString(q));
        for (auto& x : st) x.status = MG_ERR_CUDA;
      }
      for (size_t k = 0; k < B->reqs.size(); ++k) {
        B->reqs[k]->stats = st[k];
        finish(c, B->reqs[k], st[k].status);
      }
      c->free_runs.push_back(B->run);
      c->free_streams.push_back(B->stream);
      c->batches.erase(c->batches.begin() + i);
      progress = true;
    }
    // the queued requests that fit the batched kernel (first precision found)
    // go out together as one launch, which takes one slot
    if (c->serve_batch > 0 && (int)(c->running.size() + c->batches.size()) < c->max_slots) {
      std::vector<std::shared_ptr<ServeRequest>> grp;
      for (auto& r : c->queue) {
        if ((int)grp.size() >= c->serve_batch) break;
        if (r->batchable < 0) r->batchable = batch_check(r->h, r->prec) == MG_OK ? 1 : 0;
        if (r->batchable == 1 && (grp.empty() || r->prec == grp[0]->prec)) grp.push_back(r);
      }
      if ((int)grp.size() < c->serve_batch_min) grp.clear();   // too few: they take the graph path
      for (auto& r : grp) c->queue.erase(std::find(c->queue.begin(), c->queue.end(), r));
      if (!grp.empty()) {
        auto B = std::make_shared<ServeBatch>();
        if (c->free_runs.empty()) c->free_runs.push_back(new BatchRun());
        B->run = c->free_runs.back();
        c->free_runs.pop_back();
        if (c->free_streams.empty()) {
          cudaStream_t s;
          cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
          c->free_streams.push_back(s);
        }
        B->stream = c->free_streams.back();
        c->free_streams.pop_back();
        const size_t k = grp.size();
        std::vector<mg_hier*> hs(k);
        std::vector<const double*> bs(k);
        std::vector<double*> xs(k);
        std::vector<double> rt(k);
        std::vector<int> mi(k);
        const auto now = std::chrono::steady_clock::now();
        for (size_t i = 0; i < k; ++i) {
          hs[i] = grp[i]->h; bs[i] = grp[i]->b; xs[i] = grp[i]->x; rt[i] = grp[i]->rtol; mi[i] = grp[i]->max_it;
          grp[i]->state = 1;
          grp[i]->t_start = now;
        }
        int rc = batch_enqueue(c, *B->run, (int)k, hs.data(), bs.data(), xs.data(), rt.data(), mi.data(),
                               grp[0]->prec, B->stream);
        if (rc == MG_OK) {
          B->reqs = std::move(grp);
          c->batches.push_back(B);
        } else {
          // no room for the batch's work vectors: these requests are solved alone
          c->free_runs.push_back(B->run);
          c->free_streams.push_back(B->stream);
          for (size_t i = k; i-- > 0;) {
            grp[i]->batchable = 0;
            grp[i]->state = 0;
            c->queue.push_front(grp[i]);
          }
        }
        progress = true;
      }
    }
    // admissions: first come first served, later requests may pass one that
    // does not fit yet
    for (auto it = c->queue.begin(); it != c->queue.end() && (int)c->running.size() < c->max_slots;) {
      auto r = *it;
      if (c->free_streams.empty()) {
        cudaStream_t s;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        c->free_streams.push_back(s);
      }
      // a pooled workspace was last used on another stream: that solve has
      // finished (its ev1 completed) before the workspace went back to the pool
      Workspace* w = acquire_ws(r->h, c->free_streams.back());
      if (!w) { ++it; continue; }
      r->stream = c->free_streams.back();
      c->free_streams.pop_back();
      r->ws = w;
      r->state = 1;
      r->t_start = std::chrono::steady_clock::now();
      int rc = solve_start(r->h, *w, r->b, false, r->x, false, r->x, false, r->rtol, r->max_it, r->prec, r->stream);
      it = c->queue.erase(it);
      if (rc != MG_OK) finish(c, r, rc);
      else c->running.push_back(r);
      progress = true;
    }
    if (c->running.empty() && c->batches.empty() && c->queue.empty()) {
      c->cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
    } else if (!progress) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

}  // namespace

extern "C" {

const char* mg_strerror(int code) {
  switch (code) {
    case MG_OK: return "ok";
    case MG_PENDING: return "pending";
    case MG_ERR_INVALID: return "invalid argument";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_ADMISSION: return "request exceeds the HBM budget";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_BREAKDOWN: return "Krylov breakdown";
    case MG_ERR_NAN: return "NaN or Inf in a reduction";
    case MG_ERR_TIMEOUT: return "device wait timed out";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

const char* mg_last_error(void) { return last_error(); }

void mg_default_opts(mg_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = -1.0;
  o->min_level = -1;
  o->max_levels = 0;
  o->krylov = MG_KRYLOV_AUTO;
  o->restart = 30;
  o->store_fp64 = 1;
  o->store_fp32 = 1;
  o->launch_mode = 0;
  o->tail_rows = 4096;
  o->store_bf16 = 0;
  o->autotune = 1;
  o->inner_rtol = 0.0;
  o->sell_sigma = -1;
  o->col16 = -1;
  o->row_lanes = -1;
  o->smoother = MG_SMOOTHER_JACOBI;
  o->vanka_rows = 0;
  o->vanka_omega = 1.0;
  o->stage_x = 0;
}

int mg_init(int device, size_t budget, const mg_allocator* alloc, void* stream, mg_ctx** out) {
  if (!out) return fail(MG_ERR_INVALID, "out is NULL");
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(MG_ERR_INVALID, "no such device");
  CU(cudaSetDevice(device));
  int smem_optin = 0;
  CU(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  if (smem_optin < (int)kTailSmemMax + 1024)
    return fail(MG_ERR_INVALID, "device gives a block less shared memory than the staged tail needs");
  mg_ctx* c = new mg_ctx();
  c->device = device;
  c->budget = budget;
  if (alloc && alloc->malloc_fn && alloc->free_fn) { c->alloc = *alloc; c->has_alloc = true; }
  if (stream) c->stream = (cudaStream_t)stream;
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return fail(MG_ERR_CUDA, "stream"); }
    c->own_stream = true;
  }
  *out = c;
  return MG_OK;
}

int mg_destroy(mg_ctx* c) {
  if (!c) return MG_ERR_INVALID;
  if (c->live_hiers.load() > 0) return fail(MG_ERR_INVALID, "context still has hierarchies: mg_free them first");
  {
    std::unique_lock<std::mutex> lk(c->mu);
    c->stop = true;
  }
  c->cv.notify_all();
  if (c->worker.joinable()) c->worker.join();
  for (auto& r : c->running) cudaStreamSynchronize(r->stream);
  for (auto& B : c->batches) {
    cudaStreamSynchronize(B->stream);
    cudaStreamDestroy(B->stream);
    free_run(c, *B->run);
    delete B->run;
  }
  c->batches.clear();
  for (BatchRun* run : c->free_runs) {
    free_run(c, *run);
    delete run;
  }
  c->free_runs.clear();
  for (cudaStream_t s : c->free_streams) cudaStreamDestroy(s);
  for (auto& r : c->running)
    if (r->stream) cudaStreamDestroy(r->stream);
  cudaStreamSynchronize(c->stream);
  free_run(c, c->batch);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return MG_OK;
}

int mg_setup(mg_ctx* ctx, const mg_mesh* mesh, const mg_problem* prob, const mg_opts* opts_in, mg_hier** out) {
  if (!ctx || !mesh || !prob || !out) return fail(MG_ERR_INVALID, "NULL argument");
  CU(cudaSetDevice(ctx->device));
  mg_opts opts;
  if (opts_in) opts = *opts_in;
  else mg_default_opts(&opts);
  if (opts.nu1 < 1 || opts.nu2 < 0 || opts.nu1 > 16 || opts.nu2 > 16) return fail(MG_ERR_INVALID, "nu1 must be >= 1");
  if (std::isnan(opts.omega)) return fail(MG_ERR_INVALID, "omega is NaN");
  if (!(opts.inner_rtol >= 0.0 && opts.inner_rtol < 1.0)) return fail(MG_ERR_INVALID, "inner_rtol must be in [0, 1)");
  if (opts.col16 < -1 || opts.col16 > 1) return fail(MG_ERR_INVALID, "col16 must be -1, 0 or 1");
  if (opts.row_lanes != -1 && opts.row_lanes != 1) return fail(MG_ERR_INVALID, "row_lanes must be -1 or 1");
  if (opts.stage_x < -1 || opts.stage_x > 1) return fail(MG_ERR_INVALID, "stage_x must be -1, 0 or 1");
  if (opts.smoother != MG_SMOOTHER_JACOBI && opts.smoother != MG_SMOOTHER_VANKA)
    return fail(MG_ERR_INVALID, "unknown smoother");
  if (opts.vanka_rows < 0 || !(opts.vanka_omega > 0) || !std::isfinite(opts.vanka_omega))
    return fail(MG_ERR_INVALID, "vanka_rows must be >= 0 and vanka_omega > 0");
  if (opts.sell_sigma < -1 || (opts.sell_sigma > 0 && opts.sell_sigma % 32 != 0))
    return fail(MG_ERR_INVALID, "sell_sigma must be -1, 0 or a positive multiple of 32");
  if (!opts.store_fp64 && !opts.store_fp32 && !opts.store_bf16) return fail(MG_ERR_INVALID, "no precision stored");
  if (!opts.store_fp64 && !(opts.store_fp32 || opts.store_bf16))
    return fail(MG_ERR_INVALID, "no precision stored");
  HostHierarchy H;
  Status st = build_hierarchy(*mesh, *prob, opts, &H);
  if (!st.good()) return fail(st.code, st.msg);
  auto h = std::make_unique<mg_hier>();
  h->ctx = ctx;
  h->dim = H.dim;
  h->nc = H.nc;
  h->nlev = (int)H.levels.size();
  const HostLevel& F = H.levels.back();
  h->n_nodes = F.topo.n_nodes;
  h->n_dofs = h->n_nodes * H.nc;
  h->n_free = H.n_free;
  h->prob = *prob;
  h->prob.conv = nullptr;   // read during setup only
  h->opts = opts;
  // the mesh, for re-assembly with new coefficients (mg_update_problem)
  h->mesh = *mesh;
  h->mesh_lev.assign(mesh->leaf_level, mesh->leaf_level + mesh->n_leaves);
  h->mesh_anc.assign(mesh->leaf_anchor, mesh->leaf_anchor + mesh->n_leaves * mesh->dim);
  for (int d = 0; d < 3; ++d) {
    h->mesh_axis[d] = H.axis[d];
    h->mesh.axis[d] = nullptr;
  }
  h->mesh.leaf_level = nullptr;
  h->mesh.leaf_anchor = nullptr;
  h->has_fp64 = opts.store_fp64 != 0;
  h->has_fp32 = opts.store_fp32 != 0;
  h->has_bf16 = opts.store_bf16 != 0;
  if (method_of(h.get()) == 3) h->gmres_m = std::max(2, std::min(opts.restart > 0 ? opts.restart : 30, 64));
  for (int64_t i = 0; i < h->n_nodes; ++i) h->n_hanging += F.topo.hanging[i];
  h->coords.resize(h->n_nodes * H.dim);
  for (int64_t i = 0; i < h->n_nodes; ++i) {
    int64_t X[3];
    F.topo.lattice_coords(i, X);
    for (int d = 0; d < H.dim; ++d)
      h->coords[i * H.dim + d] = H.axis_L >= 0 ? H.axis[d][X[d] << (H.axis_L - F.topo.L)]
                                               : H.origin[d] + (double)X[d] * (H.extent[d] / (double)F.topo.ncell[d]);
  }
  // admission, first a lower bound without allocating anything (stored
  // values of the level operators); the exact check follows the upload
  {
    size_t lower = 0;
    const int nb = H.nc * H.nc;
    for (const HostLevel& lv : H.levels) {
      if (opts.store_fp64 || &lv == &H.levels.back()) lower += (size_t)lv.A.nnzb() * nb * 8;
      if (opts.store_fp32) lower += (size_t)lv.A.nnzb() * nb * 4;
    }
    if (ctx->budget && ctx->used + lower > ctx->budget)
      return fail(MG_ERR_ADMISSION, "hierarchy needs more than " + std::to_string(lower) + " bytes, budget left " +
                                        std::to_string(ctx->budget - std::min(ctx->budget, (size_t)ctx->used)));
  }
  mg_hier* hp = h.get();
  int rc = upload_hierarchy(hp, H);
  if (rc == MG_OK) {
    hp->ws_bytes = workspace_bytes(hp);
    rc = ws_create(hp, true, ctx->stream, &hp->ws0);
  }
  if (rc == MG_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = fail(MG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc == MG_OK && opts.autotune)
    rc = autotune(hp, hp->has_fp32 ? MG_MIXED_FP32 : (hp->has_bf16 ? MG_MIXED_BF16 : MG_FP64));
  if (rc == MG_OK && ctx->budget && ctx->used > ctx->budget)
    rc = fail(MG_ERR_ADMISSION, "hierarchy and its workspace need " + std::to_string(hp->bytes + hp->ws0->bytes) +
                                    " bytes, over the HBM budget");
  if (rc != MG_OK) {
    free_hierarchy(hp);
    return rc;
  }
  ctx->resident += hp->bytes + hp->ws0->bytes;
  ctx->live_hiers++;
  *out = h.release();
  return MG_OK;
}

int mg_hier_info(const mg_hier* h, mg_info* info) {
  if (!h || !info) return fail(MG_ERR_INVALID, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->dim = h->dim;
  info->nc = h->nc;
  info->levels = h->nlev;
  info->n_nodes = h->n_nodes;
  info->n_dofs = h->n_dofs;
  info->n_free = h->n_free;
  for (int l = 0; l < h->nlev && l < 32; ++l) {
    info->level_nodes[l] = h->level_nodes[l];
    info->level_nnzb[l] = h->level_nnzb[l];
    info->level_rows_nnzb[l] = h->level_real_nnzb[l];
    info->level_col16[l] = h->level_col16[l];
  }
  info->bytes_device = h->bytes + (h->ws0 ? h->ws0->bytes : 0);
  info->bytes_workspace = h->ws_bytes;
  info->tail_levels = h->tail_top > 0 ? h->tail_top + 1 : 0;
  info->tail_cluster = h->tail_cluster;
  info->vcycle_ms = h->tuned_vcycle_ms;
  info->col16_slices = h->col16_slices;
  info->col32_slices = h->col32_slices;
  info->n_hanging = h->n_hanging;
  info->omega = h->L.back().omega;
  for (int l = 0; l < h->nlev && l < 32; ++l) {
    info->level_omega[l] = h->L[l].omega;
    info->level_block_values[l] = h->level_block_values[l];
    info->level_sigma[l] = h->level_sigma[l];
    info->level_lanes[l] = h->L[l].A32.slots ? h->L[l].A32.v.tpr : 1;
    info->level_smoother[l] = h->L[l].vanka ? MG_SMOOTHER_VANKA : MG_SMOOTHER_JACOBI;
    info->level_vanka_nnzb[l] = h->L[l].vanka ? std::max(h->L[l].V32.nnz_real, h->L[l].V64.nnz_real) : 0;
  }
  return MG_OK;
}

int mg_mesh_nodes(const mg_mesh* mesh, int64_t* n_nodes, double* xyz) {
  if (!mesh || !n_nodes) return fail(MG_ERR_INVALID, "NULL argument");
  LeafSet s;
  Status st = validate_mesh(*mesh, &s);
  if (!st.good()) return fail(st.code, st.msg);
  std::vector<double> axis[3];
  int L = -1;
  st = read_axes(*mesh, s, axis, &L);
  if (!st.good()) return fail(st.code, st.msg);
  Topology T;
  build_topology(s, &T);
  *n_nodes = T.n_nodes;
  if (xyz)
    for (int64_t i = 0; i < T.n_nodes; ++i) {
      int64_t X[3];
      T.lattice_coords(i, X);
      for (int d = 0; d < mesh->dim; ++d)
        xyz[i * mesh->dim + d] = L >= 0 ? axis[d][X[d] << (L - T.L)]
                                        : mesh->origin[d] + (double)X[d] * (mesh->extent[d] / (double)T.ncell[d]);
    }
  return MG_OK;
}

int mg_node_coords(const mg_hier* h, double* xyz) {
  if (!h || !xyz) return fail(MG_ERR_INVALID, "NULL argument");
  std::memcpy(xyz, h->coords.data(), h->coords.size() * sizeof(double));
  return MG_OK;
}

int mg_free(mg_hier* h) {
  if (!h) return MG_ERR_INVALID;
  cudaSetDevice(h->ctx->device);
  cudaDeviceSynchronize();
  h->ctx->resident -= h->bytes + (h->ws0 ? h->ws0->bytes : 0);
  h->ctx->live_hiers--;
  free_hierarchy(h);
  delete h;
  return MG_OK;
}

int mg_assemble_rhs(mg_hier* h, const double* f, const double* g, double* b) {
  if (!h || !f || !b) return fail(MG_ERR_INVALID, "NULL argument");
  CU(cudaSetDevice(h->ctx->device));
  cudaStream_t s = h->ctx->stream;
  launch_rhs(h->F.v, h->nc, f, h->fixmask, h->dirmask, g, b, s);
  if (g) launch_lift(h->Lift.v, h->nc, g, b, s);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

static int solve_sync(mg_hier* h, const double* b, bool bh, double* x, bool xh, double rtol, int max_it, int prec,
                      mg_stats* stats) {
  if (!h || !b || !x || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaSetDevice(h->ctx->device));
  cudaStream_t s = h->ctx->stream;
  Workspace& w = *h->ws0;
  rc = solve_start(h, w, b, bh, x, xh, x, xh, rtol, max_it, prec, s);
  while (rc == MG_OK || rc == MG_PENDING) {
    CU(cudaEventSynchronize(w.ev1));
    rc = solve_check(h, w, s, stats);
    if (rc != MG_PENDING) break;
  }
  CU(cudaGetLastError());
  return rc;
}

int mg_time_steps(mg_hier* h, double* theta, const double* f, const double* g, int n_steps, double rtol, int max_it,
                  int prec, mg_stats* steps) {
  if (!h || !theta || n_steps < 0 || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  if (!(h->prob.mass > 0)) return fail(MG_ERR_INVALID, "time stepping needs a problem with mass = 1/dt > 0");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaSetDevice(h->ctx->device));
  cudaStream_t s = h->ctx->stream;
  Workspace& w = *h->ws0;
  const int64_t n = h->n_dofs;
  for (int k = 0; k < n_steps; ++k) {
    // right-hand side of step k+1 straight into the solve's b buffer; the
    // step's nodal load field goes through w.t, which the solve overwrites
    const double* fk = f ? f + (int64_t)k * n : nullptr;
    const double* gk = g ? g + (int64_t)k * n : nullptr;
    launch_step_load(n, h->prob.mass, theta, fk, w.t, s);
    launch_rhs(h->F.v, h->nc, w.t, h->fixmask, h->dirmask, gk, w.bi, s);
    if (gk) launch_lift(h->Lift.v, h->nc, gk, w.bi, s);
    h->launch_count += gk ? 3 : 2;
    mg_stats st{};
    rc = solve_start(h, w, w.bi, false, theta, false, theta, false, rtol, max_it, prec, s);
    while (rc == MG_OK || rc == MG_PENDING) {
      CU(cudaEventSynchronize(w.ev1));
      rc = solve_check(h, w, s, &st);
      if (rc != MG_PENDING) break;
    }
    st.launches += gk ? 3 : 2;
    if (steps) steps[k] = st;
    if (rc != MG_OK) break;
  }
  CU(cudaGetLastError());
  return rc;
}

int mg_time_steps2(mg_hier* h, double* u, double* v, const double* f, const double* g, int n_steps, double dt,
                   double rtol, int max_it, int prec, mg_stats* steps) {
  if (!h || !u || !v || n_steps < 0 || !(dt > 0) || !(rtol > 0) || max_it < 1)
    return fail(MG_ERR_INVALID, "bad argument");
  if (!(std::fabs(h->prob.mass * dt * dt - 1.0) <= 1e-12))
    return fail(MG_ERR_INVALID, "second-order steps need a problem with mass = 1/dt^2");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaSetDevice(h->ctx->device));
  cudaStream_t s = h->ctx->stream;
  Workspace& w = *h->ws0;
  const int64_t n = h->n_dofs;
  const double inv_dt = 1.0 / dt;
  for (int k = 0; k < n_steps; ++k) {
    const double* fk = f ? f + (int64_t)k * n : nullptr;
    const double* gk = g ? g + (int64_t)k * n : nullptr;
    launch_step_load2(n, inv_dt, u, v, fk, w.t, s);   // v now holds -u_{n-1}/dt
    launch_rhs(h->F.v, h->nc, w.t, h->fixmask, h->dirmask, gk, w.bi, s);
    if (gk) launch_lift(h->Lift.v, h->nc, gk, w.bi, s);
    mg_stats st{};
    rc = solve_start(h, w, w.bi, false, u, false, u, false, rtol, max_it, prec, s);
    while (rc == MG_OK || rc == MG_PENDING) {
      CU(cudaEventSynchronize(w.ev1));
      rc = solve_check(h, w, s, &st);
      if (rc != MG_PENDING) break;
    }
    launch_step_velocity(n, inv_dt, u, v, s);           // v = (u_n - u_{n-1}) / dt
    h->launch_count += gk ? 4 : 3;
    st.launches += gk ? 4 : 3;
    if (steps) steps[k] = st;
    if (rc != MG_OK) break;
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return rc;
}

// "k_smooth<float, float, 1, false, 1>" from the kernel's symbol: demangled,
// without the return type, namespace and parameter list.
static void kernel_label(const void* fn, char* out, size_t cap) {
  const char* mangled = nullptr;
  std::string name = "?";
  if (cudaFuncGetName(&mangled, fn) == cudaSuccess && mangled) {
    int st = 0;
    char* dem = abi::__cxa_demangle(mangled, nullptr, nullptr, &st);
    name = (st == 0 && dem) ? dem : mangled;
    std::free(dem);
  }
  const std::string anon = "(anonymous namespace)::";
  for (size_t p; (p = name.find(anon)) != std::string::npos;) name.erase(p, anon.size());
  if (name.compare(0, 5, "void ") == 0) name.erase(0, 5);
  int depth = 0;
  for (size_t i = 0; i < name.size(); ++i) {   // cut at the parameter list
    if (name[i] == '<') ++depth;
    else if (name[i] == '>') --depth;
    else if (name[i] == '(' && depth == 0) {
      name.resize(i);
      break;
    }
  }
  const size_t ns = name.rfind("::", name.find('<'));   // namespace qualifiers
  if (ns != std::string::npos) name.erase(0, ns + 2);
  std::snprintf(out, cap, "%s", name.c_str());
}

int mg_solve_profiled(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats,
                      mg_prof_entry* entries, int cap, int* n_entries) {
  if (!h || !n_entries || cap < 0 || (cap > 0 && !entries)) return fail(MG_ERR_INVALID, "bad argument");
  EventProfiler prof;
  int rc = prof.init(2 * 4096);
  if (rc) return rc;
  LaunchProfiler* prev = t_prof;
  t_prof = &prof;
  rc = solve_sync(h, b, false, x, false, rtol, max_it, prec, stats);
  t_prof = prev;
  if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED && rc != MG_ERR_BREAKDOWN && rc != MG_ERR_NAN) return rc;
  CU(cudaStreamSynchronize(h->ctx->stream));
  prof.collect_direct();
  std::vector<std::pair<std::pair<const void*, int>, std::pair<int64_t, double>>> v(prof.acc.begin(), prof.acc.end());
  std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.second.second > b.second.second; });
  *n_entries = (int)v.size();
  for (int i = 0; i < cap && i < (int)v.size(); ++i) {
    kernel_label(v[i].first.first, entries[i].kernel, sizeof(entries[i].kernel));
    entries[i].level = v[i].first.second;
    entries[i].launches = v[i].second.first;
    entries[i].ms = v[i].second.second;
  }
  return rc;
}

int mg_solve(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats) {
  return solve_sync(h, b, false, x, false, rtol, max_it, prec, stats);
}

int mg_solve_host(mg_hier* h, const double* b_host, double* x_host, double rtol, int max_it, int prec,
                  mg_stats* stats) {
  return solve_sync(h, b_host, true, x_host, true, rtol, max_it, prec, stats);
}

int mg_vcycle(mg_hier* h, const void* r, void* z, int prec) {
  if (!h || !r || !z) return fail(MG_ERR_INVALID, "NULL argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  if (prec == MG_FP64) enqueue_vcycle<double>(h, *h->ws0, h->nlev - 1, (const double*)r, (double*)z, nullptr, s);
  else enqueue_vcycle<float>(h, *h->ws0, h->nlev - 1, (const float*)r, (float*)z, nullptr, s, false,
                             prec == MG_MIXED_BF16);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

// one level operator on the given vectors (shared by mg_apply and mg_time_op)
static int level_op(mg_hier* h, int level, int op, const void* in, const void* in2, void* out, int prec,
                    cudaStream_t s) {
  LevelMats& L = h->L[level];
  LevelVecs& V = h->ws0->lv[level];
  const int nc = h->nc;
  const bool d = prec == MG_FP64;
  const SellView& A32 = prec == MG_MIXED_BF16 ? L.A16.v : L.A32.v;
  switch (op) {
    case MG_OP_MATVEC:
      if (d) launch_matvec<double>(L.A64.v, nc, (const double*)in, (double*)out, nullptr, s);
      else launch_matvec<float>(A32, nc, (const float*)in, (float*)out, nullptr, s);
      return MG_OK;
    case MG_OP_SMOOTH:
      if (!in2) return fail(MG_ERR_INVALID, "smooth needs b");
      if (L.vanka) {      // residual into the level's r buffer, then out = in + w S r
        if (d) {
          launch_residual<double>(L.A64.v, nc, (const double*)in, (const double*)in2, V.r64, nullptr, s);
          launch_vanka<double>(L.V64.v, nc, V.r64, (const double*)in, (double*)out, L.omega, nullptr, s);
        } else {
          launch_residual<float>(A32, nc, (const float*)in, (const float*)in2, V.r32, nullptr, s);
          launch_vanka<float>(L.V32.v, nc, V.r32, (const float*)in, (float*)out, L.omega, nullptr, s);
        }
        return MG_OK;
      }
      if (d) launch_smooth<double>(L.A64.v, nc, (const double*)in, (const double*)in2, L.S64, (double*)out, L.omega, false, nullptr, s);
      else launch_smooth<float>(A32, nc, (const float*)in, (const float*)in2, L.S32, (float*)out, L.omega, false, nullptr, s);
      return MG_OK;
    case MG_OP_RESTRICT:
      if (level == 0 || !in2) return fail(MG_ERR_INVALID, "restrict needs level >= 1 and b");
      if (d) {
        launch_residual<double>(L.A64.v, nc, (const double*)in, (const double*)in2, V.r64, nullptr, s);
        launch_restrict<double>(L.R.t, nc, V.r64, (double*)out, nullptr, nullptr, 0.0, nullptr, s);
      } else {
        launch_residual<float>(A32, nc, (const float*)in, (const float*)in2, V.r32, nullptr, s);
        launch_restrict<float>(L.R.t, nc, V.r32, (float*)out, nullptr, nullptr, 0.0, nullptr, s);
      }
      return MG_OK;
    case MG_OP_PROLONG_ADD:
      if (level == 0 || !in2) return fail(MG_ERR_INVALID, "prolong needs level >= 1 and x");
      if (d) launch_prolong_add<double>(L.P.t, nc, (const double*)in, (const double*)in2, (double*)out, nullptr, s);
      else launch_prolong_add<float>(L.P.t, nc, (const float*)in, (const float*)in2, (float*)out, nullptr, s);
      return MG_OK;
    case MG_OP_COARSE:
      if (level != 0) return fail(MG_ERR_INVALID, "coarse solve is on level 0");
      if (d) launch_coarse<double>(h->coarse_inv, h->coarse_n, (const double*)in, (double*)out, nullptr, s);
      else launch_coarse<float>(h->coarse_inv, h->coarse_n, (const float*)in, (float*)out, nullptr, s);
      return MG_OK;
    default:
      return fail(MG_ERR_INVALID, "unknown op");
  }
}

int mg_apply(mg_hier* h, int level, int op, const void* in, const void* in2, void* out, int prec) {
  if (!h || !in || !out || level < 0 || level >= h->nlev) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  rc = level_op(h, level, op, in, in2, out, prec, s);
  if (rc) return rc;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

int mg_time_op(mg_hier* h, int level, int op, int prec, int reps, double* ms) {
  if (!h || !ms || level < 0 || level >= h->nlev || reps < 1) return fail(MG_ERR_INVALID, "bad argument");
  if (op == MG_OP_COARSE || ((op == MG_OP_RESTRICT || op == MG_OP_PROLONG_ADD) && level == 0))
    return fail(MG_ERR_INVALID, "operator not timed on this level");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  Workspace& w = *h->ws0;
  if (op == MG_TIME_VCYCLE || op == MG_TIME_VCYCLE_GRAPH) {
    LevelVecs& V = w.lv[level];
    const bool bf = prec == MG_MIXED_BF16;
    auto cycle = [&]() {
      if (prec == MG_FP64) enqueue_vcycle<double>(h, w, level, V.b64, V.t64, nullptr, s);
      else enqueue_vcycle<float>(h, w, level, V.b32, V.t32, nullptr, s, false, bf);
    };
    cycle();                          // warm (also the first-use setup of every kernel)
    CU(cudaStreamSynchronize(s));
    float t = 0;
    if (op == MG_TIME_VCYCLE) {
      CU(cudaEventRecord(w.ev0, s));
      for (int i = 0; i < reps; ++i) cycle();
      CU(cudaEventRecord(w.ev1, s));
    } else {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int i = 0; i < reps; ++i) cycle();
      CU(cudaStreamEndCapture(s, &g));
      cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
      CU(cudaGraphLaunch(ge, s));     // warm
      CU(cudaEventRecord(w.ev0, s));
      CU(cudaGraphLaunch(ge, s));
      CU(cudaEventRecord(w.ev1, s));
      CU(cudaEventSynchronize(w.ev1));
      cudaGraphExecDestroy(ge);
    }
    CU(cudaEventSynchronize(w.ev1));
    CU(cudaEventElapsedTime(&t, w.ev0, w.ev1));
    *ms = (double)t / reps;
    CU(cudaGetLastError());
    return MG_OK;
  }
  LevelVecs& V = w.lv[level];
  const bool d = prec == MG_FP64;
  const void* x = d ? (const void*)V.o64 : (const void*)V.o32;
  const void* b = d ? (const void*)V.b64 : (const void*)V.b32;
  void* y = d ? (void*)V.t64 : (void*)V.t32;
  void* yc = nullptr;
  const void* xc = nullptr;
  if (level > 0) {
    yc = d ? (void*)w.lv[level - 1].b64 : (void*)w.lv[level - 1].b32;
    xc = d ? (const void*)w.lv[level - 1].o64 : (const void*)w.lv[level - 1].o32;
  }
  auto once = [&]() -> int {
    if (op == MG_OP_RESTRICT) return level_op(h, level, op, x, b, yc, prec, s);
    if (op == MG_OP_PROLONG_ADD) return level_op(h, level, op, xc, x, y, prec, s);
    return level_op(h, level, op, x, b, y, prec, s);
  };
  if ((rc = once())) return rc;
  CU(cudaEventRecord(w.ev0, s));
  for (int i = 0; i < reps; ++i) once();
  CU(cudaEventRecord(w.ev1, s));
  CU(cudaEventSynchronize(w.ev1));
  float t = 0;
  CU(cudaEventElapsedTime(&t, w.ev0, w.ev1));
  *ms = (double)t / reps;
  CU(cudaGetLastError());
  return MG_OK;
}

int64_t mg_launch_count(const mg_hier* h) { return h ? (int64_t)h->launch_count : 0; }

int mg_tune(mg_hier* h, int prec, int tail_rows, int cluster) {
  if (!h || (tail_rows >= 0 && (cluster < -16 || cluster > 16))) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  if (tail_rows < 0) return autotune(h, prec);
  return set_tail(h, tail_rows, cluster);
}

int mg_submit(mg_ctx* c, mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec,
              uint64_t* ticket) {
  if (!c || !h || !b || !x || !ticket || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  if (h->ctx != c) return fail(MG_ERR_INVALID, "hierarchy belongs to another context");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  // a request can never run if one more workspace does not fit next to the
  // resident hierarchies
  if (c->budget && (size_t)c->resident + h->ws_bytes > c->budget)
    return fail(MG_ERR_ADMISSION, "a solve workspace of " + std::to_string(h->ws_bytes) +
                                      " bytes never fits the HBM budget next to the resident hierarchies");
  auto r = std::make_shared<ServeRequest>();
  r->h = h; r->b = b; r->x = x; r->rtol = rtol; r->max_it = max_it; r->prec = prec;
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->worker_started) {
      c->worker = std::thread(serve_worker, c);
      c->worker_started = true;
    }
    r->ticket = c->next_ticket++;
    c->tickets[r->ticket] = r;
    c->queue.push_back(r);
    *ticket = r->ticket;
  }
  c->cv.notify_one();
  return MG_OK;
}

int mg_poll(mg_ctx* c, uint64_t ticket, mg_stats* stats) {
  if (!c) return fail(MG_ERR_INVALID, "NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->tickets.find(ticket);
  if (it == c->tickets.end()) return fail(MG_ERR_INVALID, "unknown ticket");
  auto r = it->second;
  if (r->state != 2) return MG_PENDING;
  if (stats) {
    *stats = r->stats;
    stats->status = r->status;
  }
  int st = r->status;
  c->tickets.erase(it);
  return st;
}

int mg_cancel(mg_ctx* c, uint64_t ticket) {
  if (!c) return fail(MG_ERR_INVALID, "NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->tickets.find(ticket);
  if (it == c->tickets.end()) return fail(MG_ERR_INVALID, "unknown ticket");
  auto r = it->second;
  if (r->state != 0) return fail(MG_ERR_INVALID, "request already running or finished");
  for (auto q = c->queue.begin(); q != c->queue.end(); ++q)
    if ((*q)->ticket == ticket) { c->queue.erase(q); break; }
  r->state = 2;
  r->status = MG_ERR_CANCELLED;
  return MG_OK;
}

int mg_serve_reserve(mg_ctx* c, mg_hier* h, int slots, int prec) {
  if (!c || !h || h->ctx != c || slots < 1 || slots > 256) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  CU(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(c->mu);      // the scheduler does not touch the pool meanwhile
  const int method = method_of(h);
  int have;
  {
    std::lock_guard<std::mutex> pk(h->pool_mu);
    have = (int)h->all_ws.size();
  }
  for (; have < slots; ++have) {
    if (c->budget && c->used + h->ws_bytes > c->budget)
      return fail(MG_ERR_ADMISSION, "reserved solve slots exceed the HBM budget");
    Workspace* w = nullptr;
    if ((rc = ws_create(h, true, c->stream, &w))) return rc;
    std::lock_guard<std::mutex> pk(h->pool_mu);
    h->all_ws.push_back(w);
    h->pool.push_back(w);
  }
  std::vector<Workspace*> ws;
  {
    std::lock_guard<std::mutex> pk(h->pool_mu);
    ws = h->pool;
    h->serve_cap = std::max(h->serve_cap, slots);
  }
  for (Workspace* w : ws) {       // idle workspaces: build their solve graphs now, not on the first request
    SolveGraph* g = nullptr;
    if (h->opts.launch_mode != 1 && (rc = get_graph(h, *w, method, prec, &g))) return rc;
  }
  CU(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

int mg_update_problem(mg_hier* h, const mg_problem* prob) {
  if (!h || !prob) return fail(MG_ERR_INVALID, "NULL argument");
  const mg_problem& o = h->prob;
  if (prob->kind != o.kind || prob->pin_origin != o.pin_origin ||
      std::memcmp(prob->dirichlet_mask, o.dirichlet_mask, sizeof(o.dirichlet_mask)) != 0)
    return fail(MG_ERR_INVALID, "the problem kind, Dirichlet faces and pin must stay the same");
  mg_ctx* c = h->ctx;
  {
    // no request of h queued or in flight
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& r : c->queue)
      if (r->h == h) return fail(MG_ERR_INVALID, "the hierarchy has serving requests queued");
    for (auto& r : c->running)
      if (r->h == h) return fail(MG_ERR_INVALID, "the hierarchy has serving requests running");
    for (auto& B : c->batches)
      for (auto& r : B->reqs)
        if (r->h == h) return fail(MG_ERR_INVALID, "the hierarchy has serving requests running");
  }
  CU(cudaSetDevice(c->device));
  mg_mesh m = h->mesh;
  m.leaf_level = h->mesh_lev.data();
  m.leaf_anchor = h->mesh_anc.data();
  for (int d = 0; d < 3; ++d) m.axis[d] = h->mesh_axis[d].empty() ? nullptr : h->mesh_axis[d].data();
  HostHierarchy H;
  Status st = build_hierarchy(m, *prob, h->opts, &H);
  if (!st.good()) return fail(st.code, st.msg);
  // no synchronous batched solve (which reads the images being rebuilt) and
  // no solve of h on the context's stream meanwhile
  std::lock_guard<std::mutex> bk(c->batch_mu);
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaStreamSynchronize(c->stream));
  int rc = update_hierarchy(h, H);
  if (rc) return rc;
  h->prob = *prob;
  h->prob.conv = nullptr;
  return MG_OK;
}

int mg_solve_batch(mg_ctx* c, int count, mg_hier* const* h, const double* const* b, double* const* x, double rtol,
                   int max_it, int prec, mg_stats* stats) {
  return solve_batch(c, count, h, b, x, rtol, max_it, prec, stats);
}

int mg_batch_fits(mg_hier* h, int prec) {
  if (!h) return fail(MG_ERR_INVALID, "NULL hierarchy");
  return batch_check(h, prec) == MG_OK ? 1 : 0;
}

int mg_serve_batching(mg_ctx* c, int max_batch, int min_batch) {
  if (!c || max_batch < 0 || max_batch > 65536 || min_batch < 1)
    return fail(MG_ERR_INVALID, "max_batch must be in [0, 65536] and min_batch >= 1");
  std::lock_guard<std::mutex> lk(c->mu);
  c->serve_batch = max_batch;
  c->serve_batch_min = min_batch;
  return MG_OK;
}

int mg_serve_config(mg_ctx* c, int max_slots) {
  if (!c || max_slots < 1 || max_slots > 256) return fail(MG_ERR_INVALID, "max_slots must be in [1, 256]");
  std::lock_guard<std::mutex> lk(c->mu);
  c->max_slots = max_slots;
  return MG_OK;
}

}  // extern "C"
