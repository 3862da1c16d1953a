// Device hierarchy, V-cycle and Krylov drivers, C-ABI entry points.
//
// The V-cycle follows Algorithm "Geometric multigrid solver" of the paper
// (Sec. 2.2): Step 0 coarse solve, Step 1 pre-smoothing, Step 2 restriction of
// the residual, Step 3 recursion with zero initial guess, Step 4 prolongation
// and correction, Step 5 post-smoothing.  It preconditions CG (flexible,
// Polak-Ribiere) or BiCGStab (Sec. 4.1.5: multigrid as preconditioner of a
// Krylov method).  All Krylov scalars stay on the device; one Krylov
// iteration is captured into the body of a CUDA-graph `while` node whose
// condition is set by the convergence test on the device, so a whole solve is
// one graph launch and only the final status crosses to the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"

using namespace mgi;

// ------------------------------------------------------------------ context
struct ServeRequest;

struct mg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mg_allocator alloc{};
  bool has_alloc = false;
  size_t budget = 0;
  std::atomic<size_t> used{0};
  std::string last_error;
  // serving
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  bool worker_started = false;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<ServeRequest>> queue;
  std::map<uint64_t, std::shared_ptr<ServeRequest>> tickets;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CU(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Alloc {
  void* p = nullptr;
  size_t bytes = 0;
};

struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  int method = 0, prec = 0;
  int64_t launches_per_iter = 0;
};

}  // namespace

struct SellBuf {
  SellView v;
  TransferView t;
  int64_t nnz_real = 0;
  int64_t slots = 0;
};

struct LevelBufs {
  int64_t n = 0;                         // nodes
  SellBuf A64, A32, P, R;
  double* S64 = nullptr;
  float* S32 = nullptr;
  // V-cycle vectors per precision: rhs, out, tmp, residual
  double* b64 = nullptr; double* o64 = nullptr; double* t64 = nullptr; double* r64 = nullptr;
  float* b32 = nullptr; float* o32 = nullptr; float* t32 = nullptr; float* r32 = nullptr;
};

struct mg_hier {
  mg_ctx* ctx = nullptr;
  int dim = 2, nc = 1, nlev = 0;
  int64_t n_nodes = 0, n_dofs = 0, n_free = 0, n_hanging = 0;
  mg_problem prob{};
  mg_opts opts{};
  std::vector<double> coords;            // finest nodes, external order
  std::vector<int64_t> level_nodes, level_nnzb, level_real_nnzb;
  std::vector<Alloc> allocs;
  size_t bytes = 0;
  std::vector<LevelBufs> L;              // [0] coarsest
  double* coarse_inv = nullptr;          // (n0 nc)^2
  int64_t coarse_n = 0;
  SellBuf F;                             // load matrix (finest)
  SellBuf Hc;                            // hanging rows of H (finest)
  uint8_t* fixmask = nullptr;            // finest, per node
  bool has_fp64 = true, has_fp32 = true;
  // Krylov workspace (finest, FP64)
  double *xi = nullptr, *bi = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *rhat = nullptr,
         *sv = nullptr, *t = nullptr, *ph = nullptr, *shat = nullptr;
  float *r32 = nullptr, *ph32 = nullptr, *sh32 = nullptr;
  Partials part;
  KrylovState* st = nullptr;
  KrylovState* st_host = nullptr;        // pinned
  int nred = 1;
  std::vector<SolveGraph> graphs;
  int tail_top = 0;                      // levels 0..tail_top run in the single-CTA tail kernel
  TailParams tail64, tail32;
  GmresView gm;                          // GMRES workspace (allocated when opts.krylov == MG_GMRES)
  double* vcur = nullptr;                // FP64 V-cycle input of the current Arnoldi vector
  int64_t launch_count = 0;              // kernels enqueued (host-side count)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::mutex solve_mu;                   // one solve at a time per hierarchy
};

namespace {

void* dev_alloc(mg_hier* h, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  mg_ctx* c = h->ctx;
  if (c->has_alloc) p = c->alloc.malloc_fn(bytes, c->alloc.user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (!p) return nullptr;
  h->allocs.push_back({p, bytes});
  h->bytes += bytes;
  c->used += bytes;
  return p;
}

void free_all(mg_hier* h) {
  mg_ctx* c = h->ctx;
  for (auto& a : h->allocs) {
    if (c->has_alloc) c->alloc.free_fn(a.p, c->alloc.user);
    else cudaFree(a.p);
    c->used -= a.bytes;
  }
  h->allocs.clear();
  h->bytes = 0;
}

size_t rnd(size_t b) { return ((b + 255) & ~(size_t)255) + (b == 0 ? 256 : 0); }

// SELL-C packing of a block CSR matrix.
template <typename VT>
void pack_sell(const BlockCSR& M, std::vector<int64_t>& sptr, std::vector<int32_t>& col, std::vector<VT>& val) {
  const int nb = M.nc * M.nc;
  const int64_t n = M.n, ns = (n + kSlice - 1) / kSlice;
  sptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t w = 0;
    for (int64_t r = s * kSlice; r < std::min(n, (s + 1) * kSlice); ++r) w = std::max(w, M.ptr[r + 1] - M.ptr[r]);
    sptr[s + 1] = sptr[s] + kSlice * w;
  }
  const int64_t slots = sptr[ns];
  col.assign(slots, 0);
  val.assign(slots * nb, VT(0));
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t w = (sptr[s + 1] - sptr[s]) / kSlice;
    for (int lane = 0; lane < kSlice; ++lane) {
      const int64_t r = s * kSlice + lane;
      const int64_t len = r < n ? M.ptr[r + 1] - M.ptr[r] : 0;
      for (int64_t j = 0; j < w; ++j) {
        const int64_t g = sptr[s] + kSlice * j, o = g + lane;
        if (j < len) {
          col[o] = (int32_t)M.col[M.ptr[r] + j];
          for (int e = 0; e < nb; ++e) val[g * nb + (int64_t)e * kSlice + lane] = (VT)M.val[(M.ptr[r] + j) * nb + e];
        } else {
          col[o] = (int32_t)(r < n ? std::min<int64_t>(r, M.m - 1) : 0);
        }
      }
    }
  }
}

size_t sell_bytes(const BlockCSR& M, int vbytes) {
  const int64_t n = M.n, ns = (n + kSlice - 1) / kSlice;
  int64_t slots = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t w = 0;
    for (int64_t r = s * kSlice; r < std::min(n, (s + 1) * kSlice); ++r) w = std::max(w, M.ptr[r + 1] - M.ptr[r]);
    slots += kSlice * w;
  }
  return rnd((ns + 1) * 8) + rnd(slots * 4) + rnd(slots * M.nc * M.nc * vbytes);
}

template <typename VT>
int upload_sell(mg_hier* h, const BlockCSR& M, SellBuf* out, bool transfer) {
  std::vector<int64_t> sptr;
  std::vector<int32_t> col;
  std::vector<VT> val;
  pack_sell<VT>(M, sptr, col, val);
  void* dp = dev_alloc(h, sptr.size() * 8);
  void* dc = dev_alloc(h, col.size() * 4);
  void* dv = dev_alloc(h, val.size() * sizeof(VT));
  if (!dp || !dc || !dv) return fail(MG_ERR_OOM, "device allocation failed");
  CU(cudaMemcpy(dp, sptr.data(), sptr.size() * 8, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(dc, col.data(), col.size() * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(dv, val.data(), val.size() * sizeof(VT), cudaMemcpyHostToDevice));
  out->v.sptr = out->t.sptr = (const int64_t*)dp;
  out->v.col = out->t.col = (const int32_t*)dc;
  out->v.val = dv;
  out->t.w = (const float*)dv;
  out->v.n = out->t.n = M.n;
  out->v.nslices = out->t.nslices = (int64_t)sptr.size() - 1;
  out->slots = (int64_t)col.size();
  out->nnz_real = M.nnzb();
  (void)transfer;
  return MG_OK;
}

template <typename T>
T* alloc_vec(mg_hier* h, int64_t n) {
  return (T*)dev_alloc(h, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
}

// ------------------------------------------------------------------ V-cycle
template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const TailParams& tail(mg_hier* h) { return h->tail64; }
  static const SellView& A(LevelBufs& l) { return l.A64.v; }
  static const double* S(LevelBufs& l) { return l.S64; }
  static double* b(LevelBufs& l) { return l.b64; }
  static double* o(LevelBufs& l) { return l.o64; }
  static double* t(LevelBufs& l) { return l.t64; }
  static double* r(LevelBufs& l) { return l.r64; }
};
template <>
struct Prec<float> {
  static const TailParams& tail(mg_hier* h) { return h->tail32; }
  static const SellView& A(LevelBufs& l) { return l.A32.v; }
  static const float* S(LevelBufs& l) { return l.S32; }
  static float* b(LevelBufs& l) { return l.b32; }
  static float* o(LevelBufs& l) { return l.o32; }
  static float* t(LevelBufs& l) { return l.t32; }
  static float* r(LevelBufs& l) { return l.r32; }
};

// z = GMG(l, 0, b): the V-cycle of Algorithm "Geometric multigrid solver".
// first_done: the first pre-smoothing sweep (from x = 0) was already written
// into its buffer by the restriction kernel of the finer level.
template <typename T>
void enqueue_vcycle(mg_hier* h, int l, const T* b, T* out, const int* done, cudaStream_t s, bool first_done = false) {
  const int nc = h->nc;
  if (l == 0) {                                                  // Step 0
    launch_coarse<T>(h->coarse_inv, h->coarse_n, b, out, done, s);
    h->launch_count++;
    return;
  }
  LevelBufs& L = h->L[l];
  LevelBufs& C = h->L[l - 1];
  if (l <= h->tail_top) {                                        // small levels: one CTA
    launch_tail<T>(Prec<T>::tail(h), nc, b, out, first_done, done, s);
    h->launch_count++;
    return;
  }
  const int nu1 = h->opts.nu1, nu2 = h->opts.nu2, ns = nu1 + nu2;
  auto bufof = [&](LevelBufs& X, T* o, int k) -> T* { return ((ns - 1 - k) % 2 == 0) ? o : Prec<T>::t(X); };
  const double om = h->opts.omega;
  T* cur = nullptr;
  for (int k = 0; k < nu1; ++k) {                                // Step 1
    T* dst = bufof(L, out, k);
    if (!(k == 0 && first_done)) {
      launch_smooth<T>(Prec<T>::A(L), nc, cur, b, Prec<T>::S(L), dst, om, k == 0, done, s);
      h->launch_count++;
    }
    cur = dst;
  }
  launch_residual<T>(Prec<T>::A(L), nc, cur, b, Prec<T>::r(L), done, s);   // Step 2
  const bool fuse = l - 1 > 0;
  T* cfirst = fuse ? bufof(C, Prec<T>::o(C), 0) : nullptr;
  launch_restrict<T>(L.R.t, nc, Prec<T>::r(L), Prec<T>::b(C), Prec<T>::S(C), cfirst, om, done, s);
  h->launch_count += 2;
  enqueue_vcycle<T>(h, l - 1, Prec<T>::b(C), Prec<T>::o(C), done, s, fuse);   // Step 3
  T* pdst = nu2 == 0 ? out : cur;                                          // Step 4
  launch_prolong_add<T>(L.P.t, nc, Prec<T>::o(C), cur, pdst, done, s);
  cur = pdst;
  h->launch_count++;
  for (int k = nu1; k < ns; ++k) {                               // Step 5
    T* dst = bufof(L, out, k);
    launch_smooth<T>(Prec<T>::A(L), nc, cur, b, Prec<T>::S(L), dst, om, false, done, s);
    cur = dst;
    h->launch_count++;
  }
}

// ------------------------------------------------------------------ Krylov
enum { M_CG = 1, M_BICG = 2, M_GMRES = 3 };

int method_of(const mg_hier* h) {
  int k = h->opts.krylov;
  if (k == MG_KRYLOV_AUTO) k = (h->prob.kind == MG_TRANSPORT) ? MG_BICGSTAB : MG_CG;
  return k == MG_BICGSTAB ? M_BICG : (k == MG_GMRES ? M_GMRES : M_CG);
}

// One Krylov iteration (the body of the graph's while node).  The last kernel
// of the iteration runs the convergence test and sets the while condition.
void enqueue_iteration(mg_hier* h, int method, int prec, unsigned long long cond, cudaStream_t s) {
  const int nc = h->nc;
  const int fine = h->nlev - 1;
  const int64_t n = h->n_dofs;
  const SellView& A = h->L[fine].A64.v;
  const int* done = &h->st->done;
  const bool mixed = prec != MG_FP64;
  if (method == M_CG) {
    PVec z;
    if (mixed) {
      launch_to_f32(n, h->r, h->r32, h->st, s);
      enqueue_vcycle<float>(h, fine, h->r32, h->ph32, done, s);
      z.f = h->ph32;
      h->launch_count++;
    } else {
      enqueue_vcycle<double>(h, fine, h->r, h->z, done, s);
      z.d = h->z;
    }
    launch_cg_dots(n, z, h->r, h->q, h->part, h->st, s);
    launch_cg_update_p(n, z, h->p, h->st, s);
    PVec pp;
    pp.d = h->p;
    launch_spmv_dot(A, nc, pp, nullptr, h->q, h->part, Q_PQ, h->st, s);
    launch_cg_update_xr(n, h->p, h->q, h->xi, h->r, h->part, h->st, cond, s);
    h->launch_count += 4;
  } else if (method == M_GMRES) {
    // one Arnoldi step of flexible GMRES(m); cycle end and restart are gated
    // on the device (gm_end / gm_j)
    PVec z;
    if (mixed) { enqueue_vcycle<float>(h, fine, h->r32, h->ph32, done, s); z.f = h->ph32; }
    else { enqueue_vcycle<double>(h, fine, h->vcur, h->z, done, s); z.d = h->z; }
    launch_gm_spmv(A, nc, z, h->q, h->gm, h->st, s);
    launch_gm_orth(n, h->q, h->gm, h->st, 0, h->part, s);
    launch_gm_orth(n, h->q, h->gm, h->st, 1, h->part, s);
    launch_gm_givens(h->gm, h->st, s);
    launch_gm_next(n, h->q, mixed ? h->r32 : nullptr, mixed ? nullptr : h->vcur, h->gm, h->st, s);
    launch_gm_update_x(n, h->xi, h->gm, h->st, s);
    launch_gm_residual(A, nc, h->xi, h->bi, h->r, h->part, h->st, cond, s);
    launch_gm_start(n, h->r, mixed ? h->r32 : nullptr, mixed ? nullptr : h->vcur, h->gm, h->st, s);
    h->launch_count += 1 + 3 * 2 + 1 + 2 + 1 + 1 + 1;
  } else {
    // in mixed mode bicg_p / bicg_s also write the FP32 preconditioner input
    launch_bicg_p(n, h->r, h->t /* v */, h->p, mixed ? h->r32 : nullptr, h->st, s);
    PVec ph;
    if (mixed) { enqueue_vcycle<float>(h, fine, h->r32, h->ph32, done, s); ph.f = h->ph32; }
    else { enqueue_vcycle<double>(h, fine, h->p, h->ph, done, s); ph.d = h->ph; }
    launch_spmv_dot(A, nc, ph, h->rhat, h->t /* v */, h->part, Q_RHV, h->st, s);
    launch_bicg_s(n, h->r, h->t, h->sv, mixed ? h->r32 : nullptr, h->st, s);
    PVec sh;
    if (mixed) { enqueue_vcycle<float>(h, fine, h->r32, h->sh32, done, s); sh.f = h->sh32; }
    else { enqueue_vcycle<double>(h, fine, h->sv, h->shat, done, s); sh.d = h->shat; }
    launch_spmv_2dots(A, nc, sh, h->sv, h->q /* t */, h->part, h->st, s);
    launch_bicg_x(n, ph, sh, h->sv, h->q, h->rhat, h->xi, h->r, h->part, h->st, cond, s);
    h->launch_count += 5;
  }
}

int build_graph(mg_hier* h, int method, int prec, SolveGraph* out) {
  cudaStream_t cs;
  CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  CU(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle handle;
  CU(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CU(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int64_t before = h->launch_count;
  enqueue_iteration(h, method, prec, (unsigned long long)handle, cs);
  out->launches_per_iter = h->launch_count - before;
  h->launch_count = before;
  cudaGraph_t captured;
  cudaError_t e = cudaStreamEndCapture(cs, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return fail(MG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&out->exec, g, 0);
  cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  out->method = method;
  out->prec = prec;
  return MG_OK;
}

int get_graph(mg_hier* h, int method, int prec, SolveGraph** g) {
  for (auto& x : h->graphs)
    if (x.method == method && x.prec == prec) { *g = &x; return MG_OK; }
  SolveGraph ng;
  int rc = build_graph(h, method, prec, &ng);
  if (rc) return rc;
  h->graphs.push_back(ng);
  *g = &h->graphs.back();
  return MG_OK;
}

int check_prec(const mg_hier* h, int prec) {
  if (prec == MG_FP64 && !h->has_fp64) return fail(MG_ERR_INVALID, "hierarchy built without FP64 level matrices");
  if (prec == MG_MIXED_FP32 && !h->has_fp32) return fail(MG_ERR_INVALID, "hierarchy built without FP32 level matrices");
  if (prec != MG_FP64 && prec != MG_MIXED_FP32) return fail(MG_ERR_INVALID, "unsupported precision");
  return MG_OK;
}

// Device part of a solve on the internal buffers (bi, xi already set).
int solve_device(mg_hier* h, double rtol, int max_it, int prec, cudaStream_t s, mg_stats* stats) {
  const int method = method_of(h);
  const int nc = h->nc;
  const int fine = h->nlev - 1;
  const SellView& A = h->L[fine].A64.v;
  SolveGraph* g = nullptr;
  SolveGraph direct;   // direct launches are counted as they are enqueued
  if (h->opts.launch_mode == 1) {
    g = &direct;
  } else {
    int rc = get_graph(h, method, prec, &g);
    if (rc) return rc;
  }
  int64_t launches = 0;
  CU(cudaEventRecord(h->ev0, s));
  launch_norm_init(h->n_nodes, nc, h->fixmask, h->bi, h->part, h->st, rtol, max_it, s);
  launches += 1;
  int total_iters = 0;
  int status = MG_OK;
  double rel = 0.0;
  for (int round = 0; round < 4; ++round) {
    launch_residual_norm(A, nc, h->xi, h->bi, h->r, h->part, h->st, 1, s);
    launches += 1;
    if (method == M_GMRES) {
      if (!h->gm.V) return fail(MG_ERR_INVALID, "hierarchy set up without GMRES workspace (opts.krylov)");
      launch_gm_start(h->n_dofs, h->r, prec != MG_FP64 ? h->r32 : nullptr, prec != MG_FP64 ? nullptr : h->vcur,
                      h->gm, h->st, s);
      launches += 1;
    } else if (method == M_BICG) {
      // rhat = r0, (rhat, r) = (r, r)
      CU(cudaMemcpyAsync(h->rhat, h->r, h->n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(cudaMemcpyAsync(&h->st->red[Q_RHR], &h->st->red[Q_RR], sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(cudaMemsetAsync(h->t, 0, h->n_dofs * sizeof(double), s));
    } else {
      CU(cudaMemsetAsync(h->q, 0, h->n_dofs * sizeof(double), s));
    }
    if (h->opts.launch_mode == 1) {
      // direct launches: one iteration at a time, status read back after each
      const int64_t before = h->launch_count;
      for (int it = 0; it < max_it + 1; ++it) {
        CU(cudaMemcpyAsync(h->st_host, h->st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (h->st_host->done) break;
        enqueue_iteration(h, method, prec, 0ull, s);
      }
      launches += h->launch_count - before;
      h->launch_count = before;
    } else {
      CU(cudaGraphLaunch(g->exec, s));
    }
    // true residual of the final iterate
    launch_residual_norm(A, nc, h->xi, h->bi, h->r, h->part, h->st, 0, s);
    launches += 1;
    CU(cudaMemcpyAsync(h->st_host, h->st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const KrylovState& S = *h->st_host;
    const double rr = S.red[Q_RR];
    int it_round = S.iter;
    launches += (int64_t)it_round * g->launches_per_iter + (it_round == 0 ? 0 : 0);
    total_iters = it_round;
    rel = std::sqrt(rr) / S.bnorm;
    if (S.status == -6) { status = MG_ERR_NAN; break; }
    if (S.status == -5) { status = MG_ERR_BREAKDOWN; break; }
    if (rel <= rtol) { status = MG_OK; break; }
    if (S.iter >= max_it) { status = MG_ERR_NOT_CONVERGED; break; }
    // recursive residual converged but the true one did not: restart from
    // the true residual with the iteration count kept
    KrylovState fix = S;
    fix.done = 0;
    fix.status = 0;
    fix.restart_pos = fix.iter;
    fix.gm_j = 0;
    fix.gm_end = 0;
    CU(cudaMemcpyAsync(h->st, &fix, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    status = MG_ERR_NOT_CONVERGED;
  }
  CU(cudaEventRecord(h->ev1, s));
  CU(cudaEventSynchronize(h->ev1));
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  if (stats) {
    stats->status = status;
    stats->iters = total_iters;
    stats->vcycles = total_iters * (method == M_BICG ? 2 : 1);
    stats->precision = prec;
    stats->rel_res = rel;
    stats->solve_ms = ms;
    stats->launches = launches;
  }
  h->launch_count += launches;
  return status;
}

}  // namespace

// ------------------------------------------------------------------ serving
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
  std::chrono::steady_clock::time_point t_submit, t_start;
};

static int solve_impl(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats,
                      cudaStream_t s) {
  const int64_t n = h->n_dofs;
  CU(cudaMemcpyAsync(h->bi, b, n * 8, cudaMemcpyDeviceToDevice, s));
  launch_copy_fixed(h->n_nodes, h->nc, h->fixmask, h->bi, x, h->xi, s);
  int rc = solve_device(h, rtol, max_it, prec, s, stats);
  if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED && rc != MG_ERR_NAN && rc != MG_ERR_BREAKDOWN) return rc;
  launch_fill_hanging(h->Hc.t, h->nc, h->xi, s);
  CU(cudaMemcpyAsync(x, h->xi, n * 8, cudaMemcpyDeviceToDevice, s));
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return rc;
}


static void serve_worker(mg_ctx* c) {
  cudaSetDevice(c->device);
  while (true) {
    std::shared_ptr<ServeRequest> r;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      c->cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      if (c->stop) return;
      r = c->queue.front();
      c->queue.pop_front();
      r->state = 1;
      r->t_start = std::chrono::steady_clock::now();
    }
    mg_stats st{};
    int rc;
    {
      std::lock_guard<std::mutex> lk(r->h->solve_mu);
      rc = solve_impl(r->h, r->b, r->x, r->rtol, r->max_it, r->prec, &st, c->stream);
    }
    std::lock_guard<std::mutex> lk(c->mu);
    st.setup_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    r->stats = st;
    r->status = rc;
    r->state = 2;
  }
}

// ------------------------------------------------------------------ C ABI
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

const char* mg_last_error(void) { return g_last_error.c_str(); }

void mg_default_opts(mg_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.8;
  o->min_level = -1;
  o->max_levels = 0;
  o->krylov = MG_KRYLOV_AUTO;
  o->restart = 30;
  o->store_fp64 = 1;
  o->store_fp32 = 1;
  o->launch_mode = 0;
  o->tail_rows = 4096;
}

int mg_init(int device, size_t budget, const mg_allocator* alloc, void* stream, mg_ctx** out) {
  if (!out) return fail(MG_ERR_INVALID, "out is NULL");
  int ndev = 0;
  CU(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(MG_ERR_INVALID, "no such device");
  CU(cudaSetDevice(device));
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
  {
    std::unique_lock<std::mutex> lk(c->mu);
    c->stop = true;
  }
  c->cv.notify_all();
  if (c->worker.joinable()) c->worker.join();
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
  if (!(opts.omega > 0.0)) return fail(MG_ERR_INVALID, "omega must be positive");
  if (!opts.store_fp64 && !opts.store_fp32) return fail(MG_ERR_INVALID, "no precision stored");
  HostHierarchy H;
  Status st = build_hierarchy(*mesh, *prob, opts, &H);
  if (!st.good()) return fail(st.code, st.msg);
  const int nc = H.nc, nb = nc * nc;
  const int nlev = (int)H.levels.size();
  const HostLevel& F = H.levels.back();
  const int64_t nn = F.topo.n_nodes, n = nn * nc;
  // ---- admission: total device bytes of hierarchy + workspace
  size_t need = 0;
  for (int l = 0; l < nlev; ++l) {
    const HostLevel& lv = H.levels[l];
    const int64_t m = lv.topo.n_nodes * nc;
    if (opts.store_fp64) need += sell_bytes(lv.A, 8) + rnd(lv.topo.n_nodes * nb * 8) + 4 * rnd(m * 8);
    if (opts.store_fp32) need += sell_bytes(lv.A, 4) + rnd(lv.topo.n_nodes * nb * 4) + 4 * rnd(m * 4);
    if (l > 0) need += sell_bytes(lv.P, 4) + sell_bytes(lv.R, 4);
  }
  {
    int kk = opts.krylov;
    if (kk == MG_KRYLOV_AUTO) kk = prob->kind == MG_TRANSPORT ? MG_BICGSTAB : MG_CG;
    if (kk == MG_GMRES) {
      const int64_t m = std::max(2, std::min(opts.restart > 0 ? opts.restart : 30, 64));
      need += rnd((m + 1) * n * 8) + (opts.store_fp64 ? rnd(m * n * 8) : 0) + (opts.store_fp32 ? rnd(m * n * 4) : 0) +
              rnd(n * 8) + rnd((m + 1) * kMaxRedBlocks * 8) + 8 * rnd((m + 1) * m * 8);
    }
  }
  need += rnd(H.coarse_inv.size() * 8) + sell_bytes(H.load, 8) + rnd(nn) + 16 * rnd(n * 8) + 3 * rnd(n * 4) +
          rnd(Q_NUM * kMaxRedBlocks * 8) + rnd(sizeof(KrylovState));
  if (ctx->budget && ctx->used + need > ctx->budget)
    return fail(MG_ERR_ADMISSION, "hierarchy needs " + std::to_string(need) + " bytes, budget left " +
                                      std::to_string(ctx->budget - std::min(ctx->budget, (size_t)ctx->used)));
  mg_hier* h = new mg_hier();
  h->ctx = ctx;
  h->dim = H.dim;
  h->nc = nc;
  h->nlev = nlev;
  h->n_nodes = nn;
  h->n_dofs = n;
  h->n_free = H.n_free;
  h->prob = *prob;
  h->opts = opts;
  h->has_fp64 = opts.store_fp64 != 0;
  h->has_fp32 = opts.store_fp32 != 0;
  for (int64_t i = 0; i < nn; ++i) h->n_hanging += F.topo.hanging[i];
  h->coords.resize(nn * H.dim);
  for (int64_t i = 0; i < nn; ++i) {
    int64_t X[3];
    F.topo.lattice_coords(i, X);
    for (int d = 0; d < H.dim; ++d)
      h->coords[i * H.dim + d] = H.origin[d] + (double)X[d] * (H.extent[d] / (double)F.topo.ncell[d]);
  }
  auto bail = [&](int rc) {
    free_all(h);
    delete h;
    return rc;
  };
  h->L.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    HostLevel& lv = H.levels[l];
    LevelBufs& B = h->L[l];
    B.n = lv.topo.n_nodes;
    const int64_t m = B.n * nc;
    h->level_nodes.push_back(B.n);
    h->level_real_nnzb.push_back(lv.A.nnzb());
    int rc;
    if (opts.store_fp64) {
      if ((rc = upload_sell<double>(h, lv.A, &B.A64, false))) return bail(rc);
      B.S64 = alloc_vec<double>(h, B.n * nb);
      if (!B.S64) return bail(fail(MG_ERR_OOM, "alloc"));
      CU(cudaMemcpy(B.S64, lv.Sinv.data(), B.n * nb * 8, cudaMemcpyHostToDevice));
      B.b64 = alloc_vec<double>(h, m); B.o64 = alloc_vec<double>(h, m);
      B.t64 = alloc_vec<double>(h, m); B.r64 = alloc_vec<double>(h, m);
      if (!B.b64 || !B.o64 || !B.t64 || !B.r64) return bail(fail(MG_ERR_OOM, "alloc"));
    }
    if (opts.store_fp32) {
      if ((rc = upload_sell<float>(h, lv.A, &B.A32, false))) return bail(rc);
      std::vector<float> s32(lv.Sinv.begin(), lv.Sinv.end());
      B.S32 = alloc_vec<float>(h, B.n * nb);
      if (!B.S32) return bail(fail(MG_ERR_OOM, "alloc"));
      CU(cudaMemcpy(B.S32, s32.data(), B.n * nb * 4, cudaMemcpyHostToDevice));
      B.b32 = alloc_vec<float>(h, m); B.o32 = alloc_vec<float>(h, m);
      B.t32 = alloc_vec<float>(h, m); B.r32 = alloc_vec<float>(h, m);
      if (!B.b32 || !B.o32 || !B.t32 || !B.r32) return bail(fail(MG_ERR_OOM, "alloc"));
    }
    h->level_nnzb.push_back(opts.store_fp64 ? B.A64.slots : B.A32.slots);
    if (l > 0) {
      if ((rc = upload_sell<float>(h, lv.P, &B.P, true))) return bail(rc);
      if ((rc = upload_sell<float>(h, lv.R, &B.R, true))) return bail(rc);
    }
    // release host copies of what is now on the device
    if (l < nlev - 1) { lv.A = BlockCSR(); lv.leaves = LeafSet(); }
    lv.P = BlockCSR();
    lv.R = BlockCSR();
  }
  h->coarse_n = H.levels[0].topo.n_nodes * nc;
  h->coarse_inv = alloc_vec<double>(h, h->coarse_n * h->coarse_n);
  if (!h->coarse_inv) return bail(fail(MG_ERR_OOM, "alloc"));
  CU(cudaMemcpy(h->coarse_inv, H.coarse_inv.data(), H.coarse_inv.size() * 8, cudaMemcpyHostToDevice));
  int rc;
  if ((rc = upload_sell<double>(h, H.load, &h->F, false))) return bail(rc);
  {
    // hanging rows of H on the finest level (regular rows empty)
    BlockCSR Hm;
    Hm.n = Hm.m = nn;
    Hm.nc = 1;
    Hm.ptr.assign(nn + 1, 0);
    for (int64_t i = 0; i < nn; ++i)
      Hm.ptr[i + 1] = Hm.ptr[i] + (F.topo.hanging[i] ? F.topo.con_ptr[i + 1] - F.topo.con_ptr[i] : 0);
    for (int64_t i = 0; i < nn; ++i)
      if (F.topo.hanging[i])
        for (int64_t o = F.topo.con_ptr[i]; o < F.topo.con_ptr[i + 1]; ++o) {
          Hm.col.push_back(F.topo.con_node[o]);
          Hm.val.push_back(F.topo.con_w[o]);
        }
    if ((rc = upload_sell<float>(h, Hm, &h->Hc, true))) return bail(rc);
  }
  h->fixmask = (uint8_t*)dev_alloc(h, nn);
  if (!h->fixmask) return bail(fail(MG_ERR_OOM, "alloc"));
  CU(cudaMemcpy(h->fixmask, F.fixmask.data(), nn, cudaMemcpyHostToDevice));
  double** vecs[] = {&h->xi, &h->bi, &h->r, &h->p, &h->q, &h->z, &h->rhat, &h->sv, &h->t, &h->ph, &h->shat};
  for (double** v : vecs) {
    *v = alloc_vec<double>(h, n);
    if (!*v) return bail(fail(MG_ERR_OOM, "alloc"));
    CU(cudaMemset(*v, 0, n * 8));
  }
  float** v32[] = {&h->r32, &h->ph32, &h->sh32};
  for (float** v : v32) {
    *v = alloc_vec<float>(h, n);
    if (!*v) return bail(fail(MG_ERR_OOM, "alloc"));
  }
  if (method_of(h) == M_GMRES) {
    const int m = std::max(2, std::min(opts.restart > 0 ? opts.restart : 30, 64));
    GmresView& G = h->gm;
    G.m = m;
    G.H = alloc_vec<double>(h, (int64_t)(m + 1) * m);
    G.cs = alloc_vec<double>(h, m);
    G.sn = alloc_vec<double>(h, m);
    G.g = alloc_vec<double>(h, m + 1);
    G.hv = alloc_vec<double>(h, m + 1);
    G.y = alloc_vec<double>(h, m);
    G.zs = alloc_vec<double>(h, m);
    G.part = alloc_vec<double>(h, (int64_t)(m + 1) * kMaxRedBlocks);
    G.V = alloc_vec<double>(h, (int64_t)(m + 1) * n);
    if (opts.store_fp64) G.Z64 = alloc_vec<double>(h, (int64_t)m * n);
    if (opts.store_fp32) G.Z32 = alloc_vec<float>(h, (int64_t)m * n);
    h->vcur = alloc_vec<double>(h, n);
    if (!G.H || !G.V || !G.part || !h->vcur || (opts.store_fp64 && !G.Z64) || (opts.store_fp32 && !G.Z32))
      return bail(fail(MG_ERR_OOM, "alloc"));
  }
  h->part.p = alloc_vec<double>(h, Q_NUM * kMaxRedBlocks);
  h->st = (KrylovState*)dev_alloc(h, sizeof(KrylovState));
  if (!h->part.p || !h->st) return bail(fail(MG_ERR_OOM, "alloc"));
  CU(cudaMemset(h->part.p, 0, Q_NUM * kMaxRedBlocks * 8));
  CU(cudaMemset(h->st, 0, sizeof(KrylovState)));
  CU(cudaMallocHost(&h->st_host, sizeof(KrylovState)));
  CU(cudaEventCreate(&h->ev0));
  CU(cudaEventCreate(&h->ev1));
  h->nred = grid_for_rows(((nn + 31) / 32) * 32);
  // tail: the largest prefix of levels (from the coarsest) with <= tail_rows dofs
  h->tail_top = 0;
  if (opts.tail_rows > 0)
    for (int l = 1; l < nlev && l < kTailMax; ++l)
      if (h->L[l].n * nc <= opts.tail_rows) h->tail_top = l;
      else break;
  for (int pi = 0; pi < 2; ++pi) {
    TailParams& P = pi == 0 ? h->tail64 : h->tail32;
    const bool d = pi == 0;
    if (d ? !opts.store_fp64 : !opts.store_fp32) continue;
    P.nt = h->tail_top + 1;
    P.nu1 = opts.nu1;
    P.nu2 = opts.nu2;
    P.omega = opts.omega;
    P.cinv = h->coarse_inv;
    P.cn = h->coarse_n;
    for (int l = 0; l <= h->tail_top; ++l) {
      LevelBufs& B = h->L[l];
      TailLevel& T = P.lv[l];
      T.A = d ? B.A64.v : B.A32.v;
      T.P = B.P.t;
      T.R = B.R.t;
      T.S = d ? (const void*)B.S64 : (const void*)B.S32;
      T.b = d ? (void*)B.b64 : (void*)B.b32;
      T.o = d ? (void*)B.o64 : (void*)B.o32;
      T.t = d ? (void*)B.t64 : (void*)B.t32;
      T.r = d ? (void*)B.r64 : (void*)B.r32;
    }
  }
  CU(cudaDeviceSynchronize());
  *out = h;
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
  }
  info->bytes_device = h->bytes;
  info->n_hanging = h->n_hanging;
  info->omega = h->opts.omega;
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
  cudaStreamSynchronize(h->ctx->stream);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  free_all(h);
  delete h;
  return MG_OK;
}

int mg_assemble_rhs(mg_hier* h, const double* f, double* b) {
  if (!h || !f || !b) return fail(MG_ERR_INVALID, "NULL argument");
  cudaStream_t s = h->ctx->stream;
  launch_rhs(h->F.v, h->nc, f, h->fixmask, b, s);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

int mg_solve(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats) {
  if (!h || !b || !x || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaSetDevice(h->ctx->device));
  return solve_impl(h, b, x, rtol, max_it, prec, stats, h->ctx->stream);
}

int mg_solve_host(mg_hier* h, const double* b_host, double* x_host, double rtol, int max_it, int prec,
                  mg_stats* stats) {
  if (!h || !b_host || !x_host || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  CU(cudaSetDevice(h->ctx->device));
  cudaStream_t s = h->ctx->stream;
  const int64_t n = h->n_dofs;
  // stage through the Krylov workspace: bi <- b, p <- x0 (p is rewritten by the solve)
  CU(cudaMemcpyAsync(h->bi, b_host, n * 8, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(h->p, x_host, n * 8, cudaMemcpyHostToDevice, s));
  launch_copy_fixed(h->n_nodes, h->nc, h->fixmask, h->bi, h->p, h->xi, s);
  rc = solve_device(h, rtol, max_it, prec, s, stats);
  if (rc != MG_OK && rc != MG_ERR_NOT_CONVERGED && rc != MG_ERR_NAN && rc != MG_ERR_BREAKDOWN) return rc;
  launch_fill_hanging(h->Hc.t, h->nc, h->xi, s);
  CU(cudaMemcpyAsync(x_host, h->xi, n * 8, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return rc;
}

int mg_vcycle(mg_hier* h, const void* r, void* z, int prec) {
  if (!h || !r || !z) return fail(MG_ERR_INVALID, "NULL argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  if (prec == MG_FP64) enqueue_vcycle<double>(h, h->nlev - 1, (const double*)r, (double*)z, nullptr, s);
  else enqueue_vcycle<float>(h, h->nlev - 1, (const float*)r, (float*)z, nullptr, s);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

int mg_apply(mg_hier* h, int level, int op, const void* in, const void* in2, void* out, int prec) {
  if (!h || !in || !out || level < 0 || level >= h->nlev) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  LevelBufs& L = h->L[level];
  const int nc = h->nc;
  const bool d = prec == MG_FP64;
  switch (op) {
    case MG_OP_MATVEC:
      if (d) launch_matvec<double>(L.A64.v, nc, (const double*)in, (double*)out, nullptr, s);
      else launch_matvec<float>(L.A32.v, nc, (const float*)in, (float*)out, nullptr, s);
      break;
    case MG_OP_SMOOTH:
      if (!in2) return fail(MG_ERR_INVALID, "smooth needs b");
      if (d) launch_smooth<double>(L.A64.v, nc, (const double*)in, (const double*)in2, L.S64, (double*)out, h->opts.omega, false, nullptr, s);
      else launch_smooth<float>(L.A32.v, nc, (const float*)in, (const float*)in2, L.S32, (float*)out, h->opts.omega, false, nullptr, s);
      break;
    case MG_OP_RESTRICT:
      if (level == 0 || !in2) return fail(MG_ERR_INVALID, "restrict needs level >= 1 and b");
      if (d) {
        launch_residual<double>(L.A64.v, nc, (const double*)in, (const double*)in2, L.r64, nullptr, s);
        launch_restrict<double>(L.R.t, nc, L.r64, (double*)out, nullptr, nullptr, 0.0, nullptr, s);
      } else {
        launch_residual<float>(L.A32.v, nc, (const float*)in, (const float*)in2, L.r32, nullptr, s);
        launch_restrict<float>(L.R.t, nc, L.r32, (float*)out, nullptr, nullptr, 0.0, nullptr, s);
      }
      break;
    case MG_OP_PROLONG_ADD:
      if (level == 0 || !in2) return fail(MG_ERR_INVALID, "prolong needs level >= 1 and x");
      if (d) launch_prolong_add<double>(L.P.t, nc, (const double*)in, (const double*)in2, (double*)out, nullptr, s);
      else launch_prolong_add<float>(L.P.t, nc, (const float*)in, (const float*)in2, (float*)out, nullptr, s);
      break;
    case MG_OP_COARSE:
      if (level != 0) return fail(MG_ERR_INVALID, "coarse solve is on level 0");
      if (d) launch_coarse<double>(h->coarse_inv, h->coarse_n, (const double*)in, (double*)out, nullptr, s);
      else launch_coarse<float>(h->coarse_inv, h->coarse_n, (const float*)in, (float*)out, nullptr, s);
      break;
    default:
      return fail(MG_ERR_INVALID, "unknown op");
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

int mg_submit(mg_ctx* c, mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec,
              uint64_t* ticket) {
  if (!c || !h || !b || !x || !ticket || !(rtol > 0) || max_it < 1) return fail(MG_ERR_INVALID, "bad argument");
  if (h->ctx != c) return fail(MG_ERR_INVALID, "hierarchy belongs to another context");
  int rc = check_prec(h, prec);
  if (rc) return rc;
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
  if (stats) *stats = r->stats;
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

int64_t mg_launch_count(const mg_hier* h) { return h ? h->launch_count : 0; }

int mg_time_op(mg_hier* h, int level, int op, int prec, int reps, double* ms) {
  if (!h || !ms || level < 0 || level >= h->nlev || reps < 1) return fail(MG_ERR_INVALID, "bad argument");
  int rc = check_prec(h, prec);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(h->solve_mu);
  cudaStream_t s = h->ctx->stream;
  LevelBufs& L = h->L[level];
  const int nc = h->nc;
  const bool d = prec == MG_FP64;
  auto once = [&]() {
    switch (op) {
      case MG_OP_MATVEC:
        if (d) launch_matvec<double>(L.A64.v, nc, L.o64, L.r64, nullptr, s);
        else launch_matvec<float>(L.A32.v, nc, L.o32, L.r32, nullptr, s);
        break;
      case MG_OP_SMOOTH:
        if (d) launch_smooth<double>(L.A64.v, nc, L.o64, L.b64, L.S64, L.t64, h->opts.omega, false, nullptr, s);
        else launch_smooth<float>(L.A32.v, nc, L.o32, L.b32, L.S32, L.t32, h->opts.omega, false, nullptr, s);
        break;
      case MG_OP_RESTRICT:
        if (level == 0) break;
        if (d) {
          launch_residual<double>(L.A64.v, nc, L.o64, L.b64, L.r64, nullptr, s);
          launch_restrict<double>(L.R.t, nc, L.r64, h->L[level - 1].b64, nullptr, nullptr, 0.0, nullptr, s);
        } else {
          launch_residual<float>(L.A32.v, nc, L.o32, L.b32, L.r32, nullptr, s);
          launch_restrict<float>(L.R.t, nc, L.r32, h->L[level - 1].b32, nullptr, nullptr, 0.0, nullptr, s);
        }
        break;
      case MG_OP_PROLONG_ADD:
        if (level == 0) break;
        if (d) launch_prolong_add<double>(L.P.t, nc, h->L[level - 1].o64, L.o64, L.t64, nullptr, s);
        else launch_prolong_add<float>(L.P.t, nc, h->L[level - 1].o32, L.o32, L.t32, nullptr, s);
        break;
      default:
        break;
    }
  };
  once();
  CU(cudaEventRecord(h->ev0, s));
  for (int i = 0; i < reps; ++i) once();
  CU(cudaEventRecord(h->ev1, s));
  CU(cudaEventSynchronize(h->ev1));
  float t = 0;
  CU(cudaEventElapsedTime(&t, h->ev0, h->ev1));
  *ms = (double)t / reps;
  CU(cudaGetLastError());
  return MG_OK;
}

}  // extern "C"
