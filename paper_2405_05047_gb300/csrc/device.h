// Device-side hierarchy, solve workspaces and the asynchronous solve driver.
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"

namespace mgi {

struct Alloc {
  void* p = nullptr;
  size_t bytes = 0;
  bool cuda = false;          // allocated with cudaMalloc (not the context allocator)
};

struct SellBuf {
  SellView v;
  TransferView t;
  int64_t nnz_real = 0;
  int64_t slots = 0;
  int64_t sigma = 0;          // SELL-C-sigma window it was packed with
  size_t val_bytes = 0;       // bytes of its value array
};

// Read-only matrices of one level.
struct LevelMats {
  int64_t n = 0;              // nodes
  double omega = 0.8;         // smoother damping of this level
  SellBuf A64, A32, A16, P, R;   // A16: BF16-stored values
  double* S64 = nullptr;
  float* S32 = nullptr;
  bool vanka = false;         // smoothed by the cell-patch Vanka matrix V instead of Jacobi
  SellBuf V64, V32;           // Vanka matrix (FP32 copy also serves the BF16-values path)
};

// V-cycle vectors of one level in one workspace: rhs, out, ping-pong, residual.
struct LevelVecs {
  double *b64 = nullptr, *o64 = nullptr, *t64 = nullptr, *r64 = nullptr;
  float *b32 = nullptr, *o32 = nullptr, *t32 = nullptr, *r32 = nullptr;
};

struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  int method = 0, prec = 0;
  int64_t launches_per_iter = 0;
};

// Everything one solve writes: a hierarchy can run as many solves at once as
// it has workspaces.
struct Workspace {
  std::vector<LevelVecs> lv;
  double *xi = nullptr, *bi = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *rhat = nullptr,
         *sv = nullptr, *t = nullptr, *ph = nullptr, *shat = nullptr, *vcur = nullptr;
  float *r32 = nullptr, *ph32 = nullptr, *sh32 = nullptr;
  Partials part;
  KrylovState* st = nullptr;
  KrylovState* st_host = nullptr;   // pinned mirror, written at the end of every round
  GmresView gm;
  TailParams tail64, tail32, tail16;
  std::vector<SolveGraph> graphs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<Alloc> allocs;
  size_t bytes = 0;
  // the solve in flight
  int method = 0, prec = 0, rounds = 0, max_it = 0, iter_base = 0;
  double rtol = 0.0;
  int64_t launches = 0;
  bool graph_round = false;       // the current round's iterations run as the cached solve graph
  double* x_out = nullptr;
  bool x_out_host = false;
};

// Per-kernel timing of a solve (mg_solve_profiled).  Launches made while a
// stream is being captured use a fixed pool of events and are timed as a
// chain: one event before the first kernel and one after every run of
// consecutive launches of the same kernel on the same level (the launches of
// a run follow each other as in the solve, with no event node between them),
// so an interval runs from the end of the previous run to the end of its own
// and the intervals add up to the captured iteration.  The graph re-records
// the same events on every run (collect_graph after each).  Other launches
// are bracketed by events of their own, read once at the end.  Results are
// summed per (kernel, multigrid level).
struct EventProfiler : LaunchProfiler {
  struct Rec {
    const void* fn;
    int level;
    cudaEvent_t e0, e1;
    int64_t n = 1;               // launches in the interval (a run of the same kernel and level)
  };
  std::vector<cudaEvent_t> graph_pool, direct_pool;
  size_t graph_used = 0;
  std::vector<Rec> graph_recs, direct_recs;
  bool pending = false;          // the last before() recorded a start event
  bool run_open = false;         // the captured run's end event is not recorded yet
  cudaStream_t run_stream = nullptr;
  int64_t dropped = 0;           // launches beyond the graph pool
  std::map<std::pair<const void*, int>, std::pair<int64_t, double>> acc;   // launches, ms
  int init(size_t graph_events);
  void before(const void* fn, cudaStream_t s) override;
  void after(cudaStream_t s) override;
  void begin_capture() {
    graph_used = 0;
    graph_recs.clear();
    run_open = false;
  }
  void close_run();              // record the end event of the open captured run
  void end_capture() { close_run(); }   // before the capture ends
  void collect_graph();          // after the graph's run completed
  void collect_direct();         // after every direct launch completed
  ~EventProfiler() override;
};

// One batched launch (k_batch) and its buffers: a device arena (work list,
// order, counters, FP64 work vectors) and a pinned mirror of the work list,
// both grown to the largest batch run through them.  batch_enqueue puts the
// uploads, the launches (between ev0 and ev1) and the download of the
// results on a stream, then records done; batch_collect reads the results
// once done completed.
struct BatchRun {
  std::vector<Alloc> allocs;
  size_t bytes = 0;
  void* arena = nullptr;
  size_t cap = 0;
  void* host = nullptr;
  size_t host_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, done = nullptr;
  int count = 0, prec = 0, launches = 0;
};

int fail(int code, const std::string& msg);
const char* last_error();

}  // namespace mgi

struct mg_ctx;
namespace mgi {
// Device allocation through the context's allocator (ctx_alloc) or
// cudaMalloc, recorded in list and counted against the context; free_list
// releases a list.
void* ctx_alloc(mg_ctx* c, std::vector<Alloc>& list, size_t& total, size_t bytes, bool ctx_alloc);
void ctx_free(mg_ctx* c, std::vector<Alloc>& list, size_t& total);
}  // namespace mgi

struct ServeRequest;
struct ServeBatch;

struct mg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mg_allocator alloc{};
  bool has_alloc = false;
  size_t budget = 0;
  std::atomic<size_t> used{0};          // every device byte allocated through this context
  std::atomic<size_t> resident{0};      // hierarchies and their default workspaces
  std::atomic<int> live_hiers{0};       // hierarchies not yet freed
  // serving
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  bool worker_started = false;
  uint64_t next_ticket = 1;
  int max_slots = 16;
  std::deque<std::shared_ptr<ServeRequest>> queue;
  std::vector<std::shared_ptr<ServeRequest>> running;
  std::map<uint64_t, std::shared_ptr<ServeRequest>> tickets;
  std::vector<cudaStream_t> free_streams;
  // batched solves: the run of mg_solve_batch (one call at a time), and the
  // serving scheduler's runs (idle ones pooled)
  std::mutex batch_mu;
  mgi::BatchRun batch;
  int serve_batch = 0;                  // most requests per batched launch (0: no batching)
  int serve_batch_min = 2;              // fewest queued fitting requests that go out as one
  std::vector<std::shared_ptr<ServeBatch>> batches;   // batched launches in flight
  std::vector<mgi::BatchRun*> free_runs;
};

struct mg_hier {
  mg_ctx* ctx = nullptr;
  int dim = 2, nc = 1, nlev = 0;
  int64_t n_nodes = 0, n_dofs = 0, n_free = 0, n_hanging = 0;
  mg_problem prob{};
  mg_opts opts{};
  std::vector<double> coords;            // finest nodes, external order
  std::vector<int64_t> level_nodes, level_nnzb, level_real_nnzb;
  std::vector<int> level_block_values;   // values stored per slot (nc*nc, or 6: velocity-pressure pattern)
  std::vector<mgi::Alloc> allocs;        // matrices
  size_t bytes = 0;
  std::vector<mgi::LevelMats> L;         // [0] coarsest
  double* coarse_inv = nullptr;          // (n0 nc)^2
  int64_t coarse_n = 0;
  mgi::SellBuf F;                        // load matrix (finest)
  mgi::SellBuf Hc;                       // hanging rows of H (finest)
  uint8_t* fixmask = nullptr;            // finest, per node: fixed-dof bits (hanging or Dirichlet)
  uint8_t* dirmask = nullptr;            // finest, per node: Dirichlet bits
  mgi::SellBuf Lift;                     // finest: free-row x Dirichlet-column couplings (n = 0: none)
  bool has_fp64 = true, has_fp32 = true, has_bf16 = false;
  int tail_top = 0;                      // levels 0..tail_top run in the tail kernel
  int tail_cluster = 1;                  // 0: one CTA in shared memory, > 0: cluster CTAs over device
                                         // memory, < 0: -CTAs of a cluster-resident tail
  struct TailImage {
    void* p = nullptr;
    uint32_t image_bytes = 0, smem = 0, staged_mask = 0;
    uint32_t section = 0;                  // cluster-resident image: bytes per CTA section
  };
  // (precision slot, top | CTAs << 8) -> shared-memory image (CTAs = 0: one CTA)
  std::map<std::pair<int, int>, TailImage> tail_img;
  double tuned_vcycle_ms = 0.0;
  int64_t col16_slices = 0, col32_slices = 0;   // over the matrices stored with 16-bit columns
  std::vector<int> level_col16;                 // per level: operator copies with 16-bit columns
  std::vector<int64_t> level_sigma;             // per level: SELL-C-sigma window of the operator copies
  int gmres_m = 0;                       // > 0: workspaces carry GMRES(m) arrays
  mgi::Workspace* ws0 = nullptr;         // default workspace (mg_solve, mg_vcycle, mg_apply)
  std::mutex solve_mu;                   // guards ws0
  std::mutex pool_mu;
  std::vector<mgi::Workspace*> pool;     // idle serving workspaces
  std::vector<mgi::Workspace*> all_ws;   // every serving workspace
  size_t ws_bytes = 0;                   // device bytes of one workspace
  int serve_cap = 0;                     // > 0: serving never holds more workspaces (mg_serve_reserve)
  // the mesh it was set up on (leaf arrays and graded axes owned here), for
  // re-assembly with new coefficients
  mg_mesh mesh{};
  std::vector<int32_t> mesh_lev, mesh_anc;
  std::vector<double> mesh_axis[3];
  // batched solves: device copy of the staged tail over every level, per
  // precision slot (built on first use), and its shared-memory bytes
  const mgi::TailParams* batch_tp[3] = {nullptr, nullptr, nullptr};
  uint32_t batch_smem[3] = {0, 0, 0};
  std::atomic<int64_t> launch_count{0};  // kernels enqueued (host-side count)
};

namespace mgi {

int method_of(const mg_hier* h);
int check_prec(const mg_hier* h, int prec);
size_t workspace_bytes(const mg_hier* h);
// New workspace; its buffers are initialised in stream order on `s`, the
// stream its solves will run on.
int ws_create(mg_hier* h, bool ctx_alloc, cudaStream_t s, Workspace** out);
void ws_destroy(mg_hier* h, Workspace* ws);
int upload_hierarchy(mg_hier* h, HostHierarchy& H);
// Rewrites the values of an uploaded hierarchy in place from H, a host
// hierarchy of the same mesh with new coefficients (same levels, patterns
// and layouts): operators, smoother blocks and damping, Vanka matrices,
// coarse inverse, load and lifting matrices; rebuilds the small-level images,
// refreshes the workspaces' level parameters and drops their solve graphs.
int update_hierarchy(mg_hier* h, HostHierarchy& H);
// Tail threshold (levels <= rows dofs) and cluster size for every workspace;
// cached solve graphs are dropped (they embed the old configuration).
// cluster 0: one CTA with the tail in shared memory (the threshold is lowered
// until its vectors fit).
int set_tail(mg_hier* h, int rows, int cluster);
// Time V-cycles over tail thresholds x cluster sizes, keep the fastest.
int autotune(mg_hier* h, int prec);
void free_hierarchy(mg_hier* h);

// bf16 (T = float only): level operators with BF16-stored values.  out64
// (optional): the result also in FP64 times *scale, written by the last sweep;
// returns false when the cycle could not produce it (the caller then reads out).
template <typename T>
bool enqueue_vcycle(mg_hier* h, Workspace& w, int l, const T* b, T* out, const int* done, cudaStream_t s,
                    bool first_done = false, bool bf16 = false, double* out64 = nullptr,
                    const double* scale = nullptr);

// Asynchronous solve: solve_start copies the inputs (device or host
// pointers) into the workspace and enqueues the first round; a round ends
// with the outputs written to x_out and the state mirrored to st_host, then
// ev1 recorded.  solve_check (after ev1 completed) either returns the final
// status or enqueues another round (true residual above rtol) and returns
// MG_PENDING.
int solve_start(mg_hier* h, Workspace& w, const double* b, bool b_host, const double* x0, bool x0_host,
                double* x_out, bool x_out_host, double rtol, int max_it, int prec, cudaStream_t s);
int solve_check(mg_hier* h, Workspace& w, cudaStream_t s, mg_stats* stats);
// The cached solve graph of (method, prec) of a workspace, built on first use.
int get_graph(mg_hier* h, Workspace& w, int method, int prec, SolveGraph** g);
// MG_OK when h can be solved by the batched kernel at prec (else the reason,
// through fail()).
int batch_check(const mg_hier* h, int prec);
// Batched solve of count problems (mg_solve_batch).
int solve_batch(mg_ctx* c, int count, mg_hier* const* hs, const double* const* b, double* const* x, double rtol,
                int max_it, int prec, mg_stats* stats);
// Enqueues a batched solve on s (problems checked by batch_check; rtol and
// max_it per problem) into run; MG_OK or an allocation / admission error
// (nothing enqueued).
int batch_enqueue(mg_ctx* c, BatchRun& run, int count, mg_hier* const* hs, const double* const* b,
                  double* const* x, const double* rtol, const int* max_it, int prec, cudaStream_t s);
// After run.done completed: per-problem stats; returns MG_OK when all converged,
// else the status of the first problem that did not.
int batch_collect(BatchRun& run, mg_stats* stats);
// Releases a run's buffers and events.
void free_run(mg_ctx* c, BatchRun& run);

}  // namespace mgi
