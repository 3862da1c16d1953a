// Launchers of the CUDA kernels (implemented in kernels.cu).  Host code calls
// only these; every pointer is a device pointer.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mgi {

constexpr int kBlock = 256;               // threads per block for every kernel
constexpr int kMaxRedBlocks = 1216;       // 152 SMs x 8: upper bound of reduction partials

// View of a SELL-C matrix of nc x nc blocks (C = 32 block rows per slice).
// Slot o of slice s lies in [sptr[s], sptr[s+1]); slot o = sptr[s] + 32 j + lane
// holds block column col[o]; block entry e (row-major i*nc+k) is stored at
// val[(o - lane) * nc*nc + e*32 + lane].
struct SellView {
  const int64_t* sptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  int64_t n = 0;          // block rows
  int64_t nslices = 0;
  int bf16 = 0;           // values stored as BF16 (read by the FP32 kernels, widened to FP32)
  const int32_t* perm = nullptr;   // SELL row -> node row (rows sorted by length within windows), or NULL
  // 16-bit column indices (FP32/BF16 copies of large levels): column =
  // (slice / 8) * 256 + col16[o].  A slice whose columns do not fit has bit 0
  // of sptr[slice] set and uses col[] instead; slot offsets are multiples of
  // 32, so readers mask sptr with kSptrMask.
  const int16_t* col16 = nullptr;
  int tpr = 1;                // lanes per block row (1 or 4; small FP32/BF16 block levels use 4)
  // Staged x (scalar FP32 / BF16 copies, one lane per row): per window of
  // 256 SELL rows (8 slices) the range [wlo, wlo + wlen) of every column its
  // stored slots name (padding included); windows of at most kStageMax
  // columns are gathered from shared memory.  NULL: not staged.
  const int32_t* wlo = nullptr;
  const int32_t* wlen = nullptr;
  // 3x3 blocks of the velocity-pressure pattern [[a, 0, g1], [0, a, g2],
  // [d1, d2, c]] (both velocity components share one operator, no coupling
  // between them) are stored as the 6 values (a, g1, g2, d1, d2, c) per slot;
  // 0: nc x nc values per slot
  int bpat = 0;
};
// values stored per slot of a block matrix
inline int block_values(const SellView& A, int nc) { return A.bpat ? 6 : nc * nc; }
constexpr int64_t kSptrMask = ~int64_t(31);
constexpr int kCol16Window = 256;       // rows per base of the 16-bit column offsets
constexpr int kStageMax = 4096;         // x entries a staged window holds (16 KB of FP32)

// Transfer matrices (P, R) are scalar SELL with float weights, applied to
// every component.  fix (block problems with partly fixed nodes, else NULL):
// per row node the bits of the components whose output stays untouched (P)
// or zero (R) -- the per-component rows of the constrained dofs.
struct TransferView {
  const int64_t* sptr = nullptr;
  const int32_t* col = nullptr;
  const float* w = nullptr;
  int64_t n = 0;
  int64_t nslices = 0;
  const uint8_t* fix = nullptr;    // indexed by node row
  const int32_t* perm = nullptr;   // SELL row -> node row, or NULL
};

// Scalars of the Krylov loop, resident in device memory.
struct KrylovState {
  double rho, rho_prev, alpha, omega, beta;
  double rnorm, bnorm, rtol, scale;  // scale: factor of the FP32 preconditioner input
  // step scalars formed once by the kernel that finishes their reductions
  // (GB300 has little FP64 throughput: a division per thread of a vector
  // kernel costs more than its memory traffic)
  double inv_scale;                  // 1 / scale
  double beta_next;                  // BiCGStab: beta of the next iteration
  double gm_inv;                     // GMRES: 1 / h_{j+1,j}
  int iter, max_it, done, status;
  int restart_pos;
  unsigned int counter;              // arrival counter of the last-block reductions
  int gm_j;                          // GMRES: current Arnoldi column
  int gm_end;                        // GMRES: 1 when the current cycle ends after this step
  double red[16];                    // finished reductions, indexed by Q_*
};

// GMRES(m) work arrays on the device (doubles): Hessenberg (m+1) x m
// column-major, Givens cosines/sines, rhs g, current coefficients h, y.
struct GmresView {
  int m = 30;
  double* H = nullptr;               // (m+1) * m
  double* cs = nullptr;              // m
  double* sn = nullptr;              // m
  double* g = nullptr;               // m + 1
  double* hv = nullptr;              // m + 1 (projection coefficients of the current sweep)
  double* y = nullptr;               // m
  double* V = nullptr;               // (m+1) * n, FP64 Krylov basis
  double* Z64 = nullptr;             // m * n preconditioned vectors (FP64 mode)
  float* Z32 = nullptr;              // m * n preconditioned vectors (mixed mode, times zs[j])
  double* zs = nullptr;              // m scales of Z32
  double* part = nullptr;            // (m+1) * kMaxRedBlocks dot partials
};

// Reduction partials: one slot array per quantity, kMaxRedBlocks each.
struct Partials {
  double* p = nullptr;                 // [nq][kMaxRedBlocks]
  double* q(int k) const { return p + (int64_t)k * kMaxRedBlocks; }
};

int grid_for_rows(int64_t rows);       // blocks for one thread per row, capped for grid-stride
int grid_for_vec(int64_t n);

// ---- level operators (T = double or float; nc = 1 or 3) --------------------
// xo64 (optional): FP64 copy of the output times *scale
template <typename T>
void launch_smooth(const SellView& A, int nc, const T* x, const T* b, const T* Sinv, T* xo, double omega,
                   bool from_zero, const int* done, cudaStream_t s, double* xo64 = nullptr,
                   const double* scale = nullptr);
template <typename T>
void launch_residual(const SellView& A, int nc, const T* x, const T* b, T* r, const int* done, cudaStream_t s);
// cell-patch Vanka update: xo = xin + omega S r (xin == NULL: xo = omega S r)
template <typename T>
void launch_vanka(const SellView& S, int nc, const T* r, const T* xin, T* xo, double omega, const int* done,
                  cudaStream_t s, double* xo64 = nullptr, const double* scale = nullptr);
template <typename T>
void launch_matvec(const SellView& A, int nc, const T* x, T* y, const int* done, cudaStream_t s);
// d = R r; when x0 != nullptr also x0 = omega S d (first sweep of the coarser level from zero)
template <typename T>
void launch_restrict(const TransferView& R, int nc, const T* r, T* d, const T* Sinv, T* x0, double omega,
                     const int* done, cudaStream_t s);
void set_pdl(bool on);
// Launch timing: while a profiler is installed on the calling thread, every
// kernel launch is bracketed by two CUDA events on its stream and recorded
// with the multigrid level the caller set (-1 outside a V-cycle).
struct LaunchProfiler {
  virtual void before(const void* fn, cudaStream_t s) = 0;
  virtual void after(cudaStream_t s) = 0;
  virtual ~LaunchProfiler() = default;
};
extern thread_local LaunchProfiler* t_prof;
extern thread_local int t_prof_level;
void launch_prof_empty(cudaStream_t s);
template <typename T>
void launch_prolong_add(const TransferView& P, int nc, const T* y, const T* xin, T* xo, const int* done,
                        cudaStream_t s);
template <typename T>
void launch_coarse(const double* Ainv, int64_t n, const T* d, T* z, const int* done, cudaStream_t s);

// ---- single-CTA tail V-cycle over the smallest levels -------------------------
constexpr int kTailMax = 16;
constexpr int kTailThreads = 1024;
struct TailLevel {
  SellView A;
  TransferView P, R;          // P, R of this level (unused on level 0)
  const void* S = nullptr;    // smoother blocks
  void* b = nullptr;          // rhs (written by the restriction from level+1)
  void* o = nullptr;          // output
  void* t = nullptr;          // ping-pong buffer
  void* r = nullptr;          // residual
  double omega = 0.8;         // smoother damping of this level
  int csh = 0;                // cluster-resident mode: rows per CTA chunk = 2^csh
  int c16 = 0;                // cluster-resident mode: A.col16 is a staged offset
};
struct TailParams {
  TailLevel lv[kTailMax];     // [0] = coarsest level of the hierarchy
  int nt = 0;                 // levels in the tail (top = nt - 1)
  int nu1 = 2, nu2 = 2;
  const double* cinv = nullptr;   // coarse inverse
  int64_t cn = 0;
  int cluster = 1;            // CTAs of the one thread-block cluster that runs the tail (1..8);
                              // 0: one CTA working in shared memory (below)
  // Shared-memory image of the tail (cluster == 0).  image[0, image_bytes) is
  // copied into dynamic shared memory at kernel start: TailLevel hdr[nt] whose
  // pointers are byte offsets into that memory (the vectors b, o, t, r of every
  // level, and the matrices A, S, P, R of the levels whose bit is set in
  // staged_mask; the other levels keep device pointers), followed by the
  // staged matrix arrays.  The vectors occupy [image_bytes, smem).
  const void* image = nullptr;
  uint32_t image_bytes = 0;
  uint32_t smem = 0;
  uint32_t staged_mask = 0;
  // Cluster-resident mode (dsm = 1, scalar problems): a cluster of `cluster`
  // CTAs, CTA k holding chunk k (rows [k 2^csh, (k+1) 2^csh) of every level)
  // of every vector at the same shared-memory offset in each CTA, and the rows
  // of its chunks of the level and transfer matrices; gathers of other CTAs'
  // entries go through distributed shared memory.  The image has one section
  // of `section` bytes per CTA (header, then the matrices; vectors follow in
  // shared memory at offsets equal in every CTA); its header pointers are
  // byte offsets relative to the CTA's shared memory, shifted by the chunk's
  // first row so that rows keep their level-wide indices.
  int dsm = 0;
  uint32_t section = 0;
};
// dynamic shared memory of the staged tail: sm_100 / sm_103 give a block up
// to 227 KB (232448 B) on opt-in; 1 KB stays for the static arrays of the
// batched kernel
constexpr uint32_t kTailSmemMax = 226 * 1024;
// true when the GPU schedules a cluster of cl tail CTAs (always for cl <= 8)
bool tail_cluster_fits(int cl);
// true when the GPU schedules a cluster-resident tail of cl CTAs with smem
// bytes of dynamic shared memory each
bool tail_dsm_fits(int cl, uint32_t smem);
template <typename T>
// o64 (optional): FP64 copy of the output times *scale, written by the last
// post-smoothing sweep (nothing when nu2 == 0)
void launch_tail(const TailParams& P, int nc, const T* b, T* out, bool first_done, const int* done, cudaStream_t s,
                 double* o64 = nullptr, const double* scale = nullptr);

// ---- batched solves of small problems ---------------------------------------
// One problem of a batched launch.  The thread block that takes it runs the
// whole Krylov solve: FP64 outer vectors in device memory, the V-cycle as the
// staged tail over every level of the hierarchy (vectors and matrices in
// shared memory).  Scalars and the status stay in the block.
struct BatchItem {
  const TailParams* tail = nullptr;   // device copy of the hierarchy's staged tail (nt = all levels)
  SellView A;                         // finest FP64 operator
  TransferView Hc;                    // hanging rows of H (finest)
  const uint8_t* fix = nullptr;       // per node: fixed-dof bits (hanging or Dirichlet)
  const double* b = nullptr;          // assembled right-hand side, n entries
  double* x = nullptr;                // in: initial guess; out: solution, hanging values filled
  double *xi = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;   // work vectors, n each
  double *rhat = nullptr, *v = nullptr, *s = nullptr, *ph = nullptr, *sh = nullptr;   // BiCGStab
  int64_t n_nodes = 0, n = 0;         // nodes, dofs (n = n_nodes * nc)
  int method = 1;                     // 1: flexible CG, 2: BiCGStab
  int max_it = 1;
  double rtol = 1e-8;
  // results, written by the block
  int status = 0;                     // 0, -4 (max_it), -5 (breakdown), -6 (not finite),
                                      // -7 (refused: inconsistent item, nothing computed)
  int iters = 0, rounds = 0;
  double rel_res = 0.0;               // true ||b - A x|| / ||b_free||
};
// Solves count items, taken in the order order[0..count) by grid blocks of
// kTailThreads threads (a block takes the next item when it finishes one);
// *next must be 0 at launch.  prec 0: FP64 V-cycle, 1: FP32, 2: FP32 with
// BF16-stored values.  smem: the largest staged tail of the items.
void launch_batch(BatchItem* items, const int* order, int count, unsigned int* next, int nc, int prec, uint32_t smem,
                  int grid, cudaStream_t s);
// Blocks of the batched kernel resident on one SM with smem bytes of shared memory
int batch_blocks_per_sm(int nc, int prec, uint32_t smem);

// ---- vector kernels --------------------------------------------------------
void launch_rhs(const SellView& F, int nc, const double* f, const uint8_t* fixmask, const uint8_t* dirmask,
                const double* g, double* b, cudaStream_t s);
void launch_lift(const SellView& L, int nc, const double* g, double* b, cudaStream_t s);
// out = sc * theta + f (f NULL: out = sc * theta), n entries
void launch_step_load(int64_t n, double sc, const double* theta, const double* f, double* out, cudaStream_t s);
// out = (u / dt + v) / dt + f, then v = -u / dt (f NULL: no source)
void launch_step_load2(int64_t n, double inv_dt, const double* u, double* v, const double* f, double* out,
                       cudaStream_t s);
// v += u / dt
void launch_step_velocity(int64_t n, double inv_dt, const double* u, double* v, cudaStream_t s);
void launch_fill_hanging(const TransferView& Hc, int nc, double* x, cudaStream_t s);
void launch_copy_fixed(int64_t n_nodes, int nc, const uint8_t* fixmask, const double* b, const double* xin,
                       double* x, cudaStream_t s);
// ---- Krylov kernels (FP64 outer loop) --------------------------------------
// Preconditioned vectors come either as double (zs == nullptr) or as float
// times the scalar st->scale (z32 != nullptr).
struct PVec {
  const double* d = nullptr;
  const float* f = nullptr;
};

// Clears the CUDA-graph while condition (first kernel of every loop body).
void launch_cond_reset(unsigned long long cond, cudaStream_t s);

// Quantity slots of the partial arrays and of KrylovState::red
enum { Q_RR = 0, Q_RZ = 1, Q_QZ = 2, Q_PQ = 3, Q_BB = 4, Q_RHV = 5, Q_SS = 6, Q_TS = 7, Q_TT = 8, Q_RHR = 9, Q_NUM = 10 };

// r = b - A x and ||r||^2 -> red[Q_RR]; test 1: initial convergence test; test 2:
// end of a multigrid-solver iteration (counts it and sets the while condition)
void launch_residual_norm(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                          KrylovState* st, int test, cudaStream_t s, unsigned long long cond = 0ull);
// x += z for the multigrid iteration
void launch_mgi_update(int64_t n, PVec z, double* x, KrylovState* st, cudaStream_t s);
// ||b_free||^2 -> bnorm, and the initial Krylov state
void launch_norm_init(int64_t n_nodes, int nc, const uint8_t* fixmask, const double* b, Partials part,
                      KrylovState* st, double rtol, int max_it, cudaStream_t s);
void launch_to_f32(int64_t n, const double* v, float* v32, const KrylovState* st, cudaStream_t s);
// CG (flexible, Polak-Ribiere beta): dots -> Q_RZ, Q_QZ; update_p; spmv_dot -> Q_PQ; update_xr -> Q_RR + test
void launch_cg_dots(int64_t n, PVec z, const double* r, const double* q, Partials part, KrylovState* st,
                    cudaStream_t s);
void launch_cg_update_p(int64_t n, PVec z, double* p, KrylovState* st, cudaStream_t s);
void launch_spmv_dot(const SellView& A64, int nc, PVec p, const double* w, double* out, Partials part, int k,
                     KrylovState* st, cudaStream_t s);
void launch_cg_update_xr(int64_t n, const double* p, const double* q, double* x, double* r, Partials part,
                         KrylovState* st, unsigned long long cond, cudaStream_t s);
// BiCGStab (right preconditioned): p ; spmv_dot -> Q_RHV ; s ; spmv_2dots -> Q_TS, Q_TT ; x -> Q_RR, Q_RHR + test.
// p32 / s32 (optional): FP32 copies scaled by 1 / st->scale for the FP32 preconditioner
void launch_bicg_p(int64_t n, const double* r, const double* v, double* p, float* p32, KrylovState* st,
                   cudaStream_t s);
void launch_bicg_s(int64_t n, const double* r, const double* v, double* sv, float* s32, KrylovState* st,
                   cudaStream_t s);
void launch_spmv_2dots(const SellView& A64, int nc, PVec sh, const double* sv, double* t, Partials part,
                       KrylovState* st, cudaStream_t s);
void launch_bicg_x(int64_t n, PVec ph, PVec sh, const double* sv, const double* t, const double* rhat, double* x,
                   double* r, Partials part, KrylovState* st, unsigned long long cond, cudaStream_t s);

// ---- GMRES(m), flexible, right preconditioned (Sec. 4.1.5; Saad 2003) -------
// start: v0 = r / ||r|| (+ FP32 copy), g = ||r|| e1, j = 0 (gated: cycle start)
void launch_gm_start(int64_t n, const double* r, float* v32, double* v64, GmresView G, KrylovState* st,
                     cudaStream_t s);
// w = A z_j, z_j = preconditioner output (FP64 z64 or FP32 z32 x 1); also stores z_j into Z[j]
void launch_gm_spmv(const SellView& A64, int nc, PVec z, double* w, GmresView G, KrylovState* st, cudaStream_t s);
// one classical Gram-Schmidt sweep: h_i = (v_i, w), w -= sum h_i v_i, i <= j; pass 0 or 1
void launch_gm_orth(int64_t n, double* w, GmresView G, KrylovState* st, int pass, Partials part, cudaStream_t s);
// Givens update of column j, convergence test, triangular solve at the cycle end
void launch_gm_givens(GmresView G, KrylovState* st, cudaStream_t s);
// v_{j+1} = w / h_{j+1,j} (+ FP32 copy) when the cycle continues
void launch_gm_next(int64_t n, const double* w, float* v32, double* v64, GmresView G, KrylovState* st,
                    cudaStream_t s);
// x += sum_i y_i z_i at the cycle end
void launch_gm_update_x(int64_t n, double* x, GmresView G, KrylovState* st, cudaStream_t s);
// r = b - A x and the convergence test at the cycle end (true residual)
void launch_gm_residual(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                        KrylovState* st, unsigned long long cond, cudaStream_t s);

}  // namespace mgi
