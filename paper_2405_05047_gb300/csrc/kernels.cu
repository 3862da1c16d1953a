// CUDA kernels of the multigrid-preconditioned Krylov solve (sm_103a).
//
// Layout: level operators in SELL-C (C = 32 block rows per slice, one thread
// per block row, slots of a slice stored column-major so that the 32 threads
// of a warp read consecutive addresses); nc x nc blocks store entry e of the
// 32 blocks of one slot group contiguously.  Transfers are scalar SELL with
// float weights (all weights are dyadic, exact in FP32).
//
// Reductions are deterministic: every kernel that produces a dot product
// writes one partial per block (fixed grid, fixed order inside the block),
// the consuming kernel sums the partials in a fixed order.  No floating-point
// atomics anywhere.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "kernels.h"
#include "rows.cuh"
namespace mgi {

namespace {

// ------------------------------------------------------------------ level ops
// x_out = x + omega S (b - A x)  (Sec. 4.1.4), S = inverse diagonal block.
// xo64 (optional): the sweep's output also written in FP64 times *scale (the
// last sweep of an FP32 V-cycle hands the FP64 Krylov loop its result).
template <typename T, typename VT, int NC, bool FROM_ZERO, int TPR>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 8 : 4) k_smooth(SellView A, const T* __restrict__ x, const T* __restrict__ b,
                                                    const T* __restrict__ Sinv, T* __restrict__ xo, T omega,
                                                    const int* done, double* __restrict__ xo64,
                                                    const double* scale) {
  pdl_wait();
  if (stopped(done)) return;
  const double sc = xo64 ? *scale : 1.0;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = A.nslices * 32 * TPR;   // TPR lanes per row (1 or 4)
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += nthreads)
    row_smooth<T, NC, 0, VT, TPR>(A, t / TPR, x, b, Sinv, xo, omega, FROM_ZERO, (int)(t % TPR), xo64, sc);
}

// The scalar FP32 sweep with each window's x staged in shared memory: the
// 256 rows of a window (8 slices) gather x over a column range [wlo,
// wlo + wlen) a few thousand entries wide on most windows of a lexicographic
// mesh; the block loads that range once (coalesced, every load independent),
// and each gather becomes a shared-memory read instead of an L2 round trip
// behind the column load.  Windows with a wider range gather from device
// memory as in k_smooth.  Same row function, same summation order: the same
// bits as k_smooth.
template <typename VT>
__global__ void __launch_bounds__(kBlock, 8) k_smooth_staged(SellView A, const float* __restrict__ x,
                                                             const float* __restrict__ b,
                                                             const float* __restrict__ Sinv, float* __restrict__ xo,
                                                             float omega, const int* done, double* __restrict__ xo64,
                                                             const double* scale) {
  static_assert(kBlock == kCol16Window, "one block per 256-row window");
  __shared__ float xs[kStageMax];
  pdl_wait();
  if (stopped(done)) return;
  const double sc = xo64 ? *scale : 1.0;
  const int64_t rows = A.nslices * 32;
  const int64_t nwin = (rows + kBlock - 1) / kBlock;
  for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
    const int32_t lo = __ldg(A.wlo + w), len = __ldg(A.wlen + w);
    const bool staged = len <= kStageMax;
    __syncthreads();                                   // the previous window's gathers are done
    if (staged)
      for (int i = threadIdx.x; i < len; i += blockDim.x) xs[i] = __ldg(x + lo + i);
    __syncthreads();
    const int64_t row = w * kBlock + threadIdx.x;
    if (row < rows) {
      if (staged) row_smooth<float, 1, 4, VT, 1>(A, row, xs - lo, b, Sinv, xo, omega, false, 0, xo64, sc);
      else row_smooth<float, 1, 0, VT, 1>(A, row, x, b, Sinv, xo, omega, false, 0, xo64, sc);
    }
  }
}

template <typename T, typename VT, int NC, int MODE, int TPR>   // MODE 0: y = A x; 1: y = b - A x
__global__ void __launch_bounds__(kBlock, NC == 1 ? 8 : 4) k_apply(SellView A, const T* __restrict__ x, const T* __restrict__ b,
                                                   T* __restrict__ y, const int* done) {
  pdl_wait();
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  constexpr int tpr = TPR;
  const int64_t total = A.nslices * 32 * tpr;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += nthreads) {
    const int64_t row = t / tpr;
    const int sub = (int)(t % tpr);
    if (MODE == 1) {
      row_residual<T, NC, 0, VT, TPR>(A, row, x, b, y, sub);
      continue;
    }
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      T r = sell_dot1<T, 0, VT, TPR>(A, slice, lane, x, sub);
      if (row < A.n && sub == 0) y[orow] = r;
    } else {
      T acc[3];
      sell_dot3<T, 0, VT, TPR>(A, slice, lane, x, acc, sub);
      if (row < A.n) {
        const int i0 = tpr > 1 ? sub : 0, i1 = tpr > 1 ? sub + 1 : 3;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i >= i0 && i < i1) y[3 * orow + i] = acc[i];
      }
    }
  }
}

// Cell-patch Vanka update x_out = x_in + omega S r with the assembled Vanka
// matrix S = W sum_T P_T A_T^-1 P_T^T (block SELL, dense nc x nc blocks) and
// r = b - A x_in from the preceding residual kernel; from zero (x_in = NULL)
// r is b itself and x_out = omega S b.  xo64 (optional): the output also in
// FP64 times *scale (last sweep of an FP32 V-cycle).
template <typename T, typename VT, int NC, int TPR>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 8 : 4) k_vanka(SellView S, const T* __restrict__ r,
                                                   const T* __restrict__ xin, T* __restrict__ xo, T omega,
                                                   const int* done, double* __restrict__ xo64,
                                                   const double* scale) {
  pdl_wait();
  if (stopped(done)) return;
  const double sc = xo64 ? *scale : 1.0;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = S.nslices * 32 * TPR;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += nthreads) {
    const int64_t row = t / TPR;
    const int sub = (int)(t % TPR);
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t orow = srow<0>(S, row);
    if (NC == 1) {
      const T c = sell_dot1<T, 0, VT, TPR>(S, slice, lane, r, sub);
      if (row < S.n && sub == 0) {
        const T v = xin ? fmad(omega, c, xin[orow]) : omega * c;
        xo[orow] = v;
        if (xo64) xo64[orow] = (double)v * sc;
      }
    } else {
      T acc[3];
      sell_dot3<T, 0, VT, TPR>(S, slice, lane, r, acc, sub);
      if (row < S.n) {
        const int i0 = TPR > 1 ? sub : 0, i1 = TPR > 1 ? sub + 1 : 3;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i < i0 || i >= i1) continue;
          const T v = xin ? fmad(omega, acc[i], xin[3 * orow + i]) : omega * acc[i];
          xo[3 * orow + i] = v;
          if (xo64) xo64[3 * orow + i] = (double)v * sc;
        }
      }
    }
  }
}

// d_j = sum_i R(j,i) r_i (R = P^T stored as its own gather matrix: no atomics).
// With S0 the same pass also performs the coarser level's first smoothing
// sweep from a zero guess, x0_j = omega S_j d_j (it needs no matrix).
template <typename T, int NC, bool S0>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 3) k_restrict(TransferView R, const T* __restrict__ r, T* __restrict__ d,
                                                      const T* __restrict__ Sinv, T* __restrict__ x0, T omega,
                                                      const int* done) {
  pdl_wait();
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < R.nslices * 32; row += nthreads)
    row_restrict<T, NC, 0>(R, row, r, d, Sinv, S0 ? x0 : nullptr, omega);
}

// x_out_i = x_in_i + sum_j P(i,j) y_j: the coarse correction interpolated and added (Sec. 2.2)
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 3) k_prolong(TransferView P, const T* __restrict__ y, const T* xin, T* xo,
                                                     const int* done) {
  pdl_wait();
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < P.nslices * 32; row += nthreads)
    row_prolong<T, NC, 0>(P, row, y, xin, xo);
}

template <typename T, typename VT, int NC, int TLM>
__global__ void __launch_bounds__(kTailThreads) k_tail(TailParams P, const T* btop, T* otop, int first_done,
                                                        const int* done, double* o64, const double* scale) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  int64_t me = 0;                                // CTA rank in the cluster (TLM 3)
  if constexpr (TLM == 3) me = (int64_t)cooperative_groups::this_cluster().block_rank();
  const TailLevel* LV = P.lv;
  // the image holds only matrices and offsets: copy it before waiting on the
  // preceding kernel
  if constexpr (TLM == 2 || TLM == 3) LV = tail_stage<TLM>(P, tail_smem, me);
  pdl_wait();
  if (stopped(done)) return;
  tail_cycle<T, VT, NC, TLM>(P, LV, btop, otop, first_done, o64, scale, me);
}

// z = A_0^{-1} d with the FP64 inverse of the coarse matrix; one warp per row.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_coarse(const double* __restrict__ Ainv, int64_t n, const T* __restrict__ d,
                                                    T* __restrict__ z, const int* done) {
  pdl_wait();
  if (stopped(done)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) acc = fma(Ainv[row * n + j], (double)d[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) z[row] = (T)acc;
  }
}

// ------------------------------------------------------------------ vectors
// b = H^T (F f) on free dofs; Dirichlet dofs take g (0 without g), hanging
// dofs 0.  fix: fixed-dof bits per node, dir: Dirichlet bits per node.
__global__ void k_rhs(SellView F, int nc, const double* __restrict__ f, const uint8_t* __restrict__ fix,
                      const uint8_t* __restrict__ dir, const double* __restrict__ g, double* __restrict__ b) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < F.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    double acc[3] = {0.0, 0.0, 0.0};
    const double* val = (const double*)F.val;
    for (int64_t o = F.sptr[slice] + lane; o < F.sptr[slice + 1]; o += 32) {
      const double w = val[o];
      const int j = F.col[o];
      for (int c = 0; c < nc; ++c) acc[c] = fma(w, f[(int64_t)nc * j + c], acc[c]);
    }
    if (row < F.n)
      for (int c = 0; c < nc; ++c) {
        double v = acc[c];
        if ((dir[row] >> c) & 1) v = g ? g[nc * row + c] : 0.0;
        else if ((fix[row] >> c) & 1) v = 0.0;
        b[nc * row + c] = v;
      }
  }
}

// b -= Lift g on the free dofs: Lift holds the couplings of free rows to
// Dirichlet columns of the condensed operator (symmetric elimination).
template <int NC>
__global__ void k_lift(SellView L, const double* __restrict__ g, double* __restrict__ b) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < L.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const double* val = (const double*)L.val;
    double acc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) acc[i] = 0.0;
    for (int64_t o = L.sptr[slice] + lane; o < L.sptr[slice + 1]; o += 32) {
      const int64_t j = L.col[o];
      const int64_t vb = (o - lane) * NC * NC + lane;
#pragma unroll
      for (int i = 0; i < NC; ++i)
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[i] = fma(val[vb + (int64_t)(i * NC + k) * 32], g[NC * j + k], acc[i]);
    }
    if (row < L.n)
#pragma unroll
      for (int i = 0; i < NC; ++i) b[NC * row + i] -= acc[i];
  }
}

// x_i = sum_j H(i,j) x_j on hanging rows (H restricted to hanging rows;
// row i of the view is node Hc.rowmap...); here the view rows are all nodes
// and regular rows are empty.
__global__ void k_fill_hanging(TransferView Hc, int nc, double* x) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < Hc.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t o0 = Hc.sptr[slice] + lane, o1 = Hc.sptr[slice + 1];
    bool any = false;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t o = o0; o < o1; o += 32) {
      const double w = (double)Hc.w[o];
      if (w == 0.0) continue;
      any = true;
      const int j = Hc.col[o];
      for (int c = 0; c < nc; ++c) acc[c] = fma(w, x[(int64_t)nc * j + c], acc[c]);
    }
    if (row < Hc.n && any)
      for (int c = 0; c < nc; ++c) x[nc * row + c] = acc[c];
  }
}

__global__ void k_copy_fixed(int64_t n, int nc, const uint8_t* __restrict__ fix, const double* __restrict__ b,
                             const double* __restrict__ xin, double* __restrict__ x) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    for (int c = 0; c < nc; ++c) x[nc * i + c] = ((fix[i] >> c) & 1) ? b[nc * i + c] : xin[nc * i + c];
}

// Nodal field of one backward-Euler step's load: out = s theta + f (f may be
// NULL: no source).  Scalar loads: theta and f are caller pointers (f is a
// block of a steps x n array) with no alignment beyond 8 bytes.
__global__ void k_step_load(int64_t n, double s, const double* __restrict__ theta, const double* __restrict__ f,
                            double* __restrict__ out) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    out[i] = f ? fma(s, theta[i], f[i]) : s * theta[i];
}

// Second-order-in-time steps (d_t^2 u + A u = f as the first-order system in
// (u, v), backward Euler): the step's nodal load (u/dt + v)/dt + f, and v
// replaced by -u/dt so that k_step_velocity can finish v_n = (u_n - u_{n-1})/dt
// after the solve without another buffer.
__global__ void k_step_load2(int64_t n, double inv_dt, const double* __restrict__ u, double* __restrict__ v,
                             const double* __restrict__ f, double* __restrict__ out) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) {
    const double ui = u[i];
    const double l = fma(ui, inv_dt, v[i]) * inv_dt;
    out[i] = f ? l + f[i] : l;
    v[i] = -ui * inv_dt;
  }
}

__global__ void k_step_velocity(int64_t n, double inv_dt, const double* __restrict__ u, double* __restrict__ v) {
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    v[i] = fma(u[i], inv_dt, v[i]);
}

// ------------------------------------------------------------------ Krylov
// All Krylov kernels run one thread per node (nc dofs) or per vector entry.
// A kernel that produces dot products writes one partial per block; the block
// that finishes last (integer arrival counter, no floating-point atomics)
// sums the partials of every quantity in a fixed order and stores the scalars
// in st->red[], so consumers read one double.  Kernels that end an iteration
// run the convergence test in that last block and set the condition of the
// CUDA-graph while loop there.
__device__ __forceinline__ double pv(const PVec& p, int64_t i, double scale) {
  return p.f ? (double)p.f[i] * scale : p.d[i];
}

// First kernel of every loop body: the while condition is cleared here, so the
// loop only continues if the convergence test at the end of the body sets it
// again (a body that fails to reach its test ends the loop instead of
// spinning).
__global__ void k_cond_reset(unsigned long long cond) {
  pdl_wait();
  if (threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
}

// Convergence test, thread 0 of the last block.  count: increment iter.
__device__ void converge_step(KrylovState* st, bool count, unsigned long long cond) {
  if (count) st->iter += 1;
  const double rn = sqrt(st->red[Q_RR]);
  st->rnorm = rn;
  st->scale = rn > 0.0 ? rn : 1.0;
  st->inv_scale = 1.0 / st->scale;
  int done = 0, status = st->status;
  if (!isfinite(rn)) { done = 1; status = status ? status : -6; }
  else if (status != 0) done = 1;
  else if (rn <= st->rtol * st->bnorm) { done = 1; status = 0; }
  else if (st->iter >= st->max_it) { done = 1; status = -4; }
  st->status = status;
  st->done = done;
  if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, done ? 0u : 1u);
}

// Writes this block's partials of nq quantities; returns true (in every
// thread) in the block that arrived last, after it stored the sums in st->red.
__device__ bool reduce_partials(double* part, int nq, const int* q, const double* v, KrylovState* st, double* sh) {
  __shared__ int amlast;
  for (int k = 0; k < nq; ++k) {
    double t = block_sum(v[k], sh);
    if (threadIdx.x == 0) part[(int64_t)q[k] * kMaxRedBlocks + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) amlast = atomicAdd(&st->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
  for (int k = 0; k < nq; ++k) {
    const double* pk = part + (int64_t)q[k] * kMaxRedBlocks;
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(pk + i);
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) st->red[q[k]] = t;
  }
  if (threadIdx.x == 0) st->counter = 0;
  __syncthreads();
  return true;
}

// r = b - A x and ||r||^2; test 1: initial convergence test; test 2: end of
// an iteration of the multigrid solver (counts it, sets the loop condition)
template <int NC>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 4) k_residual_norm(SellView A, const double* __restrict__ x,
                                                           const double* __restrict__ b, double* __restrict__ r,
                                                           double* part, KrylovState* st, int test,
                                                           unsigned long long cond) {
  __shared__ double sh[40];
  pdl_wait();
  if (test == 2 && st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
  const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      double ax = sell_dot1<double>(A, slice, lane, x);
      if (row < A.n) { double ri = b[orow] - ax; r[orow] = ri; acc = fma(ri, ri, acc); }
    } else {
      double a3[3];
      sell_dot3<double>(A, slice, lane, x, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) { double ri = b[3 * orow + i] - a3[i]; r[3 * orow + i] = ri; acc = fma(ri, ri, acc); }
    }
  }
  const int q[1] = {Q_RR};
  if (reduce_partials(part, 1, q, &acc, st, sh) && test && threadIdx.x == 0) converge_step(st, test == 2, cond);
}

// x += z (z = preconditioner output, FP64 or FP32 times st->scale)
__global__ void __launch_bounds__(kBlock) k_mgi_update(int64_t n, PVec z, double* __restrict__ x, KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double zi[4], xi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { zi[k] = pv(z, j, sc); xi[k] = x[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) x[j] = xi[k] + zi[k];
    }
  }
}

// ||b_free||^2 and the initial state of the Krylov loop
__global__ void k_norm_init(int64_t n, int nc, const uint8_t* __restrict__ fix, const double* __restrict__ b,
                            double* part, KrylovState* st, double rtol, int max_it) {
  __shared__ double sh[40];
  pdl_wait();
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) {
    const uint8_t f = fix[i];
    for (int c = 0; c < nc; ++c)
      if (!((f >> c) & 1)) acc = fma(b[nc * i + c], b[nc * i + c], acc);
  }
  const int q[1] = {Q_BB};
  if (reduce_partials(part, 1, q, &acc, st, sh) && threadIdx.x == 0) {
    st->bnorm = st->red[Q_BB] > 0.0 ? sqrt(st->red[Q_BB]) : 1.0;
    st->rtol = rtol; st->max_it = max_it; st->iter = 0; st->done = 0; st->status = 0;
    st->rho = st->rho_prev = st->alpha = st->omega = 1.0; st->beta = 0.0; st->scale = 1.0; st->restart_pos = 0;
    st->inv_scale = 1.0; st->beta_next = 0.0; st->gm_inv = 0.0;
    st->gm_j = 0; st->gm_end = 0;
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ v, float* __restrict__ v32, const KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const double inv = st->inv_scale;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 + 3 < n) {
    const double2 a = *reinterpret_cast<const double2*>(v + i0), b = *reinterpret_cast<const double2*>(v + i0 + 2);
    float4 o;
    o.x = __double2float_rn(a.x * inv); o.y = __double2float_rn(a.y * inv);
    o.z = __double2float_rn(b.x * inv); o.w = __double2float_rn(b.y * inv);
    *reinterpret_cast<float4*>(v32 + i0) = o;
  } else {
    for (int64_t i = i0; i < n; ++i) v32[i] = __double2float_rn(v[i] * inv);
  }
}

// (r, z) and (q, z) for flexible CG
__global__ void __launch_bounds__(kBlock, 4) k_cg_dots(int64_t n, PVec z, const double* __restrict__ r,
                                                     const double* __restrict__ q, double* part, KrylovState* st) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double zi[4], ri[4], qi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { zi[k] = pv(z, j, sc); ri[k] = r[j]; qi[k] = q[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i + k * nthreads < n) { a = fma(ri[k], zi[k], a); c = fma(qi[k], zi[k], c); }
  }
  const int qs[2] = {Q_RZ, Q_QZ};
  const double v[2] = {a, c};
  // Polak-Ribiere: beta = (z_new, r_new - r_old) / rho_old, r_new - r_old = -alpha q
  if (reduce_partials(part, 2, qs, v, st, sh) && threadIdx.x == 0)
    st->beta_next = -st->alpha * st->red[Q_QZ] / st->rho_prev;
}

__global__ void __launch_bounds__(kBlock) k_cg_update_p(int64_t n, PVec z, double* __restrict__ p, KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const double rz = st->red[Q_RZ];
  const bool first = st->iter == st->restart_pos;
  const double beta = first ? 0.0 : st->beta_next;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double zi[4], pi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { zi[k] = pv(z, j, sc); pi[k] = first ? 0.0 : p[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) p[j] = first ? zi[k] : fma(beta, pi[k], zi[k]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { st->rho = rz; st->beta = beta; }
}

// out = A p (p given as PVec), partial of (w, out) (w = p when w == nullptr)
template <int NC, bool F32>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 4) k_spmv_dot(SellView A, PVec p, const double* __restrict__ w,
                                                      double* __restrict__ out, double* part, int qk,
                                                      KrylovState* st) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
  const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      const double ax = F32 ? sell_dot1x<double>(A.sptr, A.col, (const double*)A.val, slice, lane, p.f, A.col16) * sc
                            : sell_dot1<double>(A, slice, lane, p.d);
      if (row < A.n) {
        out[orow] = ax;
        acc = fma(w ? w[orow] : (F32 ? (double)p.f[orow] * sc : p.d[orow]), ax, acc);
      }
    } else {
      double a3[3];
      if (F32) sell_dot3<double, float>(A, slice, lane, p.f, 1.0, a3);
      else sell_dot3<double>(A, slice, lane, p.d, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) {
          const double y = F32 ? a3[i] * sc : a3[i];
          out[3 * orow + i] = y;
          acc = fma(w ? w[3 * orow + i] : (F32 ? (double)p.f[3 * orow + i] * sc : p.d[3 * orow + i]), y, acc);
        }
    }
  }
  const int qs[1] = {qk};
  // CG: alpha = (r, z) / (p, A p); BiCGStab: alpha = rho / (r^, A p^)
  if (reduce_partials(part, 1, qs, &acc, st, sh) && threadIdx.x == 0) st->alpha = st->rho / st->red[qk];
}

// x += alpha p, r -= alpha q, ||r||^2, then (last block) the convergence test
__global__ void __launch_bounds__(kBlock, 4) k_cg_update_xr(int64_t n, const double* __restrict__ p,
                                                          const double* __restrict__ q, double* __restrict__ x,
                                                          double* __restrict__ r, double* part, KrylovState* st,
                                                          unsigned long long cond) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) {   // already converged: the device loop must still end here
    if (blockIdx.x == 0 && threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  const double pq = st->red[Q_PQ];
  const double alpha = st->alpha;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double pi[4], qi[4], xi[4], ri[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { pi[k] = p[j]; qi[k] = q[j]; xi[k] = x[j]; ri[k] = r[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) {
        x[j] = fma(alpha, pi[k], xi[k]);
        const double rr = fma(-alpha, qi[k], ri[k]);
        r[j] = rr;
        acc = fma(rr, rr, acc);
      }
    }
  }
  const int qs[1] = {Q_RR};
  if (reduce_partials(part, 1, qs, &acc, st, sh) && threadIdx.x == 0) {
    st->rho_prev = st->rho;
    if (pq == 0.0) st->status = -5;
    converge_step(st, true, cond);
  }
}

// BiCGStab (van der Vorst), right preconditioned.  p = r + beta (p - omega v);
// with p32 also the FP32 preconditioner input p / scale.
__global__ void __launch_bounds__(kBlock) k_bicg_p(int64_t n, const double* __restrict__ r,
                                                    const double* __restrict__ v, double* __restrict__ p,
                                                    float* __restrict__ p32, KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const double rho = st->red[Q_RHR];
  const bool first = st->iter == st->restart_pos;
  const double beta = first ? 0.0 : st->beta_next;   // (rho / rho_prev) (alpha / omega)
  const double om = st->omega;
  const double inv = st->inv_scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double ri[4], vi[4], pi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { ri[k] = r[j]; vi[k] = first ? 0.0 : v[j]; pi[k] = first ? 0.0 : p[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) {
        const double pn = first ? ri[k] : fma(beta, fma(-om, vi[k], pi[k]), ri[k]);
        p[j] = pn;
        if (p32) p32[j] = __double2float_rn(pn * inv);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rho = rho;
    st->beta = beta;
    if (rho == 0.0) st->status = -5;
  }
}

// s = r - alpha v (alpha = rho / (rhat, v)); with s32 the FP32 copy s / scale
__global__ void __launch_bounds__(kBlock) k_bicg_s(int64_t n, const double* __restrict__ r,
                                                    const double* __restrict__ v, double* __restrict__ s,
                                                    float* __restrict__ s32, KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const double rhv = st->red[Q_RHV];
  const double alpha = st->alpha;     // rho / rhv
  const double inv = st->inv_scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * nthreads) {
    double ri[4], vi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) { ri[k] = r[j]; vi[k] = v[j]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) {
        const double si = fma(-alpha, vi[k], ri[k]);
        s[j] = si;
        if (s32) s32[j] = __double2float_rn(si * inv);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && rhv == 0.0) st->status = -5;
}

// t = A sh, partials (t, s) and (t, t)
template <int NC, bool F32>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 4) k_spmv_2dots(SellView A, PVec shv, const double* __restrict__ sv,
                                                        double* __restrict__ t, double* part, KrylovState* st) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double a = 0.0, c = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
  const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      const double ax = F32 ? sell_dot1x<double>(A.sptr, A.col, (const double*)A.val, slice, lane, shv.f, A.col16) * sc
                            : sell_dot1<double>(A, slice, lane, shv.d);
      if (row < A.n) { t[orow] = ax; a = fma(ax, sv[orow], a); c = fma(ax, ax, c); }
    } else {
      double a3[3];
      if (F32) sell_dot3<double, float>(A, slice, lane, shv.f, 1.0, a3);
      else sell_dot3<double>(A, slice, lane, shv.d, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) {
          const double y = F32 ? a3[i] * sc : a3[i];
          t[3 * orow + i] = y;
          a = fma(y, sv[3 * orow + i], a);
          c = fma(y, y, c);
        }
    }
  }
  const int qs[2] = {Q_TS, Q_TT};
  const double v[2] = {a, c};
  if (reduce_partials(part, 2, qs, v, st, sh) && threadIdx.x == 0) {
    const double ts = st->red[Q_TS], tt = st->red[Q_TT];
    st->omega = tt > 0.0 ? ts / tt : 0.0;
  }
}

// omega = (t,s)/(t,t); x += alpha ph + omega sh; r = s - omega t; (r,r), (rhat,r)
__global__ void __launch_bounds__(kBlock, 4) k_bicg_x(int64_t n, PVec ph, PVec shv, const double* __restrict__ sv,
                                                    const double* __restrict__ t, const double* __restrict__ rhat,
                                                    double* __restrict__ x, double* __restrict__ r, double* part,
                                                    KrylovState* st, unsigned long long cond) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) {   // already converged: the device loop must still end here
    if (blockIdx.x == 0 && threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  const double tt = st->red[Q_TT];
  const double om = st->omega;        // (t, s) / (t, t)
  const double alpha = st->alpha;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * nthreads) {
    double phi[2], shi[2], si[2], ti[2], rh[2], xi[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) {
        phi[k] = pv(ph, j, sc); shi[k] = pv(shv, j, sc); si[k] = sv[j]; ti[k] = t[j]; rh[k] = rhat[j]; xi[k] = x[j];
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t j = i + k * nthreads;
      if (j < n) {
        x[j] = fma(om, shi[k], fma(alpha, phi[k], xi[k]));
        const double rr = fma(-om, ti[k], si[k]);
        r[j] = rr;
        a = fma(rr, rr, a);
        c = fma(rh[k], rr, c);
      }
    }
  }
  const int qs[2] = {Q_RR, Q_RHR};
  const double v[2] = {a, c};
  if (reduce_partials(part, 2, qs, v, st, sh) && threadIdx.x == 0) {
    st->beta_next = (st->red[Q_RHR] / st->rho) * (alpha / om);
    st->rho_prev = st->rho;
    if (!(tt > 0.0) || om == 0.0) st->status = -5;
    converge_step(st, true, cond);
  }
}


// ------------------------------------------------------------------ GMRES
// Flexible GMRES(m) with right preconditioning: Arnoldi on A M^-1 with the
// preconditioned vectors z_j kept (Saad 2003, Sec. 9.4.1), orthogonalisation
// by classical Gram-Schmidt applied twice (two sweeps of one block-dot pass
// and one update pass each), Hessenberg QR by Givens rotations (Sec. 6.5.3).
// The Hessenberg matrix, the rotations and the small triangular solve stay on
// the device.  Phase flags in the state gate the cycle-start and cycle-end
// kernels, so every Arnoldi step is the same fixed kernel sequence.
__global__ void __launch_bounds__(kBlock) k_gm_start(int64_t n, const double* __restrict__ r, float* __restrict__ v32,
                                                     double* __restrict__ v64, GmresView G, KrylovState* st) {
  pdl_wait();
  if (st->done || st->gm_j != 0) return;
  const double rn = st->rnorm;                        // sqrt(red[Q_RR]), set with inv_scale = 1 / rn
  const double inv = rn > 0.0 ? st->inv_scale : 0.0;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) {
    const double v = r[i] * inv;
    G.V[i] = v;
    if (v32) v32[i] = __double2float_rn(v);
    if (v64) v64[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x <= G.m) G.g[threadIdx.x] = threadIdx.x == 0 ? rn : 0.0;
}

template <int NC, bool F32>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 4) k_gm_spmv(SellView A, PVec z, double* __restrict__ w,
                                                                      GmresView G, KrylovState* st) {
  pdl_wait();
  if (st->done) return;
  const int j = st->gm_j;
  const int64_t n = A.n * NC;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
  const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      const double ax = F32 ? sell_dot1x<double>(A.sptr, A.col, (const double*)A.val, slice, lane, z.f, A.col16)
                            : sell_dot1<double>(A, slice, lane, z.d);
      if (row < A.n) {
        w[orow] = ax;
        if (F32) G.Z32[(int64_t)j * n + orow] = z.f[orow];
        else G.Z64[(int64_t)j * n + orow] = z.d[orow];
      }
    } else {
      double a3[3];
      if (F32) sell_dot3<double, float>(A, slice, lane, z.f, 1.0, a3);
      else sell_dot3<double>(A, slice, lane, z.d, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) {
          w[3 * orow + i] = a3[i];
          if (F32) G.Z32[(int64_t)j * n + 3 * orow + i] = z.f[3 * orow + i];
          else G.Z64[(int64_t)j * n + 3 * orow + i] = z.d[3 * orow + i];
        }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && F32) G.zs[j] = 1.0;
}

// partial dots (v_i, w) for the vectors i = 4 blockIdx.y + k <= j: w is read
// once per four basis vectors, and a partial chunk runs a loop of its own
// length (no idle FP64 multiply-adds)
constexpr int kGmDotVecs = 4;
template <int K>
__device__ __forceinline__ void gm_dots_k(int64_t n, const double* __restrict__ w, const double* __restrict__ v,
                                          double (&acc)[kGmDotVecs]) {
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += nthreads) {
    const double we = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(v[(int64_t)k * n + e], we, acc[k]);
  }
}

__global__ void __launch_bounds__(kBlock) k_gm_dots(int64_t n, const double* __restrict__ w, GmresView G,
                                                    KrylovState* st) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const int i0 = kGmDotVecs * blockIdx.y, j = st->gm_j;
  if (i0 > j) return;
  const int kn = min(kGmDotVecs, j + 1 - i0);
  const double* __restrict__ v = G.V + (int64_t)i0 * n;
  double acc[kGmDotVecs] = {0.0, 0.0, 0.0, 0.0};
  switch (kn) {
    case 4: gm_dots_k<4>(n, w, v, acc); break;
    case 3: gm_dots_k<3>(n, w, v, acc); break;
    case 2: gm_dots_k<2>(n, w, v, acc); break;
    default: gm_dots_k<1>(n, w, v, acc); break;
  }
#pragma unroll
  for (int k = 0; k < kGmDotVecs; ++k) {
    if (k >= kn) break;
    const double t = block_sum(acc[k], sh);
    if (threadIdx.x == 0) G.part[(int64_t)(i0 + k) * kMaxRedBlocks + blockIdx.x] = t;
  }
}

// h_i = sum of the partials (one block per i), added into column j of H
__global__ void k_gm_reduce(GmresView G, KrylovState* st, int nparts, int pass) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const int i = blockIdx.x, j = st->gm_j;
  if (i > j) return;
  const double* p = G.part + (int64_t)i * kMaxRedBlocks;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) acc += p[k];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    G.hv[i] = t;
    double* Hc = G.H + (int64_t)j * (G.m + 1);
    Hc[i] = pass == 0 ? t : Hc[i] + t;
  }
}

// w -= sum_{i <= j} h_i v_i ; on the second sweep also ||w||^2 -> red[Q_SS]
__global__ void __launch_bounds__(kBlock) k_gm_axpy(int64_t n, double* __restrict__ w, GmresView G, KrylovState* st,
                                                    double* part, int pass) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) return;
  const int j = st->gm_j;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += nthreads) {
    double we = w[e];
    for (int i = 0; i <= j; ++i) we = fma(-G.hv[i], G.V[(int64_t)i * n + e], we);
    w[e] = we;
    acc = fma(we, we, acc);
  }
  if (pass == 1) {
    const int q[1] = {Q_SS};
    reduce_partials(part, 1, q, &acc, st, sh);
  }
}

// Givens rotations on column j, new rotation, residual estimate |g_{j+1}|;
// at the end of a cycle the triangular system H y = g is solved here.
__global__ void k_gm_givens(GmresView G, KrylovState* st) {
  pdl_wait();
  if (st->done || threadIdx.x != 0) return;
  const int j = st->gm_j, m = G.m;
  double* Hc = G.H + (int64_t)j * (m + 1);
  Hc[j + 1] = sqrt(st->red[Q_SS]);
  for (int i = 0; i < j; ++i) {
    const double t = G.cs[i] * Hc[i] + G.sn[i] * Hc[i + 1];
    Hc[i + 1] = -G.sn[i] * Hc[i] + G.cs[i] * Hc[i + 1];
    Hc[i] = t;
  }
  const double den = hypot(Hc[j], Hc[j + 1]);
  const double c = den > 0.0 ? Hc[j] / den : 1.0, sn = den > 0.0 ? Hc[j + 1] / den : 0.0;
  G.cs[j] = c;
  G.sn[j] = sn;
  st->red[Q_TT] = Hc[j + 1];           // h_{j+1,j} before the rotation: norm of the new basis vector
  st->gm_inv = 1.0 / Hc[j + 1];
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  G.g[j + 1] = -sn * G.g[j];
  G.g[j] = c * G.g[j];
  st->iter += 1;
  const double est = fabs(G.g[j + 1]);
  const bool end = est <= st->rtol * st->bnorm || j + 1 >= m || st->iter >= st->max_it || !(den > 0.0) ||
                   !isfinite(est);
  st->gm_end = end ? 1 : 0;
  if (end) {
    const int k = j + 1;
    for (int r = k - 1; r >= 0; --r) {
      double acc = G.g[r];
      for (int c2 = r + 1; c2 < k; ++c2) acc -= G.H[(int64_t)c2 * (m + 1) + r] * G.y[c2];
      G.y[r] = acc / G.H[(int64_t)r * (m + 1) + r];
    }
    st->restart_pos = k;               // number of columns used in this cycle
  }
}

__global__ void __launch_bounds__(kBlock) k_gm_next(int64_t n, const double* __restrict__ w, float* __restrict__ v32,
                                                    double* __restrict__ v64, GmresView G, KrylovState* st) {
  pdl_wait();
  if (st->done || st->gm_end) return;
  const int j = st->gm_j;
  const double inv = st->gm_inv;      // 1 / h_{j+1,j}
  double* vn = G.V + (int64_t)(j + 1) * n;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += nthreads) {
    const double v = w[e] * inv;
    vn[e] = v;
    if (v32) v32[e] = __double2float_rn(v);
    if (v64) v64[e] = v;
  }
}

// advance the column counter once every block of k_gm_next has read it
__global__ void k_gm_advance(KrylovState* st) {
  pdl_wait();
  if (threadIdx.x != 0 || st->done) return;
  if (!st->gm_end) st->gm_j += 1;
}

__global__ void __launch_bounds__(kBlock) k_gm_update_x(int64_t n, double* __restrict__ x, GmresView G,
                                                        KrylovState* st) {
  pdl_wait();
  if (st->done || !st->gm_end) return;
  const int k = st->restart_pos;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += nthreads) {
    double xe = x[e];
    for (int i = 0; i < k; ++i) {
      const double zi = G.Z32 ? (double)G.Z32[(int64_t)i * n + e] * G.zs[i] : G.Z64[(int64_t)i * n + e];
      xe = fma(G.y[i], zi, xe);
    }
    x[e] = xe;
  }
}

// cycle end: true residual, convergence test, next cycle starts at column 0
template <int NC>
__global__ void __launch_bounds__(kBlock, NC == 1 ? 6 : 4) k_gm_residual(SellView A, const double* __restrict__ x,
                                                                          const double* __restrict__ b,
                                                                          double* __restrict__ r, double* part,
                                                                          KrylovState* st, unsigned long long cond) {
  __shared__ double sh[40];
  pdl_wait();
  if (st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  if (!st->gm_end) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 1u);
    return;
  }
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
  const int64_t orow = srow<0>(A, row);
    if (NC == 1) {
      double ax = sell_dot1<double>(A, slice, lane, x);
      if (row < A.n) { double ri = b[orow] - ax; r[orow] = ri; acc = fma(ri, ri, acc); }
    } else {
      double a3[3];
      sell_dot3<double>(A, slice, lane, x, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) { double ri = b[3 * orow + i] - a3[i]; r[3 * orow + i] = ri; acc = fma(ri, ri, acc); }
    }
  }
  const int q[1] = {Q_RR};
  if (reduce_partials(part, 1, q, &acc, st, sh) && threadIdx.x == 0) {
    const int iters = st->iter;
    converge_step(st, false, cond);     // sets done / status / the while condition
    st->iter = iters;
    st->gm_j = 0;
    st->gm_end = 0;
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
static bool g_pdl = true;
void set_pdl(bool on) { g_pdl = on; }
thread_local LaunchProfiler* t_prof = nullptr;
thread_local int t_prof_level = -1;

template <typename... KArgs, typename... Args>
static void launch_ex(cudaLaunchConfig_t& cfg, void (*kernel)(KArgs...), Args... args) {
  if (t_prof) t_prof->before((const void*)kernel, cfg.stream);
  cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
  if (t_prof) t_prof->after(cfg.stream);
}



template <typename... KArgs, typename... Args>
static void launch(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  int na = 0;
  if (g_pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  launch_ex(cfg, kernel, args...);
}

// Row grids stop at 1216 blocks (152 SMs x 8).  A kernel with more than 32
// registers per thread holds fewer than 8 blocks of kBlock threads per SM;
// where that leaves a last wave filling less than half of the SMs' block
// slots (6 per SM: 1216 = 1.33 waves), the grid-stride kernel gets one full
// wave instead.  Applied to the scalar row kernels and the vector kernels;
// the 3x3-block kernels keep their grid (one wave was measured slower there:
// their rows of 9 to 27 blocks balance better over two waves).
static int wave_grid(const void* fn, int grid) {
  thread_local std::map<const void*, int> cap;
  auto it = cap.find(fn);
  int c;
  if (it != cap.end()) {
    c = it->second;
  } else {
    int dev = 0, sms = 0, occ = 0;
    c = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, 0) == cudaSuccess && occ > 0 && sms > 0)
      c = sms * occ;
    cap[fn] = c;
  }
  return (c > 0 && grid > c && 2 * grid < 3 * c) ? c : grid;
}

// launch() for grid-stride kernels over rows or vector entries
template <typename... KArgs, typename... Args>
static void launch_rows(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  launch(kernel, wave_grid((const void*)kernel, grid), s, args...);
}

// launch_rows for scalar kernels (NC = 1), launch() for 3x3-block ones
template <int NC, typename... KArgs, typename... Args>
static void launch_nc(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  if constexpr (NC == 1) launch_rows(kernel, grid, s, args...);
  else launch(kernel, grid, s, args...);
}

int grid_for_rows(int64_t rows) {
  int64_t g = (rows + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  return (int)(g > kMaxRedBlocks ? kMaxRedBlocks : g);
}
int grid_for_vec(int64_t n) { return grid_for_rows(n); }

static int grid_sell(int64_t nslices) { return grid_for_rows(nslices * 32); }

template <typename T, typename V, int NC, int TPR>
void launch_smooth_k(const SellView& A, int g, cudaStream_t s, const T* x, const T* b, const T* Sinv, T* xo, T om,
                     bool from_zero, const int* done, double* xo64, const double* scale) {
  if constexpr (std::is_same<T, float>::value && NC == 1 && TPR == 1) {
    if (!from_zero && A.wlo) {   // x staged per window
      launch_rows(k_smooth_staged<V>, g, s, A, x, b, Sinv, xo, om, done, xo64, scale);
      return;
    }
  }
  if (from_zero) launch_nc<NC>(k_smooth<T, V, NC, true, TPR>, g, s, A, x, b, Sinv, xo, om, done, xo64, scale);
  else launch_nc<NC>(k_smooth<T, V, NC, false, TPR>, g, s, A, x, b, Sinv, xo, om, done, xo64, scale);
}

template <typename T, typename V>
void launch_smooth_v(const SellView& A, int nc, int g, cudaStream_t s, const T* x, const T* b, const T* Sinv, T* xo,
                     T om, bool from_zero, const int* done, double* xo64, const double* scale) {
  const bool four = A.tpr == 4;
  if (nc == 1) {
    if (four) launch_smooth_k<T, V, 1, 4>(A, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
    else launch_smooth_k<T, V, 1, 1>(A, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
  } else {
    if (four) launch_smooth_k<T, V, 3, 4>(A, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
    else launch_smooth_k<T, V, 3, 1>(A, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
  }
}

template <typename T>
void launch_smooth(const SellView& A, int nc, const T* x, const T* b, const T* Sinv, T* xo, double omega,
                   bool from_zero, const int* done, cudaStream_t s, double* xo64, const double* scale) {
  const int g = grid_for_rows(A.nslices * 32 * A.tpr);
  const T om = (T)omega;
  if constexpr (std::is_same<T, float>::value) {
    if (A.bf16) {
      launch_smooth_v<T, __nv_bfloat16>(A, nc, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
      return;
    }
  }
  launch_smooth_v<T, T>(A, nc, g, s, x, b, Sinv, xo, om, from_zero, done, xo64, scale);
}

template <typename T, typename V, int MODE>
void launch_apply_v(const SellView& A, int nc, int g, cudaStream_t s, const T* x, const T* b, T* y, const int* done) {
  const bool four = A.tpr == 4;
  if (nc == 1) {
    if (four) launch_rows(k_apply<T, V, 1, MODE, 4>, g, s, A, x, b, y, done);
    else launch_rows(k_apply<T, V, 1, MODE, 1>, g, s, A, x, b, y, done);
  } else {
    if (four) launch(k_apply<T, V, 3, MODE, 4>, g, s, A, x, b, y, done);
    else launch(k_apply<T, V, 3, MODE, 1>, g, s, A, x, b, y, done);
  }
}

template <typename T>
void launch_residual(const SellView& A, int nc, const T* x, const T* b, T* r, const int* done, cudaStream_t s) {
  const int g = grid_for_rows(A.nslices * 32 * A.tpr);
  if constexpr (std::is_same<T, float>::value) {
    if (A.bf16) {
      launch_apply_v<T, __nv_bfloat16, 1>(A, nc, g, s, x, b, r, done);
      return;
    }
  }
  launch_apply_v<T, T, 1>(A, nc, g, s, x, b, r, done);
}

template <typename T>
void launch_matvec(const SellView& A, int nc, const T* x, T* y, const int* done, cudaStream_t s) {
  const int g = grid_for_rows(A.nslices * 32 * A.tpr);
  if constexpr (std::is_same<T, float>::value) {
    if (A.bf16) {
      launch_apply_v<T, __nv_bfloat16, 0>(A, nc, g, s, x, (const T*)nullptr, y, done);
      return;
    }
  }
  launch_apply_v<T, T, 0>(A, nc, g, s, x, (const T*)nullptr, y, done);
}

template <typename T>
void launch_restrict(const TransferView& R, int nc, const T* r, T* d, const T* Sinv, T* x0, double omega,
                     const int* done, cudaStream_t s) {
  const int g = grid_sell(R.nslices);
  const T om = (T)omega;
  if (x0) {
    if (nc == 1) launch_rows(k_restrict<T, 1, true>, g, s, R, r, d, Sinv, x0, om, done);
    else launch(k_restrict<T, 3, true>, g, s, R, r, d, Sinv, x0, om, done);
  } else {
    if (nc == 1) launch_rows(k_restrict<T, 1, false>, g, s, R, r, d, Sinv, x0, om, done);
    else launch(k_restrict<T, 3, false>, g, s, R, r, d, Sinv, x0, om, done);
  }
}

template <typename T>
void launch_prolong_add(const TransferView& P, int nc, const T* y, const T* xin, T* xo, const int* done,
                        cudaStream_t s) {
  const int g = grid_sell(P.nslices);
  if (nc == 1) launch_rows(k_prolong<T, 1>, g, s, P, y, xin, xo, done);
  else launch(k_prolong<T, 3>, g, s, P, y, xin, xo, done);
}

template <typename T>
void launch_vanka(const SellView& S, int nc, const T* r, const T* xin, T* xo, double omega, const int* done,
                  cudaStream_t s, double* xo64, const double* scale) {
  const int g = grid_for_rows(S.nslices * 32 * S.tpr);
  const T om = (T)omega;
  const bool four = S.tpr == 4;
  if (nc == 1) {
    if (four) launch_rows(k_vanka<T, T, 1, 4>, g, s, S, r, xin, xo, om, done, xo64, scale);
    else launch_rows(k_vanka<T, T, 1, 1>, g, s, S, r, xin, xo, om, done, xo64, scale);
  } else {
    if (four) launch(k_vanka<T, T, 3, 4>, g, s, S, r, xin, xo, om, done, xo64, scale);
    else launch(k_vanka<T, T, 3, 1>, g, s, S, r, xin, xo, om, done, xo64, scale);
  }
}

template <typename T>
void launch_coarse(const double* Ainv, int64_t n, const T* d, T* z, const int* done, cudaStream_t s) {
  int64_t g = (n + 7) / 8;
  if (g > kMaxRedBlocks) g = kMaxRedBlocks;
  launch(k_coarse<T>, (int)g, s, Ainv, n, d, z, done);
}

#define MGI_INST(T)                                                                                                \
  template void launch_smooth<T>(const SellView&, int, const T*, const T*, const T*, T*, double, bool, const int*, \
                                 cudaStream_t, double*, const double*);                                            \
  template void launch_residual<T>(const SellView&, int, const T*, const T*, T*, const int*, cudaStream_t);        \
  template void launch_matvec<T>(const SellView&, int, const T*, T*, const int*, cudaStream_t);                    \
  template void launch_restrict<T>(const TransferView&, int, const T*, T*, const T*, T*, double, const int*,       \
                                   cudaStream_t);                                                                  \
  template void launch_prolong_add<T>(const TransferView&, int, const T*, const T*, T*, const int*, cudaStream_t); \
  template void launch_coarse<T>(const double*, int64_t, const T*, T*, const int*, cudaStream_t);              \
  template void launch_vanka<T>(const SellView&, int, const T*, const T*, T*, double, const int*, cudaStream_t,   \
                                double*, const double*);
MGI_INST(double)
MGI_INST(float)
#undef MGI_INST

template <typename T, typename V, int NC, int TLM>
void launch_tail_k(cudaLaunchConfig_t& cfg, const TailParams& P, const T* b, T* out, int fd, const int* done,
                   double* o64, const double* scale) {
  if constexpr (TLM == 2 || TLM == 3) {
    static std::once_flag once;   // opt in to the large dynamic shared memory, once per instantiation
    std::call_once(once, [] {
      cudaFuncSetAttribute(k_tail<T, V, NC, TLM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
      if (TLM == 3) cudaFuncSetAttribute(k_tail<T, V, NC, TLM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
  } else {
    static std::once_flag once;   // clusters of up to 16 CTAs (beyond the portable 8)
    std::call_once(once, [] {
      cudaFuncSetAttribute(k_tail<T, V, NC, TLM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
  }
  launch_ex(cfg, k_tail<T, V, NC, TLM>, P, b, out, fd, done, o64, scale);
}

template <typename T, typename V>
void launch_tail_v(cudaLaunchConfig_t& cfg, const TailParams& P, int nc, const T* b, T* out, int fd, const int* done,
                   double* o64, const double* scale) {
  const bool staged = P.cluster == 0;
  if (nc == 1) {
    if (P.dsm) launch_tail_k<T, V, 1, 3>(cfg, P, b, out, fd, done, o64, scale);
    else if (staged) launch_tail_k<T, V, 1, 2>(cfg, P, b, out, fd, done, o64, scale);
    else launch_tail_k<T, V, 1, 1>(cfg, P, b, out, fd, done, o64, scale);
  } else {
    if (staged) launch_tail_k<T, V, 3, 2>(cfg, P, b, out, fd, done, o64, scale);
    else launch_tail_k<T, V, 3, 1>(cfg, P, b, out, fd, done, o64, scale);
  }
}

template <typename T>
void launch_tail(const TailParams& P, int nc, const T* b, T* out, bool first_done, const int* done, cudaStream_t s,
                 double* o64, const double* scale) {
  const bool staged = P.cluster == 0;
  const int cl = staged ? 1 : P.cluster;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = (staged || P.dsm) ? P.smem : 0;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (!staged) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cl;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  if (g_pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  const int fd = first_done ? 1 : 0;
  if constexpr (std::is_same<T, float>::value) {
    if (P.lv[0].A.bf16) {
      launch_tail_v<T, __nv_bfloat16>(cfg, P, nc, b, out, fd, done, o64, scale);
      return;
    }
  }
  launch_tail_v<T, T>(cfg, P, nc, b, out, fd, done, o64, scale);
}
template void launch_tail<double>(const TailParams&, int, const double*, double*, bool, const int*, cudaStream_t,
                                  double*, const double*);

// Whether this GPU schedules a cluster of `cl` tail CTAs (kTailThreads each):
// sizes above 8 are not portable and need that many SMs free in one GPC.
bool tail_cluster_fits(int cl) {
  if (cl <= 8) return true;
  static std::mutex mu;
  static std::map<int, bool> known;
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find(cl);
  if (it != known.end()) return it->second;
  const void* fn = (const void*)k_tail<float, float, 1, 1>;
  bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0;
  }
  cudaGetLastError();   // a refused query leaves no sticky error
  known[cl] = ok;
  return ok;
}
template void launch_tail<float>(const TailParams&, int, const float*, float*, bool, const int*, cudaStream_t,
                                 double*, const double*);

bool tail_dsm_fits(int cl, uint32_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, uint32_t>, bool> known;
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find({cl, smem});
  if (it != known.end()) return it->second;
  const void* fn = (const void*)k_tail<float, float, 1, 3>;
  bool ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0;
  }
  cudaGetLastError();   // a refused query leaves no sticky error
  known[{cl, smem}] = ok;
  return ok;
}

void launch_rhs(const SellView& F, int nc, const double* f, const uint8_t* fixmask, const uint8_t* dirmask,
                const double* g, double* b, cudaStream_t s) {
  launch_rows(k_rhs, grid_sell(F.nslices), s, F, nc, f, fixmask, dirmask, g, b);
}
void launch_lift(const SellView& L, int nc, const double* g, double* b, cudaStream_t s) {
  if (L.n == 0) return;
  if (nc == 1) launch_rows(k_lift<1>, grid_sell(L.nslices), s, L, g, b);
  else launch(k_lift<3>, grid_sell(L.nslices), s, L, g, b);
}
void launch_fill_hanging(const TransferView& Hc, int nc, double* x, cudaStream_t s) {
  launch_rows(k_fill_hanging, grid_sell(Hc.nslices), s, Hc, nc, x);
}
void launch_copy_fixed(int64_t n, int nc, const uint8_t* fixmask, const double* b, const double* xin, double* x,
                       cudaStream_t s) {
  launch_rows(k_copy_fixed, grid_for_rows(n), s, n, nc, fixmask, b, xin, x);
}
void launch_step_load2(int64_t n, double inv_dt, const double* u, double* v, const double* f, double* out,
                       cudaStream_t s) {
  launch_rows(k_step_load2, grid_for_rows(n), s, n, inv_dt, u, v, f, out);
}
void launch_step_velocity(int64_t n, double inv_dt, const double* u, double* v, cudaStream_t s) {
  launch_rows(k_step_velocity, grid_for_rows(n), s, n, inv_dt, u, v);
}
void launch_step_load(int64_t n, double sc, const double* theta, const double* f, double* out, cudaStream_t s) {
  launch_rows(k_step_load, grid_for_rows(n), s, n, sc, theta, f, out);
}
void launch_residual_norm(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                          KrylovState* st, int test, cudaStream_t s, unsigned long long cond) {
  const int g = grid_sell(A64.nslices);
  if (nc == 1) launch_rows(k_residual_norm<1>, g, s, A64, x, b, r, part.p, st, test, cond);
  else launch(k_residual_norm<3>, g, s, A64, x, b, r, part.p, st, test, cond);
}

void launch_norm_init(int64_t n_nodes, int nc, const uint8_t* fixmask, const double* b, Partials part,
                      KrylovState* st, double rtol, int max_it, cudaStream_t s) {
  launch_rows(k_norm_init, grid_for_rows(n_nodes), s, n_nodes, nc, fixmask, b, part.p, st, rtol, max_it);
}
static int grid_vec4(int64_t n) {  // 4 entries per thread (k_bicg_x: 2, capped grid)
  int64_t g = (n + 4 * kBlock - 1) / (4 * kBlock);
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxRedBlocks));
}
void launch_mgi_update(int64_t n, PVec z, double* x, KrylovState* st, cudaStream_t s) {
  launch_rows(k_mgi_update, grid_vec4(n), s, n, z, x, st);
}
void launch_to_f32(int64_t n, const double* v, float* v32, const KrylovState* st, cudaStream_t s) {
  int64_t g = (n + 4 * kBlock - 1) / (4 * kBlock);
  launch(k_to_f32, (int)std::max<int64_t>(1, g), s, n, v, v32, st);
}
void launch_cg_dots(int64_t n, PVec z, const double* r, const double* q, Partials part, KrylovState* st,
                    cudaStream_t s) {
  launch_rows(k_cg_dots, grid_vec4(n), s, n, z, r, q, part.p, st);
}
void launch_cg_update_p(int64_t n, PVec z, double* p, KrylovState* st, cudaStream_t s) {
  launch_rows(k_cg_update_p, grid_vec4(n), s, n, z, p, st);
}
void launch_spmv_dot(const SellView& A64, int nc, PVec p, const double* w, double* out, Partials part, int k,
                     KrylovState* st, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  if (p.f) {
    if (nc == 1) launch_rows(k_spmv_dot<1, true>, g, s, A64, p, w, out, part.p, k, st);
    else launch(k_spmv_dot<3, true>, g, s, A64, p, w, out, part.p, k, st);
  } else {
    if (nc == 1) launch_rows(k_spmv_dot<1, false>, g, s, A64, p, w, out, part.p, k, st);
    else launch(k_spmv_dot<3, false>, g, s, A64, p, w, out, part.p, k, st);
  }
}
void launch_cg_update_xr(int64_t n, const double* p, const double* q, double* x, double* r, Partials part,
                         KrylovState* st, unsigned long long cond, cudaStream_t s) {
  launch_rows(k_cg_update_xr, grid_vec4(n), s, n, p, q, x, r, part.p, st, cond);
}
void launch_bicg_p(int64_t n, const double* r, const double* v, double* p, float* p32, KrylovState* st,
                   cudaStream_t s) {
  launch_rows(k_bicg_p, grid_vec4(n), s, n, r, v, p, p32, st);
}
void launch_bicg_s(int64_t n, const double* r, const double* v, double* sv, float* s32, KrylovState* st,
                   cudaStream_t s) {
  launch_rows(k_bicg_s, grid_vec4(n), s, n, r, v, sv, s32, st);
}
void launch_spmv_2dots(const SellView& A64, int nc, PVec sh, const double* sv, double* t, Partials part,
                       KrylovState* st, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  if (sh.f) {
    if (nc == 1) launch_rows(k_spmv_2dots<1, true>, g, s, A64, sh, sv, t, part.p, st);
    else launch(k_spmv_2dots<3, true>, g, s, A64, sh, sv, t, part.p, st);
  } else {
    if (nc == 1) launch_rows(k_spmv_2dots<1, false>, g, s, A64, sh, sv, t, part.p, st);
    else launch(k_spmv_2dots<3, false>, g, s, A64, sh, sv, t, part.p, st);
  }
}
void launch_bicg_x(int64_t n, PVec ph, PVec sh, const double* sv, const double* t, const double* rhat, double* x,
                   double* r, Partials part, KrylovState* st, unsigned long long cond, cudaStream_t s) {
  launch_rows(k_bicg_x, grid_vec4(n), s, n, ph, sh, sv, t, rhat, x, r, part.p, st, cond);
}

void launch_cond_reset(unsigned long long cond, cudaStream_t s) { launch(k_cond_reset, 1, s, cond); }

// ---- GMRES launchers
void launch_gm_start(int64_t n, const double* r, float* v32, double* v64, GmresView G, KrylovState* st,
                     cudaStream_t s) {
  launch_rows(k_gm_start, grid_for_rows(n), s, n, r, v32, v64, G, st);
}
void launch_gm_spmv(const SellView& A64, int nc, PVec z, double* w, GmresView G, KrylovState* st, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  if (z.f) {
    if (nc == 1) launch_rows(k_gm_spmv<1, true>, g, s, A64, z, w, G, st);
    else launch(k_gm_spmv<3, true>, g, s, A64, z, w, G, st);
  } else {
    if (nc == 1) launch_rows(k_gm_spmv<1, false>, g, s, A64, z, w, G, st);
    else launch(k_gm_spmv<3, false>, g, s, A64, z, w, G, st);
  }
}
// an empty kernel: the per-launch floor of the per-kernel event timing
__global__ void k_prof_empty() { pdl_wait(); }
void launch_prof_empty(cudaStream_t s) { launch(k_prof_empty, 1, s); }

void launch_gm_orth(int64_t n, double* w, GmresView G, KrylovState* st, int pass, Partials part, cudaStream_t s) {
  const int gx = grid_vec4(n);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)gx, (unsigned)((G.m + kGmDotVecs) / kGmDotVecs));
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 1 : 0;
    launch_ex(cfg, k_gm_dots, n, (const double*)w, G, st);
  }
  launch(k_gm_reduce, G.m + 1, s, G, st, gx, pass);
  launch_rows(k_gm_axpy, grid_for_rows(n), s, n, w, G, st, part.p, pass);
}
void launch_gm_givens(GmresView G, KrylovState* st, cudaStream_t s) { launch(k_gm_givens, 1, s, G, st); }
void launch_gm_next(int64_t n, const double* w, float* v32, double* v64, GmresView G, KrylovState* st,
                    cudaStream_t s) {
  launch_rows(k_gm_next, grid_for_rows(n), s, n, w, v32, v64, G, st);
  launch(k_gm_advance, 1, s, st);
}
void launch_gm_update_x(int64_t n, double* x, GmresView G, KrylovState* st, cudaStream_t s) {
  launch_rows(k_gm_update_x, grid_for_rows(n), s, n, x, G, st);
}
void launch_gm_residual(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                        KrylovState* st, unsigned long long cond, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  if (nc == 1) launch_rows(k_gm_residual<1>, g, s, A64, x, b, r, part.p, st, cond);
  else launch(k_gm_residual<3>, g, s, A64, x, b, r, part.p, st, cond);
}

}  // namespace mgi
