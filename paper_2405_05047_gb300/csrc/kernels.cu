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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "kernels.h"

namespace mgi {

namespace {

__device__ __forceinline__ bool stopped(const int* done) { return done != nullptr && *(volatile const int*)done; }

template <typename T>
__device__ __forceinline__ T fmad(T a, T b, T c);
template <>
__device__ __forceinline__ double fmad<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmad<float>(float a, float b, float c) { return fmaf(a, b, c); }

// Warp + block sum in a fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

// Sum of the first n partials of one quantity, identical in every block;
// result broadcast to all threads.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  double t = block_sum(v, sh);
  __syncthreads();
  if (threadIdx.x == 0) sh[32] = t;
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// y_row = sum_j A(row, j) x_j for a scalar SELL row (thread = row).
template <typename T>
__device__ __forceinline__ T sell_dot1(const SellView& A, int64_t slice, int lane, const T* __restrict__ x) {
  const int64_t s0 = A.sptr[slice] + lane, s1 = A.sptr[slice + 1];
  const T* __restrict__ val = (const T*)A.val;
  T acc = T(0);
  int64_t o = s0;
  for (; o + 96 < s1; o += 128) {
    const int c0 = __ldg(A.col + o), c1 = __ldg(A.col + o + 32), c2 = __ldg(A.col + o + 64),
              c3 = __ldg(A.col + o + 96);
    const T v0 = __ldg(val + o), v1 = __ldg(val + o + 32), v2 = __ldg(val + o + 64), v3 = __ldg(val + o + 96);
    const T x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
    acc = fmad(v0, x0, acc);
    acc = fmad(v1, x1, acc);
    acc = fmad(v2, x2, acc);
    acc = fmad(v3, x3, acc);
  }
  for (; o < s1; o += 32) acc = fmad(__ldg(val + o), __ldg(x + __ldg(A.col + o)), acc);
  return acc;
}

// acc[0..2] = sum_j A(row, j) x_j for a 3x3-block SELL row.
template <typename T, typename XT>
__device__ __forceinline__ void sell_dot3(const SellView& A, int64_t slice, int lane, const XT* __restrict__ x,
                                          double xs, T acc[3]) {
  const int64_t s0 = A.sptr[slice], s1 = A.sptr[slice + 1];
  const T* __restrict__ val = (const T*)A.val;
  acc[0] = acc[1] = acc[2] = T(0);
  for (int64_t g = s0; g < s1; g += 32) {
    const int c = __ldg(A.col + g + lane);
    const T* __restrict__ v = val + g * 9 + lane;
    const T x0 = (T)((double)__ldg(x + 3 * c) * xs), x1 = (T)((double)__ldg(x + 3 * c + 1) * xs),
            x2 = (T)((double)__ldg(x + 3 * c + 2) * xs);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = acc[i];
      a = fmad(__ldg(v + (3 * i + 0) * 32), x0, a);
      a = fmad(__ldg(v + (3 * i + 1) * 32), x1, a);
      a = fmad(__ldg(v + (3 * i + 2) * 32), x2, a);
      acc[i] = a;
    }
  }
}

template <typename T>
__device__ __forceinline__ void sell_dot3(const SellView& A, int64_t slice, int lane, const T* __restrict__ x,
                                          T acc[3]) {
  const int64_t s0 = A.sptr[slice], s1 = A.sptr[slice + 1];
  const T* __restrict__ val = (const T*)A.val;
  acc[0] = acc[1] = acc[2] = T(0);
  for (int64_t g = s0; g < s1; g += 32) {
    const int c = __ldg(A.col + g + lane);
    const T* __restrict__ v = val + g * 9 + lane;
    const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = acc[i];
      a = fmad(__ldg(v + (3 * i + 0) * 32), x0, a);
      a = fmad(__ldg(v + (3 * i + 1) * 32), x1, a);
      a = fmad(__ldg(v + (3 * i + 2) * 32), x2, a);
      acc[i] = a;
    }
  }
}

// ------------------------------------------------------------------ level ops
// x_out = x + omega S (b - A x)  (Sec. 4.1.4), S = inverse diagonal block.
template <typename T, int NC, bool FROM_ZERO>
__global__ void __launch_bounds__(kBlock) k_smooth(SellView A, const T* __restrict__ x, const T* __restrict__ b,
                                                    const T* __restrict__ Sinv, T* __restrict__ xo, T omega,
                                                    const int* done) {
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    if (NC == 1) {
      T r = FROM_ZERO ? T(0) : sell_dot1<T>(A, slice, lane, x);
      if (row < A.n) {
        const T bi = b[row];
        if (FROM_ZERO) xo[row] = omega * Sinv[row] * bi;
        else xo[row] = fmad(omega * Sinv[row], bi - r, x[row]);
      }
    } else {
      T acc[3] = {T(0), T(0), T(0)};
      if (!FROM_ZERO) sell_dot3<T>(A, slice, lane, x, acc);
      if (row < A.n) {
        T res[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) res[i] = b[3 * row + i] - acc[i];
        const T* S = Sinv + 9 * row;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T c = S[3 * i] * res[0];
          c = fmad(S[3 * i + 1], res[1], c);
          c = fmad(S[3 * i + 2], res[2], c);
          xo[3 * row + i] = FROM_ZERO ? omega * c : fmad(omega, c, x[3 * row + i]);
        }
      }
    }
  }
}

template <typename T, int NC, int MODE>   // MODE 0: y = A x; 1: y = b - A x
__global__ void __launch_bounds__(kBlock) k_apply(SellView A, const T* __restrict__ x, const T* __restrict__ b,
                                                   T* __restrict__ y, const int* done) {
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    if (NC == 1) {
      T r = sell_dot1<T>(A, slice, lane, x);
      if (row < A.n) y[row] = MODE ? b[row] - r : r;
    } else {
      T acc[3];
      sell_dot3<T>(A, slice, lane, x, acc);
      if (row < A.n)
#pragma unroll
        for (int i = 0; i < 3; ++i) y[3 * row + i] = MODE ? b[3 * row + i] - acc[i] : acc[i];
    }
  }
}

// d_j = sum_i R(j,i) r_i (R = P^T stored as its own gather matrix: no atomics)
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock) k_restrict(TransferView R, const T* __restrict__ r, T* __restrict__ d,
                                                      const int* done) {
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < R.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    for (int64_t o = R.sptr[slice] + lane; o < R.sptr[slice + 1]; o += 32) {
      const T w = (T)__ldg(R.w + o);
      const int j = __ldg(R.col + o);
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = fmad(w, __ldg(r + (int64_t)NC * j + c), acc[c]);
    }
    if (row < R.n)
#pragma unroll
      for (int c = 0; c < NC; ++c) d[NC * row + c] = acc[c];
  }
}

// x_out_i = x_in_i + sum_j P(i,j) y_j   (Algorithm "Geometric multigrid solver", Step 4)
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock) k_prolong(TransferView P, const T* __restrict__ y, const T* xin, T* xo,
                                                     const int* done) {
  if (stopped(done)) return;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < P.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    for (int64_t o = P.sptr[slice] + lane; o < P.sptr[slice + 1]; o += 32) {
      const T w = (T)__ldg(P.w + o);
      const int j = __ldg(P.col + o);
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = fmad(w, __ldg(y + (int64_t)NC * j + c), acc[c]);
    }
    if (row < P.n)
#pragma unroll
      for (int c = 0; c < NC; ++c) xo[NC * row + c] = xin[NC * row + c] + acc[c];
  }
}

// z = A_0^{-1} d with the FP64 inverse of the coarse matrix; one warp per row.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_coarse(const double* __restrict__ Ainv, int64_t n, const T* __restrict__ d,
                                                    T* __restrict__ z, const int* done) {
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
__global__ void k_rhs(SellView F, int nc, const double* __restrict__ f, const uint8_t* __restrict__ fix,
                      double* __restrict__ b) {
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
      for (int c = 0; c < nc; ++c) b[nc * row + c] = ((fix[row] >> c) & 1) ? 0.0 : acc[c];
  }
}

// x_i = sum_j H(i,j) x_j on hanging rows (H restricted to hanging rows;
// row i of the view is node Hc.rowmap...); here the view rows are all nodes
// and regular rows are empty.
__global__ void k_fill_hanging(TransferView Hc, int nc, double* x) {
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
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    for (int c = 0; c < nc; ++c) x[nc * i + c] = ((fix[i] >> c) & 1) ? b[nc * i + c] : xin[nc * i + c];
}

__global__ void k_norm_free(int64_t n, int nc, const uint8_t* __restrict__ fix, const double* __restrict__ b,
                            double* __restrict__ part) {
  __shared__ double sh[40];
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    for (int c = 0; c < nc; ++c)
      if (!((fix[i] >> c) & 1)) acc = fma(b[nc * i + c], b[nc * i + c], acc);
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// ------------------------------------------------------------------ Krylov
// All Krylov kernels run one thread per node (nc dofs) with the same grid as
// the finest-level SpMV, so that every reduction has the same partial count.
__device__ __forceinline__ double pv(const PVec& p, int64_t i, double scale) {
  return p.f ? (double)p.f[i] * scale : p.d[i];
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_residual_norm(SellView A, const double* __restrict__ x,
                                                           const double* __restrict__ b, double* __restrict__ r,
                                                           double* __restrict__ part) {
  __shared__ double sh[40];
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    if (NC == 1) {
      double ax = sell_dot1<double>(A, slice, lane, x);
      if (row < A.n) { double ri = b[row] - ax; r[row] = ri; acc = fma(ri, ri, acc); }
    } else {
      double a3[3];
      sell_dot3<double>(A, slice, lane, x, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) { double ri = b[3 * row + i] - a3[i]; r[3 * row + i] = ri; acc = fma(ri, ri, acc); }
    }
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_init_state(KrylovState* st, const double* part_bb, int nred, double rtol, int max_it) {
  __shared__ double sh[40];
  double bb = sum_partials(part_bb, nred, sh);
  if (threadIdx.x == 0) {
    st->bnorm = bb > 0.0 ? sqrt(bb) : 1.0;
    st->rtol = rtol;
    st->max_it = max_it;
    st->iter = 0;
    st->done = 0;
    st->status = 0;
    st->rho = st->rho_prev = st->alpha = st->omega = 1.0;
    st->beta = 0.0;
    st->scale = 1.0;
    st->restart_pos = 0;
  }
}

__global__ void k_finalize(const double* part_rr, int nred, KrylovState* st, int first,
                           unsigned long long cond_handle) {
  __shared__ double sh[40];
  if (st->done) {
    if (threadIdx.x == 0 && cond_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, 0);
    return;
  }
  double rr = sum_partials(part_rr, nred, sh);
  if (threadIdx.x == 0) {
    if (!first) st->iter += 1;
    double rn = sqrt(rr);
    st->rnorm = rn;
    st->scale = rn > 0.0 ? rn : 1.0;
    int done = 0, status = st->status;
    if (!isfinite(rn)) { done = 1; status = status ? status : -6; }
    else if (status != 0) done = 1;
    else if (rn <= st->rtol * st->bnorm) { done = 1; status = 0; }
    else if (st->iter >= st->max_it) { done = 1; status = -4; }
    st->status = status;
    st->done = done;
    if (cond_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_handle, done ? 0u : 1u);
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ v, float* __restrict__ v32, const KrylovState* st) {
  if (st->done) return;
  const double inv = 1.0 / st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    v32[i] = __double2float_rn(v[i] * inv);
}

// (r, z) and (q, z) partials for flexible CG
template <int NC>
__global__ void __launch_bounds__(kBlock) k_cg_dots(int64_t nn, PVec z, const double* __restrict__ r,
                                                     const double* __restrict__ q, double* part_rz, double* part_qz,
                                                     const KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double a = 0.0, c = 0.0;
  const int64_t lim = ((nn + 31) / 32) * 32;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < lim; node += nthreads) {
    if (node < nn)
      for (int k = 0; k < NC; ++k) {
        const int64_t i = NC * node + k;
        const double zi = pv(z, i, sc);
        a = fma(r[i], zi, a);
        c = fma(q[i], zi, c);
      }
  }
  double t = block_sum(a, sh);
  if (threadIdx.x == 0) part_rz[blockIdx.x] = t;
  t = block_sum(c, sh);
  if (threadIdx.x == 0) part_qz[blockIdx.x] = t;
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_cg_update_p(int64_t nn, PVec z, double* __restrict__ p,
                                                         const double* part_rz, const double* part_qz, int nred,
                                                         KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double rz = sum_partials(part_rz, nred, sh);
  const double qz = sum_partials(part_qz, nred, sh);
  const bool first = st->iter == st->restart_pos;
  // Polak-Ribiere: beta = (z_new, r_new - r_old) / rho_old, r_new - r_old = -alpha q
  const double beta = first ? 0.0 : -st->alpha * qz / st->rho_prev;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t lim = ((nn + 31) / 32) * 32;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < lim; node += nthreads)
    if (node < nn)
      for (int k = 0; k < NC; ++k) {
        const int64_t i = NC * node + k;
        p[i] = first ? pv(z, i, sc) : fma(beta, p[i], pv(z, i, sc));
      }
  if (blockIdx.x == 0 && threadIdx.x == 0) { st->rho = rz; st->beta = beta; }
}

// out = A p (p given as PVec), partial of (w, out) (w = p when w == nullptr)
template <int NC>
__global__ void __launch_bounds__(kBlock) k_spmv_dot(SellView A, PVec p, const double* __restrict__ w,
                                                      double* __restrict__ out, double* part, const KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    if (NC == 1) {
      double ax;
      if (p.f) {
        // A (scale * p32): accumulate in FP64 from FP32 operands
        const int64_t s0 = A.sptr[slice] + lane, s1 = A.sptr[slice + 1];
        const double* val = (const double*)A.val;
        double a = 0.0;
        for (int64_t o = s0; o < s1; o += 32) a = fma(__ldg(val + o), (double)__ldg(p.f + __ldg(A.col + o)), a);
        ax = a * sc;
      } else {
        ax = sell_dot1<double>(A, slice, lane, p.d);
      }
      if (row < A.n) {
        out[row] = ax;
        acc = fma(w ? w[row] : pv(p, row, sc), ax, acc);
      }
    } else {
      double a3[3];
      if (p.f) sell_dot3<double, float>(A, slice, lane, p.f, 1.0, a3);
      else sell_dot3<double>(A, slice, lane, p.d, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) {
          const double y = p.f ? a3[i] * sc : a3[i];
          out[3 * row + i] = y;
          acc = fma(w ? w[3 * row + i] : pv(p, 3 * row + i, sc), y, acc);
        }
    }
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_cg_update_xr(int64_t nn, const double* __restrict__ p,
                                                          const double* __restrict__ q, double* __restrict__ x,
                                                          double* __restrict__ r, const double* part_pq, int nred,
                                                          double* part_rr, KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double pq = sum_partials(part_pq, nred, sh);
  const double alpha = st->rho / pq;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t lim = ((nn + 31) / 32) * 32;
  double acc = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < lim; node += nthreads)
    if (node < nn)
      for (int k = 0; k < NC; ++k) {
        const int64_t i = NC * node + k;
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
      }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    part_rr[blockIdx.x] = t;
    if (blockIdx.x == 0) {
      st->alpha = alpha;
      st->rho_prev = st->rho;
      if (pq == 0.0) st->status = -5;
    }
  }
}

// BiCGStab (van der Vorst), right preconditioned
template <int NC>
__global__ void __launch_bounds__(kBlock) k_bicg_p(int64_t nn, const double* __restrict__ r,
                                                    const double* __restrict__ v, double* __restrict__ p,
                                                    const double* part_rhr, int nred, KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double rho = sum_partials(part_rhr, nred, sh);
  const bool first = st->iter == st->restart_pos;
  const double beta = first ? 0.0 : (rho / st->rho_prev) * (st->alpha / st->omega);
  const double om = st->omega;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = nn * NC;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads)
    p[i] = first ? r[i] : fma(beta, fma(-om, v[i], p[i]), r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rho = rho;
    st->beta = beta;
    if (rho == 0.0) st->status = -5;
  }
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_bicg_s(int64_t nn, const double* __restrict__ r,
                                                    const double* __restrict__ v, double* __restrict__ s,
                                                    const double* part_rhv, int nred, KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double rhv = sum_partials(part_rhv, nred, sh);
  const double alpha = st->rho / rhv;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = nn * NC;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += nthreads) s[i] = fma(-alpha, v[i], r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->alpha = alpha;
    if (rhv == 0.0) st->status = -5;
  }
}

// t = A sh, partials (t, s) and (t, t)
template <int NC>
__global__ void __launch_bounds__(kBlock) k_spmv_2dots(SellView A, PVec shv, const double* __restrict__ sv,
                                                        double* __restrict__ t, double* part_ts, double* part_tt,
                                                        const KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double a = 0.0, c = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.nslices * 32; row += nthreads) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    if (NC == 1) {
      double ax;
      if (shv.f) {
        const int64_t s0 = A.sptr[slice] + lane, s1 = A.sptr[slice + 1];
        const double* val = (const double*)A.val;
        double acc = 0.0;
        for (int64_t o = s0; o < s1; o += 32) acc = fma(__ldg(val + o), (double)__ldg(shv.f + __ldg(A.col + o)), acc);
        ax = acc * sc;
      } else {
        ax = sell_dot1<double>(A, slice, lane, shv.d);
      }
      if (row < A.n) { t[row] = ax; a = fma(ax, sv[row], a); c = fma(ax, ax, c); }
    } else {
      double a3[3];
      if (shv.f) sell_dot3<double, float>(A, slice, lane, shv.f, 1.0, a3);
      else sell_dot3<double>(A, slice, lane, shv.d, a3);
      if (row < A.n)
        for (int i = 0; i < 3; ++i) {
          const double y = shv.f ? a3[i] * sc : a3[i];
          t[3 * row + i] = y;
          a = fma(y, sv[3 * row + i], a);
          c = fma(y, y, c);
        }
    }
  }
  double tt = block_sum(a, sh);
  if (threadIdx.x == 0) part_ts[blockIdx.x] = tt;
  tt = block_sum(c, sh);
  if (threadIdx.x == 0) part_tt[blockIdx.x] = tt;
}

template <int NC>
__global__ void __launch_bounds__(kBlock) k_bicg_x(int64_t nn, PVec ph, PVec shv, const double* __restrict__ sv,
                                                    const double* __restrict__ t, const double* __restrict__ rhat,
                                                    double* __restrict__ x, double* __restrict__ r,
                                                    const double* part_ts, const double* part_tt, int nred,
                                                    double* part_rr, double* part_rhr, KrylovState* st) {
  __shared__ double sh[40];
  if (st->done) return;
  const double ts = sum_partials(part_ts, nred, sh);
  const double tt = sum_partials(part_tt, nred, sh);
  const double om = tt > 0.0 ? ts / tt : 0.0;
  const double alpha = st->alpha;
  const double sc = st->scale;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t lim = ((nn + 31) / 32) * 32;
  double a = 0.0, c = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < lim; node += nthreads)
    if (node < nn)
      for (int k = 0; k < NC; ++k) {
        const int64_t i = NC * node + k;
        x[i] = fma(om, pv(shv, i, sc), fma(alpha, pv(ph, i, sc), x[i]));
        const double ri = fma(-om, t[i], sv[i]);
        r[i] = ri;
        a = fma(ri, ri, a);
        c = fma(rhat[i], ri, c);
      }
  double s1 = block_sum(a, sh);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = s1;
  s1 = block_sum(c, sh);
  if (threadIdx.x == 0) {
    part_rhr[blockIdx.x] = s1;
    if (blockIdx.x == 0) {
      st->omega = om;
      st->rho_prev = st->rho;
      if (!(tt > 0.0) || om == 0.0) st->status = -5;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
int grid_for_rows(int64_t rows) {
  int64_t g = (rows + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  return (int)(g > kMaxRedBlocks ? kMaxRedBlocks : g);
}
int grid_for_vec(int64_t n) { return grid_for_rows(n); }

static int grid_sell(int64_t nslices) { return grid_for_rows(nslices * 32); }

template <typename T>
void launch_smooth(const SellView& A, int nc, const T* x, const T* b, const T* Sinv, T* xo, double omega,
                   bool from_zero, const int* done, cudaStream_t s) {
  const int g = grid_sell(A.nslices);
  if (nc == 1) {
    if (from_zero) k_smooth<T, 1, true><<<g, kBlock, 0, s>>>(A, x, b, Sinv, xo, (T)omega, done);
    else k_smooth<T, 1, false><<<g, kBlock, 0, s>>>(A, x, b, Sinv, xo, (T)omega, done);
  } else {
    if (from_zero) k_smooth<T, 3, true><<<g, kBlock, 0, s>>>(A, x, b, Sinv, xo, (T)omega, done);
    else k_smooth<T, 3, false><<<g, kBlock, 0, s>>>(A, x, b, Sinv, xo, (T)omega, done);
  }
}

template <typename T>
void launch_residual(const SellView& A, int nc, const T* x, const T* b, T* r, const int* done, cudaStream_t s) {
  const int g = grid_sell(A.nslices);
  if (nc == 1) k_apply<T, 1, 1><<<g, kBlock, 0, s>>>(A, x, b, r, done);
  else k_apply<T, 3, 1><<<g, kBlock, 0, s>>>(A, x, b, r, done);
}

template <typename T>
void launch_matvec(const SellView& A, int nc, const T* x, T* y, const int* done, cudaStream_t s) {
  const int g = grid_sell(A.nslices);
  if (nc == 1) k_apply<T, 1, 0><<<g, kBlock, 0, s>>>(A, x, nullptr, y, done);
  else k_apply<T, 3, 0><<<g, kBlock, 0, s>>>(A, x, nullptr, y, done);
}

template <typename T>
void launch_restrict(const TransferView& R, int nc, const T* r, T* d, const int* done, cudaStream_t s) {
  const int g = grid_sell(R.nslices);
  if (nc == 1) k_restrict<T, 1><<<g, kBlock, 0, s>>>(R, r, d, done);
  else k_restrict<T, 3><<<g, kBlock, 0, s>>>(R, r, d, done);
}

template <typename T>
void launch_prolong_add(const TransferView& P, int nc, const T* y, const T* xin, T* xo, const int* done,
                        cudaStream_t s) {
  const int g = grid_sell(P.nslices);
  if (nc == 1) k_prolong<T, 1><<<g, kBlock, 0, s>>>(P, y, xin, xo, done);
  else k_prolong<T, 3><<<g, kBlock, 0, s>>>(P, y, xin, xo, done);
}

template <typename T>
void launch_coarse(const double* Ainv, int64_t n, const T* d, T* z, const int* done, cudaStream_t s) {
  int64_t g = (n + 7) / 8;
  if (g > kMaxRedBlocks) g = kMaxRedBlocks;
  k_coarse<T><<<(int)g, kBlock, 0, s>>>(Ainv, n, d, z, done);
}

#define MGI_INST(T)                                                                                                \
  template void launch_smooth<T>(const SellView&, int, const T*, const T*, const T*, T*, double, bool, const int*, \
                                 cudaStream_t);                                                                    \
  template void launch_residual<T>(const SellView&, int, const T*, const T*, T*, const int*, cudaStream_t);        \
  template void launch_matvec<T>(const SellView&, int, const T*, T*, const int*, cudaStream_t);                    \
  template void launch_restrict<T>(const TransferView&, int, const T*, T*, const int*, cudaStream_t);              \
  template void launch_prolong_add<T>(const TransferView&, int, const T*, const T*, T*, const int*, cudaStream_t); \
  template void launch_coarse<T>(const double*, int64_t, const T*, T*, const int*, cudaStream_t);
MGI_INST(double)
MGI_INST(float)
#undef MGI_INST

void launch_rhs(const SellView& F, int nc, const double* f, const uint8_t* fixmask, double* b, cudaStream_t s) {
  k_rhs<<<grid_sell(F.nslices), kBlock, 0, s>>>(F, nc, f, fixmask, b);
}
void launch_fill_hanging(const TransferView& Hc, int nc, double* x, cudaStream_t s) {
  k_fill_hanging<<<grid_sell(Hc.nslices), kBlock, 0, s>>>(Hc, nc, x);
}
void launch_copy_fixed(int64_t n, int nc, const uint8_t* fixmask, const double* b, const double* xin, double* x,
                       cudaStream_t s) {
  k_copy_fixed<<<grid_for_rows(n), kBlock, 0, s>>>(n, nc, fixmask, b, xin, x);
}
void launch_norm_free(int64_t n, int nc, const uint8_t* fixmask, const double* b, Partials part, int k,
                      cudaStream_t s) {
  k_norm_free<<<grid_for_rows(((n + 31) / 32) * 32), kBlock, 0, s>>>(n, nc, fixmask, b, part.q(k));
}
void launch_residual_norm(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                          int k, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  if (nc == 1) k_residual_norm<1><<<g, kBlock, 0, s>>>(A64, x, b, r, part.q(k));
  else k_residual_norm<3><<<g, kBlock, 0, s>>>(A64, x, b, r, part.q(k));
}
void launch_init_state(KrylovState* st, Partials part, int k_bb, int nred, double rtol, int max_it, cudaStream_t s) {
  k_init_state<<<1, kBlock, 0, s>>>(st, part.q(k_bb), nred, rtol, max_it);
}
void launch_finalize(Partials part, int k_rr, int nred, KrylovState* st, int first, unsigned long long cond_handle,
                     cudaStream_t s) {
  k_finalize<<<1, kBlock, 0, s>>>(part.q(k_rr), nred, st, first, cond_handle);
}
void launch_to_f32(int64_t n, const double* v, float* v32, const KrylovState* st, cudaStream_t s) {
  k_to_f32<<<grid_for_rows(n), kBlock, 0, s>>>(n, v, v32, st);
}

// Krylov launchers: grid = the finest-level SpMV grid (one thread per node)
static int grid_nodes(int64_t nn) { return grid_for_rows(((nn + 31) / 32) * 32); }

#define MGI_NC(call1, call3) \
  do {                          \
    if (nc == 1) call1;         \
    else call3;                 \
  } while (0)

void launch_cg_dots(int64_t nn, int nc, PVec z, const double* r, const double* q, Partials part,
                    const KrylovState* st, cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_cg_dots<1><<<g, kBlock, 0, s>>>(nn, z, r, q, part.q(1), part.q(2), st)),
         (k_cg_dots<3><<<g, kBlock, 0, s>>>(nn, z, r, q, part.q(1), part.q(2), st)));
}
void launch_cg_update_p(int64_t nn, int nc, PVec z, double* p, Partials part, int nred, KrylovState* st,
                        cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_cg_update_p<1><<<g, kBlock, 0, s>>>(nn, z, p, part.q(1), part.q(2), nred, st)),
         (k_cg_update_p<3><<<g, kBlock, 0, s>>>(nn, z, p, part.q(1), part.q(2), nred, st)));
}
void launch_spmv_dot(const SellView& A64, int nc, PVec p, const double* w, double* out, Partials part, int k,
                     const KrylovState* st, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  MGI_NC((k_spmv_dot<1><<<g, kBlock, 0, s>>>(A64, p, w, out, part.q(k), st)),
         (k_spmv_dot<3><<<g, kBlock, 0, s>>>(A64, p, w, out, part.q(k), st)));
}
void launch_cg_update_xr(int64_t nn, int nc, const double* p, const double* q, double* x, double* r, Partials part,
                         int nred, KrylovState* st, cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_cg_update_xr<1><<<g, kBlock, 0, s>>>(nn, p, q, x, r, part.q(3), nred, part.q(0), st)),
         (k_cg_update_xr<3><<<g, kBlock, 0, s>>>(nn, p, q, x, r, part.q(3), nred, part.q(0), st)));
}
void launch_bicg_p(int64_t nn, int nc, const double* r, const double* v, double* p, Partials part, int nred,
                   KrylovState* st, cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_bicg_p<1><<<g, kBlock, 0, s>>>(nn, r, v, p, part.q(9), nred, st)),
         (k_bicg_p<3><<<g, kBlock, 0, s>>>(nn, r, v, p, part.q(9), nred, st)));
}
void launch_bicg_s(int64_t nn, int nc, const double* r, const double* v, double* sv, Partials part, int nred,
                   KrylovState* st, cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_bicg_s<1><<<g, kBlock, 0, s>>>(nn, r, v, sv, part.q(5), nred, st)),
         (k_bicg_s<3><<<g, kBlock, 0, s>>>(nn, r, v, sv, part.q(5), nred, st)));
}
void launch_spmv_2dots(const SellView& A64, int nc, PVec sh, const double* sv, double* t, Partials part,
                       const KrylovState* st, cudaStream_t s) {
  const int g = grid_sell(A64.nslices);
  MGI_NC((k_spmv_2dots<1><<<g, kBlock, 0, s>>>(A64, sh, sv, t, part.q(7), part.q(8), st)),
         (k_spmv_2dots<3><<<g, kBlock, 0, s>>>(A64, sh, sv, t, part.q(7), part.q(8), st)));
}
void launch_bicg_x(int64_t nn, int nc, PVec ph, PVec sh, const double* sv, const double* t, const double* rhat,
                   double* x, double* r, Partials part, int nred, KrylovState* st, cudaStream_t s) {
  const int g = grid_nodes(nn);
  MGI_NC((k_bicg_x<1><<<g, kBlock, 0, s>>>(nn, ph, sh, sv, t, rhat, x, r, part.q(7), part.q(8), nred, part.q(0),
                                            part.q(9), st)),
         (k_bicg_x<3><<<g, kBlock, 0, s>>>(nn, ph, sh, sv, t, rhat, x, r, part.q(7), part.q(8), nred, part.q(0),
                                            part.q(9), st)));
}
#undef MGI_NC

}  // namespace mgi
