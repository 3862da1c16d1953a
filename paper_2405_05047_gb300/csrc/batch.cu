// Batched solve of many small problems in one launch (k_batch): one thread
// block per problem runs the whole Krylov solve with the V-cycle of every
// level in shared memory (tail_cycle of rows.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "kernels.h"
#include "rows.cuh"

namespace mgi {

namespace {
// ------------------------------------------------------------- batched solves
// Many small problems in one launch: the launch overhead that dominates a
// small solve (Sec. 6.1: thousands of kernel launches per time step) is paid
// once for all of them.  A block takes the next problem of the work list and
// runs its whole solve (the algorithms of the graph-driven solve: flexible CG
// or right-preconditioned BiCGStab on FP64 vectors, an FP32 or FP64 V-cycle
// as the preconditioner, restarts from the true residual), then takes the
// next.  The V-cycle is the staged tail over every level, so smoothing,
// transfers and the coarse solve run out of shared memory; the FP64 vectors
// stay in the block's L1 / L2.  Dots are block sums in a fixed order, and no
// block ever waits for another.

// a and b summed over the block: butterfly in each warp, then the warp sums
// in warp order, read by every thread (the same bits everywhere)
__device__ __forceinline__ void bsum2(double& a, double& b, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();                   // readers of the previous sums are done with sh
  if ((threadIdx.x & 31) == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < nw; ++i) { a += sh[2 * i]; b += sh[2 * i + 1]; }
}

// y = A x over the rows of the finest FP64 operator, f(first dof, y[NC]) per
// node row; x was written by this block (plain loads)
template <int NC, typename F>
__device__ __forceinline__ void batch_spmv(const SellView& A, const double* x, F f) {
  for (int64_t row = threadIdx.x; row < A.nslices * 32; row += blockDim.x) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t orow = srow<2>(A, row);
    double y[NC];
    if constexpr (NC == 1) y[0] = sell_dot1<double, 2>(A, slice, lane, x);
    else sell_dot3<double, 2>(A, slice, lane, x, y);
    if (row < A.n) f(NC * orow, y);
  }
}

// Convergence test of the graph-driven solve (converge_step).
__device__ __forceinline__ bool batch_converged(double rr, double bnorm, double rtol, int iter, int max_it,
                                                int& status, double& scale) {
  const double rn = sqrt(rr);
  scale = rn > 0.0 ? rn : 1.0;
  if (!isfinite(rn)) { if (!status) status = -6; return true; }
  if (status != 0) return true;
  if (rn <= rtol * bnorm) return true;
  if (iter >= max_it) { status = -4; return true; }
  return false;
}

template <typename T, typename VT, int NC>
__device__ void batch_solve(BatchItem& it, unsigned char* smem, double* sh) {
  constexpr bool mixed = !std::is_same<T, double>::value;
  const TailParams& P = *it.tail;
  {
    // the item must describe a staged tail over all its levels that fits the
    // launch's shared memory, with the top level's vectors as long as x
    unsigned dyn = 0;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    __shared__ int bad;
    if (threadIdx.x == 0) {
      int e = 0;
      if (P.nt < 1 || P.nt > kTailMax || P.cluster != 0 || P.smem > dyn || P.image_bytes > P.smem) e = 1;
      else if (it.n != it.n_nodes * NC || it.n < 1) e = 1;
      bad = e;
    }
    __syncthreads();
    const int e = bad;
    __syncthreads();
    if (e) {
      if (threadIdx.x == 0) { it.status = -7; it.iters = 0; it.rounds = 0; it.rel_res = 0.0; }
      return;
    }
  }
  const TailLevel* LV = tail_stage<2>(P, smem, 0);
  __syncthreads();
  const int top = P.nt - 1;
  if (LV[top].A.n * NC != it.n) {      // the top level is not this problem's finest level
    __syncthreads();
    if (threadIdx.x == 0) { it.status = -7; it.iters = 0; it.rounds = 0; it.rel_res = 0.0; }
    __syncthreads();
    return;
  }
  T* cb = (T*)LV[top].b;               // V-cycle input (shared memory)
  const T* co = (const T*)LV[top].o;   // V-cycle output (shared memory)
  const SellView A = it.A;
  const int64_t n = it.n, nn = it.n_nodes;
  const double* __restrict__ b = it.b;
  double* xi = it.xi;
  double* r = it.r;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double rtol = it.rtol;
  const int max_it = it.max_it;
  // iterate: the initial guess with the fixed entries from b; ||b_free||
  double bb = 0.0, un = 0.0;
  for (int64_t i = tid; i < nn; i += nth) {
    const unsigned f = it.fix[i];
    for (int c = 0; c < NC; ++c) {
      const int64_t k = NC * i + c;
      const double bk = b[k];
      const bool fx = (f >> c) & 1u;
      xi[k] = fx ? bk : it.x[k];
      if (!fx) bb = fma(bk, bk, bb);
    }
  }
  bsum2(bb, un, sh);
  const double bnorm = bb > 0.0 ? sqrt(bb) : 1.0;
  auto residual = [&]() {              // r = b - A xi, returns (r, r)
    double rr = 0.0, z = 0.0;
    batch_spmv<NC>(A, xi, [&](int64_t k, const double* y) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double ri = b[k + c] - y[c];
        r[k + c] = ri;
        rr = fma(ri, ri, rr);
      }
    });
    bsum2(rr, z, sh);
    return rr;
  };
  // V-cycle on v (mixed: v / scale in FP32); the output is read as co[i] * zs
  auto vcycle = [&](const double* v, double inv) {
    for (int64_t i = tid; i < n; i += nth) cb[i] = mixed ? (T)__double2float_rn(v[i] * inv) : (T)v[i];
    tail_cycle<T, VT, NC, 2>(P, LV, nullptr, nullptr, 0, nullptr, nullptr, 0);
  };
  int iter = 0, status = 0, rounds = 0;
  double rel = 0.0;
  for (;;) {
    double rr = residual(), scale = 1.0;
    const int restart = iter;
    bool done = batch_converged(rr, bnorm, rtol, iter, max_it, status, scale);
    if (it.method == 1) {
      // flexible CG (Polak-Ribiere beta)
      double* p = it.p;
      double* q = it.q;
      double alpha = 1.0, rho_prev = 1.0;
      while (!done) {
        const double zs = mixed ? scale : 1.0;
        vcycle(r, 1.0 / scale);
        const bool first = iter == restart;
        double rz = 0.0, qz = 0.0;
        for (int64_t i = tid; i < n; i += nth) {
          const double z = (double)co[i] * zs;
          rz = fma(r[i], z, rz);
          if (!first) qz = fma(q[i], z, qz);
        }
        bsum2(rz, qz, sh);
        const double beta = first ? 0.0 : -alpha * qz / rho_prev;
        const double rho = rz;
        for (int64_t i = tid; i < n; i += nth) {
          const double z = (double)co[i] * zs;
          p[i] = first ? z : fma(beta, p[i], z);
        }
        __syncthreads();
        double pq = 0.0, un2 = 0.0;
        batch_spmv<NC>(A, p, [&](int64_t k, const double* y) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            q[k + c] = y[c];
            pq = fma(p[k + c], y[c], pq);
          }
        });
        bsum2(pq, un2, sh);
        alpha = rho / pq;
        double rr2 = 0.0;
        for (int64_t i = tid; i < n; i += nth) {
          xi[i] = fma(alpha, p[i], xi[i]);
          const double ri = fma(-alpha, q[i], r[i]);
          r[i] = ri;
          rr2 = fma(ri, ri, rr2);
        }
        bsum2(rr2, un2, sh);
        rho_prev = rho;
        iter += 1;
        if (pq == 0.0) status = -5;
        done = batch_converged(rr2, bnorm, rtol, iter, max_it, status, scale);
      }
    } else {
      // BiCGStab (van der Vorst), right preconditioned
      double *p = it.p, *v = it.v, *s = it.s, *t = it.q, *ph = it.ph, *rhat = it.rhat, *shv = it.sh;
      for (int64_t i = tid; i < n; i += nth) { rhat[i] = r[i]; v[i] = 0.0; }
      double rhr = rr, om = 1.0, alpha = 1.0, beta_next = 0.0;
      __syncthreads();
      while (!done) {
        const double zs = mixed ? scale : 1.0, inv = 1.0 / scale;
        const double rho = rhr;
        const bool first = iter == restart;
        const double beta = first ? 0.0 : beta_next;
        for (int64_t i = tid; i < n; i += nth) {
          const double pn = first ? r[i] : fma(beta, fma(-om, v[i], p[i]), r[i]);
          p[i] = pn;
        }
        if (rho == 0.0) status = -5;
        __syncthreads();
        vcycle(p, inv);
        for (int64_t i = tid; i < n; i += nth) ph[i] = (double)co[i] * zs;
        __syncthreads();
        double rhv = 0.0, un2 = 0.0;
        batch_spmv<NC>(A, ph, [&](int64_t k, const double* y) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[k + c] = y[c];
            rhv = fma(rhat[k + c], y[c], rhv);
          }
        });
        bsum2(rhv, un2, sh);
        alpha = rho / rhv;
        for (int64_t i = tid; i < n; i += nth) s[i] = fma(-alpha, v[i], r[i]);
        if (rhv == 0.0) status = -5;
        __syncthreads();
        vcycle(s, inv);
        for (int64_t i = tid; i < n; i += nth) shv[i] = (double)co[i] * zs;
        __syncthreads();
        double ts = 0.0, tt = 0.0;
        batch_spmv<NC>(A, shv, [&](int64_t k, const double* y) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            t[k + c] = y[c];
            ts = fma(y[c], s[k + c], ts);
            tt = fma(y[c], y[c], tt);
          }
        });
        bsum2(ts, tt, sh);
        om = tt > 0.0 ? ts / tt : 0.0;
        double rr2 = 0.0, rh2 = 0.0;
        for (int64_t i = tid; i < n; i += nth) {
          xi[i] = fma(om, shv[i], fma(alpha, ph[i], xi[i]));
          const double ri = fma(-om, t[i], s[i]);
          r[i] = ri;
          rr2 = fma(ri, ri, rr2);
          rh2 = fma(rhat[i], ri, rh2);
        }
        bsum2(rr2, rh2, sh);
        rhr = rh2;
        beta_next = (rhr / rho) * (alpha / om);
        if (!(tt > 0.0) || om == 0.0) status = -5;
        iter += 1;
        done = batch_converged(rr2, bnorm, rtol, iter, max_it, status, scale);
      }
    }
    // true residual of the iterate; restart from it while it is above rtol
    const double tr = residual();
    rel = sqrt(tr) / bnorm;
    if (status == -6 || status == -5 || rel <= rtol) break;
    if (iter >= max_it || rounds >= 3) { status = -4; break; }
    status = 0;
    rounds += 1;
    for (int64_t i = tid; i < nn; i += nth) {   // hanging / Dirichlet entries back from b
      const unsigned f = it.fix[i];
      for (int c = 0; c < NC; ++c)
        if ((f >> c) & 1u) xi[NC * i + c] = b[NC * i + c];
    }
    __syncthreads();
  }
  if (status == 0 && !(rel <= rtol)) status = -4;
  // solution: fixed entries from b, then the hanging values x_h = H x
  double* x = it.x;
  for (int64_t i = tid; i < nn; i += nth) {
    const unsigned f = it.fix[i];
    for (int c = 0; c < NC; ++c) x[NC * i + c] = ((f >> c) & 1u) ? b[NC * i + c] : xi[NC * i + c];
  }
  __syncthreads();
  const TransferView Hc = it.Hc;
  for (int64_t row = tid; row < Hc.nslices * 32; row += nth) {
    const int64_t slice = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t o0 = Hc.sptr[slice] + lane, o1 = Hc.sptr[slice + 1];
    bool any = false;
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int64_t o = o0; o < o1; o += 32) {
      const double w = (double)Hc.w[o];
      if (w == 0.0) continue;
      any = true;
      const int64_t j = Hc.col[o];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = fma(w, x[NC * j + c], acc[c]);
    }
    if (row < Hc.n && any)
#pragma unroll
      for (int c = 0; c < NC; ++c) x[NC * row + c] = acc[c];
  }
  if (tid == 0) {
    it.status = status;
    it.iters = iter;
    it.rounds = rounds;
    it.rel_res = rel;
  }
  __syncthreads();                     // shared memory is free for the next problem
}

template <typename T, typename VT, int NC>
__global__ void __launch_bounds__(kTailThreads) k_batch(BatchItem* items, const int* order, int count,
                                                         unsigned int* next) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ double sh[2 * (kTailThreads / 32)];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int k = cur;
    __syncthreads();
    if (k >= count) return;
    batch_solve<T, VT, NC>(items[order[k]], tail_smem, sh);
  }
}

}  // namespace

template <typename T, typename V, int NC>
static const void* batch_fn() {
  static std::once_flag once;   // opt in to the large dynamic shared memory, once per instantiation
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_batch<T, V, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  });
  return (const void*)k_batch<T, V, NC>;
}

template <typename T, typename V, int NC>
static void batch_k(BatchItem* items, const int* order, int count, unsigned int* next, uint32_t smem, int grid,
                    cudaStream_t s) {
  batch_fn<T, V, NC>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  if (t_prof) t_prof->before((const void*)k_batch<T, V, NC>, s);
  cudaLaunchKernelEx(&cfg, k_batch<T, V, NC>, items, order, count, next);
  if (t_prof) t_prof->after(s);
}

void launch_batch(BatchItem* items, const int* order, int count, unsigned int* next, int nc, int prec, uint32_t smem,
                  int grid, cudaStream_t s) {
  if (nc == 1) {
    if (prec == 0) batch_k<double, double, 1>(items, order, count, next, smem, grid, s);
    else if (prec == 1) batch_k<float, float, 1>(items, order, count, next, smem, grid, s);
    else batch_k<float, __nv_bfloat16, 1>(items, order, count, next, smem, grid, s);
  } else {
    if (prec == 0) batch_k<double, double, 3>(items, order, count, next, smem, grid, s);
    else if (prec == 1) batch_k<float, float, 3>(items, order, count, next, smem, grid, s);
    else batch_k<float, __nv_bfloat16, 3>(items, order, count, next, smem, grid, s);
  }
}

int batch_blocks_per_sm(int nc, int prec, uint32_t smem) {
  const void* fn;
  if (nc == 1) fn = prec == 0 ? batch_fn<double, double, 1>() : (prec == 1 ? batch_fn<float, float, 1>()
                                                                          : batch_fn<float, __nv_bfloat16, 1>());
  else fn = prec == 0 ? batch_fn<double, double, 3>() : (prec == 1 ? batch_fn<float, float, 3>()
                                                                   : batch_fn<float, __nv_bfloat16, 3>());
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTailThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

}  // namespace mgi
