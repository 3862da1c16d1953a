// Device functions shared by the CUDA translation units of the library: load
// helpers, the SELL row sums, the row steps of every level operation (the
// grid kernels, the small-level kernel and the batched solve call the same
// functions, so their results are bitwise identical) and the small-level
// V-cycle (tail_stage / tail_cycle).  Everything is in an unnamed namespace:
// each translation unit instantiates what it uses.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.h"

namespace mgi {

namespace {

// Programmatic dependent launch: kernels are launched while their predecessor
// drains; every kernel waits here until the preceding kernel of the stream
// has completed and its writes are visible.  (Triggering the next
// launch early was measured slower: the waiting blocks of the next kernel
// take SM slots from the running one.)
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }

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

// Vector loads: through the read-only path where the vector is constant for
// the kernel's lifetime, plain (coherent) loads in the single-CTA tail kernel
// that rewrites its vectors between __syncthreads().
// Load modes: 0 grid kernels (read-only path), 1 unstaged tail kernel (its
// CTAs run on several SMs: vectors L2-coherent), 2 shared-memory-staged tail
// kernel (plain generic loads, operands may sit in shared memory), 4 the
// staged sweep (matrices through the read-only path, vectors by plain
// generic loads: the gathered x sits in shared memory).
template <int LM, typename T>
__device__ __forceinline__ T vld(const T* p) {
  if (LM == 0) return __ldg(p);
  if (LM == 1) return __ldcg(p);
  return *p;
}

// Stored matrix values: float/double as they are, BF16 widened to FP32.
// Matrix loads: read-only path in the grid kernels; plain generic loads in
// the tail kernel, whose matrices may sit in shared memory.
template <int LM, typename T>
__device__ __forceinline__ T mld(const T* p) {
  if (LM <= 1 || LM == 4) return __ldg(p);   // matrices never change during a kernel
  return *p;
}
template <typename AT, int LM = 0, typename VT>
__device__ __forceinline__ AT ldv(const VT* p) {
  if constexpr (std::is_same<VT, __nv_bfloat16>::value) return (AT)__bfloat162float(mld<LM>(p));
  else return (AT)mld<LM>(p);
}

// Entry c of a gathered vector.  LM 3 (the cluster-resident small levels):
// the CTAs of the cluster hold the vector in chunks of 2^gsh entries, chunk k
// in CTA k, each at the same shared-memory offset, and v is this CTA's chunk
// minus its first index.  Entry c is in CTA c >> gsh: its address is v + c
// moved by whole chunks into this CTA's window, then mapped into the owner's
// window (mapa) when the owner is another CTA.
template <int LM, typename T>
__device__ __forceinline__ T xg(const T* v, int64_t c, int gsh) {
  if constexpr (LM == 3) {
    namespace cg = cooperative_groups;
    const int64_t me = (int64_t)cg::this_cluster().block_rank();
    const int64_t owner = c >> gsh;
    const T* p = v + (c - (owner - me) * ((int64_t)1 << gsh));
    if (owner == me) return *p;
    return *cg::this_cluster().map_shared_rank(const_cast<T*>(p), (unsigned)owner);
  } else {
    return vld<LM>(v + c);
  }
}

// Output row of SELL row `row` (< A.n): rows may be sorted by length within
// windows (SELL-C-sigma); perm maps them back to node order.
template <int LM = 0, typename V>
__device__ __forceinline__ int64_t srow(const V& A, int64_t row) {
  if (A.perm && row < A.n) return (int64_t)mld<LM>(A.perm + row);
  return row;
}

// y_row = sum_j A(row, j) x_j for a scalar SELL row (thread = row).  Slots
// are processed in batches of 4 (column and value loads of a batch issued
// together, then the 4 gathers, then the FMAs in slot order); the slice width
// is the same for the 32 threads of a warp, so the remainder switch is
// warp-uniform.  The summation order is the plain sequential one.
template <typename AT, int LM, typename VT, typename XT, typename CF>
__device__ __forceinline__ AT sell_dot1x_loop(int64_t o, int64_t s1, const VT* __restrict__ val, const XT* __restrict__ x,
                                              CF colat, int64_t S = 32, int gsh = 0) {
  AT acc = AT(0);
  for (; o + 3 * S < s1; o += 4 * S) {
    const int c0 = colat(o), c1 = colat(o + S), c2 = colat(o + 2 * S), c3 = colat(o + 3 * S);
    const AT v0 = ldv<AT, LM>(val + o), v1 = ldv<AT, LM>(val + o + S), v2 = ldv<AT, LM>(val + o + 2 * S),
             v3 = ldv<AT, LM>(val + o + 3 * S);
    const XT x0 = xg<LM>(x, c0, gsh), x1 = xg<LM>(x, c1, gsh), x2 = xg<LM>(x, c2, gsh), x3 = xg<LM>(x, c3, gsh);
    acc = fmad(v0, (AT)x0, acc);
    acc = fmad(v1, (AT)x1, acc);
    acc = fmad(v2, (AT)x2, acc);
    acc = fmad(v3, (AT)x3, acc);
  }
  const int rem = (int)((s1 - o + S - 1) / S);   // 0..3 (identical across a warp when S = 32)
  if (rem == 3) {
    const int c0 = colat(o), c1 = colat(o + S), c2 = colat(o + 2 * S);
    const AT v0 = ldv<AT, LM>(val + o), v1 = ldv<AT, LM>(val + o + S), v2 = ldv<AT, LM>(val + o + 2 * S);
    const XT x0 = xg<LM>(x, c0, gsh), x1 = xg<LM>(x, c1, gsh), x2 = xg<LM>(x, c2, gsh);
    acc = fmad(v0, (AT)x0, acc);
    acc = fmad(v1, (AT)x1, acc);
    acc = fmad(v2, (AT)x2, acc);
  } else if (rem == 2) {
    const int c0 = colat(o), c1 = colat(o + S);
    const AT v0 = ldv<AT, LM>(val + o), v1 = ldv<AT, LM>(val + o + S);
    const XT x0 = xg<LM>(x, c0, gsh), x1 = xg<LM>(x, c1, gsh);
    acc = fmad(v0, (AT)x0, acc);
    acc = fmad(v1, (AT)x1, acc);
  } else if (rem == 1) {
    acc = fmad(ldv<AT, LM>(val + o), (AT)xg<LM>(x, colat(o), gsh), acc);
  }
  return acc;
}

// y_row = sum_j A(row, j) x_j for a scalar SELL row (thread = row).  Slots
// are processed in batches of 4 (column and value loads of a batch issued
// together, then the 4 gathers, then the FMAs in slot order); the slice width
// is the same for the 32 threads of a warp, so the remainder switch is
// warp-uniform.  The summation order is the plain sequential one.  Columns
// come from the 16-bit offsets when the view has them and the slice fits.
template <typename AT, int LM = 0, typename VT, typename XT>
__device__ __forceinline__ AT sell_dot1x(const int64_t* __restrict__ sptr, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, int64_t slice, int lane,
                                         const XT* __restrict__ x, const int16_t* __restrict__ col16 = nullptr,
                                         int sub = 0, int tpr = 1, int gsh = 0) {
  const int64_t r0 = mld<LM>(sptr + slice), r1 = mld<LM>(sptr + slice + 1);
  const int64_t s0 = (r0 & kSptrMask) + lane + 32 * sub, s1 = r1 & kSptrMask;
  const int64_t S = 32 * (int64_t)tpr;
  if (col16 && !(r0 & 1)) {
    const int base = (int)((slice >> 3) * kCol16Window);
    return sell_dot1x_loop<AT, LM>(s0, s1, val, x, [&](int64_t o) { return base + (int)mld<LM>(col16 + o); }, S,
                                   gsh);
  }
  return sell_dot1x_loop<AT, LM>(s0, s1, val, x, [&](int64_t o) { return (int)mld<LM>(col + o); }, S, gsh);
}

// Scalar row sum; with tpr > 1 lane sub of the row's group takes slot groups
// sub, sub + tpr, ... and a butterfly adds the partial sums (same bits on
// every lane of the group).
template <typename T, int LM = 0, typename VT = T, int TPR = 1>
__device__ __forceinline__ T sell_dot1(const SellView& A, int64_t slice, int lane, const T* __restrict__ x,
                                       int sub = 0, int gsh = 0) {
  T acc = sell_dot1x<T, LM>(A.sptr, A.col, (const VT*)A.val, slice, lane, x, A.col16, sub, TPR, gsh);
#pragma unroll
  for (int o = 1; o < TPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// One 3x3 block of the velocity-pressure pattern (SellView::bpat = 1)
// [[a, 0, g1], [0, a, g2], [d1, d2, c]], stored as m = (a, g1, g2, d1, d2, c):
// the FMAs of the dense block without its structural zeros, in the same order.
template <typename T, typename M>
__device__ __forceinline__ void block_fma_p6(const M& m, T x0, T x1, T x2, T acc[3]) {
  acc[0] = fmad((T)m[0], x0, acc[0]);
  acc[0] = fmad((T)m[1], x2, acc[0]);
  acc[1] = fmad((T)m[0], x1, acc[1]);
  acc[1] = fmad((T)m[2], x2, acc[1]);
  acc[2] = fmad((T)m[3], x0, acc[2]);
  acc[2] = fmad((T)m[4], x1, acc[2]);
  acc[2] = fmad((T)m[5], x2, acc[2]);
}

// acc[0..2] = sum_j A(row, j) x_j for a 3x3-block SELL row.
template <typename T, typename XT>
__device__ __forceinline__ void sell_dot3(const SellView& A, int64_t slice, int lane, const XT* __restrict__ x,
                                          double xs, T acc[3]) {
  const int64_t r0 = A.sptr[slice];
  const int64_t s0 = r0 & kSptrMask, s1 = A.sptr[slice + 1] & kSptrMask;
  const T* __restrict__ val = (const T*)A.val;
  const bool narrow = A.col16 && !(r0 & 1);
  const int base = (int)((slice >> 3) * kCol16Window);
  auto colat = [&](int64_t o) { return narrow ? base + (int)__ldg(A.col16 + o) : __ldg(A.col + o); };
  acc[0] = acc[1] = acc[2] = T(0);
  if (A.bpat) {
    for (int64_t g = s0; g < s1; g += 32) {
      const int c = colat(g + lane);
      const T* __restrict__ v = val + g * 6 + lane;
      const T x0 = (T)((double)__ldg(x + 3 * c) * xs), x1 = (T)((double)__ldg(x + 3 * c + 1) * xs),
              x2 = (T)((double)__ldg(x + 3 * c + 2) * xs);
      T m[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) m[e] = __ldg(v + e * 32);
      block_fma_p6(m, x0, x1, x2, acc);
    }
    return;
  }
  for (int64_t g = s0; g < s1; g += 32) {
    const int c = colat(g + lane);
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

template <typename T, int LM, typename VT, typename CF>
__device__ __forceinline__ void sell_dot3_loop(int64_t g, int64_t s1, int lane, const VT* __restrict__ val,
                                               const T* __restrict__ x, T acc[3], CF colat, int64_t stride = 32) {
  acc[0] = acc[1] = acc[2] = T(0);
  for (; g + stride < s1; g += 2 * stride) {
    const int ca = colat(g + lane), cb = colat(g + stride + lane);
    const VT* __restrict__ va = val + g * 9 + lane;
    const VT* __restrict__ vb = va + stride * 9;
    T ma[9], mb[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) { ma[e] = ldv<T, LM>(va + e * 32); mb[e] = ldv<T, LM>(vb + e * 32); }
    const T xa0 = vld<LM>(x + 3 * ca), xa1 = vld<LM>(x + 3 * ca + 1), xa2 = vld<LM>(x + 3 * ca + 2);
    const T xb0 = vld<LM>(x + 3 * cb), xb1 = vld<LM>(x + 3 * cb + 1), xb2 = vld<LM>(x + 3 * cb + 2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = acc[i];
      a = fmad(ma[3 * i + 0], xa0, a);
      a = fmad(ma[3 * i + 1], xa1, a);
      a = fmad(ma[3 * i + 2], xa2, a);
      acc[i] = a;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = acc[i];
      a = fmad(mb[3 * i + 0], xb0, a);
      a = fmad(mb[3 * i + 1], xb1, a);
      a = fmad(mb[3 * i + 2], xb2, a);
      acc[i] = a;
    }
  }
  if (g < s1) {
    const int c = colat(g + lane);
    const VT* __restrict__ v = val + g * 9 + lane;
    const T x0 = vld<LM>(x + 3 * c), x1 = vld<LM>(x + 3 * c + 1), x2 = vld<LM>(x + 3 * c + 2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T a = acc[i];
      a = fmad(ldv<T, LM>(v + (3 * i + 0) * 32), x0, a);
      a = fmad(ldv<T, LM>(v + (3 * i + 1) * 32), x1, a);
      a = fmad(ldv<T, LM>(v + (3 * i + 2) * 32), x2, a);
      acc[i] = a;
    }
  }
}

// sell_dot3_loop for blocks stored in the velocity-pressure pattern (6 values)
template <typename T, int LM, typename VT, typename CF>
__device__ __forceinline__ void sell_dot3p_loop(int64_t g, int64_t s1, int lane, const VT* __restrict__ val,
                                                const T* __restrict__ x, T acc[3], CF colat, int64_t stride = 32) {
  acc[0] = acc[1] = acc[2] = T(0);
  for (; g + stride < s1; g += 2 * stride) {
    const int ca = colat(g + lane), cb = colat(g + stride + lane);
    const VT* __restrict__ va = val + g * 6 + lane;
    const VT* __restrict__ vb = va + stride * 6;
    T ma[6], mb[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) { ma[e] = ldv<T, LM>(va + e * 32); mb[e] = ldv<T, LM>(vb + e * 32); }
    const T xa0 = vld<LM>(x + 3 * ca), xa1 = vld<LM>(x + 3 * ca + 1), xa2 = vld<LM>(x + 3 * ca + 2);
    const T xb0 = vld<LM>(x + 3 * cb), xb1 = vld<LM>(x + 3 * cb + 1), xb2 = vld<LM>(x + 3 * cb + 2);
    block_fma_p6(ma, xa0, xa1, xa2, acc);
    block_fma_p6(mb, xb0, xb1, xb2, acc);
  }
  if (g < s1) {
    const int c = colat(g + lane);
    const VT* __restrict__ v = val + g * 6 + lane;
    const T x0 = vld<LM>(x + 3 * c), x1 = vld<LM>(x + 3 * c + 1), x2 = vld<LM>(x + 3 * c + 2);
    T m[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) m[e] = ldv<T, LM>(v + e * 32);
    block_fma_p6(m, x0, x1, x2, acc);
  }
}

// acc[0..2] = sum_j A(row, j) x_j for a 3x3-block SELL row (same types).
// Slot groups are processed two at a time (both column loads, then both
// blocks' values and gathers, then the FMAs in slot order), so a thread keeps
// two dependent load chains in flight; the group count is warp-uniform.
// With tpr > 1 (small FP32 block levels) the tpr consecutive lanes of a row
// share its slot groups (lane sub takes groups sub, sub + tpr, ...), and a
// butterfly over those lanes adds the partial sums; every lane of the group
// ends with the same bits (the pairwise additions commute).
template <typename T, int LM = 0, typename VT = T, int TPR = 1>
__device__ __forceinline__ void sell_dot3(const SellView& A, int64_t slice, int lane, const T* __restrict__ x,
                                          T acc[3], int sub = 0) {
  constexpr int tpr = TPR;
  const int64_t r0 = mld<LM>(A.sptr + slice), r1 = mld<LM>(A.sptr + slice + 1);
  const int64_t s0 = (r0 & kSptrMask) + 32 * sub, s1 = r1 & kSptrMask;
  const VT* __restrict__ val = (const VT*)A.val;
  const int64_t stride = 32 * (int64_t)tpr;
  const int base = (int)((slice >> 3) * kCol16Window);
  const int16_t* c16 = A.col16;
  const int32_t* c32 = A.col;
  auto col16at = [&](int64_t o) { return base + (int)mld<LM>(c16 + o); };
  auto col32at = [&](int64_t o) { return (int)mld<LM>(c32 + o); };
  const bool narrow = c16 && !(r0 & 1);
  if (A.bpat) {
    if (narrow) sell_dot3p_loop<T, LM>(s0, s1, lane, val, x, acc, col16at, stride);
    else sell_dot3p_loop<T, LM>(s0, s1, lane, val, x, acc, col32at, stride);
  } else {
    if (narrow) sell_dot3_loop<T, LM>(s0, s1, lane, val, x, acc, col16at, stride);
    else sell_dot3_loop<T, LM>(s0, s1, lane, val, x, acc, col32at, stride);
  }
#pragma unroll
  for (int o = 1; o < tpr; o <<= 1)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
}

// acc[c] += sum_j W(row, j) v[NC j + c] for a transfer matrix row: batches
// of 4 slots (loads first), warp-uniform remainder, sequential summation.
template <typename T, int NC, int LM>
__device__ __forceinline__ void transfer_gather(const TransferView& W, int64_t slice, int lane, const T* v,
                                                T acc[NC], int gsh = 0) {
  const int64_t s0 = mld<LM>(W.sptr + slice) + lane, s1 = mld<LM>(W.sptr + slice + 1);
  int64_t o = s0;
  for (; o < s1; o += 4 * 32) {
    const int m = (int)min((int64_t)4, (s1 - o + 31) >> 5);   // warp-uniform
    int j[4];
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < m) { j[k] = mld<LM>(W.col + o + 32 * k); w[k] = mld<LM>(W.w + o + 32 * k); }
    T xv[4][NC];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < m)
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[k][c] = xg<LM>(v, (int64_t)NC * j[k] + c, gsh);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < m)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmad((T)w[k], xv[k][c], acc[c]);
  }
}

// ------------------------------------------------------------------ row steps
// One row (block row) of each level step.  The grid kernels below and the
// single-CTA tail kernel call the same functions, so both produce bitwise
// identical results.
// sub: lane of the row's lane group (A.tpr lanes per row, block levels);
// xo64 (optional): also write the output in FP64 times sc.
template <typename T, int NC, int LM, typename VT = T, int TPR = 1>
__device__ __forceinline__ void row_smooth(const SellView& A, int64_t row, const T* x, const T* b, const T* Sinv,
                                           T* xo, T omega, bool from_zero, int sub = 0, double* xo64 = nullptr,
                                           double sc = 1.0, int gsh = 0) {
  const int64_t slice = row >> 5;
  const int lane = (int)(row & 31);
  const int64_t orow = srow<LM>(A, row);
  if (NC == 1) {
    T r = from_zero ? T(0) : sell_dot1<T, LM, VT, TPR>(A, slice, lane, x, sub, gsh);
    if (row < A.n && sub == 0) {
      const T bi = vld<LM>(b + orow);
      const T v = from_zero ? omega * Sinv[orow] * bi : fmad(omega * Sinv[orow], bi - r, vld<LM>(x + orow));
      xo[orow] = v;
      if (xo64) xo64[orow] = (double)v * sc;
    }
  } else {
    constexpr int tpr = TPR;
    T acc[3] = {T(0), T(0), T(0)};
    if (!from_zero) sell_dot3<T, LM, VT, TPR>(A, slice, lane, x, acc, sub);
    if (row < A.n) {
      T res[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) res[i] = vld<LM>(b + 3 * orow + i) - acc[i];
      const T* S = Sinv + 9 * orow;
      // one lane per component when the row has several lanes
      const int i0 = tpr > 1 ? sub : 0, i1 = tpr > 1 ? sub + 1 : 3;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i < i0 || i >= i1) continue;
        T c = S[3 * i] * res[0];
        c = fmad(S[3 * i + 1], res[1], c);
        c = fmad(S[3 * i + 2], res[2], c);
        const T v = from_zero ? omega * c : fmad(omega, c, vld<LM>(x + 3 * orow + i));
        xo[3 * orow + i] = v;
        if (xo64) xo64[3 * orow + i] = (double)v * sc;
      }
    }
  }
}

template <typename T, int NC, int LM, typename VT = T, int TPR = 1>
__device__ __forceinline__ void row_residual(const SellView& A, int64_t row, const T* x, const T* b, T* y,
                                             int sub = 0, int gsh = 0) {
  const int64_t slice = row >> 5;
  const int lane = (int)(row & 31);
  const int64_t orow = srow<LM>(A, row);
  if (NC == 1) {
    T r = sell_dot1<T, LM, VT, TPR>(A, slice, lane, x, sub, gsh);
    if (row < A.n && sub == 0) y[orow] = vld<LM>(b + orow) - r;
  } else {
    constexpr int tpr = TPR;
    T acc[3];
    sell_dot3<T, LM, VT, TPR>(A, slice, lane, x, acc, sub);
    if (row < A.n) {
      const int i0 = tpr > 1 ? sub : 0, i1 = tpr > 1 ? sub + 1 : 3;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i >= i0 && i < i1) y[3 * orow + i] = vld<LM>(b + 3 * orow + i) - acc[i];
    }
  }
}

template <typename T, int NC, int LM>
__device__ __forceinline__ void row_restrict(const TransferView& R, int64_t row, const T* r, T* d, const T* Sinv,
                                             T* x0, T omega, int gsh = 0) {
  const int64_t slice = row >> 5;
  const int lane = (int)(row & 31);
  const int64_t orow = srow<LM>(R, row);
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  transfer_gather<T, NC, LM>(R, slice, lane, r, acc, gsh);
  if (row < R.n) {
    if constexpr (NC > 1)
      if (R.fix) {
        const unsigned m = mld<LM>(R.fix + orow);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if ((m >> c) & 1u) acc[c] = T(0);
      }
#pragma unroll
    for (int c = 0; c < NC; ++c) d[NC * orow + c] = acc[c];
    if (x0) {
      if (NC == 1) {
        x0[orow] = omega * Sinv[orow] * acc[0];
      } else {
        const T* S = Sinv + NC * NC * orow;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          T c = S[NC * i] * acc[0];
#pragma unroll
          for (int k = 1; k < NC; ++k) c = fmad(S[NC * i + k], acc[k], c);
          x0[NC * orow + i] = omega * c;
        }
      }
    }
  }
}

template <typename T, int NC, int LM>
__device__ __forceinline__ void row_prolong(const TransferView& P, int64_t row, const T* y, const T* xin, T* xo,
                                            int gsh = 0) {
  const int64_t slice = row >> 5;
  const int lane = (int)(row & 31);
  const int64_t orow = srow<LM>(P, row);
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  transfer_gather<T, NC, LM>(P, slice, lane, y, acc, gsh);
  if (row < P.n) {
    if constexpr (NC > 1)
      if (P.fix) {
        const unsigned m = mld<LM>(P.fix + orow);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if ((m >> c) & 1u) acc[c] = T(0);
      }
#pragma unroll
    for (int c = 0; c < NC; ++c) xo[NC * orow + c] = vld<LM>(xin + NC * orow + c) + acc[c];
  }
}

// The V-cycle below (and including) level `nt - 1` in one launch: smoothing,
// restriction, coarse solve and correction of the small levels, separated
// by block or cluster barriers instead of kernel boundaries.  Same row
// functions as the grid kernels, so the result is bitwise identical to the
// multi-kernel cycle.
//   TLM 1: one thread-block cluster of gridDim.x CTAs over the device arrays;
//          barriers are hardware cluster barriers (release/acquire at cluster
//          scope) and vectors are read with L2-coherent loads.
//   TLM 2: one CTA whose vectors (and the matrices of the staged levels) live
//          in dynamic shared memory, copied from the tail image at start; each
//          step then runs at shared-memory latency instead of L2 latency.
__device__ __forceinline__ void tail_sync() {
  if (gridDim.x > 1) cooperative_groups::this_cluster().sync();
  else __syncthreads();
}
// Barrier between two steps of the tail.  TLM 3: cluster-wide only when the
// data written by the step is read by another CTA in the next one (a level
// cut into several chunks on either side); levels held by one CTA whole
// need only its own barrier.  Every CTA evaluates the same condition, so all
// take the same sequence of cluster barriers.
template <int TLM>
__device__ __forceinline__ void tail_bar(bool wide) {
  if constexpr (TLM == 3) {
    if (wide) cooperative_groups::this_cluster().sync();
    else __syncthreads();
  } else if constexpr (TLM == 2) {
    __syncthreads();                 // one CTA (also one of many in a batched launch)
  } else {
    tail_sync();
  }
}

template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, int64_t n) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Copies the tail image into shared memory (TLM 2: the whole image; TLM 3:
// CTA me's section) and turns the header's offsets into shared-memory
// pointers; returns the level headers.
template <int TLM>
__device__ __forceinline__ TailLevel* tail_stage(const TailParams& P, unsigned char* tail_smem, int64_t me) {
  // four 16-byte loads in flight per thread
  const uint4* src = (const uint4*)((const unsigned char*)P.image + (TLM == 3 ? (size_t)me * P.section : 0));
  uint4* dst = (uint4*)tail_smem;
  const uint32_t n16 = P.image_bytes / 16, step = blockDim.x;
  uint32_t i = threadIdx.x;
  for (; i + 3 * step < n16; i += 4 * step) {
    const uint4 a = __ldg(src + i), b = __ldg(src + i + step), c = __ldg(src + i + 2 * step),
                d = __ldg(src + i + 3 * step);
    dst[i] = a; dst[i + step] = b; dst[i + 2 * step] = c; dst[i + 3 * step] = d;
  }
  for (; i < n16; i += step) dst[i] = __ldg(src + i);
  __syncthreads();
  TailLevel* hdr = (TailLevel*)tail_smem;
  for (int l = threadIdx.x; l < P.nt; l += blockDim.x) {
    TailLevel& L = hdr[l];
    // offsets relative to this CTA's shared memory (TLM 3: shifted by the
    // chunk's first row, so they may be negative)
    auto at = [&](const void* off) -> unsigned char* { return tail_smem + (intptr_t)off; };
    L.b = at(L.b); L.o = at(L.o); L.t = at(L.t); L.r = at(L.r);
    if ((P.staged_mask >> l) & 1u) {
      L.A.sptr = (const int64_t*)at(L.A.sptr);
      L.A.col = (const int32_t*)at(L.A.col);
      L.A.val = at(L.A.val);
      if (TLM == 3 && L.c16) L.A.col16 = (const int16_t*)at(L.A.col16);
      L.S = at(L.S);
      if (l > 0) {
        L.P.sptr = (const int64_t*)at(L.P.sptr); L.P.col = (const int32_t*)at(L.P.col); L.P.w = (const float*)at(L.P.w);
        L.R.sptr = (const int64_t*)at(L.R.sptr); L.R.col = (const int32_t*)at(L.R.col); L.R.w = (const float*)at(L.R.w);
      }
    }
  }
  return hdr;
}

// One V-cycle of levels 0..P.nt-1 (the body of k_tail after staging).  LV:
// the level headers (P.lv, or tail_stage's copy in shared memory).  SM modes:
// btop NULL means the top level's right-hand side is already in LV[top].b;
// otop NULL leaves the result in LV[top].o.
template <typename T, typename VT, int NC, int TLM>
__device__ __forceinline__ void tail_cycle(const TailParams& P, const TailLevel* LV, const T* btop, T* otop,
                                           int first_done, double* o64, const double* scale, int64_t me) {
  constexpr bool SM = TLM == 2 || TLM == 3;      // vectors (and staged matrices) in shared memory
  const int top = P.nt - 1, ns = P.nu1 + P.nu2;
  // rows of a level this thread block works on: every row (TLM 1, 2) or the
  // CTA's chunk (TLM 3)
  auto own = [&](int64_t rows, int csh, int64_t& lo, int64_t& hi) {
    if constexpr (TLM == 3) {
      lo = min(rows, me << csh);
      hi = min(rows, (me + 1) << csh);
    } else {
      lo = 0;
      hi = rows;
    }
  };
  if constexpr (SM) {
    __syncthreads();
    int64_t lo, hi;
    own(LV[top].A.n * NC, TLM == 3 ? LV[top].csh : 0, lo, hi);
    T* bt = (T*)LV[top].b;
    if (btop)
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) bt[i] = btop[i];
    if (first_done && P.nu1 > 0) {   // first pre-smoothing sweep, written by the finer level's restriction
      const bool in_o = (ns - 1) % 2 == 0;
      T* d = (T*)(in_o ? LV[top].o : LV[top].t);
      const T* sv = in_o ? (const T*)otop : (const T*)P.lv[top].t;
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) d[i] = sv[i];
    }
    tail_bar<TLM>(true);             // TLM 3: every chunk is in place before any gather
  }
  const int tid = SM ? threadIdx.x : blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = SM ? blockDim.x : gridDim.x * blockDim.x;
  auto bvec = [&](int l) -> T* { return (TLM == 1 && l == top) ? const_cast<T*>(btop) : (T*)LV[l].b; };
  auto ovec = [&](int l) -> T* { return (TLM == 1 && l == top) ? otop : (T*)LV[l].o; };
  auto bufof = [&](int l, int k) -> T* { return ((ns - 1 - k) % 2 == 0) ? ovec(l) : (T*)LV[l].t; };
  auto csh = [&](int l) -> int { return TLM == 3 ? LV[l].csh : 0; };
  // TLM 3: level l is cut into several chunks (else CTA 0 holds it whole)
  auto dist = [&](int l) -> bool { return TLM == 3 && ((int64_t)1 << LV[l].csh) < LV[l].A.n * NC; };
  int fdone = first_done;
  for (int l = top; l >= 1; --l) {
    const TailLevel& L = LV[l];
    const T* S = (const T*)L.S;
    const T om = (T)L.omega;
    const int tpr = L.A.tpr;
    int64_t lo, hi, clo, chi;
    own(L.A.nslices * 32, csh(l), lo, hi);
    own(L.R.nslices * 32, csh(l - 1), clo, chi);
    T* cur = nullptr;
    for (int k = 0; k < P.nu1; ++k) {
      T* dst = bufof(l, k);
      if (!(k == 0 && fdone)) {
        if (tpr == 4)
          for (int64_t t = lo * 4 + tid; t < hi * 4; t += nth)
            row_smooth<T, NC, TLM, VT, 4>(L.A, t / 4, cur, bvec(l), S, dst, om, k == 0, (int)(t % 4), nullptr, 1.0,
                                          csh(l));
        else
          for (int64_t t = lo + tid; t < hi; t += nth)
            row_smooth<T, NC, TLM, VT, 1>(L.A, t, cur, bvec(l), S, dst, om, k == 0, 0, nullptr, 1.0, csh(l));
        tail_bar<TLM>(dist(l));
      }
      cur = dst;
    }
    if (tpr == 4)
      for (int64_t t = lo * 4 + tid; t < hi * 4; t += nth)
        row_residual<T, NC, TLM, VT, 4>(L.A, t / 4, cur, bvec(l), (T*)L.r, (int)(t % 4), csh(l));
    else
      for (int64_t t = lo + tid; t < hi; t += nth)
        row_residual<T, NC, TLM, VT, 1>(L.A, t, cur, bvec(l), (T*)L.r, 0, csh(l));
    tail_bar<TLM>(dist(l) || dist(l - 1));
    T* x0 = l - 1 > 0 ? bufof(l - 1, 0) : nullptr;
    for (int64_t row = clo + tid; row < chi; row += nth)
      row_restrict<T, NC, TLM>(L.R, row, (const T*)L.r, bvec(l - 1), (const T*)LV[l - 1].S, x0, (T)LV[l - 1].omega,
                               csh(l));
    tail_bar<TLM>(dist(l - 1));
    fdone = l - 1 > 0;
  }
  {   // coarse direct solve, one warp per row
    const int lane = threadIdx.x & 31;
    const T* d = bvec(0);
    T* z = ovec(0);
    int64_t lo, hi;
    own(P.cn, csh(0), lo, hi);
    for (int64_t row = lo + (tid >> 5); row < hi; row += nth >> 5) {
      double acc = 0.0;
      for (int64_t j = lane; j < P.cn; j += 32)
        acc = fma(P.cinv[row * P.cn + j], (double)xg<TLM == 3 ? 3 : TLM>(d, j, csh(0)), acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) z[row] = (T)acc;
    }
    tail_bar<TLM>(dist(0) || (top >= 1 && dist(1)));
  }
  for (int l = 1; l <= top; ++l) {
    const TailLevel& L = LV[l];
    const T om = (T)L.omega;
    const int tpr = L.A.tpr;
    int64_t lo, hi, plo, phi;
    own(L.A.nslices * 32, csh(l), lo, hi);
    own(L.P.nslices * 32, csh(l), plo, phi);
    T* cur = bufof(l, P.nu1 - 1);       // output of the last pre-smoothing sweep (nu1 >= 1)
    T* pdst = P.nu2 == 0 ? ovec(l) : cur;
    for (int64_t row = plo + tid; row < phi; row += nth)
      row_prolong<T, NC, TLM>(L.P, row, ovec(l - 1), cur, pdst, csh(l - 1));
    tail_bar<TLM>(dist(l) || (P.nu2 == 0 && l < top && dist(l + 1)));
    cur = pdst;
    for (int k = P.nu1; k < ns; ++k) {
      T* dst = bufof(l, k);
      const bool out64 = o64 && l == top && k == ns - 1;   // last sweep: also the FP64 copy times *scale
      const double sc = out64 ? *scale : 1.0;
      if (tpr == 4)
        for (int64_t t = lo * 4 + tid; t < hi * 4; t += nth)
          row_smooth<T, NC, TLM, VT, 4>(L.A, t / 4, cur, bvec(l), (const T*)L.S, dst, om, false, (int)(t % 4),
                                        out64 ? o64 : nullptr, sc, csh(l));
      else
        for (int64_t t = lo + tid; t < hi; t += nth)
          row_smooth<T, NC, TLM, VT, 1>(L.A, t, cur, bvec(l), (const T*)L.S, dst, om, false, 0,
                                        out64 ? o64 : nullptr, sc, csh(l));
      // the last sweep of a level feeds the prolongation of the next finer one
      tail_bar<TLM>(dist(l) || (k == ns - 1 && l < top && dist(l + 1)));
      cur = dst;
    }
  }
  if constexpr (SM) {
    int64_t lo, hi;
    own(LV[top].A.n * NC, csh(top), lo, hi);
    const T* o = (const T*)LV[top].o;
    if (otop)
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) otop[i] = o[i];
  }
}


}  // namespace

}  // namespace mgi
