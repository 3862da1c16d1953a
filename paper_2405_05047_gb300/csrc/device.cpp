// Device hierarchy (SELL packing + upload), solve workspaces, the V-cycle and
// the Krylov loop as one CUDA graph.
//
// The V-cycle is the recursive geometric multigrid cycle of Sec. 2.2: on the
// coarsest level a direct solve; on every finer level damped smoothing sweeps,
// the residual carried to the next coarser level, the cycle there from a zero
// guess, its result interpolated back and added, then smoothing again.  It
// preconditions flexible CG
// (Polak-Ribiere), BiCGStab or flexible GMRES(m) (Sec. 4.1.5: multigrid as
// preconditioner of a Krylov method).  All Krylov scalars stay on the device;
// one Krylov iteration is captured into the body of a CUDA-graph `while` node
// whose condition is set by the convergence test on the device, so a whole
// solve is one graph launch and only the final state crosses to the host.
#include "device.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

namespace mgi {

namespace {
thread_local std::string g_last_error;
}

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
const char* last_error() { return g_last_error.c_str(); }

#define CU(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

size_t rnd(size_t b) { return b == 0 ? 256 : ((b + 255) & ~(size_t)255); }

// Device allocation through the context allocator (or cudaMalloc), recorded
// in `list` and counted against the context.
void* dev_alloc(mg_ctx* c, std::vector<Alloc>& list, size_t& total, size_t bytes, bool ctx_alloc) {
  bytes = rnd(bytes);
  void* p = nullptr;
  const bool use_ctx = ctx_alloc && c->has_alloc;
  if (use_ctx) p = c->alloc.malloc_fn(bytes, c->alloc.user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (!p) return nullptr;
  list.push_back({p, bytes, !use_ctx});
  total += bytes;
  c->used += bytes;
  return p;
}

// Frees the one allocation of list that starts at p (nothing if absent).
void free_one(mg_ctx* c, std::vector<Alloc>& list, size_t& total, const void* p) {
  for (size_t i = 0; i < list.size(); ++i)
    if (list[i].p == p) {
      if (!list[i].cuda) c->alloc.free_fn(list[i].p, c->alloc.user);
      else cudaFree(list[i].p);
      c->used -= list[i].bytes;
      total -= list[i].bytes;
      list.erase(list.begin() + (int64_t)i);
      return;
    }
}

void free_list(mg_ctx* c, std::vector<Alloc>& list, size_t& total) {
  for (auto& a : list) {
    if (!a.cuda) c->alloc.free_fn(a.p, c->alloc.user);
    else cudaFree(a.p);
    c->used -= a.bytes;
  }
  list.clear();
  total = 0;
}

template <typename VT>
VT to_vt(double v) { return (VT)v; }
template <>
__nv_bfloat16 to_vt<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }   // via FP32, round to nearest even

// SELL-C-sigma packing of a block CSR matrix (C = kSlice block rows per
// slice).  With sigma > 0 the rows of every window of sigma consecutive rows
// are ordered by decreasing length before slicing, so rows of similar length
// share a slice (less padding); perm[sell row] = matrix row.  A window is one
// thread block of the kernels (kBlock rows), so the permuted vector accesses
// stay within one block's rows.
// pat6: 3x3 blocks in the velocity-pressure pattern, stored as the 6 values
// (a, g1, g2, d1, d2, c) of [[a, 0, g1], [0, a, g2], [d1, d2, c]]
// (block entries 0, 2, 5, 6, 7, 8).
constexpr int kPat6Entries[6] = {0, 2, 5, 6, 7, 8};

template <typename VT>
void pack_sell(const BlockCSR& M, int64_t sigma, std::vector<int64_t>& sptr, std::vector<int32_t>& col,
               std::vector<VT>& val, std::vector<int32_t>& perm, bool pat6 = false) {
  const int nbm = M.nc * M.nc, nb = pat6 ? 6 : nbm;
  const int64_t n = M.n, ns = (n + kSlice - 1) / kSlice;
  perm.clear();
  if (sigma > 0) {
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
      const int64_t w1 = std::min(n, w0 + sigma);
      std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int32_t a, int32_t b) {
        return M.ptr[a + 1] - M.ptr[a] > M.ptr[b + 1] - M.ptr[b];
      });
    }
    bool identity = true;
    for (int64_t r = 0; r < n && identity; ++r) identity = perm[r] == r;
    if (identity) perm.clear();
  }
  auto mrow = [&](int64_t r) -> int64_t { return perm.empty() ? r : perm[r]; };
  sptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t w = 0;
    for (int64_t r = s * kSlice; r < std::min(n, (s + 1) * kSlice); ++r) {
      const int64_t q = mrow(r);
      w = std::max(w, M.ptr[q + 1] - M.ptr[q]);
    }
    sptr[s + 1] = sptr[s] + kSlice * w;
  }
  const int64_t slots = sptr[ns];
  col.assign(slots, 0);
  val.assign(slots * nb, to_vt<VT>(0.0));
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t w = (sptr[s + 1] - sptr[s]) / kSlice;
    for (int lane = 0; lane < kSlice; ++lane) {
      const int64_t r = s * kSlice + lane;
      const int64_t q = r < n ? mrow(r) : -1;
      const int64_t len = q >= 0 ? M.ptr[q + 1] - M.ptr[q] : 0;
      for (int64_t j = 0; j < w; ++j) {
        const int64_t g = sptr[s] + kSlice * j, o = g + lane;
        if (j < len) {
          col[o] = (int32_t)M.col[M.ptr[q] + j];
          const double* blk = &M.val[(M.ptr[q] + j) * nbm];
          for (int e = 0; e < nb; ++e)
            val[g * nb + (int64_t)e * kSlice + lane] = to_vt<VT>(blk[pat6 ? kPat6Entries[e] : e]);
        } else {
          col[o] = (int32_t)(q >= 0 ? std::min<int64_t>(q, M.m - 1) : 0);
        }
      }
    }
  }
}

// 16-bit column offsets relative to each slice's 256-row window base;
// slices with an offset outside int16 are flagged in bit 0 of sptr[slice]
// and keep using the 32-bit columns.
void pack_col16(const std::vector<int64_t>& sptr, const std::vector<int32_t>& col, std::vector<int64_t>& sptr_out,
                std::vector<int16_t>& col16) {
  const int64_t ns = (int64_t)sptr.size() - 1;
  sptr_out = sptr;
  col16.assign(col.size(), 0);
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t base = (s / (kCol16Window / kSlice)) * kCol16Window;
    bool fits = true;
    for (int64_t o = sptr[s]; o < sptr[s + 1] && fits; ++o) {
      const int64_t rel = (int64_t)col[o] - base;
      fits = rel >= -32768 && rel <= 32767;
    }
    if (!fits) { sptr_out[s] |= 1; continue; }
    for (int64_t o = sptr[s]; o < sptr[s + 1]; ++o) col16[o] = (int16_t)((int64_t)col[o] - base);
  }
}

// Every 3x3 block of M has the velocity-pressure pattern (exact zeros at
// (0,1) and (1,0), equal entries at (0,0) and (1,1)): the 2D Oseen operator,
// whose two velocity components share one convection-diffusion operator.
bool velocity_pressure_pattern(const BlockCSR& M) {
  if (M.nc != 3) return false;
  const int64_t nb = M.nnzb();
  for (int64_t k = 0; k < nb; ++k) {
    const double* b = &M.val[k * 9];
    if (b[1] != 0.0 || b[3] != 0.0 || b[0] != b[4]) return false;
  }
  return true;
}

// Upload a matrix as SELL-C-sigma in one device allocation (sptr, col,
// optional 16-bit columns, values, optional permutation; each 256-byte
// aligned).  sigma: window of the row sort (0: rows in matrix order); idx16:
// also store 16-bit column offsets.
template <typename VT>
int upload_sell(mg_hier* h, const BlockCSR& M, SellBuf* out, int64_t sigma = 0, bool idx16 = false,
                bool pat6 = false, std::vector<Alloc>* list = nullptr, size_t* list_bytes = nullptr) {
  std::vector<int64_t> sptr;
  std::vector<int32_t> col;
  std::vector<VT> val;
  std::vector<int32_t> perm;
  std::vector<int16_t> col16;
  pack_sell<VT>(M, sigma, sptr, col, val, perm, pat6);
  if (idx16) {
    std::vector<int64_t> flagged;
    pack_col16(sptr, col, flagged, col16);
    sptr.swap(flagged);
    if (!list)
      for (size_t k = 0; k + 1 < sptr.size(); ++k) {
        if (sptr[k] & 1) h->col32_slices++;
        else h->col16_slices++;
      }
  }
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_sptr = sptr.size() * 8, b_col = col.size() * 4, b_c16 = col16.size() * 2,
               b_val = val.size() * sizeof(VT), b_perm = perm.size() * 4;
  // 16-bit columns and values adjacent: the part a sweep streams
  const size_t o_c16 = 0, o_val = r256(b_c16), o_col = o_val + r256(b_val), o_sptr = o_col + r256(b_col),
               o_perm = o_sptr + r256(b_sptr), total = o_perm + r256(b_perm);
  unsigned char* base = (unsigned char*)dev_alloc(h->ctx, list ? *list : h->allocs, list ? *list_bytes : h->bytes,
                                                  std::max<size_t>(total, 256), true);
  if (!base) return fail(MG_ERR_OOM, "device allocation failed");
  CU(cudaMemcpy(base + o_sptr, sptr.data(), b_sptr, cudaMemcpyHostToDevice));
  if (b_col) CU(cudaMemcpy(base + o_col, col.data(), b_col, cudaMemcpyHostToDevice));
  if (b_c16) CU(cudaMemcpy(base + o_c16, col16.data(), b_c16, cudaMemcpyHostToDevice));
  if (b_val) CU(cudaMemcpy(base + o_val, val.data(), b_val, cudaMemcpyHostToDevice));
  if (b_perm) CU(cudaMemcpy(base + o_perm, perm.data(), b_perm, cudaMemcpyHostToDevice));
  // pageable copies may still be in flight on the legacy stream: complete
  // them before the setup tuner times the matrix on the context's stream
  CU(cudaStreamSynchronize(cudaStreamLegacy));
  out->v.perm = out->t.perm = b_perm ? (const int32_t*)(base + o_perm) : nullptr;
  out->v.col16 = b_c16 ? (const int16_t*)(base + o_c16) : nullptr;
  out->v.sptr = out->t.sptr = (const int64_t*)(base + o_sptr);
  out->v.col = out->t.col = (const int32_t*)(base + o_col);
  out->v.val = base + o_val;
  out->v.bpat = pat6 ? 1 : 0;
  out->t.w = (const float*)(base + o_val);
  out->v.n = out->t.n = M.n;
  out->v.nslices = out->t.nslices = (int64_t)sptr.size() - 1;
  out->slots = (int64_t)col.size();
  out->sigma = sigma;
  out->val_bytes = b_val;
  out->nnz_real = M.nnzb();
  return MG_OK;
}

template <typename T>
T* halloc(mg_hier* h, int64_t n) {
  return (T*)dev_alloc(h->ctx, h->allocs, h->bytes, (size_t)std::max<int64_t>(n, 1) * sizeof(T), true);
}

// SELL-C-sigma window of the level operators and transfers, used on levels
// with at least kSigmaMinRows rows: there the padding costs bandwidth, while
// on the small, latency-bound levels the extra permutation load would cost
// more than it saves.
constexpr int64_t kSigma = kBlock;
constexpr int64_t kSigmaMinRows = 32768;
// 16-bit column offsets for the level operators of the large levels, every
// precision (streamed bytes per scalar entry: FP32 8 -> 6, FP64 12 -> 10).
bool idx16_for(const mg_hier* h, int64_t rows) {
  const int o = h->opts.col16;
  return o >= 0 ? o != 0 : rows >= kSigmaMinRows;
}
// Lanes per row of the FP32/BF16 level operators: the small levels are
// latency-bound (one thread walks all slots of its row one dependent batch
// after another), so four lanes share a row there.
int tpr_for(const mg_hier* h, int nc, int64_t rows) {
  if (h->opts.row_lanes == 1) return 1;
  if (nc == 3) return rows < 65536 ? 4 : 1;
  // scalar rows are short: the smallest levels (the shared-memory tail's,
  // where threads are few) keep one lane per row
  return (rows >= 1024 && rows < 32768) ? 4 : 1;
}
int64_t sigma_for(const mg_hier* h, int64_t rows) {
  const int o = h->opts.sell_sigma;
  if (o >= 0) return o;
  return rows >= kSigmaMinRows ? kSigma : 0;
}

// Column range of every 256-row window of a scalar SELL packing (all stored
// slots, padding included), on the device, for the staged sweep; nullptr
// arrays when no window is narrow enough to be staged.
int stage_windows(mg_hier* h, const BlockCSR& M, int64_t sigma, SellView& v) {
  std::vector<int64_t> sptr;
  std::vector<int32_t> col, perm;
  std::vector<float> val;
  pack_sell<float>(M, sigma, sptr, col, val, perm);
  const int64_t ns = (int64_t)sptr.size() - 1, per = kCol16Window / kSlice;
  const int64_t nw = (ns + per - 1) / per;
  std::vector<int32_t> lo(nw), len(nw);
  int64_t staged = 0;
  for (int64_t w = 0; w < nw; ++w) {
    int32_t mn = INT32_MAX, mx = INT32_MIN;
    for (int64_t o = sptr[w * per]; o < sptr[std::min(ns, (w + 1) * per)]; ++o) {
      mn = std::min(mn, col[o]);
      mx = std::max(mx, col[o]);
    }
    if (mn > mx) mn = mx = 0;
    lo[w] = mn;
    len[w] = mx - mn + 1;
    staged += len[w] <= kStageMax;
  }
  if (staged == 0) return MG_OK;
  int32_t* d = (int32_t*)dev_alloc(h->ctx, h->allocs, h->bytes, (size_t)nw * 8, true);
  if (!d) return fail(MG_ERR_OOM, "alloc");
  CU(cudaMemcpy(d, lo.data(), nw * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(d + nw, len.data(), nw * 4, cudaMemcpyHostToDevice));
  v.wlo = d;
  v.wlen = d + nw;
  return MG_OK;
}

// New values for a packed matrix whose pattern is unchanged: packs M the way
// upload_sell packed it (same window, same pattern flag) and copies only the
// value array into the existing device buffer.
template <typename VT>
int refill_sell(const BlockCSR& M, SellBuf& buf, bool pat6 = false) {
  if (!buf.v.val || buf.val_bytes == 0) return MG_OK;
  std::vector<int64_t> sptr;
  std::vector<int32_t> col;
  std::vector<VT> val;
  std::vector<int32_t> perm;
  pack_sell<VT>(M, buf.sigma, sptr, col, val, perm, pat6);
  if (val.size() * sizeof(VT) != buf.val_bytes || (int64_t)col.size() != buf.slots)
    return fail(MG_ERR_INVALID, "re-assembly changed a matrix pattern");
  CU(cudaMemcpy(const_cast<void*>(buf.v.val), val.data(), buf.val_bytes, cudaMemcpyHostToDevice));
  return MG_OK;
}

// ---------------------------------------------------------------- precision helpers
template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const TailParams& tail(Workspace& w) { return w.tail64; }
  static const SellView& A(LevelMats& l) { return l.A64.v; }
  static const SellView& V(LevelMats& l) { return l.V64.v; }
  static const double* S(LevelMats& l) { return l.S64; }
  static double* b(LevelVecs& v) { return v.b64; }
  static double* o(LevelVecs& v) { return v.o64; }
  static double* t(LevelVecs& v) { return v.t64; }
  static double* r(LevelVecs& v) { return v.r64; }
};
template <>
struct Prec<float> {
  static const TailParams& tail(Workspace& w) { return w.tail32; }
  static const SellView& A(LevelMats& l) { return l.A32.v; }
  static const SellView& V(LevelMats& l) { return l.V32.v; }
  static const float* S(LevelMats& l) { return l.S32; }
  static float* b(LevelVecs& v) { return v.b32; }
  static float* o(LevelVecs& v) { return v.o32; }
  static float* t(LevelVecs& v) { return v.t32; }
  static float* r(LevelVecs& v) { return v.r32; }
};

}  // namespace

// ---------------------------------------------------------------- tail tuning
namespace {
int tail_top_for(const mg_hier* h, int rows) {
  int top = 0;
  if (rows > 0)   // the small-level kernel smooths with Jacobi: it stops below the first Vanka level
    for (int l = 1; l < h->nlev && l < kTailMax; ++l)
      if (h->L[l].n * h->nc <= rows && !h->L[l].vanka) top = l;
      else break;
  return top;
}
uint32_t rnd16(uint64_t b) { return (uint32_t)((b + 15) & ~uint64_t(15)); }

// Precision slot pi (0 FP64, 1 FP32, 2 BF16-stored values) of a hierarchy.
bool has_slot(const mg_hier* h, int pi) { return pi == 0 ? h->has_fp64 : (pi == 1 ? h->has_fp32 : h->has_bf16); }
const SellBuf& slot_A(const LevelMats& B, int pi) { return pi == 0 ? B.A64 : (pi == 1 ? B.A32 : B.A16); }
uint32_t slot_tsize(int pi) { return pi == 0 ? 8 : 4; }
uint32_t slot_vsize(int pi) { return pi == 0 ? 8 : (pi == 1 ? 4 : 2); }

// Bytes of the header and the vectors of a staged tail over levels 0..top.
uint64_t tail_vec_bytes(const mg_hier* h, int pi, int top) {
  uint64_t b = rnd16((uint64_t)(top + 1) * sizeof(TailLevel));
  for (int l = 0; l <= top; ++l) b += 4 * (uint64_t)rnd16((uint64_t)h->L[l].n * h->nc * slot_tsize(pi));
  return b;
}

// Largest tail top whose staged vectors fit in shared memory, for every slot.
int staged_top_cap(const mg_hier* h, int top) {
  for (int pi = 0; pi < 3; ++pi)
    if (has_slot(h, pi))
      while (top > 0 && tail_vec_bytes(h, pi, top) > kTailSmemMax) --top;
  return top;
}

// Shared-memory image of levels 0..top (layout in kernels.h, TailParams).
// Matrices are staged level by level from the coarsest while they fit.
int tail_image(mg_hier* h, int pi, int top, mg_hier::TailImage* out) {
  auto it = h->tail_img.find({pi, top});
  if (it != h->tail_img.end()) { *out = it->second; return MG_OK; }
  const int nc = h->nc, nb = nc * nc, nt = top + 1;
  const uint32_t ts = slot_tsize(pi), vs = slot_vsize(pi);
  struct Piece { const void* src; uint64_t bytes; uint32_t off; };
  std::vector<Piece> pieces;
  std::vector<TailLevel> hdr(nt);
  uint64_t off = rnd16((uint64_t)nt * sizeof(TailLevel));
  const uint64_t vec_bytes = tail_vec_bytes(h, pi, top) - off;
  uint32_t mask = 0;
  bool staging = true;
  for (int l = 0; l < nt; ++l) {
    const LevelMats& B = h->L[l];
    const SellBuf& A = slot_A(B, pi);
    TailLevel& T = hdr[l];
    T.A = A.v;
    T.omega = B.omega;
    T.P = B.P.t;
    T.R = B.R.t;
    T.S = pi == 0 ? (const void*)B.S64 : (const void*)B.S32;
    std::vector<Piece> lp;
    uint64_t lo = off;
    auto add = [&](const void* src, uint64_t bytes) -> const void* {
      lp.push_back({src, bytes, (uint32_t)lo});
      const void* o = (const void*)(uintptr_t)lo;
      lo += rnd16(bytes);
      return o;
    };
    TailLevel S = T;
    S.A.sptr = (const int64_t*)add(A.v.sptr, (A.v.nslices + 1) * 8);
    S.A.col = (const int32_t*)add(A.v.col, A.slots * 4);
    S.A.val = add(A.v.val, A.slots * block_values(A.v, nc) * vs);
    S.S = add(T.S, B.n * nb * ts);
    if (l > 0)
      for (TransferView* V : {&S.P, &S.R}) {
        const SellBuf& X = V == &S.P ? B.P : B.R;
        V->sptr = (const int64_t*)add(X.t.sptr, (X.t.nslices + 1) * 8);
        V->col = (const int32_t*)add(X.t.col, X.slots * 4);
        V->w = (const float*)add(X.t.w, X.slots * 4);
      }
    if (staging && lo + vec_bytes <= kTailSmemMax) {
      T = S;
      mask |= 1u << l;
      pieces.insert(pieces.end(), lp.begin(), lp.end());
      off = lo;
    } else {
      staging = false;   // levels only grow: stage a prefix
    }
  }
  const uint32_t image_bytes = (uint32_t)off;
  uint64_t v = image_bytes;
  for (int l = 0; l < nt; ++l) {
    const uint64_t m = rnd16((uint64_t)h->L[l].n * nc * ts);
    hdr[l].b = (void*)(uintptr_t)v; v += m;
    hdr[l].o = (void*)(uintptr_t)v; v += m;
    hdr[l].t = (void*)(uintptr_t)v; v += m;
    hdr[l].r = (void*)(uintptr_t)v; v += m;
  }
  if (v > kTailSmemMax) return fail(MG_ERR_INVALID, "tail levels do not fit in shared memory");
  unsigned char* img = (unsigned char*)dev_alloc(h->ctx, h->allocs, h->bytes, image_bytes, true);
  if (!img) return fail(MG_ERR_OOM, "alloc");
  CU(cudaMemset(img, 0, image_bytes));
  CU(cudaMemcpy(img, hdr.data(), nt * sizeof(TailLevel), cudaMemcpyHostToDevice));
  for (const Piece& p : pieces) CU(cudaMemcpy(img + p.off, p.src, p.bytes, cudaMemcpyDeviceToDevice));
  // the memset and the copies ran on the legacy stream, and device-to-device
  // copies return before they complete: finish them before any stream (also
  // a non-blocking one, unordered with the legacy stream) reads the image
  CU(cudaStreamSynchronize(cudaStreamLegacy));
  mg_hier::TailImage ti;
  ti.p = img;
  ti.image_bytes = image_bytes;
  ti.smem = (uint32_t)v;
  ti.staged_mask = mask;
  h->tail_img[{pi, top}] = ti;
  *out = ti;
  return MG_OK;
}

// Cluster-resident image of levels 0..top for a cluster of C CTAs (scalar
// problems, levels without row permutation).  Level l is cut into chunks of
// 2^csh_l rows, chunk k belonging to CTA k; each CTA's section holds the
// header and the rows of its chunks of A, S, P (rows: level l) and R (rows:
// level l-1), copied from the device arrays; its vectors (b, o, t, r of every
// level, one chunk each) follow the largest section in shared memory, at the
// same offsets in every CTA.  Header offsets are shifted by the first index
// of the CTA's part of each array, so level-wide row, slot and column indices
// address the staged arrays directly.
constexpr int64_t kDsmWhole = 1024;

int tail_image_dsm(mg_hier* h, int pi, int top, int C, mg_hier::TailImage* out) {
  const int key = top | (C << 8);
  if (h->L[top].n <= kDsmWhole) return fail(MG_ERR_INVALID, "cluster-resident tail: no level to distribute");
  auto it = h->tail_img.find({pi, key});
  if (it != h->tail_img.end()) { *out = it->second; return MG_OK; }
  if (h->nc != 1) return fail(MG_ERR_INVALID, "cluster-resident tail: scalar problems only");
  const int nt = top + 1;
  const uint32_t ts = slot_tsize(pi), vs = slot_vsize(pi);
  struct Arr {
    std::vector<unsigned char> bytes;
  };
  auto down = [&](const void* src, size_t bytes, std::vector<unsigned char>& dst) -> int {
    dst.resize(bytes);
    if (bytes) CU(cudaMemcpy(dst.data(), src, bytes, cudaMemcpyDeviceToHost));
    return MG_OK;
  };
  std::vector<int> csh(nt);
  std::vector<TailLevel> base(nt);
  // host copies of the tail levels' arrays
  struct LevelHost {
    std::vector<unsigned char> sptr, col, col16, val, S, Psptr, Pcol, Pw, Rsptr, Rcol, Rw;
  };
  std::vector<LevelHost> LH(nt);
  int rc;
  for (int l = 0; l < nt; ++l) {
    const LevelMats& B = h->L[l];
    const SellBuf& A = slot_A(B, pi);
    if (A.v.perm || (l > 0 && (B.P.t.perm || B.R.t.perm || B.P.t.fix || B.R.t.fix)) || B.vanka)
      return fail(MG_ERR_INVALID, "cluster-resident tail: permuted, masked or Vanka level");
    // levels of at most kDsmWhole rows stay whole in CTA 0 (their steps need
    // no cluster barrier); larger ones are cut into C chunks
    int c = 5;
    if (B.n <= kDsmWhole)
      while (((int64_t)1 << c) < B.n) ++c;
    else
      while (((int64_t)C << c) < B.n) ++c;
    csh[l] = c;
    TailLevel& T = base[l];
    T.A = A.v;
    T.omega = B.omega;
    T.P = B.P.t;
    T.R = B.R.t;
    T.S = pi == 0 ? (const void*)B.S64 : (const void*)B.S32;   // device arrays unless the level is staged
    T.csh = c;
    LevelHost& H = LH[l];
    const int64_t slots = A.slots;
    if ((rc = down(A.v.sptr, (A.v.nslices + 1) * 8, H.sptr))) return rc;
    if ((rc = down(A.v.col, slots * 4, H.col))) return rc;
    if (A.v.col16 && (rc = down(A.v.col16, slots * 2, H.col16))) return rc;
    if ((rc = down(A.v.val, slots * vs, H.val))) return rc;
    if ((rc = down(pi == 0 ? (const void*)B.S64 : (const void*)B.S32, B.n * ts, H.S))) return rc;
    if (l > 0) {
      if ((rc = down(B.P.t.sptr, (B.P.t.nslices + 1) * 8, H.Psptr))) return rc;
      if ((rc = down(B.P.t.col, B.P.slots * 4, H.Pcol))) return rc;
      if ((rc = down(B.P.t.w, B.P.slots * 4, H.Pw))) return rc;
      if ((rc = down(B.R.t.sptr, (B.R.t.nslices + 1) * 8, H.Rsptr))) return rc;
      if ((rc = down(B.R.t.col, B.R.slots * 4, H.Rcol))) return rc;
      if ((rc = down(B.R.t.w, B.R.slots * 4, H.Rw))) return rc;
    }
  }
  // every column index a gather can meet must be a row of the gathered level
  for (int l = 0; l < nt; ++l) {
    const LevelHost& H = LH[l];
    const int32_t* col = (const int32_t*)H.col.data();
    for (size_t k = 0; k < H.col.size() / 4; ++k)
      if (col[k] < 0 || col[k] >= h->L[l].n) return fail(MG_ERR_INVALID, "cluster-resident tail: column out of range");
    if (l > 0) {
      const int32_t* pc = (const int32_t*)H.Pcol.data();
      for (size_t k = 0; k < H.Pcol.size() / 4; ++k)
        if (pc[k] < 0 || pc[k] >= h->L[l - 1].n) return fail(MG_ERR_INVALID, "cluster-resident tail: P column");
      const int32_t* rcl = (const int32_t*)H.Rcol.data();
      for (size_t k = 0; k < H.Rcol.size() / 4; ++k)
        if (rcl[k] < 0 || rcl[k] >= h->L[l].n) return fail(MG_ERR_INVALID, "cluster-resident tail: R column");
    }
  }
  const uint64_t hdr_bytes = rnd16((uint64_t)nt * sizeof(TailLevel));
  // vectors: one chunk per level and vector, at the same offsets in every CTA
  // (after the largest section, known once the sections are built)
  uint64_t vec_bytes = 0;
  for (int l = 0; l < nt; ++l) vec_bytes += 4 * (uint64_t)rnd16(((uint64_t)1 << csh[l]) * ts);
  if (hdr_bytes + vec_bytes > kTailSmemMax)
    return fail(MG_ERR_INVALID, "cluster-resident tail does not fit in shared memory");
  // per CTA: header + its rows of the matrices of the staged levels (coarsest
  // first while every CTA's section fits next to the vectors; the other
  // levels read the device arrays, whose level-wide indices work for any row)
  std::vector<std::vector<unsigned char>> sec(C, std::vector<unsigned char>(hdr_bytes, 0));
  std::vector<std::vector<TailLevel>> hdrs(C, base);
  uint32_t mask = 0;
  for (int l = 0; l < nt; ++l) {
    std::vector<std::vector<unsigned char>> trial = sec;
    std::vector<std::vector<TailLevel>> th = hdrs;
    uint64_t worst = 0;
    for (int c = 0; c < C; ++c) {
      std::vector<unsigned char>& out_c = trial[c];
      auto put = [&](const unsigned char* src, uint64_t bytes, int64_t first, uint32_t esize) -> const void* {
        const uint64_t q = out_c.size();
        out_c.resize(q + rnd16(bytes), 0);
        if (bytes) std::memcpy(out_c.data() + q, src, bytes);
        return (const void*)(intptr_t)((int64_t)q - first * (int64_t)esize);
      };
      // slices [s0, s1) of a SELL array whose chunk is rows [c 2^sh, (c+1) 2^sh)
      auto slices = [&](int64_t nslices, int sh, int64_t& s0, int64_t& s1) {
        s0 = std::min<int64_t>(nslices, ((int64_t)c << sh) >> 5);
        s1 = std::min<int64_t>(nslices, ((int64_t)(c + 1) << sh) >> 5);
      };
      const LevelHost& H = LH[l];
      TailLevel& T = th[c][l];
      int64_t s0, s1;
      slices(T.A.nslices, csh[l], s0, s1);
      const int64_t* sp = (const int64_t*)H.sptr.data();
      const int64_t o0 = sp[s0] & kSptrMask, o1 = sp[s1] & kSptrMask;
      T.A.sptr = (const int64_t*)put((const unsigned char*)(sp + s0), (s1 - s0 + 1) * 8, s0, 8);
      T.A.col = (const int32_t*)put(H.col.data() + o0 * 4, (o1 - o0) * 4, o0, 4);
      if (!H.col16.empty()) {
        T.A.col16 = (const int16_t*)put(H.col16.data() + o0 * 2, (o1 - o0) * 2, o0, 2);
        T.c16 = 1;
      }
      T.A.val = put(H.val.data() + o0 * vs, (o1 - o0) * vs, o0, vs);
      const int64_t r0 = std::min<int64_t>(h->L[l].n, (int64_t)c << csh[l]);
      const int64_t r1 = std::min<int64_t>(h->L[l].n, (int64_t)(c + 1) << csh[l]);
      T.S = put(H.S.data() + r0 * ts, (r1 - r0) * ts, r0, ts);
      if (l > 0) {
        for (int which = 0; which < 2; ++which) {     // P: rows of level l; R: rows of level l - 1
          TransferView& V = which == 0 ? T.P : T.R;
          const std::vector<unsigned char>& vsp = which == 0 ? H.Psptr : H.Rsptr;
          const std::vector<unsigned char>& vcol = which == 0 ? H.Pcol : H.Rcol;
          const std::vector<unsigned char>& vw = which == 0 ? H.Pw : H.Rw;
          int64_t t0, t1;
          slices(V.nslices, which == 0 ? csh[l] : csh[l - 1], t0, t1);
          const int64_t* tsp = (const int64_t*)vsp.data();
          const int64_t q0 = tsp[t0], q1 = tsp[t1];
          V.sptr = (const int64_t*)put((const unsigned char*)(tsp + t0), (t1 - t0 + 1) * 8, t0, 8);
          V.col = (const int32_t*)put(vcol.data() + q0 * 4, (q1 - q0) * 4, q0, 4);
          V.w = (const float*)put(vw.data() + q0 * 4, (q1 - q0) * 4, q0, 4);
        }
      }
      worst = std::max<uint64_t>(worst, out_c.size());
    }
    if (rnd16(worst) + vec_bytes > kTailSmemMax) break;   // levels only grow: stage a prefix
    sec.swap(trial);
    hdrs.swap(th);
    mask |= 1u << l;
  }
  // the levels left in device memory must have every array there
  for (int l = 0; l < nt; ++l) {
    if ((mask >> l) & 1u) continue;
    const TailLevel& T = base[l];
    if (!T.A.sptr || !T.A.col || !T.A.val || !T.S || (l > 0 && (!T.P.sptr || !T.P.col || !T.P.w || !T.R.sptr ||
                                                               !T.R.col || !T.R.w)))
      return fail(MG_ERR_INVALID, "cluster-resident tail: a level's arrays are missing");
  }
  uint64_t section = 0;
  for (auto& x : sec) section = std::max<uint64_t>(section, x.size());
  section = rnd16(section);
  uint64_t v = section;
  std::vector<uint64_t> vb(nt);
  for (int l = 0; l < nt; ++l) {
    vb[l] = v;
    v += 4 * (uint64_t)rnd16(((uint64_t)1 << csh[l]) * ts);
  }
  if (v > kTailSmemMax) return fail(MG_ERR_INVALID, "cluster-resident tail does not fit in shared memory");
  for (int c = 0; c < C; ++c) {
    std::vector<TailLevel>& hdr = hdrs[c];
    for (int l = 0; l < nt; ++l) {
      const int64_t chunk = rnd16(((uint64_t)1 << csh[l]) * ts), shift = ((int64_t)c << csh[l]) * (int64_t)ts;
      hdr[l].b = (void*)(intptr_t)((int64_t)vb[l] - shift);
      hdr[l].o = (void*)(intptr_t)((int64_t)vb[l] + chunk - shift);
      hdr[l].t = (void*)(intptr_t)((int64_t)vb[l] + 2 * chunk - shift);
      hdr[l].r = (void*)(intptr_t)((int64_t)vb[l] + 3 * chunk - shift);
    }
    std::memcpy(sec[c].data(), hdr.data(), nt * sizeof(TailLevel));
    sec[c].resize(section, 0);
  }
  unsigned char* img = (unsigned char*)dev_alloc(h->ctx, h->allocs, h->bytes, section * C, true);
  if (!img) return fail(MG_ERR_OOM, "alloc");
  for (int c = 0; c < C; ++c) CU(cudaMemcpy(img + c * section, sec[c].data(), section, cudaMemcpyHostToDevice));
  mg_hier::TailImage ti;
  ti.p = img;
  ti.image_bytes = (uint32_t)section;
  ti.section = (uint32_t)section;
  ti.smem = (uint32_t)v;
  ti.staged_mask = mask;
  CU(cudaStreamSynchronize(cudaStreamLegacy));   // complete before any stream reads it (see tail_image)
  h->tail_img[{pi, key}] = ti;
  *out = ti;
  return MG_OK;
}

void apply_tail(mg_hier* h, Workspace* w) {
  for (int pi = 0; pi < 3; ++pi) {
    TailParams* P = pi == 0 ? &w->tail64 : (pi == 1 ? &w->tail32 : &w->tail16);
    P->nt = h->tail_top + 1;
    P->cluster = h->tail_cluster < 0 ? -h->tail_cluster : h->tail_cluster;
    P->dsm = h->tail_cluster < 0 ? 1 : 0;
    P->image = nullptr;
    P->image_bytes = P->smem = P->staged_mask = P->section = 0;
    if (h->tail_cluster <= 0 && h->tail_top > 0 && has_slot(h, pi)) {
      const int key = h->tail_top | (h->tail_cluster < 0 ? (-h->tail_cluster) << 8 : 0);
      auto it = h->tail_img.find({pi, key});
      if (it != h->tail_img.end()) {
        P->image = it->second.p;
        P->image_bytes = it->second.image_bytes;
        P->smem = it->second.smem;
        P->staged_mask = it->second.staged_mask;
        P->section = it->second.section;
      }
    }
  }
  for (auto& g : w->graphs) cudaGraphExecDestroy(g.exec);
  w->graphs.clear();
}
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, std::pair<int, int>> g_tune_cache;   // shape -> (rows, cluster)
}  // namespace

// ---------------------------------------------------------------- layout tuning
// Layout of the FP32 / BF16 copies of one level operator (the V-cycle's in
// the mixed modes): the SELL-C-sigma window and the 16-bit column offsets.
// Both keep the summation order of every row, so no choice changes a bit of a
// V-cycle (the FP64 copies keep the size rule: the finest one is also the
// outer Krylov operator, whose SpMV kernels form dot products in SELL row
// order).  With opts.autotune the FP32 sweep of a level of >= 32768 rows is timed
// for a few windows, with and without 16-bit columns, and the fastest is kept
// (the size rule unless another is faster by 2 %), cached per level shape
// (dimension, components, row count in quarter-octaves, blocks per row);
// otherwise, or when opts fixes sell_sigma / col16, the size rules apply.
struct Layout {
  int64_t sigma;
  bool idx16;
};
std::mutex g_layout_mu;
std::map<std::vector<int64_t>, Layout> g_layout_cache;

Layout level_layout(mg_hier* h, const BlockCSR& A, bool pat6) {
  const int64_t n = A.n;
  const Layout rule{sigma_for(h, n), idx16_for(h, n)};
  const mg_opts& o = h->opts;
  // the small levels keep rows in node order (the cluster-resident tail
  // needs that; there the window barely changes the padding)
  if (!o.autotune || o.sell_sigma >= 0 || o.col16 >= 0 || !o.store_fp32 || n < kSigmaMinRows) return rule;
  const int nc = h->nc;
  const std::vector<int64_t> key = {h->dim, nc, (int64_t)std::llround(4.0 * std::log2((double)n)),
                                    (A.nnzb() * 8) / std::max<int64_t>(n, 1), pat6 ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_layout_mu);
    auto it = g_layout_cache.find(key);
    if (it != g_layout_cache.end()) return it->second;
  }
  std::vector<Alloc> tmp;
  size_t tb = 0;
  auto fbuf = [&](int64_t k) { return (float*)dev_alloc(h->ctx, tmp, tb, (size_t)k * 4, true); };
  float *x = fbuf(n * nc), *b = fbuf(n * nc), *out = fbuf(n * nc), *S = fbuf(n * nc * nc);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Layout best = rule;
  if (x && b && out && S && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    cudaStream_t s = h->ctx->stream;
    cudaMemsetAsync(x, 0, n * nc * 4, s);
    cudaMemsetAsync(b, 0, n * nc * 4, s);
    cudaMemsetAsync(S, 0, n * nc * nc * 4, s);
    std::vector<Layout> cands = {rule};
    for (int64_t sg : {int64_t(0), int64_t(256), int64_t(1024)})
      for (bool i16 : {false, true})
        if (sg != rule.sigma || i16 != rule.idx16) cands.push_back({sg, i16});
    double best_ms = 1e30;
    for (const Layout& c : cands) {
      SellBuf cand;
      std::vector<Alloc> ca;
      size_t cb = 0;
      if (upload_sell<float>(h, A, &cand, c.sigma, c.idx16, pat6, &ca, &cb) != MG_OK) {
        free_list(h->ctx, ca, cb);
        continue;
      }
      cand.v.tpr = tpr_for(h, nc, n);
      for (int i = 0; i < 2; ++i) launch_smooth<float>(cand.v, nc, x, b, S, out, 0.8, false, nullptr, s);
      cudaEventRecord(e0, s);
      for (int i = 0; i < 10; ++i) launch_smooth<float>(cand.v, nc, x, b, S, out, 0.8, false, nullptr, s);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      free_list(h->ctx, ca, cb);
      if (!ok) continue;
      if (best_ms == 1e30 || ms < 0.98 * best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(h->ctx->stream);
  free_list(h->ctx, tmp, tb);
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_layout_mu);
  g_layout_cache[key] = best;
  return best;
}

// ---------------------------------------------------------------- hierarchy
int upload_hierarchy(mg_hier* h, HostHierarchy& H) {
  const int nc = H.nc, nb = nc * nc;
  const int nlev = (int)H.levels.size();
  const mg_opts& opts = h->opts;
  h->L.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    HostLevel& lv = H.levels[l];
    LevelMats& B = h->L[l];
    B.n = lv.topo.n_nodes;
    B.omega = lv.omega;
    h->level_nodes.push_back(B.n);
    h->level_real_nnzb.push_back(lv.A.nnzb());
    int rc;
    const bool pat6 = velocity_pressure_pattern(lv.A);
    h->level_block_values.push_back(pat6 ? 6 : nb);
    const Layout lay = level_layout(h, lv.A, pat6);
    h->level_sigma.push_back(lay.sigma);
    // The finest FP64 operator is the outer Krylov residual's matrix in every
    // precision mode, so it is kept even without store_fp64 (which then only
    // drops the FP64 V-cycle: coarser FP64 operators and FP64 smoother blocks).
    if (opts.store_fp64 || l == nlev - 1) {
      // the FP64 copy keeps the size rule: it is also the outer Krylov
      // operator, whose SpMV kernels form dot products in SELL row order
      if ((rc = upload_sell<double>(h, lv.A, &B.A64, sigma_for(h, lv.A.n), idx16_for(h, lv.A.n), pat6))) return rc;
    }
    if (opts.store_fp64) {
      B.S64 = halloc<double>(h, B.n * nb);
      if (!B.S64) return fail(MG_ERR_OOM, "alloc");
      CU(cudaMemcpy(B.S64, lv.Sinv.data(), B.n * nb * 8, cudaMemcpyHostToDevice));
    }
    if (opts.store_fp32) {
      if ((rc = upload_sell<float>(h, lv.A, &B.A32, lay.sigma, lay.idx16, pat6))) return rc;
      B.A32.v.tpr = tpr_for(h, nc, lv.A.n);
      std::vector<float> s32(lv.Sinv.begin(), lv.Sinv.end());
      B.S32 = halloc<float>(h, B.n * nb);
      if (!B.S32) return fail(MG_ERR_OOM, "alloc");
      CU(cudaMemcpy(B.S32, s32.data(), B.n * nb * 4, cudaMemcpyHostToDevice));
    }
    if (opts.store_bf16) {
      if ((rc = upload_sell<__nv_bfloat16>(h, lv.A, &B.A16, lay.sigma, lay.idx16, pat6)))
        return rc;
      B.A16.v.bf16 = 1;
      B.A16.v.tpr = tpr_for(h, nc, lv.A.n);
      if (!B.S32) {
        std::vector<float> s32(lv.Sinv.begin(), lv.Sinv.end());
        B.S32 = halloc<float>(h, B.n * nb);
        if (!B.S32) return fail(MG_ERR_OOM, "alloc");
        CU(cudaMemcpy(B.S32, s32.data(), B.n * nb * 4, cudaMemcpyHostToDevice));
      }
    }
    if (lv.vanka) {
      B.vanka = true;
      if (opts.store_fp64 && (rc = upload_sell<double>(h, lv.Sv, &B.V64, sigma_for(h, lv.Sv.n), idx16_for(h, lv.Sv.n))))
        return rc;
      if (opts.store_fp32 || opts.store_bf16) {
        if ((rc = upload_sell<float>(h, lv.Sv, &B.V32, sigma_for(h, lv.Sv.n), idx16_for(h, lv.Sv.n)))) return rc;
        B.V32.v.tpr = tpr_for(h, nc, lv.Sv.n);
      }
    }
    // x staged per window for the one-lane scalar FP32 / BF16 sweeps
    const SellView& av = B.A32.slots ? B.A32.v : B.A16.v;
    const bool stage = nc == 1 && av.tpr == 1 && (B.A32.slots || B.A16.slots) &&
                       (opts.stage_x == 1 || (opts.stage_x < 0 && lv.A.n >= kSigmaMinRows));
    if (stage) {
      SellView w;
      if ((rc = stage_windows(h, lv.A, lay.sigma, w))) return rc;
      B.A32.v.wlo = B.A16.v.wlo = w.wlo;
      B.A32.v.wlen = B.A16.v.wlen = w.wlen;
    }
    h->level_nnzb.push_back(opts.store_fp64 ? B.A64.slots : B.A32.slots);
    h->level_col16.push_back(lay.idx16 ? 1 : 0);   // of the FP32 / BF16 copies
    if (l > 0) {
      if ((rc = upload_sell<float>(h, lv.P, &B.P, sigma_for(h, lv.P.n)))) return rc;
      if ((rc = upload_sell<float>(h, lv.R, &B.R, sigma_for(h, lv.R.n)))) return rc;
      // per-component rows of partly fixed nodes (block problems)
      auto partial_mask = [&](const HostLevel& X, const uint8_t** out) -> int {
        const uint8_t all = (uint8_t)((1 << nc) - 1);
        bool partial = false;
        for (uint8_t m : X.fixmask) partial |= (m != 0 && m != all);
        if (!partial) return MG_OK;
        uint8_t* d = (uint8_t*)dev_alloc(h->ctx, h->allocs, h->bytes, X.fixmask.size(), true);
        if (!d) return fail(MG_ERR_OOM, "alloc");
        CU(cudaMemcpy(d, X.fixmask.data(), X.fixmask.size(), cudaMemcpyHostToDevice));
        *out = d;
        return MG_OK;
      };
      if ((rc = partial_mask(lv, &B.P.t.fix))) return rc;
      if ((rc = partial_mask(H.levels[l - 1], &B.R.t.fix))) return rc;
    }
    // release host copies of what is now on the device
    if (l < nlev - 1) { lv.A = BlockCSR(); lv.leaves = LeafSet(); }
    lv.P = BlockCSR();
    lv.R = BlockCSR();
  }
  h->coarse_n = H.levels[0].topo.n_nodes * nc;
  h->coarse_inv = halloc<double>(h, h->coarse_n * h->coarse_n);
  if (!h->coarse_inv) return fail(MG_ERR_OOM, "alloc");
  CU(cudaMemcpy(h->coarse_inv, H.coarse_inv.data(), H.coarse_inv.size() * 8, cudaMemcpyHostToDevice));
  int rc;
  if ((rc = upload_sell<double>(h, H.load, &h->F))) return rc;
  const HostLevel& F = H.levels.back();
  const int64_t nn = F.topo.n_nodes;
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
    if ((rc = upload_sell<float>(h, Hm, &h->Hc))) return rc;
  }
  h->fixmask = (uint8_t*)dev_alloc(h->ctx, h->allocs, h->bytes, nn, true);
  if (!h->fixmask) return fail(MG_ERR_OOM, "alloc");
  CU(cudaMemcpy(h->fixmask, F.fixmask.data(), nn, cudaMemcpyHostToDevice));
  {
    std::vector<uint8_t> dm(nn);
    for (int64_t i = 0; i < nn; ++i) dm[i] = F.topo.hanging[i] ? 0 : F.fixmask[i];
    h->dirmask = (uint8_t*)dev_alloc(h->ctx, h->allocs, h->bytes, nn, true);
    if (!h->dirmask) return fail(MG_ERR_OOM, "alloc");
    CU(cudaMemcpy(h->dirmask, dm.data(), nn, cudaMemcpyHostToDevice));
  }
  if (H.lift.nnzb() > 0 && (rc = upload_sell<double>(h, H.lift, &h->Lift))) return rc;
  // tail: the largest prefix of levels (from the coarsest) with <= tail_rows dofs
  h->tail_top = tail_top_for(h, opts.tail_rows);
  h->tail_cluster = 1;
  return MG_OK;
}

void free_hierarchy(mg_hier* h) {
  for (Workspace* w : h->all_ws) ws_destroy(h, w);
  h->all_ws.clear();
  h->pool.clear();
  if (h->ws0) ws_destroy(h, h->ws0);
  h->ws0 = nullptr;
  free_list(h->ctx, h->allocs, h->bytes);
}

// ---------------------------------------------------------------- workspaces
size_t workspace_bytes(const mg_hier* h) {
  const int nc = h->nc;
  const int64_t n = h->n_dofs;
  size_t b = 0;
  for (const LevelMats& L : h->L) {
    const int64_t m = L.n * nc;
    if (h->has_fp64) b += 4 * rnd(m * 8);
    if (h->has_fp32 || h->has_bf16) b += 4 * rnd(m * 4);
  }
  b += 12 * rnd(n * 8) + 3 * rnd(n * 4) + rnd(Q_NUM * kMaxRedBlocks * 8) + rnd(sizeof(KrylovState));
  if (h->gmres_m > 0) {
    const int64_t m = h->gmres_m;
    b += rnd((m + 1) * n * 8) + (h->has_fp64 ? rnd(m * n * 8) : 0) + (h->has_fp32 || h->has_bf16 ? rnd(m * n * 4) : 0) +
         rnd((m + 1) * kMaxRedBlocks * 8) + 8 * rnd((m + 1) * (m + 1) * 8);
  }
  return b;
}

int ws_create(mg_hier* h, bool ctx_alloc, cudaStream_t s, Workspace** out) {
  auto w = std::make_unique<Workspace>();
  mg_ctx* c = h->ctx;
  const int nc = h->nc;
  const int64_t n = h->n_dofs;
  auto A8 = [&](int64_t k) { return (double*)dev_alloc(c, w->allocs, w->bytes, (size_t)std::max<int64_t>(k, 1) * 8, ctx_alloc); };
  auto A4 = [&](int64_t k) { return (float*)dev_alloc(c, w->allocs, w->bytes, (size_t)std::max<int64_t>(k, 1) * 4, ctx_alloc); };
  bool ok = true;
  w->lv.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    LevelVecs& v = w->lv[l];
    const int64_t m = h->L[l].n * nc;
    if (h->has_fp64) { v.b64 = A8(m); v.o64 = A8(m); v.t64 = A8(m); v.r64 = A8(m); ok &= v.b64 && v.o64 && v.t64 && v.r64; }
    if (h->has_fp32 || h->has_bf16) { v.b32 = A4(m); v.o32 = A4(m); v.t32 = A4(m); v.r32 = A4(m); ok &= v.b32 && v.o32 && v.t32 && v.r32; }
  }
  double** vecs[] = {&w->xi, &w->bi, &w->r, &w->p, &w->q, &w->z, &w->rhat, &w->sv, &w->t, &w->ph, &w->shat, &w->vcur};
  for (double** v : vecs) { *v = A8(n); ok &= *v != nullptr; }
  float** v32[] = {&w->r32, &w->ph32, &w->sh32};
  for (float** v : v32) { *v = A4(n); ok &= *v != nullptr; }
  w->part.p = A8(Q_NUM * kMaxRedBlocks);
  w->st = (KrylovState*)dev_alloc(c, w->allocs, w->bytes, sizeof(KrylovState), ctx_alloc);
  ok &= w->part.p && w->st;
  if (h->gmres_m > 0 && ok) {
    const int m = h->gmres_m;
    GmresView& G = w->gm;
    G.m = m;
    G.H = A8((int64_t)(m + 1) * m);
    G.cs = A8(m); G.sn = A8(m); G.g = A8(m + 1); G.hv = A8(m + 1); G.y = A8(m); G.zs = A8(m);
    G.part = A8((int64_t)(m + 1) * kMaxRedBlocks);
    G.V = A8((int64_t)(m + 1) * n);
    if (h->has_fp64) G.Z64 = A8((int64_t)m * n);
    if (h->has_fp32 || h->has_bf16) G.Z32 = A4((int64_t)m * n);
    ok &= G.H && G.cs && G.sn && G.g && G.hv && G.y && G.zs && G.part && G.V && (!h->has_fp64 || G.Z64) &&
          (!(h->has_fp32 || h->has_bf16) || G.Z32);
  }
  if (!ok) {
    free_list(c, w->allocs, w->bytes);
    return fail(MG_ERR_OOM, "workspace allocation failed");
  }
  // initialised in stream order on the stream the solves will use
  for (double** v : vecs) CU(cudaMemsetAsync(*v, 0, n * 8, s));
  CU(cudaMemsetAsync(w->part.p, 0, Q_NUM * kMaxRedBlocks * 8, s));
  CU(cudaMemsetAsync(w->st, 0, sizeof(KrylovState), s));
  CU(cudaMallocHost(&w->st_host, sizeof(KrylovState)));
  CU(cudaEventCreate(&w->ev0));
  CU(cudaEventCreate(&w->ev1));
  // tail parameters: matrices of the hierarchy, vectors of this workspace
  for (int pi = 0; pi < 3; ++pi) {
    TailParams& P = pi == 0 ? w->tail64 : (pi == 1 ? w->tail32 : w->tail16);
    const bool d = pi == 0;
    if (pi == 0 ? !h->has_fp64 : (pi == 1 ? !h->has_fp32 : !h->has_bf16)) continue;
    P.nu1 = h->opts.nu1;
    P.nu2 = h->opts.nu2;

    P.cinv = h->coarse_inv;
    P.cn = h->coarse_n;
    for (int l = 0; l < h->nlev && l < kTailMax; ++l) {
      LevelMats& B = h->L[l];
      LevelVecs& V = w->lv[l];
      TailLevel& T = P.lv[l];
      T.A = d ? B.A64.v : (pi == 1 ? B.A32.v : B.A16.v);
      T.omega = B.omega;
      T.P = B.P.t;
      T.R = B.R.t;
      T.S = d ? (const void*)B.S64 : (const void*)B.S32;
      T.b = d ? (void*)V.b64 : (void*)V.b32;
      T.o = d ? (void*)V.o64 : (void*)V.o32;
      T.t = d ? (void*)V.t64 : (void*)V.t32;
      T.r = d ? (void*)V.r64 : (void*)V.r32;
    }
  }
  apply_tail(h, w.get());
  *out = w.release();
  return MG_OK;
}

void ws_destroy(mg_hier* h, Workspace* w) {
  if (!w) return;
  for (auto& g : w->graphs) cudaGraphExecDestroy(g.exec);
  if (w->st_host) cudaFreeHost(w->st_host);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  free_list(h->ctx, w->allocs, w->bytes);
  delete w;
}

int set_tail(mg_hier* h, int rows, int cluster) {
  int top = tail_top_for(h, rows);
  cluster = std::max(-16, std::min(cluster, 16));
  if (cluster < 0) {   // cluster-resident tail of -cluster CTAs
    if (cluster != -2 && cluster != -4 && cluster != -8 && cluster != -16)
      return fail(MG_ERR_INVALID, "cluster-resident tail: 2, 4, 8 or 16 CTAs");
    if (top == 0) cluster = 1;
    for (int pi = 0; pi < 3 && top > 0; ++pi) {
      mg_hier::TailImage ti;
      int rc;
      if (!has_slot(h, pi)) continue;
      if ((rc = tail_image_dsm(h, pi, top, -cluster, &ti))) return rc;
      if (!tail_dsm_fits(-cluster, ti.smem)) return fail(MG_ERR_INVALID, "cluster-resident tail not schedulable");
    }
  } else if (!tail_cluster_fits(cluster)) {
    return fail(MG_ERR_INVALID, "tail cluster size not schedulable on this GPU");
  }
  if (cluster == 0) {
    top = staged_top_cap(h, top);
    for (int pi = 0; pi < 3 && top > 0; ++pi) {
      mg_hier::TailImage ti;
      int rc;
      if (has_slot(h, pi) && (rc = tail_image(h, pi, top, &ti))) return rc;
    }
  }
  h->tail_top = top;
  h->tail_cluster = cluster;
  if (h->ws0) apply_tail(h, h->ws0);
  std::lock_guard<std::mutex> lk(h->pool_mu);
  for (Workspace* w : h->all_ws) apply_tail(h, w);
  return MG_OK;
}

int autotune(mg_hier* h, int prec) {
  std::vector<int64_t> key = {h->dim, h->nc, prec, h->opts.nu1, h->opts.nu2};
  for (const LevelMats& L : h->L) key.push_back(L.vanka ? -L.n : L.n);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      return set_tail(h, it->second.first, it->second.second);
    }
  }
  Workspace& w = *h->ws0;
  cudaStream_t s = h->ctx->stream;
  const int fine = h->nlev - 1;
  const int rows_c[] = {0, 256, 1024, 4096, 16384, 65536};
  // 0: one CTA in shared memory.  The cluster-resident shapes (mg_tune with a
  // negative cluster) are not among the candidates: on the adaptive
  // transport hierarchy every one of them was slower than the shared-memory
  // CTA (V(5,5) cycle 487-575 us against 460 us; the gathers that cross CTA
  // chunks wait on distributed-shared-memory latency in every batch)
  const int cl_c[] = {1, 0, 2, 4, 8, 16};
  double best = 1e30;
  int best_rows = 0, best_cl = 1, last_top = -1;
  for (int rows : rows_c) {
    const int top = tail_top_for(h, rows);
    if (top == last_top) continue;      // same split as a smaller threshold
    last_top = top;
    for (int cl : cl_c) {
      if (top == 0 && cl != 1) break;
      if (!tail_cluster_fits(cl)) continue;
      int rc = set_tail(h, rows, cl);
      if (rc) return rc;
      auto once = [&]() {
        if (prec == MG_FP64) enqueue_vcycle<double>(h, w, fine, w.r, w.z, nullptr, s);
        else enqueue_vcycle<float>(h, w, fine, w.r32, w.ph32, nullptr, s, false, prec == MG_MIXED_BF16);
      };
      once();
      CU(cudaEventRecord(w.ev0, s));
      for (int i = 0; i < 8; ++i) once();
      CU(cudaEventRecord(w.ev1, s));
      CU(cudaEventSynchronize(w.ev1));
      float ms = 0.0f;
      CU(cudaEventElapsedTime(&ms, w.ev0, w.ev1));
      CU(cudaGetLastError());
      const double t = ms / 8.0;
      if (t < best * 0.98) { best = t; best_rows = rows; best_cl = cl; }
    }
  }
  int rc = set_tail(h, best_rows, best_cl);
  if (rc) return rc;
  h->tuned_vcycle_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_rows, best_cl};
  return MG_OK;
}

// ---------------------------------------------------------------- V-cycle
// z = GMG(l, 0, b): one V-cycle on level l from a zero initial guess (Sec. 2.2).
// first_done: the first pre-smoothing sweep (from x = 0) was already written
// into its buffer by the restriction kernel of the finer level.
template <typename T>
bool enqueue_vcycle(mg_hier* h, Workspace& w, int l, const T* b, T* out, const int* done, cudaStream_t s,
                    bool first_done, bool bf16, double* out64, const double* scale) {
  const int nc = h->nc;
  struct LevelTag {          // launches below belong to level l (per-kernel timing)
    int prev;
    explicit LevelTag(int l) : prev(t_prof_level) { t_prof_level = l; }
    ~LevelTag() { t_prof_level = prev; }
  } tag(l);
  if (l == 0) {                                                  // coarse solve
    launch_coarse<T>(h->coarse_inv, h->coarse_n, b, out, done, s);
    h->launch_count++;
    return false;
  }
  if (l <= h->tail_top) {                                        // small levels: one cluster
    const TailParams& TP = bf16 ? w.tail16 : Prec<T>::tail(w);
    if (l < h->tail_top) {
      // a cycle started below the tail's top level (measurement only): the
      // kernel's top must be level l, whose vectors b and out are given
      TailParams sub = TP;
      sub.nt = l + 1;
      launch_tail<T>(sub, nc, b, out, first_done, done, s, out64, scale);
    } else {
      launch_tail<T>(TP, nc, b, out, first_done, done, s, out64, scale);
    }
    h->launch_count++;
    return out64 != nullptr && h->opts.nu2 > 0;
  }
  LevelMats& L = h->L[l];
  const SellView& AL = bf16 ? L.A16.v : Prec<T>::A(L);
  LevelVecs& V = w.lv[l];
  LevelMats& C = h->L[l - 1];
  LevelVecs& CV = w.lv[l - 1];
  const int nu1 = h->opts.nu1, nu2 = h->opts.nu2, ns = nu1 + nu2;
  auto bufof = [&](LevelVecs& X, T* o, int k) -> T* { return ((ns - 1 - k) % 2 == 0) ? o : Prec<T>::t(X); };
  const double om = L.omega, omc = C.omega;
  // one smoothing sweep cur -> dst: fused residual + Jacobi, or (Vanka) the
  // residual into the level's r buffer, then dst = cur + w S r (from zero:
  // dst = w S b, no residual)
  auto sweep = [&](const T* in, T* dst, bool from_zero, double* o64, const double* sc) {
    if (!L.vanka) {
      launch_smooth<T>(AL, nc, in, b, Prec<T>::S(L), dst, om, from_zero, done, s, o64, sc);
      h->launch_count++;
      return;
    }
    if (!from_zero) {
      launch_residual<T>(AL, nc, in, b, Prec<T>::r(V), done, s);
      h->launch_count++;
    }
    launch_vanka<T>(Prec<T>::V(L), nc, from_zero ? b : Prec<T>::r(V), from_zero ? nullptr : in, dst, om, done, s,
                    o64, sc);
    h->launch_count++;
  };
  T* cur = nullptr;
  for (int k = 0; k < nu1; ++k) {                                // pre-smoothing
    T* dst = bufof(V, out, k);
    if (!(k == 0 && first_done)) sweep(cur, dst, k == 0, nullptr, nullptr);
    cur = dst;
  }
  launch_residual<T>(AL, nc, cur, b, Prec<T>::r(V), done, s);   // residual, restricted below
  // the restriction also performs the coarser level's first (Jacobi) sweep
  const bool fuse = l - 1 > 0 && !C.vanka;
  T* cfirst = fuse ? bufof(CV, Prec<T>::o(CV), 0) : nullptr;
  launch_restrict<T>(L.R.t, nc, Prec<T>::r(V), Prec<T>::b(CV), Prec<T>::S(C), cfirst, omc, done, s);
  h->launch_count += 2;
  enqueue_vcycle<T>(h, w, l - 1, Prec<T>::b(CV), Prec<T>::o(CV), done, s, fuse, bf16);   // coarser cycle
  T* pdst = nu2 == 0 ? out : cur;                                                   // correction
  launch_prolong_add<T>(L.P.t, nc, Prec<T>::o(CV), cur, pdst, done, s);
  cur = pdst;
  h->launch_count++;
  for (int k = nu1; k < ns; ++k) {                               // post-smoothing
    T* dst = bufof(V, out, k);
    const bool last = k == ns - 1;
    sweep(cur, dst, false, last ? out64 : nullptr, last ? scale : nullptr);
    cur = dst;
  }
  return out64 != nullptr && nu2 > 0;
}
template bool enqueue_vcycle<double>(mg_hier*, Workspace&, int, const double*, double*, const int*, cudaStream_t,
                                     bool, bool, double*, const double*);
template bool enqueue_vcycle<float>(mg_hier*, Workspace&, int, const float*, float*, const int*, cudaStream_t, bool,
                                    bool, double*, const double*);

// ---------------------------------------------------------------- Krylov
enum { M_CG = 1, M_BICG = 2, M_GMRES = 3, M_MGI = 4 };

int method_of(const mg_hier* h) {
  int k = h->opts.krylov;
  if (k == MG_KRYLOV_AUTO)
    k = h->prob.kind == MG_TRANSPORT ? MG_BICGSTAB : (h->prob.kind == MG_OSEEN ? MG_GMRES : MG_CG);
  if (k == MG_MGITER) return M_MGI;
  return k == MG_BICGSTAB ? M_BICG : (k == MG_GMRES ? M_GMRES : M_CG);
}

int check_prec(const mg_hier* h, int prec) {
  if (h->L.empty() || h->L.back().A64.v.nslices == 0)
    return fail(MG_ERR_INVALID, "hierarchy has no FP64 finest-level operator for the outer residual");
  if (prec == MG_FP64 && !h->has_fp64) return fail(MG_ERR_INVALID, "hierarchy built without FP64 level matrices");
  if (prec == MG_MIXED_FP32 && !h->has_fp32) return fail(MG_ERR_INVALID, "hierarchy built without FP32 level matrices");
  if (prec == MG_MIXED_BF16 && !h->has_bf16) return fail(MG_ERR_INVALID, "hierarchy built without BF16 level matrices");
  if (prec != MG_FP64 && prec != MG_MIXED_FP32 && prec != MG_MIXED_BF16) return fail(MG_ERR_INVALID, "unsupported precision");
  return MG_OK;
}

namespace {

// One Krylov iteration (the body of the graph's while node).  The last kernel
// of the iteration runs the convergence test and sets the while condition.
void enqueue_iteration(mg_hier* h, Workspace& w, int method, int prec, unsigned long long cond, cudaStream_t s) {
  const int nc = h->nc;
  const int fine = h->nlev - 1;
  const int64_t n = h->n_dofs;
  const SellView& A = h->L[fine].A64.v;
  const int* done = &w.st->done;
  const bool mixed = prec != MG_FP64;
  const bool bf16 = prec == MG_MIXED_BF16;
  if (cond) {
    launch_cond_reset(cond, s);
    h->launch_count++;
  }
  const double* scale = &w.st->scale;
  if (method == M_MGI) {
    // the multigrid cycle as the solver: x <- x + GMG(0, b - A x)
    PVec z;
    if (mixed) {
      launch_to_f32(n, w.r, w.r32, w.st, s);
      if (enqueue_vcycle<float>(h, w, fine, w.r32, w.ph32, done, s, false, bf16, w.z, scale)) z.d = w.z;
      else z.f = w.ph32;
      h->launch_count++;
    } else {
      enqueue_vcycle<double>(h, w, fine, w.r, w.z, done, s);
      z.d = w.z;
    }
    launch_mgi_update(n, z, w.xi, w.st, s);
    launch_residual_norm(A, nc, w.xi, w.bi, w.r, w.part, w.st, 2, s, cond);
    h->launch_count += 2;
  } else if (method == M_CG) {
    PVec z;
    if (mixed) {
      launch_to_f32(n, w.r, w.r32, w.st, s);
      if (enqueue_vcycle<float>(h, w, fine, w.r32, w.ph32, done, s, false, bf16, w.z, scale)) z.d = w.z;
      else z.f = w.ph32;
      h->launch_count++;
    } else {
      enqueue_vcycle<double>(h, w, fine, w.r, w.z, done, s);
      z.d = w.z;
    }
    launch_cg_dots(n, z, w.r, w.q, w.part, w.st, s);
    launch_cg_update_p(n, z, w.p, w.st, s);
    PVec pp;
    pp.d = w.p;
    launch_spmv_dot(A, nc, pp, nullptr, w.q, w.part, Q_PQ, w.st, s);
    launch_cg_update_xr(n, w.p, w.q, w.xi, w.r, w.part, w.st, cond, s);
    h->launch_count += 4;
  } else if (method == M_GMRES) {
    // one Arnoldi step of flexible GMRES(m); cycle end and restart are gated
    // on the device (gm_end / gm_j).  The view carries only the preconditioned
    // vectors of the active precision.
    GmresView gm = w.gm;
    if (mixed) gm.Z64 = nullptr;
    else gm.Z32 = nullptr;
    PVec z;
    if (mixed) { enqueue_vcycle<float>(h, w, fine, w.r32, w.ph32, done, s, false, bf16); z.f = w.ph32; }
    else { enqueue_vcycle<double>(h, w, fine, w.vcur, w.z, done, s); z.d = w.z; }
    launch_gm_spmv(A, nc, z, w.q, gm, w.st, s);
    launch_gm_orth(n, w.q, gm, w.st, 0, w.part, s);
    launch_gm_orth(n, w.q, gm, w.st, 1, w.part, s);
    launch_gm_givens(gm, w.st, s);
    launch_gm_next(n, w.q, mixed ? w.r32 : nullptr, mixed ? nullptr : w.vcur, gm, w.st, s);
    launch_gm_update_x(n, w.xi, gm, w.st, s);
    launch_gm_residual(A, nc, w.xi, w.bi, w.r, w.part, w.st, cond, s);
    launch_gm_start(n, w.r, mixed ? w.r32 : nullptr, mixed ? nullptr : w.vcur, gm, w.st, s);
    h->launch_count += 1 + 3 * 2 + 1 + 2 + 1 + 1 + 1;
  } else {
    // in mixed mode bicg_p / bicg_s also write the FP32 preconditioner input
    launch_bicg_p(n, w.r, w.t /* v */, w.p, mixed ? w.r32 : nullptr, w.st, s);
    PVec ph;
    if (mixed) {
      if (enqueue_vcycle<float>(h, w, fine, w.r32, w.ph32, done, s, false, bf16, w.ph, scale)) ph.d = w.ph;
      else ph.f = w.ph32;
    } else {
      enqueue_vcycle<double>(h, w, fine, w.p, w.ph, done, s);
      ph.d = w.ph;
    }
    launch_spmv_dot(A, nc, ph, w.rhat, w.t /* v */, w.part, Q_RHV, w.st, s);
    launch_bicg_s(n, w.r, w.t, w.sv, mixed ? w.r32 : nullptr, w.st, s);
    PVec sh;
    if (mixed) {
      if (enqueue_vcycle<float>(h, w, fine, w.r32, w.sh32, done, s, false, bf16, w.shat, scale)) sh.d = w.shat;
      else sh.f = w.sh32;
    } else {
      enqueue_vcycle<double>(h, w, fine, w.sv, w.shat, done, s);
      sh.d = w.shat;
    }
    launch_spmv_2dots(A, nc, sh, w.sv, w.q /* t */, w.part, w.st, s);
    launch_bicg_x(n, ph, sh, w.sv, w.q, w.rhat, w.xi, w.r, w.part, w.st, cond, s);
    h->launch_count += 5;
  }
}

int build_graph(mg_hier* h, Workspace& w, int method, int prec, SolveGraph* out) {
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
  const int64_t before = h->launch_count;
  enqueue_iteration(h, w, method, prec, (unsigned long long)handle, cs);
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

}  // namespace

int get_graph(mg_hier* h, Workspace& w, int method, int prec, SolveGraph** g) {
  for (auto& x : w.graphs)
    if (x.method == method && x.prec == prec) { *g = &x; return MG_OK; }
  SolveGraph ng;
  int rc = build_graph(h, w, method, prec, &ng);
  if (rc) return rc;
  w.graphs.push_back(ng);
  *g = &w.graphs.back();
  return MG_OK;
}

namespace {

// One round: residual of the current iterate, the device loop (graph or
// direct launches), the true residual, outputs and the state mirror.
int enqueue_round(mg_hier* h, Workspace& w, cudaStream_t s) {
  const int nc = h->nc;
  const int fine = h->nlev - 1;
  const SellView& A = h->L[fine].A64.v;
  const int method = w.method, prec = w.prec;
  SolveGraph* g = nullptr;
  // a profiled solve captures its own graph: the cached one must not pick up
  // the profiler's event nodes
  EventProfiler* prof = dynamic_cast<EventProfiler*>(t_prof);
  if (h->opts.launch_mode != 1 && !prof) {
    int rc = get_graph(h, w, method, prec, &g);
    if (rc) return rc;
  }
  w.graph_round = g != nullptr;
  launch_residual_norm(A, nc, w.xi, w.bi, w.r, w.part, w.st, 1, s);
  w.launches += 1;
  if (method == M_GMRES) {
    GmresView gm = w.gm;
    launch_gm_start(h->n_dofs, w.r, prec != MG_FP64 ? w.r32 : nullptr, prec != MG_FP64 ? nullptr : w.vcur, gm,
                    w.st, s);
    w.launches += 1;
  } else if (method == M_BICG) {
    // rhat = r0, (rhat, r) = (r, r)
    CU(cudaMemcpyAsync(w.rhat, w.r, h->n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(&w.st->red[Q_RHR], &w.st->red[Q_RR], sizeof(double), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(w.t, 0, h->n_dofs * sizeof(double), s));
  } else {
    CU(cudaMemsetAsync(w.q, 0, h->n_dofs * sizeof(double), s));
  }
  if (prof) {
    // per-kernel timing: one iteration captured as a plain graph (an
    // event-record node after every run of the same kernel), run once per
    // iteration, status polled
    cudaStream_t cs;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    prof->begin_capture();
    cudaGraph_t g1 = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int64_t before = h->launch_count;
    if (e == cudaSuccess) {
      const int lv = t_prof_level;
      t_prof_level = -2;             // the floor of an interval: an empty kernel
      launch_prof_empty(cs);
      t_prof_level = lv;
      before = h->launch_count;
      enqueue_iteration(h, w, method, prec, 0ull, cs);
      prof->end_capture();
      e = cudaStreamEndCapture(cs, &g1);
    }
    const int64_t per_iter = h->launch_count - before;
    h->launch_count = before;
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g1, 0);
    if (g1) cudaGraphDestroy(g1);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("profiled iteration graph: ") + cudaGetErrorString(e));
    struct ExecGuard {           // the graph goes on every return path
      cudaGraphExec_t x;
      ~ExecGuard() { cudaGraphExecDestroy(x); }
    } guard{ex};
    bool ran = false;
    for (int it = 0; it < w.max_it + 1; ++it) {
      CU(cudaMemcpyAsync(w.st_host, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (ran) prof->collect_graph();
      ran = false;
      if (w.st_host->done) break;
      CU(cudaGraphLaunch(ex, s));
      w.launches += per_iter;
      ran = true;
    }
    if (ran) {
      CU(cudaStreamSynchronize(s));
      prof->collect_graph();
    }
  } else if (h->opts.launch_mode == 1) {
    // direct launches (profilers): one iteration at a time, status polled
    const int64_t before = h->launch_count;
    for (int it = 0; it < w.max_it + 1; ++it) {
      CU(cudaMemcpyAsync(w.st_host, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (w.st_host->done) break;
      enqueue_iteration(h, w, method, prec, 0ull, s);
    }
    w.launches += h->launch_count - before;
    h->launch_count = before;
  } else {
    CU(cudaGraphLaunch(g->exec, s));
  }
  // true residual of the final iterate, solution with hanging values, state
  launch_residual_norm(A, nc, w.xi, w.bi, w.r, w.part, w.st, 0, s);
  launch_copy_fixed(h->n_nodes, nc, h->fixmask, w.bi, w.xi, w.p, s);     // p <- x (hanging/Dirichlet from b)
  launch_fill_hanging(h->Hc.t, nc, w.p, s);
  w.launches += 3;
  CU(cudaMemcpyAsync(w.x_out, w.p, h->n_dofs * 8, w.x_out_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     s));
  CU(cudaMemcpyAsync(w.st_host, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  CU(cudaEventRecord(w.ev1, s));
  return MG_OK;
}

}  // namespace

// ------------------------------------------------------------ EventProfiler
int EventProfiler::init(size_t graph_events) {
  graph_pool.resize(graph_events);
  for (auto& e : graph_pool) CU(cudaEventCreate(&e));
  return MG_OK;
}

void EventProfiler::before(const void* fn, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  pending = false;
  if (cap == cudaStreamCaptureStatusActive) {
    if (run_open && graph_recs.back().fn == fn && graph_recs.back().level == t_prof_level) {
      graph_recs.back().n += 1;          // the run goes on: no event between its launches
      return;
    }
    close_run();
    const bool first = graph_recs.empty();
    if (graph_used + (first ? 2 : 1) > graph_pool.size()) {
      ++dropped;
      return;
    }
    Rec r{fn, t_prof_level, nullptr, nullptr};
    if (first) {
      r.e0 = graph_pool[graph_used++];
      cudaEventRecordWithFlags(r.e0, s, cudaEventRecordExternal);
    } else {
      r.e0 = graph_recs.back().e1;
    }
    r.e1 = graph_pool[graph_used++];
    graph_recs.push_back(r);
    run_open = true;                     // its end event follows the run's last launch
    run_stream = s;
    return;
  } else {
    Rec r{fn, t_prof_level, nullptr, nullptr};
    if (cudaEventCreate(&r.e0) != cudaSuccess) return;
    if (cudaEventCreate(&r.e1) != cudaSuccess) {
      cudaEventDestroy(r.e0);
      return;
    }
    direct_pool.push_back(r.e0);
    direct_pool.push_back(r.e1);
    cudaEventRecord(r.e0, s);
    direct_recs.push_back(r);
  }
  pending = true;
}

void EventProfiler::after(cudaStream_t s) {
  if (!pending) return;                  // captured launches: the run's end event comes later
  pending = false;
  cudaEventRecord(direct_recs.back().e1, s);
}

void EventProfiler::close_run() {
  if (!run_open) return;
  run_open = false;
  cudaEventRecordWithFlags(graph_recs.back().e1, run_stream, cudaEventRecordExternal);
}

static void add_recs(std::map<std::pair<const void*, int>, std::pair<int64_t, double>>& acc,
                     const std::vector<EventProfiler::Rec>& recs) {
  for (const auto& r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) continue;
    auto& a = acc[{r.fn, r.level}];
    a.first += r.n;
    a.second += ms;
  }
}

void EventProfiler::collect_graph() { add_recs(acc, graph_recs); }

void EventProfiler::collect_direct() {
  add_recs(acc, direct_recs);
  direct_recs.clear();
}

EventProfiler::~EventProfiler() {
  for (auto e : graph_pool) cudaEventDestroy(e);
  for (auto e : direct_pool) cudaEventDestroy(e);
}

int solve_start(mg_hier* h, Workspace& w, const double* b, bool b_host, const double* x0, bool x0_host,
                double* x_out, bool x_out_host, double rtol, int max_it, int prec, cudaStream_t s) {
  const int64_t n = h->n_dofs;
  w.method = method_of(h);
  w.prec = prec;
  w.rtol = rtol;
  w.max_it = max_it;
  w.rounds = 0;
  w.iter_base = 0;
  w.launches = 0;
  w.x_out = x_out;
  w.x_out_host = x_out_host;
  if (w.method == M_GMRES && !w.gm.V) return fail(MG_ERR_INVALID, "hierarchy set up without GMRES workspace");
  CU(cudaEventRecord(w.ev0, s));
  CU(cudaMemsetAsync(&w.st->counter, 0, sizeof(unsigned int), s));   // reduction arrival counter
  if (b != w.bi)   // a time step assembles its right-hand side in place
    CU(cudaMemcpyAsync(w.bi, b, n * 8, b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  CU(cudaMemcpyAsync(w.p, x0, n * 8, x0_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  launch_copy_fixed(h->n_nodes, h->nc, h->fixmask, w.bi, w.p, w.xi, s);
  // defect correction: the first round stops at inner_rtol (relative to b; x0
  // contributes through the recomputed defect of the next round)
  const double inner = h->opts.inner_rtol;
  launch_norm_init(h->n_nodes, h->nc, h->fixmask, w.bi, w.part, w.st, inner > 0 ? std::max(rtol, inner) : rtol,
                   max_it, s);
  w.launches += 2;
  return enqueue_round(h, w, s);
}

int solve_check(mg_hier* h, Workspace& w, cudaStream_t s, mg_stats* stats) {
  const KrylovState& S = *w.st_host;
  const double rel = std::sqrt(S.red[Q_RR]) / S.bnorm;
  SolveGraph* g = nullptr;   // the round's device loop ran as this graph (launches counted per iteration)
  if (w.graph_round)
    for (auto& x : w.graphs)
      if (x.method == w.method && x.prec == w.prec) g = &x;
  int status;
  if (S.status == -6) status = MG_ERR_NAN;
  else if (S.status == -5) status = MG_ERR_BREAKDOWN;
  else if (rel <= w.rtol) status = MG_OK;
  else if (S.iter >= w.max_it || w.rounds >= (h->opts.inner_rtol > 0 ? 200 : 3)) status = MG_ERR_NOT_CONVERGED;
  else status = MG_PENDING;
  const int iters_round = S.iter - w.iter_base;
  if (status == MG_PENDING) {
    // the recursive residual converged but the true one did not: restart
    // from the true residual, keeping the iteration count
    KrylovState fix = S;
    fix.done = 0;
    fix.status = 0;
    fix.restart_pos = fix.iter;
    fix.gm_j = 0;
    fix.gm_end = 0;
    // defect correction: this round reduces the current true defect by inner_rtol
    if (h->opts.inner_rtol > 0) fix.rtol = std::max(w.rtol, h->opts.inner_rtol * rel);
    *w.st_host = fix;
    CU(cudaMemcpyAsync(w.st, w.st_host, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
    // reset hanging / Dirichlet entries of the iterate
    launch_copy_fixed(h->n_nodes, h->nc, h->fixmask, w.bi, w.xi, w.xi, s);
    w.launches += 1;
    w.rounds += 1;
    w.iter_base = S.iter;
    if (g) w.launches += (int64_t)iters_round * g->launches_per_iter;
    int rc = enqueue_round(h, w, s);
    return rc ? rc : MG_PENDING;
  }
  if (g) w.launches += (int64_t)iters_round * g->launches_per_iter;
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, w.ev0, w.ev1);
  if (stats) {
    stats->status = status;
    stats->iters = S.iter;
    stats->vcycles = S.iter * (w.method == M_BICG ? 2 : 1);
    stats->precision = w.prec;
    stats->rel_res = rel;
    stats->solve_ms = ms;
    stats->launches = w.launches;
  }
  h->launch_count += w.launches;
  return status;
}


void* ctx_alloc(mg_ctx* c, std::vector<Alloc>& list, size_t& total, size_t bytes, bool use_ctx) {
  return dev_alloc(c, list, total, bytes, use_ctx);
}
void ctx_free(mg_ctx* c, std::vector<Alloc>& list, size_t& total) { free_list(c, list, total); }

// ---------------------------------------------------------------- batched solves
// Many small problems in one launch (k_batch): every level of each hierarchy
// runs in the staged tail of the thread block that takes the problem, so a
// problem qualifies when the vectors of all its levels fit in shared memory
// at the V-cycle precision.
int batch_check(const mg_hier* h, int prec) {
  int rc = check_prec(h, prec);
  if (rc) return rc;
  const int method = method_of(h);
  if (method != M_CG && method != M_BICG)
    return fail(MG_ERR_INVALID, "batched solves run CG or BiCGStab (not GMRES or the plain multigrid iteration)");
  if (h->opts.inner_rtol > 0) return fail(MG_ERR_INVALID, "batched solves do not run defect correction");
  if (h->nlev > kTailMax) return fail(MG_ERR_INVALID, "hierarchy has more levels than the staged tail holds");
  for (const LevelMats& L : h->L)
    if (L.vanka) return fail(MG_ERR_INVALID, "batched solves smooth with Jacobi only (no Vanka levels)");
  const int pi = prec == MG_FP64 ? 0 : (prec == MG_MIXED_FP32 ? 1 : 2);
  if (tail_vec_bytes(h, pi, h->nlev - 1) > kTailSmemMax)
    return fail(MG_ERR_INVALID, "the V-cycle vectors of every level do not fit in shared memory");
  return MG_OK;
}

namespace {

// Device copy of the staged tail over every level of h for slot pi.
int batch_tail(mg_hier* h, int pi) {
  if (h->batch_tp[pi]) return MG_OK;
  const int top = h->nlev - 1;
  TailParams P;
  P.nt = top + 1;
  P.nu1 = h->opts.nu1;
  P.nu2 = h->opts.nu2;
  P.cinv = h->coarse_inv;
  P.cn = h->coarse_n;
  P.cluster = 0;
  mg_hier::TailImage ti;
  int rc = tail_image(h, pi, top, &ti);
  if (rc) return rc;
  P.image = ti.p;
  P.image_bytes = ti.image_bytes;
  P.smem = ti.smem;
  P.staged_mask = ti.staged_mask;
  void* d = dev_alloc(h->ctx, h->allocs, h->bytes, sizeof(TailParams), true);
  if (!d) return fail(MG_ERR_OOM, "alloc");
  CU(cudaMemcpy(d, &P, sizeof(TailParams), cudaMemcpyHostToDevice));
  // the batched kernel may run on a non-blocking stream, unordered with the
  // legacy stream of the copy: complete it first
  CU(cudaStreamSynchronize(cudaStreamLegacy));
  h->batch_tp[pi] = (const TailParams*)d;
  h->batch_smem[pi] = P.smem;
  return MG_OK;
}

constexpr size_t kBatchAlign = 256;
size_t balign(size_t b) { return (b + kBatchAlign - 1) & ~(kBatchAlign - 1); }

}  // namespace

void free_run(mg_ctx* c, BatchRun& run) {
  free_list(c, run.allocs, run.bytes);
  run.arena = nullptr;
  run.cap = 0;
  if (run.host) cudaFreeHost(run.host);
  run.host = nullptr;
  run.host_cap = 0;
  if (run.ev0) cudaEventDestroy(run.ev0);
  if (run.ev1) cudaEventDestroy(run.ev1);
  if (run.done) cudaEventDestroy(run.done);
  run.ev0 = run.ev1 = run.done = nullptr;
}

int batch_enqueue(mg_ctx* c, BatchRun& run, int count, mg_hier* const* hs, const double* const* b,
                  double* const* x, const double* rtol, const int* max_it, int prec, cudaStream_t s) {
  const int pi = prec == MG_FP64 ? 0 : (prec == MG_MIXED_FP32 ? 1 : 2);
  for (int k = 0; k < count; ++k) {
    mg_hier* h = hs[k];
    std::lock_guard<std::mutex> lk(h->solve_mu);   // the tail image map
    int rc = batch_tail(h, pi);
    if (rc) return rc;
  }
  // arena: work list, order, two counters, then the FP64 work vectors
  auto nvec = [&](const mg_hier* h) { return method_of(h) == M_CG ? 4 : 9; };
  const size_t items_b = balign((size_t)count * sizeof(BatchItem));
  const size_t order_b = balign((size_t)count * sizeof(int));
  size_t total = items_b + order_b + kBatchAlign;
  for (int k = 0; k < count; ++k) total += (size_t)nvec(hs[k]) * balign((size_t)hs[k]->n_dofs * 8);
  if (total > run.cap) {
    free_list(c, run.allocs, run.bytes);
    run.arena = nullptr;
    run.cap = 0;
    if (c->budget && c->used + total > c->budget)
      return fail(MG_ERR_ADMISSION, "batch work vectors exceed the HBM budget");
    run.arena = dev_alloc(c, run.allocs, run.bytes, total, true);
    if (!run.arena) return fail(MG_ERR_OOM, "batch arena");
    run.cap = total;
  }
  const size_t host_b = items_b + order_b;
  if (host_b > run.host_cap) {
    if (run.host) cudaFreeHost(run.host);
    run.host = nullptr;
    run.host_cap = 0;
    CU(cudaMallocHost(&run.host, host_b));
    run.host_cap = host_b;
  }
  if (!run.ev0) CU(cudaEventCreate(&run.ev0));
  if (!run.ev1) CU(cudaEventCreate(&run.ev1));
  if (!run.done) CU(cudaEventCreate(&run.done));
  unsigned char* dev = (unsigned char*)run.arena;
  BatchItem* d_items = (BatchItem*)dev;
  int* d_order = (int*)(dev + items_b);
  unsigned int* d_next = (unsigned int*)(dev + items_b + order_b);
  BatchItem* items = (BatchItem*)run.host;
  int* order = (int*)((unsigned char*)run.host + items_b);
  unsigned char* vp = dev + items_b + order_b + kBatchAlign;
  for (int k = 0; k < count; ++k) {
    const mg_hier* h = hs[k];
    const size_t vb = balign((size_t)h->n_dofs * 8);
    auto vec = [&]() {
      double* p = (double*)vp;
      vp += vb;
      return p;
    };
    BatchItem it;
    it.tail = h->batch_tp[pi];
    it.A = h->L.back().A64.v;
    it.Hc = h->Hc.t;
    it.fix = h->fixmask;
    it.b = b[k];
    it.x = x[k];
    it.xi = vec(); it.r = vec(); it.p = vec(); it.q = vec();
    if (method_of(h) == M_BICG) { it.rhat = vec(); it.v = vec(); it.s = vec(); it.ph = vec(); it.sh = vec(); }
    it.n_nodes = h->n_nodes;
    it.n = h->n_dofs;
    it.method = method_of(h) == M_CG ? 1 : 2;
    it.max_it = max_it[k];
    it.rtol = rtol[k];
    items[k] = it;
  }
  // work list: scalar problems first, then block problems (one launch each),
  // largest first within each so that the long solves start early
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int q) {
    if (hs[a]->nc != hs[q]->nc) return hs[a]->nc < hs[q]->nc;
    return hs[a]->n_dofs > hs[q]->n_dofs;
  });
  std::copy(idx.begin(), idx.end(), order);
  int n1 = 0;
  while (n1 < count && hs[idx[n1]]->nc == 1) ++n1;
  CU(cudaMemcpyAsync(d_items, items, (size_t)count * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_order, order, (size_t)count * sizeof(int), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(d_next, 0, 2 * sizeof(unsigned int), s));
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  CU(cudaEventRecord(run.ev0, s));
  run.launches = 0;
  for (int g = 0; g < 2; ++g) {
    const int lo = g == 0 ? 0 : n1, hi = g == 0 ? n1 : count;
    if (hi <= lo) continue;
    const int nc = g == 0 ? 1 : 3;
    uint32_t smem = 0;
    for (int k = lo; k < hi; ++k) smem = std::max(smem, hs[idx[k]]->batch_smem[pi]);
    const int per_sm = batch_blocks_per_sm(nc, pi, smem);
    const int grid = std::min(hi - lo, sms * per_sm);
    launch_batch(d_items, d_order + lo, hi - lo, d_next + g, nc, pi, smem, grid, s);
    ++run.launches;
  }
  CU(cudaGetLastError());
  CU(cudaEventRecord(run.ev1, s));
  CU(cudaMemcpyAsync(items, d_items, (size_t)count * sizeof(BatchItem), cudaMemcpyDeviceToHost, s));
  CU(cudaEventRecord(run.done, s));      // results readable once it completed
  run.count = count;
  run.prec = prec;
  for (int k = 0; k < count; ++k) hs[k]->launch_count++;
  return MG_OK;
}

int batch_collect(BatchRun& run, mg_stats* stats) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, run.ev0, run.ev1);
  const BatchItem* items = (const BatchItem*)run.host;
  int first_bad = MG_OK;
  for (int k = 0; k < run.count; ++k) {
    const BatchItem& it = items[k];
    int st;
    if (it.status == -7) st = MG_ERR_INVALID;   // the kernel refused the item (inconsistent sizes)
    else if (it.status == -6) st = MG_ERR_NAN;
    else if (it.status == -5) st = MG_ERR_BREAKDOWN;
    else if (it.status == 0 && it.rel_res <= it.rtol) st = MG_OK;
    else st = MG_ERR_NOT_CONVERGED;
    if (st != MG_OK && first_bad == MG_OK) first_bad = st;
    if (stats) {
      mg_stats& o = stats[k];
      o = mg_stats{};
      o.status = st;
      o.iters = it.iters;
      o.vcycles = it.iters * (it.method == 2 ? 2 : 1);
      o.precision = run.prec;
      o.rel_res = it.rel_res;
      o.solve_ms = ms;
      o.launches = run.launches;
    }
  }
  return first_bad;
}

int solve_batch(mg_ctx* c, int count, mg_hier* const* hs, const double* const* b, double* const* x, double rtol,
                int max_it, int prec, mg_stats* stats) {
  if (!c || count < 0 || (count > 0 && (!hs || !b || !x)) || !(rtol > 0) || max_it < 1)
    return fail(MG_ERR_INVALID, "bad argument");
  if (count == 0) return MG_OK;
  for (int k = 0; k < count; ++k) {
    mg_hier* h = hs[k];
    if (!h || h->ctx != c || !b[k] || !x[k]) return fail(MG_ERR_INVALID, "bad problem " + std::to_string(k));
    int rc = batch_check(h, prec);
    if (rc) return rc;
  }
  CU(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(c->batch_mu);
  std::vector<double> rt(count, rtol);
  std::vector<int> mi(count, max_it);
  int rc = batch_enqueue(c, c->batch, count, hs, b, x, rt.data(), mi.data(), prec, c->stream);
  if (rc) return rc;
  CU(cudaEventSynchronize(c->batch.done));
  return batch_collect(c->batch, stats);
}


// ---------------------------------------------------------------- re-assembly
int update_hierarchy(mg_hier* h, HostHierarchy& H) {
  const int nc = h->nc, nb = nc * nc;
  if ((int)H.levels.size() != h->nlev) return fail(MG_ERR_INVALID, "re-assembly changed the number of levels");
  int rc;
  for (int l = 0; l < h->nlev; ++l) {
    HostLevel& lv = H.levels[l];
    LevelMats& B = h->L[l];
    const bool pat6 = velocity_pressure_pattern(lv.A);
    if (lv.topo.n_nodes != B.n || lv.vanka != B.vanka || (pat6 ? 6 : nb) != h->level_block_values[l])
      return fail(MG_ERR_INVALID, "re-assembly changed a level");
    B.omega = lv.omega;
    if (B.A64.slots && (rc = refill_sell<double>(lv.A, B.A64, pat6))) return rc;
    if (B.A32.slots && (rc = refill_sell<float>(lv.A, B.A32, pat6))) return rc;
    if (B.A16.slots && (rc = refill_sell<__nv_bfloat16>(lv.A, B.A16, pat6))) return rc;
    if (B.S64) CU(cudaMemcpy(B.S64, lv.Sinv.data(), B.n * nb * 8, cudaMemcpyHostToDevice));
    if (B.S32) {
      std::vector<float> s32(lv.Sinv.begin(), lv.Sinv.end());
      CU(cudaMemcpy(B.S32, s32.data(), B.n * nb * 4, cudaMemcpyHostToDevice));
    }
    if (B.vanka) {
      if (B.V64.slots && (rc = refill_sell<double>(lv.Sv, B.V64))) return rc;
      if (B.V32.slots && (rc = refill_sell<float>(lv.Sv, B.V32))) return rc;
    }
  }
  if ((int64_t)H.coarse_inv.size() != h->coarse_n * h->coarse_n)
    return fail(MG_ERR_INVALID, "re-assembly changed the coarse level");
  CU(cudaMemcpy(h->coarse_inv, H.coarse_inv.data(), H.coarse_inv.size() * 8, cudaMemcpyHostToDevice));
  if ((rc = refill_sell<double>(H.load, h->F))) return rc;
  if ((H.lift.nnzb() > 0) != (h->Lift.slots > 0)) return fail(MG_ERR_INVALID, "re-assembly changed the lifting");
  if (h->Lift.slots && (rc = refill_sell<double>(H.lift, h->Lift))) return rc;
  // the copies ran on the legacy stream: complete them before any stream reads
  CU(cudaStreamSynchronize(cudaStreamLegacy));
  // the small-level images hold copies of the level matrices and damping:
  // rebuild them for the current tail configuration
  for (int pi = 0; pi < 3; ++pi)
    if (h->batch_tp[pi]) {
      free_one(h->ctx, h->allocs, h->bytes, h->batch_tp[pi]);
      h->batch_tp[pi] = nullptr;
      h->batch_smem[pi] = 0;
    }
  for (auto& kv : h->tail_img) free_one(h->ctx, h->allocs, h->bytes, kv.second.p);
  h->tail_img.clear();
  const int top = h->tail_top, cl = h->tail_cluster;
  for (int pi = 0; pi < 3 && top > 0 && cl <= 0; ++pi) {
    if (!has_slot(h, pi)) continue;
    mg_hier::TailImage ti;
    rc = cl < 0 ? tail_image_dsm(h, pi, top, -cl, &ti) : tail_image(h, pi, top, &ti);
    if (rc) return rc;
  }
  // every workspace: the levels' damping in its tail parameters, the new
  // images, and no cached graph (kernel arguments carry the damping)
  auto refresh = [&](Workspace* w) {
    for (TailParams* P : {&w->tail64, &w->tail32, &w->tail16})
      for (int l = 0; l < h->nlev && l < kTailMax; ++l) P->lv[l].omega = h->L[l].omega;
    apply_tail(h, w);
  };
  if (h->ws0) refresh(h->ws0);
  std::lock_guard<std::mutex> lk(h->pool_mu);
  for (Workspace* w : h->all_ws) refresh(w);
  return MG_OK;
}

}  // namespace mgi
