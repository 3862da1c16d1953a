// Explicit Navier-Stokes pressure correction on the driven cavity (Sec. 5.3):
// host setup (meshes, per-axis 1D operators, the pressure hierarchy) and the
// time-step driver; the kernels are in ns_kernels.cu.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device.h"
#include "ns.h"

using namespace mgi;

#define CU(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct mg_ns {
  mg_ctx* ctx = nullptr;
  mg_hier* hp = nullptr;                 // pressure hierarchy (graded, pure Neumann)
  mg_ns_params par{};
  std::vector<Alloc> allocs;
  size_t bytes = 0;
  NsView V;
  double *u = nullptr, *un = nullptr, *pt = nullptr, *dv = nullptr;   // velocity mesh
  double *p = nullptr, *q = nullptr, *d = nullptr, *b = nullptr, *mp = nullptr, *mp_inv = nullptr;   // pressure mesh
  double mp_total = 0.0;                 // sum of the lumped pressure masses (the volume)
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

// Node coordinates of the pressure mesh along an axis with n cells on
// [0, len]: cosine-graded (Sec. 5.3) or equidistant.
std::vector<double> pressure_axis(int n, double len, bool graded) {
  std::vector<double> x(n + 1);
  const double pi = std::acos(-1.0);
  for (int i = 0; i <= n; ++i)
    x[i] = graded ? 0.5 * len * (1.0 - std::cos(i * pi / n)) : len * (double)i / n;
  x[0] = 0.0;
  x[n] = len;
  return x;
}

// Equidistant refinement: every cell halved.
std::vector<double> refine(const std::vector<double>& a) {
  std::vector<double> r(2 * a.size() - 1);
  for (size_t i = 0; i < a.size(); ++i) r[2 * i] = a[i];
  for (size_t i = 0; i + 1 < a.size(); ++i) r[2 * i + 1] = 0.5 * (a[i] + a[i + 1]);
  return r;
}

// The 1D Q1 operators of an axis (layout in ns.h): exact integrals of
// products of hat functions over the cells left (h_l) and right (h_r) of a
// node: (phi_{i-1}, phi_i) = h_l / 6, (phi_i, phi_i) = (h_l + h_r) / 3,
// stiffness 1/h per cell, and int phi_j phi_i' = +1/2 over the left cell
// (phi_i rises) and -1/2 over the right one, for j either node of the cell.
struct Axis1D {
  std::vector<double> M, K, G, GT, m1;
};
Axis1D axis_ops(const std::vector<double>& x) {
  const int n = (int)x.size();
  Axis1D A;
  A.M.assign(3 * n, 0.0);
  A.K.assign(3 * n, 0.0);
  A.G.assign(3 * n, 0.0);
  A.GT.assign(3 * n, 0.0);
  A.m1.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double hl = i > 0 ? x[i] - x[i - 1] : 0.0, hr = i + 1 < n ? x[i + 1] - x[i] : 0.0;
    A.M[3 * i] = hl / 6.0;
    A.M[3 * i + 1] = (hl + hr) / 3.0;
    A.M[3 * i + 2] = hr / 6.0;
    A.K[3 * i] = hl > 0 ? -1.0 / hl : 0.0;
    A.K[3 * i + 1] = (hl > 0 ? 1.0 / hl : 0.0) + (hr > 0 ? 1.0 / hr : 0.0);
    A.K[3 * i + 2] = hr > 0 ? -1.0 / hr : 0.0;
    A.G[3 * i] = hl > 0 ? 0.5 : 0.0;
    A.G[3 * i + 1] = (hl > 0 ? 0.5 : 0.0) - (hr > 0 ? 0.5 : 0.0);
    A.G[3 * i + 2] = hr > 0 ? -0.5 : 0.0;
    A.m1[i] = 0.5 * (hl + hr);
  }
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      const int j = i + a - 1;
      A.GT[3 * i + a] = (j >= 0 && j < n) ? A.G[3 * j + 2 - a] : 0.0;
    }
  return A;
}

int largest_level(int nx, int ny, int nz) {
  int L = 0;
  while (nx % (2 << L) == 0 && ny % (2 << L) == 0 && nz % (2 << L) == 0) ++L;
  return L;
}

double* dvec(mg_ns* ns, int64_t n) {
  return (double*)ctx_alloc(ns->ctx, ns->allocs, ns->bytes, (size_t)std::max<int64_t>(n, 1) * 8, true);
}

void ns_release(mg_ns* ns) {
  if (!ns) return;
  if (ns->hp) mg_free(ns->hp);
  ns->hp = nullptr;
  ctx_free(ns->ctx, ns->allocs, ns->bytes);
  for (auto& e : ns->ev)
    if (e) cudaEventDestroy(e);
  delete ns;
}

}  // namespace

extern "C" {

void mg_ns_default_params(mg_ns_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = 32;
  p->ny = 32;
  p->nz = 64;
  p->graded = 1;
  p->re = 1000.0;
  p->dt = 1e-4;
  p->lid = 1.0;
  p->prec = MG_MIXED_FP32;
  p->krylov = MG_GMRES;
  p->rtol = 1e-8;
  p->max_it = 200;
  p->nu = 4;
  p->smoother = MG_SMOOTHER_JACOBI;
}

int mg_ns_setup(mg_ctx* ctx, const mg_ns_params* par, mg_ns** out) {
  if (!ctx || !par || !out) return fail(MG_ERR_INVALID, "NULL argument");
  const mg_ns_params& P = *par;
  if (P.nx < 2 || P.ny < 2 || P.nz < 2 || P.nx > 4096 || P.ny > 4096 || P.nz > 4096)
    return fail(MG_ERR_INVALID, "nx, ny, nz must be in [2, 4096]");
  if (!(P.re > 0) || !(P.dt > 0) || !std::isfinite(P.lid) || !(P.rtol > 0) || P.max_it < 1 || P.nu < 1 || P.nu > 16)
    return fail(MG_ERR_INVALID, "need re > 0, dt > 0, a finite lid speed, rtol > 0, max_it >= 1, nu in [1, 16]");
  if (P.smoother != MG_SMOOTHER_JACOBI && P.smoother != MG_SMOOTHER_VANKA)
    return fail(MG_ERR_INVALID, "unknown smoother");
  if (P.prec != MG_FP64 && P.prec != MG_MIXED_FP32 && P.prec != MG_MIXED_BF16)
    return fail(MG_ERR_INVALID, "unknown precision");
  if (P.krylov != MG_KRYLOV_AUTO && P.krylov != MG_CG && P.krylov != MG_BICGSTAB && P.krylov != MG_GMRES)
    return fail(MG_ERR_INVALID, "the pressure solve runs CG, BiCGStab or GMRES");
  CU(cudaSetDevice(ctx->device));
  mg_ns* ns = new mg_ns();
  ns->ctx = ctx;
  ns->par = P;
  const int nc[3] = {P.nx, P.ny, P.nz};
  const double len[3] = {1.0, 1.0, 2.0};
  std::vector<double> ax[3], vx[3];
  for (int d = 0; d < 3; ++d) {
    ax[d] = pressure_axis(nc[d], len[d], P.graded != 0);
    vx[d] = refine(ax[d]);
  }
  // pressure hierarchy: the uniform leaf set of the largest level L that
  // divides every cell count, on the macro grid (n >> L), graded by ax
  const int L = largest_level(P.nx, P.ny, P.nz);
  const int64_t ncell = (int64_t)P.nx * P.ny * P.nz;
  std::vector<int32_t> lev(ncell, L), anc(ncell * 3);
  for (int64_t c = 0; c < ncell; ++c) {
    anc[3 * c] = (int32_t)(c % P.nx);
    anc[3 * c + 1] = (int32_t)((c / P.nx) % P.ny);
    anc[3 * c + 2] = (int32_t)(c / ((int64_t)P.nx * P.ny));
  }
  mg_mesh m{};
  m.dim = 3;
  for (int d = 0; d < 3; ++d) {
    m.origin[d] = 0.0;
    m.extent[d] = len[d];
    m.macro[d] = nc[d] >> L;
    m.axis[d] = ax[d].data();
  }
  m.n_leaves = ncell;
  m.leaf_level = lev.data();
  m.leaf_anchor = anc.data();
  mg_problem pr{};
  pr.kind = MG_POISSON;
  pr.eps = 1.0;
  pr.mu = 1.0;
  pr.lambda = 1.0;
  pr.supg_delta0 = 0.5;
  pr.dt = INFINITY;
  // no Dirichlet face: the pure Neumann problem (its coarse solve applies the
  // pseudo-inverse; the increment is shifted to mean zero after each solve)
  mg_opts o;
  mg_default_opts(&o);
  o.krylov = P.krylov;
  o.nu1 = o.nu2 = P.nu;
  o.smoother = P.smoother;
  o.store_bf16 = P.prec == MG_MIXED_BF16 ? 1 : 0;
  int rc = mg_setup(ctx, &m, &pr, &o, &ns->hp);
  if (rc != MG_OK) {
    ns_release(ns);
    return rc;
  }
  // velocity operators: per-axis 1D coefficients
  NsView& V = ns->V;
  V.nu = 1.0 / P.re;
  for (int d = 0; d < 3; ++d) {
    const Axis1D A = axis_ops(vx[d]);
    const int64_t n = (int64_t)vx[d].size();
    double* buf = dvec(ns, 17 * n);
    if (!buf) { ns_release(ns); return fail(MG_ERR_OOM, "alloc"); }
    std::vector<double> h(17 * n);
    std::copy(A.M.begin(), A.M.end(), h.begin());
    std::copy(A.K.begin(), A.K.end(), h.begin() + 3 * n);
    std::copy(A.G.begin(), A.G.end(), h.begin() + 6 * n);
    std::copy(A.GT.begin(), A.GT.end(), h.begin() + 9 * n);
    std::copy(A.m1.begin(), A.m1.end(), h.begin() + 12 * n);
    for (int64_t e = 0; e < 3 * n; ++e) h[13 * n + e] = -V.nu * A.K[e];
    for (int64_t i = 0; i < n; ++i) h[16 * n + i] = 1.0 / A.m1[i];
    if (cudaMemcpy(buf, h.data(), 17 * n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      ns_release(ns);
      return fail(MG_ERR_CUDA, "upload");
    }
    V.ax[d].M = buf;
    V.ax[d].K = buf + 3 * n;
    V.ax[d].G = buf + 6 * n;
    V.ax[d].GT = buf + 9 * n;
    V.ax[d].m1 = buf + 12 * n;
    V.ax[d].Kn = buf + 13 * n;
    V.ax[d].im1 = buf + 16 * n;
    V.nv[d] = (int)n;
    V.np[d] = nc[d] + 1;
  }
  V.dt = P.dt;
  V.lid = P.lid;
  const int64_t nv = (int64_t)V.nv[0] * V.nv[1] * V.nv[2], np = (int64_t)V.np[0] * V.np[1] * V.np[2];
  ns->u = dvec(ns, 3 * nv);
  ns->un = dvec(ns, 3 * nv);
  ns->pt = dvec(ns, nv);
  ns->dv = dvec(ns, nv);
  ns->p = dvec(ns, np);
  ns->q = dvec(ns, np);
  ns->d = dvec(ns, np);
  ns->b = dvec(ns, np);
  ns->mp_inv = dvec(ns, np);
  ns->mp = dvec(ns, np);
  if (!ns->u || !ns->un || !ns->pt || !ns->dv || !ns->p || !ns->q || !ns->d || !ns->b || !ns->mp_inv || !ns->mp) {
    ns_release(ns);
    return fail(MG_ERR_OOM, "alloc");
  }
  {
    Axis1D Ap[3] = {axis_ops(ax[0]), axis_ops(ax[1]), axis_ops(ax[2])};
    std::vector<double> mi(np), mm(np);
    for (int64_t t = 0; t < np; ++t) {
      const int64_t i = t % V.np[0], j = (t / V.np[0]) % V.np[1], k = t / ((int64_t)V.np[0] * V.np[1]);
      mm[t] = Ap[0].m1[i] * Ap[1].m1[j] * Ap[2].m1[k];
      mi[t] = 1.0 / mm[t];
      ns->mp_total += mm[t];
    }
    if (cudaMemcpy(ns->mp_inv, mi.data(), np * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ns->mp, mm.data(), np * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      ns_release(ns);
      return fail(MG_ERR_CUDA, "upload");
    }
  }
  cudaStream_t s = ctx->stream;
  bool ok = cudaMemsetAsync(ns->u, 0, 3 * nv * 8, s) == cudaSuccess && cudaMemsetAsync(ns->un, 0, 3 * nv * 8, s) == cudaSuccess &&
            cudaMemsetAsync(ns->p, 0, np * 8, s) == cudaSuccess && cudaMemsetAsync(ns->q, 0, np * 8, s) == cudaSuccess;
  for (auto& e : ns->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  // the uploads ran on the legacy stream: complete them before the solver's stream uses them
  ok = ok && cudaStreamSynchronize(cudaStreamLegacy) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    ns_release(ns);
    return fail(MG_ERR_CUDA, "initialisation");
  }
  *out = ns;
  return MG_OK;
}

int mg_ns_sizes(const mg_ns* ns, int n_vel[3], int n_pres[3]) {
  if (!ns) return fail(MG_ERR_INVALID, "NULL argument");
  for (int d = 0; d < 3; ++d) {
    if (n_vel) n_vel[d] = ns->V.nv[d];
    if (n_pres) n_pres[d] = ns->V.np[d];
  }
  return MG_OK;
}

mg_hier* mg_ns_pressure_hierarchy(mg_ns* ns) { return ns ? ns->hp : nullptr; }

int mg_ns_state(mg_ns* ns, double* u, double* p, double* q, int dir) {
  if (!ns || (dir != 0 && dir != 1)) return fail(MG_ERR_INVALID, "bad argument");
  CU(cudaSetDevice(ns->ctx->device));
  const NsView& V = ns->V;
  const int64_t nv = (int64_t)V.nv[0] * V.nv[1] * V.nv[2], np = (int64_t)V.np[0] * V.np[1] * V.np[2];
  cudaStream_t s = ns->ctx->stream;
  auto cp = [&](double* ext, double* mine, int64_t n) -> cudaError_t {
    if (!ext) return cudaSuccess;
    return dir == 0 ? cudaMemcpyAsync(mine, ext, n * 8, cudaMemcpyDeviceToDevice, s)
                    : cudaMemcpyAsync(ext, mine, n * 8, cudaMemcpyDeviceToDevice, s);
  };
  CU(cp(u, ns->u, 3 * nv));
  CU(cp(p, ns->p, np));
  CU(cp(q, ns->q, np));
  CU(cudaStreamSynchronize(s));
  return MG_OK;
}

int mg_ns_steps(mg_ns* ns, int n_steps, mg_ns_stats* stats) {
  if (!ns || n_steps < 0) return fail(MG_ERR_INVALID, "bad argument");
  CU(cudaSetDevice(ns->ctx->device));
  mg_ns_stats st{};
  const auto t0 = std::chrono::steady_clock::now();
  mg_hier* h = ns->hp;
  const NsView& V = ns->V;
  const int64_t np = (int64_t)V.np[0] * V.np[1] * V.np[2];
  cudaStream_t s = ns->ctx->stream;
  int status = MG_OK;
  {
    std::lock_guard<std::mutex> lk(h->solve_mu);
    Workspace& w = *h->ws0;
    for (int k = 0; k < n_steps; ++k) {
      CU(cudaEventRecord(ns->ev[0], s));
      ns_interp(V, ns->p, ns->q, ns->pt, s);                 // P (p^{m-1} + q^{m-1})
      ns_momentum(V, ns->u, ns->pt, ns->un, s);              // Step 1
      std::swap(ns->u, ns->un);
      CU(cudaEventRecord(ns->ev[1], s));
      ns_div(V, ns->u, ns->dv, s);                           // Step 2: d = P^T (div u^m, phi)
      ns_restrict(V, ns->dv, ns->d, ns->b, s);
      CU(cudaEventRecord(ns->ev[2], s));
      mg_stats ss{};
      int rc = solve_start(h, w, ns->b, false, ns->q, false, ns->q, false, ns->par.rtol, ns->par.max_it,
                           ns->par.prec, s);
      while (rc == MG_OK || rc == MG_PENDING) {
        CU(cudaEventSynchronize(w.ev1));
        rc = solve_check(h, w, s, &ss);
        if (rc != MG_PENDING) break;
      }
      ns_meanfree(np, ns->mp, ns->mp_total, ns->q, s);      // the increment of mean zero
      CU(cudaEventRecord(ns->ev[3], s));
      ns_pupdate(np, V.nu, ns->q, ns->d, ns->mp_inv, ns->p, s);   // Step 3
      CU(cudaEventRecord(ns->ev[4], s));
      CU(cudaEventSynchronize(ns->ev[4]));
      CU(cudaGetLastError());
      float t01 = 0.f, t12 = 0.f, t23 = 0.f, t34 = 0.f;
      cudaEventElapsedTime(&t01, ns->ev[0], ns->ev[1]);
      cudaEventElapsedTime(&t12, ns->ev[1], ns->ev[2]);
      cudaEventElapsedTime(&t23, ns->ev[2], ns->ev[3]);
      cudaEventElapsedTime(&t34, ns->ev[3], ns->ev[4]);
      st.ms_momentum += t01;
      st.ms_pres_rhs += t12;
      st.ms_pres_solve += t23;
      st.ms_pres_up += t34;
      st.steps += 1;
      st.iters += ss.iters;
      st.iters_max = std::max(st.iters_max, ss.iters);
      st.rel_res_max = std::max(st.rel_res_max, ss.rel_res);
      h->launch_count += 6;
      if (rc != MG_OK) {
        status = rc;
        break;
      }
    }
  }
  st.status = status;
  st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return status;
}

int mg_ns_free(mg_ns* ns) {
  if (!ns) return MG_ERR_INVALID;
  cudaSetDevice(ns->ctx->device);
  cudaStreamSynchronize(ns->ctx->stream);
  ns_release(ns);
  return MG_OK;
}

}  // extern "C"
