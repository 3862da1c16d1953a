// Device view of the driven-cavity Navier-Stokes operators (ns_kernels.cu) and the
// launchers of its kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mgi {

// 1D operators along one axis of the velocity mesh (n nodes), 3 entries per
// node for the offsets -1, 0, +1 (zero where the neighbour cell is missing):
//   M[3i + a]  = (phi_{i+a-1}, phi_i)        consistent mass
//   K[3i + a]  = (phi_{i+a-1}', phi_i')      stiffness
//   G[3i + a]  = (phi_{i+a-1}, phi_i')       convection (rows of C_d along d)
//   GT[3i + a] = G[3(i+a-1) + 2 - a]         transposed (the divergence)
//   m1[i]      = sum_a M[3i + a]             lumped mass
//   Kn[3i + a] = -nu K[3i + a]               (the viscous factor of Step 1)
//   im1[i]     = 1 / m1[i]
struct NsAxis {
  const double* M = nullptr;
  const double* K = nullptr;
  const double* G = nullptr;
  const double* GT = nullptr;
  const double* m1 = nullptr;
  const double* Kn = nullptr;
  const double* im1 = nullptr;
};

struct NsView {
  NsAxis ax[3];
  int nv[3] = {0, 0, 0};      // velocity nodes per axis (2 np - 1)
  int np[3] = {0, 0, 0};      // pressure nodes per axis
  double nu = 1e-3, dt = 1e-4, lid = 1.0;
};

// pt = P (p + q) (velocity nodes)
void ns_interp(const NsView& V, const double* p, const double* q, double* pt, cudaStream_t s);
// Step 1: un from u (both node-major n_v x 3) and pt
void ns_momentum(const NsView& V, const double* u, const double* pt, double* un, cudaStream_t s);
// dv = ((div u, phi_i))_i (velocity nodes)
void ns_div(const NsView& V, const double* u, double* dv, cudaStream_t s);
// d = P^T dv, b = -d / dt
void ns_restrict(const NsView& V, const double* dv, double* d, double* b, cudaStream_t s);
// q <- q - (sum_j m_j q_j) / total (mean zero with the lumped masses m)
void ns_meanfree(int64_t np, const double* m, double total, double* q, cudaStream_t s);
// Step 3: p <- p + q - nu d / m^p
void ns_pupdate(int64_t np, double nu, const double* q, const double* d, const double* mp_inv, double* p,
                cudaStream_t s);

}  // namespace mgi
