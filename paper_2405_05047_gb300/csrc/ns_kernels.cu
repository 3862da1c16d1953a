// Kernels of the explicit Navier-Stokes pressure correction (Sec. 5.3,
// Algorithm "The fully discrete solution procedure for the Navier-Stokes
// equations") on the tensor-product meshes of the driven cavity (host side: ns.cpp).
//
// Velocity: Q1 on Omega_{h/2}, pressure: Q1 on Omega_h (its equidistant
// refinement is Omega_{h/2}).  On a tensor grid every velocity operator is a
// Kronecker product of tridiagonal 1D operators along x, y, z:
//   consistent mass  M1[i][a] = (phi_{i+a}, phi_i)          a = -1, 0, 1
//   stiffness        K1[i][a] = (phi_{i+a}', phi_i')
//   convection       G1[i][a] = (phi_{i+a}, phi_i')          (C_d = G1 along d, M1 across)
//   transposed       GT1[i][a] = G1[i+a][-a]                  (the divergence)
//   lumped mass      m1[i] = sum_a M1[i][a]
// so K = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1, C_x = G1 x M1 x M1 (and
// so on), and the lumped 3D mass is m1 x m1 x m1.  The kernels apply them as
// 27-point stencils with the per-axis coefficients (nothing is stored per
// node but the vectors).  The interpolation P from the pressure grid (node J
// -> velocity node 2J, midpoints get 1/2 of each neighbour per axis) and its
// transpose are tensor products too.  Arithmetic in FP64 throughout.
#include <cuda_runtime.h>

#include "kernels.h"
#include "ns.h"

namespace mgi {

namespace {

constexpr int kNsBlock = 256;

__device__ __forceinline__ void node_of(int64_t t, const int* n, int& i, int& j, int& k) {
  i = (int)(t % n[0]);
  const int64_t r = t / n[0];
  j = (int)(r % n[1]);
  k = (int)(r / n[1]);
}

// pt = P (p + q) at every velocity node
__global__ void __launch_bounds__(kNsBlock) k_ns_interp(NsView V, const double* __restrict__ p,
                                                        const double* __restrict__ q, double* __restrict__ pt) {
  const int64_t nv = (int64_t)V.nv[0] * V.nv[1] * V.nv[2];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    int I[3];
    node_of(t, V.nv, I[0], I[1], I[2]);
    int lo[3], hi[3];
    double wl[3], wh[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = I[d] >> 1;
      const bool odd = I[d] & 1;
      hi[d] = odd ? lo[d] + 1 : lo[d];
      wl[d] = odd ? 0.5 : 1.0;
      wh[d] = odd ? 0.5 : 0.0;
    }
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int jx = (c & 1) ? hi[0] : lo[0], jy = (c & 2) ? hi[1] : lo[1], jz = (c & 4) ? hi[2] : lo[2];
      const double w = ((c & 1) ? wh[0] : wl[0]) * ((c & 2) ? wh[1] : wl[1]) * ((c & 4) ? wh[2] : wl[2]);
      if (w == 0.0) continue;
      const int64_t J = jx + (int64_t)V.np[0] * (jy + (int64_t)V.np[1] * jz);
      acc = fma(w, p[J] + q[J], acc);
    }
    pt[t] = acc;
  }
}

// Step 1: un = u + dt / m_i (-nu K u + N(u) + C P (p + q)) at interior nodes,
// the Dirichlet data on the boundary (lid: (0, lid, 0) on x = 1).
//   N(u)_{i,c} = sum_b sum_j C_b[i, j] u_{j,b} u_{j,c}  (Eqs. "tp", "multC")
__global__ void __launch_bounds__(kNsBlock) k_ns_momentum(NsView V, const double* __restrict__ u,
                                                          const double* __restrict__ pt, double* __restrict__ un) {
  const int64_t nv = (int64_t)V.nv[0] * V.nv[1] * V.nv[2];
  const int64_t sy = V.nv[0], sz = (int64_t)V.nv[0] * V.nv[1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(t, V.nv, i, j, k);
    if (i == 0 || j == 0 || k == 0 || i == V.nv[0] - 1 || j == V.nv[1] - 1 || k == V.nv[2] - 1) {
      un[3 * t] = 0.0;
      un[3 * t + 1] = i == V.nv[0] - 1 ? V.lid : 0.0;
      un[3 * t + 2] = 0.0;
      continue;
    }
    // per-axis factors; -nu folded into the stiffness ones
    double Mx[3], Kx[3], Gx[3], My[3], Ky[3], Gy[3], Mz[3], Kz[3], Gz[3];
    for (int a = 0; a < 3; ++a) {
      Mx[a] = V.ax[0].M[3 * i + a]; Kx[a] = -V.nu * V.ax[0].K[3 * i + a]; Gx[a] = V.ax[0].G[3 * i + a];
      My[a] = V.ax[1].M[3 * j + a]; Ky[a] = -V.nu * V.ax[1].K[3 * j + a]; Gy[a] = V.ax[1].G[3 * j + a];
      Mz[a] = V.ax[2].M[3 * k + a]; Kz[a] = -V.nu * V.ax[2].K[3 * k + a]; Gz[a] = V.ax[2].G[3 * k + a];
    }
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      for (int b = 0; b < 3; ++b) {
        const double myz = My[b] * Mz[c], kyz = fma(Ky[b], Mz[c], My[b] * Kz[c]);
        const double gyz = Gy[b] * Mz[c], mygz = My[b] * Gz[c];
        const int64_t row = t + (b - 1) * sy + (c - 1) * sz;
        for (int a = 0; a < 3; ++a) {
          const int64_t s = row + (a - 1);
          const double ux = u[3 * s], uy = u[3 * s + 1], uz = u[3 * s + 2], ps = pt[s];
          const double cx = Gx[a] * myz, cy = Mx[a] * gyz, cz = Mx[a] * mygz;
          // w = sum_b C_b u_b - nu K(a, b, c): acc_c += w u_c + C_c ps
          const double w = fma(cx, ux, fma(cy, uy, fma(cz, uz, fma(Kx[a], myz, Mx[a] * kyz))));
          acc0 = fma(w, ux, fma(cx, ps, acc0));
          acc1 = fma(w, uy, fma(cy, ps, acc1));
          acc2 = fma(w, uz, fma(cz, ps, acc2));
        }
      }
    }
    const double s = V.dt / (V.ax[0].m1[i] * V.ax[1].m1[j] * V.ax[2].m1[k]);
    un[3 * t] = fma(s, acc0, u[3 * t]);
    un[3 * t + 1] = fma(s, acc1, u[3 * t + 1]);
    un[3 * t + 2] = fma(s, acc2, u[3 * t + 2]);
  }
}

// dv_i = sum_j sum_c C_c[j, i] u_{j,c} = ((div u, phi_i))_i at every velocity node
__global__ void __launch_bounds__(kNsBlock) k_ns_div(NsView V, const double* __restrict__ u, double* __restrict__ dv) {
  const int64_t nv = (int64_t)V.nv[0] * V.nv[1] * V.nv[2];
  const int64_t sy = V.nv[0], sz = (int64_t)V.nv[0] * V.nv[1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(t, V.nv, i, j, k);
    double acc = 0.0;
    for (int c = 0; c < 3; ++c) {
      const int kk = k + c - 1;
      if (kk < 0 || kk >= V.nv[2]) continue;
      const double mz = V.ax[2].M[3 * k + c], gz = V.ax[2].GT[3 * k + c];
      for (int b = 0; b < 3; ++b) {
        const int jj = j + b - 1;
        if (jj < 0 || jj >= V.nv[1]) continue;
        const double my = V.ax[1].M[3 * j + b], gy = V.ax[1].GT[3 * j + b];
        const double myz = my * mz, gyz = gy * mz, mygz = my * gz;
        for (int a = 0; a < 3; ++a) {
          const int ii = i + a - 1;
          if (ii < 0 || ii >= V.nv[0]) continue;
          const double mx = V.ax[0].M[3 * i + a], gx = V.ax[0].GT[3 * i + a];
          const int64_t s = t + (a - 1) + (b - 1) * sy + (c - 1) * sz;
          acc = fma(gx * myz, u[3 * s], acc);
          acc = fma(mx * gyz, u[3 * s + 1], acc);
          acc = fma(mx * mygz, u[3 * s + 2], acc);
        }
      }
    }
    dv[t] = acc;
  }
}

// d = P^T dv at every pressure node; the pressure-increment right-hand side
// b = -d / dt
__global__ void __launch_bounds__(kNsBlock) k_ns_restrict(NsView V, const double* __restrict__ dv,
                                                          double* __restrict__ d, double* __restrict__ b) {
  const int64_t np = (int64_t)V.np[0] * V.np[1] * V.np[2];
  const int64_t sy = V.nv[0], sz = (int64_t)V.nv[0] * V.nv[1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np; t += (int64_t)gridDim.x * blockDim.x) {
    int J[3];
    node_of(t, V.np, J[0], J[1], J[2]);
    const int64_t centre = 2 * J[0] + 2 * J[1] * sy + 2 * J[2] * sz;
    double acc = 0.0;
    for (int c = -1; c <= 1; ++c) {
      const int kk = 2 * J[2] + c;
      if (kk < 0 || kk >= V.nv[2]) continue;
      const double wz = c == 0 ? 1.0 : 0.5;
      for (int bb = -1; bb <= 1; ++bb) {
        const int jj = 2 * J[1] + bb;
        if (jj < 0 || jj >= V.nv[1]) continue;
        const double wyz = (bb == 0 ? 1.0 : 0.5) * wz;
        for (int a = -1; a <= 1; ++a) {
          const int ii = 2 * J[0] + a;
          if (ii < 0 || ii >= V.nv[0]) continue;
          acc = fma((a == 0 ? 1.0 : 0.5) * wyz, dv[centre + a + bb * sy + c * sz], acc);
        }
      }
    }
    d[t] = acc;
    b[t] = -acc / V.dt;
  }
}

// q <- q - (sum_j m_j q_j) / total: the mean-zero increment (one block; the
// sum in a fixed order: per-thread partial sums, then the block's)
__global__ void __launch_bounds__(1024) k_ns_meanfree(int64_t np, const double* __restrict__ m, double total,
                                                      double* __restrict__ q) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) acc = fma(m[t], q[t], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  const double shift = s / total;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) q[t] -= shift;
}

// Step 3: p <- p + q - nu d / m^p
__global__ void __launch_bounds__(kNsBlock) k_ns_pupdate(int64_t np, double nu, const double* __restrict__ q,
                                                         const double* __restrict__ d,
                                                         const double* __restrict__ mp_inv, double* __restrict__ p) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = fma(-nu * d[t], mp_inv[t], p[t] + q[t]);
}

int grid_of(int64_t n) {
  int64_t g = (n + kNsBlock - 1) / kNsBlock;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

template <typename K, typename... A>
void ns_launch(K kernel, int64_t n, cudaStream_t s, A... args) {
  const int g = grid_of(n);
  if (t_prof) t_prof->before((const void*)kernel, s);
  kernel<<<g, kNsBlock, 0, s>>>(args...);
  if (t_prof) t_prof->after(s);
}

}  // namespace

void ns_interp(const NsView& V, const double* p, const double* q, double* pt, cudaStream_t s) {
  ns_launch(k_ns_interp, (int64_t)V.nv[0] * V.nv[1] * V.nv[2], s, V, p, q, pt);
}
void ns_momentum(const NsView& V, const double* u, const double* pt, double* un, cudaStream_t s) {
  ns_launch(k_ns_momentum, (int64_t)V.nv[0] * V.nv[1] * V.nv[2], s, V, u, pt, un);
}
void ns_div(const NsView& V, const double* u, double* dv, cudaStream_t s) {
  ns_launch(k_ns_div, (int64_t)V.nv[0] * V.nv[1] * V.nv[2], s, V, u, dv);
}
void ns_restrict(const NsView& V, const double* dv, double* d, double* b, cudaStream_t s) {
  ns_launch(k_ns_restrict, (int64_t)V.np[0] * V.np[1] * V.np[2], s, V, dv, d, b);
}
void ns_meanfree(int64_t np, const double* m, double total, double* q, cudaStream_t s) {
  if (t_prof) t_prof->before((const void*)k_ns_meanfree, s);
  k_ns_meanfree<<<1, 1024, 0, s>>>(np, m, total, q);
  if (t_prof) t_prof->after(s);
}
void ns_pupdate(int64_t np, double nu, const double* q, const double* d, const double* mp_inv, double* p,
                cudaStream_t s) {
  ns_launch(k_ns_pupdate, np, s, np, nu, q, d, mp_inv, p);
}

}  // namespace mgi
