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
// so on), and the lumped 3D mass is m1 x m1 x m1.  The momentum and
// divergence kernels apply them axis by axis on shared-memory tiles (sum
// factorisation), the others as stencils with the per-axis coefficients
// (nothing is stored per node but the vectors).  The interpolation P from the pressure grid (node J
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
// Every term is a Kronecker product X (x) Y (x) Z of the 1D operators, so the
// 27-point sum is taken axis by axis (sum factorisation) on a tile of
// kTx x kTy x kTz nodes with a one-node halo, staged in shared memory:
//   z pass, at (i', j', k):  A_c = Mz (u_x u_c)  [+ Mz ps for c = x]
//                            B_c = Mz (u_y u_c)  [+ Mz ps for c = y]
//                            D_c = Gz (u_z u_c) - nu Kz u_c  [+ Gz ps for c = z]
//                            E_c = Mz u_c
//   y pass, at (i', j, k):   Y1_c = My A_c
//                            Y2_c = Gy B_c + My D_c - nu Ky E_c
//                            Y3_c = My E_c
//   x pass, at (i, j, k):    acc_c = Gx Y1_c + Mx Y2_c - nu Kx Y3_c
// which is sum_b C_b (u_b u_c) - nu K u_c + C_c ps with C_x = Gx My Mz,
// C_y = Mx Gy Mz, C_z = Mx My Gz and K = Kx My Mz + Mx Ky Mz + Mx My Kz:
// about 180 FP64 operations per node instead of about 420 for the 27-point
// stencil (the kernel is bound by the FP64 pipe); -nu K and 1 / m1 come per
// axis from the setup.
constexpr int kTx = 8, kTy = 8, kTz = 4;
constexpr int kHx = kTx + 2, kHy = kTy + 2, kHz = kTz + 2;
constexpr int kNIn = kHx * kHy * kHz;          // input nodes (halo on every side)
constexpr int kNZ = kHx * kHy * kTz;           // z-pass nodes (halo in x and y)
constexpr int kNY = kHx * kTy * kTz;           // y-pass nodes (halo in x)
constexpr size_t kMomentumSmem = sizeof(double) * (4 * kNIn + 12 * kNZ + 9 * kNY);
static_assert(kTx * kTy * kTz == kNsBlock, "one output node per thread in the x pass");

__global__ void __launch_bounds__(kNsBlock) k_ns_momentum(NsView V, const double* __restrict__ u,
                                                          const double* __restrict__ pt, double* __restrict__ un) {
  extern __shared__ double sm[];
  double* ux = sm;                 // [kNIn] each
  double* uy = ux + kNIn;
  double* uz = uy + kNIn;
  double* ps = uz + kNIn;
  double* Z = ps + kNIn;           // [12][kNZ]: A_c, B_c, D_c, E_c for c = 0..2
  double* Y = Z + 12 * kNZ;        // [9][kNY]: Y1_c, Y2_c, Y3_c for c = 0..2
  const int n0 = V.nv[0], n1 = V.nv[1], n2 = V.nv[2];
  const int i0 = blockIdx.x * kTx, j0 = blockIdx.y * kTy, k0 = blockIdx.z * kTz;
  const int tid = threadIdx.x;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  // this thread's output node (x pass)
  const int ox = tid % kTx, oy = (tid / kTx) % kTy, oz = tid / (kTx * kTy);
  const int gi = i0 + ox, gj = j0 + oy, gk = k0 + oz;
  const bool inside = gi < n0 && gj < n1 && gk < n2;
  const bool interior = gi > 0 && gj > 0 && gk > 0 && gi < n0 - 1 && gj < n1 - 1 && gk < n2 - 1;
  // a tile with no interior node only writes boundary values
  const bool work = i0 + kTx - 1 >= 1 && i0 <= n0 - 2 && j0 + kTy - 1 >= 1 && j0 <= n1 - 2 &&
                    k0 + kTz - 1 >= 1 && k0 <= n2 - 2;
  if (work) {
    // inputs u and ps on the tile with its halo (zero outside the mesh)
    for (int n = tid; n < kNIn; n += kNsBlock) {
      const int a = n % kHx, b = (n / kHx) % kHy, c = n / (kHx * kHy);
      const int i = i0 - 1 + a, j = j0 - 1 + b, k = k0 - 1 + c;
      double vx = 0.0, vy = 0.0, vz = 0.0, vp = 0.0;
      if (i >= 0 && j >= 0 && k >= 0 && i < n0 && j < n1 && k < n2) {
        const int64_t t = i + j * sy + k * sz;
        vx = u[3 * t];
        vy = u[3 * t + 1];
        vz = u[3 * t + 2];
        vp = pt[t];
      }
      ux[n] = vx;
      uy[n] = vy;
      uz[n] = vz;
      ps[n] = vp;
    }
    __syncthreads();
    // z pass
    for (int n = tid; n < kNZ; n += kNsBlock) {
      const int a = n % kHx, b = (n / kHx) % kHy, c = n / (kHx * kHy);
      const int i = i0 - 1 + a, j = j0 - 1 + b, k = k0 + c;
      double A[3] = {0.0, 0.0, 0.0}, Bv[3] = {0.0, 0.0, 0.0}, D[3] = {0.0, 0.0, 0.0}, E[3] = {0.0, 0.0, 0.0};
      if (i >= 0 && j >= 0 && i < n0 && j < n1 && k < n2) {
        double pm = 0.0, pg = 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const int q = a + kHx * (b + kHy * (c + e));     // input node (i', j', k + e - 1)
          const double mz = V.ax[2].M[3 * k + e], gz = V.ax[2].G[3 * k + e], kz = V.ax[2].Kn[3 * k + e];
          const double vx = ux[q], vy = uy[q], vz = uz[q], vp = ps[q];
          const double g = fma(gz, vz, kz);                // Gz u_z - nu Kz, shared by the components
          pm = fma(mz, vp, pm);
          pg = fma(gz, vp, pg);
          const double vc[3] = {vx, vy, vz};
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            const double w = mz * vc[cc];
            A[cc] = fma(w, vx, A[cc]);
            Bv[cc] = fma(w, vy, Bv[cc]);
            E[cc] += w;
            D[cc] = fma(g, vc[cc], D[cc]);
          }
        }
        A[0] += pm;
        Bv[1] += pm;
        D[2] += pg;
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        Z[(0 + cc) * kNZ + n] = A[cc];
        Z[(3 + cc) * kNZ + n] = Bv[cc];
        Z[(6 + cc) * kNZ + n] = D[cc];
        Z[(9 + cc) * kNZ + n] = E[cc];
      }
    }
    __syncthreads();
    // y pass
    for (int n = tid; n < kNY; n += kNsBlock) {
      const int a = n % kHx, b = (n / kHx) % kTy, c = n / (kHx * kTy);
      const int i = i0 - 1 + a, j = j0 + b, k = k0 + c;
      double Y1[3] = {0.0, 0.0, 0.0}, Y2[3] = {0.0, 0.0, 0.0}, Y3[3] = {0.0, 0.0, 0.0};
      if (i >= 0 && i < n0 && j < n1 && k < n2) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const int q = a + kHx * ((b + e) + kHy * c);     // z-pass node (i', j + e - 1, k)
          const double my = V.ax[1].M[3 * j + e], gy = V.ax[1].G[3 * j + e], ky = V.ax[1].Kn[3 * j + e];
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            const double zA = Z[(0 + cc) * kNZ + q], zB = Z[(3 + cc) * kNZ + q], zD = Z[(6 + cc) * kNZ + q],
                         zE = Z[(9 + cc) * kNZ + q];
            Y1[cc] = fma(my, zA, Y1[cc]);
            Y2[cc] = fma(gy, zB, fma(my, zD, fma(ky, zE, Y2[cc])));
            Y3[cc] = fma(my, zE, Y3[cc]);
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        Y[(0 + cc) * kNY + n] = Y1[cc];
        Y[(3 + cc) * kNY + n] = Y2[cc];
        Y[(6 + cc) * kNY + n] = Y3[cc];
      }
    }
    __syncthreads();
  }
  if (!inside) return;
  const int64_t t = gi + gj * sy + gk * sz;
  if (!interior) {
    un[3 * t] = 0.0;
    un[3 * t + 1] = gi == n0 - 1 ? V.lid : 0.0;
    un[3 * t + 2] = 0.0;
    return;
  }
  // x pass
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int q = (ox + e) + kHx * (oy + kTy * oz);         // y-pass node (i + e - 1, j, k)
    const double mx = V.ax[0].M[3 * gi + e], gx = V.ax[0].G[3 * gi + e], kx = V.ax[0].Kn[3 * gi + e];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      acc[cc] = fma(gx, Y[(0 + cc) * kNY + q], fma(mx, Y[(3 + cc) * kNY + q], fma(kx, Y[(6 + cc) * kNY + q], acc[cc])));
  }
  const double s = V.dt * V.ax[0].im1[gi] * V.ax[1].im1[gj] * V.ax[2].im1[gk];
  un[3 * t] = fma(s, acc[0], u[3 * t]);
  un[3 * t + 1] = fma(s, acc[1], u[3 * t + 1]);
  un[3 * t + 2] = fma(s, acc[2], u[3 * t + 2]);
}

// dv_i = sum_j sum_c C_c[j, i] u_{j,c} = ((div u, phi_i))_i at every velocity node:
// dv = (GTx My Mz) u_x + (Mx GTy Mz) u_y + (Mx My GTz) u_z, summed axis by axis
// on the same tiles as the momentum step:
//   z pass, at (i', j', k):  a = Mz u_x, b = Mz u_y, c = GTz u_z
//   y pass, at (i', j, k):   Y1 = My a, Y2 = GTy b + My c
//   x pass, at (i, j, k):    dv = GTx Y1 + Mx Y2
// (the 1D factors are zero towards a missing neighbour, and the halo outside
// the mesh is zero, so boundary nodes need no special case).
constexpr size_t kDivSmem = sizeof(double) * (3 * kNIn + 3 * kNZ + 2 * kNY);

__global__ void __launch_bounds__(kNsBlock) k_ns_div(NsView V, const double* __restrict__ u, double* __restrict__ dv) {
  extern __shared__ double sm[];
  double* ux = sm;                 // [kNIn] each
  double* uy = ux + kNIn;
  double* uz = uy + kNIn;
  double* Z = uz + kNIn;           // [3][kNZ]: a, b, c
  double* Y = Z + 3 * kNZ;         // [2][kNY]: Y1, Y2
  const int n0 = V.nv[0], n1 = V.nv[1], n2 = V.nv[2];
  const int i0 = blockIdx.x * kTx, j0 = blockIdx.y * kTy, k0 = blockIdx.z * kTz;
  const int tid = threadIdx.x;
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  for (int n = tid; n < kNIn; n += kNsBlock) {
    const int a = n % kHx, b = (n / kHx) % kHy, c = n / (kHx * kHy);
    const int i = i0 - 1 + a, j = j0 - 1 + b, k = k0 - 1 + c;
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (i >= 0 && j >= 0 && k >= 0 && i < n0 && j < n1 && k < n2) {
      const int64_t t = i + j * sy + k * sz;
      vx = u[3 * t];
      vy = u[3 * t + 1];
      vz = u[3 * t + 2];
    }
    ux[n] = vx;
    uy[n] = vy;
    uz[n] = vz;
  }
  __syncthreads();
  for (int n = tid; n < kNZ; n += kNsBlock) {
    const int a = n % kHx, b = (n / kHx) % kHy, c = n / (kHx * kHy);
    const int i = i0 - 1 + a, j = j0 - 1 + b, k = k0 + c;
    double za = 0.0, zb = 0.0, zc = 0.0;
    if (i >= 0 && j >= 0 && i < n0 && j < n1 && k < n2) {
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int q = a + kHx * (b + kHy * (c + e));       // input node (i', j', k + e - 1)
        const double mz = V.ax[2].M[3 * k + e], gz = V.ax[2].GT[3 * k + e];
        za = fma(mz, ux[q], za);
        zb = fma(mz, uy[q], zb);
        zc = fma(gz, uz[q], zc);
      }
    }
    Z[n] = za;
    Z[kNZ + n] = zb;
    Z[2 * kNZ + n] = zc;
  }
  __syncthreads();
  for (int n = tid; n < kNY; n += kNsBlock) {
    const int a = n % kHx, b = (n / kHx) % kTy, c = n / (kHx * kTy);
    const int i = i0 - 1 + a, j = j0 + b, k = k0 + c;
    double y1 = 0.0, y2 = 0.0;
    if (i >= 0 && i < n0 && j < n1 && k < n2) {
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int q = a + kHx * ((b + e) + kHy * c);       // z-pass node (i', j + e - 1, k)
        const double my = V.ax[1].M[3 * j + e], gy = V.ax[1].GT[3 * j + e];
        y1 = fma(my, Z[q], y1);
        y2 = fma(gy, Z[kNZ + q], fma(my, Z[2 * kNZ + q], y2));
      }
    }
    Y[n] = y1;
    Y[kNY + n] = y2;
  }
  __syncthreads();
  const int ox = tid % kTx, oy = (tid / kTx) % kTy, oz = tid / (kTx * kTy);
  const int gi = i0 + ox, gj = j0 + oy, gk = k0 + oz;
  if (gi >= n0 || gj >= n1 || gk >= n2) return;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int q = (ox + e) + kHx * (oy + kTy * oz);         // y-pass node (i + e - 1, j, k)
    acc = fma(V.ax[0].GT[3 * gi + e], Y[q], fma(V.ax[0].M[3 * gi + e], Y[kNY + q], acc));
  }
  dv[gi + gj * sy + gk * sz] = acc;
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
  static const bool attr_set =
      cudaFuncSetAttribute(k_ns_momentum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMomentumSmem) ==
      cudaSuccess;
  (void)attr_set;
  const dim3 grid((V.nv[0] + kTx - 1) / kTx, (V.nv[1] + kTy - 1) / kTy, (V.nv[2] + kTz - 1) / kTz);
  if (t_prof) t_prof->before((const void*)k_ns_momentum, s);
  k_ns_momentum<<<grid, kNsBlock, kMomentumSmem, s>>>(V, u, pt, un);
  if (t_prof) t_prof->after(s);
}
void ns_div(const NsView& V, const double* u, double* dv, cudaStream_t s) {
  const dim3 grid((V.nv[0] + kTx - 1) / kTx, (V.nv[1] + kTy - 1) / kTy, (V.nv[2] + kTz - 1) / kTz);
  if (t_prof) t_prof->before((const void*)k_ns_div, s);
  k_ns_div<<<grid, kNsBlock, kDivSmem, s>>>(V, u, dv);
  if (t_prof) t_prof->after(s);
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
