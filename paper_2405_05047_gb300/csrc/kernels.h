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
};

// Transfer matrices (P, R) are scalar SELL with float weights.
struct TransferView {
  const int64_t* sptr = nullptr;
  const int32_t* col = nullptr;
  const float* w = nullptr;
  int64_t n = 0;
  int64_t nslices = 0;
};

// Scalars of the Krylov loop, resident in device memory.
struct KrylovState {
  double rho, rho_prev, alpha, omega, beta;
  double rnorm, bnorm, rtol, scale;  // scale: factor of the FP32 preconditioner input
  int iter, max_it, done, status;
  int restart_pos;
  int pad[3];
};

// Reduction partials: one slot array per quantity, kMaxRedBlocks each.
struct Partials {
  double* p = nullptr;                 // [nq][kMaxRedBlocks]
  double* q(int k) const { return p + (int64_t)k * kMaxRedBlocks; }
};

int grid_for_rows(int64_t rows);       // blocks for one thread per row, capped for grid-stride
int grid_for_vec(int64_t n);

// ---- level operators (T = double or float; nc = 1 or 3) --------------------
template <typename T>
void launch_smooth(const SellView& A, int nc, const T* x, const T* b, const T* Sinv, T* xo, double omega,
                   bool from_zero, const int* done, cudaStream_t s);
template <typename T>
void launch_residual(const SellView& A, int nc, const T* x, const T* b, T* r, const int* done, cudaStream_t s);
template <typename T>
void launch_matvec(const SellView& A, int nc, const T* x, T* y, const int* done, cudaStream_t s);
template <typename T>
void launch_restrict(const TransferView& R, int nc, const T* r, T* d, const int* done, cudaStream_t s);
template <typename T>
void launch_prolong_add(const TransferView& P, int nc, const T* y, const T* xin, T* xo, const int* done,
                        cudaStream_t s);
template <typename T>
void launch_coarse(const double* Ainv, int64_t n, const T* d, T* z, const int* done, cudaStream_t s);

// ---- vector kernels --------------------------------------------------------
void launch_rhs(const SellView& F, int nc, const double* f, const uint8_t* fixmask, double* b, cudaStream_t s);
void launch_fill_hanging(const TransferView& Hc, int nc, double* x, cudaStream_t s);
void launch_copy_fixed(int64_t n_nodes, int nc, const uint8_t* fixmask, const double* b, const double* xin,
                       double* x, cudaStream_t s);
// partial of sum over free dofs of b^2 (quantity k of part)
void launch_norm_free(int64_t n_nodes, int nc, const uint8_t* fixmask, const double* b, Partials part, int k,
                      cudaStream_t s);

// ---- Krylov kernels (FP64 outer loop) --------------------------------------
// Preconditioned vectors come either as double (zs == nullptr) or as float
// times the scalar st->scale (z32 != nullptr).
struct PVec {
  const double* d = nullptr;
  const float* f = nullptr;
};

void launch_residual_norm(const SellView& A64, int nc, const double* x, const double* b, double* r, Partials part,
                          int k, cudaStream_t s);
void launch_finalize(Partials part, int k_rr, int nred, KrylovState* st, int first, unsigned long long cond_handle,
                     cudaStream_t s);
void launch_init_state(KrylovState* st, Partials part, int k_bb, int nred, double rtol, int max_it, cudaStream_t s);
void launch_to_f32(int64_t n, const double* v, float* v32, const KrylovState* st, cudaStream_t s);
// Quantity slots of the partial arrays
enum { Q_RR = 0, Q_RZ = 1, Q_QZ = 2, Q_PQ = 3, Q_BB = 4, Q_RHV = 5, Q_SS = 6, Q_TS = 7, Q_TT = 8, Q_RHR = 9, Q_NUM = 10 };
// CG (flexible, Polak-Ribiere beta): dots -> Q_RZ, Q_QZ; update_p; spmv_dot -> Q_PQ; update_xr -> Q_RR
void launch_cg_dots(int64_t nn, int nc, PVec z, const double* r, const double* q, Partials part,
                    const KrylovState* st, cudaStream_t s);
void launch_cg_update_p(int64_t nn, int nc, PVec z, double* p, Partials part, int nred, KrylovState* st,
                        cudaStream_t s);
void launch_spmv_dot(const SellView& A64, int nc, PVec p, const double* w, double* out, Partials part, int k,
                     const KrylovState* st, cudaStream_t s);
void launch_cg_update_xr(int64_t nn, int nc, const double* p, const double* q, double* x, double* r, Partials part,
                         int nred, KrylovState* st, cudaStream_t s);
// BiCGStab (right preconditioned): p (Q_RHR) ; spmv_dot -> Q_RHV ; s ; spmv_2dots -> Q_TS, Q_TT ; x -> Q_RR, Q_RHR
void launch_bicg_p(int64_t nn, int nc, const double* r, const double* v, double* p, Partials part, int nred,
                   KrylovState* st, cudaStream_t s);
void launch_bicg_s(int64_t nn, int nc, const double* r, const double* v, double* sv, Partials part, int nred,
                   KrylovState* st, cudaStream_t s);
void launch_spmv_2dots(const SellView& A64, int nc, PVec sh, const double* sv, double* t, Partials part,
                       const KrylovState* st, cudaStream_t s);
void launch_bicg_x(int64_t nn, int nc, PVec ph, PVec sh, const double* sv, const double* t, const double* rhat,
                   double* x, double* r, Partials part, int nred, KrylovState* st, cudaStream_t s);

}  // namespace mgi
