/*
 * mg_debug.h -- host-only inspection of the hierarchy the library builds.
 *
 * These entry points run the same host setup as mg_setup (leaf validation,
 * global coarsening of Sec. 2.2, condensed Q1 operators with the hanging-node
 * matrix H_h of Sec. 2.2, transfers of Eq. "prolongation" with R = P^T,
 * Sec. 4.1.4) but stop before anything is packed or uploaded, so they need no
 * GPU.  They exist for testing and inspection; the solve path never uses them.
 *
 * Ownership: mg_host_build allocates the returned object; mg_host_free
 * releases it.  Arrays returned by mg_host_level point into that object and
 * stay valid until mg_host_free.  Errors: negative MG_ERR_* codes as in mg.h.
 */
#ifndef MG_GB300_DEBUG_H
#define MG_GB300_DEBUG_H

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_host_hier mg_host_hier;

/* Build the host hierarchy; opts may be NULL (defaults). */
int mg_host_build(const mg_mesh* mesh, const mg_problem* problem, const mg_opts* opts, mg_host_hier** out);
int mg_host_levels(const mg_host_hier* h);
/* Matrix `which` of a level as block CSR with nc x nc row-major blocks:
 *   0 = A_l (condensed level operator), 1 = P_l (scalar, rows = level l
 *   nodes, columns = level l-1 nodes), 2 = R_l = P_l^T (scalar), 3 = load
 *   matrix of the finest level (b = load * f before Dirichlet zeroing),
 *   4 = smoother blocks as a block-diagonal matrix, 5 = hanging-node matrix
 *   H (scalar, all nodes), 6 = lifting matrix of the finest level (the
 *   couplings (H^T A H)[free dof, Dirichlet dof], zero elsewhere), 7 = the
 *   cell-patch Vanka matrix S of the level (n = 0 on levels that smooth with
 *   Jacobi).  n/m: block
 *   rows/columns; nc: block size. */
int mg_host_level(const mg_host_hier* h, int level, int which, int64_t* n, int64_t* m, int* nc, int64_t* nnzb,
                  const int64_t** ptr, const int64_t** col, const double** val);
/* Per node of a level: fixed-dof bit mask (bit c set: dof c is hanging or
 * Dirichlet) and lattice coordinates (n_nodes * dim int64, finest lattice of
 * that level). */
int mg_host_nodes(const mg_host_hier* h, int level, const uint8_t** fixmask, int64_t* n_nodes);
/* Smoother damping of a level (opts.omega, or the automatic per-level rule). */
int mg_host_omega(const mg_host_hier* h, int level, double* omega);
/* Dense inverse of the coarse operator, (n0 nc)^2 row-major. */
int mg_host_coarse_inverse(const mg_host_hier* h, int64_t* n, const double** inv);
int mg_host_free(mg_host_hier* h);

#ifdef __cplusplus
}
#endif
#endif /* MG_GB300_DEBUG_H */
