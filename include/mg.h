/*
 * mg.h -- C ABI of the GB300 geometric-multigrid Krylov solver for adaptive
 * Q1 finite elements on quad/hex meshes with hanging nodes.
 *
 * The method is that of arXiv:2405.05047 ("An adaptive finite element
 * multigrid solver using GPU acceleration"):
 *   - Q1 elements on 1-irregular meshes, hanging nodes eliminated through the
 *     interpolation matrix H_h (Sec. 2.1, 2.2);
 *   - a hierarchy built by global coarsening of the finest mesh (Sec. 2.2);
 *   - the V-cycle of Algorithm "Geometric multigrid solver" with a damped
 *     (block-)Jacobi smoother x <- x + omega S (b - A x) and transfers given by
 *     the local embedding P_l, R_l = P_l^T (Sec. 4.1.4, Eq. "prolongation");
 *   - the V-cycle as preconditioner of a Krylov method (Sec. 4.1.5).
 *
 * Conventions for every entry point:
 *   - return value: MG_OK (0) or a negative MG_ERR_* code; mg_strerror() names
 *     it.  No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device; "host" pointers are ordinary CPU memory.  Pointers passed in are
 *     only read during the call unless stated; the library never frees memory
 *     it did not allocate.
 *   - vectors are node-major: entry (node i, component c) is at i*nc + c, with
 *     nodes in the *external order*: integer lattice coordinates of the finest
 *     level sorted lexicographically, x fastest, then y, then z.
 *   - a context is used from one host thread at a time; calls run on the
 *     context's stream and return after the device work has finished unless
 *     stated otherwise.
 */
#ifndef MG_GB300_H
#define MG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  MG_OK = 0,
  MG_PENDING = 1,              /* mg_poll: request still queued or running      */
  MG_ERR_INVALID = -1,         /* bad argument, malformed mesh, unknown ticket  */
  MG_ERR_OOM = -2,             /* device allocation failed                      */
  MG_ERR_ADMISSION = -3,       /* request can never fit the HBM budget          */
  MG_ERR_NOT_CONVERGED = -4,   /* max_it reached; x and stats are still valid   */
  MG_ERR_BREAKDOWN = -5,       /* Krylov breakdown (zero denominator)           */
  MG_ERR_NAN = -6,             /* NaN/Inf met in a reduction                    */
  MG_ERR_TIMEOUT = -7,         /* a bounded device-side wait gave up            */
  MG_ERR_CUDA = -8,            /* CUDA runtime error                            */
  MG_ERR_CANCELLED = -9        /* mg_cancel'ed request                          */
};

typedef enum { MG_FP64 = 0, MG_MIXED_FP32 = 1, MG_MIXED_BF16 = 2 } mg_precision;
typedef enum { MG_POISSON = 0, MG_TRANSPORT = 1, MG_ELASTICITY = 2, MG_OSEEN = 3 } mg_kind;
/* MG_MGITER: the multigrid iteration itself as the solver, x <- x + GMG(0, b - A x)
 * with the defect computed in FP64 (defect correction when the V-cycle runs
 * in FP32). */
typedef enum { MG_KRYLOV_AUTO = 0, MG_CG = 1, MG_BICGSTAB = 2, MG_GMRES = 3, MG_MGITER = 4 } mg_krylov;
/* Smoother of the multigrid levels (Sec. 4.1.4: damped block Jacobi; Sec. 6
 * names Vanka smoothers for saddle-point problems as the next step). */
typedef enum { MG_SMOOTHER_JACOBI = 0, MG_SMOOTHER_VANKA = 1 } mg_smoother;

typedef struct mg_ctx mg_ctx;
typedef struct mg_hier mg_hier;

/* Device allocator callbacks (optional).  malloc_fn returns a device pointer
 * aligned to >= 256 bytes or NULL; free_fn releases it.  With alloc == NULL
 * the library uses cudaMalloc/cudaFree. */
typedef struct {
  void* (*malloc_fn)(size_t bytes, void* user);
  void (*free_fn)(void* ptr, void* user);
  void* user;
} mg_allocator;

/* Leaf mesh (host memory, copied by mg_setup).  Domain: the box
 * origin + [0, extent]; level 0 is a macro[0] x macro[1] (x macro[2]) grid;
 * leaf k has level leaf_level[k] and integer anchor
 * leaf_anchor[k*dim + d] in [0, macro[d] << level).  The leaves must tile the
 * box exactly and be 1-irregular: face neighbours differ by <= 1 level
 * (Sec. 2.2: "We allow a level jump of 1 for neighboring elements"). */
typedef struct {
  int dim;                     /* 2 or 3 */
  double origin[3];
  double extent[3];
  int macro[3];
  int64_t n_leaves;
  const int32_t* leaf_level;   /* host, n_leaves */
  const int32_t* leaf_anchor;  /* host, n_leaves * dim */
  const double* axis[3];       /* optional tensor-product (graded) geometry:
                                  NULL, or for every d < dim a host array of
                                  (macro[d] << L) + 1 strictly increasing node
                                  coordinates along axis d, L the finest leaf
                                  level; node (i, j, k) of the finest lattice
                                  sits at (axis[0][i], axis[1][j], axis[2][k])
                                  and a coarser lattice's nodes at the same
                                  points (every 2^(L-l)-th entry).  Cells stay
                                  axis-aligned boxes, each with its own sizes;
                                  origin and extent are then taken from the
                                  arrays.  Every leaf must have the same level
                                  (a hanging node would not sit at its edge's
                                  middle).  Not for OSEEN.                     */
} mg_mesh;

/* Problem: bilinear form and Dirichlet faces.  Face bit 2d = face x_d = min,
 * bit 2d+1 = face x_d = max; dirichlet_mask[c] selects the faces on which
 * component c is prescribed (values from mg_assemble_rhs's g, else 0).
 * A POISSON problem with no prescribed dof at all (no Dirichlet face, no
 * pin, no mass) is the pure Neumann problem: its null space are the
 * constants, right-hand sides must be compatible (sum of b = 0), and the
 * solve returns one solution (determined up to a constant; the coarse solve
 * applies the pseudo-inverse of A_0).
 *   POISSON      (grad u, grad v)                                  nc = 1
 *   TRANSPORT    eps (grad u, grad v) + (beta.grad u, v)
 *                + sum_T delta_T (beta.grad u, beta.grad v)_T,
 *                delta_T = supg_delta0 h_T^2 / (6 eps + |beta| h_T)   nc = 1
 *   ELASTICITY   2 mu (eps(u), eps(v)) + lambda (div u, div v), 3D  nc = 3
 *   OSEEN        one linearised backward-Euler step of incompressible flow
 *                (Sec. 5.3's equations), 2D, unknowns (u, v, p), nc = 3:
 *                (1/dt)(u, v) + nu (grad u, grad v) + ((beta_h.grad) u, v)
 *                - (p, div v) + (div u, q)
 *                + sum_P alpha_P [(grad kp, grad kq)_P
 *                                 + (beta_P.grad ku, beta_P.grad kv)_P]
 *                with local projection stabilisation on patches P (the
 *                parents of the sibling families: the mesh must be a patch
 *                mesh, every leaf in a complete family), k = id - i_2h the
 *                fluctuation w.r.t. the patch's coarse Q1 interpolant,
 *                alpha_P = lps_alpha0 h_P^2 / (nu + |beta_P| h_P), h_P the
 *                patch diameter, beta_h the cell-wise Q1 interpolant of the
 *                nodal field conv, beta_P its value at the patch centre.
 *                Coarser levels inject conv at their nodes and are coarsened
 *                so that they stay patch meshes (coarsest >= level 1). */
typedef struct {
  int kind;
  double eps;
  double beta[3];
  double mu;
  double lambda;
  double supg_delta0;
  uint32_t dirichlet_mask[3];
  double nu;                   /* OSEEN: viscosity                              */
  double dt;                   /* OSEEN: time step (INFINITY: no mass term)     */
  double lps_alpha0;           /* OSEEN: LPS parameter (0.5 is customary)       */
  const double* conv;          /* OSEEN: host, n_nodes * dim doubles, the nodal
                                  convection field at the finest nodes in the
                                  external order (see mg_mesh_nodes); read
                                  during mg_setup only                          */
  double mass;                 /* POISSON, TRANSPORT, ELASTICITY: coefficient
                                  s >= 0 of an added mass term s (u, v) (every
                                  component); s = 1/dt gives the matrix of one
                                  backward-Euler step of a first-order-in-time
                                  problem (Sec. 5.1), s = 1/dt^2 that of
                                  d_t^2 u + A u = f (Sec. 5.2).  With SUPG the
                                  stabilisation also tests it:
                                  + sum_T delta_T s (u, beta.grad v)_T.
                                  0: stationary                                 */
  int pin_origin;              /* 1: the node at the origin corner is also
                                  prescribed (every component, every level;
                                  value from g, else 0): with no Dirichlet face
                                  this picks one solution of the pure Neumann
                                  problem (constants are its null space), e.g.
                                  the pressure increment of Sec. 5.3           */
} mg_problem;

typedef struct {
  int nu1, nu2;                /* pre/post smoothing sweeps (default 2, 2)    */
  double omega;                /* damping of the (block-)Jacobi smoother: > 0
                                  on every level; <= 0 (default -1): 0.8 for
                                  scalar problems on uniform boxes, 1.2 /
                                  lambda_max(S_l A_l) per level for the
                                  point-block smoothers and on graded meshes
                                  (20 power iterations at setup)             */
  int min_level;               /* coarsest level allowed (-1: automatic)      */
  int max_levels;              /* cap on the number of levels (0: no cap)     */
  int krylov;                  /* mg_krylov                                   */
  int restart;                 /* GMRES restart length (default 30)           */
  int store_fp64;              /* keep FP64 level matrices (1) for MG_FP64    */
  int store_fp32;              /* keep FP32 level matrices (1) for mixed modes*/
  int launch_mode;             /* 0: whole solve as one CUDA-graph while loop;
                                  1: direct kernel launches, host polls the
                                  status after every iteration (profilers)   */
  int tail_rows;               /* levels with at most this many dofs (and all
                                  coarser ones) run as one single-CTA kernel
                                  per V-cycle (0: off; default 4096)          */
  int store_bf16;              /* keep BF16 copies of the level matrices for
                                  MG_MIXED_BF16 (FP32 vectors and arithmetic,
                                  values rounded to BF16: an ablation)        */
  int autotune;                /* 1 (default): at setup, time V-cycles over
                                  tail thresholds x cluster sizes and keep the
                                  fastest (cached per hierarchy shape); and per
                                  level of >= 32768 rows time the FP32 sweep over
                                  SELL windows {0, 256, 1024} x 16-bit columns
                                  {off, on} and keep the fastest for the
                                  FP32 / BF16 copies (cached per level shape;
                                  only where sell_sigma and col16 are
                                  automatic).  V-cycles do not depend on
                                  either choice.                              */
  double inner_rtol;           /* > 0: defect correction -- every round runs
                                  the Krylov method until its residual fell by
                                  this factor (or reached rtol), then the FP64
                                  defect b - A x is recomputed and the next
                                  round solves for the correction (0: off)    */
  int sell_sigma;              /* SELL-C-sigma window: rows of each window of
                                  sigma rows sorted by length before slicing
                                  (-1: automatic, 256 on levels of >= 32768
                                  rows; 0: never; > 0: this window on every
                                  level, a multiple of 32)                    */
  int col16;                   /* 16-bit column offsets in the level matrices,
                                  every stored precision (-1: automatic,
                                  levels of >= 32768 rows; 0: never; 1: every
                                  level)                                      */
  int row_lanes;               /* lanes per row of the FP32/BF16 level matrices
                                  (-1: automatic, 4 on the small latency-bound
                                  levels; 1: one lane per row everywhere)     */
  int smoother;                /* MG_SMOOTHER_JACOBI (default): damped
                                  (point-block) Jacobi on every level;
                                  MG_SMOOTHER_VANKA: the additive cell-patch
                                  Vanka smoother x <- x + w S (b - A x) with
                                  S = W sum_T P_T A_T^-1 P_T^T (A_T: the level
                                  operator on the 2^dim nc unknowns of cell T,
                                  inverted densely at setup; W = 1/(cells
                                  containing the node)) on the levels >= 1
                                  with at least vanka_rows unknowns, Jacobi
                                  below; the small-level kernel only takes
                                  Jacobi levels                               */
  int vanka_rows;              /* see smoother (default 0: every level >= 1)  */
  double vanka_omega;          /* damping w of the Vanka levels (default 1)   */
  int stage_x;                 /* FP32 / BF16 scalar sweeps with one lane per
                                  row gather x from shared memory: each block
                                  first loads the range of x its 256 rows'
                                  columns span (when at most 4096 entries)
                                  (-1: levels of >= 32768 rows; 0 (default):
                                  never; 1: every such level).  Same bits
                                  either way; off by default because the
                                  gathers it replaces already hit in L1/L2
                                  and the staging pass plus its barriers cost
                                  more than they save.                         */
} mg_opts;

typedef struct {
  int dim, nc, levels;
  int64_t n_nodes, n_dofs, n_free;      /* finest level                        */
  int64_t level_nodes[32];              /* [0] = coarsest                      */
  int64_t level_nnzb[32];               /* stored blocks (incl. padding)       */
  int64_t level_rows_nnzb[32];          /* blocks without SELL padding         */
  size_t bytes_device;                  /* hierarchy + workspace               */
  int64_t n_hanging;
  double omega;
  size_t bytes_workspace;               /* one extra solve workspace (serving)   */
  int tail_levels;                      /* levels run by the cluster tail kernel  */
  int tail_cluster;                     /* CTAs in that kernel's cluster (0: one
                                           CTA working in shared memory; < 0: a
                                           cluster-resident tail of -tail_cluster
                                           CTAs, see mg_tune)                    */
  double vcycle_ms;                     /* tuned V-cycle time (0 if not tuned)    */
  int64_t col16_slices;                 /* slices read with 16-bit columns        */
  int64_t col32_slices;                 /* slices of those matrices that keep
                                           32-bit columns (offsets outside int16) */
  int level_col16[32];                  /* 1: the level's operator copies store
                                           16-bit column offsets                 */
  double level_omega[32];               /* smoother damping per level            */
  int level_block_values[32];           /* values stored per block of the level
                                           operator: nc*nc, or 6 for 3x3 blocks of
                                           the velocity-pressure pattern
                                           [[a,0,g1],[0,a,g2],[d1,d2,c]]          */
  int level_smoother[32];               /* mg_smoother used on the level          */
  int64_t level_vanka_nnzb[32];         /* blocks of the level's Vanka matrix
                                           (0 on Jacobi levels)                   */
  int64_t level_sigma[32];              /* SELL-C-sigma window of the level
                                           operator's FP32 / BF16 copies (0: rows
                                           in node order); with opts.autotune it
                                           and level_col16 are the fastest of a
                                           timed set for the FP32 sweep (both keep
                                           every row's summation order: no V-cycle
                                           bit depends on them; the FP64 copies
                                           keep the size rule)                    */
  int level_lanes[32];                  /* lanes per row of the level operator's
                                           FP32 / BF16 copies (1 or 4, the size
                                           rule of opts.row_lanes)                */
} mg_info;

typedef struct {
  int status;                  /* MG_OK, MG_ERR_NOT_CONVERGED, ...            */
  int iters;                   /* Krylov iterations                           */
  int vcycles;                 /* preconditioner applications                 */
  int precision;               /* mg_precision used                           */
  double rel_res;              /* true ||b - A x||_2 / ||b_free||_2 (FP64)    */
  double solve_ms;             /* device time of the solve                    */
  double setup_ms;             /* for mg_poll: time from submit to start      */
  int64_t launches;            /* kernels launched by the solve               */
} mg_stats;

const char* mg_strerror(int code);
/* Message of the last error raised on the calling thread (static storage,
 * valid until the next call on that thread). */
const char* mg_last_error(void);
void mg_default_opts(mg_opts* opts);

/* Context: one device, one stream (a cudaStream_t from the caller, e.g.
 * torch.cuda.current_stream().cuda_stream, or NULL for a private stream),
 * an HBM budget (bytes; 0 = no limit) that bounds every hierarchy and
 * workspace allocated through this context.  The allocator struct is copied.
 * MG_ERR_INVALID for a device that gives a block less than 227 KB of shared
 * memory on opt-in (the staged small-level kernel needs 226 KB). */
int mg_init(int device, size_t hbm_budget_bytes, const mg_allocator* alloc, void* stream, mg_ctx** out);
/* MG_ERR_INVALID while hierarchies of this context are still alive. */
int mg_destroy(mg_ctx* ctx);

/* Build the hierarchy (Sec. 2.2 global coarsening; level operators by
 * rediscretisation; transfers from the local embedding, Eq. "prolongation")
 * on the host, pack it in the device layouts and upload it.  mesh, problem and
 * opts are copied; the library owns all device memory of the hierarchy.
 * MG_ERR_INVALID for a malformed mesh (overlap, gap, 2:1 violation),
 * MG_ERR_ADMISSION when the hierarchy would exceed the context's budget. */
int mg_setup(mg_ctx* ctx, const mg_mesh* mesh, const mg_problem* problem, const mg_opts* opts,
             mg_hier** out);
int mg_hier_info(const mg_hier* h, mg_info* info);
/* Finest-level nodes of a leaf mesh before any setup: *n_nodes receives their
 * number and, when xyz_host != NULL, their physical coordinates (host buffer
 * of n_nodes * dim doubles, external order).  MG_ERR_INVALID for a malformed
 * mesh.  Needs no context and no GPU. */
int mg_mesh_nodes(const mg_mesh* mesh, int64_t* n_nodes, double* xyz_host);
/* Physical coordinates of the finest-level nodes, external order, host
 * buffer of n_nodes * dim doubles. */
int mg_node_coords(const mg_hier* h, double* xyz_host);
int mg_free(mg_hier* h);

/* b = H^T (M I_h f) (+ SUPG load term) with the Dirichlet data eliminated
 * symmetrically: b -= (H^T A H)[:, D] g_D on the free rows, b = g on the
 * Dirichlet rows, 0 on hanging rows (Sec. 2.2 for H, H^T).
 * f_nodal: device, n_nodes * nc doubles (nodal source values at every node,
 * hanging ones included); g_nodal: device, n_nodes * nc doubles or NULL
 * (homogeneous data), only its Dirichlet entries are read; b: device,
 * n_nodes * nc doubles. */
int mg_assemble_rhs(mg_hier* h, const double* f_nodal, const double* g_nodal, double* b);

/* Backward-Euler time stepping with the hierarchy resident (Sec. 5.1;
 * Algorithm "Nonstationary Linear Problem": the matrices are assembled and
 * uploaded once, every step assembles its right-hand side and solves on the
 * device).  The hierarchy's problem must have mass = 1/dt > 0; its operator
 * is then the step matrix M/dt + A.  For n = 1..n_steps:
 *   b_n = H^T F (theta_{n-1} / dt + f_n)   (F: the load matrix of
 *         mg_assemble_rhs, i.e. the consistent mass, plus the SUPG load when
 *         stabilised), Dirichlet data g_n eliminated as in mg_assemble_rhs;
 *   theta_n = solution of (M/dt + A) theta_n = b_n, the Krylov method
 *         started from theta_{n-1} (warm start) and stopped at
 *         ||b_n - A theta_n|| <= rtol ||b_n,free||.
 * theta: device, n_nodes * nc doubles; in: theta_0, out: theta_{n_steps}
 * (all nodes; hanging values filled by H, Dirichlet values g_n).
 * f: device, n_steps blocks of n_nodes * nc doubles (nodal source values at
 * t_1, ..., t_n_steps, block n-1 for step n) or NULL (no source).
 * g: device, the same layout, nodal Dirichlet data (only its Dirichlet
 * entries are read) or NULL (homogeneous data).
 * steps: host array of n_steps mg_stats (per-step statistics) or NULL.
 * Returns MG_OK when every step converged; otherwise stops at the first step
 * that did not and returns its status (theta holds that step's iterate and
 * steps[] is filled up to it).  MG_ERR_INVALID if the problem has no mass
 * term.  Buffers for the step's source and right-hand side come from the
 * hierarchy's solve workspace; nothing is allocated. */
int mg_time_steps(mg_hier* h, double* theta, const double* f, const double* g, int n_steps, double rtol,
                  int max_it, int prec, mg_stats* steps);

/* Backward-Euler steps of the second-order-in-time problem d_t^2 u + A u = f
 * (Sec. 5.2: elastodynamics d_t^2 u - div sigma(u) = f), written as the
 * first-order system d_t u - v = 0, d_t v + A u = f in the unknowns (u, v).
 * Eliminating v_n = (u_n - u_{n-1})/dt from the step's coupled equations
 * leaves one system for u_n with the matrix M/dt^2 + A: the hierarchy's
 * problem must have mass = 1/dt^2 (checked to 1e-12 relative).  For
 * n = 1..n_steps:
 *   b_n = H^T F ((u_{n-1}/dt + v_{n-1})/dt + f_n), Dirichlet data g_n of u
 *         eliminated as in mg_assemble_rhs;
 *   u_n = solution of (M/dt^2 + A) u_n = b_n from u_{n-1} (warm start);
 *   v_n = (u_n - u_{n-1}) / dt on every dof (Dirichlet dofs included, so
 *         v follows the data's difference quotient there).
 * u, v: device, n_nodes * nc doubles each; in: u_0, v_0; out: u_n, v_n.
 * f, g: as in mg_time_steps (NULL: no source / homogeneous data).
 * Returns MG_OK when every step converged, else the first failing step's
 * status (u and v then hold that step's iterate).  Buffers come from the
 * hierarchy's solve workspace; nothing is allocated. */
int mg_time_steps2(mg_hier* h, double* u, double* v, const double* f, const double* g, int n_steps, double dt,
                   double rtol, int max_it, int prec, mg_stats* steps);

/* Krylov solve (CG / BiCGStab / GMRES per opts.krylov) preconditioned by one
 * V-cycle per iteration (Sec. 4.1.5).  b, x: device, n_nodes * nc doubles,
 * caller-owned.  x in: initial guess; out: solution on all nodes, hanging
 * values filled by H (Sec. 2.2), Dirichlet values taken from b.  Stops when
 * the true FP64 residual satisfies ||b - A x|| <= rtol ||b_free||; prec selects the
 * V-cycle precision (MG_FP64, or FP32 inside the FP64 Krylov loop).  Returns
 * MG_ERR_NOT_CONVERGED after max_it iterations (x and stats valid). */
int mg_solve(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats);
/* The same with HOST b and x: copies b to the device, solves, copies x back. */
int mg_solve_host(mg_hier* h, const double* b_host, double* x_host, double rtol, int max_it, int prec,
                  mg_stats* stats);

/* z = M^-1 r: one V-cycle with zero initial guess (Algorithm "Geometric
 * multigrid solver" started at the finest level).  r, z: device vectors of
 * n_dofs entries of type double (prec = MG_FP64) or float (mixed modes). */
int mg_vcycle(mg_hier* h, const void* r, void* z, int prec);

/* Single level operators, for tests and custom outer loops.  level 0 is the
 * coarsest.  Vectors are device arrays of double (MG_FP64) or float (mixed):
 *   MG_OP_MATVEC       out = A_l in
 *   MG_OP_SMOOTH       out = in + omega S_l (in2 - A_l in)     (one sweep)
 *   MG_OP_RESTRICT     out = R_l (in2 - A_l in)   (out on level l-1)
 *   MG_OP_PROLONG_ADD  out = in2 + P_l in         (in on level l-1)
 *   MG_OP_COARSE       out = A_0^-1 in            (level must be 0) */
enum { MG_OP_MATVEC = 0, MG_OP_SMOOTH = 1, MG_OP_RESTRICT = 2, MG_OP_PROLONG_ADD = 3, MG_OP_COARSE = 4 };
int mg_apply(mg_hier* h, int level, int op, const void* in, const void* in2, void* out, int prec);

/* Launch shape of the smallest levels: levels with at most tail_rows dofs
 * (and all coarser ones) run as one kernel on a cluster of `cluster` CTAs
 * (1..16; sizes above the portable 8 only where the GPU schedules such a
 * cluster of 1024-thread CTAs), or, for cluster == 0, on one CTA that first copies their vectors
 * and, coarsest first, as many of their matrices as fit into 226 KB of
 * shared memory (the threshold is lowered until the vectors fit), or, for
 * cluster = -2, -4, -8, -16 (scalar problems), cluster-resident on that many
 * CTAs: every level is cut into equal power-of-two row chunks, one per CTA;
 * each CTA keeps its chunks of the vectors and its rows of the level and
 * transfer matrices in shared memory and reads the other CTAs' vector entries
 * through distributed shared memory (MG_ERR_INVALID when the levels do not
 * fit 226 KB per CTA or the cluster is not schedulable).
 * tail_rows < 0: time V-cycles of precision prec over a set of thresholds and
 * launch shapes and keep the fastest (what opts.autotune does at setup).
 * Results are bitwise identical for every choice.  Errors: MG_ERR_INVALID
 * (cluster outside -16..16 or not schedulable, unknown precision), MG_ERR_OOM (the shared-memory
 * image of the tail could not be allocated). */
int mg_tune(mg_hier* h, int prec, int tail_rows, int cluster);

/* Allocation-free residual + restriction (no counterpart in the paper: it
 * exists for callers that cannot allocate device memory -- applications whose
 * device memory is owned up front by another allocator or a fixed pool, which
 * pass inputs and outputs but have nothing to give for temporaries, and
 * real-time loops that must not enter the CUDA allocator at all).
 *   d = R_l (b - A_l x) on level l >= 1, the same result as
 *   mg_apply(h, l, MG_OP_RESTRICT, x, b, d, prec).
 * x, b: device vectors of level l (n_l * nc entries); d: device vector of level
 * l-1; double for MG_FP64, float for MG_MIXED_FP32 and MG_MIXED_BF16 (the
 * latter reads the BF16-stored operator copy: store_bf16).  The residual is kept in a
 * fixed device array of 2^20 doubles (8 MiB) compiled into the library, so
 * the level may have at most 2^20 dofs in FP64 and 2^21 in FP32; larger levels
 * are refused with MG_ERR_INVALID before anything runs.  Every device that
 * loads the library holds that array until the process exits.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture.  All calls share the one array and
 * it keeps the last call's contents; calls that overlap on the GPU (other
 * threads, other contexts) race on it.  Runs on the context's stream and
 * returns after the work has finished; calls no allocator of any kind. */
int mg_restrict_static(mg_hier* h, int level, const void* x, const void* b, void* d, int prec);

/* Device time of one level operator: launches op (as mg_apply, on the
 * library's own level buffers, FP64 or FP32 per prec) `reps` times back to
 * back on the context's stream between two CUDA events and returns the mean
 * milliseconds per launch in *ms.  Two more ops time whole V-cycles started on
 * `level` (levels below it included, current tail configuration):
 * MG_TIME_VCYCLE launches their kernels directly, MG_TIME_VCYCLE_GRAPH
 * captures `reps` cycles into one CUDA graph and times its launch (the form
 * the solves use).  For measurement only. */
enum { MG_TIME_VCYCLE = 5, MG_TIME_VCYCLE_GRAPH = 6 };
int mg_time_op(mg_hier* h, int level, int op, int prec, int reps, double* ms);

/* Per-kernel device time of one solve.  Runs the solve of mg_solve (same
 * kernels in the same order, so x and stats are bitwise the same) but issues
 * one Krylov iteration at a time as a plain CUDA graph with a CUDA
 * event-record node before the first kernel and after every run of
 * consecutive launches of the same kernel on the same level (e.g. the
 * smoothing sweeps of one level, which follow each other as in mg_solve with
 * no event node between them): an interval runs from the end of the previous
 * run to the end of its own, so the intervals of an iteration add up to its
 * device time and a run's launches share one interval.  The graph
 * starts with an empty kernel (`k_prof_empty`, level -2, not part of the
 * solve and not counted in stats->launches) whose interval is the floor of
 * any interval: launch latency plus event overhead, which the chained kernels
 * of mg_solve partly hide.  Launches outside the iterations are bracketed by
 * two events on the context's stream.  Intervals are summed per
 * (kernel, level):
 *   kernel:   the kernel's name with its template arguments (truncated to 127
 *             characters, NUL-terminated);
 *   level:    the multigrid level whose V-cycle step launched it (restriction
 *             and the fused first sweep below count for the finer level; the
 *             small-level kernel for the top level it covers), -1 for Krylov
 *             and bookkeeping kernels, -2 for the empty kernel;
 *   launches, ms: launches and summed milliseconds.
 * Entries are sorted by ms, largest first; at most `cap` are written and
 * *n_entries receives the number of distinct pairs.  Launches beyond 8190 per
 * iteration are not timed.  For measurement: the solve itself runs slower
 * than mg_solve (host round trip per iteration, no overlap of neighbouring
 * kernels). */
typedef struct {
  char kernel[128];
  int level;
  int64_t launches;
  double ms;
} mg_prof_entry;
int mg_solve_profiled(mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec, mg_stats* stats,
                      mg_prof_entry* entries, int cap, int* n_entries);

/* New coefficients for a resident hierarchy (Algorithm "Nonstationary Linear
 * Problem": the matrices stay on the device; only their values change): the
 * host assembly runs again on the mesh the hierarchy was set up on, and the
 * level operators, smoother blocks and damping, Vanka matrices, coarse
 * inverse, load and lifting matrices and the small-level images are
 * rewritten in place (same device memory, same SELL layouts and tuning);
 * workspaces and serving reservations are kept, cached solve graphs are
 * rebuilt on their next use.  The kind, the Dirichlet faces and pin_origin
 * must stay the same (eps, beta, mu, lambda, supg_delta0, mass, nu, dt,
 * lps_alpha0 and conv may change).  A solve afterwards equals a solve on a
 * hierarchy set up with the new problem (same tuning) bit for bit.
 * MG_ERR_INVALID if a request of h is queued or running, or the new problem
 * changes the hierarchy's structure.  The call waits for synchronous solves
 * of h and for batched solves of the context; the caller must not submit
 * requests of h while it runs. */
int mg_update_problem(mg_hier* h, const mg_problem* problem);

/* Batched solve of many small problems in one kernel launch (the per-kernel
 * launch overhead that dominates small solves, Sec. 6.1, paid once for the
 * batch).  Problem k: hierarchy h[k], right-hand side b[k] (device, n_dofs
 * doubles, e.g. from mg_assemble_rhs) and x[k] (device, n_dofs doubles; in:
 * initial guess, out: solution on all nodes with hanging values filled, as
 * mg_solve).  A thread block takes the next problem of a work list (largest
 * first) and runs its whole solve: the Krylov method of mg_solve (CG or
 * BiCGStab; the same iteration formulas, FP64 vectors, restarts from the
 * true residual) with the V-cycle of every level in shared memory at
 * precision prec.  Dot products are summed in a different order than in
 * mg_solve, so iterates agree with it to rounding, not bit for bit.  The same
 * hierarchy may appear several times.  Every problem must pass
 * mg_batch_fits.  Scalar and 3-component problems may be mixed (one launch
 * each).  stats (optional): count entries, per problem; solve_ms is the whole
 * batch's device time.  Returns MG_OK when every problem converged, else the
 * status of the first one that did not (all stats are filled either way);
 * MG_ERR_INVALID (nothing run) when a problem does not fit.  count = 0: no-op.
 * Work vectors come from a context arena that grows to the largest batch. */
int mg_solve_batch(mg_ctx* ctx, int count, mg_hier* const* h, const double* const* b, double* const* x,
                   double rtol, int max_it, int prec, mg_stats* stats);
/* 1 when mg_solve_batch can solve h at precision prec (a CG or BiCGStab
 * problem without defect correction or Vanka levels, at most 16 levels, the
 * V-cycle vectors of all levels within 200 KiB of shared memory: about 90^2
 * nodes in 2D or 21^3 in 3D with an FP32 V-cycle), 0 otherwise (the reason in
 * mg_last_error), MG_ERR_INVALID for a NULL hierarchy. */
int mg_batch_fits(mg_hier* h, int prec);

/* Serving: continuous batching of solves on resident hierarchies.
 * mg_submit queues a solve of h (b, x device buffers, caller-owned, not to be
 * touched until mg_poll returns a final status) and returns at once with a
 * ticket; MG_ERR_ADMISSION if the request's workspace can never fit the
 * budget.  The context's scheduler thread admits queued requests as solve
 * slots and workspace memory free up and launches each admitted solve (one
 * CUDA graph) on a stream of its own, so the solves overlap on the device.
 * mg_poll returns MG_PENDING, or the final status with stats filled in.
 * mg_cancel removes a queued request (MG_ERR_CANCELLED on its next poll). */
int mg_submit(mg_ctx* ctx, mg_hier* h, const double* b, double* x, double rtol, int max_it, int prec,
              uint64_t* ticket);
int mg_poll(mg_ctx* ctx, uint64_t ticket, mg_stats* stats);
int mg_cancel(mg_ctx* ctx, uint64_t ticket);
/* Maximum number of solves the scheduler keeps in flight at once (default 16;
 * each runs on its own stream with its own workspace). */
int mg_serve_config(mg_ctx* ctx, int max_slots);
/* Batched launches in serving (off by default: max_batch = 0).  With
 * max_batch > 0, whenever at least min_batch queued requests of one
 * precision pass mg_batch_fits, up to max_batch of them (oldest first) go out
 * as one mg_solve_batch-style launch on a stream of its own, taking one
 * solve slot; fewer than min_batch take the graph path as without batching.
 * A batched request's result equals mg_solve_batch of that request alone bit
 * for bit (a block solves each problem; nothing depends on the batch's
 * other problems); it agrees with mg_solve to rounding only, so with
 * batching on, which of the two a request gets depends on the queue. */
int mg_serve_batching(mg_ctx* ctx, int max_batch, int min_batch);
/* Reserve `slots` solve slots of hierarchy h for serving: up to that many
 * workspaces are allocated now (through the context's allocator, on the
 * calling thread) and their solve graphs for precision prec are built, and
 * the scheduler never holds more than `slots` workspaces of h at once (a
 * request waits for a free one instead of allocating on the serving path).
 * Without a reservation the scheduler creates a workspace (cudaMalloc) and
 * builds its graph when a request finds none free.  MG_ERR_ADMISSION when the
 * slots do not fit the budget (the ones created stay reserved). */
int mg_serve_reserve(mg_ctx* ctx, mg_hier* h, int slots, int prec);
/* Kernels the library has enqueued on behalf of this hierarchy so far. */
int64_t mg_launch_count(const mg_hier* h);

/* ------------------------------------------------------------------------
 * Explicit Navier-Stokes pressure correction: the 3D driven cavity of
 * Sec. 5.3 (Algorithm "The fully discrete solution procedure for the
 * Navier-Stokes equations"), Re = 1/nu, on the box (0,1) x (0,1) x (0,2).
 * Pressure Q1 on the nx x ny x nz mesh Omega_h (cosine-graded node
 * coordinates x_i = (1 - cos(i pi/nx))/2, y alike, z_k = 1 - cos(k pi/nz)),
 * velocity Q1 on its equidistant refinement Omega_{h/2} (the
 * Q1-iso-Q2/Q1 pair); lumped masses; the convective term through the nodal
 * interpolant of u (x) u and C_d = (phi_j, d_d phi_i) (Eqs. "tp", "multC").
 * One step:
 *   1. u^m = u^{m-1} + k M^-1 (-nu K u^{m-1} + N(u^{m-1}) + C P (p + q))
 *      on interior velocity nodes; u = (0, lid, 0) on x = 1, 0 on the
 *      other walls;
 *   2. K_p q^m = -(1/k) d, d = ((div u^m, psi_j))_j: the pure Neumann
 *      pressure-increment problem, solved by the library's Krylov + geometric
 *      multigrid on the graded pressure mesh (warm start from q^{m-1}), then
 *      shifted to mean zero (sum_j m^p_j q_j = 0: the space Q of Sec. 5.3);
 *   3. p^m = p^{m-1} + q^m - nu d / m^p.
 * Node numbering: lexicographic, x fastest; velocity vectors node-major
 * (n_v x 3 doubles), pressure vectors n_p doubles; all on the device. */
typedef struct mg_ns mg_ns;
typedef struct {
  int nx, ny, nz;              /* pressure cells per axis (each >= 2)          */
  int graded;                  /* 1 (default): cosine-graded coordinates,
                                  0: equidistant                               */
  double re;                   /* Reynolds number (default 1000)               */
  double dt;                   /* time step k (default 1e-4)                   */
  double lid;                  /* lid speed (default 1)                        */
  int prec;                    /* precision of the pressure solve (default
                                  MG_MIXED_FP32: FP32 multigrid, FP64 Krylov)  */
  int krylov;                  /* Krylov method of the pressure solve (default
                                  MG_GMRES, as in Sec. 5.3)                    */
  double rtol;                 /* pressure solve tolerance (default 1e-8)      */
  int max_it;                  /* pressure solve iteration cap (default 200)   */
  int nu;                      /* smoothing sweeps before and after the coarse
                                  correction on every level (default 4: on the
                                  graded cavity the fastest of 2, 3, 4, 6, 8)  */
  int smoother;                /* mg_smoother of the pressure multigrid
                                  (default MG_SMOOTHER_JACOBI)                 */
} mg_ns_params;
typedef struct {
  int steps;                   /* steps run                                    */
  int status;                  /* MG_OK or the first failing solve's status    */
  int64_t iters;               /* Krylov iterations of all pressure solves     */
  int iters_max;               /* most iterations of one pressure solve        */
  double rel_res_max;          /* largest true relative residual               */
  double ms_momentum;          /* device time of Step 1 (interpolation of p+q
                                  and the fused momentum update)               */
  double ms_pres_rhs;          /* divergence and its restriction (Step 2 rhs)  */
  double ms_pres_solve;        /* the pressure-increment solves                */
  double ms_pres_up;           /* Step 3                                       */
  double ms_total;             /* wall time of mg_ns_steps                     */
} mg_ns_stats;
void mg_ns_default_params(mg_ns_params* p);
/* Builds the meshes, the velocity operators (per-axis 1D coefficients) and
 * the pressure hierarchy; velocity and pressure start at 0. */
int mg_ns_setup(mg_ctx* ctx, const mg_ns_params* params, mg_ns** out);
/* Velocity and pressure nodes per axis (n_v[d] = 2 n_p[d] - 1). */
int mg_ns_sizes(const mg_ns* ns, int n_vel[3], int n_pres[3]);
/* Copies the state in (dir = 0: u, p, q device buffers -> the solver) or
 * out (dir = 1); any pointer may be NULL (that field is skipped). */
int mg_ns_state(mg_ns* ns, double* u, double* p, double* q, int dir);
/* Runs n_steps steps on the context's stream; stats may be NULL.  Returns
 * MG_OK, or the status of the first pressure solve that failed (the state
 * after that step is kept). */
int mg_ns_steps(mg_ns* ns, int n_steps, mg_ns_stats* stats);
/* The pressure hierarchy (for inspection: mg_hier_info and so on). */
mg_hier* mg_ns_pressure_hierarchy(mg_ns* ns);
int mg_ns_free(mg_ns* ns);

#ifdef __cplusplus
}
#endif
#endif /* MG_GB300_H */
