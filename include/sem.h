/*
 * sem.h - C ABI of libsem: the matrix-free spectral-element elliptic solver
 * path of NekRS (Fischer et al., "NekRS, a GPU-accelerated spectral element
 * Navier-Stokes solver"), written for one NVIDIA GB300 (sm_103a).
 *
 * Problem (Section 2.3, eq. aip/A and the Helmholtz substep eq. ns_wrt2):
 *   find u with  A u = b,  A = R Q^T A_L Q R^T,
 *   A^e = D^T (h1 G^e) D + h2 B^e            (eq. Ae, eq. gij, eq. vBu)
 * on E hexahedral elements of order N with GLL points. Q is the Boolean
 * global-to-local map built from per-point global ids (eq. dssum and the
 * gs_setup interface of Section 3.2, "Parallel Communication"); R removes
 * Dirichlet rows (footnote below eq. dssum).
 *
 * Vectors. Every vector passed to the library is an L-vector: E blocks of
 * (N+1)^3 values, point (i,j,k) of element e at index
 * i + (N+1)*(j + (N+1)*(k + (N+1)*e)) (eq. uijk). A "continuous" L-vector
 * holds the same value in every local copy of a global node. Solver inputs
 * and outputs are continuous L-vectors.
 *
 * Memory and streams. Unless stated otherwise vector arguments are DEVICE
 * pointers owned by the caller (e.g. torch tensors), contiguous, 8-byte (FP64)
 * or 4-byte (FP32) aligned; the library keeps no reference to them after the
 * call returns. Mesh arrays in sem_setup are HOST pointers, copied. All
 * internal device memory (geometric factors, gather-scatter maps, multigrid
 * levels, solver workspace) is allocated in sem_setup and released by
 * sem_free; sem_ax, sem_gs and the level operators allocate nothing.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 * calls are asynchronous on it except where noted.
 *
 * Errors. Every int-returning call returns SEM_OK (0) or a negative code
 * below; sem_strerror gives a message and sem_last_error_detail the last
 * failure's context. No call exits, aborts or traps.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_OK 0
#define SEM_EINVAL (-1)      /* bad argument: N, E, id, pointer, level, flag */
#define SEM_ENOMEM (-2)      /* device allocation failed */
#define SEM_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define SEM_ENOTCONV (-4)    /* maxit reached before the tolerance; info is filled */
#define SEM_EBREAKDOWN (-5)  /* Krylov breakdown: p^T A p <= 0 or a NaN/Inf scalar */
#define SEM_EMESH (-6)       /* mesh rejected: non-positive Jacobian in some element */

#define SEM_MAX_N 11         /* orders 1..SEM_MAX_N are compiled */
#define SEM_MAX_LEVELS 6

/* Arithmetic of an operator application. */
#define SEM_FP64 0           /* FP64 geometric factors and arithmetic */
#define SEM_FP32 1           /* FP32 geometric factors and arithmetic */
#define SEM_BF16G 2          /* BF16 geometric factors, FP32 arithmetic */
#define SEM_FP64P 3          /* FP64 in and out, arithmetic in FP32 pairs (~48 bits; see sem_ax) */

/* sem_ax / sem_level_ax flags */
#define SEM_AX_LOCAL 0       /* w_L = A_L u_L only (no assembly) */
#define SEM_AX_ASSEMBLE 1    /* w_L = R QQ^T A_L u_L (gs_op(+) then Dirichlet mask) */
#define SEM_AX_PAIRS 2       /* evaluate A_L with FP32-pair arithmetic instead of FP64 instructions */

/* sem_gs flags */
#define SEM_GS_ADD 0         /* w_L <- QQ^T w_L */
#define SEM_GS_ADD_MASK 1    /* w_L <- R QQ^T w_L (zero every copy of a Dirichlet node) */

/* multigrid smoothers (sem_opts.smoother), Section 3.4 */
#define SEM_SMOOTH_JACOBI 0  /* Chebyshev-accelerated Jacobi (CHEBY-JAC) */
#define SEM_SMOOTH_ASM 1     /* Chebyshev-accelerated overlapping Schwarz with FDM local solves (CHEBY-ASM) */

/* execution of the coarse Jacobi-PCG (sem_opts.coarse_mode); the algorithm is the same in both.
 * Values 1 and 3 are not used (SEM_EINVAL). */
#define SEM_COARSE_AUTO 0     /* PIPE where it fits, else KERNELS */
#define SEM_COARSE_KERNELS 2  /* a few kernels per iteration, launched in batches (waits on the host:
                                 the preconditioner step is then launched directly, not from a graph) */
#define SEM_COARSE_PIPE 4     /* pipelined PCG on one sub-domain per SM in one cooperative launch; blocks
                                 exchange tagged words, no grid barrier; when it fits, else KERNELS */

/* sem_solve preconditioners and flags */
#define SEM_PC_JACOBI 0      /* Jacobi-PCG (the viscous-substep solver, Section 2.2) */
#define SEM_PC_PMG 1         /* flexible PCG + p-multigrid V-cycle with Chebyshev-Jacobi smoothing */
#define SEM_RHS_NODAL 0      /* f_L is a nodal function: b = R Q^T B_L f_L, replicated */
#define SEM_RHS_ASSEMBLED 1  /* f_L already holds the assembled b, replicated on copies */
#define SEM_X0_GIVEN 2       /* use u_L on entry as the initial guess (else x0 = 0) */
#define SEM_OUTER_PAIRS 4    /* the outer (FP64) operator uses the FP32-pair kernel (SEM_AX_PAIRS) */

/* precision bits in sem_opts.prec_copies: which preconditioner copies to build */
#define SEM_BUILD_FP32 1
#define SEM_BUILD_BF16G 2
#define SEM_BUILD_PAIRS 4    /* (hi, lo) FP32 split of the FP64 factors for SEM_FP64P / SEM_AX_PAIRS */

typedef struct sem_ctx sem_ctx;
typedef struct sem_proj sem_proj;    /* projection space of earlier solutions (sem_proj_create) */
typedef struct sem_halo sem_halo;    /* interface nodes shared with other ranks (sem_halo_create) */
#define SEM_PROJ_MAX 16              /* largest basis a projection space may keep */

/* Mesh description (all HOST pointers, copied during sem_setup). */
typedef struct {
  int32_t E;                 /* number of elements, >= 1 */
  int32_t N;                 /* polynomial order, 1..SEM_MAX_N */
  const double* x;           /* E*(N+1)^3 nodal coordinates at the GLL points (eq. xijk) */
  const double* y;
  const double* z;
  const int64_t* gid;        /* E*(N+1)^3 global node ids, >= 0; 0 marks a singleton (gs_setup) */
  const uint8_t* dirichlet;  /* E*(N+1)^3 flags, 1 = Dirichlet point; NULL = pure Neumann */
} sem_mesh;

/* Solver/multigrid options. sem_default_opts fills the defaults given here. */
typedef struct {
  int32_t mg_nlevels;        /* 0: schedule N, N/2, ..., 1; else the number of orders in mg_orders */
  int32_t mg_orders[SEM_MAX_LEVELS]; /* strictly decreasing, mg_orders[0] == N */
  int32_t cheb_degree;       /* Chebyshev-Jacobi steps per smoothing application (2) */
  double cheb_lmin_factor;   /* smoothed interval [lmin*est, lmax*est] (0.1) */
  double cheb_lmax_factor;   /* (1.1) */
  int32_t lanczos_steps;     /* Lanczos steps for the eigenvalue estimate of D^-1 A (10) */
  uint64_t lanczos_seed;     /* SplitMix64 seed of the Lanczos start vector (1) */
  double coarse_tol;         /* relative residual of the coarsest-level Jacobi-PCG (1e-1) */
  int32_t coarse_maxit;      /* iteration cap of the coarse solve (100) */
  int32_t prec_copies;       /* SEM_BUILD_* bits: factor copies to build (default: all three) */
  int32_t smoother;          /* SEM_SMOOTH_JACOBI (CHEBY-JAC, default) or SEM_SMOOTH_ASM (CHEBY-ASM) */
  int32_t coarse_mode;       /* how the order-1 coarse Jacobi-PCG runs: SEM_COARSE_* (default AUTO) */
  int64_t spin_limit;        /* SM clock cycles a device-side wait may spin before it gives up (2^31, about a
                                second at GB300's clock; >= 0). A wait that gives up makes the solve that
                                launched it return SEM_EBREAKDOWN (the coarse solve's exchange waits) or turns
                                the outputs of the waiting block into NaN (the FP32 operator's bulk-copy wait,
                                which then waits once more, with the default limit, for its copies to land) */
} sem_opts;

/* Coefficients h1 (diffusion) and h2 (mass) of A = D^T h1 G D + h2 B. */
typedef struct {
  double h1;
  double h2;
  const double* h1_L;        /* DEVICE, optional nodal h1 on the fine level (L-vector); NULL = scalar h1 */
} sem_coef;

/* Per-solve report. */
typedef struct {
  int32_t iters;             /* outer Krylov iterations */
  double relres;             /* final ||r|| / ||b|| (unique-node 2-norm) */
  double bnorm;              /* ||b|| */
  int32_t coarse_iters;      /* total coarse-level PCG iterations (PMG only) */
  int32_t nlevels;
  double lmax[SEM_MAX_LEVELS]; /* Lanczos estimates of lambda_max(D^-1 A) per smoothed level */
  double relres0;            /* sem_solve_proj: ||b - A xbar|| / ||b|| after projection; else -1 */
  int32_t proj_count;        /* sem_solve_proj: basis size after the solve; else 0 */
  int32_t graph_steps;       /* p-MG: preconditioner steps (V-cycle, beta, direction) replayed from a
                                CUDA graph in this solve; 0 where the context launches them directly */
} sem_info;

/* Per-level sizes. */
typedef struct {
  int32_t N, E;
  int64_t nL;                /* E*(N+1)^3 local points */
  int64_t nG;                /* unique global nodes */
  int64_t n_ids;             /* distinct nonzero global ids */
  int64_t n_idx;             /* local points with a nonzero id */
  int64_t n_seg;             /* gather-scatter segments (shared or Dirichlet nodes) */
  int64_t n_seg_idx;         /* local points in those segments */
} sem_level_desc;

void sem_default_opts(sem_opts* opts);
const char* sem_strerror(int code);
const char* sem_last_error_detail(void);

/* Build everything the path needs on the current CUDA device (Sections 2.3,
 * 3.2 and 3.4): GLL rule and D_hat (eq. dh) per order, geometric
 * factors G and B in FP64 (eq. grad, eq. gij, eq. vBu) plus FP32/BF16 copies,
 * the canonical gather-scatter maps (gs_setup), the Dirichlet mask and the
 * multigrid levels. Synchronous. Errors: SEM_EINVAL (bad N/E/pointer, negative
 * id), SEM_EMESH (J <= 0 somewhere), SEM_ENOMEM, SEM_ECUDA. On error *out is NULL. */
int sem_setup(const sem_mesh* mesh, const sem_opts* opts, sem_ctx** out);
void sem_free(sem_ctx* ctx);

int sem_num_levels(const sem_ctx* ctx);
int sem_level_info(const sem_ctx* ctx, int level, sem_level_desc* out);

/* w_L = A_L u_L (flags SEM_AX_LOCAL) or R QQ^T A_L u_L (SEM_AX_ASSEMBLE) on the
 * fine level in FP64, A^e = D^T h1 G D + h2 B (eq. Ae). With SEM_AX_PAIRS the
 * element operator runs in FP32-pair arithmetic (every value an unevaluated sum
 * of two floats, error-free TwoProduct/TwoSum; about 48 significant bits and
 * the FP32 exponent range, |values| within ~1e-30..1e30; a nodal h1_L is split into
 * pairs as it is read), which
 * GB300 executes far faster than FP64 instructions. The Dirichlet entries
 * of u_L are used as given; pass a masked u_L (zero at Dirichlet nodes, as every
 * solver vector is) to apply A = R Q^T A_L Q R^T. u_L and w_L must not alias.
 * Errors: SEM_EINVAL, SEM_ECUDA. */
int sem_ax(sem_ctx* ctx, const double* u_L, double* w_L, const sem_coef* coef, int flags, void* stream);

/* w_L <- QQ^T w_L (SEM_GS_ADD) or R QQ^T w_L (SEM_GS_ADD_MASK) on the fine
 * level in FP64: the gs_op(+) of Section 3.2. In place. */
int sem_gs(sem_ctx* ctx, double* w_L, int flags, void* stream);

/* Level operators (level 0 = fine, 1.. coarser). `prec` selects SEM_FP64
 * (double vectors) or SEM_FP32/SEM_BF16G (float vectors; the copy must have
 * been built). h1/h2 are scalars here. */
int sem_level_ax(sem_ctx* ctx, int level, int prec, const void* u_L, void* w_L, double h1, double h2,
                 int flags, void* stream);
int sem_level_gs(sem_ctx* ctx, int level, int prec, void* w_L, int flags, void* stream);

/* Inverse of the exact assembled diagonal of A on `level` (Jacobi, Section
 * 2.2), replicated on copies, 0 at Dirichlet nodes. FP64 output. */
int sem_level_dinv(sem_ctx* ctx, int level, double h1, double h2, double* dinv_L, void* stream);

/* Multigrid transfers between level `level` (fine) and `level`+1 (coarse)
 * (Section 3.4, orders N, N/2, ..., 1):
 *   prolong : x_f += R_f J e_c  (J: tensor interpolation, e_c continuous)
 *   restrict: r_c  = R_c QQ^T_c J^T (W_f r_f), W_f the counting weight 1/m. */
int sem_prolong_add(sem_ctx* ctx, int level, int prec, const void* ec_L, void* xf_L, void* stream);
int sem_restrict(sem_ctx* ctx, int level, int prec, const void* rf_L, void* rc_L, void* stream);

/* Set up the preconditioner for coefficients (h1, h2): Jacobi diagonals and,
 * on every smoothed level, an estimate of lambda_max of the smoothed operator:
 * the largest Ritz value of Lanczos on D^-1 A (CHEBY-JAC), or for CHEBY-ASM
 * the largest eigenvalue of the symmetric part of the Arnoldi Hessenberg
 * matrix of M_ASM A (an upper bound on the real parts of its Ritz values),
 * lanczos_steps steps from the seeded start vector, in FP64. Synchronous. */
int sem_precond_setup(sem_ctx* ctx, double h1, double h2, int prec, void* stream);
/* sem_precond_setup for A = D^T (h1 G) D + h2 B with a nodal h1 (h1_L: DEVICE, fine-level
 * L-vector, continuous): the fine values are carried to every coarser level by evaluating
 * each element's fine interpolant at the coarse GLL points (as the coarse coordinates are,
 * eq. xijk), and every level's operator, Jacobi diagonal and eigenvalue estimate use them
 * point by point; the order-1 coarse solve gets factors with G scaled by h1. CHEBY-JAC only
 * (the Schwarz local solves take a scalar h1: SEM_EINVAL). h1_L is copied; synchronous.
 * sem_solve with SEM_PC_PMG and coef->h1_L sets this up itself (again whenever the h1_L
 * pointer, h2 or the precision changes). */
int sem_precond_setup_nodal(sem_ctx* ctx, const double* h1_L, double h2, int prec, void* stream);
/* Chebyshev smoothing (Jacobi or Schwarz, per sem_opts.smoother) on `level` (needs sem_precond_setup): x <- S(b, x);
 * x_is_zero != 0 treats x as 0 on entry. Vectors in the V-cycle's precision. */
int sem_cheb_smooth(sem_ctx* ctx, int level, const void* b_L, void* x_L, int x_is_zero, void* stream);
/* Weighted overlapping additive Schwarz on `level` (Section 3.4): z = W sum_e
 * P_e^T F_e P_e r, masked. P_e gathers r on element e's (N+3)^3 extended box:
 * its own (N+1)^3 nodes and, across each face with a neighbour, the
 * neighbour's nodes one step inside from the shared face (the box's edge and
 * corner strips stay zero); P_e^T adds those slots back. F_e is the fast-
 * diagonalisation inverse of the separable operator h1 (B x B x A + B x A x B +
 * A x B x B) + h2 (B x B x B) of a box with the element's mean lengths, built
 * from the 1-D GLL stiffness A and mass B of the extended segment (the element
 * and same-length neighbours, Dirichlet one node beyond the overlap; a
 * Dirichlet boundary side drops its boundary node, a Neumann side keeps it).
 * W = 1 / (number of subdomain slots holding the node), 0 at Dirichlet nodes.
 * Needs 2 <= N on the level; the data are built on the first call (synchronous).
 * prec: SEM_FP64 (double vectors), SEM_FP32 (float vectors, FP32 local solves) or
 * SEM_BF16G (float vectors; the local solves on the TF32 tensor cores, operands
 * rounded to 11 significant bits, FP32 accumulation: the smoother of the BF16-G
 * V-cycle). */
int sem_asm_apply(sem_ctx* ctx, int level, int prec, const void* r_L, void* z_L, double h1, double h2,
                  void* stream);
/* z_L = M r_L: one V-cycle (needs sem_precond_setup), FP64 in and out. */
int sem_vcycle(sem_ctx* ctx, const double* r_L, double* z_L, void* stream);
/* Read back the lambda_max estimates (after sem_precond_setup). */
int sem_get_lmax(const sem_ctx* ctx, double* lmax, int n);

/* Solve A u = b to ||r||/||b|| <= tol with Jacobi-PCG (SEM_PC_JACOBI) or
 * flexible PCG preconditioned by the p-MG V-cycle (SEM_PC_PMG) whose
 * smoother and levels run in `prec` (SEM_FP64, SEM_FP32, SEM_BF16G); the
 * outer iteration, residual and dot products are always FP64. A nodal
 * coef->h1_L works with both (p-MG: CHEBY-JAC, see sem_precond_setup_nodal) and
 * with SEM_OUTER_PAIRS. f_L: nodal
 * function or assembled b (rhs_flags). u_L: solution (continuous L-vector).
 * Blocks until done (reads one residual norm per iteration). Errors:
 * SEM_ENOTCONV (info filled, u_L holds the last iterate), SEM_EBREAKDOWN,
 * SEM_EINVAL, SEM_ECUDA. info may be NULL. */
int sem_solve(sem_ctx* ctx, const double* f_L, const sem_coef* coef, double tol, int maxit, int precond,
              int prec, int rhs_flags, double* u_L, sem_info* info, void* stream);

/* ---- Projection of successive right-hand sides (Section 3.4, "projection-based
 * initial guesses"; Fischer, CMAME 163, 1998) ----
 * A space keeps up to max_vectors earlier solution directions x_i, A-orthonormal
 * (x_i^T A x_j = delta_ij, unique-node inner products), and b_i = A x_i beside
 * them, as FP64 fine-level L-vectors in DEVICE memory the space owns
 * (2 * max_vectors * nL * 8 bytes, allocated by sem_proj_create). A space
 * belongs to one context and one operator: a solve or update with other
 * coefficients (h1, h2, the h1_L pointer, SEM_OUTER_PAIRS) empties it first;
 * a caller that changes the values behind h1_L must call sem_proj_reset. */
int sem_proj_create(sem_ctx* ctx, int max_vectors, sem_proj** out);   /* 1 <= max_vectors <= SEM_PROJ_MAX */
void sem_proj_free(sem_proj* pj);
int sem_proj_reset(sem_proj* pj);                                     /* forget every vector */
int sem_proj_count(const sem_proj* pj);                               /* vectors held (or SEM_EINVAL) */
/* Read-only DEVICE pointers to x_i and b_i = A x_i, valid until the next update or free. */
int sem_proj_vectors(const sem_proj* pj, int i, const double** x_L, const double** ax_L);
/* xbar = sum_i (x_i, b) x_i, the A-norm-closest element of the span to A^-1 b,
 * and r0 = b - sum_i (x_i, b) b_i = b - A xbar (no operator application).
 * b_L: assembled, masked, replicated right-hand side. r0 may alias b; xbar may not.
 * Asynchronous on `stream`. */
int sem_proj_project(sem_proj* pj, const double* b_L, double* xbar_L, double* r0_L, void* stream);
/* Add one direction: v = dx_L, or x_L when the space is full (it then restarts
 * from x alone; x_L may be NULL, then dx_L is used). v is A-orthogonalised
 * against the space by classical Gram-Schmidt applied twice (one FP64
 * operator application A v, or the FP32-pair one with flags SEM_OUTER_PAIRS),
 * scaled to unit A-norm and kept unless orthogonalisation left less than
 * 1e-20 of its squared A-norm. *added (may be NULL) says whether it was kept.
 * Synchronous (reads two norms). */
int sem_proj_update(sem_proj* pj, const sem_coef* coef, int flags, const double* x_L, const double* dx_L,
                    int* added, void* stream);
/* sem_solve with the initial guess projected from the space: b is formed as in
 * sem_solve, xbar and r0 = b - A xbar come from sem_proj_project, the Krylov
 * solve finds dx from r0 with x0 = 0 and stops at ||r|| <= tol ||b|| (the
 * unprojected b), u_L = xbar + dx, and the space takes the new direction
 * (sem_proj_update). info->relres0 reports ||r0|| / ||b||. SEM_X0_GIVEN is
 * rejected (SEM_EINVAL). Errors as sem_solve. */
int sem_solve_proj(sem_ctx* ctx, sem_proj* pj, const double* f_L, const sem_coef* coef, double tol, int maxit,
                   int precond, int prec, int rhs_flags, double* u_L, sem_info* info, void* stream);

/* Dealiased advection operator (Section 2.1: the nonlinear term of eq. stdadv and the
 * hyperbolic substeps of eq. hyp; Section 3.3: evaluated on N_q^3 quadrature points):
 * for each of ncomp fields u, w = C(c) u with
 *   (C u)_i = sum_q w_q J_q phi_i(x_q) (c . grad u)(x_q),
 * q over nq^3 Gauss-Legendre points per element, nq = ceil(3 (N+1) / 2) (N = 7: 12),
 * on the fine level; element-local (SEM_ADV_LOCAL) or summed over the copies of each
 * node, Q Q^T C_L u (SEM_ADV_ASSEMBLE; no Dirichlet mask: the term is explicit).
 * c_L: 3 DEVICE L-vectors back to back ([3][nL], components x, y, z); u_L and w_L:
 * ncomp L-vectors back to back ([ncomp][nL]); w_L must not alias c_L or u_L.
 * prec SEM_FP64 (double vectors), SEM_FP64P (double vectors, the operator in FP32-pair
 * arithmetic: about 48 significant bits, FP32 exponent range; the pair copies of the
 * cubature factors, 9 nq^3 float2 per element, are built on the first such call) or SEM_FP32
 * (float vectors, FP32 arithmetic).
 * The cubature factors w J dr/dx at the Gauss points are built on the first call
 * (synchronous; 9 nq^3 values per element in FP64 and FP32). Compiled for 2 <= N <= 8. */
#define SEM_ADV_LOCAL 0
#define SEM_ADV_ASSEMBLE 1
int sem_advect(sem_ctx* ctx, int prec, const void* c_L, const void* u_L, void* w_L, int ncomp, int flags,
               void* stream);

/* The hyperbolic subproblem of the characteristics (semi-Lagrangian) scheme, Section 2.1
 * eq. hyp: w_t + c . grad w = 0 on [t0, t1], advanced in place by nsub classical RK4 steps of
 *   dw/dt = -M^-1 Q Q^T C(c(t)) w
 * with the dealiased operator of sem_advect and the assembled diagonal GLL mass M
 * (no boundary condition is imposed: winds tangent to the walls need none). The
 * wind is linear in time between c0 (at t0) and c1 (at t1); c1 = NULL freezes it at c0.
 * c0_L, c1_L: [3][nL]; w_L: ncomp L-vectors [ncomp][nL], continuous, updated in place
 * (must not alias the winds). prec SEM_FP64 / SEM_FP64P (the operator in FP32 pairs, the
 * Runge-Kutta stages in FP64) / SEM_FP32. Workspace (3 ncomp + 3
 * L-vectors) and the inverse mass are allocated on first use and kept. */
int sem_char_advance(sem_ctx* ctx, int prec, const void* c0_L, const void* c1_L, void* w_L, int ncomp, double t0,
                     double t1, int nsub, void* stream);

/* Adjoint gradient with respect to nodal h1 (no counterpart in the paper's
 * solver; built on eq. Ae): g_L = -sum_{m,m'} (D_m lam)(G_mm')(D_m' u) at every
 * local point, with G excluding h1. For L = loss(u(h1)), A lam = dL/du gives
 * dL/dh1 = g. flags 0: per-point contributions (the gradient with respect to
 * an L-vector h1); SEM_GRAD_SUM: summed over the copies of each node (QQ^T),
 * the gradient with respect to the unique nodal values, replicated. */
#define SEM_GRAD_SUM 1
int sem_grad_h1(sem_ctx* ctx, const double* u_L, const double* lam_L, double* g_L, int flags, void* stream);

/* b_L = R QQ^T (B_L f_L): the GLL inner products b_i = (phi_i, f)_N (eq. qN-vBu). */
int sem_rhs(sem_ctx* ctx, const double* f_L, double* b_L, void* stream);
/* out_L = B_L f_L, the local diagonal mass (eq. vBu), no assembly. */
int sem_mass_local(sem_ctx* ctx, const double* f_L, double* out_L, void* stream);

/* Unique-node dot product (a, b) of two continuous FP64 L-vectors: the sum
 * over one owner copy of each non-Dirichlet node. Result in *out (HOST). Synchronous. */
int sem_dot(sem_ctx* ctx, const double* a_L, const double* b_L, double* out, void* stream);

/* Dot product sum_l mask_l a_l b_l of two FP64 device vectors (mask: DEVICE
 * uint8 flags, NULL = all ones) written to *out (DEVICE), that allocates no
 * memory and needs no context. The paper has no counterpart: this is for
 * callers that cannot allocate device memory (a host framework that owns a
 * fixed device budget and passes only pointers into it, a latency-critical
 * loop that must not meet cudaMalloc's device-wide synchronisation, a caller
 * holding no sem_ctx). Its scratch is a file-scope static device array of
 * 64 KiB + 4 bytes per device, held until the process exits. n may be at most
 * 67,108,864; larger n returns SEM_EINVAL without launching anything. The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and must come before any stream capture on that device. Calls share the
 * array: calls that overlap on the GPU (concurrent streams) race and must be
 * serialised by the caller. Asynchronous on `stream`. To reproduce sem_dot's
 * unique-node product pass the owner mask: 1 where label[l] == l and dmask[l] == 0
 * (sem_get_maps). */
int sem_dot_static(const double* a, const double* b, const uint8_t* mask, int64_t n, double* out, void* stream);

/* ---- Element partitioning across GPUs and the interface exchange (Section 3.1,
 * "Domain Partitioning": elements are split among ranks; Section 3.2, "Parallel
 * Communication": the gather-scatter becomes each rank's own QQ^T plus the exchange
 * of partial sums at the nodes shared with other ranks, and the elements on the
 * partition boundary are computed first so that the exchange overlaps the others).
 * A rank builds a context from its own elements (global ids kept); the sum over
 * ranks of the halo buffers is the caller's collective (e.g. an all-reduce). ---- */

/* Recursive coordinate bisection of E element centroids (cx, cy, cz: HOST, E each)
 * into nparts parts of sizes within one of each other: part[e] in 0..nparts-1 (HOST,
 * caller-allocated). Each bisection splits the longest extent of the part's centroids
 * at the median (ties by element index). No GPU. Errors: SEM_EINVAL (1 <= nparts <= E). */
int sem_partition_rcb(int32_t E, const double* cx, const double* cy, const double* cz, int32_t nparts,
                      int32_t* part);
/* w_L = A_L u_L on elements e0 .. e1-1 of the fine level only (eq. Ae; other elements'
 * entries of w_L are not touched). u_L, w_L and coef->h1_L are whole L-vectors. flags 0
 * (FP64) or SEM_AX_PAIRS (FP32-pair arithmetic). Errors: SEM_EINVAL. */
int sem_ax_elements(sem_ctx* ctx, int32_t e0, int32_t e1, const double* u_L, double* w_L, const sem_coef* coef,
                    int flags, void* stream);
/* Interface of this rank: n global ids (HOST, each held by this context's fine level)
 * and for each its position pos[i] in an exchange buffer of nbuf doubles (HOST arrays,
 * copied). Synchronous. Errors: SEM_EINVAL (an id not held here, a position outside
 * 0..nbuf-1), SEM_ENOMEM, SEM_ECUDA. */
int sem_halo_create(sem_ctx* ctx, int64_t n, const int64_t* gid, const int64_t* pos, int64_t nbuf,
                    sem_halo** out);
void sem_halo_free(sem_halo* halo);
/* buf (DEVICE, nbuf doubles) <- 0, then buf[pos[i]] = the sum of this rank's local
 * copies of interface node i in w_L (ascending local index). Asynchronous. */
int sem_halo_gather(sem_halo* halo, const double* w_L, double* buf, void* stream);
/* every local copy of interface node i in w_L <- buf[pos[i]] (with SEM_GS_ADD_MASK: 0 at
 * Dirichlet nodes). With buf the sum over ranks of the gathered buffers and w_L this
 * rank's own QQ^T of A_L u, this completes the gather-scatter of the whole mesh.
 * Asynchronous. */
int sem_halo_scatter(sem_halo* halo, const double* buf, double* w_L, int flags, void* stream);

/* Arithmetic peaks of the current device, measured with plain kernels and CUDA
 * events on the legacy default stream (the paper has no counterpart; the
 * library's roofline reports divide by these). out[0]: FP64 FMA, out[1]: FP64
 * mma.sync (m16n8k8, changing operands), out[2]: FP32 FMA, all in TFLOP/s
 * (2 flops per multiply-add). Allocates and frees a scratch of 8 blocks x 256
 * doubles per SM; takes about 0.1 s. Synchronous. Errors: SEM_EINVAL (NULL),
 * SEM_ENOMEM, SEM_ECUDA. */
int sem_measure_peaks(double* out);

/* ---- read-back of setup products, for validation (HOST outputs, synchronous) ---- */
/* Canonical gather-scatter maps of `level` (any pointer may be NULL):
 * ids[n_ids]: distinct nonzero global ids ascending; off[n_ids+1]: CSR offsets;
 * idx[n_idx]: local indices sorted by (id, local index); mult[nL]: multiplicity;
 * node[nL]: unique-node number (ids in order, then singletons in local order);
 * label[nL]: smallest local index of the point's node; dmask[nL]: 1 at Dirichlet nodes. */
int sem_get_maps(const sem_ctx* ctx, int level, int64_t* ids, int64_t* off, int32_t* idx, int32_t* mult,
                 int64_t* node, int64_t* label, uint8_t* dmask);
/* FP64 geometric factors [E][7][(N+1)^3] (G11,G12,G13,G22,G23,G33,B) of `level`. */
int sem_get_geom(const sem_ctx* ctx, int level, double* G);
/* BF16 / FP32 copies as raw bits (uint16 / uint32 per value, same layout). */
int sem_get_geom_lowp(const sem_ctx* ctx, int level, int prec, void* G);
/* Nodal coordinates and global ids of `level` (coarse levels are derived). */
int sem_get_coords(const sem_ctx* ctx, int level, double* x, double* y, double* z, int64_t* gid);
/* GLL nodes, weights and D_hat (row-major, D[a*(N+1)+b] = h_b'(xi_a)) for order N. */
int sem_gll(int N, double* xi, double* rho, double* D);

/* Sub-domain partition of an order-1 level as the pipelined coarse solve (SEM_COARSE_PIPE)
 * builds it: HOST-only (no GPU), for inspection and tests. Direct-stiffness summation
 * QQ^T (Section 3.2) becomes, per sub-domain, a sum over every copy of each node it holds.
 * In: E elements of 8 points (point l = 8e + i + 2j + 4k); node[8E] the unique node of each
 * point, 0 <= node < nG; dmask[8E] 1 at Dirichlet nodes; owner[8E] 1 at the copy of each
 * non-Dirichlet node that counts in dot products; x, y, z[8E] coordinates (element centroids
 * are split by recursive coordinate bisection); nblocks sub-domains, 1 <= nblocks <= E.
 * Out, caller-allocated: el_off[nblocks+1] and el[E]: elements grouped by sub-domain, ascending
 * within one. p2n[8E]: for the points in el order, the point's sub-domain node, with bit 31 set
 * when that node has copies in other sub-domains. nd_off[nblocks+1]: offsets of each
 * sub-domain's nodes, numbered by first appearance. nd_src[cap_nodes]: one local point of each
 * node. nd_fl[cap_nodes]: bit 0 set where the sub-domain holds the owner copy, bit 1 at
 * Dirichlet nodes. cp_off[cap_nodes+1] and cp[cap_copies]: every copy of each node in
 * ascending local index; an entry >= 0 is a point of the sub-domain (offset from its first
 * point in el order), an entry < 0 is -(local point + 1) in another sub-domain.
 * counts[5]: nodes, copies, then the largest sub-domain's elements, nodes and copies.
 * Errors: SEM_EINVAL for a NULL pointer, bad sizes or node numbers, or capacities that are
 * too small (counts is filled in that case). */
int sem_coarse_partition(int32_t E, int64_t nG, const int32_t* node, const uint8_t* dmask,
                         const uint8_t* owner, const double* x, const double* y, const double* z,
                         int32_t nblocks, int64_t cap_nodes, int64_t cap_copies, int32_t* el_off,
                         int32_t* el, int32_t* p2n, int32_t* nd_off, int32_t* nd_src, uint8_t* nd_fl,
                         int32_t* cp_off, int32_t* cp, int64_t* counts);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H */
