/*
 * thm.h -- C ABI of the GB300 DDM-GMRES solver for the Nedelec-discretised
 * time-harmonic Maxwell (THM) system
 *
 *     curl(mu^{-1} curl E) - omega^2 E = 0                  in Omega
 *     mu^{-1} gamma^t(curl E) - i kappa omega gamma^T(E) = 0 on Gamma^inf
 *     gamma^T(E) = gamma^T(E^inc)                            on Gamma^inc
 *
 * (Beuchler, Kinnewig, Wick, "Parallel domain decomposition solvers for the
 * time harmonic Maxwell equations", Section 2, Eq. 1), solved by the
 * non-overlapping optimized-Schwarz DDM with impedance transmission
 * (Section 3.1, Eqs. 4-6, S = identity), GMRES on the interface system (Eq. 8)
 * and block-preconditioned GMRES inside every subdomain (Section 3.2, Eq. 7).
 *
 * Conventions for every call
 *  - Return value: THM_OK (0) or a negative THM_E* code; thm_last_error()
 *    then returns a thread-local message.  No call aborts the process.
 *  - Complex vectors are interleaved (re, im) pairs of doubles.
 *  - "host" pointers are read/written with plain CPU loads; "device" pointers
 *    must be CUDA device (or managed) memory of the current device.
 *  - The caller owns every buffer it passes in; the library only reads or
 *    writes it during the call.  Handles (thm_mesh*, thm_sys*) and all their
 *    workspace are owned by the library and freed by thm_*_destroy.
 *  - Work is issued on the stream given to thm_assemble (0 = legacy default);
 *    calls that return results to host memory synchronise that stream.
 *  - Every step of the solve runs in this library's CUDA kernels for sm_103a;
 *    there is no CPU fallback.  A missing or unusable GPU is THM_ECUDA.
 */
#ifndef THM_H
#define THM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THM_OK           0
#define THM_EINVAL      -1   /* bad argument, shape, tag or unsupported combination */
#define THM_ENOCONV     -2   /* iteration limit hit: u holds the last iterate, stats filled */
#define THM_EBREAKDOWN  -3   /* Krylov breakdown / non-finite value */
#define THM_ESINGULAR   -4   /* zero pivot while factorising a block of P_i (Eq. 7) */
#define THM_ETIMEOUT    -5   /* a bounded device-side wait gave up */
#define THM_ECUDA       -6   /* CUDA runtime error (message has the CUDA string) */
#define THM_ENOMEM      -7   /* device allocation failed */

typedef struct thm_mesh thm_mesh;   /* opaque: numbering + subdomain structure */
typedef struct thm_sys thm_sys;     /* opaque: assembled operators + preconditioner */

/* Boundary face tags. */
#define THM_TAG_IMPEDANCE 0   /* Gamma^inf: impedance condition of Eq. 1 */
#define THM_TAG_DIRICHLET 1   /* Gamma^inc: gamma^T E = gamma^T E^inc, imposed strongly */
#define THM_TAG_NATURAL   2   /* no boundary term (homogeneous natural condition) */

/* Precision modes of thm_ddm_solve. */
#define THM_MODE_FP64  0      /* every kernel in FP64 */
#define THM_MODE_MIXED 1      /* FP32 operator/preconditioner/inner Krylov, FP64 outer
                                 GMRES, Givens, true residual and refinement */

/*
 * thm_mesh -- build the DOF numbering, orientation signs and the subdomain /
 * interface structure of a mesh of axis-aligned quads (dim 2) or hexes (dim 3).
 * Section 2 (the space N_h^p) and Section 3.1 (partition into Omega_i, Sigma_ij).
 *
 *  dim          2 or 3;  order 1 (dim 2 or 3) or 2 (dim 2 only).
 *  coords       host double [n_vert][dim].
 *  cells        host int64  [n_cell][4 | 8]: corner vertex ids in tensor order
 *               (2-D: 00,10,01,11; 3-D: v = i + 2j + 4k); any of the square's
 *               (cube's) symmetric re-listings is accepted.
 *  cell_sub     host int32  [n_cell]: subdomain id of each cell, 0..n_sub-1,
 *               every id used.
 *  bfaces       host int64  [n_bface][2 | 4]: boundary faces (2-D: the edge's two
 *               vertices; 3-D: the quad's four vertices in tensor order).
 *  btag         host uint8  [n_bface]: THM_TAG_*.
 *  max_block    largest block of the level-block-tridiagonal factorisation of
 *               P_i (<= 0: library default); 0 < max_block sets the trade-off
 *               between sequential depth and bytes of the preconditioner.
 *
 *  Numbering (bit-exact contract): edges are the distinct vertex pairs of the
 *  cells' local edges, numbered in lexicographic order of (min id, max id);
 *  order 1: DOF = edge id; order 2: Whitney 2e, gradient 2e+1, cell bubble k
 *  of cell c -> 2E + 4c + k.  A cell's local edge (a->b) has sign +1 iff
 *  id(a) < id(b); gradient and bubble DOFs have sign +1.
 *  Errors: THM_EINVAL for bad sizes/tags/ids or non-axis-aligned cells.
 */
int thm_mesh_create(thm_mesh** out, int dim, int order,
                    int64_t n_vert, const double* coords,
                    int64_t n_cell, const int64_t* cells, const int32_t* cell_sub,
                    int64_t n_bface, const int64_t* bfaces, const uint8_t* btag,
                    int max_block);

/*
 * thm_mesh_info -- sizes, and optionally the per-cell DOF ids and signs.
 *  n_dof, n_edge, n_sub, dofs_per_cell: host outputs (any may be NULL).
 *  dof_of_cell  host int64 [n_cell][dofs_per_cell] or NULL.
 *  sign_of_cell host int8  [n_cell][dofs_per_cell] or NULL.
 * The DOF map and signs are computed by a device kernel at thm_mesh_create.
 */
int thm_mesh_info(const thm_mesh* m, int64_t* n_dof, int64_t* n_edge, int32_t* n_sub,
                  int32_t* dofs_per_cell, int64_t* dof_of_cell, int8_t* sign_of_cell);

void thm_mesh_destroy(thm_mesh* m);

/*
 * thm_assemble -- assemble the subdomain operators and factorise the block
 * preconditioner.  Section 2, the integrals (A), (M), (B) and Eq. 3; Section
 * 3.1, Eq. 5 (transmission term on Sigma_ij); Section 3.2, Eq. 7.
 *
 *  Per subdomain i:  T_i = P_i + i B_i,  P_i = mu^{-1} A_i - omega^2 M_i (real),
 *  B_i = kappa omega (M_{Gamma^inf,i} + sum_j M_{Sigma_ij})  (tangential face
 *  masses), on the free DOFs of Omega_i.  P_i is factorised once here and
 *  reused by every solve (Section 3.2: the expensive preconditioner set-up is
 *  reused across DDM iterations).
 *
 *  mu_inv       double [n_cell] (host or device, see mu_inv_on_device).
 *  omega>0, kappa>=0.
 *  pol          host double [dim][2] complex polarisation, dir host double[dim]:
 *               E^inc(x) = pol * exp(-i omega dir.x) (time factor e^{i omega t}).
 *               The Dirichlet DOFs get the tangential moments of E^inc.
 *  stream       cudaStream_t (as void*) for all work of this system.
 *  Errors: THM_EINVAL, THM_ESINGULAR (a block of P_i is singular: omega^2 is an
 *  eigenvalue of the subdomain's natural-boundary problem), THM_ENOMEM, THM_ECUDA.
 */
int thm_assemble(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                 double omega, double kappa, const double* pol, const double* dir,
                 void* stream);

/*
 * thm_mesh_dirichlet_dofs -- the Dirichlet DOFs of the mesh (those on
 * THM_TAG_DIRICHLET faces, Gamma^inc of Eq. 1), in increasing global order:
 * the order in which thm_assemble_dirichlet takes their values.
 *  n_dir  host output (may be NULL);  ids  host int64 [n_dir] or NULL.
 */
int thm_mesh_dirichlet_dofs(const thm_mesh* m, int64_t* n_dir, int64_t* ids);

/*
 * thm_assemble_dirichlet -- thm_assemble with the Dirichlet data of Eq. 1
 * (gamma^T E = gamma^T E^inc on Gamma^inc) given by the caller instead of a
 * plane wave: the values of the Dirichlet DOFs themselves (order 1: the
 * tangential moment of E^inc along the edge; order 2 also the second edge
 * moment; the same DOF definition the plane-wave path evaluates).
 *
 *  u_dir            complex double [n_dir] (interleaved re, im) in the order
 *                   of thm_mesh_dirichlet_dofs; host or device
 *                   (u_dir_on_device).  May be NULL only when n_dir = 0.
 *  Other arguments as in thm_assemble.  A single problem only (a batch mesh
 *  gets THM_EINVAL).  The values are copied during the call.  The adjoint of
 *  such a system treats the data as independent of omega and kappa.
 *  Errors: as thm_assemble; THM_EINVAL for a non-finite host value.
 */
int thm_assemble_dirichlet(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                           double omega, double kappa, const double* u_dir, int u_dir_on_device, void* stream);

/*
 * thm_assemble_ex -- thm_assemble / thm_assemble_batch / thm_assemble_dirichlet
 * with the options below (opts may be NULL: all defaults).
 *
 *  omega   host double [n_prob] (one value unless the mesh is a batch).
 *  pol, dir  the plane wave, as in thm_assemble; ignored when opts->u_dir is set.
 *
 *  eps     relative permittivity per cell (double [n_cell], > 0, host or
 *          device per eps_on_device): the mass term becomes omega^2 M_eps,
 *          M_eps = sum_c eps_c M_c, i.e. curl(mu^{-1} curl E) - omega^2 eps E = 0.
 *          Eq. 1 is printed with eps = 1 (NULL); the paper's Example 1 (Section 4)
 *          describes its block by a refractive index n, eps = n^2.  The Gamma^inf
 *          and Sigma coefficients stay kappa omega; the adjoint differentiates
 *          the weighted mass term.
 *  trans_re, trans_im
 *          transmission coefficient on Sigma_ij in units of kappa omega; both 0
 *          means (0, 1): i kappa omega, the impedance condition of Eq. 5 with
 *          S = 1 (Section 3.1).  Subdomain i then solves
 *          (K_i + c kappa omega M_Sigma) u_i = s_i + G and the exchange is
 *          G_{i<-j} = -G_{j<-i} + 2 c kappa omega M_Sigma u_j, c = trans_re + i trans_im;
 *          the fixed point is the monolithic solution for every c != 0.  A large
 *          real c is the penalty form of the Dirichlet-like classical Schwarz
 *          interface condition that Section 3.1 says cannot be expected to
 *          converge for large omega.  The block preconditioner of Eq. 7
 *          factorises P_i = Re(T_i), which then includes trans_re kappa omega M_Sigma.
 *  u_dir, u_dir_on_device
 *          caller-given Dirichlet values as in thm_assemble_dirichlet (single
 *          problems only), or NULL for the plane wave (pol, dir).
 *  Errors: as thm_assemble.
 */
typedef struct thm_assemble_opts {
    const double* eps;
    int eps_on_device;
    double trans_re, trans_im;
    const double* u_dir;
    int u_dir_on_device;
} thm_assemble_opts;

int thm_assemble_ex(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                    const double* omega, double kappa, const double* pol, const double* dir,
                    const thm_assemble_opts* opts, void* stream);

/*
 * Batches of independent problems (the paper solves one problem at a time;
 * this is the batched form of the same solve).  A batch mesh is the disjoint
 * union of the problems' meshes, built with thm_mesh_create: subdomain ids are
 * unique across the batch, each problem's subdomains form a contiguous,
 * increasing range of ids and its vertices a contiguous range of vertex ids
 * (so its global DOFs are a contiguous range).
 *
 * thm_mesh_set_problems -- declare the batch: sub_problem (host int32
 *   [n_sub]) gives each subdomain's problem in [0, n_prob), non-decreasing.
 *   Must come before the first thm_assemble on the mesh.  Errors: THM_EINVAL
 *   when the ranges are not contiguous, problems share a DOF or an interface.
 *
 * thm_assemble_batch -- thm_assemble with one omega per problem (host double
 *   [n_prob]); mu_inv, kappa, pol and dir as in thm_assemble (shared).  A batch
 *   mesh must be assembled with this call.
 *
 * thm_ddm_solve on a batch system runs every problem's DDM together: one set
 * of kernel launches per step covers all subdomains of all problems, the
 * interface GMRES keeps one Krylov segment (Hessenberg, Givens, convergence
 * flag) per problem, and the refinement stops when every problem's relative
 * FP64 residual is <= rtol (stats->rel_residual is the largest).  The adjoint
 * takes single problems only.
 */
int thm_mesh_set_problems(thm_mesh* m, int32_t n_prob, const int32_t* sub_problem);
int thm_assemble_batch(thm_sys** out, const thm_mesh* m, const double* mu_inv, int mu_inv_on_device,
                       const double* omega, double kappa, const double* pol, const double* dir, void* stream);

typedef struct thm_solve_opts {
    int    mode;           /* THM_MODE_FP64 or THM_MODE_MIXED */
    double rtol;           /* target ||f - K u|| / ||f|| (global, FP64), e.g. 1e-8 */
    int    inner_restart;  /* subdomain GMRES restart length m (<=0: 120) */
    double inner_tol;      /* subdomain solve relative tolerance on the FP64 residual (<=0: 1e-11);
                              mixed mode refines FP32 GMRES cycles (each to 1e-5) on the FP64
                              residual; a subdomain also stops when a cycle fails to halve its
                              residual (the attainable accuracy is reached) */
    int    inner_maxit;    /* Arnoldi steps per subdomain solve (<=0: 2000) */
    int    outer_restart;  /* interface GMRES restart (<=0: 600) */
    double outer_tol;      /* interface GMRES relative tolerance (<=0: 1e-9) */
    int    outer_maxit;    /* (<=0: 2000) */
    int    max_refine;     /* iterative-refinement steps (<=0: 6) */
    int    relax;          /* 1: inexact-Krylov relaxation of the subdomain tolerance as the
                              interface residual falls (clamp(1e-2 * outer_tol/||r_k||,
                              inner_tol, 1e-6)); the refinement on the FP64 residual still
                              decides convergence.  0: fixed inner_tol */
    int    outer_method;   /* THM_OUTER_GMRES (0): GMRES on (I - A) g = b (Eq. 8);
                              THM_OUTER_JACOBI (1): the fixed-point iteration
                              g <- A g + b of the same map, stopped when
                              ||(I - A) g - b|| <= outer_tol ||b|| (norms over
                              the whole interface vector, also for a batch) */
    int    precond;        /* preconditioner of the subdomain GMRES (Section 3.2):
                              THM_PRECOND_BLOCKDIAG (0): blockdiag(P_i, P_i)^{-1} of
                              Eq. 7 on the real/imaginary splitting (default);
                              THM_PRECOND_FULL (1): the exact inverse of the full
                              2x2 block operator [[P_i, -B_i], [B_i, P_i]] (the real
                              form of T_i, Eq. 3), i.e. T_i^{-1} from complex
                              factors: GMRES then needs one step per solve (FP64)
                              for twice the factor memory.  2-D meshes only. */
} thm_solve_opts;

#define THM_OUTER_GMRES 0
#define THM_OUTER_JACOBI 1
#define THM_PRECOND_BLOCKDIAG 0
#define THM_PRECOND_FULL 1

typedef struct thm_stats {
    int    outer_iters;        /* interface GMRES iterations, summed over refinement */
    int    sweeps;             /* DDM sweeps (each: all subdomain solves + exchange) */
    int    refine_steps;       /* DDM solves performed */
    int64_t inner_iters;       /* sum over sweeps and subdomains of inner GMRES steps */
    int64_t dof_iters;         /* sum over the same of n_i * inner steps */
    int    max_inner_iters;    /* largest single subdomain solve */
    double rel_residual;       /* final ||f - K u|| / ||f|| in FP64 */
    double seconds;            /* wall time of thm_ddm_solve */
} thm_stats;

/*
 * thm_ddm_solve -- solve for the discrete field.  Section 3.1 (Eqs. 4-6, the
 * interface system Eq. 8 by GMRES), Section 3.2 (inner GMRES with Eq. 7).
 * Each DDM solve is wrapped in iterative refinement on the FP64 true residual
 * f - K u, assembled from the subdomain pieces, until rel_residual <= rtol.
 *
 *  u      complex double [n_dof] (device), caller-owned; on return holds all
 *         DOFs (Dirichlet DOFs = the tangential moments of E^inc).
 *  stats  host, may be NULL.
 *  Errors: THM_ENOCONV (u holds the last iterate), THM_EBREAKDOWN, THM_ECUDA.
 */
int thm_ddm_solve(thm_sys* s, const thm_solve_opts* opts, double* u, thm_stats* stats);

/*
 * thm_ddm_solve_host -- as thm_ddm_solve, but u is a host buffer
 * (complex double [n_dof]); the device->host copy is part of the call.
 */
int thm_ddm_solve_host(thm_sys* s, const thm_solve_opts* opts, double* u_host, thm_stats* stats);

/*
 * thm_adjoint -- gradient of a real loss L(u) through the solve (no counterpart
 * in the paper).  Given dLdu_conj = dL/d(conj u) as a complex device vector
 * [n_dof] (for L = u^H M_R u this is M_R u), solves K^T lambda = dLdu_conj on
 * the free DOFs (K^T = K, the same DDM-GMRES solve) and returns
 *   grad_mu_inv[c] = -2 Re(lambda_c^T A_c u_c)           (device double [n_cell])
 *   grad_omega     = -2 Re(lambda^T [(dK/domega) u + K du_D/domega])
 *                    + 2 Re(a^T du_D/domega)              (host double)
 *   grad_kappa     = -2 Re(lambda^T (i omega M_Gamma) u)     (host double, or
 *                    NULL when not wanted)
 * with dK/domega = -2 omega M + i kappa M_Gamma, a = dLdu_conj and du_D/domega
 * the derivative of the Dirichlet moments (0 for caller-given Dirichlet data,
 * thm_assemble_dirichlet).  Since s K(mu^{-1}, omega, kappa) = K(s mu^{-1},
 * sqrt(s) omega, sqrt(s) kappa), the three gradients satisfy
 * sum_c mu^{-1}_c grad_mu_inv[c] + (omega/2) grad_omega + (kappa/2) grad_kappa
 * = 0 whenever the Dirichlet data do not depend on omega.  2-D (orders 1, 2)
 * and 3-D.  u is the forward solution (device complex [n_dof]); lambda is
 * zero on Dirichlet DOFs.
 */
int thm_adjoint(thm_sys* s, const thm_solve_opts* opts, const double* u, const double* dLdu_conj,
                double* grad_mu_inv, double* grad_omega, double* grad_kappa, thm_stats* stats);

void thm_sys_destroy(thm_sys* s);

const char* thm_last_error(void);

/* ------------------------------------------------------------------------
 * Diagnostic entry points: expose the pieces of the path so that each kernel
 * can be checked on its own.  "local" vectors concatenate the free DOFs of all
 * subdomains (interface DOFs appear once per subdomain); "interface" vectors
 * concatenate the dual data G_{i<-j} of all directed subdomain pairs.
 * ------------------------------------------------------------------------ */

/* Sizes: n_local (sum of free DOFs over subdomains), n_iface, n_sub. */
int thm_sys_info(const thm_sys* s, int64_t* n_local, int64_t* n_iface, int32_t* n_sub,
                 int64_t* nnz_stored);

/* Global DOF id and subdomain of every local index (host int64/int32 [n_local]). */
int thm_local_dofs(const thm_sys* s, int64_t* gdof, int32_t* sub);

/* Receiver i, sender j and global DOF of every interface entry (host [n_iface]). */
int thm_iface_dofs(const thm_sys* s, int32_t* recv, int32_t* send, int64_t* gdof);

/* Operators on local vectors (device complex [n_local], FP64):
 *   THM_OP_T     y = T_i x   for all i (Eq. 5's subdomain operator)
 *   THM_OP_PINV  y = P_i^{-1} x  (Eq. 7: the same real P_i^{-1} on Re and Im)
 *   THM_OP_KLOC  y = (T_i - i kappa omega sum_j M_Sigma_ij) x  (no transmission term)
 *   THM_OP_TINV  y = T_i^{-1} x  (the full 2x2 block preconditioner; 2-D only)
 * mode selects FP64 or FP32 storage of the operator (vectors stay FP64 here). */
#define THM_OP_T    0
#define THM_OP_PINV 1
#define THM_OP_KLOC 2
#define THM_OP_TINV 3
int thm_apply_local(thm_sys* s, int op, int mode, const double* x, double* y);

/* One DDM sweep (Eqs. 5-6) on interface data g_in (device complex [n_iface]):
 * subdomain solves with right-hand side (with_sources ? lifting : 0) + G,
 * then the exchange.  Writes g_out and the local solution u_loc
 * (device complex [n_local]). */
int thm_sweep(thm_sys* s, const thm_solve_opts* opts, int with_sources,
              const double* g_in, double* g_out, double* u_loc, thm_stats* stats);

/* Dirichlet lifting right-hand side on local vectors (device complex [n_local]). */
int thm_local_sources(thm_sys* s, double* f_loc);

/* Dirichlet values on all DOFs (device complex [n_dof], 0 on free DOFs). */
int thm_dirichlet_values(thm_sys* s, double* u_d);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper): a process-wide count of this
 * library's kernel launches, and CUDA-event timing of launch classes on the
 * stream each kernel is launched on.
 * ------------------------------------------------------------------------ */
#define THM_K_SPMV      0   /* subdomain operator T_i (or K_i) apply            */
#define THM_K_PINV      1   /* block-preconditioner apply P_i^{-1} (Eq. 7)      */
#define THM_K_DOTS      2   /* Arnoldi: segmented dot products                  */
#define THM_K_UPDATE    3   /* Arnoldi: w -= V h (and norms)                    */
#define THM_K_KRYLOV    4   /* other Krylov kernels (scale, Givens, reductions) */
#define THM_K_DDM       5   /* right-hand sides, exchange, glue, residual, IR   */
#define THM_K_SETUP     6   /* numbering, assembly, factorisation               */
#define THM_K_NCLASSES  7

/* Algorithmic bytes one launch of class cls must move in mode (THM_MODE_*),
 * from the system's sizes (index streams and SELL padding are layout
 * overhead and not counted):
 *   THM_K_SPMV: nnz(P_i) values + 2 diagonal face terms per row
 *               + x read + y written (complex vectors)
 *   THM_K_PINV: the inverse blocks W_l of the forward sweeps and the middle
 *               level (sum_l m_l^2 per subdomain), the backward-sweep blocks
 *               H_l = W_l F_l resp. W_l E_l (sum_{l != k} m_l m_{l+-1}), the
 *               level coupling values of the forward and middle steps, the
 *               order-2 condensation tables, x read + y written
 * Other classes: THM_EINVAL. */
int thm_alg_bytes(const thm_sys* s, int mode, int cls, double* bytes);

/* Algorithmic bytes of the work that this system has actually done so far in
 * `mode`'s precision: inside the Arnoldi steps the kernels skip the
 * subdomains whose Krylov segment has converged, so the work per launch
 * varies and thm_alg_bytes (every subdomain) overstates it.  The kernels count
 * on the device, one atomic per block; this call reads the sums (synchronising
 * the system's stream).
 *   THM_K_PINV:   values and rows of the subdomains processed, by the byte
 *                 model of thm_alg_bytes
 *   THM_K_SPMV:   rows processed x thm_alg_bytes(THM_K_SPMV) / n_local
 *   THM_K_DOTS:   the dot-product passes over the Krylov basis (basis vectors
 *                 and the vectors they are dotted with, read once per pass)
 *   THM_K_UPDATE: the update passes (vectors read, vectors written)
 * Other classes: THM_EINVAL. */
int thm_work_bytes(const thm_sys* s, int mode, int cls, double* bytes);

/* ------------------------------------------------------------------------
 * thm_residual_noalloc -- the FP64 true residual of a field u without any
 * device allocation (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory when they need the check:
 * programs that hand all device memory to their own pool allocator up front
 * (a cudaMalloc then fails, or the pool forbids it), and loops that must not
 * call cudaMalloc or cudaFree because those synchronise the whole device.
 *
 *  u    device complex double [n_dof]: a field on all DOFs (Dirichlet entries
 *       are ignored; the Dirichlet lifting already sits in f).
 *  out  device double[2], written on the system's stream: out[0] = ||f - K u||,
 *       out[1] = ||f||, global FP64 norms over all free DOFs.  For a single
 *       problem out[0] / out[1] is thm_stats.rel_residual; for a batch it is
 *       the ratio over the whole batch vector, whereas thm_stats.rel_residual
 *       reports the largest per-problem ratio.
 *  Limit: n_dof <= 4,194,304 (4096 partial-sum blocks of 1024 DOFs); larger
 *       systems get THM_EINVAL with the limit in the message.
 *  Scratch: a file-scope device array of 64 KB, held by every GPU that loads
 *       the library until the process exits; every call overwrites the
 *       partials it uses (nothing has to start at zero).  Calls that overlap
 *       on the GPU (on different streams, or from threads on one device) race
 *       on that array and must be serialised by the caller.
 *  First call on a device: looks up the array's device address with
 *       cudaGetSymbolAddress (no allocation) and caches it; make that first
 *       call before any stream capture.
 *  No cudaMalloc, cudaFree or allocating library call is made.
 * ------------------------------------------------------------------------ */
int thm_residual_noalloc(const thm_sys* s, const double* u, double* out);

/* Bytes of the stored preconditioner factors (the dense inverse blocks W_l of
 * the twisted block factorisation and the backward-sweep blocks H_l^T =
 * (W_l F_l)^T resp. (W_l E_l)^T of every level but the middle one, row strides
 * padded to 4 entries) for precond THM_PRECOND_* in mode
 * THM_MODE_*: real values for Eq. 7, complex ones for the full 2x2 block
 * operator.  From the sizes alone (nothing is factorised by this call). */
int thm_factor_bytes(const thm_sys* s, int precond, int mode, double* bytes);

/* Kernel launches issued by this library since the process started. */
int64_t thm_kernel_launches(void);

/* Time the classes in mask (bit 1 << THM_K_*) with CUDA events from now on;
 * resets all totals.  0 disables timing (launches are always counted). */
int thm_profile_enable(unsigned mask);

/* Launches and summed event time (ms) of one class since thm_profile_enable;
 * waits for that class's pending events. */
int thm_profile_read(int cls, int64_t* launches, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* THM_H */
