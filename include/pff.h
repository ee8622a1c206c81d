/*
 * pff.h -- C-ABI of the GB300 (sm_103a) phase-field fracture library (libpff.so).
 *
 * Computes, on one GPU, the hot path of the matrix-free monolithic multigrid solver of
 * Jodlbauer, Langer, Wick, "Parallel matrix-free higher-order finite element solvers for
 * phase-field fracture problems": the residual of Eq. (residual), the Jacobian of Eq. (G)
 * applied matrix-free by sum factorisation (Sec. 3.4), the primal-dual active-set step of
 * Alg. 1, and the geometric-multigrid preconditioner of Sec. 3.3 (block-diagonal
 * Chebyshev-Jacobi smoother, nested-mesh transfers, coarse solve) inside flexible GMRES.
 *
 * Discretisation. Unit square (dim 2) or cube (dim 3), N^dim cells of edge h = 1/N, Q_p
 * Lagrange elements on Gauss-Lobatto-Legendre nodes, (p+1)^dim Gauss points per cell.
 * Nodes are numbered lexicographically over (pN+1)^dim points, x fastest. A global vector
 * ("DoF vector") is component blocked: [u_1 | ... | u_dim | phi], n_nodes values per block,
 * n_dofs = (dim+1) n_nodes. Boundary data of the single-edge notched tension test (Sec. 5.1):
 * every displacement component is fixed on the bottom and top faces (last coordinate 0 and 1).
 *
 * Conventions of every entry point:
 *  - Pointers to vectors are DEVICE pointers owned by the caller, contiguous, in the DoF
 *    layout above (or one value per node where stated). The library never frees them.
 *  - Work is enqueued on the CUDA stream passed to pff_setup_mesh and is asynchronous with
 *    respect to the host unless stated otherwise.
 *  - The return value is PFF_OK (0) or a negative PFF_ERR_* code; pff_strerror() names it.
 *    No C++ exception crosses this interface. After PFF_ERR_CUDA the context must be destroyed.
 *  - The context is not thread safe: one host thread per context.
 */
#ifndef PFF_H
#define PFF_H

#ifdef __cplusplus
extern "C" {
#endif

#define PFF_OK 0
#define PFF_ERR_INVALID_ARG (-1)   /* bad size, degree, pointer or mode */
#define PFF_ERR_OOM (-2)           /* device allocation failed */
#define PFF_ERR_CUDA (-3)          /* a CUDA runtime call or kernel launch failed */
#define PFF_ERR_NAN (-4)           /* a non-finite value appeared in a norm */
#define PFF_ERR_NOT_CONVERGED (-5) /* FGMRES reached its iteration cap */
#define PFF_ERR_BREAKDOWN (-6)     /* Krylov breakdown (zero norm before convergence) */
#define PFF_ERR_NO_STATE (-7)      /* pff_set_state has not been called */
#define PFF_ERR_TOO_LARGE (-8)     /* problem exceeds the fixed scratch of pff_param_grad_noalloc, the
                                      32-bit indices of the assembled comparator matrix, or 2^31 - 1
                                      DoFs (the operator kernels index DoFs with 32-bit integers) */
#define PFF_ERR_UNAVAILABLE (-9)   /* an optional library (cuSPARSE, for pff_csr_spmv) cannot be loaded */

/* Splits of the elastic energy (Sec. 2.1): none = isotropic model, miehe = spectral split. */
#define PFF_SPLIT_NONE 0
#define PFF_SPLIT_MIEHE 1

/* Jacobian modes (low two bits of `mode`). */
#define PFF_MODE_FULL 0       /* G of Eq. (G) */
#define PFF_MODE_BLOCKDIAG 1  /* diag(G_uu, G_phiphi): coupling block G_phiu dropped (Sec. 3.3 smoother) */
#define PFF_MODE_TRANSPOSE 2  /* G^T */
/* Masking flags (OR-ed into `mode`). Default: rows and columns of Dirichlet DoFs and of the
 * active set are replaced by the identity (x is zeroed there on input, y = x there on output). */
#define PFF_MASK_RAW 4        /* no masking at all: the plain sum over cells of Sec. 3.4 */
#define PFF_MASK_ADJOINT 8    /* x zeroed on Dirichlet DoFs only, output unmasked: d(R)/dU^T v
                                 for the residual of pff_residual (whose Dirichlet rows are 0) */

/* Node flag bits returned by pff_node_flags. */
#define PFF_FLAG_FIXED(c) (1u << (c))  /* field c masked: c < dim Dirichlet; c == dim active phi */
#define PFF_FLAG_TOP 0x10u            /* node on the top face */
#define PFF_FLAG_BOTTOM 0x20u         /* node on the bottom face */
#define PFF_FLAG_SLIT 0x40u           /* node on the slit / notch (last coord 1/2, x <= 1/2) */
#define PFF_FLAG_COPY 0x80u           /* copy of a slit node used by the cells below a cut slit */

typedef struct pff_ctx pff_ctx; /* opaque: mesh hierarchy, states, per-point data, workspaces */

typedef struct {
  int dim;            /* 2 or 3 */
  int degree;         /* p = 1..4 */
  int n_cells_1d;     /* N >= 1 cells per direction on the finest mesh */
  int coarse_min;     /* levels halve N while N is even and N/2 >= coarse_min (default 3) */
  int split;          /* PFF_SPLIT_NONE or PFF_SPLIT_MIEHE */
  double lambda, mu;  /* Lame parameters (used where no nodal field is given) */
  double gc;          /* critical energy release rate G_c (used where no nodal field is given) */
  double eps;         /* phase-field length scale epsilon */
  double kappa;       /* degradation regularisation: g(phi) = (1 - kappa) phi^2 + kappa */
  double as_c;        /* constant c of the active-set rule of Alg. 1 (default 1) */
  int mg_precision;   /* 64: FP64 multigrid; 32: FP32 levels, smoothers, transfers (coarse solve per
                         coarse_precision) */
  int cheb_degree;    /* Chebyshev-Jacobi smoother degree (paper: 5) */
  double cheb_lo;     /* smoothing interval [cheb_lo, cheb_hi] * lambda_max (paper: 0.24, 1.2) */
  double cheb_hi;
  int eig_iters;      /* CG-Lanczos iterations for lambda_max (default 15) */
  unsigned long long eig_seed; /* SplitMix64 seed of the CG start vector */
  int gmres_restart;  /* FGMRES restart length (default 50) */
  int gmres_max_iters;/* FGMRES iteration cap per linear solve (default 500) */
  double lin_rtol;    /* FGMRES relative tolerance (paper: 1e-6) */
  int fp64_mode;      /* FP64 Jacobian applies: 0 native FP64 arithmetic; 1 double-word (float-float)
                         arithmetic on the FP32 pipe, about 48 significant bits */
  int coarse_precision; /* coarse solve of the FP32 multigrid: 64 (default) FP64 inverses of the FP64
                           coarse blocks, the cycle's vector cast to FP64 and back around it; 32 FP32
                           inverses of the rounded blocks. Ignored (always 64) by the FP64 multigrid. */
  int slit_cut;       /* 0 (default): one node per grid point, the slit enters through the state (phi = 0
                         on its nodes). 1: the slit is cut into the finest mesh (Sec. 5.1): every node
                         on the slit except the tip (last coordinate 1/2, x < 1/2) gets a second copy,
                         which the cells below the slit use. The copies are numbered after the
                         (pN+1)^dim grid nodes, x fastest (then y in 3D), and carry PFF_FLAG_COPY, so
                         n_nodes = (pN+1)^dim + pN/2 (2D) or + (pN/2)(pN+1) (3D); in 2D the DoF counts are
                         those of the paper's table of slit DoFs. Needs N even with N/2 a multiple of
                         the tile height along the last axis (2D: 16 cells for p = 1, 8 for p = 2, 4 for
                         p = 3, 4; 3D: 2 for p <= 3, 1 for p = 4), else INVALID_ARG. Coarse levels keep one
                         node per grid point (the prolongation gives a copy its slit node's value, the
                         restriction adds it back). The assembled-matrix comparator is not available. */
  int fp32_tangent;   /* FP32 Jacobian applies in 2D (the FP32 multigrid): 0 (default) read stored
                         per-point values (precomputed in FP64 and rounded); 1 recompute the tangent of
                         Eq. (G) at every Gauss point from the nodal state (u, phi, phi~), which the apply
                         reads instead: the method's minimum of DRAM traffic, but more arithmetic (slower
                         on GB300 at 2D Q2). Nodal material fields and 3D always use stored values. */
} pff_params;

typedef struct {
  double res_norm;       /* ||R~||: residual with Dirichlet and active rows zeroed, before the update */
  double gmres_rel;      /* final relative residual of the linear solve */
  int gmres_iters;       /* FGMRES iterations */
  int n_active;          /* |A_k| */
  int n_changed;         /* phase-field DoFs whose active flag changed against A_{k-1} */
  int status;            /* PFF_OK or the error of the linear solve */
  double t_residual_ms, t_setup_ms, t_solve_ms; /* host wall time of the phases */
} pff_report;

/* Defaults: the paper's tension test (lambda 121.15, mu 80.77, G_c 2.7e-3, kappa 1e-10), split none,
 * dim 2, p 1, N 32, eps 2/N, c 1, FP32 multigrid with FP64 coarse solve, Chebyshev degree 5 on
 * [0.24, 1.2] lambda_max,
 * 15 eigen iterations, restart 50, relative tolerance 1e-6 (Sec. 5.1, Sec. 6.2), native FP64 applies.
 * Never fails. */
void pff_default_params(pff_params* p);

/* Builds the mesh hierarchy and allocates per-level storage (Sec. 3.3 nested meshes).
 * `stream` is a cudaStream_t (NULL = legacy default stream). On success *out owns the context.
 * Errors: INVALID_ARG (dim, degree, N, tolerances out of range), TOO_LARGE (more than 2^31 - 1 DoFs
 * on the finest level, counting a cut slit's copies; far above what device memory holds), OOM, CUDA. */
int pff_setup_mesh(pff_ctx** out, const pff_params* p, void* stream);

/* Frees everything the context owns (synchronises its stream first). NULL is allowed. */
void pff_destroy(pff_ctx* ctx);

/* Sizes of level 0 (finest) and the number of levels. Host pointers, any may be NULL. */
int pff_sizes(const pff_ctx* ctx, long long* n_dofs, long long* n_nodes, int* n_levels);

/* Sizes of level `level` (0 = finest): nodes and cells per direction. Host pointers. */
int pff_level_sizes(const pff_ctx* ctx, int level, long long* n_nodes, int* n_cells_1d);

/* Per-node flags of the finest mesh (PFF_FLAG_*), one byte per node, device pointer. The
 * active bit reflects the active set of the last pff_set_state / Newton step. */
int pff_node_flags(pff_ctx* ctx, int level, unsigned char* flags);

/* Sets the Newton state (Alg. 1, Eq. (residual)):
 *   U        DoF vector [u | phi] with the Dirichlet values already lifted in (required);
 *   phi_old  previous load step's phase field, one per node (required): bound phi <= phi_old;
 *   phi_tilde extrapolated phase field used in g(phi~) of the u-equation (NULL: phi_old);
 *   active   one byte per node, nonzero = phase-field DoF in the active set A (NULL: the set is
 *            computed by the rule of Alg. 1 from the residual at U and phi is reset to phi_old on it;
 *            that is the first step of Alg. 1, so the next pff_solve_newton_step goes on from it
 *            instead of determining the set again);
 *   gc_field, lambda_field, mu_field: nodal material fields (NULL: the constants of the params).
 * Copies every input. Computes the per-quadrature-point tangent data of the finest level in FP64
 * (and FP32 when mg_precision is 32). Multigrid level data are built lazily by the first
 * pff_vcycle / pff_solve_newton_step after it. Errors: NO_STATE never; INVALID_ARG on NULL U/phi_old. */
int pff_set_state(pff_ctx* ctx, const double* U, const double* phi_old, const double* phi_tilde,
                  const unsigned char* active, const double* gc_field, const double* lambda_field,
                  const double* mu_field);

/* Current Newton state U (DoF vector) into `U_out` (device). */
int pff_get_state(pff_ctx* ctx, double* U_out);

/* Active set of the current state, one byte per node (1 = active), device pointer. */
int pff_get_active(pff_ctx* ctx, unsigned char* active_out);

/* y = G x on level `level` (0 = finest) with G of Eq. (G) at the current state, matrix free
 * (Sec. 3.4). precision 64: x, y are double*; 32: float* (tangent data rounded to FP32, FP32
 * accumulation). mode: PFF_MODE_* | PFF_MASK_* (see above). x and y must not alias.
 * Level > 0 builds the multigrid data first if needed. Errors: NO_STATE, INVALID_ARG. */
int pff_apply_jacobian(pff_ctx* ctx, int level, const void* x, void* y, int precision, int mode);

/* r = R(U) of Eq. (residual) at the current state, FP64, rows of Dirichlet DoFs set to 0. */
int pff_residual(pff_ctx* ctx, double* r);

/* Force on the loaded top face (tension test, Sec. 5.1; shear test, Sec. 5.2), the ordinate of the
 * load-displacement curve, at the current state: the rows of R(U) (Dirichlet rows kept) of the loaded
 * component (pff_set_load_component; u_dim by default) summed over the nodes of the top face, i.e.
 * the residual's u-equation tested with the unit displacement of that face in the loading direction
 * (the consistent nodal reaction; for a uniform stress it is the face integral of sigma_{comp,dim}).
 * *force is a host double. Synchronous. Errors: INVALID_ARG, NO_STATE. */
int pff_reaction_force(pff_ctx* ctx, double* force);

/* Diagonal of the masked block-diagonal operator diag(G_uu, G_phiphi) on `level` (masked rows 1),
 * the Jacobi scaling of the smoother (Sec. 3.3). precision 64 or 32. With mg_precision 32 the
 * multigrid's diagonal is computed in FP32 from the FP32 per-point data (what precision 32 returns);
 * precision 64 computes the FP64 diagonals of all levels on first request. */
int pff_diagonal(pff_ctx* ctx, int level, void* diag, int precision);

/* lambda_max estimates of D^{-1} G_uu and D^{-1} G_phiphi on `level` (host double[2]). */
int pff_lambda_max(pff_ctx* ctx, int level, double* lam2);

/* Multigrid state of `level`: the Newton state carried to that mesh (DoF vector of the level). */
int pff_level_state(pff_ctx* ctx, int level, double* U_level);

/* Prolongation from level+1 (coarse) to level (fine): y_fine = Z P x_coarse, Z zeroing masked
 * fine rows. Restriction: y_coarse = Z_c P^T x_fine (transpose, masked coarse rows zeroed).
 * precision 64 or 32, vectors in the layout of their level. */
int pff_prolongate(pff_ctx* ctx, int level, const void* x_coarse, void* y_fine, int precision);
int pff_restrict(pff_ctx* ctx, int level, const void* x_fine, void* y_coarse, int precision);

/* One application of the block-diagonal Chebyshev-Jacobi smoother on `level` with zero initial
 * guess: x = S(G_uu, G_phiphi) f (Sec. 3.3), with the level's lambda_max estimate and the diagonal
 * of the requested precision. */
int pff_smooth(pff_ctx* ctx, int level, const void* f, void* x, int precision);

/* Coarse-level solve: z = G_c^{-1} r by block forward substitution over the block lower triangular
 * coarse matrix (Sec. 3.3), r and z FP64 in the coarsest level's layout. The dense inverses of the
 * diagonal blocks are FP64 (Gauss-Jordan on the FP64 coarse blocks), the precision the FP32 V-cycle
 * uses too; only with mg_precision 32 and coarse_precision 32 are they FP32 copies, computed and
 * applied in FP32 (r is then rounded to FP32 on entry). */
int pff_coarse_solve(pff_ctx* ctx, const double* r, double* z);

/* One V-cycle of GMG(G) (Sec. 3.3) on the finest level: z = M^{-1} r, FP64 in and out; inside it
 * runs in the params' mg_precision. */
int pff_vcycle(pff_ctx* ctx, const double* r, double* z);

/* Solves G dU = b by right-preconditioned flexible GMRES with the V-cycle (FP64 outer). Host
 * pointers iters/rel may be NULL. Synchronises the stream once per iteration. */
int pff_solve_linear(pff_ctx* ctx, const double* b, double* x, int* iters, double* rel);

/* One primal-dual active-set iteration (Alg. 1) from the current state: residual, active set,
 * reset phi to phi_old on it, level setup, FGMRES + GMG solve of G dU = -R on the inactive DoFs,
 * update U += dU. The context's state becomes the new iterate; it is also copied to U_out when
 * non-NULL. `rep` (host, may be NULL) receives the report. Synchronous. */
int pff_solve_newton_step(pff_ctx* ctx, double* U_out, pff_report* rep);

/* Alg. 1 repeated from the current state until the active set no longer changes and
 * ||R~_k|| <= newton_rtol * ||R~_0|| (paper: 1e-8), or max_iters steps. Reports of the steps go to
 * `reps` (host array of max_iters entries, may be NULL); *n_steps receives the number of steps.
 * Returns PFF_ERR_NOT_CONVERGED if the loop ended by max_iters, or the first failing step's status.
 * The final state is the context's state (and is copied to U_out when non-NULL). Synchronous. */
int pff_solve_pdas(pff_ctx* ctx, int max_iters, double newton_rtol, double* U_out, pff_report* reps, int* n_steps);

/* Displacement component that the load steps prescribe on the top face and in which
 * pff_reaction_force measures: dim - 1 (the default; the tension test of Sec. 5.1, top face pulled)
 * or 0 (the shear test of Sec. 5.2, top face moved to the right; the other components stay as the
 * state has them, 0 for that test). Both tests fix every displacement component on the top and bottom
 * faces, so the masks do not change. Errors: INVALID_ARG (comp outside 0..dim-1). */
int pff_set_load_component(pff_ctx* ctx, int comp);

/* One quasi-static load step of the tension test (Sec. 5.1; of the shear test with
 * pff_set_load_component) from the current state: the loaded displacement component (u_dim by
 * default) on the top face is set to `load` (all other Dirichlet values kept), phi_old becomes
 * the phase field of the last solved load step (the state's own before the first) and phi~ the linear
 * extrapolation from the solutions of the last two load steps, clamp(2 phi^{n-1} - phi^{n-2}, 0, 1)
 * (Sec. 3.2), or phi_old while fewer than two load steps have been solved (the phase field given to
 * pff_set_state is not the solution of a load step); then pff_solve_pdas. The history is cleared by
 * pff_set_state and advances only when the step converges. Same outputs and errors as
 * pff_solve_pdas. */
int pff_solve_load_step(pff_ctx* ctx, double load, int max_iters, double newton_rtol, pff_report* reps,
                        int* n_steps);

/* Phase-field history of the load-step loop, for checkpoint and resume: phi1 = phase field after the
 * last converged load step, phi2 = the one before (device arrays of n_nodes doubles); n_hist (host
 * int) = how many converged load steps are known (0, 1 or 2; 2 once phi~ is extrapolated). pff_get_history copies the known ones (outputs may be NULL;
 * unknown ones are left untouched). pff_set_history installs a history after pff_set_state (which
 * clears it): with the state U and the history of a checkpoint taken after a converged load step, the
 * next pff_solve_load_step continues that run (same iterates up to the order of the floating-point
 * sums of shared nodes). Synchronous. Errors: INVALID_ARG (n_hist outside 0..2, or a needed array
 * NULL), NO_STATE (pff_set_history before pff_set_state). */
int pff_get_history(pff_ctx* ctx, double* phi1, double* phi2, int* n_hist);
int pff_set_history(pff_ctx* ctx, const double* phi1, const double* phi2, int n_hist);

/* Parameter gradients of the residual (not in the paper; needed for adjoints): for a test vector v
 * (DoF layout), g_gc = (dR/dG_c)^T v, g_lambda = (dR/dlambda)^T v, g_mu = (dR/dmu)^T v with the
 * material parameters as nodal fields, one value per node each, at the current state. Entries of v
 * on Dirichlet DoFs are ignored (those rows of the residual are zero). Any output may be NULL;
 * outputs are overwritten. */
int pff_param_grad(pff_ctx* ctx, const double* v, double* g_gc, double* g_lambda, double* g_mu);

/* Allocation-free variant of pff_param_grad (the paper has no counterpart: this exists for callers
 * of this library that must not allocate device memory, e.g. code running while a CUDA graph is
 * being captured, where cudaMalloc is illegal, or a host that owns all device memory through its
 * own pool). pff_param_grad allocates its per-point scratch (3 x cells x points-per-cell doubles)
 * on first use; this entry point uses a fixed array in device global memory instead, of
 * PFF_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB), which every GPU that loads the library holds until
 * the process exits. Problems that need more (3 * N^dim * (p+1)^dim doubles) are rejected with
 * PFF_ERR_TOO_LARGE before any work is queued. The context's device (that of the stream given to
 * pff_setup_mesh) must be the current device, else PFF_ERR_INVALID_ARG: the array's address is a
 * per-device one. The first call on a device looks up that address (cudaGetSymbolAddress); make
 * that first call before any stream capture. No call allocates (no cudaMalloc, cudaFree or allocating library routine).
 * All calls share the array: calls whose work overlaps on the GPU (other streams, other contexts)
 * race on it, so serialise them. Every scratch entry read is written earlier in the same call, so
 * the contents left by a previous call do not matter. Same arguments, results and requirements as
 * pff_param_grad otherwise (the state must have been set; outputs are overwritten). */
#define PFF_NOALLOC_SCRATCH_DOUBLES (2LL * 1024 * 1024)
int pff_param_grad_noalloc(pff_ctx* ctx, const double* v, double* g_gc, double* g_lambda, double* g_mu);

/* ---- Assembled-matrix comparator (Sec. 6.3, fig. compare:vmult) ------------------------------
 * The paper times the matrix-free product against a sparse-matrix product with the assembled
 * Jacobian. pff_csr_assemble assembles the finest level's operator of the linear solve,
 * Z G Z + (I - Z) (Eq. (G) at the current state; Dirichlet and active DoFs masked as by
 * pff_apply_jacobian's default mask), into a context-owned device CSR matrix (32-bit indices, FP64
 * values, columns ascending, rows and columns in the DoF layout): the pattern comes from the mesh
 * and the masks (pff_csr_pattern), the values from (d+1)(2p+1)^d products of the native FP64
 * matrix-free operator with coloured probe vectors (two nodes of one colour never share a row).
 * The matrix is a snapshot of the state: later state changes do not update it; assembling again
 * replaces it. *nnz (host, may be NULL) receives the number of entries. Synchronous.
 * Errors: INVALID_ARG (a context with a cut slit), NO_STATE, TOO_LARGE (n_dofs + 1 or nnz above
 * 2^31 - 1), OOM, CUDA. */
int pff_csr_assemble(pff_ctx* ctx, long long* nnz);

/* y = A x with the assembled matrix, by cuSPARSE SpMV (FP64, default algorithm; the library is
 * loaded on first use) on the context's stream. x, y: device arrays of n_dofs doubles, not aliased.
 * Errors: INVALID_ARG, NO_STATE (nothing assembled), UNAVAILABLE (cuSPARSE not found), CUDA. */
int pff_csr_spmv(pff_ctx* ctx, const double* x, double* y);

/* Host only: 1 when cuSPARSE can be loaded and every entry point pff_csr_spmv uses resolves, else 0
 * (loads the library on the first call; no GPU work). */
int pff_csr_spmv_available(void);

/* Copies the assembled matrix into device arrays: rowptr (n_dofs + 1 ints), col (nnz ints), val
 * (nnz doubles); each may be NULL. Synchronous. Errors: INVALID_ARG, NO_STATE (nothing assembled). */
int pff_csr_export(pff_ctx* ctx, int* rowptr, int* col, double* val);

/* Host only (no GPU work): the pattern that pff_csr_assemble uses, for a mesh of n_cells_1d^dim Q_p
 * cells and host node flags (one byte per node; bit f set = DoF of component f masked). A masked row
 * holds its diagonal; an unmasked row of node i holds the unmasked DoFs of every node sharing a cell
 * with i, of the displacement components for a displacement row (G_uphi = 0) and of all components
 * for a phase-field row, columns ascending. *nnz (required) receives the number of entries; rowptr
 * (n_dofs + 1 ints) and col (nnz ints) are host arrays filled when not NULL, so a first call with
 * both NULL sizes them. Errors: INVALID_ARG, TOO_LARGE. */
int pff_csr_pattern(int dim, int degree, int n_cells_1d, const unsigned char* flags, int* rowptr, int* col,
                    long long* nnz);

/* Host only: the probing plan of pff_csr_assemble. For component f and colour `color` (0 <=
 * color < (2p+1)^dim; a node's colour is sum_t (i_t mod (2p+1)) (2p+1)^t over its indices i_t),
 * targets[r] (host, n_dofs entries) receives, for every row r, the one column of component f and that
 * colour among the nodes sharing a cell with r's node, or -1 when there is none; the assembly stores
 * the probe's y[r] there when the pattern holds that column. Errors: INVALID_ARG. */
int pff_csr_probe_targets(int dim, int degree, int n_cells_1d, int f, int color, long long* targets);

/* Device memory the context holds (Sec. 6.1 compares memory requirements), in bytes, host outputs,
 * each may be NULL: level_bytes[l] for each of the n_levels levels (node flags, state, nodal fields,
 * per-point data in all precisions, diagonals, multigrid work vectors), the FGMRES basis (krylov), the
 * dense coarse blocks and their inverses (coarse), everything else including the assembled
 * comparator matrix (other), and the sum (total). Buffers allocated on first use (multigrid work
 * vectors, gradient scratch, comparator matrix) count once they exist. Errors: INVALID_ARG. */
int pff_memory(pff_ctx* ctx, long long* level_bytes, long long* krylov, long long* coarse, long long* other,
               long long* total);

/* Device timing of one kernel family with CUDA events recorded on the context's stream around
 * each launch of that family (for throughput and roofline figures; off by default):
 *   PFF_PROF_OFF, PFF_PROF_JAC64_L0 / PFF_PROF_JAC32_L0 (FP64 / FP32 Jacobian kernels on the finest
 *   level, any mode), PFF_PROF_JAC64 / PFF_PROF_JAC32 (any level), PFF_PROF_RESIDUAL.
 * pff_profile resets the counters; pff_profile_result synchronises the stream and returns the
 * number of timed launches and their summed device time in milliseconds (at most 16384 launches
 * are timed; later ones are not). */
#define PFF_PROF_OFF 0
#define PFF_PROF_JAC64_L0 1
#define PFF_PROF_JAC32_L0 2
#define PFF_PROF_JAC64 3
#define PFF_PROF_JAC32 4
#define PFF_PROF_RESIDUAL 5
int pff_profile(pff_ctx* ctx, int family);
int pff_profile_result(pff_ctx* ctx, int* launches, double* total_ms);

/* Number of CUDA kernels this library has launched since it was loaded (all contexts), counting
 * the kernels inside each replay of a captured graph (captured launches themselves are not counted). */
long long pff_launch_count(void);

/* Human-readable name of a status code. */
const char* pff_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PFF_H */
