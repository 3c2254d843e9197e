/*
 * mg.h -- C ABI of libmg.so, a GB300 (sm_103a) geometric multigrid solver for the
 * sparse finite element systems of conforming Q1 and nonconforming rotated-Q1
 * (Rannacher-Turek) elements on uniformly refined grids of the unit square / cube.
 *
 * The operation is the multigrid solve of the paper "An object oriented parallel
 * finite element scheme for computations of PDEs: Design and implementation"
 * (Ganesan et al.): V-cycles (Sec. 5.3, Algorithm "Parallel Multigrid Solver
 * (V-Cycle)") of smoothing sweeps, restriction of the residual, an exact solve on the
 * coarsest level, prolongation with correction, on a hierarchy of meshes obtained by
 * uniform refinement (Sec. 5.1), with grid transfers between the levels (Sec. 5.4).
 * The V-cycle is applied to the defect inside a defect-correction loop that stops at
 * a relative residual.
 *
 * Conventions for every entry point:
 *   - Return value: MG_OK (0) or a negative MG_E* code; mg_last_error() then returns a
 *     thread-local message. No C++ exception crosses this interface.
 *   - "device pointer": memory of the CUDA device current when mg_setup was called.
 *     "host pointer": ordinary (pageable or pinned) CPU memory.
 *   - The library owns hierarchies and servers; the caller owns every array it passes.
 *   - DOF order: interior DOFs only (homogeneous Dirichlet boundary eliminated).
 *     Q1: vertices (ix, iy[, iz]) in [1, N-1]^d, index (ix-1) + (N-1)*((iy-1) +
 *     (N-1)*(iz-1)). Rotated Q1: faces normal to x, then y, then z; a face normal to x
 *     at x = i/N over cell (j, k) has index (i-1) + (N-1)*(j + N*k), normal to y at
 *     y = j/N over cell (i, k): (N-1)N^2 + i + N*((j-1) + (N-1)*k), normal to z at
 *     z = k/N over cell (i, j): 2(N-1)N^2 + i + N*(j + N*(k-1)).
 *   - Thread safety: calls on different hierarchies may run concurrently; calls on one
 *     hierarchy must not overlap.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mg_status;
#define MG_OK 0
#define MG_PENDING 1      /* mg_serve_poll: the request is not finished yet */
#define MG_EINVAL (-1)    /* invalid argument (sizes, enum values, NULL where required) */
#define MG_ENOMEM (-2)    /* host or device allocation failed */
#define MG_ENOCONV (-3)   /* max_iters reached before the tolerance; x holds the last iterate */
#define MG_ECUDA (-4)     /* a CUDA runtime call failed */
#define MG_ETIMEOUT (-5)  /* a bounded wait ran out */
#define MG_EBUDGET (-6)   /* a serving request can never fit the device-memory budget */
#define MG_ENOTFOUND (-7) /* unknown serving ticket */

/* element */
#define MG_Q1 0  /* conforming bi/trilinear, vertex DOFs, 2D or 3D */
#define MG_RQ1 1 /* nonconforming rotated Q1 with face-mean DOFs, 3D */
/* Conforming P1 / P2 on tetrahedra (the paper's elements, Sec. 6), 3D: every cell of the
 * grid is split into the six Kuhn tetrahedra along its main diagonal (cell (c), axis
 * permutation pi: vertices c, c + e_pi0, c + e_pi0 + e_pi1, c + (1,1,1)); halving the grid
 * splits each into eight of the finer grid's, so the spaces are nested and P is
 * interpolation. P1 DOFs: the interior vertices (numbered like Q1; storage DIA, ELL or
 * CSR). P2 DOFs: vertices and edge midpoints, i.e. the interior points of the grid of
 * 2 n_cells cells, numbered like Q1 there (ELL or CSR). Load vector: b = M f_I (the mass
 * matrix times f at the nodes). Gauss-Seidel colours: P1 (vx + vy + vz) mod 4, P2
 * (wx + 2wy + 4wz) mod 15 on the grid of 2 n_cells cells. */
#define MG_P1 2
#define MG_P2 3
/* smoother */
#define MG_JACOBI 0    /* damped Jacobi x <- x + omega D^-1 (b - A x) */
#define MG_CHEBYSHEV 1 /* Chebyshev polynomial in D^-1 A of degree cheb_degree */
#define MG_GAUSS_SEIDEL 2 /* multicolour Gauss-Seidel (the paper's Eq. GS on DOFs numbered
                             colour-wise, Sec. 4 "DOF Reordering"): one application visits
                             every colour once, x_i <- x_i + (b_i - (A x)_i) / a_ii for all
                             DOFs of a colour at once; colours ascending before the coarse
                             correction, descending after it, so the V-cycle is symmetric.
                             Q1 colours: parity classes of the vertex coordinates (2^dim);
                             rotated Q1: face family x parity of the normal position (6);
                             P1, P2: see MG_P1.
                             Not available to the serving API. */
/* precision */
#define MG_FP64 0  /* every step in FP64 */
#define MG_MIXED 1 /* FP32 V-cycle (matrices, smoother, transfers) inside FP64 defect correction */
/* device storage of the level matrices */
#define MG_STORAGE_AUTO 0 /* chosen by timing the candidates on the device at setup */
#define MG_STORAGE_CSR 1  /* compressed sparse rows, one thread per row */
#define MG_STORAGE_ELL 2  /* column-major ELLPACK with explicit 32-bit column indices */
#define MG_STORAGE_DIA 3  /* column-major ELLPACK whose columns are row + fixed offsets (Q1, P1) */
#define MG_STORAGE_SELL 4 /* sliced ELLPACK: rows sorted by length, slices of 32 rows stored
                             column-major with their own width, 32-bit columns */
#define MG_STORAGE_STENCIL 5 /* constant stencil (Q1, P1, rotated Q1; FP32 levels of a mixed
                                hierarchy): one value per stencil position (rotated Q1: the
                                three values of a face's row: itself, the opposite faces of its
                                two cells, their other faces), used where every row of the
                                level matrix is the same stencil (constant coefficient,
                                rediscretised), boundary neighbours masked from the grid
                                coordinates; no matrix is stored or streamed. Checked exactly
                                on the host; levels that fail the check, Galerkin levels and
                                levels of at most 32768 rows keep DIA (rotated Q1: ELL). Not
                                with Gauss-Seidel. */
#define MG_STORAGE_COEF 6 /* per-cell coefficient (3D Q1; FP32 levels of a mixed hierarchy):
                             where the level matrix is the rediscretisation of a per-cell
                             coefficient k_e (every level above the Galerkin ones, no mass
                             shift), one FP32 value k_e h / 12 per cell is stored and the
                             sweep forms each row from the 8 cells around its vertex and the
                             Q1 element stiffness; 4 bytes per cell instead of 21 values per
                             row. Checked on the host against the assembled FP64 matrix
                             (every entry within 1e-12 of the row's diagonal); levels that
                             fail the check and levels of at most 32768 rows keep DIA. Not
                             with Gauss-Seidel. */
/* grid transfers P (prolongation, Sec. 5.1) and R = P^T of a level (mg_info.transfer) */
#define MG_TRANSFER_NONE 0 /* level 0 (no coarser level) */
#define MG_TRANSFER_GRID 1 /* Q1: weights computed from the grid in the kernel */
#define MG_TRANSFER_SELL 2 /* rotated Q1, P1, P2: explicit P and R in SELL-32 */

#define MG_MAX_LEVELS 16

/* The problem: a uniform grid of n_cells^dim cells on the unit square / cube, refined
 * n_levels-1 times from the coarsest grid of n_cells / 2^(n_levels-1) cells per axis
 * (which must be an integer >= 2). k_cell: host pointer to the per-cell diffusion
 * coefficient of the finest grid (n_cells^dim values, x fastest), or NULL for k = 1.
 * mass: sigma >= 0; the operator of every level is A + sigma M with M the consistent
 * mass matrix (Q1 only), the system of a Crank-Nicolson step scaled by sigma = 2/dt
 * (mg_heat); 0 for the stiffness matrix alone. Zero-initialise unused fields. */
typedef struct {
    int dim;
    int element;
    int n_cells;
    int n_levels;
    const double *k_cell;
    double mass;
} mg_problem;

/* Solver options. mg_options_default() fills in damped Jacobi (omega 0.8), V(2,2),
 * FP64, automatic storage, 100 iterations, CUDA graphs on. nu_pre / nu_post count
 * smoother applications; a Chebyshev application performs cheb_degree matrix-vector
 * products, a Gauss-Seidel application one sweep over all colours. Chebyshev targets [lambda_u / cheb_ratio, lambda_u] with lambda_u =
 * cheb_hi * lambda_hat and lambda_hat from power_iters steps of the power method on
 * D^-1 A (start vector from SplitMix64(power_seed)). */
typedef struct {
    int smoother;
    double omega;
    int cheb_degree;
    int nu_pre, nu_post;
    double cheb_hi, cheb_ratio;
    int power_iters;
    uint64_t power_seed;
    int precision;
    int storage;
    int max_iters;
    int use_graph;
    int use_pdl; /* launch V-cycle kernels with programmatic dependent launch (default 1) */
    int coarse_tail; /* the levels of at most 4096 rows as one thread-block-cluster launch:
                        0 never, 1 whenever it applies, 2 (default) where setup measures the
                        captured V-cycle faster with it than without (always when use_graph
                        is 0); every choice computes the same bits */
    int fuse_first; /* the first pre-smoothing step of a level starts from x = 0 and needs
                       only the level's right-hand side and D^-1 (Sec. 5.3, the smoothing
                       steps of the V-cycle): 1 (default) takes it in the kernel that makes
                       that right-hand side (the restriction from the finer level; on the
                       finest level of a mixed hierarchy the FP64 outer residual), 0 as a
                       sweep of its own; the same bits either way (Jacobi and Chebyshev) */
} mg_options;

/* Right-hand side f of -div(k grad u) = f: the constant f_const if n_modes == 0, else
 * f = -Laplace(u) of the manufactured u = sum_m amp[m] prod_d sin(freq[3m+d] pi x_d).
 * amp: host, n_modes values; freq: host, 3*n_modes integers (third ignored in 2D). */
typedef struct {
    int n_modes;
    const double *amp;
    const int *freq;
    double f_const;
} mg_rhs;

/* Device memory and ordering. alloc/free: the only source of device memory (NULL:
 * cudaMalloc/cudaFree); alloc returns NULL on failure and must return 256-byte aligned
 * memory. stream: the cudaStream_t the caller orders its work on (NULL: the legacy
 * default stream); the library runs on a private stream joined to it by events. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *ctx);
    void *ctx;
    void *stream;
} mg_device;

typedef struct mg_hierarchy mg_hierarchy;

/* Description of a built hierarchy (level 0 = coarsest). */
typedef struct {
    int n_levels;
    int precision;
    int64_t n[MG_MAX_LEVELS];       /* DOFs per level */
    int64_t nnz[MG_MAX_LEVELS];     /* stored structural nonzeros per level matrix */
    int storage[MG_MAX_LEVELS];     /* MG_STORAGE_* chosen per level */
    int galerkin[MG_MAX_LEVELS];    /* 1 if the level matrix is R A P of the finer level */
    double lambda[MG_MAX_LEVELS];   /* power-method estimate of lambda_max(D^-1 A), 0 if unused */
    size_t device_bytes;            /* device memory held by the hierarchy */
    int kernels_per_cycle;          /* kernel launches in one defect-correction iteration */
    int tail_levels;                /* levels replayed by the coarse-level tail launch (0: none) */
    int transfer[MG_MAX_LEVELS];    /* MG_TRANSFER_* between level l and l-1 */
} mg_info;

void mg_options_default(mg_options *o);

/* Number of interior DOFs; -1 for an invalid combination. The DOF sets are those of the
 * paper's elements on the uniformly refined grid (Sec. 5.1; P1/P2 counts of Sec. 6.4). */
int64_t mg_ndofs(int dim, int element, int n_cells);

/* Load vector b_i = integral of f phi_i over the finest grid, 3-point Gauss rule per
 * axis per cell (host computation): the right-hand side of the sparse FE system A x = b
 * of Sec. 2 ("FEM and iterative methods"). b_host: n DOFs, caller-owned. MG_EINVAL for
 * an invalid problem. */
mg_status mg_load_vector(const mg_problem *p, const mg_rhs *f, double *b_host);

/* (Sec. 2, as mg_load_vector.) The same Q1 load vector with the tensor Gauss rule factorised per sine mode and axis
 * (b = sum_m c_m X_m (x) Y_m [(x) Z_m]): O(modes * n) instead of O(modes * 3^d * n) sine
 * evaluations, equal to mg_load_vector up to rounding. Q1 only. */
mg_status mg_load_vector_separable(const mg_problem *p, const mg_rhs *f, double *b_host);

/* The level operators of Sec. 5.1 (system matrix per level) and Sec. 5.4 (transfers), as
 * assembled on the host, without a GPU: which = 0:
 * A_level, 1: P_level (rows: level, columns: level-1), 2: R_level = P_level^T, in CSR
 * with ascending columns and FP64 values (the same matrices mg_setup stores). Call with
 * rowptr = NULL to get *nrows and *nnz only; then rowptr holds nrows+1 entries and
 * col/val nnz entries (caller-owned host arrays). */
mg_status mg_assemble_operator(const mg_problem *p, int level, int which, int64_t *nrows, int64_t *nnz,
                               int64_t *rowptr, int32_t *col, double *val);

/* Host only: *is_stencil = 1 if every row of the level-`level` matrix (as mg_setup
 * assembles it, mass shift included) is the same stencil: no entry outside the 3^d box
 * of the grid point, the interior row's FP64 values at every in-grid neighbour, zero
 * elsewhere. The paper stores every level matrix (Sec. 5.1); this is the per-level
 * condition under which a stored FP32 level can be replaced by its stencil. It is
 * necessary, not sufficient: mg_setup uses MG_STORAGE_STENCIL only on levels l >= 1 of
 * at least 32768 rows of a mixed-precision hierarchy without Gauss-Seidel, requested
 * by MG_STORAGE_STENCIL or chosen by the MG_STORAGE_AUTO timing, and keeps DIA
 * elsewhere even where this check returns 1. Q1 and P1 only (0 for the other elements
 * and for grids of fewer than 4 cells per axis). */
mg_status mg_constant_stencil(const mg_problem *p, int level, int *is_stencil);

/* Build the level hierarchy of Sec. 5.1 (uniform refinement of the coarsest grid, the
 * system matrix assembled on every level) with the transfers of Sec. 5.4: per-level
 * stiffness matrices (rediscretised; R A P of the
 * finer level where the coefficient is not resolved by the coarse cells), transfer
 * operators P (Q1 nodal interpolation, rotated-Q1 face averaging) and R = P^T, device
 * storage, the coarsest-level LU factorisation for the exact coarse solve of the V-cycle
 * (Sec. 5.3; FP64, on the device), smoother parameters and the CUDA graphs of one
 * iteration. p, o: host structs (read only, not kept); dev may be NULL (cudaMalloc);
 * *out receives a hierarchy owned by the library until mg_hierarchy_free. MG_EINVAL for
 * invalid sizes or options, MG_ENOMEM when dev->alloc fails, MG_ECUDA on a CUDA error;
 * nothing is left allocated on failure. */
mg_status mg_setup(const mg_problem *p, const mg_options *o, const mg_device *dev, mg_hierarchy **out);
/* Release everything mg_setup allocated (through dev->free). NULL is MG_EINVAL. */
mg_status mg_hierarchy_free(mg_hierarchy *h);
/* Describe a built hierarchy (sizes, storage per level, Sec. 5.1 levels); info: host. */
mg_status mg_get_info(const mg_hierarchy *h, mg_info *info);

/* The solve of the paper: the V-cycle of Sec. 5.3 (Algorithm "Parallel Multigrid Solver
 * (V-Cycle)": pre-smoothing, restriction of the defect, exact coarsest solve,
 * prolongation and correction, post-smoothing) applied in a defect-correction loop
 * until ||b - A x||_2 <= rel_tol * ||b||_2 (the paper gives no stopping rule):
 *   r_k = b - A x_k (FP64), stop test, c = V(r_k), x_{k+1} = x_k + c.
 * b_dev, x_dev: device pointers to n doubles; x_dev holds the initial guess on entry
 * and the result on exit. iters (may be NULL): V-cycles performed. res_hist (host, may
 * be NULL, max_iters + 1 doubles): ||r_k|| / ||b|| for k = 0..iters. Returns MG_ENOCONV
 * if max_iters cycles do not reach the tolerance. Synchronises with the caller's
 * stream on return. */
mg_status mg_solve(mg_hierarchy *h, const double *b_dev, double *x_dev, double rel_tol, int *iters,
                   double *res_hist);

/* mg_solve (Sec. 5.3) with host arrays: copies b to the device, solves, copies x back
 * (x_host also supplies the initial guess). Errors as mg_solve. */
mg_status mg_solve_host(mg_hierarchy *h, const double *b_host, double *x_host, double rel_tol, int *iters,
                        double *res_hist);

/* Conjugate gradients preconditioned by one V-cycle (the paper, Sec. 1: multigrid is
 * most often used as the preconditioner of a Krylov method such as CG or GMRES; for
 * these symmetric positive definite systems that is CG, Saad Alg. 9.1, M^-1 r = V(r)):
 *   r_0 = b - A x_0; per iteration z = V(r), rz = (r, z), p = z + (rz / rz_old) p
 *   (p = z first), q = A p, alpha = rz / (p, q), x += alpha p, r -= alpha q,
 * in FP64 on the finest operator (the V-cycle in the hierarchy's precision). Stops when
 * ||r|| <= rel_tol ||b|| for the recursively updated r; iters counts V-cycles and
 * res_hist (host, may be NULL, max_iters + 1 doubles) holds ||r_k|| / ||b||. The
 * V-cycle must be symmetric: MG_EINVAL unless nu_pre == nu_post (Gauss-Seidel runs
 * its colours backward after the correction). MG_ENOCONV after max_iters iterations,
 * x holding the last iterate. Arguments, ownership and synchronisation as mg_solve. */
mg_status mg_pcg(mg_hierarchy *h, const double *b_dev, double *x_dev, double rel_tol, int *iters,
                 double *res_hist);

/* mg_pcg (Sec. 1, Saad Alg. 9.1) with host arrays (x_host also supplies the initial
 * guess). Errors as mg_pcg. */
mg_status mg_pcg_host(mg_hierarchy *h, const double *b_host, double *x_host, double rel_tol, int *iters,
                      double *res_hist);

/* Crank-Nicolson time stepping of the heat equation u_t - div(k grad u) = f with
 * homogeneous Dirichlet data (the paper's model problem, Sec. 6: Galerkin FE in space,
 * Crank-Nicolson in time; here on Q1 hexahedra). The hierarchy must be set up with
 * problem.mass = sigma = 2/dt. For a source f(t, x) = g(t) F(x) with load vector bF of
 * F, step k = 0..n_steps-1 solves
 *     (A + sigma M) u_{k+1} = (sigma M - A) u_k + (g_k + g_{k+1}) bF
 * (the step (M + dt/2 A) u' = (M - dt/2 A) u + dt/2 (b' + b) times 2/dt; the right-hand
 * side row sums column-ascending by fused multiply-adds, then + t*bF_i), starting from
 * u_k, by defect correction (method MG_METHOD_DC) or V-cycle CG (MG_METHOD_PCG) to
 * ||r|| <= rel_tol ||rhs||. bF_dev, u_dev: device arrays of n doubles (u: u_0 in, u_n
 * out); g_host: n_steps + 1 values g(t_k); iters (host, n_steps ints, may be NULL):
 * V-cycles of each step. MG_ENOCONV if a step does not converge (u holds its last
 * iterate, later steps are not taken); MG_EINVAL if the hierarchy has no mass shift. */
#define MG_METHOD_DC 0
#define MG_METHOD_PCG 1
mg_status mg_heat(mg_hierarchy *h, const double *bF_dev, const double *g_host, int n_steps, double *u_dev,
                  double rel_tol, int method, int *iters);

/* mg_heat (Sec. 6.2) with host arrays bF_host, u_host (copied in, u copied back). */
mg_status mg_heat_host(mg_hierarchy *h, const double *bF_host, const double *g_host, int n_steps, double *u_host,
                       double rel_tol, int method, int *iters);

/* Exactly n_cycles defect-correction iterations with the V-cycle of Sec. 5.3, without a
 * stop test (no host synchronisation between them). b_dev, x_dev as mg_solve. rel_res
 * (host, may be NULL): ||r|| / ||b|| of the last residual computed, i.e. before the last
 * correction. MG_EINVAL for NULL vectors or n_cycles < 0. */
mg_status mg_cycle(mg_hierarchy *h, const double *b_dev, double *x_dev, int n_cycles, double *rel_res);

/* The device copy of a level operator of Sec. 5.1 / 5.4, to the host as CSR (FP64
 * values, structural pattern):
 * which = 0: A_level (precision MG_FP64 or MG_MIXED selects the stored copy),
 * 1: P_level (rows: level, columns: level-1), 2: R_level = P_level^T.
 * Call with rowptr = NULL to get *nnz only; otherwise rowptr holds nrows+1, col/val nnz. */
mg_status mg_export_operator(const mg_hierarchy *h, int level, int which, int precision, int64_t *nrows,
                             int64_t *nnz, int64_t *rowptr, int32_t *col, double *val);

/* Measurement, not part of the method: the paper reports the solve's cost per step
 * class (Sec. 5.5 "Computational complexity": every step O(N)); these time each kernel
 * class per level. Per-kernel timing with CUDA events recorded around every launch
 * (kernel classes below); off by default. mg_profile_read returns the accumulated device time and
 * launch count of one (class, level) since the last enable, and the algorithmic
 * bytes one such launch moves. */
#define MG_K_SMOOTH 0   /* smoother sweep (fused residual + update) */
#define MG_K_RESID 1    /* residual before restriction */
#define MG_K_RESTRICT 2 /* b_{l-1} = R r */
#define MG_K_PROLONG 3  /* x_l += P x_{l-1} */
#define MG_K_COARSE 4   /* coarsest-level LU solve */
#define MG_K_OUTER 5    /* FP64 outer residual and its norm */
#define MG_K_UPDATE 6   /* x += c */
#define MG_K_SMOOTH0 7  /* first smoother step from x = 0 (diagonal only, no matrix-vector product) */
#define MG_K_KRYLOV 8   /* conjugate gradients: inner products, search direction, A p, x and r update */
#define MG_K_COUNT 9
/* enable: 0 off, else on for launches whose class bit is set in class_mask and whose
 * level bit is set in level_mask (~0u: all). Resets the accumulated profile. With
 * profiling on, mg_cycle synchronises after every iteration to read the events. */
mg_status mg_profile_enable(mg_hierarchy *h, int enable, unsigned class_mask, unsigned level_mask);
mg_status mg_profile_read(const mg_hierarchy *h, int kclass, int level, double *ms_total, int64_t *launches,
                          double *bytes_per_launch, double *flops_per_launch);

/* r = b - A x on the finest level in FP64 and rnorm = ||r||_2, without allocating
 * anything. The paper has no counterpart: this entry point is for callers that cannot
 * allocate device memory at the moment they need a residual, for example because a
 * memory pool owns the whole device, because they run inside a callback that must not
 * re-enter an allocator, or because their latency budget rules out an allocation. It
 * calls no cudaMalloc, cudaFree or other allocating routine: its scratch (block partial
 * sums, a completion counter, the result) is a fixed device array of about 512 KiB that
 * every GPU loading the library holds until the process exits.
 *   b_dev, x_dev: device pointers to n doubles (inputs, caller-owned; x needs no
 *   padding); r_dev: device pointer to n doubles (output, caller-owned); rnorm: host
 *   pointer to one double (output). Runs on the caller's stream of mg_device and
 *   synchronises it before returning.
 * Limit: n <= 16,777,216 rows (MG_EINVAL with a message beyond it).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. The address is then kept per device
 * for the life of the process: after a cudaDeviceReset (or any other end of the device's
 * primary context) the kept address is stale, so this entry point must not be called on
 * that device again. Every call shares the one array and it keeps the last call's
 * contents: calls that overlap on the GPU (other streams or threads) race on it and must
 * be serialised by the caller. */
mg_status mg_residual_norm_noalloc(mg_hierarchy *h, const double *b_dev, const double *x_dev, double *r_dev,
                                   double *rnorm);

/* ---------------------------------------------------------------------------------
 * Serving: a request loop that solves many Q1 Poisson problems (k = 1) of different
 * sizes and dimensions with continuous batching, in mixed precision (FP32 V-cycle
 * inside FP64 defect correction).
 *
 * The server reserves hbm_budget_bytes of device memory once (through dev, as for
 * mg_setup) and keeps everything inside it: one operator set per problem shape
 * (dim, n_cells, n_levels), shared by all requests of that shape and cached while
 * memory allows, and one workspace per admitted request. A submitted request waits
 * until a slot (max_active) and its memory are free, is then admitted at the next
 * iteration boundary, and leaves as soon as it converges; requests in flight share
 * every kernel launch: one launch per V-cycle phase covers that phase of all admitted
 * requests (tiles of 256 * rows_per_thread rows, blocks_per_sm persistent blocks per
 * SM), replayed as a CUDA graph. A request's result does not depend on the other
 * requests in flight (its arithmetic and reduction order are its own).
 * Requirements: element MG_Q1, k_cell NULL, n_levels >= 2, coarsest level <= 64 DOFs,
 * options.nu_pre >= 1, Chebyshev degree <= 4. The options are the server's; every
 * request uses them with options.precision forced to MG_MIXED.
 * Threads: one scheduler thread and one setup thread (host assembly of new shapes and
 * of right-hand sides given as mg_rhs) per server. Entry points are thread safe.
 * --------------------------------------------------------------------------------- */
typedef struct mg_server mg_server;

typedef struct {
    size_t hbm_budget_bytes; /* device memory reserved at creation and never exceeded */
    int max_active;          /* requests resident at once (1..4096) */
    int rows_per_thread;     /* tile shape: 1, 2, 4 or 8 rows per thread (256 threads) */
    int blocks_per_sm;       /* persistent blocks per SM of each phase launch (1..8) */
    mg_options options;      /* smoother, nu_pre/nu_post, max_iters, ... */
} mg_serve_config;

typedef struct {
    uint64_t completed;          /* requests finished (converged or max_iters) */
    uint64_t cycles;             /* batched iterations run */
    int active;                  /* admitted now */
    int queued;                  /* submitted, not admitted */
    int operator_sets;           /* cached problem shapes */
    double mean_batch;           /* mean admitted requests per iteration */
    double p50_ms, p99_ms, max_ms; /* latency submit -> completion of finished requests */
    double solves_per_s;         /* completed / (last completion - first submission) */
    size_t device_bytes_in_use, device_bytes_peak;
    double gpu_ms;               /* device time of the batched iterations (CUDA events) */
    double setup_ms;             /* busy time of the setup thread (operator sets, right-hand sides) */
    double span_ms;              /* first submission to last completion */
} mg_serve_stats;

/* Defaults: 4 GiB budget, 256 slots, 4 rows per thread, 4 blocks per SM, Chebyshev
 * degree 2 with one application before and after the coarse correction. */
void mg_serve_config_default(mg_serve_config *cfg);
/* Serving has no counterpart in the paper: it runs the solve of mg_solve (Sec. 5.3) for
 * many independent problems at once. cfg, dev: host structs (read only); *out is owned by
 * the library until mg_serve_destroy. MG_EINVAL for invalid options (Gauss-Seidel is not
 * served), MG_ENOMEM if the budget cannot be reserved, MG_ECUDA on a CUDA error. */
mg_status mg_serve_create(const mg_serve_config *cfg, const mg_device *dev, mg_server **out);
/* Submit A x = b (the system of Sec. 2, solved as mg_solve does) with b copied from
 * b_host (n doubles, host) before returning; the ticket identifies the request.
 * Relative tolerance on ||b - A x||_2 / ||b||_2. The request takes the server's options
 * (mg_serve_config.options): the phase launches of one iteration share one smoother.
 * MG_EINVAL for an unsupported problem, a tolerance <= 0, or a right-hand side holding a
 * NaN or an infinity. */
mg_status mg_serve_submit(mg_server *s, const mg_problem *p, const double *b_host, double rel_tol, uint64_t *ticket);
/* Submit with the right-hand side given by f (as mg_load_vector_separable); the load
 * vector is assembled on the server's setup thread. MG_EINVAL as mg_serve_submit, also
 * for a non-finite amplitude or f_const. */
mg_status mg_serve_submit_rhs(mg_server *s, const mg_problem *p, const mg_rhs *f, double rel_tol, uint64_t *ticket);
/* MG_PENDING while the request runs; otherwise its final status (MG_OK, MG_ENOCONV,
 * MG_EBUDGET, ...), with x copied to x_host (n doubles, may be NULL) and the V-cycle
 * count in iters. A finished request is forgotten after it has been returned once. */
mg_status mg_serve_poll(mg_server *s, uint64_t ticket, double *x_host, int *iters);
/* Blocking form of mg_serve_poll; MG_ETIMEOUT after timeout_s seconds. res_hist (may be
 * NULL) receives up to hist_len relative residuals, one per iteration. */
mg_status mg_serve_wait(mg_server *s, uint64_t ticket, double timeout_s, double *x_host, int *iters,
                        double *res_hist, int hist_len);
mg_status mg_serve_get_stats(mg_server *s, mg_serve_stats *out);
/* Clears the latency record and counters (for a measured run after warm-up). */
mg_status mg_serve_reset_stats(mg_server *s);
/* Autotuner for the tile shape of the phase launches: on an idle server, solves
 * `repeats` copies of each of the nshapes problems (f = 1, tolerance rel_tol) as one
 * batch for every candidate (rows per thread 1/2/4/8 x blocks per SM 2/4/8), keeps the
 * fastest and reports it. Resets the statistics. */
mg_status mg_serve_tune(mg_server *s, const mg_problem *shapes, int nshapes, int repeats, double rel_tol,
                        int *rows_per_thread, int *blocks_per_sm);
/* Stops the threads (requests in flight are dropped) and releases the budget. */
mg_status mg_serve_destroy(mg_server *s);

/* Thread-local description of the last error on this thread. */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
