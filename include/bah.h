/*
 * bah.h -- C ABI of the GB300 block-acoustic Helmholtz solver.
 *
 * Solves the mixed displacement-pressure form of the frequency-domain elastic
 * Helmholtz equation (Yovel & Treister, "A block-acoustic preconditioner for
 * the elastic Helmholtz equation", arXiv 2411.15897):
 *
 *     H [u; p] = [A  B^T; B  -C] [u; p] = b                          (Eq. 2.6)
 *
 * on a MAC-staggered grid (u_k on the x_k-faces; p, lambda, mu, rho, gamma at
 * cell centres), with flexible GMRES (FGMRES) preconditioned by the
 * block-triangular block-acoustic preconditioner P = [A B^T; 0 H_p]
 * (Eq. 3.5) applied as P^{-1} D with the distributor D = [I 0; B -A_p]
 * (Eq. 3.1-3.3), each acoustic diagonal block approximately inverted by one
 * shifted-Laplacian geometric-multigrid cycle (Sec. 2.2, Eq. 2.8, Sec. 4.4.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid:     n[0] x n[1] (x n[2]) cells, x_1 fastest, spacings h[0..dim-1].
 * Medium:   cell-centred FP64 host arrays of n[0]*n[1](*n[2]) values, x_1
 *           fastest: lambda, mu (Lame), rho (density), gamma (attenuation,
 *           absorbing layer included); angular frequency omega.  The system
 *           uses rho~ = rho (1 - i gamma/omega) in its mass terms (Eq. 2.6).
 * Vectors:  complex FP64 (interleaved re, im: 16 bytes per entry), padded
 *           layout of (dim+1) components of n[0]*n[1](*n[2]) entries each:
 *           component k < dim is u_{k+1}, stored at the cell whose lower
 *           x_k-face carries it; the entries with index 0 along x_k are the
 *           boundary-normal displacements, which are not unknowns (the
 *           normal displacement vanishes on the boundary): they are read as
 *           zero and written as zero.  Component dim is p.  nrhs vectors are
 *           stored one after another.
 * Pointers: vector arguments are DEVICE pointers on the current CUDA device
 *           unless an entry point says otherwise.  The caller owns every
 *           buffer it passes; the library owns its context and workspace,
 *           allocated in bah_create and released in bah_destroy.  Calls that
 *           take a stream enqueue their work on it (NULL = legacy default
 *           stream) and, unless stated, do not synchronise it.
 * Errors:   every int-returning call returns BAH_OK (0) or a negative
 *           status; bah_status_string names it and bah_last_error() gives
 *           the detail of the most recent failure on the calling thread.
 *           Nothing aborts or throws across this boundary.
 */
#ifndef BAH_H
#define BAH_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BAH_OK                 0
#define BAH_ERR_ARG           -1   /* invalid argument (pointer, size, option) */
#define BAH_ERR_OOM           -2   /* device or host allocation failed */
#define BAH_ERR_CUDA          -3   /* a CUDA runtime call failed */
#define BAH_ERR_NOT_CONVERGED -4   /* maxit reached; x holds the last iterate */
#define BAH_ERR_NONFINITE     -5   /* NaN/Inf met in a reduction; x holds the last finite iterate */
#define BAH_ERR_UNSUPPORTED   -6   /* a valid request the library does not implement (3-D options and
                                      calls listed at bah_create) */

/* precision of the preconditioner.  The coarsest-level inverse is computed in
 * FP64 and applied in FP64 arithmetic in both modes; the outer
 * FGMRES keeps its Hessenberg update, Givens rotations, true residual and
 * solution in FP64 in both modes (see krylov_arith for the basis) */
#define BAH_FP64   0   /* multigrid in complex FP64 with FP64 coefficients */
#define BAH_MIXED  1   /* multigrid in complex FP32, coefficients and stencils stored in bfloat16 */

/* arithmetic of the Krylov basis (Gram-Schmidt dots and updates, and, in
 * BAH_MIXED mode, the operator w = H z and the update x += Z y on the FP32
 * flexible basis); the Hessenberg least-squares update, the true residual and
 * x are FP64 always */
#define BAH_KRYLOV_FP64 0  /* IEEE FP64 */
#define BAH_KRYLOV_DF   1  /* double-FP32: each real is an FP32 pair hi + lo (48-bit significand),
                              products and sums by error-free FP32 transformations */

#define BAH_CYCLE_V 0
#define BAH_CYCLE_W 1

#define BAH_INTERGRID_BILINEAR 0   /* Eq. 4.1, 4.2: 1/4[1 2 1], 1/8[1 3 * 3 1] */
#define BAH_INTERGRID_MIXED    1   /* Eq. 4.4: 1/2[1 * 1] along cell-centred axes */

typedef struct bah_ctx bah_ctx;    /* opaque, owned by the library */

typedef struct {
    int    dim;      /* 2 or 3 */
    int    n[3];     /* cells along x_1, x_2, x_3 (n[2] ignored in 2D) */
    double h[3];     /* cell size along each axis */
} bah_grid;

typedef struct {
    const double* lambda;   /* host, cell-centred, x_1 fastest */
    const double* mu;
    const double* rho;
    const double* gamma;    /* attenuation incl. the absorbing layer */
    double        omega;    /* angular frequency, > 0 */
} bah_medium;

typedef struct {
    int    precision;        /* BAH_FP64 or BAH_MIXED */
    int    levels;           /* multigrid levels incl. the fine level; 0 = automatic */
    int    max_coarse_cells; /* automatic levels: coarsen until a level has at most this many cells */
    int    cycle;            /* BAH_CYCLE_V or BAH_CYCLE_W */
    int    nu_pre, nu_post;  /* damped-Jacobi sweeps before / after the coarse correction */
    double jacobi_w[8];      /* damping per level (the last value repeats on deeper levels) */
    int    n_jacobi_w;
    double shift_alpha;      /* complex shift alpha of Eq. 2.8; < 0 = by level count */
    int    intergrid;        /* BAH_INTERGRID_* */
    int    restart;          /* FGMRES restart length m (1..64) */
    int    maxit;            /* maximum FGMRES iterations per right-hand side */
    int    rhs_block;        /* right-hand sides solved together by bah_solve (1..256); the
                                context's workspace grows in proportion */
    int    krylov_arith;     /* BAH_KRYLOV_FP64 or BAH_KRYLOV_DF */
    /* acoustic block solves.  block_rtol = 0: each block is approximately
     * inverted by one multigrid cycle (Sec. 2.2, 4.4).  block_rtol > 0: each
     * block is solved to ||s - M e|| <= block_rtol ||s|| by an inner FGMRES in
     * FP64, preconditioned by that block's multigrid cycle -- the exact-block
     * preconditioner of Sec. 4.1 (Table 2) and of Theorem 1 (Sec. 3) as
     * block_rtol -> 0, at any grid size (inner restart length 60).  The blocks solved are shifted by
     * block_alpha (Eq. 2.8; 0 = the unshifted blocks of Eq. 3.5), while the
     * multigrid cycle keeps shift_alpha.  2-D, rhs_block = 1 only. */
    double block_rtol;
    int    block_maxit;      /* inner iterations per block solve (block_rtol > 0) */
    double block_alpha;
    /* outer Krylov method for a batch of right-hand sides: 0 = independent FGMRES
     * recurrences advanced in lockstep; 1 = block FGMRES, one Krylov space for
     * the batch (block Arnoldi with two passes of block classical Gram-Schmidt
     * and CholQR2, the block Hessenberg least squares by Householder
     * reflections); needs 2-D, 2 <= rhs_block <= 16, BAH_KRYLOV_FP64 and
     * nonzero right-hand sides.  The iteration count of a block solve is the
     * same for all its right-hand sides. */
    int    block_krylov;
} bah_opts;

typedef struct {
    int    iters;            /* FGMRES iterations (preconditioner applications) */
    int    restarts;         /* restart cycles run */
    double relres_true;      /* ||b - H x|| / ||b|| in FP64 at exit */
    double relres_est;       /* Arnoldi estimate at exit */
    int    status;           /* BAH_OK, BAH_ERR_NOT_CONVERGED or BAH_ERR_NONFINITE */
} bah_stats;

/* Fill *opts with the defaults: BAH_MIXED, automatic levels with at most 256
 * coarsest cells, V(1,2), Jacobi weights 0.8, 0.8, 0.3 (Sec. 4.4.1), shift by
 * level count (0.1 / 0.2 / 0.4 for 2 / 3 / 4 levels as in Sec. 4.4.3,
 * Table 4; 1.0 for deeper hierarchies, found by the same kind of search),
 * bilinear intergrid, FGMRES(20), maxit 5000, rhs_block 1, BAH_KRYLOV_FP64,
 * one multigrid cycle per block (block_rtol 0; block_maxit 2000, block_alpha 0),
 * lockstep batches (block_krylov 0). */
void bah_default_opts(bah_opts* opts);

/* Build a solver for one grid, medium and frequency.  Copies the host medium
 * to the device, forms the operator coefficients (Eq. 2.6), the distributor
 * (Eq. 3.2), the shifted acoustic blocks A_k,s and H_p,s (Eq. 2.8, 3.4), their
 * Galerkin hierarchies R A P (Eq. 4.3) and the FP64 inverse of every coarsest
 * block, and allocates all solve workspace.  Synchronous.  *out receives the
 * context; on failure *out is NULL and nothing is leaked.
 * block_rtol > 0 needs a 2-D grid and rhs_block = 1 (else BAH_ERR_UNSUPPORTED).
 * 3-D grids (dim 3) follow the paper's 3-D multigrid (Sec. 4.5): they need
 * intergrid = BAH_INTERGRID_MIXED (Eq. 4.4; with it every Galerkin level is a
 * 27-point stencil), krylov_arith = BAH_KRYLOV_FP64 and at least 2 levels; the
 * paper's W(2,2) cycle with Jacobi weights 0.8, 0.8, 0.2 is set through
 * cycle, nu_pre, nu_post and jacobi_w.  On a 3-D context bah_gradient,
 * bah_level_stencil and bah_residual_norm_static return BAH_ERR_UNSUPPORTED.
 * Errors: BAH_ERR_ARG (dim not 2 or 3, odd or too small sizes for the
 * requested levels, a coarsest level above 4096 cells, non-positive h or
 * omega, NULL arrays, a 3-D grid with one level), BAH_ERR_UNSUPPORTED (3-D with
 * the bilinear intergrid or the double-FP32 basis), BAH_ERR_OOM,
 * BAH_ERR_CUDA. */
int bah_create(const bah_grid* grid, const bah_medium* medium, const bah_opts* opts, bah_ctx** out);

/* Release the context and all device memory it owns.  NULL is ignored.  The
 * caller must make sure no work enqueued on the context is still running. */
void bah_destroy(bah_ctx* ctx);

/* Entries of one padded vector ((dim+1) * cells) and the number of multigrid
 * levels in use.  Either output pointer may be NULL. */
int bah_sizes(const bah_ctx* ctx, long long* vector_len, int* levels);

/* What the context chose (after defaults were applied): level count, the
 * shift alpha of Eq. 2.8, the coarsest grid's point count, and the first
 * level held in a thread-block cluster's shared memory (0: none) with the
 * CTAs per cluster and the bytes of shared memory per CTA.  The paper has no
 * counterpart; this is for reporting and tests. */
typedef struct {
    int       levels;
    double    shift_alpha;
    int       coarse_points;
    int       cluster_level;
    int       cluster_ctas;
    long long cluster_smem_bytes;
    long long block_iters;    /* inner FGMRES iterations of all block solves so far (block_rtol > 0) */
    int       block_failures; /* block solves that stopped at block_maxit above block_rtol */
} bah_info;
int bah_get_info(const bah_ctx* ctx, bah_info* out);

/* y = H x (conj_transpose = 0) or y = H^H x (conj_transpose = 1) in FP64 for
 * nrhs vectors (Eq. 2.6; H is complex symmetric, so H^H = conj(H)).  x and y
 * are device vectors and must not overlap. */
int bah_apply_operator(bah_ctx* ctx, const void* x, void* y, int nrhs, int conj_transpose, void* stream);

/* z = P^{-1} D r: one block-acoustic preconditioning step (Eq. 3.1-3.5):
 *   t_p = B r_u - A_p r_p;  e_p ~ H_p,s^{-1} t_p;  e_u ~ A_s^{-1}(r_u - B^T e_p)
 * with one multigrid cycle per block, in the context's precision.  r, z
 * device vectors (FP64), must not overlap. */
int bah_apply_preconditioner(bah_ctx* ctx, const void* r, void* z, int nrhs, void* stream);

/* Solve H x = b to ||b - H x||_2 <= rtol ||b||_2 by FGMRES(m) with the
 * block-acoustic preconditioner, x_0 = 0, for nrhs right-hand sides.
 * Right-hand sides are solved rhs_block at a time in one batch: each keeps its
 * own Krylov basis and converges on its own, while every kernel launch
 * (stencils, multigrid levels, Gram-Schmidt) serves the whole batch and
 * skips the members that have converged.  b and x
 * may both be device pointers, or both host pointers (then the copies to and
 * from the device are part of the call).  Synchronises the stream before
 * returning.  stats (may be NULL) receives nrhs records.  Returns BAH_OK when
 * every right-hand side converged, else the first failing status
 * (BAH_ERR_NOT_CONVERGED / BAH_ERR_NONFINITE) after solving all of them. */
int bah_solve(bah_ctx* ctx, const void* b, void* x, int nrhs, double rtol, bah_stats* stats, void* stream);

/* Solve the adjoint system H^H y = b (same options and stopping rule as
 * bah_solve).  H is complex symmetric (Eq. 2.6), so H^H = conj(H) and the
 * call solves H conj(y) = conj(b) with the same preconditioner. */
int bah_solve_adjoint(bah_ctx* ctx, const void* b, void* y, int nrhs, double rtol, bah_stats* stats, void* stream);

/* Receiver misfit of a least-squares data fit.  Q samples the entries
 * rec[0..nrec-1] (device int array of indices into one padded vector, e.g.
 * the u_d faces of a receiver line) of each solution x_s; d holds the
 * observed data, nrec complex values per source (device).  Writes
 * adj_s = Q^H (Q x_s - d_s) (nrhs full padded vectors, zero off the
 * receivers) and misfit[s] = 1/2 ||Q x_s - d_s||^2 (device, nrhs doubles).
 * An index listed more than once is a receiver counted more than once: its
 * data enter J once per listing and adj_s sums the residuals of every
 * listing (added in the order of rec).  Indices must lie in
 * [0, vector_len); they are not checked on the device. */
int bah_misfit(bah_ctx* ctx, const void* x, const void* d, const int* rec, int nrec, int nrhs, void* adj_src,
               double* misfit, void* stream);

/* Gradient of J = sum_s 1/2 ||Q x_s - d_s||^2 with respect to the cell values
 * of lambda, mu and rho, given the forward solutions x_s (H x_s = b_s) and
 * the adjoint solutions y_s (H^H y_s = Q^H (Q x_s - d_s)):
 *     dJ/dm_k = -Re sum_s y_s^H (dH/dm_k) x_s .
 * dH/dm_k follows Eq. 2.6: lambda enters -C = -diag(1/(lambda+mu)), mu enters
 * the edge-averaged A_e(mu) and C, rho the face mass A_f(rho(1 - i gamma/omega)).
 * The paper does not write this gradient (it uses the solver inside
 * full-waveform inversion); this is the adjoint-state derivative of the
 * discrete system.  g_lambda, g_mu, g_rho: device arrays of cells doubles,
 * ACCUMULATED into (zero them first).  FP64, one kernel. */
int bah_gradient(bah_ctx* ctx, const void* x_fwd, const void* y_adj, int nrhs, double* g_lambda, double* g_mu,
                 double* g_rho, void* stream);

/* Spectral radius of the preconditioned fixed-point iteration's error
 * operator T = I - P^{-1} D H (Sec. 3: with exact blocks, Theorem 1 gives
 * rho(T) = rho(Z), Z = Xi A^{-1} B^T H_p^{-1}; the paper estimates it by the
 * power method on a matrix-free product).  Power method from the device
 * vector x0 (FP64 complex, the vector layout above, not modified):
 * x_{k+1} = T x_k / ||T x_k||, with x_0 = x0 / ||x0||, for iters >= 1 steps,
 * using the context's preconditioner (exact blocks with levels = 1, else its
 * multigrid cycles).  history (host, iters doubles, may be NULL) receives
 * ||T x_k||; *rho the geometric mean of the last quarter of the history.
 * Uses the context's Krylov workspace (no solve may run on the context at the
 * same time).  Synchronous on the given stream. */
int bah_spectral_radius(bah_ctx* ctx, const void* x0, int iters, double* history, double* rho, void* stream);

/* Spectral radius of Z = Xi A_s^{-1} B^T H_p,s^{-1} (Theorem 1, Sec. 3), the
 * operator whose spectrum, with {0}, is that of T when the blocks are solved
 * exactly; Xi = B A - A_p B is the commutator of Eq. 3.2 (unshifted blocks)
 * and A_s, H_p,s the blocks shifted by the context's block_alpha (Eq. 2.8),
 * solved by the context's exact block solves.  Power method as in the paper
 * (a matrix-free product with Z): x_{k+1} = Z x_k / ||Z x_k|| from the device
 * vector x0 of cells complex FP64 values on the pressure lattice (not
 * modified), iters >= 1 steps; history (host, may be NULL) receives
 * ||Z x_k||, *rho the geometric mean of the last quarter.  Needs a 2-D context
 * with block_rtol > 0 (else BAH_ERR_UNSUPPORTED); uses the context's Krylov
 * workspace (no solve may run on it at the same time).  Synchronous. */
int bah_spectral_radius_z(bah_ctx* ctx, const void* x0, int iters, double* history, double* rho, void* stream);

/* Test hook: one multigrid cycle (the context's cycle type) on acoustic block
 * `block` (0..dim-1 = A_{block+1},s; dim = H_p,s) with zero initial guess.
 * b and x are device arrays of cells complex FP64 values in the padded
 * per-component layout of that block. */
int bah_block_cycle(bah_ctx* ctx, int block, const void* b, void* x, void* stream);

/* Test hook: copy the FP64 operator of block `block` on level `level` to the
 * host.  Level 0 gives the fine shifted block as a 3x3 stencil, coarser
 * levels the Galerkin stencil (Eq. 4.3) of radius (rx, rz) written to *rx,
 * *rz.  out receives (2rz+1)(2rx+1) slots x points complex values
 * (slot-major, slot index (dz+rz)(2rx+1) + (dx+rx)); out may be NULL to query
 * the radii.  Synchronous. */
int bah_level_stencil(const bah_ctx* ctx, int block, int level, double* out, int* rx, int* rz, int* n1, int* n2);

/* ---------------------------------------------------------------------------
 * Profiling.  Every context counts the kernels it launches and, per kernel
 * class, the algorithmic bytes those launches must move (the minimum traffic:
 * each input and output array touched once, coefficients once per launch).
 * For the classes set in timing_mask (bit 1 << BAH_K_*), each launch is also
 * bracketed by CUDA events recorded on the launching stream, and the summed
 * device time is reported.  Timing adds two event records per timed launch.
 * ------------------------------------------------------------------------- */
#define BAH_K_OPERATOR  0   /* y = H x or b - H x, FP64 (Eq. 2.6) */
#define BAH_K_DISTRIB   1   /* t_p = B r_u - A_p r_p (Eq. 3.1-3.3) */
#define BAH_K_URHS      2   /* s_u = r_u - B^T e_p (Eq. 3.5) */
#define BAH_K_JACOBI    3   /* damped Jacobi sweep, all levels */
#define BAH_K_RESIDUAL  4   /* multigrid residual, all levels */
#define BAH_K_RESTRICT  5   /* restriction (Eq. 4.1, 4.2, 4.4) */
#define BAH_K_PROLONG   6   /* prolongation + correction */
#define BAH_K_COARSE    7   /* coarsest-level FP64 inverse applied in FP64 */
#define BAH_K_DOT       8   /* Gram-Schmidt block dot products (2 kernels) */
#define BAH_K_AXPY      9   /* Gram-Schmidt update w -= V h */
#define BAH_K_NORM     10   /* 2-norms (2 kernels) */
#define BAH_K_UPDATE   11   /* x += Z y */
#define BAH_K_SMALL    12   /* Givens update, triangular solve, scaling, copies, conversions */
/* class 13 is unused */
#define BAH_K_CLUSTER  14   /* thread-block-cluster launch running the small levels of a cycle */
/* class 15 is unused */
#define BAH_NKCLASS    16

typedef struct {
    long long launches;             /* kernels launched since the last reset */
    long long class_launches[16];   /* kernels per class */
    long long class_calls[16];      /* launcher calls per class (a call may launch 2 kernels) */
    double    class_ms[16];         /* summed device time per timed class (ms) */
    double    class_bytes[16];      /* summed algorithmic bytes per class */
} bah_profile;

/* Select the timed classes (bit mask of 1 << BAH_K_*) and optionally zero the
 * counters (reset != 0).  Pending timings are folded in first.  Synchronous. */
int bah_profile_control(bah_ctx* ctx, unsigned timing_mask, int reset);

/* Read the counters (waits for pending timing events).  Synchronous. */
int bah_profile_read(bah_ctx* ctx, bah_profile* out);

/* ---------------------------------------------------------------------------
 * Allocation-free relative residual.  The paper has no counterpart: this is a
 * service for callers that cannot call cudaMalloc at the point where they
 * need the number -- real-time loops that forbid allocator calls after
 * start-up (an allocation can block for an unbounded time), and hosts whose
 * device memory all belongs to another allocator (a framework's caching
 * pool, which a direct cudaMalloc would bypass or find exhausted).
 *
 * relres[k] = ||b_k - H x_k||_2 / ||b_k||_2 (0 when b_k = 0) for k < nrhs,
 * written to the DEVICE array relres (nrhs doubles) on the stream, without
 * synchronising.  b, x: nrhs device vectors in the layout above
 * (boundary-normal entries read as zero).  2-D contexts only.
 *
 * Scratch: the per-block partial sums live in one file-scope device array of
 * 2 * BAH_STATIC_MAX_RHS * 296 doubles (296 KiB), which every GPU that loads
 * the library holds until the process exits.  The call launches two kernels
 * and allocates nothing (no cudaMalloc, no allocating library routine).
 * The first call on a device looks up that array's device address with the
 * device current and keeps it; make that first call before any stream
 * capture, and do not call this function on a device after cudaDeviceReset
 * (which unloads the array).  Every call overwrites the slots it reads, so
 * nothing needs clearing, but all calls share the array: calls that overlap
 * on the GPU (other streams or threads) race and must be serialised by the
 * caller.
 * Errors: BAH_ERR_ARG (NULL pointer, nrhs < 0, nrhs > BAH_STATIC_MAX_RHS),
 * BAH_ERR_UNSUPPORTED (a 3-D context), BAH_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define BAH_STATIC_MAX_RHS 64
int bah_residual_norm_static(bah_ctx* ctx, const void* b, const void* x, int nrhs, double* relres, void* stream);

/* Name of a status code (static string). */
const char* bah_status_string(int status);

/* Detail of the most recent failure on the calling thread ("" if none). */
const char* bah_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BAH_H */
