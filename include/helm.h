/*
 * helm.h -- C ABI of libhelm, a GB300 (sm_103a) solver for the heterogeneous
 * Helmholtz equation, right-preconditioned by the shifted Laplacian.
 *
 * Method (Kazemi, "Application of shifted-Laplace preconditioners for
 * heterogenous Helmholtz equation, part 1: Data modelling"):
 *   Eq. 2   -Lap u - omega^2 m^2 (1 - j alpha) u = f, m = 1/c the slowness,
 *           first-order absorbing boundary on every face (Summary, Eq. 1).
 *   Eq. 3   H u = f, the discrete system.
 *   Eq. 6   shifted Laplacian, written here as
 *           M = -Lap - (beta1 - j beta2) omega^2 m^2 (same boundary rows as H).
 *           The paper's P = -Lap + beta k^2 with beta = b1 + j b2 is
 *           M with (beta1, beta2) = (-b1, b2).
 *   Eq. 7   H M^-1 z = f, u = M^-1 z, solved by restarted flexible GMRES.
 *
 * Discretisation: second-order finite differences on a node grid; every
 * node is an unknown. Boundary rows use a centred ghost node for
 * dn u + j kappa u = 0 with kappa = omega m sqrt(1 - j alpha).
 *
 * Layout of every field: x fastest, index (iz * ny + iy) * nx + ix (2D:
 * iz * nx + ix), complex values interleaved (re, im) as helm_c128, i.e. the
 * memory layout of double2 / cuDoubleComplex / numpy complex128.
 *
 * Pointers: every array argument may be a host pointer or a CUDA device
 * pointer of the current device; the library tells them apart with
 * cudaPointerGetAttributes. Host arrays are staged through library-owned
 * device buffers; device arrays are read and written in place on the grid's
 * stream. The caller keeps ownership of every array it passes. The library
 * owns the grid and all its device memory (model, multigrid hierarchy,
 * Krylov basis) until helm_destroy_grid.
 *
 * Errors: every call returns a helm_status. On failure helm_last_error()
 * returns a message for the calling thread. A grid is not thread-safe;
 * distinct grids may be used from distinct threads.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_grid helm_grid;               /* opaque, library-owned */
typedef struct { double re, im; } helm_c128;      /* == double2 */

typedef enum {
    HELM_OK = 0,
    HELM_ERR_ARG = 1,            /* bad argument (null, size, range)               */
    HELM_ERR_NOMEM = 2,          /* device allocation failed                         */
    HELM_ERR_CUDA = 3,           /* a CUDA call failed                               */
    HELM_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; u holds the last iterate  */
    HELM_ERR_BREAKDOWN = 5,      /* Arnoldi produced a non-finite or zero pivot      */
    HELM_ERR_NONFINITE = 6,      /* input contains NaN or Inf                         */
    HELM_ERR_STATE = 7,          /* call order violated (e.g. solve before model)    */
    HELM_ERR_UNSUPPORTED = 8     /* option or grid shape the build cannot handle      */
} helm_status;

/* How M^-1 is applied inside the Krylov loop. */
typedef enum {
    HELM_PRECOND_MG = 0,     /* one geometric-multigrid V-cycle (default)            */
    HELM_PRECOND_EXACT = 1,  /* dense inverse of M (grids up to 4096 nodes)            */
    HELM_PRECOND_NONE = 2    /* M = I: plain GMRES, the paper's comparison arm        */
} helm_precond;

/* Arithmetic. The Givens/Hessenberg least squares, the solution update and
 * the true residual are always complex128. */
typedef enum {
    HELM_PREC_F64 = 0,       /* V-cycle and Arnoldi in complex128                      */
    HELM_PREC_MIXED = 1,     /* V-cycle in complex64 (z stored in complex64), Arnoldi   */
                             /* orthogonalisation in complex128                        */
    HELM_PREC_MIXED_DS = 2,  /* as MIXED, but the Arnoldi basis is stored and           */
                             /* orthogonalised in double-single arithmetic (pairs of   */
                             /* FP32 values, ~48-bit significands, FP32 pipe); H z,    */
                             /* Hessenberg, norms and the true residual in complex128  */
    HELM_PREC_MIXED_C64 = 3  /* as MIXED_DS, but the basis vectors are stored in        */
                             /* complex64 (half the bytes the Gram-Schmidt passes      */
                             /* stream); w = H z and its orthogonalisation stay        */
                             /* double-single until v_{j+1} = w / ||w|| is rounded.     */
                             /* Needs side RIGHT, reorth 0, precond MG or EXACT and a  */
                             /* constant density                                       */
} helm_precision;

/* Where M^-1 enters the Krylov operator (Eq. 5: Ml^-1 H Mr^-1 z = Ml^-1 f,
 * u = Mr^-1 z). The paper solves Eq. 7, i.e. Ml = I, Mr = M. */
typedef enum {
    HELM_SIDE_RIGHT = 0,     /* Ml = I, Mr = M (Eq. 7, default): flexible GMRES;       */
                             /* stops on ||f - H u|| <= tol ||f||                       */
    HELM_SIDE_LEFT = 1,      /* Ml = M, Mr = I: GMRES on M^-1 H u = M^-1 f              */
    HELM_SIDE_SPLIT = 2      /* Ml = Mr = M: GMRES on M^-1 H M^-1 z = M^-1 f            */
    /* LEFT and SPLIT minimise, and stop on, the preconditioned residual:        */
    /* ||M^-1 (f - H u)|| <= tol ||M^-1 f||. They need a fixed M^-1 (the V-cycle  */
    /* or the dense inverse) and a complex128 Arnoldi basis (not                 */
    /* HELM_PREC_MIXED_DS); with HELM_PRECOND_NONE the side has no effect.       */
} helm_side;

typedef struct {
    int restart;             /* Krylov dimension m per cycle (1..256); default 30     */
    int max_iters;           /* cap on inner iterations over all cycles; default 5000 */
    int precond;             /* helm_precond                                          */
    int precision;           /* helm_precision                                        */
    int nu1, nu2;            /* damped-Jacobi sweeps before / after coarse correction */
    double omega_jacobi;     /* Jacobi damping weight, (0, 1]; default 0.8            */
    int coarse_max;          /* coarsen while a level has more nodes than this         */
    int reorth;              /* Gram-Schmidt: 0 classical once (default); 1 classical  */
                             /* twice; 2 twice only where the first pass cancels more */
                             /* than half of ||w||^2 (DGKS test). The true residual   */
                             /* is recomputed after every cycle in all three.        */
    int graphs;              /* 1: replay each Arnoldi step as a captured CUDA graph   */
                             /*    (default); 0: launch kernels one by one             */
    int side;                /* helm_side; default HELM_SIDE_RIGHT                     */
    int block;               /* 0: the right-hand sides of a batch run as independent  */
                             /*    recurrences in lock-step (default); 1: block FGMRES */
                             /*    -- up to 64 sources share one block Krylov space    */
                             /*    (see helm_solve_batch)                              */
    int recycle;             /* k = 0 (default): none; 1..16: GCRO-DR, k recycled      */
                             /*    vectors per right-hand side kept across restarts   */
                             /*    and across solves (see helm_solve_batch)            */
} helm_options;

/* Fills *opt with the defaults listed above. */
void helm_default_options(helm_options *opt);

/* Creates a grid of n[0] x n[1] x n[2] nodes (unused axes: 1) with spacing
 * h > 0 in metres. dim is 1, 2 or 3; every used axis needs >= 2 nodes.
 * Device memory for the fine-level vectors is allocated here.
 * Errors: HELM_ERR_ARG, HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_create_grid(int dim, const int64_t n[3], double h, helm_grid **out);

/* Releases every device buffer of the grid. Null is ignored. */
void helm_destroy_grid(helm_grid *g);

/* Sets the CUDA stream (a cudaStream_t, may be 0) for all later work. */
helm_status helm_set_stream(helm_grid *g, void *stream);

/* Replaces the solver options. Takes effect at the next solve; a change of
 * coarse_max, precond or precision rebuilds the hierarchy.
 * Errors: HELM_ERR_ARG on an out-of-range field. */
helm_status helm_set_options(helm_grid *g, const helm_options *opt);

/* Copies the grid's current options into *opt (caller-owned).
 * Errors: HELM_ERR_ARG on a null argument. */
helm_status helm_get_options(const helm_grid *g, helm_options *opt);

/* Eq. 2: sets the medium and frequency. m: slowness 1/c in s/m, one real
 * double per node (host or device), all finite and > 0. omega: angular
 * frequency in rad/s (> 0). alpha: damping (>= 0). The library copies m.
 * Invalidates the preconditioner; it is rebuilt at the next solve or
 * helm_set_shift. Errors: HELM_ERR_ARG, HELM_ERR_NONFINITE, HELM_ERR_CUDA. */
helm_status helm_set_model(helm_grid *g, const double *m, double omega, double alpha);

/* Eq. 1: sets a variable density. rho: one real double per node (host or
 * device), all finite and > 0, the coefficient inside the divergence as the
 * paper prints it (-div(rho grad u) - omega^2 m^2 (1 - j alpha) u = f; for the
 * acoustic equation pass 1/density). Null removes it (rho = 1, Eq. 2). The
 * library copies rho. Discretisation: each face between two neighbours takes
 * the mean of rho at its two nodes; a boundary face absorbs with the local
 * wavenumber kappa / sqrt(rho) (ghost face mirrored from the inner face). M
 * keeps the same -div(rho grad) and boundary rows (Eq. 6 with rho), so H - M
 * stays diagonal; coarser levels inject rho like the slowness. With a density
 * the V-cycle runs the general (unfused) level kernels, and the
 * HELM_PREC_MIXED_DS and HELM_PREC_MIXED_C64 bases, helm_apply_H_ds and
 * helm_true_residual_noalloc are not available (HELM_ERR_UNSUPPORTED). Invalidates the preconditioner.
 * Errors: HELM_ERR_ARG, HELM_ERR_NONFINITE, HELM_ERR_UNSUPPORTED,
 * HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_set_density(helm_grid *g, const double *rho);

/* Eq. 6: sets the shift (beta1, beta2) of M = -Lap - (beta1 - j beta2) w^2 m^2
 * and builds the multigrid hierarchy and the coarse-grid inverse on the
 * device. Default (1, 0.5). Errors: HELM_ERR_STATE (no model),
 * HELM_ERR_UNSUPPORTED (grid cannot be coarsened to coarse_max, or an exact
 * preconditioner on more than 4096 nodes), HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_set_shift(helm_grid *g, double beta1, double beta2);

/* Eq. 7: solves H u = f by restarted flexible GMRES, right-preconditioned
 * by M, from u0 = 0, until ||f - H u||_2 / ||f||_2 <= tol (recomputed in
 * complex128 after each cycle). With options.side LEFT or SPLIT it runs GMRES
 * on Eq. 5 instead and stops on the preconditioned residual (see helm_side).
 * f, u: N complex values (host or device, not overlapping). iterations
 * (nullable): inner iterations used. true_rel_residual (nullable): the final
 * true relative residual ||f - H u||_2 / ||f||_2 (on every side).
 * Errors: HELM_ERR_STATE, HELM_ERR_ARG, HELM_ERR_NONFINITE (f not finite),
 * HELM_ERR_NOT_CONVERGED (u holds the last iterate), HELM_ERR_BREAKDOWN,
 * HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_solve(helm_grid *g, const helm_c128 *f, double tol, helm_c128 *u,
                       int *iterations, double *true_rel_residual);

/* Solves nrhs independent systems with the same H and M in one pass: every
 * kernel launch of the Krylov loop covers all right-hand sides, each with
 * its own Krylov space, Hessenberg matrix and stopping test. f, u: nrhs x N
 * complex values, right-hand side k at offset k*N. iterations and
 * true_rel_residual (nullable): nrhs entries each. Returns HELM_OK when all
 * converged, HELM_ERR_NOT_CONVERGED if any did not. Other errors as
 * helm_solve.
 *
 * With options.block = 1 the sources, in groups of up to 64, run block
 * flexible GMRES (Eq. 7): one block Krylov space per group, widened by one
 * vector per source at every block step, so each source minimises its
 * residual over the whole group's space. The basis is complex64; the Gram
 * matrices V^H W and the block updates run on the tensor cores (TF32 with a
 * hi/lo split, FP32 accuracy); the block Hessenberg least squares, the
 * solution and the true residual stay complex128, and a group restarts until
 * every true residual is <= tol. iterations then counts block steps. Needs
 * precision HELM_PREC_MIXED, precond MG or EXACT, side RIGHT and restart <= 32
 * (HELM_ERR_UNSUPPORTED otherwise, from helm_set_options).
 *
 * With options.recycle = k > 0 each right-hand side runs GCRO-DR: restarted
 * GMRES (Eq. 7) that keeps k recycled vectors U (with C = H U orthonormal)
 * and orthogonalises every Krylov vector against C as well. A cycle that
 * ends unconverged replaces them by the k harmonic Ritz vectors of the
 * smallest magnitude over the recycled and the new Krylov vectors, so slowly
 * converging directions are deflated across restarts. The recycled vectors
 * stay in the grid after the call: the next call with the same nrhs (e.g. the
 * next frequency of a sweep, after helm_set_model) rebuilds U and C for the
 * new H and M and starts with them, the initial guess gaining the part of
 * the solution they carry. A change of nrhs, restart, k or precision starts
 * empty; a right-hand side whose solve never ran a full cycle of restart
 * steps has none yet. Each right-hand side's result is the same alone and in
 * any batch. Needs precision HELM_PREC_F64 or HELM_PREC_MIXED, precond MG or
 * EXACT, side RIGHT, reorth 0, block 0, k <= restart <= 40. */
helm_status helm_solve_batch(helm_grid *g, int nrhs, const helm_c128 *f, double tol,
                             helm_c128 *u, int *iterations, double *true_rel_residual);

/* As helm_solve_batch, but restarted FGMRES starts from the initial guess x0
 * that u holds on entry instead of from 0 (Eq. 7 with x0 given; e.g. the
 * solution of the same source at the previous frequency of a sweep). u:
 * nrhs x N complex values, read as x0 and overwritten by the solution; host
 * or device. The stopping test stays ||f - H u||_2 / ||f||_2 <= tol; a
 * right-hand side whose x0 already meets it returns x0 with 0 iterations,
 * and one with f = 0 returns u = 0. Errors as helm_solve_batch, with
 * HELM_ERR_NONFINITE also for a non-finite x0. */
helm_status helm_solve_batch_warm(helm_grid *g, int nrhs, const helm_c128 *f, double tol,
                                  helm_c128 *u, int *iterations, double *true_rel_residual);

/* Eq. 3: y = H x on the fine grid (x, y: N complex values, host or device,
 * not overlapping). Errors: HELM_ERR_STATE, HELM_ERR_ARG, HELM_ERR_CUDA. */
helm_status helm_apply_H(helm_grid *g, const helm_c128 *x, helm_c128 *y);

/* Eq. 3 in the arithmetic of the double-single Arnoldi step: x is rounded
 * (truncated) to complex64, as the preconditioned vectors of that step are,
 * and y = H x is formed with FP32 error-free products and two-sums (about 48
 * significant bits) and returned as complex128. x, y: N complex values, host
 * or device, not overlapping. Errors as helm_apply_H, plus HELM_ERR_NOMEM. */
helm_status helm_apply_H_ds(helm_grid *g, const helm_c128 *x, helm_c128 *y);

/* Eq. 6: y = M x on multigrid level `level` (0 = fine grid), in the grid's
 * preconditioner arithmetic. x, y: the level's node count of complex values.
 * Errors: HELM_ERR_STATE, HELM_ERR_ARG, HELM_ERR_CUDA. */
helm_status helm_apply_M(helm_grid *g, int level, const helm_c128 *x, helm_c128 *y);

/* Eq. 7, inner step: z = M^-1 r as applied inside the Krylov loop (one
 * V-cycle, the dense inverse, or a copy), in the preconditioner's
 * arithmetic. r, z: N complex values. Errors as helm_apply_H. */
helm_status helm_apply_precond(helm_grid *g, const helm_c128 *r, helm_c128 *z);

/* The true relative residual ||f - H u||_2 / ||f||_2 in complex128.
 * Errors: HELM_ERR_STATE, HELM_ERR_ARG, HELM_ERR_CUDA. */
helm_status helm_true_residual(helm_grid *g, const helm_c128 *f, const helm_c128 *u,
                               double *rel);

/* Allocation-free variant of helm_true_residual for nrhs right-hand sides:
 * rel[k] = ||f_k - H u_k||_2 / ||f_k||_2 in complex128, f_k and u_k at
 * offset k*N of the device arrays f and u (both must be device pointers of
 * the current device, each holding at least nrhs*N values; nothing is
 * staged). The paper has no counterpart.
 *
 * Who needs it: callers that cannot call cudaMalloc. A serving process that
 * reserves the GPU's memory up front and hands it out from its own pool
 * leaves nothing for cudaMalloc to take, and a caller that must not stall
 * other streams cannot afford cudaMalloc/cudaFree, which may synchronise the
 * device. helm_true_residual may allocate staging and reduction buffers on
 * first use; this entry point allocates nothing (no cudaMalloc or cudaFree,
 * no allocating library call). Its scratch is one static device array of
 * 305 KiB inside the library, which every GPU that loads the library holds
 * until the process exits. Limits and behaviour:
 *  - nrhs must be 1..64 (the size of that array); larger values return
 *    HELM_ERR_ARG;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current;
 *  - it must not be called while a stream is being captured into a CUDA
 *    graph (it copies to host memory and synchronises, see below);
 *  - every call shares the array: calls whose work overlaps on the GPU (for
 *    example on two streams at once) race and give wrong results; calls in
 *    sequence on one stream are safe (each call clears what must start at 0);
 *  - it copies rel to host memory and synchronises the grid's stream before
 *    it returns;
 *  - grids with a variable-density coefficient (helm_set_density) are not
 *    served: HELM_ERR_UNSUPPORTED.
 * Errors: HELM_ERR_ARG (also for a pointer of another device),
 * HELM_ERR_STATE (no model), HELM_ERR_UNSUPPORTED, HELM_ERR_CUDA. */
helm_status helm_true_residual_noalloc(helm_grid *g, int nrhs, const helm_c128 *f,
                                       const helm_c128 *u, double *rel);

/* The two tensor-core contractions of block FGMRES (helm_solve_batch with
 * options.block = 1), exposed for checking them on their own. Vectors are
 * complex64 (float re, im interleaved), device pointers of the current
 * device, vector k at offset k*ld; ld is a multiple of 8 and >= N, and the
 * entries N..ld-1 of every vector must be zero. Arithmetic: TF32 tensor-core
 * MMAs on operands split into TF32 hi + lo parts, FP32 accumulation (FP32
 * accuracy), partial sums added in FP64.
 * helm_block_gram: G[i*s + c] = sum_p conj(V_i[p]) W_c[p] for i < nv, c < s
 *   (the Gram matrix V^H W of block Gram-Schmidt, GMRES on Eq. 7); G (nv x s
 *   complex128) may be host or device memory.
 * helm_block_combine: W_c = alpha W_c + sum_i V_i C[i*s + c] (the block
 *   update), C (nv x s complex128) host or device; W is overwritten.
 * Limits: 1 <= nv <= 2048, 1 <= s <= 64. Both allocate their scratch and
 * synchronise the device. Errors: HELM_ERR_ARG, HELM_ERR_NOMEM, HELM_ERR_CUDA. */
helm_status helm_block_gram(int nv, int s, size_t N, size_t ld, const void *V, const void *W, helm_c128 *G);
helm_status helm_block_combine(int nv, int s, size_t N, size_t ld, const void *V, const helm_c128 *C,
                               float alpha, void *W);

/* ------------------------------------------------------------ autotuning
 * Tile shapes and smoother counts of the multigrid preconditioner (the paper
 * applies P^-1 approximately without fixing how; these are implementation
 * parameters, chosen by measurement).
 *
 * Tile shapes. The fused V(1,1) level kernels of 2D/3D grids ("down":
 * pre-smoothing, residual and restriction; "up": prolongation and
 * post-smoothing) are compiled for helm_num_tile_shapes(dim) shapes each
 * (0 for 1D). helm_tile_shape gives a shape's extents and block size: the
 * block's tile of coarse nodes, computed by `threads` threads (one, two, four
 * or 2^d threads per coarse node share its 2^d fine children) for one or
 * several right-hand sides (helm_tile_rhs_per_block); for the 3D
 * down kernel that marches along z (the last 3D down shape) the extents are
 * x, y of the tile and the number of coarse planes a block walks, one thread
 * per coarse (x, y) node. The arithmetic per node does not depend on the shape:
 * results are bitwise identical for every choice. helm_set_tiles /
 * helm_get_tiles set and read the shapes used on fine level `level` (the
 * pair level, level+1); -1 (the initial setting) selects the shape
 * automatically per solve: the first shape whose grid has at least 2 blocks per
 * SM for the batch, else the shape with the most blocks.
 *
 * helm_autotune(g, nrhs, f, tol, flags, report) measures on the grid's
 * current model, shift, options and batch size nrhs:
 *   HELM_TUNE_TILES     every down and up shape on every level, each timed
 *                       with CUDA events over a graph of 20 launches on the
 *                       level's own buffers; the fastest is kept per level.
 *   HELM_TUNE_SMOOTHER  (nu1, nu2) in {(1,1), (2,1), (1,2), (2,2)}: each is
 *                       used for one untimed and one timed helm_solve_batch of
 *                       f (nrhs x N, host or device, not modified) to tol; the
 *                       fastest converged one is kept in the grid's options
 *                       (only nu = (1,1) runs the fused kernels).
 * The basis, work vectors and the solution scratch are overwritten; the
 * model and hierarchy are kept. report (caller-owned) receives the chosen
 * shapes with their times and the default shape's times per level, and each
 * smoother candidate's time to solution (-1 if it did not converge) and
 * largest iteration count. Errors: HELM_ERR_ARG, HELM_ERR_STATE (no model),
 * HELM_ERR_UNSUPPORTED (preconditioner other than HELM_PRECOND_MG),
 * HELM_ERR_NOT_CONVERGED (no smoother candidate converged; options kept),
 * HELM_ERR_NOMEM, HELM_ERR_CUDA. */
#define HELM_TUNE_TILES 1
#define HELM_TUNE_SMOOTHER 2
#define HELM_TUNE_MAX_LEVELS 16
#define HELM_TUNE_MAX_NU 4

typedef struct {
    int levels;                                   /* fine levels with a down/up pair */
    int down_shape[HELM_TUNE_MAX_LEVELS];         /* chosen shape per fine level     */
    int up_shape[HELM_TUNE_MAX_LEVELS];
    double down_us[HELM_TUNE_MAX_LEVELS];         /* us per launch, chosen shape     */
    double up_us[HELM_TUNE_MAX_LEVELS];
    double down_default_us[HELM_TUNE_MAX_LEVELS]; /* us per launch, automatic shape  */
    double up_default_us[HELM_TUNE_MAX_LEVELS];
    int n_nu;                                     /* smoother candidates tried       */
    int nu[HELM_TUNE_MAX_NU][2];
    double nu_ms[HELM_TUNE_MAX_NU];               /* time to solution, -1 = failed   */
    int nu_iterations[HELM_TUNE_MAX_NU];
    int nu1, nu2;                                 /* smoother counts now in use      */
} helm_tune_report;

/* helm_tile_shape: kernel 0 = down, 1 = up; extent[3] (caller-owned) gets the
 * tile's extents in coarse nodes (x, y, z; z = 1 in 2D), *threads the block
 * size. helm_tile_rhs_per_block: *rb (caller-owned) gets how many right-hand
 * sides of a batch one block of the shape computes: 1, or 2 or 4 for the 2D
 * shapes whose threads keep their nodes' positions, boundary tests and D^-1
 * once for several right-hand sides. Errors (both): HELM_ERR_ARG for a dim,
 * kernel or shape out of range or a null pointer. */
int         helm_num_tile_shapes(int dim);
helm_status helm_tile_shape(int dim, int kernel, int shape, int extent[3], int *threads);
helm_status helm_tile_rhs_per_block(int dim, int kernel, int shape, int *rb);
helm_status helm_set_tiles(helm_grid *g, int level, int down_shape, int up_shape);
helm_status helm_get_tiles(const helm_grid *g, int level, int *down_shape, int *up_shape);
helm_status helm_autotune(helm_grid *g, int nrhs, const helm_c128 *f, double tol, int flags,
                          helm_tune_report *report);

/* Number of multigrid levels (1 = no coarsening; 0 before helm_set_shift)
 * and the node counts and spacing of one level. */
int         helm_num_levels(const helm_grid *g);
helm_status helm_level_info(const helm_grid *g, int level, int64_t n_out[3], double *h_out);

/* Message for the last failed call on this thread ("" if none). */
const char *helm_last_error(void);

/* ---------------------------------------------------------------- serving
 * A request loop for streams of independent solves (different grids,
 * frequencies, media and source counts). A dispatcher admits queued requests
 * in arrival order (FIFO) to `workers` worker threads, each with its own CUDA
 * stream, when the device memory all admitted requests hold fits
 * `memory_budget` (footprints from helm_solve_footprint; idle workers drop
 * their cached grids to make room). With `coalesce` > 1 an admitted request
 * takes along the queued requests of the same problem (see
 * helm_server_config). Workers keep one grid resident between
 * requests of the same size. Requests on different workers run concurrently
 * and their kernels overlap on the device; each request's right-hand sides
 * are solved together by helm_solve_batch. The paper has no counterpart: it
 * solves one problem at a time. */
typedef struct helm_server helm_server;

typedef struct {
    int workers;             /* requests in flight at once (1..64)                     */
    size_t memory_budget;    /* device bytes all admitted requests may hold together  */
    helm_options options;    /* solver options for every request                      */
    double beta1, beta2;     /* shift of M (Eq. 6), as in helm_set_shift              */
    int coalesce;            /* 0 or 1: every request is solved alone. k > 1: when a    */
                             /* request is admitted, queued requests with the same     */
                             /* grid, slowness values, omega, alpha and tol join it in */
                             /* one helm_solve_batch of at most k right-hand sides     */
                             /* (each keeps its own result: a member of a lock-step    */
                             /* batch gets the bits of its solve alone, and HELM_OK    */
                             /* when its own right-hand sides met tol, with side       */
                             /* RIGHT, even if another member's did not). Ignored with */
                             /* options.block (a shared block space would change the   */
                             /* results).                                              */
} helm_server_config;

typedef struct {
    int dim;                 /* 1, 2 or 3                                              */
    int64_t n[3];            /* nodes per axis (unused axes 1)                         */
    double h;                /* spacing, m                                             */
    const double *m;         /* slowness, host, N values; copied by helm_server_submit */
    double omega, alpha;     /* angular frequency, damping (Eq. 2)                     */
    int nrhs;                /* right-hand sides                                       */
    const helm_c128 *f;      /* host, nrhs x N; copied by helm_server_submit           */
    double tol;              /* true relative residual to reach                        */
} helm_request;

typedef struct {
    uint64_t id;
    helm_status status;
    int nrhs;
    int iterations_max;            /* over the request's right-hand sides          */
    double true_rel_residual_max;
    double t_submit, t_admit, t_done;   /* seconds on the server clock             */
    size_t footprint_bytes;        /* device bytes it was admitted with            */
} helm_result;

/* Device bytes a solve of nrhs right-hand sides on an n grid holds under `opt`
 * (an upper estimate: each buffer the solver allocates -- basis x restart,
 * multigrid work vectors and coefficients, coarse inverse and its tensor-core
 * tiles, staging, Hessenberg and reduction scratch -- rounded up to 2 MiB
 * allocation pages, plus a margin for small buffers and captured graphs).
 * 0 on bad arguments. */
size_t helm_solve_footprint(int dim, const int64_t n[3], int nrhs, const helm_options *opt);

/* Creates the server on the current device and starts its threads.
 * Errors: HELM_ERR_ARG, HELM_ERR_CUDA. */
helm_status helm_server_create(const helm_server_config *cfg, helm_server **out);

/* Queues a request and returns its id at once. u: host buffer of nrhs x N
 * complex values that receives the solutions; it must stay valid until the
 * request is done. Errors: HELM_ERR_ARG. */
helm_status helm_server_submit(helm_server *s, const helm_request *req, helm_c128 *u, uint64_t *id);

/* Waits for request `id`, fills *res and forgets the request. Returns the
 * request's own status (HELM_ERR_NOMEM if its footprint can never fit the
 * budget). Errors: HELM_ERR_ARG (unknown id). */
helm_status helm_server_wait(helm_server *s, uint64_t id, helm_result *res);

/* *done = 1 once request `id` has finished (its u is then written). */
helm_status helm_server_poll(helm_server *s, uint64_t id, int *done);

/* Seconds since the server was created (the clock of helm_result times). */
double helm_server_clock(const helm_server *s);

/* Finishes the running requests, stops the threads and frees every grid. */
void helm_server_destroy(helm_server *s);

/* Per-kernel timing. helm_profile_start() turns on CUDA-event timing of every
 * launch the library makes (process-wide, all grids; it adds two event
 * records per launch). helm_profile_stop() waits for those events, turns the
 * timing off and writes a JSON object into json (cap bytes) that maps each
 * kernel name to its launch count, summed device milliseconds, algorithmic
 * bytes and FP64 flops. Errors: HELM_ERR_ARG (buffer too small),
 * HELM_ERR_CUDA. The paper has no counterpart: this is instrumentation. */
helm_status helm_profile_start(void);
helm_status helm_profile_stop(char *json, size_t cap);

/* Times one kernel of the Arnoldi step j with the data of the grid's last
 * solve: `reps` back-to-back launches are captured in a CUDA graph, replayed
 * once to warm up and once between two CUDA events on the grid's stream.
 * kernel: "multidot", "multiaxpy", "stencil_apply" (H z_j), "multidot_h" (H z_j
 * fused with the multi-dot, the kernel the complex128-basis forms run),
 * "vcycle_gemm" (the coarse-level product of one V-cycle) or "vcycle"
 * (M^-1 v_j, all its kernels). Outputs: average microseconds per launch, and
 * the launch's algorithmic bytes and FP64 flops (0 for "vcycle"); bytes and
 * flops64 are nullable. The basis and Hessenberg scratch of the last solve
 * are overwritten. Errors: HELM_ERR_STATE (no solve yet), HELM_ERR_ARG,
 * HELM_ERR_CUDA. The paper has no counterpart: this is instrumentation. */
helm_status helm_time_kernel(helm_grid *g, const char *kernel, int j, int reps,
                             double *us_per_launch, double *bytes, double *flops64);

/* Time limit of the waits in which the streamed double-single Arnoldi kernels
 * (HELM_PREC_MIXED_DS) wait for a tile copy to land in shared memory, on the
 * current device; ns = 0 restores the default of 0.5 s. A wait that runs out
 * ends the kernel early: its results become NaN and the solve returns
 * HELM_ERR_BREAKDOWN, after the copies already issued have landed (those
 * waits keep the default limit). The grid stays usable. This exists to test
 * that timeout path; leave it at the default otherwise. The paper has no
 * counterpart. Errors: HELM_ERR_CUDA. */
helm_status helm_set_wait_limit_ns(uint64_t ns);

/* Number of kernels this library has launched in this process (all grids).
 * Used to report launch counts; not thread-safe across concurrent grids. */
uint64_t    helm_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
