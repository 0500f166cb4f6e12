/*
 * gmres_gb300.h -- C-ABI of the GB300 (sm_103a) mixed-precision restarted
 * GMRES(m) library.
 *
 * The method is Algorithm 1 of Lindquist, Luszczek and Dongarra, "Improving
 * the Performance of the GMRES Method using Mixed-Precision Techniques"
 * (arXiv 2011.01850): restarted GMRES with MGS or CGSR orthogonalisation and
 * Givens rotations, where the residual z = b - A x, the convergence test and
 * the update x += u are binary64 and the whole restart cycle may run in
 * binary32 ("fully mixed", Sec. 4 and Sec. 4.1).  Every step runs in CUDA
 * kernels of this library; there is no CPU path.
 *
 * Conventions for every entry point
 *   - Return value: a gmres_status; no C++ exception crosses this boundary.
 *   - Device pointers are plain CUDA device (or managed) addresses.  Entry
 *     points that accept "host or device" buffers detect host memory with
 *     cudaPointerGetAttributes and copy through library-owned device buffers.
 *   - Matrices are CSR with int32 row pointers (n+1) and column indices
 *     (nnz, 0-based, each in [0, n)); values are binary64.
 *   - All work is issued on the handle's stream (gmres_create / gmres_set_stream)
 *     and every call returns only after that work has finished, except where a
 *     comment says otherwise.
 *   - The library owns every buffer it allocates; the caller keeps ownership
 *     of the arrays it passes in.
 */
#ifndef GMRES_GB300_H
#define GMRES_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmres_handle *gmres_t;

/* Orthogonalisation scheme (Algorithm 1, procedures MGS and CGSR). */
typedef enum { GMRES_ORTHO_MGS = 0, GMRES_ORTHO_CGSR = 1 } gmres_ortho;

/* Precision assignment.
 *   GMRES_FP64        every quantity binary64 (the double-precision baseline).
 *   GMRES_MIXED       binary64 residual, norm test and update; the restart
 *                     cycle (SpMV on a binary32 copy of A, orthogonalisation,
 *                     Givens, correction) in binary32 (Sec. 2, Sec. 4).
 *   GMRES_MIXED_BF16  as GMRES_MIXED with the Krylov basis stored as bfloat16
 *                     (round-to-nearest-even), binary32 arithmetic.
 *   GMRES_MIXED_FP16  as GMRES_MIXED with the Krylov basis stored as binary16
 *                     scaled by 2^floor(log2(n)/2), binary32 arithmetic.
 *   GMRES_MIXED_LIMITED the paper's "limited" mixed solver (Sec. 4.1):
 *                     binary64 arithmetic and vectors throughout; binary32
 *                     storage only for A as used in the Krylov step, the
 *                     preconditioner M and the Krylov basis.  Grid path only
 *                     (GMRES_PATH_AUTO picks it); not in the batched and
 *                     no-allocation solvers.
 * The 16-bit bases follow the paper's outlook on half precision (Sec. 5). */
typedef enum {
    GMRES_FP64 = 0,
    GMRES_MIXED = 1,
    GMRES_MIXED_BF16 = 2,
    GMRES_MIXED_FP16 = 3,
    GMRES_MIXED_LIMITED = 4
} gmres_precision;

typedef enum {
    GMRES_OK = 0,             /* converged: ||b - A x||_2 <= tol ||b||_2       */
    GMRES_MAXITER = 1,        /* maxiter inner iterations without converging   */
    GMRES_ERR_ARG = -1,       /* invalid argument (sizes, enums, CSR structure)*/
    GMRES_ERR_CUDA = -2,      /* a CUDA call failed                            */
    GMRES_ERR_NONFINITE = -3, /* NaN or Inf in an input or produced by a step  */
    GMRES_ERR_BREAKDOWN = -4, /* no progress possible (singular projected LS)  */
    GMRES_ERR_TIMEOUT = -5,   /* a bounded device wait ran out                 */
    GMRES_ERR_OOM = -6,       /* device allocation failed                      */
    GMRES_ERR_INDEX = -7      /* checked build only: a column index outside its
                                 system reached a kernel (see
                                 gmres_checks_enabled)                         */
} gmres_status;

/* gmres_create flags. */
#define GMRES_CREATE_DEVICE_PTRS 1 /* rowptr/colind/vals are device pointers  */
#define GMRES_CREATE_SPLIT 4       /* store A once, as the high- and low-order
                                      32 bits of each binary64 value (Sec. 4,
                                      the storage the paper points to instead of
                                      two copies): 8 bytes per nonzero instead of
                                      12; the binary32 Krylov step reads the high
                                      part (the value truncated to 20 fraction
                                      bits), binary64 work reads both.  Grid path
                                      only; not with the learned preconditioner */
#define GMRES_CREATE_TRANSPOSE 2   /* also build the CSR of A^T (preconditioner
                                      training needs A^T r)                    */

/* Restart-cycle path. */
#define GMRES_PATH_AUTO 0  /* choose by size                                  */
#define GMRES_PATH_GRID 1  /* whole-GPU kernels per inner step (large n)      */
#define GMRES_PATH_BLOCK 2 /* one thread block runs the whole solve (small n) */

/* Loss-of-orthogonality restart test (Sec. 3, fourth strategy): the norm of
 * S_k = (I + U_k)^-1 U_k, U_k the strictly upper part of V_k^T V_k. */
#define GMRES_ORTH_OFF 0
#define GMRES_ORTH_SPECTRAL 1  /* power method on S^T S                        */
#define GMRES_ORTH_FROBENIUS 2 /* ||S||_F, an upper bound of ||S||_2          */

/* Per-variable precision switches (gmres_opts.pv_mask; Sec. 4.1, the study
 * that stores one solver variable at a time in binary32 while the rest of the
 * binary64 solver is unchanged): with GMRES_FP64 on the grid path, every value
 * written to a variable whose bit is set is rounded to binary32 (round to
 * nearest even); arithmetic stays binary64.  The paper's "correction
 * variables" (the restart cycle) ... */
#define GMRES_PV_A_KRYLOV 1   /* A as used to compute the next Krylov vector */
#define GMRES_PV_M 2          /* the preconditioner M                        */
#define GMRES_PV_V 4          /* the Krylov basis                            */
#define GMRES_PV_W 8          /* the Krylov vector being orthogonalised, w   */
#define GMRES_PV_H 16         /* the Hessenberg matrix: projection
                                 coefficients, h_{j+1,j}, rotated entries    */
#define GMRES_PV_GIVENS 32    /* the least-squares vectors: rotations, the
                                 rotated right-hand side s, the solution y   */
#define GMRES_PV_Z 64         /* the non-preconditioned residual z as the
                                 cycle receives it                           */
/* ... and its "refinement variables" (the residual and the update): */
#define GMRES_PV_A_RESID 128  /* A as used for the residual z = b - A x      */
#define GMRES_PV_B 256        /* the right-hand side b                       */
#define GMRES_PV_X 512        /* the solution x (the update x += u rounds)   */
#define GMRES_PV_AX 1024      /* the product A x from which z is formed      */
/* With a refinement switch the solver tests its own (perturbed) residual; it
 * then reports the binary64 residual of the returned x in gmres_info.relres
 * and returns GMRES_OK only if that residual met tol (else GMRES_MAXITER). */

/* Solver options (gmres_default_opts gives the defaults). */
typedef struct gmres_opts {
    double tau;           /* restart when |s_{j+1}| <= tau * beta (Sec. 3, second
                             strategy); < 0 selects the precision's default:
                             0 (off) for FP64, 1e-6 MIXED, 2^-8 BF16, 2^-11
                             FP16 (one unit roundoff of the basis format)      */
    double inner_factor;  /* end a cycle once |s_{j+1}| <= inner_factor * tol *
                             ||b|| (the binary64 residual then decides); 0.5    */
    int32_t repeat_first; /* 1: cycles after the first run as long as the first
                             (Sec. 3, first strategy; Sec. 4.2); -1 = default
                             (on for the mixed precisions, off for FP64)       */
    int32_t path;         /* GMRES_PATH_*                                       */
    int32_t profile;      /* 1: time every kernel class with CUDA events and
                             report it in gmres_info.kernel_ms                  */
    int32_t spin_limit;   /* iterations a device-side wait may spin before it
                             gives up with GMRES_ERR_TIMEOUT; 0 = default       */
    int32_t precond;      /* 0: none; 1: the learned right preconditioner set
                             by gmres_spai_set; 2: ILU(0) on the left as in
                             Alg. 1 (factors made by gmres_ilu0)               */
    int32_t fallback;     /* 1: on stagnation of the preconditioned solve,
                             continue unpreconditioned (default 1)              */
    int32_t spmv_lanes;   /* lanes per CSR row in SpMV (1..32, power of two);
                             0 = the autotuned choice                           */
    int32_t cgs_kernel;   /* CGSR kernel family: 0 = register-streaming rows
                             (default; the updates split by basis vectors, and
                             with a binary32 basis the second pass keeps each
                             slice in registers between update and dot
                             products), 2 = the same passes with the update
                             split by rows (another summation order); 1 and 3
                             are retired (GMRES_ERR_ARG)                      */
    int32_t mgs_kernel;   /* MGS: 0 = one cooperative kernel per inner step with
                             w in shared memory and the block's basis rows
                             staged there one vector ahead by bulk copies
                             (default; without the staging when the rows do
                             not fit, one kernel per basis vector when w does
                             not fit either), 1 = one kernel per basis vector,
                             2 = the cooperative kernel without the staging */
    int32_t l2_prefetch;  /* register-streaming CGSR: each block prefetches the
                             basis rows of the slice this many slices ahead of
                             the one it is reading into L2 (bulk prefetch);
                             0 = off (default), 1..4                          */
    int32_t block_cluster;/* block path: thread blocks per system, 1 (one block)
                             or 8 (a cluster with distributed-shared-memory
                             reductions); 0 = automatic (8 for binary64 from
                             2048 rows, else 1)                                 */
    int32_t ilu_binary32; /* 1: with precond 2 in GMRES_FP64, use the ILU(0)
                             factors stored in binary32 (the paper's FP32-ILU
                             variant, Sec. 4.2); the binary32 cycle always does */
    double stall_factor;  /* third restart strategy (Sec. 3; Sec. 4.1 uses 1.001):
                             end the cycle once |s_{j+1}| improved by less than
                             this factor over the last stall_window inner
                             iterations; 0 = off (default)                      */
    int32_t stall_window; /* window of the stall test; 0 = ceil(0.05 m)        */
    int32_t orth_norm;    /* fourth restart strategy: GMRES_ORTH_* (default off);
                             grid path only (GMRES_PATH_AUTO picks it)          */
    double orth_threshold;/* end the cycle once ||S_k|| >= this (default 1.0)  */
    int32_t orth_iters;   /* power-method iterations (default 10, as Sec. 4.1) */
    int32_t trsv_kernel;  /* ILU(0) triangular solves, one launch per
                             triangle: 3 = cooperative, no barrier: the
                             solution entries start as an all-ones NaN
                             pattern and each warp polls its rows'
                             dependencies' entries, level after level;
                             2 = cooperative, a grid barrier between levels;
                             1 = one warp per row, rows claimed in level
                             order, per-row ready flags.  0 (default): per
                             triangle, 3 when every row has at most four
                             entries in it and every level fits the grid,
                             else 2                                          */
    int32_t pv_mask;      /* GMRES_PV_* bits (default 0): the per-variable
                             precision study; GMRES_FP64 on the grid path only
                             (not with split storage), else gmres_solve
                             returns GMRES_ERR_ARG                            */
    int32_t spmv_format;  /* storage of A for w = A v_j on the grid path and
                             for gmres_spmv: GMRES_SPMV_AUTO (default: the
                             format gmres_autotune chose per precision, CSR
                             before it runs), GMRES_SPMV_CSR, or
                             GMRES_SPMV_SLICED (slices of 32 rows stored
                             column-major, built when these options are set;
                             gmres_set_opts returns GMRES_ERR_ARG with split
                             storage or a row longer than 65535 entries).  The
                             sliced product sums each row exactly as CSR at
                             one lane per row; the limited, split and
                             binary32-A per-variable forms read CSR         */
} gmres_opts;

/* Values of gmres_opts.spmv_format. */
#define GMRES_SPMV_AUTO 0
#define GMRES_SPMV_CSR 1
#define GMRES_SPMV_SLICED 2

/* Kernel classes reported in gmres_info (index into kernel_ms / kernel_bytes). */
enum {
    GMRES_K_RESIDUAL = 0, /* z = b - A x (binary64), norms, cast               */
    GMRES_K_SPMV = 1,     /* w = A v_j in the working precision                */
    GMRES_K_ORTHO = 2,    /* MGS or CGSR (+ norm, Givens)                       */
    GMRES_K_NORMALIZE = 3,/* v_{j+1} = w / h_{j+1,j}                            */
    GMRES_K_UPDATE = 4,   /* y = H^-1 s, x += V y                               */
    GMRES_K_PRECOND = 5,  /* t = M v (learned preconditioner)                   */
    GMRES_K_BLOCK = 6,    /* the single-block whole-solve kernel                */
    GMRES_K_COUNT = 8
};

typedef struct gmres_info {
    int32_t iters;        /* total inner iterations                             */
    int32_t restarts;     /* restart cycles run                                 */
    int32_t converged;    /* 1 when the binary64 relative residual met tol      */
    int32_t first_len;    /* length of the first cycle                          */
    double relres;        /* final ||b - A x||_2 / ||b||_2 (binary64, on device)*/
    double bnorm;         /* ||b||_2                                            */
    double time_ms;       /* wall time of the call                              */
    double kernel_ms[GMRES_K_COUNT];    /* CUDA-event time per class (profile)  */
    double kernel_bytes[GMRES_K_COUNT]; /* algorithmic bytes per class          */
    int64_t kernel_launches[GMRES_K_COUNT];
    int64_t launches;     /* kernels launched by the call                       */
    int32_t path;         /* GMRES_PATH_GRID or GMRES_PATH_BLOCK                */
    int32_t fell_back;    /* 1 if the preconditioned solve fell back            */
} gmres_info;

/* Defaults for gmres_opts (never fails). */
void gmres_default_opts(gmres_opts *o);

/* Build a solver handle for the n x n CSR matrix A (Alg. 1 input A; Sec. 4:
 * the matrix is kept twice, binary64 for the residual and binary32 for the
 * restart cycle, sharing the index arrays).  The arrays are copied; flags as
 * above.  stream is a cudaStream_t (NULL = legacy default stream) that all of
 * the handle's work uses.  Errors: GMRES_ERR_ARG for n <= 0, a non-monotone
 * rowptr, rowptr[0] != 0 or a column index outside [0, n) (checked on the host
 * for host arrays, on the device for device arrays); GMRES_ERR_NONFINITE for
 * a NaN/Inf value; GMRES_ERR_OOM; GMRES_ERR_CUDA.  *out is NULL on error. */
gmres_status gmres_create(gmres_t *out, int32_t n, const int32_t *rowptr, const int32_t *colind,
                          const double *vals, int32_t flags, void *stream);

/* Release every device buffer of the handle.  NULL is ignored. */
void gmres_destroy(gmres_t h);

/* Replace A's values (same pattern; nnz binary64 values, host or device).
 * Drops the learned preconditioner and cached derived data of the old values
 * (A^T, the ILU(0) factors); A's sliced copy, when one is built, takes the
 * new values.  Synchronizes the handle's stream.  Errors: GMRES_ERR_ARG,
 * GMRES_ERR_NONFINITE (host values), GMRES_ERR_CUDA. */
gmres_status gmres_set_values(gmres_t h, const double *vals);

/* Change the stream used by later calls. */
gmres_status gmres_set_stream(gmres_t h, void *stream);

/* Replace / read the handle's options (validated: GMRES_ERR_ARG). */
gmres_status gmres_set_opts(gmres_t h, const gmres_opts *o);
gmres_status gmres_get_opts(gmres_t h, gmres_opts *o);

/* Restarted GMRES(m) (Algorithm 1) for A x = b.
 *   b     length n, binary64, host or device memory (read only)
 *   x     length n, binary64, host or device memory: x_0 on entry, the result
 *         on exit (x_0 != 0 resumes a previous solve: x is the whole state)
 *   m     restart length, 1 <= m <= 128
 *   tol   > 0: stop once ||b - A x||_2 <= tol ||b||_2, both norms binary64
 *   maxiter  cap on the total number of inner iterations (>= 0)
 *   info  may be NULL
 * Returns GMRES_OK on convergence, GMRES_MAXITER when the cap is reached, or
 * an error.  b = 0 returns x = 0 and GMRES_OK. */
gmres_status gmres_solve(gmres_t h, const double *b, double *x, int32_t m, double tol,
                         gmres_ortho ortho, gmres_precision prec, int32_t maxiter,
                         gmres_info *info);

/* y = A x with the precision's copy of A (Alg. 1, "w <- A v_j"): for
 * GMRES_FP64 x and y are binary64 device vectors, otherwise binary32.  A is
 * read in the storage gmres_spmv_format reports for the precision. */
gmres_status gmres_spmv(gmres_t h, const void *x, void *y, gmres_precision prec);

/* z = b - A x in binary64 (Alg. 1, first step of every restart) with
 * *znorm = ||z||_2.  b, x, z are device vectors; z may be NULL. */
gmres_status gmres_residual(gmres_t h, const double *b, const double *x, double *z,
                            double *znorm);

/* Normwise backward error of x, the paper's accuracy measure (Sec. 4: runs
 * stop at a backward error of 1e-10; the formula is not printed):
 *   eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf),
 * the infinity-norm form, in binary64 (maxima exact).  b and x are device
 * vectors; *eta a host double. */
gmres_status gmres_backward_error(gmres_t h, const double *b, const double *x, double *eta);

/* One restart cycle from the binary64 device vector r0, for parity checks
 * (Alg. 1 from "beta <- ||r||" to the correction u).  The cycle is the one
 * gmres_solve runs.  kmax <= m inner iterations; the cycle also ends when
 * |s_{j+1}| <= tau * beta or <= inner_abs, or on breakdown.  Host outputs
 * (NULL allowed), all binary64:
 *   V (m+1)*n column-major basis as stored (16-bit values widened),
 *   Hbar, H (m+1)*m column-major (leading dimension m+1) unrotated / rotated,
 *   s m+1, cs m, sn m, y m, u n (the correction), arn m (|s_{j+1}| per step),
 *   *jout inner iterations, *breakdown 1 if h_{j+1,j} vanished. */
gmres_status gmres_arnoldi(gmres_t h, const double *r0, int32_t m, int32_t kmax,
                           gmres_ortho ortho, gmres_precision prec, double tau, double inner_abs,
                           double *V, double *Hbar, double *H, double *s, double *cs, double *sn,
                           double *y, double *u, double *arn, int32_t *jout, int32_t *breakdown);

/* One inner iteration of Algorithm 1 from a caller-given basis, for parity
 * checks at sizes where a whole cycle drifts with the summation order: the
 * first ncols basis vectors are taken from V (host, binary64, ncols x n,
 * vector i at V + i*n, values as the precision's basis stores them: they are
 * rounded to the storage type on upload), then the iteration a solve runs
 * for column j = ncols: w = A v_j, MGS or CGSR against V_j (the kernels
 * gmres_opts selects), h_{j+1,j} = ||w|| and v_{j+1} = w / h_{j+1,j}.
 * Host outputs: hcol (ncols + 1: h_{1..j,j}, then h_{j+1,j}), vnext (n, may be
 * NULL: v_{j+1} as stored, widened).  1 <= ncols <= 128.  Errors:
 * GMRES_ERR_ARG (also with a preconditioner or split storage),
 * GMRES_ERR_BREAKDOWN when h_{j+1,j} vanished (vnext not formed). */
gmres_status gmres_arnoldi_step(gmres_t h, const double *V, int32_t ncols, gmres_ortho ortho,
                                gmres_precision prec, double *hcol, double *vnext);

/* Time every SpMV variant (lanes per CSR row 1..32, and the sliced storage
 * of A where it can be built) on this matrix in binary32 and binary64 and keep
 * the fastest for later solves (the tile autotuner).  lanes32 / lanes64 (may
 * be NULL) receive the CSR choices; gmres_spmv_format reports the storage.
 * The sliced copy is kept only when it won in one of the precisions.
 * Synchronizes the handle's stream. */
gmres_status gmres_autotune(gmres_t h, int32_t *lanes32, int32_t *lanes64);

/* 1 when this library is the checked build (compiled with -DGMRES_CHECKS, the
 * library's stand-in for a memory sanitizer), else 0.  In the checked build
 * every kernel that gathers x through a column index (the CSR and sliced
 * products, the binary64 residuals, the block and batched solvers) first
 * tests the index against its system's columns; an index outside is counted
 * in a device word and replaced by column 0, so the load stays inside x.
 * gmres_solve, gmres_spmv, gmres_batch_solve and gmres_solve_noalloc then
 * return GMRES_ERR_INDEX (their other outputs are meaningless).  Matrices
 * that pass through gmres_create or gmres_batch_create are validated on the
 * host and never trigger it; gmres_solve_noalloc checks only rowptr's ends,
 * so it is the entry point the checked build guards.  Row pointers, ILU(0)
 * factors and the learned preconditioner's kernels are not checked.  The
 * checked build is the same source with the flag
 * (paper_2011_01850_gb300.build.build(checked=True)); it costs one compare
 * per gathered entry. */
int32_t gmres_checks_enabled(void);

/* Storage of A the grid path's w = A v_j and gmres_spmv read under the current
 * options, per precision: GMRES_SPMV_CSR or GMRES_SPMV_SLICED (for the
 * mixed precisions fmt32, for GMRES_FP64 fmt64; either may be NULL).  The
 * limited and split forms always read CSR. */
gmres_status gmres_spmv_format(gmres_t h, int32_t *fmt32, int32_t *fmt64);

/* ---------------------------------------------------------------------------
 * Learned sparse-approximate-inverse right preconditioner (the paper has no
 * counterpart; it preconditions with ILU(0) on the left, Sec. 4).  M has A's
 * sparsity pattern; m_pq = g_pq / a_pp where g = MLP(features of (p, q)), an
 * 8 -> 64 -> 64 -> 1 ReLU network with binary32 parameters laid out as
 * W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3 (GMRES_SPAI_NPARAM values).
 * Features (a zero diagonal counts as 1): a_pq/a_pp, a_qq/a_pp, [p==q],
 * sum_k|a_pk|/|a_pp|, sum_k|a_kq|/|a_qq|, nnz(row p)/8, sign(a_pq), sign(q-p).
 * Training minimises L = 1/(2 P n) sum_p ||A M z_p - z_p||^2 over probes z_p.
 * ------------------------------------------------------------------------- */
#define GMRES_SPAI_NPARAM 4801

/* The 8 features per nonzero, feature-major (feat[f * nnz + k]); host or
 * device buffer of 8 * nnz binary32 values (NULL only computes and caches). */
gmres_status gmres_spai_features(gmres_t h, float *feat);

/* Loss and gradients for the parameters `params` (host or device) and the P
 * probe vectors Z (device, n x P column-major, binary32): *loss (host, may be
 * NULL), grad_params (device, GMRES_SPAI_NPARAM, may be NULL) and dL/dm on
 * A's pattern (device, nnz, may be NULL). */
gmres_status gmres_spai_loss_grad(gmres_t h, const float *params, int32_t nprobe, const float *Z,
                                  double *loss, float *grad_params, float *grad_m);

/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8) on device
 * arrays params, adam_m, adam_v (GMRES_SPAI_NPARAM each) with gradient grad;
 * step >= 1 is the 1-based step count for the bias corrections. */
gmres_status gmres_spai_adam(gmres_t h, float *params, float *adam_m, float *adam_v,
                             const float *grad, int32_t step, float lr);

/* One training step on this handle's matrix: nprobe Rademacher probes drawn
 * on the device from `seed` (a counter-based mix of seed, probe and row), plus
 * nzx extra probes Zx (device, n x nzx, e.g. residuals a solve produced), then
 * loss, gradient and one Adam step on the device arrays.  *loss (host, may be
 * NULL) is the loss before the step. */
gmres_status gmres_spai_train_step(gmres_t h, float *params, float *adam_m, float *adam_v,
                                   int32_t step, int32_t nprobe, uint64_t seed, const float *Zx,
                                   int32_t nzx, float lr, double *loss);

/* Inference: M's values from `params` (host or device) on A's pattern; the
 * solver uses them as right preconditioner when opts.precond = 1 (grid path;
 * w = A M v_j, x += M V_j y).  gmres_spai_values copies them out (nnz
 * binary64, host or device); gmres_spai_clear drops them. */
gmres_status gmres_spai_set(gmres_t h, const float *params);
gmres_status gmres_spai_values(gmres_t h, double *mvals);
gmres_status gmres_spai_clear(gmres_t h);

/* ---------------------------------------------------------------------------
 * Batched solver: many independent systems of uneven size in one persistent
 * launch.  The systems form one block-diagonal CSR matrix: system i owns rows
 * [sys_ptr[i], sys_ptr[i+1]) and its column indices must lie in that range.
 * One thread block solves one system at a time (Algorithm 1, whole solve,
 * block-wide reductions); blocks take systems from a device work queue,
 * largest first.
 * ------------------------------------------------------------------------- */
typedef struct gmres_batch *gmres_batch_t;

typedef struct gmres_batch_result {
    int32_t iters, restarts, converged, status; /* status: a gmres_status     */
    double relres;                              /* binary64 ||b-Ax|| / ||b||  */
} gmres_batch_result;

/* Copy the batch to the device.  sys_ptr (nsys+1, int64, host), rowptr
 * (sys_ptr[nsys]+1, int32, host, global nonzero offsets), colind (global
 * column indices), vals (binary64), all host arrays.  Errors: GMRES_ERR_ARG
 * for nsys <= 0, an empty system, a non-monotone rowptr, or a column outside
 * its system's rows; GMRES_ERR_NONFINITE; GMRES_ERR_OOM; GMRES_ERR_CUDA. */
gmres_status gmres_batch_create(gmres_batch_t *out, int32_t nsys, const int64_t *sys_ptr,
                                const int32_t *rowptr, const int32_t *colind, const double *vals,
                                void *stream);

void gmres_batch_destroy(gmres_batch_t b);

/* Solve every system: b and x are packed (sys_ptr[nsys] entries, binary64,
 * host or device); x holds x_0 on entry.  Same m / tol / ortho / prec /
 * maxiter meaning as gmres_solve, applied per system.  results (nsys, host,
 * may be NULL) receives each system's outcome; info (may be NULL) the
 * totals (iters = sum, restarts = sum, converged = 1 if all converged,
 * kernel_ms[GMRES_K_BLOCK] = device time of the launch).  Returns GMRES_OK
 * when every system converged, GMRES_MAXITER if any hit the cap, else the
 * first error status met.  lanes: 0 = automatic, else lanes per CSR row. */
gmres_status gmres_batch_solve(gmres_batch_t b, const double *rhs, double *x, int32_t m,
                               double tol, gmres_ortho ortho, gmres_precision prec,
                               int32_t maxiter, int32_t lanes, gmres_batch_result *results,
                               gmres_info *info);

/* Systems of at least min_rows rows are solved by a cluster of 8 thread
 * blocks (reductions through distributed shared memory), the others by one
 * block each; 0 sends every system to a single block.  Default 8192.
 * GMRES_ERR_ARG for min_rows < 0. */
gmres_status gmres_batch_set_cluster_rows(gmres_batch_t b, int32_t min_rows);

/* Threads per block of the clusters that solve the large systems (128, 256,
 * 512 or 1024; the one-block systems always use 256).  More threads give a
 * cluster fewer rows per thread, so a shorter chain of memory latencies per
 * inner iteration, and fewer clusters fit the GPU at once.  Default 256
 * (2048 uneven 2-D systems: 2.30 s, against 2.50 s at 512 and 3.09 s at
 * 1024: the batch is bound by throughput, not by its slowest system).
 * GMRES_ERR_ARG for any other value. */
gmres_status gmres_batch_set_cluster_threads(gmres_batch_t b, int32_t threads);

/* SpMV tile autotuner of the batched solver: times a capped solve (iters
 * inner iterations per system, from x0 = 0, on scratch memory; the batch's
 * x is not touched) with 1, 2, 4, 8 and 16 lanes per CSR row and keeps the
 * fastest as the batch's choice for gmres_batch_solve with lanes = 0.  rhs
 * is packed like gmres_batch_solve's (host or device); *lanes_out (may be
 * NULL) receives the choice.  Errors: GMRES_ERR_ARG, GMRES_ERR_OOM,
 * GMRES_ERR_CUDA. */
gmres_status gmres_batch_autotune(gmres_batch_t b, const double *rhs, int32_t m,
                                  gmres_ortho ortho, gmres_precision prec, int32_t iters,
                                  int32_t *lanes_out);

/* ---------------------------------------------------------------------------
 * Solve without allocating device memory.  The paper has no counterpart; this
 * is for callers that cannot allocate at the point of the solve: cudaMalloc /
 * cudaFree may synchronise the whole device, and some frameworks own the
 * entire device budget through their own allocator.
 *
 * gmres_solve_noalloc runs the single-block whole-solve kernel (the block path
 * of gmres_solve) on the caller's DEVICE arrays: CSR rowptr (n+1), colind and
 * vals (nnz, binary64), b and x (n, binary64; x = x_0 on entry, the result on
 * exit).  m, tol, ortho, prec, maxiter, info: as for gmres_solve; stream is a
 * cudaStream_t.  Every system runs on one thread block here, also binary64
 * systems of 2048 rows and more, which gmres_solve would give a cluster of 8
 * blocks (so iteration counts may differ from gmres_solve's for those).
 * rowptr[0] must be 0 and rowptr[n] must equal nnz (both read back and
 * checked: GMRES_ERR_ARG); the rest of the CSR structure is not checked.
 * All workspace (Krylov basis, work vectors, binary32 values, result record)
 * comes from one file-scope device array of GMRES_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits; a system whose
 * workspace (about (m+1) n s_V + 8 n + 4 nnz bytes) exceeds it is rejected with
 * GMRES_ERR_ARG and a message on stderr.  No call allocates: neither
 * cudaMalloc, cudaFree nor any allocating library routine.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every
 * call waits for its stream to finish before it returns (it reads the result
 * record back to the host).  All calls share the array and each overwrites
 * it: calls that overlap on the GPU race and must be serialised by the
 * caller.  Host pointers: GMRES_ERR_ARG.
 * ------------------------------------------------------------------------- */
#define GMRES_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

gmres_status gmres_solve_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colind,
                                 const double *vals, int64_t nnz, const double *b, double *x,
                                 int32_t m, double tol, gmres_ortho ortho, gmres_precision prec,
                                 int32_t maxiter, void *stream, gmres_info *info);

/* Device bytes the handle holds for the matrix (both value copies, shared
 * indices, and the sliced copy of A when one is built) and, for a solve with
 * restart length m in precision prec, the workspace (basis, vectors,
 * Hessenberg).  Matches the paper's storage model (Sec. 4) without the ILU
 * factors. */
gmres_status gmres_memory_bytes(gmres_t h, int32_t m, gmres_precision prec, int64_t *matrix_bytes,
                                int64_t *workspace_bytes);

/* ILU(0) of the handle's A, the paper's preconditioner (Sec. 4): L (unit
 * lower) and U on A's sparsity pattern, factored on the GPU one level of the
 * row-dependency graph per launch (the levels come from a host analysis of
 * the pattern), kept in binary64 and binary32.  Select it with opts.precond
 * = 2: every solve then applies M^-1 = (L U)^-1 on the left (Alg. 1:
 * r = M^-1 z, w = M^-1 A v_j; the convergence test stays on ||b - A x||), on
 * the grid path, with level-scheduled triangular solves (opts.trsv_kernel;
 * bounded waits).  gmres_set_values drops the factors.  Errors: GMRES_ERR_ARG (rows
 * not sorted, a missing diagonal entry, split storage), GMRES_ERR_BREAKDOWN
 * (a zero or non-finite pivot), GMRES_ERR_OOM, GMRES_ERR_CUDA. */
gmres_status gmres_ilu0(gmres_t h);

/* Copy the binary64 ILU(0) factors to the host array lu (nnz entries, on
 * A's pattern: L's strictly lower entries, U's upper entries with the
 * diagonal).  GMRES_ERR_ARG before gmres_ilu0. */
gmres_status gmres_ilu_factors(gmres_t h, double *lu);

/* Dependency levels of the two triangles of gmres_ilu0's factors: *lower
 * for L y = z (row i waits for the rows k < i of its pattern), *upper for
 * U x = y (row i waits for the j > i).  Each triangular solve passes its
 * levels in sequence, so its time is about levels x the per-level latency.
 * GMRES_ERR_ARG before gmres_ilu0 or for a null pointer. */
gmres_status gmres_ilu_levels(gmres_t h, int32_t *lower, int32_t *upper);

/* out = (L U)^-1 z with the factors of gmres_ilu0: z, out device vectors of
 * n binary64 (GMRES_FP64) or binary32 (otherwise) values, binary64 or
 * binary32 factors to match.  GMRES_ERR_ARG before gmres_ilu0;
 * GMRES_ERR_TIMEOUT if a bounded wait ran out. */
gmres_status gmres_ilu_apply(gmres_t h, const void *z, void *out, gmres_precision prec);

/* ||S_k|| of the loss-of-orthogonality test after each inner iteration of
 * the last restart cycle the handle ran (gmres_solve or gmres_arnoldi), for
 * k = 2 .. j+1 basis vectors: out[c] belongs to inner iteration c+1; entries
 * past the cycle's end, or with the test off, are 0.  out is a host array of
 * count <= 128 entries.  The paper reports these norms (Sec. 4.1) and has no
 * separate interface for them. */
gmres_status gmres_orth_norms(gmres_t h, double *out, int32_t count);

/* Static text for a status code. */
const char *gmres_status_str(gmres_status s);

/* Library version string. */
const char *gmres_version(void);

#ifdef __cplusplus
}
#endif
#endif
