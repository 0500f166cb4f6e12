/*
 * gmres_oracle.h -- CPU oracle for restarted mixed-precision GMRES(m).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and gmres_oracle.c form a plain,
 * slow, single-threaded restatement of Algorithm 1 of Lindquist, Luszczek and
 * Dongarra, "Improving the Performance of the GMRES Method using
 * Mixed-Precision Techniques" (arXiv 2011.01850).  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library under
 * paper_2011_01850_gb300/.
 *
 * Conventions
 *   - CSR matrices: rowptr[n+1], colind[nnz] (int32, 0-based), vals[nnz].
 *   - Basis V is column-major: vector i occupies V[i*n .. i*n+n-1].
 *   - Hessenberg matrices are column-major with leading dimension m+1:
 *     entry (row i, column j), both 0-based, lives at H[j*(m+1) + i].
 *   - Every sum is sequential in index order, in the working precision.
 *   - Return value 0 = success, negative = argument error.
 */
#ifndef GMRES_ORACLE_H
#define GMRES_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Orthogonalisation schemes (Algorithm 1, procedures MGS and CGSR). */
enum { ORC_MGS = 0, ORC_CGSR = 1 };

/* Precision assignments.
 *   ORC_FP64       every variable in binary64 (the double-precision baseline).
 *   ORC_MIXED      the paper's "fully mixed" solver (Sec. 4, 4.1): the residual
 *                  z = b - A x, its norm and the update x += u in binary64; the
 *                  whole restart cycle (Alg. 1 from the convergence test to the
 *                  correction) in binary32.
 *   ORC_MIXED_BF16 as ORC_MIXED, but each Krylov vector is stored rounded to
 *                  bfloat16 (round-to-nearest-even); arithmetic stays binary32.
 *   ORC_MIXED_FP16 as ORC_MIXED, with each Krylov vector stored as binary16
 *                  after scaling by the power of two 2^floor(log2(n)/2).
 *   ORC_ALL_FP32   negative control: residual and update in binary32 as well,
 *                  which Sec. 2 predicts cannot pass single-precision accuracy.
 *   ORC_MIXED_LIMITED the paper's "limited" mixed solver (Sec. 4.1): binary32
 *                  only for storing A as used for the next Krylov vector, the
 *                  preconditioner M and the Krylov basis V; every operation
 *                  and every other variable in binary64. */
enum { ORC_FP64 = 0, ORC_MIXED = 1, ORC_MIXED_BF16 = 2, ORC_MIXED_FP16 = 3, ORC_ALL_FP32 = 4,
       ORC_MIXED_LIMITED = 5 };

/* Per-variable precision switches (Sec. 4.1, the study that stores one
 * variable at a time in binary32 while the rest of the solver stays binary64):
 * with prec = ORC_FP64, every value written to a variable whose bit is set is
 * rounded to binary32; arithmetic stays binary64.  The paper's "correction
 * variables" (inside the restart cycle) and "refinement variables" (the
 * residual and the update):
 *   correction  ORC_PV_A_KRYLOV  A as used to compute the next Krylov vector
 *               ORC_PV_M         the preconditioner
 *               ORC_PV_V         the Krylov basis
 *               ORC_PV_W         the Krylov vector being orthogonalised (w)
 *               ORC_PV_H         the Hessenberg matrix (projection
 *                                coefficients, h_{j+1,j}, rotated entries)
 *               ORC_PV_GIVENS    the least-squares vectors: rotations
 *                                (alpha, beta), right-hand side s, solution y
 *               ORC_PV_Z         the non-preconditioned residual z as the
 *                                cycle receives it
 *   refinement  ORC_PV_A_RESID   A as used for the residual
 *               ORC_PV_B         the right-hand side b
 *               ORC_PV_X         the solution x (the update x += u rounds)
 *               ORC_PV_AX        the vector A x from which z = b - A x is formed */
enum {
    ORC_PV_A_KRYLOV = 1, ORC_PV_M = 2, ORC_PV_V = 4, ORC_PV_W = 8, ORC_PV_H = 16,
    ORC_PV_GIVENS = 32, ORC_PV_Z = 64, ORC_PV_A_RESID = 128, ORC_PV_B = 256, ORC_PV_X = 512,
    ORC_PV_AX = 1024, ORC_PV_ALL = 2047
};

typedef struct {
    int32_t m;            /* maximum inner iterations per restart cycle         */
    int32_t ortho;        /* ORC_MGS or ORC_CGSR                                 */
    int32_t prec;         /* ORC_FP64 ... ORC_MIXED_LIMITED                      */
    int32_t maxiter;      /* cap on the total number of inner iterations         */
    int32_t repeat_first; /* 1: after the first cycle, every cycle is limited to
                             the first cycle's length (Sec. 3, first strategy)  */
    int32_t stall_window; /* third strategy window w (inner iterations); 0 selects
                             ceil(0.05 m)                                        */
    double tol;           /* stop when ||b - A x||_2 <= tol * ||b||_2 (binary64) */
    double tau;           /* restart when |s_{j+1}| <= tau * beta (Sec. 3,
                             second strategy); 0 disables                       */
    double inner_factor;  /* end a cycle once |s_{j+1}| <= inner_factor*tol*||b||*/
    double stall_factor;  /* third strategy: restart once |s| improved by less
                             than this factor over the last w iterations of the
                             cycle (Sec. 4.1 uses 1.001); 0 disables             */
    double orth_threshold;/* fourth strategy: restart once ||S_k|| >= this     */
    int32_t orth_norm;    /* fourth strategy norm: 0 off, ORC_ORTH_SPECTRAL (power
                             method), ORC_ORTH_FROBENIUS                        */
    int32_t orth_iters;   /* power-method iterations (Sec. 4.1 uses 10)         */
    int32_t split_bytes;  /* 1: A stored once as the high- and low-order 32 bits
                             of each binary64 value (Sec. 4 outlook); the Krylov
                             step reads the high-order part only (a value
                             truncated to 20 fraction bits), the residual both */
    int32_t left_precond; /* 1: the preconditioner arguments of orc_gmres hold
                             ILU(0) factors (orc_ilu0) on their pattern, applied
                             on the left as Alg. 1 does: r = M^-1 z and
                             w = M^-1 A v_j (0: they hold a right
                             preconditioner M, applied as w = A M v_j)        */
    int32_t ilu32;        /* with left_precond in ORC_FP64: the factors stored in
                             binary32 (the paper's FP32-ILU variant, Sec. 4.2) */
    int32_t pv_mask;      /* ORC_PV_* bits (prec must be ORC_FP64); 0 = none   */
} orc_opts;

enum { ORC_ORTH_OFF = 0, ORC_ORTH_SPECTRAL = 1, ORC_ORTH_FROBENIUS = 2 };

/* The restart criteria one cycle checks after every inner iteration (Sec. 3):
 * tau and inner_abs as in orc_opts (inner_abs absolute), the stall test with
 * a window of stall_window (> 0) iterations, and the loss-of-orthogonality
 * test on S_k = (I + U_k)^-1 U_k, U_k the strictly upper part of V_k^T V_k
 * of the stored basis.  All-zero fields disable the optional tests. */
typedef struct {
    double tau;
    double inner_abs;
    double stall_factor;
    double orth_threshold;
    int32_t stall_window;
    int32_t orth_norm;
    int32_t orth_iters;
    int32_t split_bytes;  /* as in orc_opts */
    int32_t left_precond; /* as in orc_opts */
    int32_t ilu32;        /* as in orc_opts */
    int32_t pv_mask;      /* as in orc_opts (the correction variables act here) */
} orc_restart;

typedef struct {
    int32_t iters;        /* total inner iterations                              */
    int32_t restarts;     /* number of restart cycles that ran                   */
    int32_t converged;    /* 1 if the binary64 residual met tol                  */
    int32_t first_len;    /* length of the first cycle                           */
    double relres;        /* final ||b - A x|| / ||b||, binary64                 */
    double bnorm;         /* ||b||_2                                             */
} orc_info;

/* y = A x.  prec = ORC_FP64: binary64 arithmetic.  Any other prec: the values,
 * x and the running sum are binary32 (the copy of A used by the Arnoldi loop,
 * Sec. 4). */
int orc_spmv(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
             const double *x, double *y, int32_t prec);

/* z = b - A x in binary64 (Alg. 1, first line of the outer loop); returns ||z||_2. */
double orc_residual(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                    const double *b, const double *x, double *z);

/* Round each of count binary64 values as stored in a Krylov basis of the given
 * precision (ORC_FP64: unchanged; ORC_MIXED: binary32; ORC_MIXED_BF16: bfloat16
 * via binary32; ORC_MIXED_FP16: binary16 with scale 2^floor(log2(n)/2)). */
void orc_round_basis(int32_t count, const double *in, double *out, int32_t prec, int32_t n);

/* One restart cycle (Alg. 1, from "r_k <- M^-1 z_k" to the correction u_k),
 * starting from the residual r0 (length n, already in the caller's precision;
 * it is rounded to the working precision here).
 *
 *   kmax        maximum number of inner iterations (<= m)
 *   tau, inner_abs  restart when |s_{j+1}| <= tau*beta or |s_{j+1}| <= inner_abs
 *   pm_*        right preconditioner M on its own CSR pattern, or NULL for M = I;
 *               with M the loop uses w = A M v_j and u = M V_j y
 * Outputs (any may be NULL):
 *   V     (m+1)*n  basis, logical values after storage rounding
 *   Hbar  (m+1)*m  unrotated Hessenberg matrix
 *   Hrot  (m+1)*m  Hessenberg matrix after the Givens rotations (upper triangle)
 *   s     m+1      rotated right-hand side
 *   cs,sn m        rotations (alpha_i, beta_i)
 *   y     m        least-squares solution
 *   u     n        correction
 *   arn   m        |s_{j+1}| after each inner iteration
 *   jout           number of inner iterations done
 *   breakdown      1 if the cycle ended on h_{j+1,j} ~ 0
 */
int orc_arnoldi_cycle(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                      const double *r0, int32_t m, int32_t kmax, int32_t ortho, int32_t prec,
                      double tau, double inner_abs,
                      const int32_t *pm_rowptr, const int32_t *pm_colind, const double *pm_vals,
                      double *V, double *Hbar, double *Hrot, double *s, double *cs, double *sn,
                      double *y, double *u, double *arn, int32_t *jout, int32_t *breakdown);

/* One inner iteration of Alg. 1 from the given basis V (ncols columns,
 * column-major, values as the basis stores them): w = A v_ncols, MGS or CGSR
 * against V, h_{j+1,j} = ||w||, all in the working precision prec selects
 * (binary32 values and arithmetic for the mixed precisions; binary64
 * arithmetic with A rounded to binary32 for ORC_MIXED_LIMITED).  Outputs:
 * h (ncols+1: h_{1..j,j}, then h_{j+1,j}) and vnext (n: w / h_{j+1,j} in the
 * working precision, before the basis rounds it).  No Givens rotation. */
int orc_arnoldi_step(int32_t n, const int32_t *rowptr, const int32_t *colind,
                     const double *vals, const double *V, int32_t ncols, int32_t ortho,
                     int32_t prec, double *h, double *vnext);

/* orc_arnoldi_cycle with every restart criterion of orc_restart; orth
 * (length m, may be NULL) receives ||S_k|| after each inner iteration (0
 * where the test is off or the cycle broke down). */
int orc_arnoldi_cycle_ex(int32_t n, const int32_t *rowptr, const int32_t *colind,
                         const double *vals, const double *r0, int32_t m, int32_t kmax,
                         int32_t ortho, int32_t prec, const orc_restart *rs,
                         const int32_t *pm_rowptr, const int32_t *pm_colind,
                         const double *pm_vals, double *V, double *Hbar, double *Hrot, double *s,
                         double *cs, double *sn, double *y, double *u, double *arn, double *orth,
                         int32_t *jout, int32_t *breakdown);

/* ||S||_2 estimate of a k x k strictly upper triangular S (column-major,
 * leading dimension ld) by `iters` power-method iterations on S^T S from the
 * vector of equal entries; exposed for the tests. */
double orc_s_norm2(int32_t k, const double *S, int32_t ld, int32_t iters);

/* ILU(0) of A (Sec. 4's preconditioner): lu receives L (strictly lower part,
 * unit diagonal implied) and U (upper part with the diagonal) on A's pattern.
 * Rows must be sorted with a diagonal entry.  Returns 0, -1 (bad input) or
 * -3 (zero or non-finite pivot). */
int orc_ilu0(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
             double *lu);

/* out = (L U)^-1 z in binary64 (forward then backward substitution). */
int orc_ilu_apply(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *lu,
                  const double *z, double *out);

/* The high-order 32 bits of a binary64 value as a binary64 value (the low
 * 32 bits cleared: sign, exponent and the top 20 fraction bits). */
double orc_high_part(double v);

/* Threads the loops over rows and vector entries use: 1 in the parity build;
 * in the OpenMP timing build, want > 0 sets the count first.  Returns it. */
int orc_threads(int32_t want);

/* Restarted GMRES(m) (Alg. 1).  x holds x_0 on entry and the result on exit.
 * arn_hist (length maxiter) receives |s_{j+1}| of every inner iteration;
 * cyc_hist (length maxiter+1) receives ||b - A x_k|| / ||b|| at the top of every
 * cycle k and after the last one.  Either may be NULL. */
int orc_gmres(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
              const double *b, double *x, const orc_opts *o,
              const int32_t *pm_rowptr, const int32_t *pm_colind, const double *pm_vals,
              orc_info *info, double *arn_hist, double *cyc_hist);

#ifdef __cplusplus
}
#endif
#endif
