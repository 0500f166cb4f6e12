/*
 * gmres_oracle.c -- plain CPU oracle for restarted mixed-precision GMRES(m).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the CUDA library.  It restates
 * Algorithm 1 of Lindquist, Luszczek and Dongarra (arXiv 2011.01850) step by
 * step: a binary64 solver, the paper's "fully mixed" solver (binary64 residual
 * and update, binary32 restart cycle; Sec. 2 and Sec. 4), and the low-precision
 * basis variants.  Single-threaded, sequential sums, no blocking or fusion.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared gmres_oracle.c -lm
 * (-ffp-contract=off keeps every float operation separately rounded, the same
 * on x86-64 and AArch64).  The parity build is that one; the CPU-baseline
 * timing build adds -O3 -fopenmp, which runs the loops over rows and vector
 * entries on every core (inner products then sum per thread and combine the
 * threads' sums; the algorithm is unchanged).
 */
#include "gmres_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------
 * Storage rounding of Krylov vectors.
 * ------------------------------------------------------------------------- */

/* Round a binary32 value to bfloat16 (8 significand bits) with
 * round-to-nearest, ties-to-even, returned as binary32: keep the upper 16 bits
 * of the encoding after adding half an ulp of the kept part (plus the kept
 * part's lowest bit, which breaks ties towards even). */
static float round_bf16(float f)
{
    if (f != f)
        return f;
    uint32_t bits;
    memcpy(&bits, &f, 4);
    uint32_t lsb = (bits >> 16) & 1u;
    bits += 0x7fffu + lsb;
    bits &= 0xffff0000u;
    float out;
    memcpy(&out, &bits, 4);
    return out;
}

/* Round a value to IEEE binary16 (11 significand bits, exponent range
 * [-14, 15], subnormal spacing 2^-24) with round-to-nearest, ties-to-even.
 * The value is divided by its binary16 quantum (a power of two, so exactly),
 * rounded to an integer by rint (ties-to-even in the default mode) and scaled
 * back.  Magnitudes beyond the largest finite binary16 (65504) give +-inf. */
static double round_fp16(double f)
{
    if (f != f || f == 0)
        return f;
    double a = fabs(f);
    int e2;
    frexp(a, &e2);              /* a = mant * 2^e2, mant in [0.5, 1) */
    int e = e2 - 1;             /* floor(log2 a) */
    if (e < -14)
        e = -14;                /* subnormal range shares the 2^-24 quantum */
    double q = ldexp(1.0, e - 10);
    double r = rint(a / q) * q;
    if (r > 65504.0)
        r = INFINITY;
    return f < 0 ? -r : r;
}

/* Power-of-two scale of the binary16 basis: 2^floor(log2(n)/2) <= sqrt(n).
 * A unit vector's entries are at most 1 in magnitude, so scaled entries stay
 * below sqrt(n) (finite in binary16 for n < 2^32), while a typical entry
 * ~1/sqrt(n) is lifted to ~1, away from the subnormal range. */
static double fp16_scale(int32_t n)
{
    int lg = 0;
    while (lg < 31 && ((int64_t)1 << (lg + 1)) <= (int64_t)n)
        ++lg;
    return ldexp(1.0, lg / 2);
}

/* The value a basis of precision prec holds for the working value v. */
static double orc_store(double v, int32_t prec, int32_t n)
{
    switch (prec) {
    case ORC_FP64:
        return v;
    case ORC_MIXED_BF16:
        return (double)round_bf16((float)v);
    case ORC_MIXED_FP16: {
        double sc = fp16_scale(n);
        return round_fp16((double)(float)v * sc) / sc;
    }
    default:
        return (double)(float)v;
    }
}

void orc_round_basis(int32_t count, const double *in, double *out, int32_t prec, int32_t n)
{
    for (int32_t i = 0; i < count; ++i)
        out[i] = orc_store(in[i], prec, n);
}

double orc_high_part(double v)
{
    uint64_t u;
    memcpy(&u, &v, sizeof(u));
    u &= 0xFFFFFFFF00000000ull;
    memcpy(&v, &u, sizeof(v));
    return v;
}

/* ||S||_2 of a strictly upper triangular k x k S (column-major, leading
 * dimension ld) by the power method on S^T S (Sec. 3, fourth strategy; Sec.
 * 4.1 runs 10 iterations): x_0 has equal entries, x_t = S^T S x_{t-1}
 * normalised, and the estimate is ||S x_iters||. */
double orc_s_norm2(int32_t k, const double *S, int32_t ld, int32_t iters)
{
    if (k < 2)
        return 0.0;
    double *x = (double *)malloc(sizeof(double) * (size_t)k);
    double *yv = (double *)malloc(sizeof(double) * (size_t)k);
    if (!x || !yv) {
        free(x); free(yv);
        return NAN;
    }
    for (int32_t i = 0; i < k; ++i)
        x[i] = 1.0 / sqrt((double)k);
    for (int32_t t = 0; t < iters; ++t) {
        /* y = S x: y_i = sum over l > i of S_il x_l */
        for (int32_t i = 0; i < k; ++i) {
            double acc = 0;
            for (int32_t l = i + 1; l < k; ++l)
                acc += S[(size_t)l * ld + i] * x[l];
            yv[i] = acc;
        }
        /* x = S^T y: x_l = sum over i < l of S_il y_i, then normalise */
        double nn = 0;
        for (int32_t l = 0; l < k; ++l) {
            double acc = 0;
            for (int32_t i = 0; i < l; ++i)
                acc += S[(size_t)l * ld + i] * yv[i];
            x[l] = acc;
            nn += acc * acc;
        }
        nn = sqrt(nn);
        if (nn == 0) {
            free(x); free(yv);
            return 0.0;
        }
        for (int32_t l = 0; l < k; ++l)
            x[l] /= nn;
    }
    double ss = 0;
    for (int32_t i = 0; i < k; ++i) {
        double acc = 0;
        for (int32_t l = i + 1; l < k; ++l)
            acc += S[(size_t)l * ld + i] * x[l];
        ss += acc * acc;
    }
    free(x); free(yv);
    return sqrt(ss);
}

/* ---------------------------------------------------------------------------
 * The restart cycle in binary64 and in binary32.
 * ------------------------------------------------------------------------- */

/* A value written to a variable of the per-variable study (Sec. 4.1): rounded
 * to binary32 when its bit is in mask, else unchanged.  PV(x, bit) applies it
 * with the mask `pv` in scope, in the cycle's working type R. */
static double pv32(double v, int32_t mask, int32_t bit)
{
    return (mask & bit) ? (double)(float)v : v;
}
#define PV(x, bit) ((R)pv32((double)(x), pv, (bit)))

#define R double
#define FN(name) name##_f64
#define SQRT_R(x) sqrt(x)
#define U_BREAK 1e-14
#include "cycle_impl.inc"
#undef R
#undef FN
#undef SQRT_R
#undef U_BREAK

#define R float
#define FN(name) name##_f32
#define SQRT_R(x) sqrtf(x)
#define U_BREAK 1e-6
#include "cycle_impl.inc"
#undef R
#undef FN
#undef SQRT_R
#undef U_BREAK

/* ---------------------------------------------------------------------------
 * Public entry points.
 * ------------------------------------------------------------------------- */

static int csr_ok(int32_t n, const int32_t *rowptr, const int32_t *colind)
{
    if (n < 0 || !rowptr || (n > 0 && !colind && rowptr[n] > 0))
        return 0;
    if (rowptr[0] != 0)
        return 0;
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i])
            return 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colind[k] < 0 || colind[k] >= n)
                return 0;
    }
    return 1;
}

int orc_spmv(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
             const double *x, double *y, int32_t prec)
{
    if (!csr_ok(n, rowptr, colind))
        return -1;
    if (prec == ORC_FP64) {
        spmv_f64(n, rowptr, colind, vals, x, y);
        return 0;
    }
    int32_t nnz = rowptr[n];
    float *a = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    float *xf = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float *yf = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!a || !xf || !yf) {
        free(a); free(xf); free(yf);
        return -2;
    }
    for (int32_t k = 0; k < nnz; ++k)
        a[k] = (float)vals[k];
    for (int32_t i = 0; i < n; ++i)
        xf[i] = (float)x[i];
    spmv_f32(n, rowptr, colind, a, xf, yf);
    for (int32_t i = 0; i < n; ++i)
        y[i] = yf[i];
    free(a); free(xf); free(yf);
    return 0;
}

/* z = b - A x, every product and sum in binary64 (Sec. 2: the residual must be
 * formed in full precision, since it subtracts quantities of similar size). */
double orc_residual(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                    const double *b, const double *x, double *z)
{
    double ss = 0;
    #pragma omp parallel for reduction(+ : ss) schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += vals[k] * x[colind[k]];
        double zi = b[i] - acc;
        if (z)
            z[i] = zi;
        ss += zi * zi;
    }
    return sqrt(ss);
}

/* Work arrays of one cycle in precision R, exported as binary64 afterwards. */
typedef struct {
    void *V, *Hb, *H, *s, *cs, *sn, *y, *u, *r0, *a, *pm;
} cyc_buf;

static void cyc_free(cyc_buf *c)
{
    free(c->V); free(c->Hb); free(c->H); free(c->s); free(c->cs); free(c->sn);
    free(c->y); free(c->u); free(c->r0); free(c->a); free(c->pm);
    memset(c, 0, sizeof(*c));
}

static int cyc_alloc(cyc_buf *c, size_t el, int32_t n, int32_t m, int32_t nnz, int32_t pnnz)
{
    memset(c, 0, sizeof(*c));
    c->V = calloc((size_t)(m + 1) * n + 1, el);
    c->Hb = calloc((size_t)(m + 1) * m + 1, el);
    c->H = calloc((size_t)(m + 1) * m + 1, el);
    c->s = calloc((size_t)m + 2, el);
    c->cs = calloc((size_t)m + 1, el);
    c->sn = calloc((size_t)m + 1, el);
    c->y = calloc((size_t)m + 1, el);
    c->u = calloc((size_t)n + 1, el);
    c->r0 = calloc((size_t)n + 1, el);
    c->a = calloc((size_t)nnz + 1, el);
    c->pm = pnnz >= 0 ? calloc((size_t)pnnz + 1, el) : NULL;
    if (!c->V || !c->Hb || !c->H || !c->s || !c->cs || !c->sn || !c->y || !c->u || !c->r0 ||
        !c->a || (pnnz >= 0 && !c->pm)) {
        cyc_free(c);
        return -2;
    }
    return 0;
}

static void export_vec(double *dst, const void *src, size_t count, int is_f32)
{
    if (!dst)
        return;
    if (is_f32) {
        const float *f = (const float *)src;
        for (size_t i = 0; i < count; ++i)
            dst[i] = f[i];
    } else {
        memcpy(dst, src, count * sizeof(double));
    }
}

/* Run one cycle in the precision prec selects, from a binary64 residual r0. */
static int run_cycle(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                     const double *r0, int32_t m, int32_t kmax, int32_t ortho, int32_t prec,
                     const orc_restart *rs,
                     const int32_t *pm_rowptr, const int32_t *pm_colind, const double *pm_vals,
                     double *V, double *Hb, double *H, double *s, double *cs, double *sn,
                     double *y, double *u, double *arn, double *orth, int32_t *jout, int32_t *bd)
{
    const int is_f32 = (prec != ORC_FP64 && prec != ORC_MIXED_LIMITED);
    const int limited = (prec == ORC_MIXED_LIMITED);
    const size_t el = is_f32 ? sizeof(float) : sizeof(double);
    const int32_t nnz = rowptr[n];
    const int32_t pnnz = pm_vals ? pm_rowptr[n] : -1;
    cyc_buf c;
    if (cyc_alloc(&c, el, n, m, nnz, pnnz))
        return -2;
    int rc;
    if (is_f32) {
        float *a = (float *)c.a, *r = (float *)c.r0, *pm = (float *)c.pm;
        /* the Krylov step's copy of A: binary32, from the high-order part
         * when A is stored split */
        for (int32_t k = 0; k < nnz; ++k)
            a[k] = (float)(rs->split_bytes ? orc_high_part(vals[k]) : vals[k]);
        for (int32_t i = 0; i < n; ++i)
            r[i] = (float)r0[i];
        for (int32_t k = 0; k < pnnz; ++k)
            pm[k] = (float)pm_vals[k];
        rc = cycle_f32(n, rowptr, colind, a, r, m, kmax, ortho, prec, rs,
                       pm_rowptr, pm_colind, pm_vals ? pm : NULL,
                       (float *)c.V, (float *)c.Hb, (float *)c.H, (float *)c.s,
                       (float *)c.cs, (float *)c.sn, (float *)c.y, (float *)c.u, arn, orth, jout,
                       bd);
    } else {
        /* limited mixed: A for the next Krylov vector and M stored in
         * binary32, used in binary64 arithmetic (the basis is rounded by
         * orc_store); the same for the per-variable switches of A and M */
        double *a = (double *)c.a, *pm = (double *)c.pm;
        for (int32_t k = 0; k < nnz; ++k)
            a[k] = !limited ? pv32(vals[k], rs->pv_mask, ORC_PV_A_KRYLOV)
                            : (rs->split_bytes ? orc_high_part(vals[k]) : (double)(float)vals[k]);
        memcpy(c.r0, r0, sizeof(double) * (size_t)n);
        /* M in binary32 for limited mixed and for the binary32 ILU factors */
        for (int32_t k = 0; k < pnnz; ++k)
            pm[k] = (limited || (rs->left_precond && rs->ilu32)) ? (double)(float)pm_vals[k]
                                                                   : pv32(pm_vals[k], rs->pv_mask,
                                                                          ORC_PV_M);
        rc = cycle_f64(n, rowptr, colind, (double *)c.a, (double *)c.r0, m, kmax, ortho, prec,
                       rs, pm_rowptr, pm_colind, pm_vals ? (double *)c.pm : NULL,
                       (double *)c.V, (double *)c.Hb, (double *)c.H, (double *)c.s,
                       (double *)c.cs, (double *)c.sn, (double *)c.y, (double *)c.u, arn, orth,
                       jout, bd);
    }
    if (rc == 0) {
        export_vec(V, c.V, (size_t)(m + 1) * n, is_f32);
        export_vec(Hb, c.Hb, (size_t)(m + 1) * m, is_f32);
        export_vec(H, c.H, (size_t)(m + 1) * m, is_f32);
        export_vec(s, c.s, (size_t)m + 1, is_f32);
        export_vec(cs, c.cs, (size_t)m, is_f32);
        export_vec(sn, c.sn, (size_t)m, is_f32);
        export_vec(y, c.y, (size_t)m, is_f32);
        export_vec(u, c.u, (size_t)n, is_f32);
    }
    cyc_free(&c);
    return rc;
}

static int restart_ok(const orc_restart *rs)
{
    return rs && (rs->pv_mask & ~ORC_PV_ALL) == 0 && rs->tau >= 0 && rs->inner_abs >= 0 && rs->stall_factor >= 0 &&
           (rs->stall_factor == 0 || rs->stall_window >= 1) && rs->orth_norm >= ORC_ORTH_OFF &&
           rs->orth_norm <= ORC_ORTH_FROBENIUS &&
           (rs->orth_norm != ORC_ORTH_SPECTRAL || rs->orth_iters >= 1);
}

int orc_arnoldi_cycle_ex(int32_t n, const int32_t *rowptr, const int32_t *colind,
                         const double *vals, const double *r0, int32_t m, int32_t kmax,
                         int32_t ortho, int32_t prec, const orc_restart *rs,
                         const int32_t *pm_rowptr, const int32_t *pm_colind,
                         const double *pm_vals, double *V, double *Hbar, double *Hrot, double *s,
                         double *cs, double *sn, double *y, double *u, double *arn, double *orth,
                         int32_t *jout, int32_t *breakdown)
{
    if (n <= 0 || m < 1 || kmax < 1 || kmax > m || (ortho != ORC_MGS && ortho != ORC_CGSR) ||
        prec < ORC_FP64 || prec > ORC_MIXED_LIMITED || !csr_ok(n, rowptr, colind) ||
        !restart_ok(rs) || (rs->pv_mask && prec != ORC_FP64))
        return -1;
    if (pm_vals && !csr_ok(n, pm_rowptr, pm_colind))
        return -1;
    if (orth)
        memset(orth, 0, sizeof(double) * (size_t)m);
    int32_t j = 0, bd = 0;
    int rc = run_cycle(n, rowptr, colind, vals, r0, m, kmax, ortho, prec, rs, pm_rowptr,
                       pm_colind, pm_vals, V, Hbar, Hrot, s, cs, sn, y, u, arn, orth, &j, &bd);
    if (jout)
        *jout = j;
    if (breakdown)
        *breakdown = bd;
    return rc;
}

int orc_arnoldi_cycle(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                      const double *r0, int32_t m, int32_t kmax, int32_t ortho, int32_t prec,
                      double tau, double inner_abs,
                      const int32_t *pm_rowptr, const int32_t *pm_colind, const double *pm_vals,
                      double *V, double *Hbar, double *Hrot, double *s, double *cs, double *sn,
                      double *y, double *u, double *arn, int32_t *jout, int32_t *breakdown)
{
    orc_restart rs;
    memset(&rs, 0, sizeof(rs));
    rs.tau = tau;
    rs.inner_abs = inner_abs;
    return orc_arnoldi_cycle_ex(n, rowptr, colind, vals, r0, m, kmax, ortho, prec, &rs,
                                pm_rowptr, pm_colind, pm_vals, V, Hbar, Hrot, s, cs, sn, y, u,
                                arn, NULL, jout, breakdown);
}

int orc_arnoldi_step(int32_t n, const int32_t *rowptr, const int32_t *colind,
                     const double *vals, const double *V, int32_t ncols, int32_t ortho,
                     int32_t prec, double *h, double *vnext)
{
    if (n <= 0 || ncols < 1 || (ortho != ORC_MGS && ortho != ORC_CGSR) || prec < ORC_FP64 ||
        prec > ORC_MIXED_LIMITED || prec == ORC_ALL_FP32 || !V || !h || !vnext ||
        !csr_ok(n, rowptr, colind))
        return -1;
    const int is_f32 = (prec != ORC_FP64 && prec != ORC_MIXED_LIMITED);
    const int32_t nnz = rowptr[n];
    const size_t nv = (size_t)ncols * n;
    int rc;
    if (is_f32) {
        float *a = (float *)malloc(sizeof(float) * (size_t)(nnz + 1));
        float *Vf = (float *)malloc(sizeof(float) * (nv + 1));
        float *hf = (float *)malloc(sizeof(float) * (size_t)(ncols + 1));
        float *vf = (float *)malloc(sizeof(float) * (size_t)n);
        if (!a || !Vf || !hf || !vf) {
            free(a); free(Vf); free(hf); free(vf);
            return -2;
        }
        for (int32_t k = 0; k < nnz; ++k)
            a[k] = (float)vals[k];
        for (size_t i = 0; i < nv; ++i)
            Vf[i] = (float)V[i];
        rc = step_f32(n, rowptr, colind, a, Vf, ncols, ortho, hf, vf);
        if (rc == 0) {
            for (int32_t i = 0; i <= ncols; ++i)
                h[i] = hf[i];
            for (int32_t r = 0; r < n; ++r)
                vnext[r] = vf[r];
        }
        free(a); free(Vf); free(hf); free(vf);
    } else {
        /* limited mixed: the Krylov step's copy of A stored in binary32 */
        double *a = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
        if (!a)
            return -2;
        for (int32_t k = 0; k < nnz; ++k)
            a[k] = prec == ORC_MIXED_LIMITED ? (double)(float)vals[k] : vals[k];
        rc = step_f64(n, rowptr, colind, a, V, ncols, ortho, h, vnext);
        free(a);
    }
    return rc;
}

int orc_threads(int32_t want)
{
#ifdef _OPENMP
    if (want > 0)
        omp_set_num_threads(want);
    return omp_get_max_threads();
#else
    (void)want;
    return 1;
#endif
}

/* Negative control (ORC_ALL_FP32): z = b - A x formed in binary32 from
 * binary32 copies of A, b and x; returns ||z|| in binary32. */
static float residual_f32(int32_t n, const int32_t *rowptr, const int32_t *colind,
                          const float *a, const float *b, const float *x, float *z)
{
    float ss = 0;
    for (int32_t i = 0; i < n; ++i) {
        float acc = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += a[k] * x[colind[k]];
        z[i] = b[i] - acc;
        ss += z[i] * z[i];
    }
    return sqrtf(ss);
}

/* The residual of the per-variable study: z = b - A x with A and b as stored
 * (a, bs: binary32 values under ORC_PV_A_RESID / ORC_PV_B) and the product
 * A x stored in binary32 under ORC_PV_AX before the subtraction; binary64
 * arithmetic.  Returns ||z||_2. */
static double residual_pv(int32_t n, const int32_t *rowptr, const int32_t *colind,
                          const double *a, const double *bs, const double *x, double *z,
                          int32_t pv)
{
    double ss = 0;
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += a[k] * x[colind[k]];
        acc = pv32(acc, pv, ORC_PV_AX);
        double zi = bs[i] - acc;
        z[i] = zi;
        ss += zi * zi;
    }
    return sqrt(ss);
}

int orc_gmres(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
              const double *b, double *x, const orc_opts *o,
              const int32_t *pm_rowptr, const int32_t *pm_colind, const double *pm_vals,
              orc_info *info, double *arn_hist, double *cyc_hist)
{
    if (!o || n <= 0 || o->m < 1 || o->maxiter < 0 || !(o->tol > 0) ||
        (o->ortho != ORC_MGS && o->ortho != ORC_CGSR) || o->prec < ORC_FP64 ||
        o->prec > ORC_MIXED_LIMITED || !csr_ok(n, rowptr, colind) || !b || !x ||
        o->stall_factor < 0 || o->stall_window < 0 || o->orth_norm < ORC_ORTH_OFF ||
        o->orth_norm > ORC_ORTH_FROBENIUS ||
        (o->orth_norm == ORC_ORTH_SPECTRAL && o->orth_iters < 1) ||
        (o->pv_mask & ~ORC_PV_ALL) || (o->pv_mask && o->prec != ORC_FP64))
        return -1;
    if (pm_vals && !csr_ok(n, pm_rowptr, pm_colind))
        return -1;

    const int32_t m = o->m;
    /* refinement variables of the per-variable study stored in binary32 */
    const int32_t pvr = o->pv_mask & (ORC_PV_A_RESID | ORC_PV_B | ORC_PV_X | ORC_PV_AX);
    orc_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.bnorm = nrm2_f64(n, b);

    /* A zero right-hand side has the solution x = 0. */
    if (inf.bnorm == 0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        inf.converged = 1;
        if (cyc_hist)
            cyc_hist[0] = 0;
        if (info)
            *info = inf;
        return 0;
    }

    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *arn = (double *)malloc(sizeof(double) * (size_t)m);
    float *a32 = NULL, *b32 = NULL, *x32 = NULL, *z32 = NULL;
    if (o->prec == ORC_ALL_FP32) {
        int32_t nnz = rowptr[n];
        a32 = (float *)malloc(sizeof(float) * (size_t)(nnz + 1));
        b32 = (float *)malloc(sizeof(float) * (size_t)n);
        x32 = (float *)malloc(sizeof(float) * (size_t)n);
        z32 = (float *)malloc(sizeof(float) * (size_t)n);
        if (a32 && b32 && x32 && z32) {
            for (int32_t k = 0; k < nnz; ++k)
                a32[k] = (float)vals[k];
            for (int32_t i = 0; i < n; ++i) {
                b32[i] = (float)b[i];
                x32[i] = (float)x[i];
            }
        }
    }
    double *ar = NULL, *br = NULL;
    if (pvr) {
        int32_t nnz = rowptr[n];
        ar = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
        br = (double *)malloc(sizeof(double) * (size_t)n);
        if (ar && br) {
            for (int32_t k = 0; k < nnz; ++k)
                ar[k] = pv32(vals[k], pvr, ORC_PV_A_RESID);
            for (int32_t i = 0; i < n; ++i) {
                br[i] = pv32(b[i], pvr, ORC_PV_B);
                x[i] = pv32(x[i], pvr, ORC_PV_X);
            }
        }
    }
    if (!z || !u || !arn || (o->prec == ORC_ALL_FP32 && (!a32 || !b32 || !x32 || !z32)) ||
        (pvr && (!ar || !br))) {
        free(z); free(u); free(arn); free(a32); free(b32); free(x32); free(z32);
        free(ar); free(br);
        return -2;
    }

    orc_restart rs;
    memset(&rs, 0, sizeof(rs));
    rs.inner_abs = o->inner_factor * o->tol * inf.bnorm;
    rs.stall_factor = o->stall_factor;
    rs.stall_window = o->stall_window > 0 ? o->stall_window : (m + 19) / 20;
    rs.orth_norm = o->orth_norm;
    rs.orth_threshold = o->orth_threshold;
    rs.orth_iters = o->orth_iters;
    rs.split_bytes = o->split_bytes;
    rs.left_precond = o->left_precond;
    rs.ilu32 = o->ilu32;
    rs.pv_mask = o->pv_mask;
    int32_t cycle_len = m;
    int rc = 0;
    for (;;) {
        /* z_k = b - A x_k and the convergence test, in binary64 (binary32 for
         * the negative control, whose x lives in binary32). */
        double rn;
        if (o->prec == ORC_ALL_FP32) {
            for (int32_t i = 0; i < n; ++i)
                x[i] = x32[i];
            float rn32 = residual_f32(n, rowptr, colind, a32, b32, x32, z32);
            for (int32_t i = 0; i < n; ++i)
                z[i] = z32[i];
            rn = rn32;
        } else if (pvr) {
            rn = residual_pv(n, rowptr, colind, ar, br, x, z, pvr);
        } else {
            rn = orc_residual(n, rowptr, colind, vals, b, x, z);
        }
        double true_rel = (o->prec == ORC_ALL_FP32 || pvr)
                              ? orc_residual(n, rowptr, colind, vals, b, x, NULL) / inf.bnorm
                              : rn / inf.bnorm;
        if (cyc_hist)
            cyc_hist[inf.restarts] = true_rel;
        inf.relres = true_rel;
        if (rn <= o->tol * inf.bnorm) {
            inf.converged = (true_rel <= o->tol);
            break;
        }
        if (inf.iters >= o->maxiter)
            break;

        int32_t kmax = cycle_len;
        if (kmax > o->maxiter - inf.iters)
            kmax = o->maxiter - inf.iters;
        /* Two-stage restart (Sec. 3, first strategy; Sec. 4.2): with
         * repeat_first the gain threshold only ends the first cycle, later
         * cycles run for the first cycle's length. */
        rs.tau = (o->repeat_first && inf.restarts > 0) ? 0.0 : o->tau;
        int32_t j = 0, bd = 0;
        rc = run_cycle(n, rowptr, colind, vals, z, m, kmax, o->ortho, o->prec, &rs, pm_rowptr,
                       pm_colind, pm_vals, NULL, NULL, NULL, NULL, NULL, NULL, NULL, u, arn,
                       NULL, &j, &bd);
        if (rc)
            break;
        if (j == 0)
            break;  /* the working-precision residual vanished: nothing to add */

        /* x_{k+1} = x_k + u_k: binary64 addition of the (converted) correction. */
        if (o->prec == ORC_ALL_FP32) {
            for (int32_t i = 0; i < n; ++i)
                x32[i] = x32[i] + (float)u[i];
        } else {
            #pragma omp parallel for schedule(static)
            for (int32_t i = 0; i < n; ++i) {
                x[i] = x[i] + u[i];
                x[i] = pv32(x[i], pvr, ORC_PV_X);
            }
        }
        if (arn_hist)
            for (int32_t i = 0; i < j; ++i)
                arn_hist[inf.iters + i] = arn[i];
        inf.iters += j;
        inf.restarts += 1;
        if (inf.restarts == 1) {
            inf.first_len = j;
            if (o->repeat_first)
                cycle_len = j;
        }
    }
    if (o->prec == ORC_ALL_FP32)
        for (int32_t i = 0; i < n; ++i)
            x[i] = x32[i];
    if (info)
        *info = inf;
    free(z); free(u); free(arn); free(a32); free(b32); free(x32); free(z32);
    free(ar); free(br);
    return rc;
}
