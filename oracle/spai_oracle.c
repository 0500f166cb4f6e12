/*
 * spai_oracle.c -- CPU oracle for the learned sparse-approximate-inverse
 * (SpAI) right preconditioner: per-nonzero features, the 8 -> 64 -> 64 -> 1
 * MLP that predicts M's values on A's sparsity pattern, the probe loss
 * L = 1/(2 P n) sum_p ||A M z_p - z_p||^2 and its exact gradients.
 *
 * TEST INFRASTRUCTURE ONLY (see gmres_oracle.c).  Binary64 throughout, plain
 * loops, sequential sums.  The paper has no preconditioner of this kind; it
 * uses ILU(0) on the left (Sec. 4).  This is the right-preconditioned
 * variant (A M y = b, x = M y) whose values are learned.
 *
 * Features of nonzero (p, q) with value a, d_p = a_pp, d_q = a_qq (a zero
 * diagonal counts as 1):
 *   f0 = a / d_p            f1 = d_q / d_p          f2 = [p == q]
 *   f3 = sum_k |a_pk| / |d_p|                        (row weight)
 *   f4 = sum_k |a_kq| / |d_q|                        (column weight)
 *   f5 = nnz(row p) / 8     f6 = sign(a)            f7 = sign(q - p)
 * MLP: z1 = W1 f + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
 *      g = w3 . h2 + b3, and m_pq = g / d_p (so g = [p == q] gives M = D^-1).
 * Parameter layout (4801 values): W1[64][8], b1[64], W2[64][64], b2[64],
 * w3[64], b3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 8
#define NH 64
#define P_W1 0
#define P_B1 (P_W1 + NH * NF)
#define P_W2 (P_B1 + NH)
#define P_B2 (P_W2 + NH * NH)
#define P_W3 (P_B2 + NH)
#define P_B3 (P_W3 + NH)
#define NPARAM (P_B3 + 1)

int orc_spai_nparam(void) { return NPARAM; }

static double diag_of(int32_t i, const int32_t *rowptr, const int32_t *colind, const double *vals)
{
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (colind[k] == i)
            return vals[k] != 0 ? vals[k] : 1.0;
    return 1.0;
}

static double sgn(double v) { return (v > 0) - (v < 0); }

int orc_spai_features(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                      double *feat)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *rs = (double *)calloc((size_t)n, sizeof(double));
    double *cs = (double *)calloc((size_t)n, sizeof(double));
    if (!d || !rs || !cs) {
        free(d); free(rs); free(cs);
        return -2;
    }
    for (int32_t i = 0; i < n; ++i) {
        d[i] = diag_of(i, rowptr, colind, vals);
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            rs[i] += fabs(vals[k]);
            cs[colind[k]] += fabs(vals[k]);
        }
    }
    for (int32_t p = 0; p < n; ++p) {
        for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k) {
            int32_t q = colind[k];
            double *f = feat + (size_t)k * NF;
            f[0] = vals[k] / d[p];
            f[1] = d[q] / d[p];
            f[2] = (p == q) ? 1.0 : 0.0;
            f[3] = rs[p] / fabs(d[p]);
            f[4] = cs[q] / fabs(d[q]);
            f[5] = (double)(rowptr[p + 1] - rowptr[p]) / 8.0;
            f[6] = sgn(vals[k]);
            f[7] = sgn((double)q - (double)p);
        }
    }
    free(d); free(rs); free(cs);
    return 0;
}

/* Forward pass for one feature vector; keeps z1, z2 for the backward pass. */
static double mlp_fwd(const double *f, const double *w, double *z1, double *z2)
{
    double h1[NH];
    for (int o = 0; o < NH; ++o) {
        double a = w[P_B1 + o];
        for (int i = 0; i < NF; ++i)
            a += w[P_W1 + o * NF + i] * f[i];
        z1[o] = a;
        h1[o] = a > 0 ? a : 0;
    }
    double g = w[P_B3];
    for (int o = 0; o < NH; ++o) {
        double a = w[P_B2 + o];
        for (int i = 0; i < NH; ++i)
            a += w[P_W2 + o * NH + i] * h1[i];
        z2[o] = a;
        g += w[P_W3 + o] * (a > 0 ? a : 0);
    }
    return g;
}

int orc_spai_forward(int64_t nnz, const double *feat, const double *params, double *g)
{
    double z1[NH], z2[NH];
    for (int64_t k = 0; k < nnz; ++k)
        g[k] = mlp_fwd(feat + (size_t)k * NF, params, z1, z2);
    return 0;
}

/* M's values on A's pattern: m_pq = g_pq / a_pp. */
int orc_spai_values(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
                    const double *params, double *mvals)
{
    int64_t nnz = rowptr[n];
    double *feat = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1) * NF);
    if (!feat)
        return -2;
    orc_spai_features(n, rowptr, colind, vals, feat);
    orc_spai_forward(nnz, feat, params, mvals);
    for (int32_t p = 0; p < n; ++p) {
        double dp = diag_of(p, rowptr, colind, vals);
        for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k)
            mvals[k] /= dp;
    }
    free(feat);
    return 0;
}

/* y = A x with the values `v` on A's pattern. */
static void csr_mv(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *v,
                   const double *x, double *y)
{
    for (int32_t i = 0; i < n; ++i) {
        double a = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            a += v[k] * x[colind[k]];
        y[i] = a;
    }
}

/* Loss L = 1/(2 P n) sum_p ||A M z_p - z_p||^2 for M given by its values
 * mvals on A's pattern, over the P probe vectors (columns of Z, n x P
 * column-major), and dL/dm_pq = 1/(P n) sum_p (A^T r_p)_p z_p[q] with
 * r_p = A M z_p - z_p, on A's pattern (grad_m, may be NULL). */
double orc_spai_loss_grad_m(int32_t n, const int32_t *rowptr, const int32_t *colind,
                            const double *vals, const double *mvals, int32_t P, const double *Z,
                            double *grad_m)
{
    int64_t nnz = rowptr[n];
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *atr = (double *)malloc(sizeof(double) * (size_t)n);
    if (!u || !r || !atr) {
        free(u); free(r); free(atr);
        return NAN;
    }
    if (grad_m)
        memset(grad_m, 0, sizeof(double) * (size_t)nnz);
    const double scale = 1.0 / ((double)P * (double)n);
    double loss = 0;
    for (int32_t pr = 0; pr < P; ++pr) {
        const double *z = Z + (size_t)pr * n;
        csr_mv(n, rowptr, colind, mvals, z, u);  /* u = M z      */
        csr_mv(n, rowptr, colind, vals, u, r);   /* r = A u - z  */
        for (int32_t i = 0; i < n; ++i) {
            r[i] -= z[i];
            loss += r[i] * r[i];
        }
        if (!grad_m)
            continue;
        /* A^T r, scattered row by row */
        memset(atr, 0, sizeof(double) * (size_t)n);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                atr[colind[k]] += vals[k] * r[i];
        for (int32_t p = 0; p < n; ++p)
            for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k)
                grad_m[k] += atr[p] * z[colind[k]];
    }
    if (grad_m)
        for (int64_t k = 0; k < nnz; ++k)
            grad_m[k] *= scale;
    free(u); free(r); free(atr);
    return 0.5 * scale * loss;
}

/* The same loss as a function of the MLP parameters (m_pq = g_pq / a_pp),
 * with the parameter gradient by the chain rule (grad_params, may be NULL)
 * and dL/dm (grad_m, may be NULL). */
double orc_spai_loss_grad(int32_t n, const int32_t *rowptr, const int32_t *colind,
                          const double *vals, const double *params, int32_t P, const double *Z,
                          double *grad_params, double *grad_m)
{
    int64_t nnz = rowptr[n];
    double *feat = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1) * NF);
    double *m = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *gm = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    double *dg = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!feat || !m || !gm || !dg) {
        free(feat); free(m); free(gm); free(dg);
        return NAN;
    }
    orc_spai_features(n, rowptr, colind, vals, feat);
    orc_spai_forward(nnz, feat, params, m);
    for (int32_t p = 0; p < n; ++p) {
        dg[p] = diag_of(p, rowptr, colind, vals);
        for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k)
            m[k] /= dg[p];
    }
    double loss = orc_spai_loss_grad_m(n, rowptr, colind, vals, m, P, Z, gm);
    if (grad_m)
        memcpy(grad_m, gm, sizeof(double) * (size_t)nnz);
    if (grad_params) {
        memset(grad_params, 0, sizeof(double) * NPARAM);
        double z1[NH], z2[NH], d2[NH], d1[NH], h1[NH];
        for (int32_t p = 0; p < n; ++p) {
            for (int32_t k = rowptr[p]; k < rowptr[p + 1]; ++k) {
                const double *f = feat + (size_t)k * NF;
                mlp_fwd(f, params, z1, z2);
                const double dgk = gm[k] / dg[p]; /* dL/dg_pq */
                for (int o = 0; o < NH; ++o)
                    h1[o] = z1[o] > 0 ? z1[o] : 0;
                grad_params[P_B3] += dgk;
                for (int o = 0; o < NH; ++o) {
                    double h2 = z2[o] > 0 ? z2[o] : 0;
                    grad_params[P_W3 + o] += dgk * h2;
                    d2[o] = z2[o] > 0 ? dgk * params[P_W3 + o] : 0;
                    grad_params[P_B2 + o] += d2[o];
                    for (int i = 0; i < NH; ++i)
                        grad_params[P_W2 + o * NH + i] += d2[o] * h1[i];
                }
                for (int i = 0; i < NH; ++i) {
                    double a = 0;
                    for (int o = 0; o < NH; ++o)
                        a += params[P_W2 + o * NH + i] * d2[o];
                    d1[i] = z1[i] > 0 ? a : 0;
                    grad_params[P_B1 + i] += d1[i];
                    for (int j = 0; j < NF; ++j)
                        grad_params[P_W1 + i * NF + j] += d1[i] * f[j];
                }
            }
        }
    }
    free(feat); free(m); free(gm); free(dg);
    return loss;
}

/* One Adam step (Kingma and Ba, 2015) in binary64:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void orc_adam_step(int32_t np, double *p, double *m, double *v, const double *g, int32_t t,
                   double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int32_t i = 0; i < np; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
