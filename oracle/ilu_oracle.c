/*
 * ilu_oracle.c -- incomplete LU without fill, ILU(0), the preconditioner of
 * the paper's experiments (Sec. 4: left preconditioning by ILU(0), also with
 * the factors stored in binary32), and its two triangular solves.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/ and the benchmark's CPU legs,
 * never by the CUDA library.  Plain sequential code in binary64.
 *
 * ILU(0) keeps the sparsity pattern of A: L (unit lower, strictly-lower
 * entries of the pattern) and U (upper entries including the diagonal) are
 * the factors of the row-by-row Gaussian elimination that drops every update
 * falling outside the pattern (the IKJ form of ILU(0) in Saad, "Iterative
 * Methods for Sparse Linear Systems", Sec. 10.3).  The defining property the
 * tests check: (L U)_{ij} = a_{ij} for every (i, j) in the pattern.
 */
#include "gmres_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Position of column col in row i of a sorted CSR row, or -1. */
static int32_t find_in_row(const int32_t *rowptr, const int32_t *colind, int32_t i, int32_t col)
{
    int32_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (colind[mid] == col)
            return mid;
        if (colind[mid] < col)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

int orc_ilu0(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *vals,
             double *lu)
{
    if (n <= 0 || !rowptr || !colind || !vals || !lu)
        return -1;
    /* sorted rows with a diagonal entry */
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = rowptr[i] + 1; k < rowptr[i + 1]; ++k)
            if (colind[k] <= colind[k - 1])
                return -1;
        if (find_in_row(rowptr, colind, i, i) < 0)
            return -1;
    }
    memcpy(lu, vals, sizeof(double) * (size_t)rowptr[n]);
    for (int32_t i = 0; i < n; ++i) {
        /* eliminate with every earlier row k of row i's pattern, in
         * ascending order of k */
        for (int32_t p = rowptr[i]; p < rowptr[i + 1] && colind[p] < i; ++p) {
            const int32_t k = colind[p];
            const double pivot = lu[find_in_row(rowptr, colind, k, k)];
            if (pivot == 0.0 || !isfinite(pivot))
                return -3;
            lu[p] = lu[p] / pivot; /* l_ik */
            /* a_ij -= l_ik u_kj for the j > k that are in both rows */
            for (int32_t q = p + 1; q < rowptr[i + 1]; ++q) {
                const int32_t j = colind[q];
                const int32_t kj = find_in_row(rowptr, colind, k, j);
                if (kj >= 0)
                    lu[q] = lu[q] - lu[p] * lu[kj];
            }
        }
        const double d = lu[find_in_row(rowptr, colind, i, i)];
        if (d == 0.0 || !isfinite(d))
            return -3;
    }
    return 0;
}

int orc_ilu_apply(int32_t n, const int32_t *rowptr, const int32_t *colind, const double *lu,
                  const double *z, double *out)
{
    if (n <= 0 || !rowptr || !colind || !lu || !z || !out)
        return -1;
    /* L y = z, L unit lower: rows in increasing order, sums in column order */
    for (int32_t i = 0; i < n; ++i) {
        double acc = z[i];
        for (int32_t p = rowptr[i]; p < rowptr[i + 1] && colind[p] < i; ++p)
            acc -= lu[p] * out[colind[p]];
        out[i] = acc;
    }
    /* U x = y: rows in decreasing order */
    for (int32_t i = n - 1; i >= 0; --i) {
        double acc = out[i], d = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int32_t j = colind[p];
            if (j == i)
                d = lu[p];
            else if (j > i)
                acc -= lu[p] * out[j];
        }
        out[i] = acc / d;
    }
    return 0;
}
