// orth_monitor.cuh -- the loss-of-orthogonality restart test of arXiv
// 2011.01850, Sec. 3 (fourth strategy).
//
// For the k stored basis vectors V_k = [v_1 .. v_k] of the current cycle let
// U_k be the strictly upper part of V_k^T V_k and S_k = (I + U_k)^-1 U_k.
// For unit vectors ||S_k||_2 <= 1, with equality exactly when they are
// linearly dependent (Paige), so a norm near 1 signals a stalled basis.
// Appending v_k adds one column to each matrix: u = V_{k-1}^T v_k (a pass
// over the basis, k_cgs_rows MODE 3 + k_reduce_cols) and the new column of
// S_k, (I + U_{k-1})^-1 u, a unit upper triangular solve.  The norm is the
// Frobenius norm or the power method's estimate of the 2-norm on S^T S
// (10 iterations in Sec. 4.1); the cycle ends when it reaches the
// threshold.  The small dense work runs in binary64 in one block.
#pragma once

#include "grid_kernels.cuh"

namespace gmres {

constexpr int ORTH_THREADS = 256;
constexpr int ORTH_LD = MMAX + 1;  // leading dimension of U and S

struct OrthMon {
    double *U, *S;   // ORTH_LD x ORTH_LD, column-major
    double *hist;    // ||S_k|| per inner iteration of the cycle (index k - 2)
    double threshold;
    int norm;        // 1 spectral (power method), 2 Frobenius
    int iters;       // power-method iterations
};

// y_i = sum_{l > i} S_il x_l for i < k (thread per row)
__device__ __forceinline__ void s_matvec(const double *S, int k, const double *x, double *y) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double acc = 0;
        for (int l = i + 1; l < k; ++l)
            acc += S[(size_t)l * ORTH_LD + i] * x[l];
        y[i] = acc;
    }
}

// z_l = sum_{i < l} S_il y_i for l < k (thread per column)
__device__ __forceinline__ void st_matvec(const double *S, int k, const double *y, double *z) {
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        const double *col = S + (size_t)l * ORTH_LD;
        double acc = 0;
        for (int i = 0; i < l; ++i)
            acc += col[i] * y[i];
        z[l] = acc;
    }
}

// k = basis vectors including the new one (>= 2); u[0..k-2] = v_i . v_k.
// Runs only when inner iteration k-1 has just completed without breakdown
// (ctl->j == k-1), so the history covers every iteration that appended a
// vector, including the one that ends the cycle for another reason.
template <class T>
__global__ void __launch_bounds__(ORTH_THREADS) k_orth_monitor(Ctl *ctl, const T *u, int k,
                                                               OrthMon M) {
    if (ctl->j != k - 1 || ctl->breakdown || ctl->nonfinite)
        return;
    __shared__ double xs[MMAX + 2], ys[MMAX + 2], red[32];
    double *ucol = M.U + (size_t)(k - 1) * ORTH_LD;
    double *scol = M.S + (size_t)(k - 1) * ORTH_LD;
    for (int i = threadIdx.x; i < k - 1; i += blockDim.x)
        ucol[i] = (double)ldcg(u + i);
    __syncthreads();
    // new column of S: (I + U_{k-1}) x = u, rows k-2 down to 0 (warp 0)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int i = k - 2; i >= 0; --i) {
            double acc = 0;
            for (int l = i + 1 + lane; l <= k - 2; l += 32)
                acc += M.U[(size_t)l * ORTH_LD + i] * xs[l];
            acc = warp_sum(acc);
            if (lane == 0)
                xs[i] = ucol[i] - acc;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k - 1; i += blockDim.x)
        scol[i] = xs[i];
    __syncthreads();
    double nrm;
    if (M.norm == 2) {
        double ss = 0;
        for (int l = 1; l < k; ++l)
            for (int i = threadIdx.x; i < l; i += blockDim.x) {
                const double v = M.S[(size_t)l * ORTH_LD + i];
                ss += v * v;
            }
        nrm = sqrt(block_sum1(ss, red));
    } else {
        // power method on S^T S from the vector of equal entries
        for (int i = threadIdx.x; i < k; i += blockDim.x)
            xs[i] = 1.0 / sqrt((double)k);
        __syncthreads();
        bool zero = false;
        for (int t = 0; t < M.iters && !zero; ++t) {
            s_matvec(M.S, k, xs, ys);
            __syncthreads();
            st_matvec(M.S, k, ys, xs);
            double ss = 0;
            for (int l = threadIdx.x; l < k; l += blockDim.x)
                ss += xs[l] * xs[l];
            const double zn = sqrt(block_sum1(ss, red));
            if (zn == 0) {
                zero = true;
            } else {
                for (int l = threadIdx.x; l < k; l += blockDim.x)
                    xs[l] /= zn;
            }
            __syncthreads();
        }
        if (zero) {
            nrm = 0;
        } else {
            s_matvec(M.S, k, xs, ys);
            __syncthreads();
            double ss = 0;
            for (int i = threadIdx.x; i < k; i += blockDim.x)
                ss += ys[i] * ys[i];
            nrm = sqrt(block_sum1(ss, red));
        }
    }
    if (threadIdx.x == 0) {
        M.hist[k - 2] = nrm;
        if (nrm >= M.threshold)
            ctl->active = 0;
    }
}

}  // namespace gmres
