// block_solver.cuh -- one thread block runs a whole restarted GMRES(m) solve
// (Algorithm 1 of arXiv 2011.01850) for one system.
//
// Used for small systems, where whole-GPU kernels would be launch-latency
// bound, and by the batched solver: a persistent grid takes systems from a
// work queue (largest first), one block per system, so many independent
// systems of uneven size are solved in one launch.  Reductions are block-wide
// (xor-butterfly + shared memory, deterministic); the Hessenberg matrix, the
// rotations and s live in shared memory; vectors and the basis live in the
// system's global workspace (L1/L2 resident for small n).
//
// The same routine also runs on a thread-block cluster (CS > 1 CTAs): the
// system's rows are split into CS contiguous chunks, every reduction is a
// block reduction followed by an exchange of the CTAs' partials through
// distributed shared memory (double-buffered slots, summed in rank order so
// every CTA gets the same value bit for bit), the Givens step and the back
// substitution run redundantly in every CTA, and cluster barriers order the
// global writes other CTAs gather (x, v_1, v_{j+1}).  Large systems of a batch
// use clusters so that one system is not the critical path of the batch.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace gmres {

namespace cg = cooperative_groups;

constexpr int TEAM_KMAX = 8;  // values per team reduction

// A team is one thread block (CS = 1) or one thread-block cluster (CS > 1).
template <int CS>
struct Team {
    __device__ __forceinline__ static int rank() { return (int)cg::this_cluster().block_rank(); }
    __device__ __forceinline__ static void sync() { cg::this_cluster().sync(); }
};
template <>
struct Team<1> {
    __device__ __forceinline__ static int rank() { return 0; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};

// Team-wide sums of K values (every thread receives them).  red: K*32 block
// scratch; slots: 2*TEAM_KMAX shared slots (double-buffered by *buf); bc:
// TEAM_KMAX broadcast cells.
template <class T, int K, int CS>
__device__ __forceinline__ void team_sum(T (&v)[K], T *red, T *slots, T *bc, int *buf) {
    block_sum<T, K>(v, red);
    if (CS == 1)
        return;
    T *mine = slots + (*buf) * TEAM_KMAX;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            mine[k] = v[k];
    }
    Team<CS>::sync();
    if (threadIdx.x < 32) {
        // lane r reads rank r's partials (all ranks at once), then an xor
        // butterfly over the CS lanes: every block forms the same sums
        cg::cluster_group cl = cg::this_cluster();
        const int lane = threadIdx.x;
        const T *src = cl.map_shared_rank(mine, lane < CS ? lane : 0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T a = lane < CS ? src[k] : T(0);
#pragma unroll
            for (int off = CS / 2; off > 0; off >>= 1)
                a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0)
                bc[k] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
        v[k] = bc[k];
    __syncthreads();
    *buf ^= 1;
}

template <class T, int CS>
__device__ __forceinline__ T team_sum1(T v, T *red, T *slots, T *bc, int *buf) {
    T a[1] = {v};
    team_sum<T, 1, CS>(a, red, slots, bc, buf);
    return a[0];
}

// One system of a block solve.  All pointers are device pointers; V and the
// work vectors (w, r) are library workspace of at least ldv rows.
template <class T, class VT>
struct BlockSys {
    int n;
    int64_t ldv;
    const int *rowptr;
    const int *colind;
    const T *a;
    const double *a64;
    const double *b;
    double *x;
    VT *V;
    T *w;
    T *r;
    float vscale, vinv;
};

// Per-system result written by the block solver.
struct BlockResult {
    int iters, restarts, converged, first_len;
    int status;  // gmres_status value
    int pad;
    double relres, bnorm;
};

struct BlockParams {
    int m, maxiter, ortho, repeat_first;
    double tol, tau, inner_factor;
    double brk;
    int nsys;
    unsigned *queue;  // work-queue counter (reset by the host)
    const int *order; // system order (largest first)
    // third restart strategy (Sec. 3): end the cycle once |s_{j+1}| improved
    // by less than stall_factor over the last stall_w iterations (0 = off)
    double stall_factor = 0;
    int stall_w = 1;
};

// w[row] = A x for the system's rows rb..n-1 (of ncol), L lanes per row.
template <class T, class XT, int L>
__device__ __forceinline__ void block_spmv(const int *__restrict__ rowptr,
                                           const int *__restrict__ colind,
                                           const T *__restrict__ a, const XT *x, float xinv, T *y,
                                           int rb, int n, int ncol) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int G = 32 / L, gl = lane % L, gi = lane / L;
    for (int base = rb + wid * G; base < n; base += nw * G) {
        int row = base + gi;
        T acc = 0;
        if (row < n) {
            int beg = rowptr[row], end = rowptr[row + 1];
            for (int k = beg + gl; k < end; k += L)
                acc += a[k] * (T)Basis<XT>::ld(x + chk_col(colind[k], ncol), xinv);
        }
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (row < n && gl == 0)
            y[row] = acc;
    }
}

template <class T, class VT, int L, int CS>
__device__ void team_solve_one(const BlockSys<T, VT> &S, const BlockParams &P, BlockResult *res,
                               unsigned char *smem_raw) {
    const int n = S.n, m = P.m, ld = m + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    // this CTA's rows
    const int chunk = (n + CS - 1) / CS;
    const int rb = Team<CS>::rank() * chunk;
    const int re = rb + chunk < n ? rb + chunk : n;
    double *redd = reinterpret_cast<double *>(smem_raw);       // 32 (first: 8-byte aligned)
    double *slotd = redd + 32;                                 // 2 * TEAM_KMAX
    double *bcd = slotd + 2 * TEAM_KMAX;                       // TEAM_KMAX
    double *ahist = bcd + TEAM_KMAX;                           // MMAX + 2: |s_{j+1}|, j = 0..
    T *H = reinterpret_cast<T *>(ahist + MMAX + 2);            // ld x m (rotated)
    T *s = H + (size_t)ld * m;                   // m + 1
    T *cs = s + (m + 1);                         // m
    T *sn = cs + m;                              // m
    T *y = sn + m;                               // m
    T *hc = y + m;                               // MMAX + 2 (current column)
    T *hc2 = hc + (MMAX + 2);                    // MMAX + 2 (second CGS pass)
    T *red = hc2 + (MMAX + 2);                   // 8 * 32
    T *slot = red + 8 * 32;                      // 2 * TEAM_KMAX
    T *bc = slot + 2 * TEAM_KMAX;                // TEAM_KMAX
    __shared__ int s_flag;
    int bufd = 0, buft = 0;

    // ||b||
    double bb = 0;
    for (int i = rb + tid; i < re; i += nth)
        bb += S.b[i] * S.b[i];
    double bnorm = sqrt(team_sum1<double, CS>(bb, redd, slotd, bcd, &bufd));
    BlockResult out;
    out.iters = 0;
    out.restarts = 0;
    out.converged = 0;
    out.first_len = 0;
    out.status = 1;
    out.relres = 0;
    out.bnorm = bnorm;
    if (!(bnorm > 0)) {
        for (int i = rb + tid; i < re; i += nth)
            S.x[i] = 0.0;
        out.converged = isfinite(bnorm) ? 1 : 0;
        out.status = isfinite(bnorm) ? 0 : -3;
        if (tid == 0 && Team<CS>::rank() == 0)
            *res = out;
        Team<CS>::sync();
        return;
    }
    const double tol_abs = P.tol * bnorm;
    const double inner_abs = P.inner_factor * P.tol * bnorm;
    const T brk = (T)P.brk;
    int cycle_len = m;

    for (;;) {
        // every CTA's x rows are final before the residual gathers them
        Team<CS>::sync();
        // z = b - A x (binary64), r = fl(z), ||z||, ||r||.
        double acc2[2] = {0, 0};  // ||z||^2, non-finite count
        T sst = 0;
        {
            const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
            const int G = 32 / L, gl = lane % L, gi = lane / L;
            for (int base = rb + wid * G; base < re; base += nw * G) {
                int row = base + gi;
                double acc = 0;
                if (row < re) {
                    int beg = S.rowptr[row], end = S.rowptr[row + 1];
                    for (int k = beg + gl; k < end; k += L)
                        acc += S.a64[k] * S.x[chk_col(S.colind[k], S.n)];
                }
#pragma unroll
                for (int off = L / 2; off > 0; off >>= 1)
                    acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (row < re && gl == 0) {
                    double zi = S.b[row] - acc;
                    T ri = (T)zi;
                    S.r[row] = ri;
                    acc2[0] += zi * zi;
                    sst += ri * ri;
                    acc2[1] += isfinite(zi) ? 0.0 : 1.0;
                }
            }
        }
        team_sum<double, 2, CS>(acc2, redd, slotd, bcd, &bufd);
        double rn = sqrt(acc2[0]);
        T beta = wsqrt(team_sum1<T, CS>(sst, red, slot, bc, &buft));
        const bool bad = acc2[1] != 0.0;
        out.relres = rn / bnorm;
        if (bad || !isfinite(rn)) {
            out.status = -3;
            break;
        }
        if (rn <= tol_abs) {
            out.converged = 1;
            out.status = 0;
            break;
        }
        if (out.iters >= P.maxiter) {
            out.status = 1;
            break;
        }
        if (!(beta > T(0)))
            break;
        int kmax = cycle_len;
        if (kmax > P.maxiter - out.iters)
            kmax = P.maxiter - out.iters;
        const double tau = (P.repeat_first && out.restarts > 0) ? 0.0 : P.tau;

        // v_1 = r / beta, s = beta e_1
        for (int i = rb + tid; i < re; i += nth)
            Basis<VT>::st(S.V + i, S.r[i] / beta, S.vscale);
        for (int i = tid; i <= m; i += nth)
            s[i] = (i == 0) ? beta : T(0);
        if (tid == 0)
            ahist[0] = (double)beta;
        Team<CS>::sync();

        int j = 0;
        int cyc_bad = 0;
        for (;;) {
            const int c = j;
            const VT *vj = S.V + (size_t)c * S.ldv;
            block_spmv<T, VT, L>(S.rowptr, S.colind, S.a, vj, S.vinv, S.w, rb, re, S.n);
            __syncthreads();
            // ||A v_j|| (breakdown reference)
            T w0 = 0;
            for (int i = rb + tid; i < re; i += nth)
                w0 += S.w[i] * S.w[i];
            T wnorm0 = wsqrt(team_sum1<T, CS>(w0, red, slot, bc, &buft));
            if (P.ortho == 0) {
                // MGS: h_i = w . v_i, w <- w - h_i v_i, one column at a time.
                // Every thread owns the rows rb + tid + k nth, so the update
                // of column i and the dot product of column i + 1 share one
                // pass over the rows: each row is updated, then multiplied,
                // the same operations in the same order as two passes, with
                // one pass of latency per column instead of two.
                T d = 0;
                for (int r = rb + tid; r < re; r += nth)
                    d += S.w[r] * Basis<VT>::ld(S.V + r, S.vinv);
                for (int i = 0; i <= c; ++i) {
                    const T hi = team_sum1<T, CS>(d, red, slot, bc, &buft);
                    if (tid == 0)
                        hc[i] = hi;
                    const VT *vi = S.V + (size_t)i * S.ldv;
                    d = 0;
                    if (i < c) {
                        const VT *vn = vi + S.ldv;
                        for (int r = rb + tid; r < re; r += nth) {
                            const T wr = S.w[r] - hi * Basis<VT>::ld(vi + r, S.vinv);
                            S.w[r] = wr;
                            d += wr * Basis<VT>::ld(vn + r, S.vinv);
                        }
                    } else {
                        for (int r = rb + tid; r < re; r += nth)
                            S.w[r] = S.w[r] - hi * Basis<VT>::ld(vi + r, S.vinv);
                    }
                }
                __syncthreads();
            } else {
                // CGSR: two classical passes, column = sum of both
                for (int pass = 0; pass < 2; ++pass) {
                    for (int c0 = 0; c0 <= c; c0 += 8) {
                        T acc[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            acc[k] = 0;
                        for (int r = rb + tid; r < re; r += nth) {
                            T wr = S.w[r];
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                if (c0 + k <= c)
                                    acc[k] += Basis<VT>::ld(S.V + (size_t)(c0 + k) * S.ldv + r,
                                                            S.vinv) * wr;
                        }
                        team_sum<T, 8, CS>(acc, red, slot, bc, &buft);
                        if (tid == 0) {
                            T *g = pass ? hc2 : hc;
#pragma unroll
                            for (int k = 0; k < 8; ++k)
                                if (c0 + k <= c)
                                    g[c0 + k] = acc[k];
                        }
                    }
                    __syncthreads();
                    // w <- w - V g  (g = this pass's projections)
                    for (int r = rb + tid; r < re; r += nth) {
                        T t = 0;
                        for (int i = 0; i <= c; ++i) {
                            T g = pass ? hc2[i] : hc[i];
                            t += Basis<VT>::ld(S.V + (size_t)i * S.ldv + r, S.vinv) * g;
                        }
                        S.w[r] = S.w[r] - t;
                    }
                    __syncthreads();
                }
                for (int i = tid; i <= c; i += nth)
                    hc[i] = hc[i] + hc2[i];
                __syncthreads();
            }
            // h_{j+1,j} = ||w||
            T nsq = 0;
            for (int r = rb + tid; r < re; r += nth)
                nsq += S.w[r] * S.w[r];
            T hnext = wsqrt(team_sum1<T, CS>(nsq, red, slot, bc, &buft));
            // Givens step (thread 0 of every CTA, on identical data) and the
            // restart test
            if (tid == 0) {
                T *col = H + (size_t)c * ld;
                for (int i = 0; i <= c; ++i)
                    col[i] = hc[i];
                col[c + 1] = hnext;
                for (int i = 0; i < c; ++i) {
                    T hi = col[i], hi1 = col[i + 1];
                    col[i] = cs[i] * hi + sn[i] * hi1;
                    col[i + 1] = -sn[i] * hi + cs[i] * hi1;
                }
                T hjj = col[c], hj1 = col[c + 1];
                T rho = wsqrt(hjj * hjj + hj1 * hj1);
                T al, be;
                if (rho == T(0)) {
                    al = T(1);
                    be = T(0);
                } else {
                    al = hjj / rho;
                    be = hj1 / rho;
                }
                cs[c] = al;
                sn[c] = be;
                T sj = s[c];
                s[c] = al * sj;
                s[c + 1] = -be * sj;
                col[c] = al * hjj + be * hj1;
                col[c + 1] = -be * hjj + al * hj1;
                double arn = fabs((double)s[c + 1]);
                ahist[c + 1] = arn;
                int bd = hnext <= brk * wnorm0;
                int nf = !isfinite(arn);
                int stall = P.stall_factor > 0 && c + 1 >= P.stall_w &&
                            ahist[c + 1 - P.stall_w] < P.stall_factor * arn;
                int end = bd || nf || (tau > 0 && arn <= tau * (double)beta) || arn <= inner_abs ||
                          stall || (c + 1 >= kmax);
                s_flag = (end ? 1 : 0) | (bd ? 2 : 0) | (nf ? 4 : 0);
            }
            __syncthreads();
            const int flag = s_flag;
            j = c + 1;
            if (flag & 4) {
                cyc_bad = 1;
                break;
            }
            if (flag & 1)
                break;
            // v_{j+1} = w / h_{j+1,j}; every CTA's rows before the next SpMV
            VT *vn = S.V + (size_t)(c + 1) * S.ldv;
            for (int r = rb + tid; r < re; r += nth)
                Basis<VT>::st(vn + r, S.w[r] / hnext, S.vscale);
            Team<CS>::sync();
        }
        if (cyc_bad) {
            out.status = -3;
            break;
        }
        // y = H^{-1} s (back substitution), x += V_j y
        if (tid == 0) {
            for (int i = j - 1; i >= 0; --i) {
                T acc = s[i];
                for (int l = i + 1; l < j; ++l)
                    acc -= H[(size_t)l * ld + i] * y[l];
                T piv = H[(size_t)i * ld + i];
                y[i] = (piv == T(0)) ? T(0) : acc / piv;
            }
        }
        __syncthreads();
        for (int r = rb + tid; r < re; r += nth) {
            T u = 0;
            for (int i = 0; i < j; ++i)
                u += Basis<VT>::ld(S.V + (size_t)i * S.ldv + r, S.vinv) * y[i];
            S.x[r] = S.x[r] + (double)u;
        }
        __syncthreads();
        out.iters += j;
        out.restarts += 1;
        if (out.restarts == 1) {
            out.first_len = j;
            if (P.repeat_first)
                cycle_len = j;
        }
    }
    if (tid == 0 && Team<CS>::rank() == 0)
        *res = out;
    Team<CS>::sync();
}

template <class T, class VT, int L>
__device__ void block_solve_one(const BlockSys<T, VT> &S, const BlockParams &P, BlockResult *res,
                                unsigned char *smem_raw) {
    team_solve_one<T, VT, L, 1>(S, P, res, smem_raw);
}

// Launch bounds of the whole-solve kernels.  Launches of up to 1024 threads
// (single systems) use the plain bound; the batched solver's 256-thread
// launches ask for several resident blocks per SM, which caps the registers
// per thread: occupancy is what hides the latency of these block-wide
// reductions.  Measured on 2048 uneven 2-D systems, GMRES(30) MGS: binary32
// 2.25 s with 64 registers (4 blocks per SM), 1.98 s with 40 (6), 2.06 s with
// 51 (5), 2.01 s with 32 (8, spilling), 2.96 s with 80 (3) and 3.88 s
// unbounded (~125, 2); binary64 best with 5 blocks (3.12 s against 3.28 s).
template <class T, int MAXT>
struct SolveMinBlocks {
    static constexpr int value = MAXT > 256 ? 1 : (sizeof(T) == 4 ? 6 : 5);
};

// Persistent grid over a work queue of systems (largest first); one team
// (block or cluster) per system.
template <class T, class VT, int L, int CS, int MAXT = 1024>
__global__ void __launch_bounds__(MAXT, SolveMinBlocks<T, MAXT>::value)
    k_team_solve(const BlockSys<T, VT> *sys, BlockParams P, BlockResult *res) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0 && Team<CS>::rank() == 0) {
            unsigned k = atomicAdd(P.queue, 1u);
            s_idx = (k < (unsigned)P.nsys) ? (P.order ? P.order[k] : (int)k) : -1;
        }
        Team<CS>::sync();
        int idx;
        if (CS == 1) {
            idx = s_idx;
        } else {
            cg::cluster_group cl = cg::this_cluster();
            idx = *cl.map_shared_rank(&s_idx, 0);
        }
        Team<CS>::sync();
        if (idx < 0)
            return;
        BlockSys<T, VT> S = sys[idx];
        team_solve_one<T, VT, L, CS>(S, P, res + idx, smem_raw);
    }
}

template <class T, class VT, int L, int MAXT = 1024>
__global__ void __launch_bounds__(MAXT, SolveMinBlocks<T, MAXT>::value)
    k_block_solve(const BlockSys<T, VT> *sys, BlockParams P, BlockResult *res) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned k = atomicAdd(P.queue, 1u);
            s_idx = (k < (unsigned)P.nsys) ? (P.order ? P.order[k] : (int)k) : -1;
        }
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx < 0)
            return;
        BlockSys<T, VT> S = sys[idx];
        block_solve_one<T, VT, L>(S, P, res + idx, smem_raw);
        __syncthreads();
    }
}

// Shared-memory bytes of the block / team solver for restart length m.
template <class T>
inline size_t block_smem_bytes(int m) {
    size_t nt = (size_t)(m + 1) * m + (m + 1) + 3 * (size_t)m + 2 * (MMAX + 2) + 8 * 32 +
                3 * TEAM_KMAX;
    return nt * sizeof(T) + (32 + 3 * TEAM_KMAX + MMAX + 2) * sizeof(double) + 64;
}

}  // namespace gmres
