// ilu.cu -- ILU(0) left preconditioning, the preconditioner of the paper's
// experiments (arXiv 2011.01850, Sec. 4; Alg. 1 applies M^-1 on the left:
// r = M^-1 z at every restart and w = M^-1 A v_j in every inner step).
//
// Factorization.  ILU(0) keeps A's sparsity pattern; row i of the IKJ form
// eliminates with every earlier row k of its pattern in ascending order
// (l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for the j > k present in both
// rows).  Row i depends on the rows k < i of its pattern, so the rows are
// grouped into levels (host analysis of the pattern) and one launch per
// level factors every row of the level, one thread per row.  The products
// and differences are rounded separately (no fused multiply-add), as in a
// plain restatement of the elimination, so the factors are reproducible bit
// for bit.  A binary32 copy serves the binary32 restart cycle.
//
// Triangular solves.  L y = z (unit lower) and U x = y run as one persistent
// launch each, in one of three forms.  The barrier-free form polls the
// dependencies' solution entries themselves (k_trsv_wave); the level form
// walks the level schedule with a grid barrier between levels
// (k_trsv_levels).  The flag form: each warp claims the next row of the
// triangle's level schedule from a counter (every row a claimed row depends
// on sits in an earlier level, so a running warp claimed it earlier, and a
// whole level is in flight at once); its lanes wait on the dependencies'
// ready flags in parallel, lane 0 subtracts the terms in column order,
// stores the value and publishes its flag with a release store.
// Flags hold an epoch that changes every call (the host clears them before
// the 32-bit epoch wraps).  Every wait is bounded: after `spin` polls the
// warp reports a timeout in the control block and returns, and the other
// warps see the report and return too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gmres_gb300.h"
#include "common.cuh"
#include "handle.hpp"
#include "host_util.hpp"
#include "ilu.hpp"

using namespace gmres;
using namespace gmres_host;

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Factor the rows rows[0..count) (one level) in place; err[0] = 1 on a zero
// or non-finite pivot.
__global__ void __launch_bounds__(256) k_ilu0_level(const int *rowptr, const int *colind,
                                                    const int *dpos, double *lu, const int *rows,
                                                    int count, int *err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count)
        return;
    const int i = rows[t];
    const int end = rowptr[i + 1];
    for (int p = rowptr[i]; p < dpos[i]; ++p) {
        const int k = colind[p];
        const double piv = lu[dpos[k]];
        if (piv == 0.0 || !isfinite(piv)) {
            atomicExch(err, 1);
            return;
        }
        const double lik = __ddiv_rn(lu[p], piv);
        lu[p] = lik;
        // merge row i's entries after p with row k's entries after its diagonal
        int kp = dpos[k] + 1;
        const int kend = rowptr[k + 1];
        for (int q = p + 1; q < end; ++q) {
            const int j = colind[q];
            while (kp < kend && colind[kp] < j)
                ++kp;
            if (kp < kend && colind[kp] == j)
                lu[q] = __dsub_rn(lu[q], __dmul_rn(lik, lu[kp]));
        }
    }
    const double d = lu[dpos[i]];
    if (d == 0.0 || !isfinite(d))
        atomicExch(err, 1);
}

__global__ void k_ilu_cast(int64_t nnz, const double *a, float *b) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

// One triangle of (L U) x = z.  LOWER: y_i = z_i - sum_{k<i} l_ik y_k (unit
// diagonal), rows claimed in increasing order; upper: x_i = (y_i -
// sum_{j>i} u_ij x_j) / u_ii, rows claimed in decreasing order.  T is the
// arithmetic type, AT the stored factor type.
// Separately rounded multiply and subtract (no fused multiply-add), so the
// solves repeat the oracle's sums exactly.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// One triangle of (L U) x = z.  LOWER: y_i = z_i - sum_{k<i} l_ik y_k (unit
// diagonal); upper: x_i = (y_i - sum_{j>i} u_ij x_j) / u_ii.  A warp claims
// the next row of the schedule; its lanes wait on the ready flags of the
// row's dependencies (one dependency per lane, all at once) and form the
// products, and lane 0 subtracts them one by one in column order, as the
// oracle does.  T is the arithmetic type, AT the stored factor type.
template <class T, class AT, bool LOWER>
__global__ void __launch_bounds__(256) k_trsv(int n, const int *rowptr, const int *colind,
                                              const int *dpos, const int *order, const AT *lu,
                                              const T *in, T *out, unsigned *flags,
                                              unsigned epoch, unsigned *counter, long long spin,
                                              int *err) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int claim = 0;
        if (lane == 0)
            claim = (int)atomicAdd(counter, 1u);
        claim = __shfl_sync(0xffffffffu, claim, 0);
        if (claim >= n)
            return;
        const int i = order[claim];
        const int b = LOWER ? rowptr[i] : dpos[i] + 1;
        const int e = LOWER ? dpos[i] : rowptr[i + 1];
        T acc = lane == 0 ? in[i] : T(0);
        bool ok = true;
        for (int p0 = b; p0 < e; p0 += 32) {
            const int p = p0 + lane;
            T prod = 0;
            if (p < e) {
                const int j = colind[p];
                long long it = 0;
                while (ld_acquire_u32(flags + j) != epoch) {
                    if (*(volatile int *)err != 0 || ++it > spin) {
                        ok = false;
                        break;
                    }
                }
                if (ok)
                    prod = mul_rn((T)lu[p], __ldcg(out + j));
            }
            if (!__all_sync(0xffffffffu, ok))
                break;
            const int cnt = e - p0 < 32 ? e - p0 : 32;
            for (int q = 0; q < cnt; ++q) {
                const T v = __shfl_sync(0xffffffffu, prod, q);
                if (lane == 0)
                    acc = sub_rn(acc, v);
            }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0)
                atomicExch(err, 1);
            return;
        }
        if (lane == 0) {
            if (!LOWER)
                acc = acc / (T)lu[dpos[i]];
            out[i] = acc;
            st_release_u32(flags + i, epoch);
        }
    }
}

// The same triangle as one cooperative launch that walks the level schedule:
// every row of level l depends only on rows of earlier levels, so the
// threads solve the rows of a level independently and the grid passes a
// barrier between levels.  The barrier is split: a block arrives as soon as
// its rows of level l are stored, then loads the structure of its rows of
// level l + 1 (row index, entry range, right-hand side, the first TRSV_PF
// factor entries and their columns; none of it depends on the level being
// solved), and only then waits.  After the wait only the solution values of
// the dependencies remain to be read.  Warps take consecutive 32-row runs of
// a level, interleaved over the blocks so that every SM gets a share of a
// narrow level.  Each row subtracts its terms in column order with
// separately rounded products, as the oracle does.  The barrier counter
// grows by gridDim.x per level: a block arrives with one release reduction
// (its stores, ordered before it by the block barrier, are visible before
// the count), and thread 0 polls the count with acquire loads.  A wait that
// runs past `spin` polls (or sees another block's report) reports a timeout
// in *err and the block returns.
constexpr int TRSV_LV_THREADS = 1024;
constexpr int TRSV_PF = 4;

template <class T, class AT>
struct RowAhead {
    int i;  // row, -1 when the thread has none at this level
    int b, e;
    T rhs;
    AT diag;
    int col[TRSV_PF];
    AT val[TRSV_PF];
};

template <class T, class AT, bool LOWER>
__device__ __forceinline__ void trsv_load_row(RowAhead<T, AT> &r, int pos, int hi,
                                              const int *order, const int *rowptr,
                                              const int *colind, const int *dpos, const AT *lu,
                                              const T *in) {
    r.i = -1;
    if (pos >= hi)
        return;
    const int i = order[pos];
    r.i = i;
    const int d = dpos[i];
    r.b = LOWER ? rowptr[i] : d + 1;
    r.e = LOWER ? d : rowptr[i + 1];
    r.rhs = in[i];
    r.diag = LOWER ? AT(1) : lu[d];
#pragma unroll
    for (int k = 0; k < TRSV_PF; ++k) {
        if (r.b + k < r.e) {
            r.col[k] = colind[r.b + k];
            r.val[k] = lu[r.b + k];
        }
    }
}

template <class T, class AT, bool LOWER>
__device__ __forceinline__ void trsv_solve_row(const RowAhead<T, AT> &r, const int *colind,
                                               const AT *lu, T *out) {
    T acc = r.rhs;
#pragma unroll
    for (int k = 0; k < TRSV_PF; ++k)
        if (r.b + k < r.e)
            acc = sub_rn(acc, mul_rn((T)r.val[k], __ldcg(out + r.col[k])));
    for (int p = r.b + TRSV_PF; p < r.e; ++p)
        acc = sub_rn(acc, mul_rn((T)lu[p], __ldcg(out + colind[p])));
    if (!LOWER)
        acc = acc / (T)r.diag;
    out[r.i] = acc;
}

template <class T, class AT, bool LOWER>
__global__ void __launch_bounds__(TRSV_LV_THREADS, 1)
    k_trsv_levels(int nlev, const int *lptr, const int *order, const int *rowptr,
                  const int *colind, const int *dpos, const AT *lu, const T *in, T *out,
                  unsigned *bar, long long spin, int *err) {
    __shared__ int s_stop;
    const int first = (blockIdx.x + gridDim.x * (threadIdx.x >> 5)) * 32 + (threadIdx.x & 31);
    const int stride = gridDim.x * blockDim.x;
    if (threadIdx.x == 0)
        s_stop = 0;
    RowAhead<T, AT> r;
    trsv_load_row<T, AT, LOWER>(r, lptr[0] + first, lptr[1], order, rowptr, colind, dpos, lu,
                                in);
    for (int l = 0; l < nlev; ++l) {
        const int lo = lptr[l], hi = lptr[l + 1];
        if (r.i >= 0)
            trsv_solve_row<T, AT, LOWER>(r, colind, lu, out);
        for (int pos = lo + first + stride; pos < hi; pos += stride) {
            RowAhead<T, AT> q;
            trsv_load_row<T, AT, LOWER>(q, pos, hi, order, rowptr, colind, dpos, lu, in);
            trsv_solve_row<T, AT, LOWER>(q, colind, lu, out);
        }
        if (l + 1 == nlev)
            break;
        __syncthreads();
        if (threadIdx.x == 0)
            red_release_add_u32(bar, 1u);
        trsv_load_row<T, AT, LOWER>(r, hi + first, lptr[l + 2], order, rowptr, colind, dpos, lu,
                                    in);
        if (threadIdx.x == 0) {
            const unsigned target = (unsigned)(l + 1) * gridDim.x;
            long long it = 0;
            while (ld_acquire_u32(bar) < target) {
                if (*(volatile int *)err != 0 || ++it > spin) {
                    atomicExch(err, 1);
                    s_stop = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_stop)
            return;
    }
}

template <class T, class AT, bool LOWER>
cudaError_t launch_trsv_levels(gmres_handle *h, const AT *lu, const T *in, T *out,
                               unsigned *bar, long long spin, int *err) {
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_trsv_levels<T, AT, LOWER>, TRSV_LV_THREADS, 0);
        if (e != cudaSuccess)
            return e;
    }
    if (per_sm < 1)
        return cudaErrorCooperativeLaunchTooLarge;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), h->stream);
    if (e != cudaSuccess)
        return e;
    int nlev = LOWER ? h->ilu_levels : h->ilu_ulevels;
    const int *lptr = h->ilu_lptr.as<int>() + (LOWER ? 0 : h->ilu_levels + 1);
    const int *order = h->ilu_order.as<int>() + (LOWER ? 0 : h->n);
    const int *rowptr = h->rowptr.as<int>(), *colind = h->colind.as<int>(),
              *dpos = h->ilu_dpos.as<int>();
    void *args[] = {&nlev, &lptr, &order, &rowptr, &colind, &dpos, &lu, &in, &out,
                    &bar, &spin, &err};
    return cudaLaunchCooperativeKernel((const void *)k_trsv_levels<T, AT, LOWER>, dim3(h->nsm),
                                       dim3(TRSV_LV_THREADS), args, 0, h->stream);
}

// The same triangle without a barrier: the solution vector is its own
// ready flag.  Before the launch every entry of `out` is set to the all-ones
// bit pattern (a NaN that the solve never stores: a computed value with that
// pattern is stored as the canonical NaN instead); a row polls its
// dependencies' entries until none holds the pattern.  Values are single
// aligned words, stored and polled with relaxed gpu-scope accesses.  Every
// warp walks all levels in step: at each level it takes its 32-row runs
// (interleaved over the blocks, as in k_trsv_levels), and its lanes poll
// together until every lane's dependencies are in, so the warp never
// diverges across a wait.  Every dependency sits in an earlier level, which
// each warp finishes before it starts a later one, so with all blocks
// resident (cooperative launch) every wait ends; a wait that runs past `spin`
// polls, or sees another warp's report, reports a timeout in *err.
template <class T>
struct WordOf;
template <>
struct WordOf<float> {
    using U = unsigned;
    static constexpr U none = 0xffffffffu;
    static constexpr U qnan = 0x7fc00000u;
};
template <>
struct WordOf<double> {
    using U = unsigned long long;
    static constexpr U none = ~0ull;
    static constexpr U qnan = 0x7ff8000000000000ull;
};

__device__ __forceinline__ unsigned ld_relaxed_w(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_w(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_w(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_w(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ float word_value(unsigned u) { return __uint_as_float(u); }
__device__ __forceinline__ double word_value(unsigned long long u) {
    return __longlong_as_double((long long)u);
}
__device__ __forceinline__ unsigned value_word(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long value_word(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// The whole warp polls until every lane's first `cnt` (<= TRSV_PF)
// dependencies hold values (lanes without a row pass cnt = 0).  All lanes
// leave together; false (for every lane) on a timeout.
template <class T, class U>
__device__ __forceinline__ bool wave_wait_warp(const U *ob, const int *col, int cnt, T *x,
                                               long long spin, int *err) {
    unsigned pending = 0;
#pragma unroll
    for (int k = 0; k < TRSV_PF; ++k)
        if (k < cnt)
            pending |= 1u << k;
    long long it = 0;
    for (;;) {
        U w[TRSV_PF];
#pragma unroll
        for (int k = 0; k < TRSV_PF; ++k)
            if (pending & (1u << k))
                w[k] = ld_relaxed_w(ob + col[k]);
#pragma unroll
        for (int k = 0; k < TRSV_PF; ++k)
            if ((pending & (1u << k)) && w[k] != WordOf<T>::none) {
                x[k] = word_value(w[k]);
                pending &= ~(1u << k);
            }
        if (__all_sync(0xffffffffu, pending == 0))
            return true;
        const int bad = __shfl_sync(0xffffffffu, *(volatile int *)err, 0);
        if (bad != 0 || ++it > spin) {
            if ((threadIdx.x & 31) == 0)
                atomicExch(err, 1);
            return false;
        }
    }
}

// Solves the row of r (if any) with the whole warp taking part in the waits.
template <class T, class AT, bool LOWER>
__device__ __forceinline__ bool wave_solve_warp(const RowAhead<T, AT> &r, const int *colind,
                                                const AT *lu, T *out, long long spin, int *err) {
    using U = typename WordOf<T>::U;
    U *ob = reinterpret_cast<U *>(out);
    const int len = r.i >= 0 ? r.e - r.b : 0;
    const int cnt = len < TRSV_PF ? len : TRSV_PF;
    T x[TRSV_PF];
    if (!wave_wait_warp<T, U>(ob, r.col, cnt, x, spin, err))
        return false;
    T acc = r.rhs;
#pragma unroll
    for (int k = 0; k < TRSV_PF; ++k)
        if (k < cnt)
            acc = sub_rn(acc, mul_rn((T)r.val[k], x[k]));
    // entries past the first TRSV_PF: one at a time, the warp in step
    const int more = __reduce_max_sync(0xffffffffu, len > TRSV_PF ? len - TRSV_PF : 0);
    for (int q = 0; q < more; ++q) {
        const bool mine = TRSV_PF + q < len;
        const int j = mine ? colind[r.b + TRSV_PF + q] : 0;
        T xj = 0;
        if (!wave_wait_warp<T, U>(ob, &j, mine ? 1 : 0, &xj, spin, err))
            return false;
        if (mine)
            acc = sub_rn(acc, mul_rn((T)lu[r.b + TRSV_PF + q], xj));
    }
    if (r.i >= 0) {
        if (!LOWER)
            acc = acc / (T)r.diag;
        U word = value_word(acc);
        if (word == WordOf<T>::none)
            word = WordOf<T>::qnan;
        st_relaxed_w(ob + r.i, word);
    }
    return true;
}

constexpr int TRSV_WAVE_THREADS = 512;

template <class T, class AT, bool LOWER>
__global__ void __launch_bounds__(TRSV_WAVE_THREADS, 1)
    k_trsv_wave(int nlev, const int *lptr, const int *order, const int *rowptr,
                const int *colind, const int *dpos, const AT *lu, const T *in, T *out,
                long long spin, int *err) {
    const int lane = threadIdx.x & 31;
    const int wbase = (blockIdx.x + gridDim.x * (threadIdx.x >> 5)) * 32;  // warp-uniform
    const int stride = gridDim.x * blockDim.x;
    RowAhead<T, AT> r;
    int lo = __ldg(lptr), hi = __ldg(lptr + 1);
    trsv_load_row<T, AT, LOWER>(r, lo + wbase + lane, hi, order, rowptr, colind, dpos, lu, in);
    for (int l = 0; l < nlev; ++l) {
        const int hi2 = l + 1 < nlev ? __ldg(lptr + l + 2) : hi;
        RowAhead<T, AT> nx;
        trsv_load_row<T, AT, LOWER>(nx, hi + wbase + lane, hi2, order, rowptr, colind, dpos, lu,
                                    in);
        if (lo + wbase < hi && !wave_solve_warp<T, AT, LOWER>(r, colind, lu, out, spin, err))
            return;
        for (int base = lo + wbase + stride; base < hi; base += stride) {
            RowAhead<T, AT> q;
            trsv_load_row<T, AT, LOWER>(q, base + lane, hi, order, rowptr, colind, dpos, lu, in);
            if (!wave_solve_warp<T, AT, LOWER>(q, colind, lu, out, spin, err))
                return;
        }
        r = nx;
        lo = hi;
        hi = hi2;
    }
}

template <class T, class AT, bool LOWER>
cudaError_t launch_trsv_wave(gmres_handle *h, const AT *lu, const T *in, T *out, long long spin,
                             int *err) {
    static int per_sm = -1;
    if (per_sm < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_trsv_wave<T, AT, LOWER>, TRSV_WAVE_THREADS, 0);
        if (e != cudaSuccess)
            return e;
    }
    if (per_sm < 1)
        return cudaErrorCooperativeLaunchTooLarge;
    // every entry starts as the all-ones pattern (not yet solved)
    cudaError_t e = cudaMemsetAsync(out, 0xff, sizeof(T) * (size_t)h->n, h->stream);
    if (e != cudaSuccess)
        return e;
    int nlev = LOWER ? h->ilu_levels : h->ilu_ulevels;
    const int *lptr = h->ilu_lptr.as<int>() + (LOWER ? 0 : h->ilu_levels + 1);
    const int *order = h->ilu_order.as<int>() + (LOWER ? 0 : h->n);
    const int *rowptr = h->rowptr.as<int>(), *colind = h->colind.as<int>(),
              *dpos = h->ilu_dpos.as<int>();
    void *args[] = {&nlev, &lptr, &order, &rowptr, &colind, &dpos, &lu, &in, &out, &spin, &err};
    return cudaLaunchCooperativeKernel((const void *)k_trsv_wave<T, AT, LOWER>, dim3(h->nsm),
                                       dim3(TRSV_WAVE_THREADS), args, 0, h->stream);
}

template <class T, class AT, bool LOWER>
cudaError_t launch_trsv(gmres_handle *h, const AT *lu, const T *in, T *out, unsigned *flags,
                        unsigned epoch, unsigned *counter, long long spin, int *err) {
    static int grid = 0;
    if (grid == 0) {
        int per_sm = 0;
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsv<T, AT, LOWER>, 256, 0);
        if (e != cudaSuccess)
            return e;
        grid = std::max(1, per_sm) * h->nsm;
    }
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), h->stream);
    if (e != cudaSuccess)
        return e;
    const int *order = h->ilu_order.as<int>() + (LOWER ? 0 : h->n);
    k_trsv<T, AT, LOWER><<<grid, 256, 0, h->stream>>>(h->n, h->rowptr.as<int>(),
                                                       h->colind.as<int>(), h->ilu_dpos.as<int>(),
                                                       order, lu, in, out, flags, epoch, counter,
                                                       spin, err);
    return cudaGetLastError();
}

template <class T, class AT, bool LOWER>
cudaError_t launch_triangle(gmres_handle *h, const AT *lu, const T *in, T *out, unsigned *flags,
                            unsigned epoch, unsigned *ctr, long long spin, int *err) {
    switch (gmres::trsv_kind(h, LOWER)) {
    case 3: return launch_trsv_wave<T, AT, LOWER>(h, lu, in, out, spin, err);
    case 2: return launch_trsv_levels<T, AT, LOWER>(h, lu, in, out, ctr, spin, err);
    default: return launch_trsv<T, AT, LOWER>(h, lu, in, out, flags, epoch, ctr, spin, err);
    }
}

}  // namespace

namespace gmres {

gmres_status ilu_factor(gmres_handle *h) {
    const int n = h->n;
    const int64_t nnz = h->nnz;
    std::vector<int32_t> rp(n + 1), ci(std::max<int64_t>(nnz, 1));
    CK(cudaMemcpyAsync(rp.data(), h->rowptr.p, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost,
                       h->stream));
    if (nnz > 0)
        CK(cudaMemcpyAsync(ci.data(), h->colind.p, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // diagonal positions (rows sorted, diagonal present) and the levels of
    // the lower-triangular dependency graph
    std::vector<int32_t> dpos(n), level(n, 0);
    int nlev = 0;
    for (int i = 0; i < n; ++i) {
        int d = -1, lv = 0;
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (p > rp[i] && ci[p] <= ci[p - 1])
                return GMRES_ERR_ARG;  // ILU(0) needs sorted rows
            if (ci[p] == i)
                d = p;
            else if (ci[p] < i)
                lv = std::max(lv, level[ci[p]] + 1);
        }
        if (d < 0)
            return GMRES_ERR_ARG;  // and a diagonal entry in every row
        dpos[i] = d;
        level[i] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    std::vector<int32_t> lptr(nlev + 1, 0), order(n);
    for (int i = 0; i < n; ++i)
        lptr[level[i] + 1]++;
    for (int l = 0; l < nlev; ++l)
        lptr[l + 1] += lptr[l];
    {
        std::vector<int32_t> pos(lptr.begin(), lptr.end() - 1);
        for (int i = 0; i < n; ++i)
            order[pos[level[i]]++] = i;
    }
    // levels of the upper-triangular graph (row i waits for the j > i of its
    // pattern), counted from the last row
    std::vector<int32_t> ulevel(n, 0), uorder(n);
    int nulev = 0;
    for (int i = n - 1; i >= 0; --i) {
        int lv = 0;
        for (int32_t p = dpos[i] + 1; p < rp[i + 1]; ++p)
            lv = std::max(lv, ulevel[ci[p]] + 1);
        ulevel[i] = lv;
        nulev = std::max(nulev, lv + 1);
    }
    std::vector<int32_t> uptr(nulev + 1, 0);
    for (int i = 0; i < n; ++i)
        uptr[ulevel[i] + 1]++;
    for (int l = 0; l < nulev; ++l)
        uptr[l + 1] += uptr[l];
    {
        std::vector<int32_t> pos(uptr.begin(), uptr.end() - 1);
        for (int i = 0; i < n; ++i)
            uorder[pos[ulevel[i]]++] = i;
    }
    CK(h->ilu_lptr.ensure(sizeof(int32_t) * (size_t)(nlev + nulev + 2)));
    CK(cudaMemcpyAsync(h->ilu_lptr.p, lptr.data(), sizeof(int32_t) * (nlev + 1),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->ilu_lptr.as<int32_t>() + nlev + 1, uptr.data(),
                       sizeof(int32_t) * (nulev + 1), cudaMemcpyHostToDevice, h->stream));
    CK(h->ilu_order.ensure(sizeof(int32_t) * 2 * (size_t)n));
    CK(cudaMemcpyAsync(h->ilu_order.p, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(h->ilu_order.as<int32_t>() + n, uorder.data(), sizeof(int32_t) * n,
                       cudaMemcpyHostToDevice, h->stream));
    CK(h->ilu64.ensure(sizeof(double) * std::max<int64_t>(nnz, 1)));
    CK(h->ilu32.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h->ilu_dpos.ensure(sizeof(int32_t) * n));
    CK(h->ilu_flags.ensure(sizeof(unsigned) * 2 * (size_t)n + 64));
    ScopedBuf dorder, derr;
    CK(dorder.ensure(sizeof(int32_t) * n));
    CK(derr.ensure(sizeof(int)));
    CK(cudaMemcpyAsync(h->ilu_dpos.p, dpos.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(dorder.p, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemsetAsync(derr.p, 0, sizeof(int), h->stream));
    CK(cudaMemcpyAsync(h->ilu64.p, h->vals64.p, sizeof(double) * nnz, cudaMemcpyDeviceToDevice,
                       h->stream));
    for (int l = 0; l < nlev; ++l) {
        const int cnt = lptr[l + 1] - lptr[l];
        k_ilu0_level<<<(cnt + 255) / 256, 256, 0, h->stream>>>(
            h->rowptr.as<int>(), h->colind.as<int>(), h->ilu_dpos.as<int>(), h->ilu64.as<double>(),
            dorder.as<int>() + lptr[l], cnt, derr.as<int>());
    }
    CKL();
    if (nnz > 0)
        k_ilu_cast<<<h->nsm * 4, 256, 0, h->stream>>>(nnz, h->ilu64.as<double>(),
                                                       h->ilu32.as<float>());
    CKL();
    CK(cudaMemsetAsync(h->ilu_flags.p, 0, h->ilu_flags.bytes, h->stream));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, derr.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->ilu_epoch = 1;
    h->ilu_levels = nlev;
    h->ilu_ulevels = nulev;
    // the barrier-free solve suits triangles whose rows all fit the entries
    // loaded ahead (longer rows wait on one entry at a time) and whose
    // levels fit the grid in one pass
    {
        int lmax = 0, umax = 0, lwidth = 0, uwidth = 0;
        for (int i = 0; i < n; ++i) {
            lmax = std::max(lmax, dpos[i] - rp[i]);
            umax = std::max(umax, rp[i + 1] - dpos[i] - 1);
        }
        for (int l = 0; l < nlev; ++l)
            lwidth = std::max(lwidth, lptr[l + 1] - lptr[l]);
        for (int l = 0; l < nulev; ++l)
            uwidth = std::max(uwidth, uptr[l + 1] - uptr[l]);
        const int slots = h->nsm * TRSV_WAVE_THREADS;
        h->ilu_wave_ok[0] = lmax <= TRSV_PF && lwidth <= slots;
        h->ilu_wave_ok[1] = umax <= TRSV_PF && uwidth <= slots;
    }
    h->ilu_ok = bad ? 0 : 1;
    return bad ? GMRES_ERR_BREAKDOWN : GMRES_OK;
}

int trsv_kind(const gmres_handle *h, bool lower) {
    if (h->opts.trsv_kernel != 0)
        return h->opts.trsv_kernel;
    return (lower ? h->ilu_wave_ok[0] : h->ilu_wave_ok[1]) ? 3 : 2;
}

template <class T, class AT>
cudaError_t ilu_apply(gmres_handle *h, const AT *lu, const T *z, T *tmp, T *out, int *err) {
    // one epoch per call (each triangle has its own flags); clear the flags
    // before the epoch wraps
    if (h->ilu_epoch > 0x7ffffff0u) {
        cudaError_t e = cudaMemsetAsync(h->ilu_flags.p, 0, h->ilu_flags.bytes, h->stream);
        if (e != cudaSuccess)
            return e;
        h->ilu_epoch = 1;
    }
    const unsigned e0 = h->ilu_epoch;
    h->ilu_epoch += 1;
    unsigned *lflags = h->ilu_flags.as<unsigned>();
    unsigned *uflags = lflags + h->n;
    unsigned *ctr = uflags + h->n;  // two counters after the flags
    // a legitimate wait lasts at most the dependency chain (a few hundred
    // rows of latency); 2^22 polls is seconds, far beyond it
    const long long spin = h->opts.spin_limit > 0 ? h->opts.spin_limit : (1LL << 22);
    // the lower solve has read z before the upper solve starts writing out
    // (they may be the same vector)
    cudaError_t e = launch_triangle<T, AT, true>(h, lu, z, tmp, lflags, e0, ctr, spin, err);
    if (e != cudaSuccess)
        return e;
    return launch_triangle<T, AT, false>(h, lu, tmp, out, uflags, e0, ctr + 1, spin, err);
}

template cudaError_t ilu_apply<double, double>(gmres_handle *, const double *, const double *,
                                               double *, double *, int *);
template cudaError_t ilu_apply<float, float>(gmres_handle *, const float *, const float *,
                                             float *, float *, int *);
template cudaError_t ilu_apply<double, float>(gmres_handle *, const float *, const double *,
                                              double *, double *, int *);

}  // namespace gmres
