// grid_kernels.cuh -- whole-GPU kernels for one inner step of restarted
// GMRES(m) on a large system (Algorithm 1 of arXiv 2011.01850).
//
// Each kernel spreads the n rows over the grid; cross-block sums go through
// per-block partials that the last block to finish reduces in a fixed order
// (deterministic).  Every kernel of an inner step first reads ctl->active and
// returns at once when the restart cycle has ended, so the host can enqueue a
// whole cycle without waiting.
//
// Vectors (w, r, basis columns) are padded to ldv rows (a multiple of 256)
// with zero tails, so the streaming kernels always move 4 rows per thread.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "sell.cuh"

namespace gmres {

constexpr int PSTRIDE = MMAX + 8;  // partial-sum slots per block

// Leading dimension of the basis and the work vectors: n rounded up to this,
// a multiple of every row slice the streaming kernels take (512 or 1024 rows
// in the CGSR passes, 128 in pass B), so none of them needs a tail check.
constexpr int LDV_ALIGN = 2048;

// Per-variable precision study (Sec. 4.1): a set bit stores that variable in
// binary32 -- every value written to it is rounded -- while the binary64
// solver's arithmetic is unchanged (GridCtx::pv, binary64 solves only).
enum : unsigned {
    PV_A_KRYLOV = 1u, PV_M = 2u, PV_V = 4u, PV_W = 8u, PV_H = 16u, PV_GIVENS = 32u,
    PV_Z = 64u, PV_A_RESID = 128u, PV_B = 256u, PV_X = 512u, PV_AX = 1024u, PV_ALL = 2047u,
    // the switches the orthogonalisation kernels and the Givens step apply
    PV_ORTHO = PV_W | PV_H | PV_GIVENS
};

// A value written to a variable of the study: rounded to binary32 when its
// bit is set (a no-op for binary32 working values).
template <class T>
__device__ __forceinline__ T pv_round(T v, unsigned mask, unsigned bit) {
    return (mask & bit) ? (T)(float)v : v;
}

template <class T, class VT>
struct GridCtx {
    int n, m, ld;        // rows, restart length, Hessenberg leading dim (m+1)
    int64_t ldv;         // basis / vector leading dimension (padded rows)
    int64_t chunk;       // rows per block in the streaming kernels (mult. of 4)
    const int *rowptr;
    const int *colind;
    const T *a;          // matrix values in the working precision
    const double *a64;   // binary64 values (residual)
    VT *V;               // basis, column-major, ldv x (m+1)
    float vscale, vinv;  // binary16 basis scale and its reciprocal
    T *w;                // work vector (A v_j, then orthogonalised)
    T *r;                // residual in the working precision
    T *t;                // scratch vector (preconditioner)
    T *H, *Hb;           // rotated / unrotated Hessenberg, ld x m
    T *s, *cs, *sn, *y;  // rotated rhs (m+1), rotations (m), LS solution (m)
    T *h1, *h2;          // Hessenberg column: first / second projection
    T *part;             // per-block partials, gridDim x PSTRIDE
    double *part64;      // per-block binary64 partials, gridDim x 4
    Ctl *ctl;
    double tau, inner_abs, tol_abs;
    T brk;               // relative breakdown threshold for h_{j+1,j}
    int kmax;            // inner iterations allowed in this cycle
    // right preconditioner M (learned SpAI) on its own CSR, or null
    const int *prowptr;
    const int *pcolind;
    const T *pvals;
    // limited mixed precision: binary32 copies of A and M read in binary64
    // arithmetic (null otherwise; then a and pvals are used)
    const float *a_lim;
    const float *pvals_lim;
    // A stored split (Sec. 4 outlook): high- and low-order 32 bits of each
    // binary64 value; null when A is stored as binary64 + binary32 copies
    const unsigned *ahi, *alo;
    // how the Krylov step reads A: 0 the working-precision copy a, 1 the
    // binary32 copy a_lim, 2 the high part of split storage, 3 both parts
    int aform;
    // ILU(0) left preconditioning (Alg. 1: r = M^-1 z, w = M^-1 A v_j)
    int left;
    // third restart strategy (Sec. 3): |s_{j+1}| of the cycle (entry 0 =
    // beta) and the stall test's factor (0 = off) and window
    double *ahist;
    double stall_factor;
    int stall_w;
    // per-variable precision switches (PV_* bits) and A's binary32 copy for
    // the residual under PV_A_RESID
    unsigned pv;
    const float *a_res32;
    // A in sliced storage (sell.cuh) for the Krylov step, read when sfmt is
    // 1 (16-bit column offsets) or 2 (32-bit columns); 0 = the CSR arrays
    int sfmt;
    const int *sptr;
    const unsigned short *slen;
    const void *scol;
    const T *sval;
};

// 4 consecutive basis entries starting at p (16-byte aligned for fp32 /
// 32-byte for fp64 / 8-byte for 16-bit types: row index a multiple of 4).
template <class T, class VT>
__device__ __forceinline__ void ld4(const VT *p, float vinv, T (&o)[4]);

template <>
__device__ __forceinline__ void ld4<double, double>(const double *p, float, double (&o)[4]) {
    double2 a = *reinterpret_cast<const double2 *>(p);
    double2 b = *reinterpret_cast<const double2 *>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <>
__device__ __forceinline__ void ld4<float, float>(const float *p, float, float (&o)[4]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<double, float>(const float *p, float, double (&o)[4]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<float, __nv_bfloat16>(const __nv_bfloat16 *p, float,
                                                          float (&o)[4]) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
}
template <>
__device__ __forceinline__ void ld4<float, __half>(const __half *p, float vinv, float (&o)[4]) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    __half2 a = *reinterpret_cast<__half2 *>(&u.x);
    __half2 b = *reinterpret_cast<__half2 *>(&u.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    o[0] = fa.x * vinv; o[1] = fa.y * vinv; o[2] = fb.x * vinv; o[3] = fb.y * vinv;
}

template <class T>
__device__ __forceinline__ void ldv4(const T *p, T (&o)[4]) { ld4<T, T>(p, 1.f, o); }

template <class T>
__device__ __forceinline__ void st4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st4<double>(double *p, const double (&v)[4]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<float>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Store 4 working values into the basis (rounding to its storage type).
template <class T, class VT>
__device__ __forceinline__ void stb4(VT *p, const T (&v)[4], float scale) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        Basis<VT>::st(p + k, v[k], scale);
}

// Row range of block b in the streaming kernels.
template <class C>
__device__ __forceinline__ void block_rows(const C &c, int64_t &rb, int64_t &re) {
    rb = (int64_t)blockIdx.x * c.chunk;
    re = rb + c.chunk;
    if (re > c.ldv) re = c.ldv;
}

// Sum the partials of columns [0, ncols) over the grid's blocks, in the last
// block: warp w owns columns w, w+nwarps, ...; lane l sums blocks l, l+32, ...
// sequentially, then the xor-butterfly combines the lanes.
template <class T>
__device__ __forceinline__ void reduce_columns(const T *part, int nblocks, int ncols, T *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int col = wid; col < ncols; col += nw) {
        T acc = 0;
        for (int b = lane; b < nblocks; b += 32)
            acc += ldcg(part + (size_t)b * PSTRIDE + col);
        acc = warp_sum(acc);
        if (lane == 0)
            out[col] = acc;
    }
}

// ---------------------------------------------------------------------------
// SpMV: y = A x with L lanes per CSR row (L in {1,2,4,8,16,32}).  Lane l of a
// group sums the row entries k = beg + l, beg + l + L, ... in order; the
// group then combines its lanes with the xor-butterfly.
// ---------------------------------------------------------------------------
// Matrix values as a kernel reads them: a plain array, the high-order part
// of split storage (the binary64 value with its low 32 bits cleared), or the
// exact binary64 value from both parts.
template <class AT>
struct ValPlain {
    const AT *a;
    __device__ __forceinline__ AT operator()(int k) const { return __ldg(a + k); }
};
struct ValHi {
    const unsigned *hi;
    __device__ __forceinline__ double operator()(int k) const {
        return __hiloint2double((int)__ldg(hi + k), 0);
    }
};
struct ValHiLo {
    const unsigned *hi, *lo;
    __device__ __forceinline__ double operator()(int k) const {
        return __hiloint2double((int)__ldg(hi + k), (int)__ldg(lo + k));
    }
};

// The vector a row gathers from: a stored vector of type XT (scaled for
// binary16).
template <class T, class XT>
struct XPlain {
    const XT *x;
    float xinv;
    __device__ __forceinline__ T operator()(int col) const {
        return (T)Basis<XT>::ld(x + col, xinv);
    }
};

template <class T, class AV, class XV, int L>
__device__ __forceinline__ T csr_row_g(const int *__restrict__ rowptr,
                                       const int *__restrict__ colind, AV a, XV xv, int row,
                                       int n, int gl) {
    T acc = 0;
    if (row < n) {
        int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
        int k = beg + gl;
        // four independent gathers in flight per lane, also on the last,
        // partial group of a row (its missing entries are predicated off, so
        // a short row's entries are all requested at once); the sum keeps the
        // sequential order of k
        for (; k < end; k += 4 * L) {
            const bool p1 = k + L < end, p2 = k + 2 * L < end, p3 = k + 3 * L < end;
            const int c0 = chk_col(__ldg(colind + k), n);
            const int c1 = p1 ? chk_col(__ldg(colind + k + L), n) : c0;
            const int c2 = p2 ? chk_col(__ldg(colind + k + 2 * L), n) : c0;
            const int c3 = p3 ? chk_col(__ldg(colind + k + 3 * L), n) : c0;
            const T a0 = (T)a(k);
            const T a1 = p1 ? (T)a(k + L) : T(0);
            const T a2 = p2 ? (T)a(k + 2 * L) : T(0);
            const T a3 = p3 ? (T)a(k + 3 * L) : T(0);
            const T x0 = xv(c0);
            const T x1 = p1 ? xv(c1) : T(0);
            const T x2 = p2 ? xv(c2) : T(0);
            const T x3 = p3 ? xv(c3) : T(0);
            acc += a0 * x0;
            if (p1)
                acc += a1 * x1;
            if (p2)
                acc += a2 * x2;
            if (p3)
                acc += a3 * x3;
        }
    }
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
    return acc;
}

template <class T, class AV, class XT, int L>
__device__ __forceinline__ T csr_row_v(const int *__restrict__ rowptr,
                                       const int *__restrict__ colind, AV a, const XT *x,
                                       float xinv, int row, int n, int gl) {
    return csr_row_g<T, AV, XPlain<T, XT>, L>(rowptr, colind, a, XPlain<T, XT>{x, xinv}, row, n,
                                              gl);
}

template <class T, class AT, class XT, int L>
__device__ __forceinline__ T csr_row(const int *__restrict__ rowptr, const int *__restrict__ colind,
                                     const AT *__restrict__ a, const XT *x, float xinv, int row,
                                     int n, int gl) {
    return csr_row_v<T, ValPlain<AT>, XT, L>(rowptr, colind, ValPlain<AT>{a}, x, xinv, row, n,
                                             gl);
}

// A row of the Krylov step's matrix in the form the context holds: the
// binary32 copy (limited mixed), split storage (high part for the binary32
// and limited steps, both parts for binary64), or the working-precision
// copy.
template <class T, class VT, class XV, int L>
__device__ __forceinline__ T step_row_g(const GridCtx<T, VT> &c, XV xv, int row, int gl) {
    switch (c.aform) {
    case 3:
        return csr_row_g<T, ValHiLo, XV, L>(c.rowptr, c.colind, ValHiLo{c.ahi, c.alo}, xv, row,
                                            c.n, gl);
    case 2:
        return csr_row_g<T, ValHi, XV, L>(c.rowptr, c.colind, ValHi{c.ahi}, xv, row, c.n, gl);
    case 1:
        return csr_row_g<T, ValPlain<float>, XV, L>(c.rowptr, c.colind, ValPlain<float>{c.a_lim},
                                                    xv, row, c.n, gl);
    default:
        return csr_row_g<T, ValPlain<T>, XV, L>(c.rowptr, c.colind, ValPlain<T>{c.a}, xv, row,
                                                c.n, gl);
    }
}

template <class T, class VT, class XT, int L>
__device__ __forceinline__ T step_row(const GridCtx<T, VT> &c, const XT *x, int row, int gl) {
    return step_row_g<T, VT, XPlain<T, XT>, L>(c, XPlain<T, XT>{x, c.vinv}, row, gl);
}

// w = A v_col (inner step, Alg. 1 "w <- A v_j"); with a right preconditioner
// the caller first forms t = M v_col and passes x = t.
template <class T, class VT, class XT, int L>
__global__ void __launch_bounds__(256) k_spmv_step(GridCtx<T, VT> c, const XT *x, T *y) {
    if (!c.ctl->active)
        return;
    const int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int gl = lane % L, gi = lane / L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * G; base < c.n; base += nwarps * G) {
        int row = (int)(base + gi);
        T v = step_row<T, VT, XT, L>(c, x, row, gl);
        if (row < c.n && gl == 0)
            y[row] = v;
    }
}

// The same product with A in sliced storage: one warp per slice of 32 rows,
// the rows' sums bit for bit those of k_spmv_step at one lane per row.
template <class T, class VT, class XT, class CV>
__global__ void __launch_bounds__(256) k_spmv_step_sell(GridCtx<T, VT> c, const XT *x, T *y) {
    if (!c.ctl->active)
        return;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nsl = (c.n + SELL_C - 1) / SELL_C;
    const CV col = sell_cols<CV>(c.scol);
    for (int s = warp; s < nsl; s += nwarps) {
        const int row = s * SELL_C + lane;
        const T v = sell_row<T>(c.sptr, c.slen, col, ValPlain<T>{c.sval}, XPlain<T, XT>{x, c.vinv},
                                s, lane, row, c.n);
        if (row < c.n)
            y[row] = v;
    }
}

// Plain SpMV for the C-ABI entry point gmres_spmv (no control block).
template <class T, class AV, int L>
__global__ void __launch_bounds__(256) k_spmv_plain_v(int n, const int *rowptr, const int *colind,
                                                      AV a, const T *x, T *y) {
    const int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int gl = lane % L, gi = lane / L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * G; base < n; base += nwarps * G) {
        int row = (int)(base + gi);
        T v = csr_row_v<T, AV, T, L>(rowptr, colind, a, x, 1.f, row, n, gl);
        if (row < n && gl == 0)
            y[row] = v;
    }
}

template <class T, class AT, int L>
__global__ void __launch_bounds__(256) k_spmv_plain(int n, const int *rowptr, const int *colind,
                                                    const AT *a, const T *x, T *y) {
    const int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int gl = lane % L, gi = lane / L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * G; base < n; base += nwarps * G) {
        int row = (int)(base + gi);
        T v = csr_row<T, AT, T, L>(rowptr, colind, a, x, 1.f, row, n, gl);
        if (row < n && gl == 0)
            y[row] = v;
    }
}

// ---------------------------------------------------------------------------
// Residual: z = b - A x in binary64 (Alg. 1 first step; Sec. 2), its norm,
// the working-precision copy r = fl(z) and ||r|| in the working precision.
// The last block sets up the cycle: beta, s = beta e_1, active flag.
// ---------------------------------------------------------------------------
// PVR: the per-variable study's residual (A, b, A x or the cycle's copy of z
// stored in binary32 as GridCtx::pv says); a separate instantiation, so the
// default residual carries none of it.
template <class T, class VT, int L, bool PVR = false>
__global__ void __launch_bounds__(256) k_residual(GridCtx<T, VT> c, const double *b,
                                                  const double *x, double *z, int setup) {
    __shared__ double sd[32];
    __shared__ T st[32];
    const int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int gl = lane % L, gi = lane / L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double ss = 0;
    T sst = 0;
    int bad = 0;
    for (int64_t base = warp * G; base < c.n; base += nwarps * G) {
        int row = (int)(base + gi);
        double ax;
        if (c.ahi)
            ax = csr_row_v<double, ValHiLo, double, L>(c.rowptr, c.colind, ValHiLo{c.ahi, c.alo},
                                                       x, 1.f, row, c.n, gl);
        else if (PVR && (c.pv & PV_A_RESID))
            ax = csr_row<double, float, double, L>(c.rowptr, c.colind, c.a_res32, x, 1.f, row,
                                                   c.n, gl);
        else
            ax = csr_row<double, double, double, L>(c.rowptr, c.colind, c.a64, x, 1.f, row, c.n,
                                                    gl);
        if (row < c.n && gl == 0) {
            const double zi = PVR ? pv_round(b[row], c.pv, PV_B) - pv_round(ax, c.pv, PV_AX)
                                  : b[row] - ax;
            if (z)
                z[row] = zi;
            T ri = PVR ? pv_round((T)zi, c.pv, PV_Z) : (T)zi;
            c.r[row] = ri;
            ss += zi * zi;
            sst += ri * ri;
            bad |= !isfinite(zi);
        }
    }
    ss = block_sum1(ss, sd);
    sst = block_sum1(sst, st);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        c.part64[(size_t)blockIdx.x * 4 + 0] = ss;
        c.part[(size_t)blockIdx.x * PSTRIDE + 0] = sst;
        c.part64[(size_t)blockIdx.x * 4 + 1] = bad ? 1.0 : 0.0;
    }
    if (!arrive_last(&c.ctl->counter[0]))
        return;
    double a = 0, f = 0;
    T at = 0;
    for (int bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) {
        a += ldcg(c.part64 + (size_t)bb * 4 + 0);
        f += ldcg(c.part64 + (size_t)bb * 4 + 1);
        at += ldcg(c.part + (size_t)bb * PSTRIDE + 0);
    }
    a = block_sum1(a, sd);
    f = block_sum1(f, sd);
    at = block_sum1(at, st);
    if (threadIdx.x == 0) {
        Ctl *k = c.ctl;
        double rn = sqrt(a);
        T beta = wsqrt(at);
        k->rnorm = rn;
        int nf = (f != 0.0) || !isfinite(rn);
        if (nf)
            k->nonfinite = 1;
        k->converged = (!nf && rn <= c.tol_abs);
        if (setup) {
            k->beta = (double)beta;
            k->j = 0;
            k->breakdown = 0;
            k->arn = (double)beta;
            k->active = (!nf && !k->converged && beta > T(0) && isfinite((double)beta));
            c.s[0] = beta;
        }
    }
    if (setup) {
        for (int i = 1 + threadIdx.x; i <= c.m; i += blockDim.x)
            c.s[i] = T(0);
    }
}

// v_1 = r / beta (Alg. 1 "v_1 <- r_k / beta"), rounded to the basis type.
template <class T, class VT>
__global__ void __launch_bounds__(256) k_init(GridCtx<T, VT> c) {
    if (!c.ctl->active)
        return;
    const T beta = (T)c.ctl->beta;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        c.ahist[0] = c.ctl->beta;
    int64_t rb, re;
    block_rows(c, rb, re);
    for (int64_t r = rb + 4 * threadIdx.x; r < re; r += 4 * blockDim.x) {
        T v[4];
        ldv4(c.r + r, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            v[k] = v[k] / beta;
        stb4<T, VT>(c.V + r, v, c.vscale);
    }
}

// ---------------------------------------------------------------------------
// Left preconditioning, cycle start: r holds M^-1 fl(z); beta = ||r|| in the
// working precision replaces the residual kernel's set-up (Alg. 1: beta is
// the norm of the preconditioned residual; the binary64 convergence test on
// ||z|| has already been made).
// ---------------------------------------------------------------------------
template <class T, class VT>
__global__ void __launch_bounds__(256) k_pnorm(GridCtx<T, VT> c) {
    if (!c.ctl->active)
        return;
    __shared__ T st[32];
    int64_t rb, re;
    block_rows(c, rb, re);
    T ss = 0;
    for (int64_t r = rb + 4 * threadIdx.x; r < re; r += 4 * blockDim.x) {
        T v[4];
        ldv4(c.r + r, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            ss += v[k] * v[k];
    }
    ss = block_sum1(ss, st);
    if (threadIdx.x == 0)
        c.part[(size_t)blockIdx.x * PSTRIDE] = ss;
    if (!arrive_last(&c.ctl->counter[6]))
        return;
    T a = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        a += ldcg(c.part + (size_t)b * PSTRIDE);
    a = block_sum1(a, st);
    if (threadIdx.x == 0) {
        Ctl *k = c.ctl;
        const T beta = wsqrt(a);
        const bool fin = isfinite((double)beta);
        if (!fin)
            k->nonfinite = 1;
        k->beta = (double)beta;
        k->arn = (double)beta;
        k->active = fin && beta > T(0);
        c.s[0] = beta;
    }
}

// ---------------------------------------------------------------------------
// Givens step for the new Hessenberg column (Alg. 1: apply rotations
// 1..j-1, form rotation j, rotate s and the column).  Runs in the last block
// of the final orthogonalisation kernel; col is the 0-based column index,
// hc[0..col] the projections, hnext = h_{j+1,j}.
// ---------------------------------------------------------------------------
// PVS: the per-variable study's instantiation (the rotated Hessenberg entries
// under PV_H, the rotations and s under PV_GIVENS stored in binary32); the
// default one carries none of it.
template <bool PVS = false, class T, class VT>
__device__ void givens_step(GridCtx<T, VT> &c, int col, const T *hc_global, T hnext) {
    auto st32 = [&](T v, unsigned bit) { return PVS ? pv_round(v, c.pv, bit) : v; };
    __shared__ T sh[MMAX + 2], scs[MMAX], ssn[MMAX];
    for (int i = threadIdx.x; i <= col; i += blockDim.x)
        sh[i] = ldcg(hc_global + i);
    for (int i = threadIdx.x; i < col; i += blockDim.x) {
        scs[i] = c.cs[i];
        ssn[i] = c.sn[i];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        sh[col + 1] = hnext;
    __syncthreads();
    // unrotated column (for the Arnoldi relation)
    for (int i = threadIdx.x; i <= col + 1; i += blockDim.x)
        c.Hb[(size_t)col * c.ld + i] = sh[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        Ctl *k = c.ctl;
        for (int i = 0; i < col; ++i) {
            T hi = sh[i], hi1 = sh[i + 1];
            sh[i] = st32(scs[i] * hi + ssn[i] * hi1, PV_H);
            sh[i + 1] = st32(-ssn[i] * hi + scs[i] * hi1, PV_H);
        }
        T hjj = sh[col], hj1 = sh[col + 1];
        T rho = wsqrt(hjj * hjj + hj1 * hj1);
        T al, be;
        if (rho == T(0)) {
            al = T(1);
            be = T(0);
        } else {
            al = hjj / rho;
            be = hj1 / rho;
        }
        al = st32(al, PV_GIVENS);
        be = st32(be, PV_GIVENS);
        c.cs[col] = al;
        c.sn[col] = be;
        T sj = c.s[col];
        c.s[col] = st32(al * sj, PV_GIVENS);
        T snew = st32(-be * sj, PV_GIVENS);
        c.s[col + 1] = snew;
        sh[col] = st32(al * hjj + be * hj1, PV_H);
        sh[col + 1] = st32(-be * hjj + al * hj1, PV_H);
        double arn = fabs((double)snew);
        double wn0 = k->wnorm0;
        int bd = (double)hnext <= (double)c.brk * wn0;
        int nf = !isfinite(arn) || !isfinite((double)hnext);
        k->j = col + 1;
        k->arn = arn;
        k->hnext = (double)hnext;
        k->breakdown = bd;
        if (nf)
            k->nonfinite = 1;
        c.ahist[col + 1] = arn;
        int stall = c.stall_factor > 0 && col + 1 >= c.stall_w &&
                    c.ahist[col + 1 - c.stall_w] < c.stall_factor * arn;
        int end = bd || nf || (c.tau > 0 && arn <= c.tau * k->beta) || arn <= c.inner_abs ||
                  stall || (col + 1 >= c.kmax);
        k->active = !end;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= col + 1; i += blockDim.x)
        c.H[(size_t)col * c.ld + i] = sh[i];
}

// ---------------------------------------------------------------------------
// MGS chain (procedure MGS): step i applies the previous projection
// w <- w - h_{i-1} v_{i-1} and forms h_i = w . v_i in the same pass; the final
// step applies the last projection, takes ||w|| and runs the Givens step.
// ---------------------------------------------------------------------------
template <class T, class VT, bool PVS = false>
__global__ void __launch_bounds__(256) k_mgs_step(GridCtx<T, VT> c, int i) {
    if (!c.ctl->active)
        return;
    __shared__ T sred[2 * 32];
    int64_t rb, re;
    block_rows(c, rb, re);
    const T hp = (i > 0) ? c.h1[i - 1] : T(0);
    const bool rw = PVS && (c.pv & PV_W);  // per-variable w switch
    T acc[2] = {0, 0};  // [0] = w . v_i, [1] = ||w||^2 (i == 0 only)
    for (int64_t r = rb + 4 * threadIdx.x; r < re; r += 4 * blockDim.x) {
        T wv[4], vi[4];
        ldv4(c.w + r, wv);
        if (i > 0) {
            T vp[4];
            ld4<T, VT>(c.V + (size_t)(i - 1) * c.ldv + r, c.vinv, vp);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                wv[k] = wv[k] - hp * vp[k];
            if (rw) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    wv[k] = (T)(float)wv[k];
            }
            st4(c.w + r, wv);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                acc[1] += wv[k] * wv[k];
        }
        ld4<T, VT>(c.V + (size_t)i * c.ldv + r, c.vinv, vi);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            acc[0] += wv[k] * vi[k];
    }
    block_sum<T, 2>(acc, sred);
    if (threadIdx.x == 0) {
        c.part[(size_t)blockIdx.x * PSTRIDE + 0] = acc[0];
        c.part[(size_t)blockIdx.x * PSTRIDE + 1] = acc[1];
    }
    if (!arrive_last(&c.ctl->counter[1]))
        return;
    __shared__ T red[2];
    reduce_columns(c.part, gridDim.x, 2, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        c.h1[i] = PVS ? pv_round(red[0], c.pv, PV_H) : red[0];
        if (i == 0)
            c.ctl->wnorm0 = (double)wsqrt(red[1]);
    }
}

template <class T, class VT, bool PVS = false>
__global__ void __launch_bounds__(256) k_mgs_last(GridCtx<T, VT> c, int ncols) {
    if (!c.ctl->active)
        return;
    __shared__ T sred[32];
    int64_t rb, re;
    block_rows(c, rb, re);
    const int i = ncols - 1;
    const T hp = c.h1[i];
    const bool rw = PVS && (c.pv & PV_W);  // per-variable w switch
    T nsq = 0;
    for (int64_t r = rb + 4 * threadIdx.x; r < re; r += 4 * blockDim.x) {
        T wv[4], vp[4];
        ldv4(c.w + r, wv);
        ld4<T, VT>(c.V + (size_t)i * c.ldv + r, c.vinv, vp);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wv[k] = wv[k] - hp * vp[k];
            if (rw)
                wv[k] = (T)(float)wv[k];
            nsq += wv[k] * wv[k];
        }
        st4(c.w + r, wv);
    }
    nsq = block_sum1(nsq, sred);
    if (threadIdx.x == 0)
        c.part[(size_t)blockIdx.x * PSTRIDE] = nsq;
    if (!arrive_last(&c.ctl->counter[3]))
        return;
    __shared__ T stot;
    reduce_columns(c.part, gridDim.x, 1, &stot);
    __syncthreads();
    const T hn = wsqrt(stot);
    givens_step<PVS>(c, ncols - 1, c.h1, PVS ? pv_round(hn, c.pv, PV_H) : hn);
}

// v_{col} = w / h_{j+1,j} (Alg. 1 "v_{j+1} <- w / h_{j+1,j}"), rounded to the
// basis type.  Skipped when the cycle has ended.
constexpr int NORM_UNROLL = 8;
template <class T, class VT>
__global__ void __launch_bounds__(256) k_normalize(GridCtx<T, VT> c, int col, int force) {
    // force: also on the step that ended the cycle (the loss-of-orthogonality
    // test reads v_{j+1}); never after a breakdown or a skipped step
    if (!c.ctl->active &&
        !(force && c.ctl->j == col && !c.ctl->breakdown && !c.ctl->nonfinite))
        return;
    const T h = (T)c.ctl->hnext;
    int64_t rb, re;
    block_rows(c, rb, re);
    VT *dst = c.V + (size_t)col * c.ldv;
    // NORM_UNROLL groups of 4 rows per thread: all their loads are issued
    // before the first division, so enough bytes are in flight per SM to
    // stream at HBM speed with two blocks per SM
    constexpr int U = NORM_UNROLL;
    const int64_t step = 4 * (int64_t)blockDim.x;
    for (int64_t r0 = rb + 4 * threadIdx.x; r0 < re; r0 += U * step) {
        T v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (r0 + u * step < re)
                ldv4(c.w + r0 + u * step, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (r0 + u * step < re) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    v[u][k] = v[u][k] / h;
                stb4<T, VT>(dst + r0 + u * step, v[u], c.vscale);
            }
        }
    }
}

// y = H^{-1} s on the leading j x j triangle (back substitution, row-oriented
// as in the oracle; a zero pivot gives y_i = 0).  One block.
template <class T, class VT>
__global__ void k_backsolve(GridCtx<T, VT> c) {
    extern __shared__ unsigned char smraw[];
    T *Hs = reinterpret_cast<T *>(smraw);
    const int j = c.ctl->j;
    c.ctl->last_j = j;
    if (j == 0)
        return;
    for (int idx = threadIdx.x; idx < j * j; idx += blockDim.x) {
        int col = idx / j, row = idx % j;
        Hs[idx] = c.H[(size_t)col * c.ld + row];
    }
    T *ys = Hs + j * j;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = j - 1; i >= 0; --i) {
            T acc = c.s[i];
            for (int l = i + 1; l < j; ++l)
                acc -= Hs[l * j + i] * ys[l];
            T piv = Hs[i * j + i];
            T yi = (piv == T(0)) ? T(0) : acc / piv;
            if (c.pv & PV_GIVENS)
                yi = (T)(float)yi;  // the per-variable study's least-squares switch
            ys[i] = yi;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += blockDim.x)
        c.y[i] = ys[i];
}

// u = V_j y in the working precision, then x += (double) u (Alg. 1 "x_{k+1}
// <- x_k + u_k", binary64 addition, Sec. 2).  With a right preconditioner the
// kernel writes t = V_j y instead and the update is applied after t -> M t.
// PVS: the per-variable study's instantiation (x stored in binary32 under
// PV_X).
template <class T, class VT, bool PVS = false>
__global__ void __launch_bounds__(256) k_update(GridCtx<T, VT> c, double *x, int to_t) {
    __shared__ T ys[MMAX];
    const int j = c.ctl->last_j;
    if (j == 0 || c.ctl->nonfinite)
        return;
    for (int i = threadIdx.x; i < j; i += blockDim.x)
        ys[i] = c.y[i];
    __syncthreads();
    int64_t rb, re;
    block_rows(c, rb, re);
    const bool rx = PVS && (c.pv & PV_X);
    for (int64_t r = rb + 4 * threadIdx.x; r < re; r += 4 * blockDim.x) {
        T u[4] = {0, 0, 0, 0};
        for (int i = 0; i < j; ++i) {
            T v[4];
            ld4<T, VT>(c.V + (size_t)i * c.ldv + r, c.vinv, v);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                u[k] += v[k] * ys[i];
        }
        if (to_t) {
            st4(c.t + r, u);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (r + k < c.n) {
                    double xn = x[r + k] + (double)u[k];
                    if (rx)
                        xn = (double)(float)xn;  // per-variable x switch
                    x[r + k] = xn;
                }
        }
    }
}

// x += (double) u for a full-length working vector u (after u = M t).
// pv: the per-variable switches (PV_X stores x in binary32).
template <class T>
__global__ void __launch_bounds__(256) k_axpy_x(int n, const T *u, double *x, const Ctl *ctl,
                                                unsigned pv) {
    if (ctl->last_j == 0 || ctl->nonfinite)
        return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        x[r] = pv_round(x[r] + (double)u[r], pv, PV_X);
}

// v <- fl32(v) entry by entry (per-variable study: the initial x under PV_X,
// w after a left preconditioner under PV_W).  Skipped when the cycle has
// ended if ctl is given.
template <class T>
__global__ void __launch_bounds__(256) k_round32(int64_t n, T *v, const Ctl *ctl) {
    if (ctl && !ctl->active)
        return;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        v[r] = (T)(float)v[r];
}

// ||b||_2 in binary64 into ctl->bnorm (two-stage, deterministic).
template <class T, class VT>
__global__ void __launch_bounds__(256) k_bnorm(GridCtx<T, VT> c, const double *b) {
    __shared__ double sd[32];
    double ss = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < c.n;
         r += (int64_t)gridDim.x * blockDim.x) {
        double v = b[r];
        ss += v * v;
    }
    ss = block_sum1(ss, sd);
    if (threadIdx.x == 0)
        c.part64[(size_t)blockIdx.x * 4 + 2] = ss;
    if (!arrive_last(&c.ctl->counter[4]))
        return;
    double a = 0;
    for (int bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x)
        a += ldcg(c.part64 + (size_t)bb * 4 + 2);
    a = block_sum1(a, sd);
    if (threadIdx.x == 0) {
        c.ctl->bnorm = sqrt(a);
        if (!isfinite(a))
            c.ctl->nonfinite = 1;
    }
}

// Widen basis columns [0, ncols) to binary64 (for export), rows < n.
template <class T, class VT>
__global__ void k_export_basis(GridCtx<T, VT> c, int ncols, double *out) {
    const int64_t total = (int64_t)ncols * c.n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t col = idx / c.n, row = idx % c.n;
        out[idx] = (double)Basis<VT>::ld(c.V + col * c.ldv + row, c.vinv);
    }
}

// Basis columns [0, ncols) from a binary64 host-side copy (column i at
// src + i * n), rounded to the storage type; padding rows stay zero.  Used by
// the one-step replay entry point, whose inputs are basis values as stored.
template <class T, class VT>
__global__ void k_import_basis(GridCtx<T, VT> c, int ncols, const double *src) {
    const int64_t total = (int64_t)ncols * c.n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t col = idx / c.n, row = idx % c.n;
        Basis<VT>::st(c.V + col * c.ldv + row, (T)src[idx], c.vscale);
    }
}

}  // namespace gmres
