// cgs_rows.cuh -- the three passes of CGSR (procedure CGSR of Algorithm 1,
// done twice; arXiv 2011.01850) as register-streaming kernels.
//
//   MODE 0  partial h1 = V^T w per block            (+ ||w||^2)
//   MODE 1  w <- w - V h1, then partial h2 = V^T w per block
//   MODE 2  w <- w - V h2, ||w||^2 -> h_{j+1,j}; column h1 + h2; Givens step
//   MODE 3  partial u = V^T v_k per block, v_k = basis column `ncols` (the
//           loss-of-orthogonality test, Sec. 3 fourth strategy)
// k_reduce_cols sums the per-block partials of MODE 0 / 1 (one block per
// basis vector, fixed order) between the passes.
//
// A block walks slices of SR = 4 RW rows (RW = rows of one warp-step: 32
// lanes x RPL rows, RPL rows = one 16-byte vector of the basis type).  For
// the dot products the four warps split the basis vectors (warp w takes
// vectors w, w+4, ...), so a lane keeps at most 33 accumulators, and load the
// four row groups of the slice; for the update each warp takes one row group
// and all vectors.  Loads are issued in batches of CB vectors before their
// values are used, so a warp keeps CB x 512 contiguous bytes in flight.  In
// pass B the updated w of the slice goes through shared memory from the
// update step to the dot step (two block barriers per slice), and the basis
// slice the dot step reloads is still in L2: the basis crosses HBM once per
// pass.
#pragma once

#include "grid_kernels.cuh"

namespace gmres {

template <class VT>
struct RowsCfg {
    static constexpr int RPL = 16 / (int)sizeof(VT);  // rows per 16-byte vector
};

// L2 eviction policies for the basis stream: lines a pass reads once are
// marked evict-first; lines pass B reads twice are marked evict-last on the
// first read (so they are still in L2 for the second) and evict-first on the
// second.
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16 bytes through the read-only path with an L2 cache policy.
__device__ __forceinline__ uint4 ld16(const void *p, uint64_t pol) {
    uint4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

// RPL consecutive basis entries (16 bytes) widened to the working type.
template <class T, class VT, int RPL>
__device__ __forceinline__ void ld_rows(const VT *p, float vinv, T (&o)[RPL], uint64_t pol);

template <>
__device__ __forceinline__ void ld_rows<float, float, 4>(const float *p, float, float (&o)[4],
                                                         uint64_t pol) {
    uint4 u = ld16(p, pol);
    o[0] = __uint_as_float(u.x); o[1] = __uint_as_float(u.y);
    o[2] = __uint_as_float(u.z); o[3] = __uint_as_float(u.w);
}
template <>
__device__ __forceinline__ void ld_rows<double, float, 4>(const float *p, float, double (&o)[4],
                                                          uint64_t pol) {
    uint4 u = ld16(p, pol);
    o[0] = __uint_as_float(u.x); o[1] = __uint_as_float(u.y);
    o[2] = __uint_as_float(u.z); o[3] = __uint_as_float(u.w);
}
template <>
__device__ __forceinline__ void ld_rows<double, double, 2>(const double *p, float,
                                                            double (&o)[2], uint64_t pol) {
    uint4 u = ld16(p, pol);
    o[0] = __hiloint2double((int)u.y, (int)u.x);
    o[1] = __hiloint2double((int)u.w, (int)u.z);
}
template <>
__device__ __forceinline__ void ld_rows<float, __nv_bfloat16, 8>(const __nv_bfloat16 *p, float,
                                                                 float (&o)[8], uint64_t pol) {
    uint4 u = ld16(p, pol);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 f = __bfloat1622float2(h[q]);
        o[2 * q] = f.x;
        o[2 * q + 1] = f.y;
    }
}
template <>
__device__ __forceinline__ void ld_rows<float, __half, 8>(const __half *p, float vinv,
                                                          float (&o)[8], uint64_t pol) {
    uint4 u = ld16(p, pol);
    const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 f = __half22float2(h[q]);
        o[2 * q] = f.x * vinv;
        o[2 * q + 1] = f.y * vinv;
    }
}

// RPL working-precision entries of w (plain loads and stores: pass B and C
// write w).  RPL * sizeof(T) is 16 or 32 bytes.
template <class T, int RPL>
__device__ __forceinline__ void ld_w(const T *p, T (&o)[RPL]) {
    constexpr int PER = 16 / (int)sizeof(T);
#pragma unroll
    for (int q = 0; q < RPL; q += PER) {
        if (sizeof(T) == 4) {
            float4 a = *reinterpret_cast<const float4 *>(p + q);
            o[q] = a.x; o[q + 1] = a.y; o[q + 2] = a.z; o[q + 3] = a.w;
        } else {
            double2 a = *reinterpret_cast<const double2 *>(p + q);
            o[q] = a.x; o[q + 1] = a.y;
        }
    }
}
template <class T, int RPL>
__device__ __forceinline__ void st_w(T *p, const T (&v)[RPL]) {
    constexpr int PER = 16 / (int)sizeof(T);
#pragma unroll
    for (int q = 0; q < RPL; q += PER) {
        if (sizeof(T) == 4)
            *reinterpret_cast<float4 *>(p + q) =
                make_float4((float)v[q], (float)v[q + 1], (float)v[q + 2], (float)v[q + 3]);
        else
            *reinterpret_cast<double2 *>(p + q) = make_double2((double)v[q], (double)v[q + 1]);
    }
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

constexpr int ROWS_THREADS = 128;
constexpr int ROWS_WARPS = ROWS_THREADS / 32;
constexpr int ROWS_CB = 8;  // basis vectors loaded per batch

// t = sum_col h[col] * V[col][r .. r+RPL) over all ncols vectors (one warp
// row group), batched loads.
template <class T, class VT, int RPL>
__device__ __forceinline__ void rows_project(const GridCtx<T, VT> &c, int ncols, const T *hs,
                                             int64_t r, T (&t)[RPL], uint64_t pol) {
#pragma unroll
    for (int q = 0; q < RPL; ++q)
        t[q] = 0;
#pragma unroll
    for (int c0 = 0; c0 < MMAX + 1; c0 += ROWS_CB) {
        if (c0 < ncols) {
            T v[ROWS_CB][RPL];
#pragma unroll
            for (int u = 0; u < ROWS_CB; ++u) {
                if (c0 + u < ncols)
                    ld_rows<T, VT, RPL>(c.V + (size_t)(c0 + u) * c.ldv + r, c.vinv, v[u], pol);
                else {
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        v[u][q] = 0;
                }
            }
#pragma unroll
            for (int u = 0; u < ROWS_CB; ++u) {
                const T hc = (c0 + u < ncols) ? hs[c0 + u] : T(0);
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    t[q] += v[u][q] * hc;
            }
        }
    }
}

// tp[g][q] = sum over this warp's vectors (wid, wid+4, ...) of
// h[col] * V[col][slice row g*RW + lane*RPL + q]: the update's partial sums
// with every vector read as one 2 KB run per warp (as in the dot products),
// summed over the warp's vectors in ascending order, batched loads.
template <class T, class VT, int RPL, int ACC>
__device__ __forceinline__ void rows_project_split(const GridCtx<T, VT> &c, int ncols,
                                                   const T *hs, int64_t s0, int wid, int lane,
                                                   T (&tp)[4][RPL], uint64_t pol) {
    constexpr int RW = 32 * RPL;
    constexpr int KB = ROWS_CB / 4 > 0 ? ROWS_CB / 4 : 1;
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int q = 0; q < RPL; ++q)
            tp[g][q] = 0;
#pragma unroll
    for (int k0 = 0; k0 < ACC; k0 += KB) {
        if (wid + ROWS_WARPS * k0 < ncols) {
            T v[KB][4][RPL];
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const int col = wid + ROWS_WARPS * (k0 + u);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    if (k0 + u < ACC && col < ncols)
                        ld_rows<T, VT, RPL>(c.V + (size_t)col * c.ldv + s0 + g * RW + lane * RPL,
                                            c.vinv, v[u][g], pol);
                    else {
#pragma unroll
                        for (int q = 0; q < RPL; ++q)
                            v[u][g][q] = 0;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const int col = wid + ROWS_WARPS * (k0 + u);
                const T hc = (k0 + u < ACC && col < ncols) ? hs[col] : T(0);
#pragma unroll
                for (int g = 0; g < 4; ++g)
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        tp[g][q] += v[u][g][q] * hc;
            }
        }
    }
}

// acc[k] += V[wid + 4k][slice rows] . ws (the slice's w, 4 row groups in
// shared memory or registers), batched loads.
template <class T, class VT, int RPL, int ACC>
__device__ __forceinline__ void rows_dots(const GridCtx<T, VT> &c, int ncols, int64_t s0,
                                          const T (&wv)[4][RPL], int wid, int lane,
                                          T (&acc)[ACC], uint64_t pol) {
    constexpr int RW = 32 * RPL;
    constexpr int KB = ROWS_CB / 4 > 0 ? ROWS_CB / 4 : 1;  // vectors per batch (x4 groups)
#pragma unroll
    for (int k0 = 0; k0 < ACC; k0 += KB) {
        if (wid + ROWS_WARPS * k0 < ncols) {
            T v[KB][4][RPL];
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                const int col = wid + ROWS_WARPS * (k0 + u);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    if (k0 + u < ACC && col < ncols)
                        ld_rows<T, VT, RPL>(c.V + (size_t)col * c.ldv + s0 + g * RW + lane * RPL,
                                            c.vinv, v[u][g], pol);
                    else {
#pragma unroll
                        for (int q = 0; q < RPL; ++q)
                            v[u][g][q] = 0;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < KB; ++u) {
                if (k0 + u < ACC) {
                    T a = 0;
#pragma unroll
                    for (int g = 0; g < 4; ++g)
#pragma unroll
                        for (int q = 0; q < RPL; ++q)
                            a += v[u][g][q] * wv[g][q];
                    acc[k0 + u] += a;
                }
            }
        }
    }
}

// PVS: the per-variable study's instantiation (every updated entry of w under
// PV_W, the Hessenberg column and h_{j+1,j} under PV_H stored in binary32), so
// the default passes carry none of it.
template <class T, class VT, int MODE, bool SPLIT = true, bool PVS = false>
__global__ void __launch_bounds__(ROWS_THREADS)
    k_cgs_rows(GridCtx<T, VT> c, int ncols, T *part, int64_t slices_per_block, int pf) {
    // MODE 3 follows the step that appended basis column ncols, also when
    // that step ended the cycle
    if (MODE == 3 ? !(c.ctl->j == ncols && !c.ctl->breakdown && !c.ctl->nonfinite)
                  : !c.ctl->active)
        return;
    constexpr int RPL = RowsCfg<VT>::RPL;
    constexpr int RW = 32 * RPL;                   // rows per warp-step
    constexpr int SR = ROWS_WARPS * RW;            // rows per block slice
    constexpr int ACC = (MMAX + 1 + ROWS_WARPS - 1) / ROWS_WARPS;
    __shared__ T hs[MMAX + 2];
    __shared__ __align__(16) T wsl[SR];
    // SPLIT update: the four warps' partial sums of V h for the slice
    __shared__ __align__(16) T tsm[(MODE == 1 || MODE == 2) && SPLIT ? ROWS_WARPS * SR : 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (MODE == 1 || MODE == 2) {
        const T *src = (MODE == 1) ? c.h1 : c.h2;
        for (int i = threadIdx.x; i < ncols; i += blockDim.x)
            hs[i] = src[i];
        __syncthreads();
    }
    T acc[ACC];
#pragma unroll
    for (int k = 0; k < ACC; ++k)
        acc[k] = 0;
    T nsq = 0;
    const uint64_t pol_once = l2_policy_first();
    const uint64_t pol_keep = (MODE == 1) ? l2_policy_last() : pol_once;
    // each block takes an equal run of consecutive slices (the host sizes the
    // grid so the runs cover the basis with at most one short run)
    const int64_t nslices = c.ldv / SR;
    const int64_t sl0 = (int64_t)blockIdx.x * slices_per_block;
    int64_t sl1 = sl0 + slices_per_block;
    if (sl1 > nslices)
        sl1 = nslices;
    for (int64_t sl = sl0; sl < sl1; ++sl) {
        const int64_t s0 = sl * SR;
        // slice sl + pf of this block's run: one 16-byte-aligned 2 KB row
        // block per basis vector (ldv is a multiple of SR) and w's rows
        if (pf > 0 && sl + pf < sl1) {
            const int64_t p0 = (sl + pf) * SR;
            for (int col = threadIdx.x; col <= ncols; col += ROWS_THREADS) {
                if (col < ncols || MODE == 3)
                    prefetch_l2(c.V + (size_t)col * c.ldv + p0, SR * (unsigned)sizeof(VT));
                else
                    prefetch_l2(c.w + p0, SR * (unsigned)sizeof(T));
            }
        }
        T wv[4][RPL];
        if (MODE == 3) {
            const VT *vk = c.V + (size_t)ncols * c.ldv + s0 + lane * RPL;
#pragma unroll
            for (int g = 0; g < 4; ++g)
                ld_rows<T, VT, RPL>(vk + g * RW, c.vinv, wv[g], pol_once);
        } else if (MODE == 0) {
#pragma unroll
            for (int g = 0; g < 4; ++g)
                ld_w<T, RPL>(c.w + s0 + g * RW + lane * RPL, wv[g]);
            if (wid == 0) {
#pragma unroll
                for (int g = 0; g < 4; ++g)
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        nsq += wv[g][q] * wv[g][q];
            }
        } else if (SPLIT) {
            // update, split by vectors: every warp sums its vectors over the
            // whole slice (2 KB runs), the partials meet in shared memory and
            // warp wid forms row group wid as ((p0 + p1) + p2) + p3.  The
            // thread's rows of w are loaded first (only this block touches
            // the slice), so their latency hides under the basis loads.
            const int64_t r = s0 + wid * RW + lane * RPL;
            T w[RPL];
            ld_w<T, RPL>(c.w + r, w);
            T tp[4][RPL];
            rows_project_split<T, VT, RPL, ACC>(c, ncols, hs, s0, wid, lane, tp, pol_keep);
#pragma unroll
            for (int g = 0; g < 4; ++g)
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    tsm[wid * SR + g * RW + lane * RPL + q] = tp[g][q];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                const int o = wid * RW + lane * RPL + q;
                const T t = ((tsm[o] + tsm[SR + o]) + tsm[2 * SR + o]) + tsm[3 * SR + o];
                w[q] = w[q] - t;
                if (PVS)
                    w[q] = pv_round(w[q], c.pv, PV_W);
                if (MODE == 2)
                    nsq += w[q] * w[q];
                if (MODE == 1)
                    wsl[o] = w[q];
            }
            st_w<T, RPL>(c.w + r, w);
            __syncthreads();
            if (MODE == 1) {
#pragma unroll
                for (int g = 0; g < 4; ++g)
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        wv[g][q] = wsl[g * RW + lane * RPL + q];
            }
        } else {
            // update: warp wid owns row group wid of the slice
            const int64_t r = s0 + wid * RW + lane * RPL;
            T w[RPL], t[RPL];
            ld_w<T, RPL>(c.w + r, w);
            rows_project<T, VT, RPL>(c, ncols, hs, r, t, pol_keep);
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
                w[q] = w[q] - t[q];
                if (PVS)
                    w[q] = pv_round(w[q], c.pv, PV_W);
                if (MODE == 2)
                    nsq += w[q] * w[q];
            }
            st_w<T, RPL>(c.w + r, w);
            if (MODE == 1) {
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    wsl[wid * RW + lane * RPL + q] = w[q];
                __syncthreads();
#pragma unroll
                for (int g = 0; g < 4; ++g)
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        wv[g][q] = wsl[g * RW + lane * RPL + q];
                __syncthreads();
            }
        }
        if (MODE != 2)
            rows_dots<T, VT, RPL, ACC>(c, ncols, s0, wv, wid, lane, acc, pol_once);
    }
    T *mypart = part + (size_t)blockIdx.x * PSTRIDE;
    if (MODE != 2) {
#pragma unroll
        for (int k = 0; k < ACC; ++k) {
            const int col = wid + ROWS_WARPS * k;
            T v = warp_sum(acc[k]);
            if (lane == 0 && col < ncols)
                mypart[col] = v;
        }
    }
    if (MODE == 0 || MODE == 2) {
        __shared__ T sred[32];
        T tot = block_sum1(nsq, sred);
        if (threadIdx.x == 0)
            mypart[MMAX + 1] = tot;
    }
    if (MODE != 2)
        return;
    // MODE 2: ||w||^2 over blocks in the last block, then the Givens step
    if (!arrive_last(&c.ctl->counter[3]))
        return;
    __shared__ T snorm;
    reduce_columns(part + MMAX + 1, gridDim.x, 1, &snorm);
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
        const T hsum = ldcg(c.h1 + i) + ldcg(c.h2 + i);
        c.h1[i] = PVS ? pv_round(hsum, c.pv, PV_H) : hsum;
    }
    __threadfence();
    __syncthreads();
    const T hn = wsqrt(snorm);
    givens_step<PVS>(c, ncols - 1, c.h1, PVS ? pv_round(hn, c.pv, PV_H) : hn);
}

// Pass B with the slice held in registers (binary32 basis): w <- w - V h1,
// then partial h2 = V^T w, reading every basis vector once.  A block walks
// 128-row slices; its 8 warps split the basis vectors (warp w takes vectors
// w, w+8, ...) and every lane loads 4 rows of each of its at most KC vectors
// (16-byte loads, all issued before use) and keeps them: the warps' partial
// sums of V h1 meet in shared memory, threads 0..127 form the updated w of
// the slice, and the dot products then use the vectors still in registers
// instead of reading them again.  Partials of V h1 are summed over warps in
// order; the dot partials per lane over the block's slices, then by an xor
// butterfly.
constexpr int PB_THREADS = 256;
constexpr int PB_WARPS = PB_THREADS / 32;
constexpr int PB_ROWS = 128;  // rows per slice (32 lanes x 4)

template <int KC>
__global__ void __launch_bounds__(PB_THREADS)
    k_cgs_passb_reg(GridCtx<float, float> c, int ncols, float *part, int64_t slices_per_block) {
    if (!c.ctl->active)
        return;
    __shared__ float hs[MMAX + 2];
    __shared__ __align__(16) float tsm[PB_WARPS * PB_ROWS];
    __shared__ __align__(16) float wsl[PB_ROWS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < ncols; i += PB_THREADS)
        hs[i] = c.h1[i];
    __syncthreads();
    const uint64_t pol = l2_policy_first();
    float acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k)
        acc[k] = 0.f;
    const int64_t nslices = c.ldv / PB_ROWS;
    const int64_t sl0 = (int64_t)blockIdx.x * slices_per_block;
    int64_t sl1 = sl0 + slices_per_block;
    if (sl1 > nslices)
        sl1 = nslices;
    // w of a slice is read one slice ahead (only this block touches its
    // slices), so the update below does not wait for it
    float wcur = (threadIdx.x < PB_ROWS && sl0 < sl1) ? c.w[sl0 * PB_ROWS + threadIdx.x] : 0.f;
    for (int64_t sl = sl0; sl < sl1; ++sl) {
        const int64_t s0 = sl * PB_ROWS;
        const float wnext = (threadIdx.x < PB_ROWS && sl + 1 < sl1)
                                ? c.w[s0 + PB_ROWS + threadIdx.x]
                                : 0.f;
        float v[KC][4];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int col = wid + PB_WARPS * k;
            if (col < ncols)
                ld_rows<float, float, 4>(c.V + (size_t)col * c.ldv + s0 + lane * 4, 1.f, v[k],
                                         pol);
            else
                v[k][0] = v[k][1] = v[k][2] = v[k][3] = 0.f;
        }
        float tp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const int col = wid + PB_WARPS * k;
            const float hc = col < ncols ? hs[col] : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tp[q] += v[k][q] * hc;
        }
        *reinterpret_cast<float4 *>(tsm + wid * PB_ROWS + lane * 4) =
            make_float4(tp[0], tp[1], tp[2], tp[3]);
        __syncthreads();
        if (threadIdx.x < PB_ROWS) {
            const int r = threadIdx.x;
            float t = tsm[r];
#pragma unroll
            for (int w = 1; w < PB_WARPS; ++w)
                t += tsm[w * PB_ROWS + r];
            const float wn = wcur - t;
            c.w[s0 + r] = wn;
            wsl[r] = wn;
        }
        wcur = wnext;
        __syncthreads();
        const float4 wv = *reinterpret_cast<const float4 *>(wsl + lane * 4);
#pragma unroll
        for (int k = 0; k < KC; ++k)
            acc[k] += ((v[k][0] * wv.x + v[k][1] * wv.y) + v[k][2] * wv.z) + v[k][3] * wv.w;
    }
    float *mypart = part + (size_t)blockIdx.x * PSTRIDE;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int col = wid + PB_WARPS * k;
        const float a = warp_sum(acc[k]);
        if (lane == 0 && col < ncols)
            mypart[col] = a;
    }
}

// out[col] = sum over the blocks of part[b][col], col < ncols, and, when
// `extra` >= 0, ctl->wnorm0 = sqrt(sum of part[b][MMAX+1]) (the ||A v_j||
// reference of pass A).  One block per column, fixed-order tree.  pv: the
// per-variable switches (PV_H stores the projection coefficients in binary32).
template <class T>
__global__ void __launch_bounds__(256) k_reduce_cols(const T *part, int nblocks, int ncols,
                                                     T *out, Ctl *ctl, int with_norm,
                                                     unsigned pv = 0) {
    // with_norm 2: the Gram column of MODE 3 (runs under its condition)
    if (with_norm == 2 ? !(ctl->j == ncols && !ctl->breakdown && !ctl->nonfinite)
                       : !ctl->active)
        return;
    __shared__ T sred[32];
    const int col = blockIdx.x;
    const int slot = (col < ncols) ? col : MMAX + 1;
    T a = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        a += part[(size_t)b * PSTRIDE + slot];
    a = block_sum1(a, sred);
    if (threadIdx.x == 0) {
        if (col < ncols) {
            if (pv & PV_H)
                a = (T)(float)a;  // the per-variable study's Hessenberg switch
            out[col] = a;
        }
        else if (with_norm)
            ctl->wnorm0 = (double)wsqrt(a);
    }
}

}  // namespace gmres
