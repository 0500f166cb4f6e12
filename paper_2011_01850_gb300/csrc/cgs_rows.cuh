// cgs_rows.cuh -- the three passes of CGSR (procedure CGSR of Algorithm 1,
// done twice; arXiv 2011.01850) as register-streaming kernels.
//
//   MODE 0  h1 = V^T w (+ ||w||, the breakdown reference)
//   MODE 1  w <- w - V h1, then h2 = V^T w
//   MODE 2  w <- w - V h2, ||w||^2 -> h_{j+1,j}, column h1 + h2, Givens step
//
// Every warp walks its own row slices (warp-steps) in grid-stride order.  In
// a warp-step each lane holds RPL consecutive rows of w and, for every basis
// vector, loads the same RPL rows with one 16-byte vector load, so a warp
// moves 512 contiguous bytes of each column per load instruction and keeps
// many of them in flight without staging.  The dot products accumulate in
// one register per column per lane across all of the warp's slices and are
// reduced once at the end (warp butterfly, then block, then grid through the
// last block, all in a fixed order).  Pass B's second step reloads the slice
// it has just read: those lines are still in L2, so the basis crosses HBM
// once per pass.  binary64 bases split the columns over lane pairs so the
// per-column accumulators fit in registers.
#pragma once

#include "grid_kernels.cuh"

namespace gmres {

template <class T, class VT>
struct RowsCfg;
template <>
struct RowsCfg<float, float> {
    static constexpr int RPL = 4, LPR = 1;
};
template <>
struct RowsCfg<double, double> {
    static constexpr int RPL = 2, LPR = 2;
};
template <>
struct RowsCfg<float, __nv_bfloat16> {
    static constexpr int RPL = 8, LPR = 1;
};
template <>
struct RowsCfg<float, __half> {
    static constexpr int RPL = 8, LPR = 1;
};

// RPL consecutive basis entries (16 bytes) widened to the working type.
template <class T, class VT, int RPL>
__device__ __forceinline__ void ld_rows(const VT *p, float vinv, T (&o)[RPL]);

template <>
__device__ __forceinline__ void ld_rows<float, float, 4>(const float *p, float, float (&o)[4]) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
template <>
__device__ __forceinline__ void ld_rows<double, double, 2>(const double *p, float,
                                                            double (&o)[2]) {
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = a.x; o[1] = a.y;
}
template <>
__device__ __forceinline__ void ld_rows<float, __nv_bfloat16, 8>(const __nv_bfloat16 *p, float,
                                                                 float (&o)[8]) {
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
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
                                                          float (&o)[8]) {
    uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
    const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 f = __half22float2(h[q]);
        o[2 * q] = f.x * vinv;
        o[2 * q + 1] = f.y * vinv;
    }
}

// RPL working-precision entries of w (plain loads: w is written by pass B/C).
template <class T, int RPL>
__device__ __forceinline__ void ld_w(const T *p, T (&o)[RPL]) {
#pragma unroll
    for (int q = 0; q < RPL; q += 16 / (int)sizeof(T) < RPL ? 16 / (int)sizeof(T) : RPL) {
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
#pragma unroll
    for (int q = 0; q < RPL; q += 16 / (int)sizeof(T) < RPL ? 16 / (int)sizeof(T) : RPL) {
        if (sizeof(T) == 4)
            *reinterpret_cast<float4 *>(p + q) =
                make_float4((float)v[q], (float)v[q + 1], (float)v[q + 2], (float)v[q + 3]);
        else
            *reinterpret_cast<double2 *>(p + q) = make_double2((double)v[q], (double)v[q + 1]);
    }
}

constexpr int ROWS_THREADS = 128;

template <class T, class VT, int MODE>
__global__ void __launch_bounds__(ROWS_THREADS)
    k_cgs_rows(GridCtx<T, VT> c, int ncols) {
    if (!c.ctl->active)
        return;
    constexpr int RPL = RowsCfg<T, VT>::RPL, LPR = RowsCfg<T, VT>::LPR;
    constexpr int ACC = (MMAX + 1 + LPR - 1) / LPR;   // columns per lane
    constexpr int NW = ROWS_THREADS / 32;
    constexpr int RW = (32 / LPR) * RPL;                // rows per warp-step
    __shared__ T hs[MMAX + 2];
    __shared__ T red[NW][MMAX + 2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int phase = lane % LPR, slot = lane / LPR;
    if (MODE >= 1) {
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
    const int64_t nsteps = c.ldv / RW;
    const int64_t gw = (int64_t)blockIdx.x * NW + wid;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    for (int64_t st = gw; st < nsteps; st += nwarps) {
        const int64_t r = st * RW + (int64_t)slot * RPL;
        T w[RPL];
        ld_w<T, RPL>(c.w + r, w);
        if (MODE >= 1) {
            T t[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                t[q] = 0;
#pragma unroll
            for (int k = 0; k < ACC; ++k) {
                const int col = k * LPR + phase;
                if (col < ncols) {
                    T v[RPL];
                    ld_rows<T, VT, RPL>(c.V + (size_t)col * c.ldv + r, c.vinv, v);
                    const T hc = hs[col];
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        t[q] += v[q] * hc;
                }
            }
            if (LPR == 2) {
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    t[q] += __shfl_xor_sync(0xffffffffu, t[q], 1);
            }
#pragma unroll
            for (int q = 0; q < RPL; ++q)
                w[q] = w[q] - t[q];
            if (phase == 0)
                st_w<T, RPL>(c.w + r, w);
        }
        if (MODE == 0 || MODE == 2) {
            if (phase == 0) {
#pragma unroll
                for (int q = 0; q < RPL; ++q)
                    nsq += w[q] * w[q];
            }
        }
        if (MODE <= 1) {
#pragma unroll
            for (int k = 0; k < ACC; ++k) {
                const int col = k * LPR + phase;
                if (col < ncols) {
                    T v[RPL];
                    ld_rows<T, VT, RPL>(c.V + (size_t)col * c.ldv + r, c.vinv, v);
                    T a = 0;
#pragma unroll
                    for (int q = 0; q < RPL; ++q)
                        a += v[q] * w[q];
                    acc[k] += a;
                }
            }
        }
    }
    T *mypart = c.part + (size_t)blockIdx.x * PSTRIDE;
    if (MODE <= 1) {
        // lanes of one phase share their columns: butterfly over those lanes
#pragma unroll
        for (int k = 0; k < ACC; ++k) {
            T v = acc[k];
#pragma unroll
            for (int off = 16; off >= LPR; off >>= 1)
                v += __shfl_xor_sync(0xffffffffu, v, off);
            const int col = k * LPR + phase;
            if (lane < LPR && col < ncols)
                red[wid][col] = v;
        }
        __syncthreads();
        for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
            T s = 0;
#pragma unroll
            for (int w_ = 0; w_ < NW; ++w_)
                s += red[w_][col];
            mypart[col] = s;
        }
    }
    if (MODE != 1) {
        __shared__ T sred[32];
        T tot = block_sum1(nsq, sred);
        if (threadIdx.x == 0)
            mypart[MMAX + 1] = tot;
    }
    if (!arrive_last(&c.ctl->counter[MODE + 1]))
        return;
    __shared__ T snorm;
    if (MODE == 0) {
        reduce_columns(c.part, gridDim.x, ncols, c.h1);
        reduce_columns(c.part + MMAX + 1, gridDim.x, 1, &snorm);
        __syncthreads();
        if (threadIdx.x == 0)
            c.ctl->wnorm0 = (double)wsqrt(snorm);
    } else if (MODE == 1) {
        reduce_columns(c.part, gridDim.x, ncols, c.h2);
    } else {
        reduce_columns(c.part + MMAX + 1, gridDim.x, 1, &snorm);
        for (int i = threadIdx.x; i < ncols; i += blockDim.x)
            c.h1[i] = ldcg(c.h1 + i) + ldcg(c.h2 + i);
        __threadfence_block();
        __syncthreads();
        givens_step(c, ncols - 1, c.h1, wsqrt(snorm));
    }
}

}  // namespace gmres
