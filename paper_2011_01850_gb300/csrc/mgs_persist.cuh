// mgs_persist.cuh -- procedure MGS of Algorithm 1 (arXiv 2011.01850) for one
// inner step as a single cooperative kernel.
//
// MGS needs the inner product h_i = w . v_i of the already-updated w before it
// can project v_i out, so an inner step of j basis vectors has j global
// reductions in sequence.  Here every block keeps its row chunk of w in shared
// memory for the whole step; per basis vector it makes one sweep over its
// rows that applies the previous projection (w <- w - h_{i-1} v_{i-1}) and
// accumulates w . v_i, writes its partial, and meets the other blocks at a
// grid barrier; then every block sums all partials in block order (so all
// blocks see the same h_i, bit for bit).  The last sweep applies the final
// projection and takes ||w||; the blocks then write v_{j+1} = w / h_{j+1,j}
// straight into the basis and block 0 runs the Givens step.  w never goes
// back to global memory and the basis is read once from HBM per step (the
// previous vector comes back from L1/L2).
//
// The grid is launched cooperatively (all blocks resident).  Every barrier
// wait is bounded: after `spin` polls the block records a timeout in the
// control block, the other blocks see it at their next poll, and all return.
#pragma once

#include "grid_kernels.cuh"

namespace gmres {

constexpr int MGSP_THREADS = 512;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier over co-resident blocks: bar[0] arrival count, bar[1]
// generation.  Returns false (in every thread of the block) when this block
// gave up after `limit` polls or saw another block give up (*err != 0).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_gpu(bar + 1);
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            st_release_gpu(bar + 1, g + 1);
        } else {
            long long it = 0;
            while (ld_acquire_gpu(bar + 1) == g) {
                if (*(volatile int *)err != 0 || ++it > limit) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && (*(volatile int *)err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum of slot `slot` of every block's partials, in block order, broadcast to
// the whole block.
template <class T>
__device__ __forceinline__ T sum_partials(const T *part, int slot, T *sbuf) {
    if (threadIdx.x < 32) {
        T a = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
            a += ldcg(part + (size_t)b * PSTRIDE + slot);
        a = warp_sum(a);
        if (threadIdx.x == 0)
            *sbuf = a;
    }
    __syncthreads();
    T v = *sbuf;
    __syncthreads();
    return v;
}

template <class T, class VT>
__global__ void __launch_bounds__(MGSP_THREADS, 1)
    k_mgs_persist(GridCtx<T, VT> c, int ncols, int64_t chunk, long long spin, unsigned *bar) {
    if (!c.ctl->active)
        return;
    extern __shared__ __align__(16) unsigned char mgs_smem[];
    T *ws = reinterpret_cast<T *>(mgs_smem);
    __shared__ T sred[2 * 32];
    __shared__ T sval;
    __shared__ T hcol[MMAX + 2];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk;
    int64_t re = rb + chunk;
    if (re > c.ldv)
        re = c.ldv;
    const int64_t len = re > rb ? re - rb : 0;
    T *mypart = c.part + (size_t)blockIdx.x * PSTRIDE;
    int *err = &c.ctl->timeout;

    for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
        T v[4];
        ldv4(c.w + rb + q, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            ws[q + k] = v[k];
    }
    __syncthreads();
    // h_0 = w . v_0 and ||w||^2 (breakdown reference)
    {
        T acc[2] = {0, 0};
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T v[4];
            ld4<T, VT>(c.V + rb + q, c.vinv, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[0] += ws[q + k] * v[k];
                acc[1] += ws[q + k] * ws[q + k];
            }
        }
        block_sum<T, 2>(acc, sred);
        if (tid == 0) {
            mypart[0] = acc[0];
            mypart[2] = acc[1];
        }
    }
    if (!grid_barrier(bar, err, spin))
        return;
    T hprev = sum_partials(c.part, 0, &sval);
    const T wn0sq = sum_partials(c.part, 2, &sval);
    if (tid == 0)
        hcol[0] = hprev;
    // h_i for i >= 1: one sweep applies projection i-1 and dots with v_i
    for (int i = 1; i < ncols; ++i) {
        const VT *vp = c.V + (size_t)(i - 1) * c.ldv + rb;
        const VT *vi = c.V + (size_t)i * c.ldv + rb;
        T d = 0;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T a[4], b[4];
            ld4<T, VT>(vp + q, c.vinv, a);
            ld4<T, VT>(vi + q, c.vinv, b);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T wv = ws[q + k] - hprev * a[k];
                ws[q + k] = wv;
                d += wv * b[k];
            }
        }
        d = block_sum1(d, sred);
        if (tid == 0)
            mypart[i & 1] = d;
        if (!grid_barrier(bar, err, spin))
            return;
        hprev = sum_partials(c.part, i & 1, &sval);
        if (tid == 0)
            hcol[i] = hprev;
    }
    // last projection and ||w||^2
    {
        const VT *vp = c.V + (size_t)(ncols - 1) * c.ldv + rb;
        T nsq = 0;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T a[4];
            ld4<T, VT>(vp + q, c.vinv, a);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T wv = ws[q + k] - hprev * a[k];
                ws[q + k] = wv;
                nsq += wv * wv;
            }
        }
        nsq = block_sum1(nsq, sred);
        if (tid == 0)
            mypart[3] = nsq;
    }
    if (!grid_barrier(bar, err, spin))
        return;
    const T hnext = wsqrt(sum_partials(c.part, 3, &sval));
    // v_{j+1} = w / h_{j+1,j} into basis column ncols (unused if the cycle ends)
    if (hnext > T(0)) {
        VT *dst = c.V + (size_t)ncols * c.ldv + rb;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                v[k] = ws[q + k] / hnext;
            stb4<T, VT>(dst + q, v, c.vscale);
        }
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < ncols; i += nth)
            c.h1[i] = hcol[i];
        if (tid == 0)
            c.ctl->wnorm0 = (double)wsqrt(wn0sq);
        __threadfence();
        __syncthreads();
        givens_step(c, ncols - 1, c.h1, hnext);
    }
}

}  // namespace gmres
