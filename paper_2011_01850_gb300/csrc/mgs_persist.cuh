// mgs_persist.cuh -- procedure MGS of Algorithm 1 (arXiv 2011.01850) for one
// inner step as a single cooperative kernel.
//
// MGS needs the inner product h_i = w . v_i of the already-updated w before it
// can project v_i out, so an inner step of j basis vectors has j global
// reductions in sequence.  Here every block keeps its row chunk of w in shared
// memory for the whole step; per basis vector it makes one sweep over its
// rows that applies the previous projection (w <- w - h_{i-1} v_{i-1}) and
// accumulates w . v_i, then takes part in one exchange round: it publishes
// its partial with a release flag and sums every block's partial in block
// order as the flags arrive (so all blocks see the same h_i, bit for bit;
// the flags are the only synchronisation, no separate barrier).  The last
// sweep applies the final projection and takes ||w||; the blocks then write
// v_{j+1} = w / h_{j+1,j} straight into the basis and block 0 runs the
// Givens step.  w never goes back to global memory and the basis is read once
// from HBM per step (the previous vector comes back from L1/L2).
//
// The grid is launched cooperatively (all blocks resident).  Every wait is
// bounded: after `spin` polls the block records a timeout in the control
// block, the other blocks see it at their next poll, and all return.
#pragma once

#include "grid_kernels.cuh"
#include "tma.cuh"

namespace gmres {

constexpr int MGSP_THREADS = 512;

constexpr int MGSP_MAXGRID = 256;  // exchange slots read by one warp: <= 8 per lane
constexpr int MGSP_QMAX = MGSP_MAXGRID / 32;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// One round of the grid-wide exchange that replaces "barrier, then sum the
// per-block partials".  It takes every thread's NV partials in v, sums them
// over the block (warp butterflies, then warp 0 over the warp sums) and
// exchanges the block sums; the round costs two block barriers.  `bad` is a
// thread's own failure (a copy wait that gave up): if any thread of the block
// has one, the block records a timeout in *err, publishes nothing and returns
// false.  Every block owns 4 words per parity p in `slots`.
// Thread 0 publishes the block's NV partials: for binary32 each word holds
// (round << 32 | value bits), so one 64-bit store publishes a value together
// with its round; for binary64 the values go first and a release store of
// the round into word 3 follows.  Warp 0 of every block polls the words of
// all blocks at once (lane l takes blocks l, l+32, ...; every poll issues all
// of a lane's loads together), and once every block has published the round
// sums the values in block order (per lane, then an xor butterfly, so every
// block gets the same sums bit for bit) and broadcasts them.  A block may
// overwrite its words of parity p only after it has seen every block publish
// the round in between, which every block does only after reading round
// k-2's values, so two parities suffice.  Round numbers grow across launches
// and never repeat (the host clears the slots before they wrap), so a stale
// word never matches.  Returns false in every thread of the block when a
// wait gave up after `limit` polls or another block reported a timeout in
// *err.
template <class T, int NV>
__device__ __forceinline__ bool exchange_round(unsigned long long *slots, int p, unsigned round,
                                               T (&v)[NV], T (&out)[NV], int *err,
                                               long long limit, T *sred, T *sbuf, bool bad) {
    constexpr bool F32 = sizeof(T) == 4;
    const int G = (int)gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            sred[k * 32 + wid] = v[k];
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0)
            atomicExch(err, 1);
        return false;
    }
    if (threadIdx.x < 32) {
        T mine[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            mine[k] = warp_sum(lane < nw ? sred[k * 32 + lane] : T(0));
        if (lane == 0) {
            unsigned long long *my = slots + ((size_t)blockIdx.x * 2 + p) * 4;
            if constexpr (F32) {
#pragma unroll
                for (int k = 0; k < NV; ++k)
                    st_relaxed_u64(my + k, ((unsigned long long)round << 32) |
                                               (unsigned long long)__float_as_uint((float)mine[k]));
            } else {
#pragma unroll
                for (int k = 0; k < NV; ++k)
                    st_relaxed_u64(my + k,
                                   (unsigned long long)__double_as_longlong((double)mine[k]));
                st_release_u64(my + 3, (unsigned long long)round);
            }
        }
        unsigned long long w[MGSP_QMAX][NV];
        bool ok = true;
        long long it = 0;
        for (;;) {
            bool ready = true;
            // the timeout word is loaded with the slots, not after them, so
            // a poll costs one round trip to L2
            const int e = *(volatile int *)err;
#pragma unroll
            for (int q = 0; q < MGSP_QMAX; ++q) {
                const int b = lane + 32 * q;
                if (b < G) {
                    const unsigned long long *ws = slots + ((size_t)b * 2 + p) * 4;
                    if constexpr (F32) {
#pragma unroll
                        for (int k = 0; k < NV; ++k) {
                            w[q][k] = ld_relaxed_u64(ws + k);
                            ready = ready && (unsigned)(w[q][k] >> 32) == round;
                        }
                    } else {
                        ready = ready && (unsigned)ld_relaxed_u64(ws + 3) == round;
                    }
                }
            }
            if (__all_sync(0xffffffffu, ready))
                break;
            if (e != 0 || ++it > limit) {
                ok = false;
                break;
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        T acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            acc[k] = 0;
        if (ok) {
            if constexpr (!F32)
                fence_acq_rel_gpu();
#pragma unroll
            for (int q = 0; q < MGSP_QMAX; ++q) {
                const int b = lane + 32 * q;
                if (b < G) {
#pragma unroll
                    for (int k = 0; k < NV; ++k) {
                        if constexpr (F32)
                            acc[k] += (T)__uint_as_float((unsigned)(w[q][k] & 0xffffffffull));
                        else
                            acc[k] += (T)__longlong_as_double((long long)ld_relaxed_u64(
                                slots + ((size_t)b * 2 + p) * 4 + k));
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NV; ++k)
            acc[k] = warp_sum(acc[k]);
        if (lane == 0) {
            if (!ok)
                atomicExch(err, 1);
#pragma unroll
            for (int k = 0; k < NV; ++k)
                sbuf[k] = acc[k];
            sbuf[NV] = ok ? T(1) : T(0);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k)
        out[k] = sbuf[k];
    return sbuf[NV] != T(0);
}

// PVS: the per-variable study's instantiation (every updated entry of w under
// PV_W, the coefficients and h_{j+1,j} under PV_H stored in binary32); the
// default loops carry none of it.
template <class T, class VT, bool PVS = false>
__global__ void __launch_bounds__(MGSP_THREADS, 1)
    k_mgs_persist(GridCtx<T, VT> c, int ncols, int64_t chunk, long long spin,
                  unsigned long long *slots, unsigned round0) {
    if (!c.ctl->active)
        return;
    extern __shared__ __align__(16) unsigned char mgs_smem[];
    T *ws = reinterpret_cast<T *>(mgs_smem);
    __shared__ T sred[2 * 32];
    __shared__ T sx[3];
    __shared__ T hcol[MMAX + 2];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk;
    int64_t re = rb + chunk;
    if (re > c.ldv)
        re = c.ldv;
    const int64_t len = re > rb ? re - rb : 0;
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
    T hprev, wn0sq;
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
        T tot[2];
        if (!exchange_round<T, 2>(slots, 0, round0, acc, tot, err, spin, sred, sx, false))
            return;
        hprev = PVS ? pv_round(tot[0], c.pv, PV_H) : tot[0];
        wn0sq = tot[1];
    }
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
                if (PVS)
                    wv = pv_round(wv, c.pv, PV_W);
                ws[q + k] = wv;
                d += wv * b[k];
            }
        }
        T dv[1] = {d}, hv[1];
        if (!exchange_round<T, 1>(slots, i & 1, round0 + (unsigned)i, dv, hv, err, spin, sred,
                                  sx, false))
            return;
        hprev = PVS ? pv_round(hv[0], c.pv, PV_H) : hv[0];
        if (tid == 0)
            hcol[i] = hprev;
    }
    // last projection and ||w||^2
    T hnext;
    {
        const VT *vp = c.V + (size_t)(ncols - 1) * c.ldv + rb;
        T nsq = 0;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T a[4];
            ld4<T, VT>(vp + q, c.vinv, a);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T wv = ws[q + k] - hprev * a[k];
                if (PVS)
                    wv = pv_round(wv, c.pv, PV_W);
                ws[q + k] = wv;
                nsq += wv * wv;
            }
        }
        T nv[1] = {nsq}, tv[1];
        if (!exchange_round<T, 1>(slots, ncols & 1, round0 + (unsigned)ncols, nv, tv, err,
                                  spin, sred, sx, false))
            return;
        hnext = wsqrt(tv[0]);
        if (PVS)
            hnext = pv_round(hnext, c.pv, PV_H);
    }
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
        givens_step<PVS>(c, ncols - 1, c.h1, hnext);
    }
}

// The same MGS step with the block's rows of the basis staged in shared
// memory: a ring of three row-chunk buffers filled by bulk copies one basis
// vector ahead, so the copy of v_{i+1} is in flight while the block sweeps
// with v_{i-1}, v_i and waits in exchange round i; every sweep then reads
// shared memory only (w stays there too).  Same arithmetic, same order as
// k_mgs_persist, so the two give the same results bit for bit.  Needs
// chunk (sizeof(T) + 3 sizeof(VT)) + MGSS_HEAD bytes of shared memory, chunk a
// multiple of 8 (bulk copies of whole 16-byte units from 16-byte aligned
// rows).  A bulk copy that does not complete within `spin` probes is a
// timeout: the block reports it, waits (bounded) for its other copies in
// flight and returns, like every other block at its next exchange round.
constexpr int MGSS_HEAD = 64;  // three mbarriers, padded to keep the data 16-byte aligned

template <class T, class VT, bool PVS = false>
__global__ void __launch_bounds__(MGSP_THREADS, 1)
    k_mgs_staged(GridCtx<T, VT> c, int ncols, int64_t chunk, long long spin,
                 unsigned long long *slots, unsigned round0) {
    if (!c.ctl->active)
        return;
    extern __shared__ __align__(128) unsigned char mgss_smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(mgss_smem);
    T *ws = reinterpret_cast<T *>(mgss_smem + MGSS_HEAD);
    VT *vbuf = reinterpret_cast<VT *>(mgss_smem + MGSS_HEAD + (size_t)chunk * sizeof(T));
    __shared__ T sred[2 * 32];
    __shared__ T sx[3];
    __shared__ T hcol[MMAX + 2];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t rb = (int64_t)blockIdx.x * chunk;
    int64_t re = rb + chunk;
    if (re > c.ldv)
        re = c.ldv;
    const int64_t len = re > rb ? re - rb : 0;
    const uint32_t vbytes = (uint32_t)(len * (int64_t)sizeof(VT));
    int *err = &c.ctl->timeout;
    if (tid == 0) {
        for (int k = 0; k < 3; ++k)
            mbar_init(&bars[k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // a bulk copy completes unless the GPU faults: its waits get their own
    // generous bound, independent of `spin` (the bound of the exchange waits,
    // which may be set low to force a timeout), so that a block never leaves
    // while a copy of its own is still writing its shared memory
    const long long climit = spin > (1LL << 22) ? spin : (1LL << 22);
    // basis column `col` into ring buffer col % 3 (thread 0)
    int issued = 0, waited = 0;  // columns issued / waited for (same in every thread)
    auto issue = [&](int col) {
        if (len > 0 && tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&bars[col % 3], vbytes);
            bulk_g2s(vbuf + (size_t)(col % 3) * chunk, c.V + (size_t)col * c.ldv + rb, vbytes,
                     &bars[col % 3]);
        }
        ++issued;
    };
    // wait for column `col`; false in this thread on a timeout.  No barrier:
    // a thread whose wait gave up still sweeps its (in-bounds) rows, and the
    // block learns of it at the next exchange round, which then fails
    auto wait = [&](int col) -> bool {
        bool ok = true;
        if (len > 0)
            ok = mbar_wait(&bars[col % 3], (uint32_t)((col / 3) & 1), climit);
        ++waited;
        return ok;
    };
    // on the way out: let every copy still in flight land (bounded) before
    // the block's shared memory is released
    auto drain = [&]() {
        for (int col = waited; col < issued; ++col)
            if (len > 0)
                mbar_wait(&bars[col % 3], (uint32_t)((col / 3) & 1), climit);
    };
    auto vb = [&](int col) -> const VT * { return vbuf + (size_t)(col % 3) * chunk; };

    issue(0);
    if (ncols > 1)
        issue(1);
    for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
        T v[4];
        ldv4(c.w + rb + q, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            ws[q + k] = v[k];
    }
    const bool got0 = wait(0);
    // h_0 = w . v_0 and ||w||^2 (breakdown reference)
    T hprev, wn0sq;
    {
        T acc[2] = {0, 0};
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T v[4];
            ld4<T, VT>(vb(0) + q, c.vinv, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                acc[0] += ws[q + k] * v[k];
                acc[1] += ws[q + k] * ws[q + k];
            }
        }
        T tot[2];
        if (!exchange_round<T, 2>(slots, 0, round0, acc, tot, err, spin, sred, sx, !got0)) {
            drain();
            return;
        }
        hprev = PVS ? pv_round(tot[0], c.pv, PV_H) : tot[0];
        wn0sq = tot[1];
    }
    if (tid == 0)
        hcol[0] = hprev;
    for (int i = 1; i < ncols; ++i) {
        if (i + 1 < ncols)
            issue(i + 1);  // its buffer last held v_{i-2}, read before round i-1 ended
        const bool got = wait(i);
        const VT *vp = vb(i - 1);
        const VT *vi = vb(i);
        T d = 0;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T a[4], b[4];
            ld4<T, VT>(vp + q, c.vinv, a);
            ld4<T, VT>(vi + q, c.vinv, b);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T wv = ws[q + k] - hprev * a[k];
                if (PVS)
                    wv = pv_round(wv, c.pv, PV_W);
                ws[q + k] = wv;
                d += wv * b[k];
            }
        }
        T dv[1] = {d}, hv[1];
        if (!exchange_round<T, 1>(slots, i & 1, round0 + (unsigned)i, dv, hv, err, spin, sred,
                                  sx, !got)) {
            drain();
            return;
        }
        hprev = PVS ? pv_round(hv[0], c.pv, PV_H) : hv[0];
        if (tid == 0)
            hcol[i] = hprev;
    }
    // last projection and ||w||^2
    T hnext;
    {
        const VT *vp = vb(ncols - 1);
        T nsq = 0;
        for (int64_t q = 4 * tid; q < len; q += 4 * nth) {
            T a[4];
            ld4<T, VT>(vp + q, c.vinv, a);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T wv = ws[q + k] - hprev * a[k];
                if (PVS)
                    wv = pv_round(wv, c.pv, PV_W);
                ws[q + k] = wv;
                nsq += wv * wv;
            }
        }
        T nv[1] = {nsq}, tv[1];
        if (!exchange_round<T, 1>(slots, ncols & 1, round0 + (unsigned)ncols, nv, tv, err,
                                  spin, sred, sx, false))
            return;
        hnext = wsqrt(tv[0]);
        if (PVS)
            hnext = pv_round(hnext, c.pv, PV_H);
    }
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
        givens_step<PVS>(c, ncols - 1, c.h1, hnext);
    }
}

}  // namespace gmres
