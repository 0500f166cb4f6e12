// cgs_tile.cuh -- the three passes of CGSR (procedure CGSR of Algorithm 1,
// done twice; arXiv 2011.01850) as one tiled, TMA-fed kernel family.
//
//   MODE 0  h1 = V^T w                       (+ ||w||, the breakdown reference)
//   MODE 1  w <- w - V h1, then h2 = V^T w   (one read of V: the row tile of all
//                                             j basis vectors sits in shared
//                                             memory for both steps)
//   MODE 2  w <- w - V h2, ||w||^2 -> h_{j+1,j}, column h1 + h2, Givens step
//
// A persistent grid (one block per SM) walks row tiles of TR rows.  Thread 0
// streams each tile -- the TR-row segment of every basis vector plus the
// matching segment of w -- into one of S shared-memory stages with bulk
// copies completing on that stage's mbarrier, S-1 tiles ahead of the compute.
// Dot products accumulate per thread across all of a block's tiles and are
// reduced once at the end (block, then grid through the last block), so the
// inner loop has no barrier but the per-tile stage hand-off.
#pragma once

#include "grid_kernels.cuh"
#include "tma.cuh"

namespace gmres {

constexpr int CGS_THREADS = 256;
constexpr int CGS_STAGES = 3;
constexpr int CGS_TR_MAX = 2048;
constexpr int CGS_WARPS = CGS_THREADS / 32;
constexpr int CGS_COLS_PER_WARP = (MMAX + 1 + CGS_WARPS - 1) / CGS_WARPS;

__host__ __device__ inline size_t align128(size_t v) { return (v + 127) & ~(size_t)127; }

template <class T, class VT>
__host__ __device__ inline size_t cgs_stage_bytes(int ncols, int TR) {
    return align128((size_t)ncols * TR * sizeof(VT)) + align128((size_t)TR * sizeof(T));
}

// Shared-memory bytes of k_cgs_tile for ncols basis vectors and TR-row tiles.
template <class T, class VT>
__host__ __device__ inline size_t cgs_smem_bytes(int ncols, int TR) {
    return 128                                            // mbarriers
           + align128((MMAX + 2) * sizeof(T))             // projections h
           + align128(CGS_THREADS * sizeof(T))            // column-split partial rows
           + align128((size_t)TR * sizeof(T))             // updated w tile
           + CGS_STAGES * cgs_stage_bytes<T, VT>(ncols, TR);
}

// Tile height: the largest power of two in [32, 2048] whose basis tile stays
// within ~48 KB, so S stages keep ~100-150 KB in flight per SM.
template <class VT>
inline int cgs_choose_tr(int ncols) {
    int tr = CGS_TR_MAX;
    while (tr > 32 && (size_t)tr * ncols * sizeof(VT) > 48 * 1024)
        tr >>= 1;
    return tr;
}

template <class T, class VT, int MODE>
__global__ void __launch_bounds__(CGS_THREADS, 1)
    k_cgs_tile(GridCtx<T, VT> c, int ncols, int TR, long long spin_limit) {
    if (!c.ctl->active)
        return;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *p = smem + 128;
    T *hs = reinterpret_cast<T *>(p);
    p += align128((MMAX + 2) * sizeof(T));
    T *red = reinterpret_cast<T *>(p);
    p += align128(CGS_THREADS * sizeof(T));
    T *wn = reinterpret_cast<T *>(p);
    p += align128((size_t)TR * sizeof(T));
    unsigned char *stage0 = p;
    const size_t sb = cgs_stage_bytes<T, VT>(ncols, TR);
    const size_t vbytes_tile = align128((size_t)ncols * TR * sizeof(VT));
    const uint32_t copy_v = (uint32_t)(TR * sizeof(VT));
    const uint32_t copy_w = (uint32_t)(TR * sizeof(T));
    const uint32_t tx = copy_v * ncols + copy_w;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = c.ldv / TR;
    const int64_t my_tiles = (blockIdx.x < ntiles) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (MODE >= 1) {
        const T *src = (MODE == 1) ? c.h1 : c.h2;
        for (int i = tid; i < ncols; i += CGS_THREADS)
            hs[i] = src[i];
    }
    if (tid == 0) {
        for (int s = 0; s < CGS_STAGES; ++s)
            mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int64_t k) {
        const int s = (int)(k % CGS_STAGES);
        const int64_t t = blockIdx.x + k * gridDim.x;
        unsigned char *st = stage0 + s * sb;
        mbar_arrive_expect_tx(&bars[s], tx);
        const int64_t row0 = t * TR;
        for (int col = 0; col < ncols; ++col)
            bulk_g2s(st + (size_t)col * copy_v, c.V + (size_t)col * c.ldv + row0, copy_v,
                     &bars[s]);
        bulk_g2s(st + vbytes_tile, c.w + row0, copy_w, &bars[s]);
    };
    if (tid == 0) {
        for (int64_t k = 0; k < CGS_STAGES && k < my_tiles; ++k)
            issue(k);
    }

    // Step-1 mapping (update): NSPLIT column groups share each row.
    const int nsplit = TR >= CGS_THREADS ? 1 : CGS_THREADS / TR;
    const int tps = CGS_THREADS / nsplit;
    const int split = tid / tps, slot = tid % tps;
    const int rpt = TR >= CGS_THREADS ? TR / CGS_THREADS : 1;

    T acc[CGS_COLS_PER_WARP];
#pragma unroll
    for (int k = 0; k < CGS_COLS_PER_WARP; ++k)
        acc[k] = 0;
    T nsq = 0;
    bool timed_out = false;
    int64_t kbreak = 0;

    for (int64_t k = 0; k < my_tiles; ++k) {
        const int s = (int)(k % CGS_STAGES);
        const uint32_t parity = (uint32_t)((k / CGS_STAGES) & 1);
        // every thread waits (bounded); the give-up decision is block-uniform
        const bool ok = mbar_wait(&bars[s], parity, spin_limit);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            kbreak = k;
            break;
        }
        const int64_t t = blockIdx.x + k * gridDim.x;
        const VT *Vs = reinterpret_cast<const VT *>(stage0 + s * sb);
        const T *Ws = reinterpret_cast<const T *>(stage0 + s * sb + vbytes_tile);
        const T *dsrc = Ws;  // vector the dots use
        if (MODE >= 1) {
            // w' = w - V h  (rows of this tile)
            for (int q = 0; q < rpt; ++q) {
                const int r = slot + q * tps;
                T a = 0;
                for (int col = split; col < ncols; col += nsplit)
                    a += (T)Basis<VT>::ld(Vs + (size_t)col * TR + r, c.vinv) * hs[col];
                if (nsplit > 1)
                    red[split * TR + r] = a;
                else {
                    T v = Ws[r] - a;
                    wn[r] = v;
                    c.w[t * TR + r] = v;
                    nsq += v * v;
                }
            }
            if (nsplit > 1) {
                __syncthreads();
                if (split == 0) {
                    const int r = slot;
                    T a = 0;
                    for (int g = 0; g < nsplit; ++g)
                        a += red[g * TR + r];
                    T v = Ws[r] - a;
                    wn[r] = v;
                    c.w[t * TR + r] = v;
                    nsq += v * v;
                }
            }
            dsrc = wn;
            if (MODE == 1)
                __syncthreads();
        }
        if (MODE <= 1) {
            // dots with every basis vector: warp wid owns columns wid + 8 kk
#pragma unroll
            for (int kk = 0; kk < CGS_COLS_PER_WARP; ++kk) {
                const int col = wid + CGS_WARPS * kk;
                if (col < ncols) {
                    const VT *vc = Vs + (size_t)col * TR;
                    T a = 0;
                    for (int r = lane; r < TR; r += 32)
                        a += (T)Basis<VT>::ld(vc + r, c.vinv) * dsrc[r];
                    acc[kk] += a;
                }
            }
            if (MODE == 0 && wid == 0) {
                for (int r = lane; r < TR; r += 32)
                    nsq += dsrc[r] * dsrc[r];
            }
        }
        __syncthreads();  // stage s fully consumed
        if (tid == 0 && k + CGS_STAGES < my_tiles)
            issue(k + CGS_STAGES);
    }
    if (__syncthreads_or(timed_out)) {
        // Before the block's shared memory goes away, let every bulk copy it
        // issued land: wait (with its own bound) on each stage that was
        // issued and not yet consumed, then report the timeout.
        // Tiles 0 .. kbreak-1 were consumed; tiles kbreak .. kbreak+S-1 (within
        // the block's count) were issued and may still be in flight.
        if (tid == 0) {
            const long long drain = 1LL << 26;
            const int64_t issued = my_tiles < kbreak + CGS_STAGES ? my_tiles
                                                                  : kbreak + CGS_STAGES;
            for (int64_t k = kbreak; k < issued; ++k)
                mbar_wait(&bars[k % CGS_STAGES], (uint32_t)((k / CGS_STAGES) & 1), drain);
            atomicExch(&c.ctl->timeout, 1);
        }
        __syncthreads();
        return;
    }

    // block partials
    T *mypart = c.part + (size_t)blockIdx.x * PSTRIDE;
    if (MODE <= 1) {
#pragma unroll
        for (int kk = 0; kk < CGS_COLS_PER_WARP; ++kk) {
            const int col = wid + CGS_WARPS * kk;
            T v = warp_sum(acc[kk]);
            if (lane == 0 && col < ncols)
                mypart[col] = v;
        }
    }
    if (MODE != 1) {
        __shared__ T sred[32];
        T tot = block_sum1(nsq, sred);
        if (tid == 0)
            mypart[MMAX + 1] = tot;
    }
    const int slot_ctr = MODE + 1;
    if (!arrive_last(&c.ctl->counter[slot_ctr]))
        return;
    __shared__ T snorm;
    if (MODE == 0) {
        reduce_columns(c.part, gridDim.x, ncols, c.h1);
        reduce_columns(c.part + MMAX + 1, gridDim.x, 1, &snorm);
        __syncthreads();
        if (tid == 0)
            c.ctl->wnorm0 = (double)wsqrt(snorm);
    } else if (MODE == 1) {
        reduce_columns(c.part, gridDim.x, ncols, c.h2);
    } else {
        reduce_columns(c.part + MMAX + 1, gridDim.x, 1, &snorm);
        for (int i = tid; i < ncols; i += blockDim.x)
            c.h1[i] = ldcg(c.h1 + i) + ldcg(c.h2 + i);
        __threadfence();
        __syncthreads();
        givens_step(c, ncols - 1, c.h1, wsqrt(snorm));
    }
}

}  // namespace gmres
