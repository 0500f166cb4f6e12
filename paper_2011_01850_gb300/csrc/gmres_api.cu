// gmres_api.cu -- C-ABI of the GB300 mixed-precision restarted GMRES(m)
// library (declarations and contracts in include/gmres_gb300.h).
//
// Host side of Algorithm 1 of arXiv 2011.01850: it owns the device copies of
// A (binary64 values, binary32 values, shared int32 indices; Sec. 4), the
// workspace, and the per-cycle driver that enqueues the restart cycle's
// kernels on the handle's stream.  The host reads the device control block
// once per restart cycle; all arithmetic runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "../../include/gmres_gb300.h"
#include "block_solver.cuh"
#include "cgs_rows.cuh"
#include "mgs_persist.cuh"
#include "grid_kernels.cuh"
#include "orth_monitor.cuh"
#include "team_launch.hpp"
#include "ilu.hpp"
#include "handle.hpp"
#include "host_util.hpp"
#include "sell.hpp"

using namespace gmres;
using namespace gmres_host;

namespace {
constexpr int kThreads = 256;
static_assert(GMRES_PV_A_KRYLOV == PV_A_KRYLOV && GMRES_PV_M == PV_M && GMRES_PV_V == PV_V &&
                  GMRES_PV_W == PV_W && GMRES_PV_H == PV_H && GMRES_PV_GIVENS == PV_GIVENS &&
                  GMRES_PV_Z == PV_Z && GMRES_PV_A_RESID == PV_A_RESID && GMRES_PV_B == PV_B &&
                  GMRES_PV_X == PV_X && GMRES_PV_AX == PV_AX,
              "per-variable switch bits of the C-ABI and the kernels");
}  // namespace

namespace {

// max over i of |v_i| (or of the absolute row sums of A when rowptr is
// given): non-negative binary64 values order like their bit patterns, so an
// integer atomicMax gives the exact maximum in any order.
__global__ void __launch_bounds__(256) k_absmax(int n, const double *v, const int *rowptr,
                                                const unsigned *hi, const unsigned *lo,
                                                unsigned long long *out) {
    __shared__ unsigned long long sm;
    if (threadIdx.x == 0)
        sm = 0ull;
    __syncthreads();
    unsigned long long best = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a = 0.0;
        if (rowptr) {
            for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
                a += fabs(hi ? __hiloint2double((int)hi[k], (int)lo[k]) : v[k]);
        } else {
            a = fabs(v[i]);
        }
        const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
        best = bits > best ? bits : best;
    }
    atomicMax(&sm, best);
    __syncthreads();
    if (threadIdx.x == 0)
        atomicMax(out, sm);
}

__global__ void k_cast_vals(int64_t nnz, const double *a, float *b) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

// Split storage: the high- and low-order 32 bits of each binary64 value.
__global__ void __launch_bounds__(256) k_split_vals(int64_t nnz, const double *v, unsigned *hi,
                                                    unsigned *lo) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double a = v[k];
        hi[k] = (unsigned)__double2hiint(a);
        lo[k] = (unsigned)__double2loint(a);
    }
}

// Per-precision device pointers into the "small" buffer.
template <class T>
struct SmallPtrs {
    T *H, *Hb, *s, *cs, *sn, *y, *h1, *h2;
};

// The learned right preconditioner / the ILU(0) left preconditioner is on.
inline bool spai_on(const gmres_handle *h) { return h->has_precond && h->opts.precond == 1; }
inline bool ilu_on(const gmres_handle *h) { return h->ilu_ok && h->opts.precond == 2; }

inline const unsigned *split_hi(gmres_handle *h) { return h->vals64.as<unsigned>(); }
inline const unsigned *split_lo(gmres_handle *h) { return h->vals64.as<unsigned>() + h->nnz; }

// Restart-test buffers (binary64): |s_{j+1}| history of the cycle, ||S_k||
// history, then U and S of the loss-of-orthogonality test.
inline double *mon_ahist(gmres_handle *h) { return h->mon.as<double>(); }
inline double *mon_hist(gmres_handle *h) { return h->mon.as<double>() + (MMAX + 2); }
constexpr size_t MON_DOUBLES = 2 * (MMAX + 2) + 2 * (size_t)(MMAX + 1) * (MMAX + 1);

template <class T>
SmallPtrs<T> small_ptrs(gmres_handle *h) {
    const int ld = MMAX + 1;
    T *base = h->small.as<T>();
    SmallPtrs<T> p;
    p.H = base;
    p.Hb = p.H + (size_t)ld * MMAX;
    p.s = p.Hb + (size_t)ld * MMAX;
    p.cs = p.s + (MMAX + 2);
    p.sn = p.cs + (MMAX + 2);
    p.y = p.sn + (MMAX + 2);
    p.h1 = p.y + (MMAX + 2);
    p.h2 = p.h1 + (MMAX + 2);
    return p;
}

gmres_status ensure_workspace(gmres_handle *h, int m, gmres_precision prec) {
    const size_t sv = (size_t)elem_bytes(prec);
    const size_t ldv = (size_t)h->ldv;
    // The basis, padded vectors and the binary64 buffers; tails stay zero.
    size_t vbytes = ldv * (size_t)(m + 1) * sv;
    bool vgrow = vbytes > h->V.bytes;
    CK(h->V.ensure(vbytes));
    if (vgrow)
        CK(cudaMemsetAsync(h->V.p, 0, h->V.bytes, h->stream));
    // the work vectors' padding rows must read as zero in the working type:
    // clear them when the working type changes (a binary64 solve leaves
    // nonzero bytes where a binary32 view has its padding)
    const int tbytes = (prec == GMRES_FP64 || prec == GMRES_MIXED_LIMITED) ? 8 : 4;
    if (h->work_elem != 0 && h->work_elem != tbytes) {
        for (DevBuf *b : {&h->w, &h->r, &h->t, &h->t2})
            if (b->p)
                CK(cudaMemsetAsync(b->p, 0, b->bytes, h->stream));
    }
    h->work_elem = tbytes;
    for (DevBuf *b : {&h->w, &h->r, &h->t}) {
        bool grow = ldv * 8 > b->bytes;
        CK(b->ensure(ldv * 8));
        if (grow)
            CK(cudaMemsetAsync(b->p, 0, b->bytes, h->stream));
    }
    CK(h->z.ensure(ldv * 8));
    CK(h->xb.ensure(ldv * 8));
    CK(h->bb.ensure(ldv * 8));
    CK(h->small.ensure((size_t)(2 * (MMAX + 1) * MMAX + 6 * (MMAX + 2)) * 8));
    CK(h->part.ensure((size_t)std::max(h->grid, h->nsm * h->rows_blocks_per_sm) * PSTRIDE * 8));
    // binary64 partials: the reduction kernels (grid blocks) and the
    // residual, which runs on the SpMV's grid (8 blocks per SM)
    CK(h->part64.ensure((size_t)std::max(h->grid, h->nsm * 8) * 4 * 8));
    if (ilu_on(h))
        CK(h->t2.ensure(ldv * 8));
    if (ilu_on(h))
        CK(h->t2.ensure(ldv * 8));
    if (h->mon.bytes < MON_DOUBLES * sizeof(double)) {
        CK(h->mon.ensure(MON_DOUBLES * sizeof(double)));
        CK(cudaMemsetAsync(h->mon.p, 0, h->mon.bytes, h->stream));
    }
    bool cgrow = sizeof(Ctl) > h->ctl.bytes;
    CK(h->ctl.ensure(sizeof(Ctl)));
    if (cgrow)
        CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
    if (!h->hctl) {
        void *p = nullptr;
        CK(cudaMallocHost(&p, sizeof(Ctl)));
        h->hctl = reinterpret_cast<Ctl *>(p);
    }
    return GMRES_OK;
}

// Storage the product with A reads: 1 / 2 = the sliced copy (16-bit / 32-bit
// columns), 0 = CSR.  `step`: for the Krylov step of a running solve, where
// the limited form and the per-variable binary32 A read CSR.
template <class T>
int sell_fmt_for(const gmres_handle *h, bool step) {
    if (!h->sell_fmt || h->split || h->opts.spmv_format == GMRES_SPMV_CSR)
        return 0;
    if (h->opts.spmv_format == GMRES_SPMV_AUTO &&
        !(std::is_same<T, double>::value ? h->sell64 : h->sell32))
        return 0;
    if (step && (h->limited || (std::is_same<T, double>::value &&
                                (h->opts.pv_mask & GMRES_PV_A_KRYLOV))))
        return 0;
    return h->sell_fmt;
}

template <class T, class VT>
GridCtx<T, VT> make_ctx(gmres_handle *h, int m) {
    GridCtx<T, VT> c;
    memset(&c, 0, sizeof(c));
    c.n = h->n;
    c.m = m;
    c.ld = m + 1;
    c.ldv = h->ldv;
    c.chunk = h->chunk;
    c.rowptr = h->rowptr.as<int>();
    c.colind = h->colind.as<int>();
    c.a = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->vals64.p)
                                         : reinterpret_cast<const T *>(h->vals32.p);
    c.a64 = h->vals64.as<double>();
    c.V = h->V.as<VT>();
    c.vscale = std::is_same<VT, __half>::value ? fp16_scale(h->n) : 1.0f;
    c.vinv = 1.0f / c.vscale;
    c.w = h->w.as<T>();
    c.r = h->r.as<T>();
    c.t = h->t.as<T>();
    SmallPtrs<T> sp = small_ptrs<T>(h);
    c.H = sp.H;
    c.Hb = sp.Hb;
    c.s = sp.s;
    c.cs = sp.cs;
    c.sn = sp.sn;
    c.y = sp.y;
    c.h1 = sp.h1;
    c.h2 = sp.h2;
    c.part = h->part.as<T>();
    c.part64 = h->part64.as<double>();
    c.ctl = h->ctl.as<Ctl>();
    c.brk = std::is_same<T, double>::value ? T(1e-14) : T(1e-6);
    c.kmax = m;
    c.ahist = mon_ahist(h);
    c.stall_factor = h->opts.stall_factor;
    c.stall_w = h->opts.stall_window > 0 ? h->opts.stall_window : (m + 19) / 20;
    if (h->split) {
        c.a = nullptr;
        c.a64 = nullptr;
        c.ahi = split_hi(h);
        c.alo = split_lo(h);
        c.aform = (std::is_same<T, double>::value && !h->limited) ? 3 : 2;
    } else if (h->limited) {
        c.a_lim = h->vals32.as<float>();
        c.aform = 1;
    }
    c.left = ilu_on(h) ? 1 : 0;
    // per-variable precision study (binary64 solves only): A for the Krylov
    // step and M read from their binary32 copies in binary64 arithmetic, A
    // for the residual from the binary32 copy; the rest rounds in the kernels
    c.pv = (std::is_same<T, double>::value && !h->limited) ? (unsigned)h->opts.pv_mask : 0u;
    c.a_res32 = h->vals32.as<float>();
    if ((c.pv & PV_A_KRYLOV) && !h->split) {
        c.a_lim = h->vals32.as<float>();
        c.aform = 1;
    }
    if (spai_on(h)) {
        c.prowptr = c.rowptr;
        c.pcolind = c.colind;
        c.pvals = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->pvals64.p)
                                                 : reinterpret_cast<const T *>(h->pvals32.p);
        if (h->limited || (c.pv & PV_M))
            c.pvals_lim = h->pvals32.as<float>();
    }
    c.sfmt = c.aform == 0 ? sell_fmt_for<T>(h, true) : 0;
    if (c.sfmt) {
        c.sptr = h->sptr.as<int>();
        c.slen = h->slen.as<unsigned short>();
        c.scol = h->scol.p;
        c.sval = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->sval64.p)
                                                : reinterpret_cast<const T *>(h->sval32.p);
    }
    return c;
}

int spmv_grid(gmres_handle *h) { return h->nsm * 8; }

// v_1 and the update x += V_j y run 8 blocks per SM, like the SpMV, with the
// row chunk to match: more bytes in flight per SM than the reduction
// kernels' 2 (the update at 160^3: 7.1 -> 6.4 ms per solve; the
// normalisation gained nothing, a ~10 us kernel bound by its ramp, and keeps
// the 2-block grid).
template <class T, class VT>
GridCtx<T, VT> stream_ctx(const gmres_handle *h, const GridCtx<T, VT> &c, int *grid) {
    GridCtx<T, VT> s = c;
    *grid = h->nsm * 8;
    s.chunk = round_up((h->ldv + *grid - 1) / *grid, 4);
    return s;
}

// Launch helpers templated on the lanes-per-row count.
template <class T, class VT, class XT>
cudaError_t launch_spmv_step(gmres_handle *h, const GridCtx<T, VT> &c, const XT *x, T *y, int L) {
    dim3 g(spmv_grid(h)), b(kThreads);
    if (c.sfmt == 1) {
        k_spmv_step_sell<T, VT, XT, SellCol16><<<g, b, 0, h->stream>>>(c, x, y);
        return cudaGetLastError();
    }
    if (c.sfmt == 2) {
        k_spmv_step_sell<T, VT, XT, SellCol32><<<g, b, 0, h->stream>>>(c, x, y);
        return cudaGetLastError();
    }
    switch (L) {
    case 1: k_spmv_step<T, VT, XT, 1><<<g, b, 0, h->stream>>>(c, x, y); break;
    case 2: k_spmv_step<T, VT, XT, 2><<<g, b, 0, h->stream>>>(c, x, y); break;
    case 4: k_spmv_step<T, VT, XT, 4><<<g, b, 0, h->stream>>>(c, x, y); break;
    case 8: k_spmv_step<T, VT, XT, 8><<<g, b, 0, h->stream>>>(c, x, y); break;
    case 16: k_spmv_step<T, VT, XT, 16><<<g, b, 0, h->stream>>>(c, x, y); break;
    default: k_spmv_step<T, VT, XT, 32><<<g, b, 0, h->stream>>>(c, x, y); break;
    }
    return cudaGetLastError();
}

// z = b - A x gathers x like the SpMV, so it gets the SpMV's grid (more warps
// in flight per SM than the reduction kernels' two blocks).
template <class T, class VT>
cudaError_t launch_residual(gmres_handle *h, const GridCtx<T, VT> &c, const double *b,
                            const double *x, double *z, int setup) {
    dim3 g(h->nsm * 8), bl(kThreads);
    if constexpr (std::is_same<T, double>::value) {
        // the per-variable study's residual: its own instantiations
        if (c.pv & (PV_A_RESID | PV_B | PV_AX | PV_Z)) {
            switch (h->lanes64) {
            case 1: k_residual<T, VT, 1, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            case 2: k_residual<T, VT, 2, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            case 4: k_residual<T, VT, 4, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            case 8: k_residual<T, VT, 8, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            case 16: k_residual<T, VT, 16, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            default: k_residual<T, VT, 32, true><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
            }
            return cudaGetLastError();
        }
    }
    switch (h->lanes64) {
    case 1: k_residual<T, VT, 1><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    case 2: k_residual<T, VT, 2><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    case 4: k_residual<T, VT, 4><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    case 8: k_residual<T, VT, 8><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    case 16: k_residual<T, VT, 16><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    default: k_residual<T, VT, 32><<<g, bl, 0, h->stream>>>(c, b, x, z, setup); break;
    }
    return cudaGetLastError();
}

template <class T, class AT = T>
cudaError_t launch_spmv_plain(gmres_handle *h, int L, const AT *a, const T *x, T *y) {
    dim3 g(spmv_grid(h)), b(kThreads);
    const int *rp = h->rowptr.as<int>(), *ci = h->colind.as<int>();
    switch (L) {
    case 1: k_spmv_plain<T, AT, 1><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    case 2: k_spmv_plain<T, AT, 2><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    case 4: k_spmv_plain<T, AT, 4><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    case 8: k_spmv_plain<T, AT, 8><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    case 16: k_spmv_plain<T, AT, 16><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    default: k_spmv_plain<T, AT, 32><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
    }
    return cudaGetLastError();
}

// y = A x with split storage: the high part (binary32 work) or both parts.
template <class T>
cudaError_t launch_spmv_split(gmres_handle *h, int L, const T *x, T *y) {
    dim3 g(spmv_grid(h)), b(kThreads);
    const int *rp = h->rowptr.as<int>(), *ci = h->colind.as<int>();
    if (std::is_same<T, double>::value) {
        ValHiLo a{split_hi(h), split_lo(h)};
        switch (L) {
        case 1: k_spmv_plain_v<T, ValHiLo, 1><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 2: k_spmv_plain_v<T, ValHiLo, 2><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 4: k_spmv_plain_v<T, ValHiLo, 4><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 8: k_spmv_plain_v<T, ValHiLo, 8><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 16: k_spmv_plain_v<T, ValHiLo, 16><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        default: k_spmv_plain_v<T, ValHiLo, 32><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        }
    } else {
        ValHi a{split_hi(h)};
        switch (L) {
        case 1: k_spmv_plain_v<T, ValHi, 1><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 2: k_spmv_plain_v<T, ValHi, 2><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 4: k_spmv_plain_v<T, ValHi, 4><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 8: k_spmv_plain_v<T, ValHi, 8><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        case 16: k_spmv_plain_v<T, ValHi, 16><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        default: k_spmv_plain_v<T, ValHi, 32><<<g, b, 0, h->stream>>>(h->n, rp, ci, a, x, y); break;
        }
    }
    return cudaGetLastError();
}

// y = A x with the precision's copy of A, whatever the storage.
template <class T>
cudaError_t launch_spmv_any(gmres_handle *h, int L, const T *x, T *y) {
    if (h->split)
        return launch_spmv_split<T>(h, L, x, y);
    const T *a = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->vals64.p)
                                                : reinterpret_cast<const T *>(h->vals32.p);
    return launch_spmv_plain<T>(h, L, a, x, y);
}

struct Acct {
    double bytes[GMRES_K_COUNT] = {0};
    int64_t launches[GMRES_K_COUNT] = {0};
};

template <class T, class VT>
int lanes_for(gmres_handle *h) {
    int L = std::is_same<T, double>::value ? h->lanes64 : h->lanes32;
    if (h->opts.spmv_lanes > 0)
        L = h->opts.spmv_lanes;
    return L;
}

// Whether the cooperative MGS kernel can run: cooperative launches supported,
// one 512-thread block per SM resident with w's row chunk in shared memory.
template <class T, class VT>
bool mgs_persist_ok(gmres_handle *h) {
    // one entry per kernel instantiation (bfloat16 and binary16 bases have the
    // same sizes but are different kernels with their own attributes)
    const void *key = (const void *)k_mgs_persist<T, VT>;
    auto it = h->mgs_ok_cache.find(key);
    if (it != h->mgs_ok_cache.end())
        return it->second;
    bool ok = false;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (h->nsm > MGSP_MAXGRID)
        coop = 0;  // one warp reads every block's exchange slots
    // rows per block: a multiple of 8 (the staged kernel's bulk copies move
    // whole 16-byte units), the same for both kernels so they sum alike
    const int64_t chunk = round_up((h->ldv + h->nsm - 1) / h->nsm, 8);
    const size_t smem = (size_t)chunk * sizeof(T) + 16;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    cudaFuncAttributes fa;
    if (coop && cudaFuncGetAttributes(&fa, k_mgs_persist<T, VT>) == cudaSuccess &&
        smem + fa.sharedSizeBytes <= (size_t)optin &&
        cudaFuncSetAttribute(k_mgs_persist<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgs_persist<T, VT>,
                                                          MGSP_THREADS, smem) == cudaSuccess &&
            per_sm >= 1)
            ok = true;
    }
    cudaGetLastError();
    h->mgs_chunk = chunk;
    h->mgs_ok_cache[key] = ok;
    return ok;
}

// Whether the staged cooperative MGS kernel can run: the persistent kernel's
// conditions, plus w's row chunk and three basis row chunks in shared memory.
template <class T, class VT>
bool mgs_staged_ok(gmres_handle *h) {
    if (!mgs_persist_ok<T, VT>(h))
        return false;
    const void *key = (const void *)k_mgs_staged<T, VT>;
    auto it = h->mgs_ok_cache.find(key);
    if (it != h->mgs_ok_cache.end())
        return it->second;
    const int64_t chunk = round_up((h->ldv + h->nsm - 1) / h->nsm, 8);
    const size_t smem = MGSS_HEAD + (size_t)chunk * (sizeof(T) + 3 * sizeof(VT));
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    bool ok = true;
    auto prep = [&](auto fn) {
        cudaFuncAttributes fa;
        int per_sm = 0;
        ok = ok && cudaFuncGetAttributes(&fa, fn) == cudaSuccess &&
             smem + fa.sharedSizeBytes <= (size_t)optin &&
             cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                 cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, MGSP_THREADS, smem) ==
                 cudaSuccess &&
             per_sm >= 1;
    };
    prep(k_mgs_staged<T, VT>);
    if constexpr (std::is_same<T, double>::value)
        prep(k_mgs_staged<T, VT, true>);
    cudaGetLastError();
    h->mgss_chunk = chunk;
    h->mgs_ok_cache[key] = ok;
    return ok;
}

// out = (L U)^-1 z with the ILU(0) factors in the precision the solve uses:
// binary64 factors for binary64 work, binary32 factors for the binary32
// cycle, for limited mixed and on request (opts.ilu_binary32).
template <class T, class VT>
cudaError_t apply_ilu(gmres_handle *h, const T *z, T *tmp, T *out) {
    int *err = &h->ctl.as<Ctl>()->timeout;
    if constexpr (std::is_same<T, double>::value) {
        if (!h->limited && !h->opts.ilu_binary32 && !(h->opts.pv_mask & PV_M))
            return ilu_apply<double, double>(h, h->ilu64.as<double>(), z, tmp, out, err);
        return ilu_apply<double, float>(h, h->ilu32.as<float>(), z, tmp, out, err);
    } else {
        return ilu_apply<float, float>(h, h->ilu32.as<float>(), z, tmp, out, err);
    }
}

// Cycle start with the left preconditioner: r <- M^-1 r, beta = ||r||.
template <class T, class VT>
gmres_status left_start(gmres_handle *h, GridCtx<T, VT> &c, Acct &acct) {
    if (!c.left)
        return GMRES_OK;
    cudaEvent_t e = h->timer.begin();
    CK((apply_ilu<T, VT>(h, c.r, c.t, c.r)));
    k_pnorm<T, VT><<<h->grid, kThreads, 0, h->stream>>>(c);
    CKL();
    h->timer.end(GMRES_K_PRECOND, e);
    acct.launches[GMRES_K_PRECOND] += 3;
    return GMRES_OK;
}

// The three register-streaming CGSR passes (and the two column reductions)
// for an inner step with ncols basis vectors, then v_{j+1}.
template <class T, class VT, bool SPLIT>
gmres_status enqueue_cgs_rows(gmres_handle *h, GridCtx<T, VT> &c, int ncols, Acct &acct,
                              cudaEvent_t e) {
    // one resident wave per kernel: grid = SMs x resident blocks per SM
    static int per_sm[3] = {0, 0, 0};
    if (per_sm[0] == 0) {
        void (*fns[3])(GridCtx<T, VT>, int, T *, int64_t, int) = {
            k_cgs_rows<T, VT, 0, SPLIT>, k_cgs_rows<T, VT, 1, SPLIT>,
            k_cgs_rows<T, VT, 2, SPLIT>};
        for (int k = 0; k < 3; ++k) {
            int bpsm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, fns[k], ROWS_THREADS, 0));
            per_sm[k] = std::max(1, std::min(bpsm, h->rows_blocks_per_sm));
        }
    }
    // balanced grids: k = ceil(slices / resident blocks) consecutive slices
    // per block, grid = ceil(slices / k), one resident wave
    const int64_t nsl = h->ldv / (ROWS_WARPS * 32 * (16 / (int64_t)sizeof(VT)));
    int64_t kpb[3];
    int gsz[3];
    for (int k = 0; k < 3; ++k) {
        const int64_t cap = (int64_t)h->nsm * per_sm[k];
        kpb[k] = (nsl + cap - 1) / cap;
        gsz[k] = (int)((nsl + kpb[k] - 1) / kpb[k]);
    }
    // the per-variable study's instantiations (binary64 solves only)
    bool pvs = false;
    if constexpr (std::is_same<T, double>::value)
        pvs = (c.pv & PV_ORTHO) != 0;
    const int pf = h->opts.l2_prefetch;
    k_cgs_rows<T, VT, 0, SPLIT><<<gsz[0], ROWS_THREADS, 0, h->stream>>>(c, ncols, c.part, kpb[0],
                                                                        pf);
    k_reduce_cols<T><<<ncols + 1, 256, 0, h->stream>>>(c.part, gsz[0], ncols, c.h1, c.ctl, 1,
                                                       c.pv);
    if constexpr (std::is_same<T, float>::value && std::is_same<VT, float>::value) {
        // pass B with the slice in registers; KC vectors per warp
        const int kc = (ncols + PB_WARPS - 1) / PB_WARPS;
        void (*kfn)(GridCtx<float, float>, int, float *, int64_t) =
            kc <= 2 ? k_cgs_passb_reg<2>
                    : kc <= 4 ? k_cgs_passb_reg<4>
                              : kc <= 8 ? k_cgs_passb_reg<8>
                                        : kc <= 12 ? k_cgs_passb_reg<12> : k_cgs_passb_reg<17>;
        static std::map<const void *, int> pb_per_sm;
        int &bps = pb_per_sm[(const void *)kfn];
        if (bps == 0) {
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, PB_THREADS, 0));
            bps = std::max(1, bps);
        }
        const int64_t nsl_b = h->ldv / PB_ROWS;
        const int64_t cap = (int64_t)h->nsm * bps;
        const int64_t kb = (nsl_b + cap - 1) / cap;
        const int gb = (int)((nsl_b + kb - 1) / kb);
        kfn<<<gb, PB_THREADS, 0, h->stream>>>(c, ncols, c.part, kb);
        k_reduce_cols<T><<<ncols, 256, 0, h->stream>>>(c.part, gb, ncols, c.h2, c.ctl, 0, c.pv);
    } else {
        if (pvs)
            k_cgs_rows<T, VT, 1, SPLIT, true><<<gsz[1], ROWS_THREADS, 0, h->stream>>>(
                c, ncols, c.part, kpb[1], pf);
        else
            k_cgs_rows<T, VT, 1, SPLIT><<<gsz[1], ROWS_THREADS, 0, h->stream>>>(c, ncols, c.part,
                                                                                kpb[1], pf);
        k_reduce_cols<T><<<ncols, 256, 0, h->stream>>>(c.part, gsz[1], ncols, c.h2, c.ctl, 0,
                                                       c.pv);
    }
    if (pvs)
        k_cgs_rows<T, VT, 2, SPLIT, true><<<gsz[2], ROWS_THREADS, 0, h->stream>>>(c, ncols, c.part,
                                                                                  kpb[2], pf);
    else
        k_cgs_rows<T, VT, 2, SPLIT><<<gsz[2], ROWS_THREADS, 0, h->stream>>>(c, ncols, c.part,
                                                                            kpb[2], pf);
    acct.launches[GMRES_K_ORTHO] += 5;
    CKL();
    h->timer.end(GMRES_K_ORTHO, e);
    e = h->timer.begin();
    dim3 g(h->grid), b(kThreads);
    k_normalize<T, VT><<<g, b, 0, h->stream>>>(c, ncols, h->opts.orth_norm != GMRES_ORTH_OFF);
    CKL();
    h->timer.end(GMRES_K_NORMALIZE, e);
    acct.launches[GMRES_K_NORMALIZE]++;
    return GMRES_OK;
}

// Enqueue one inner step (column index `col` of the basis -> new column
// col+1) without the optional loss-of-orthogonality test.  Kernels return at
// once when the cycle has ended.
template <class T, class VT>
gmres_status enqueue_step_core(gmres_handle *h, GridCtx<T, VT> &c, int col, gmres_ortho ortho,
                               Acct &acct) {
    const int L = lanes_for<T, VT>(h);
    const VT *vj = c.V + (size_t)col * c.ldv;
    cudaEvent_t e = h->timer.begin();
    if (c.left) {
        // t = A v_j, w = M^-1 t (left preconditioning, Alg. 1); under the
        // per-variable w switch w, not t, is the stored Krylov vector
        CK((launch_spmv_step<T, VT, VT>(h, c, vj, c.t, L)));
        h->timer.end(GMRES_K_SPMV, e);
        acct.launches[GMRES_K_SPMV]++;
        e = h->timer.begin();
        CK((apply_ilu<T, VT>(h, c.t, h->t2.as<T>(), c.w)));
        if (c.pv & PV_W) {
            k_round32<T><<<h->grid, kThreads, 0, h->stream>>>(h->n, c.w, c.ctl);
            CKL();
        }
        h->timer.end(GMRES_K_PRECOND, e);
        acct.launches[GMRES_K_PRECOND] += 2;
        e = h->timer.begin();
        acct.launches[GMRES_K_SPMV]--;  // counted once below
    } else if (c.pvals) {
        // t = M v_j, w = A t (right preconditioning)
        GridCtx<T, VT> cp = c;
        cp.rowptr = c.prowptr;
        cp.colind = c.pcolind;
        cp.a = c.pvals;
        cp.a_lim = c.pvals_lim;
        cp.aform = c.pvals_lim ? 1 : 0;
        cp.sfmt = 0;  // M is on CSR
        CK((launch_spmv_step<T, VT, VT>(h, cp, vj, c.t, L)));
        acct.launches[GMRES_K_PRECOND]++;
        h->timer.end(GMRES_K_PRECOND, e);
        e = h->timer.begin();
        CK((launch_spmv_step<T, VT, T>(h, c, c.t, c.w, L)));
    } else {
        CK((launch_spmv_step<T, VT, VT>(h, c, vj, c.w, L)));
    }
    if (!c.left && (c.pv & PV_W)) {
        // the per-variable study's w switch: w = A v_j stored in binary32
        k_round32<T><<<h->grid, kThreads, 0, h->stream>>>(h->n, c.w, c.ctl);
        CKL();
    }
    h->timer.end(GMRES_K_SPMV, e);
    acct.launches[GMRES_K_SPMV]++;
    const int ncols = col + 1;
    dim3 g(h->grid), b(kThreads);
    e = h->timer.begin();
    if (ortho == GMRES_ORTHO_CGSR) {
        if (h->opts.cgs_kernel == 2)
            return enqueue_cgs_rows<T, VT, false>(h, c, ncols, acct, e);
        return enqueue_cgs_rows<T, VT, true>(h, c, ncols, acct, e);
    }
    if (h->opts.mgs_kernel != 1 && mgs_persist_ok<T, VT>(h)) {
        // one cooperative kernel: w stays in shared memory, v_{j+1} written;
        // by default with the block's basis rows staged in shared memory one
        // vector ahead (when they fit)
        const bool staged = h->opts.mgs_kernel == 0 && mgs_staged_ok<T, VT>(h);
        int64_t chunk = staged ? h->mgss_chunk : h->mgs_chunk;
        long long spin = h->opts.spin_limit > 0 ? h->opts.spin_limit : (1LL << 24);
        // exchange slots: 2 parities x 4 words per block, round numbers
        // never reused (cleared before they wrap)
        const size_t slot_bytes = (size_t)h->nsm * 2 * 4 * sizeof(unsigned long long);
        if (h->mgs_seq.bytes < slot_bytes || h->mgs_round > 0x7fffff00u - (unsigned)(ncols + 1)) {
            CK(h->mgs_seq.ensure(slot_bytes));
            CK(cudaMemsetAsync(h->mgs_seq.p, 0, h->mgs_seq.bytes, h->stream));
            h->mgs_round = 1;
        }
        unsigned long long *slots = h->mgs_seq.as<unsigned long long>();
        unsigned round0 = h->mgs_round;
        h->mgs_round += (unsigned)(ncols + 1);
        GridCtx<T, VT> cc = c;
        int nc = ncols;
        void *args[] = {&cc, &nc, &chunk, &spin, &slots, &round0};
        const void *kfn = staged ? (const void *)k_mgs_staged<T, VT>
                                 : (const void *)k_mgs_persist<T, VT>;
        size_t smem = staged ? MGSS_HEAD + (size_t)chunk * (sizeof(T) + 3 * sizeof(VT))
                             : (size_t)chunk * sizeof(T) + 16;
        if constexpr (std::is_same<T, double>::value) {
            if (c.pv & PV_ORTHO) {  // the per-variable study's instantiations
                if (staged) {
                    kfn = (const void *)k_mgs_staged<T, VT, true>;
                } else {
                    kfn = (const void *)k_mgs_persist<T, VT, true>;
                    CK(cudaFuncSetAttribute(k_mgs_persist<T, VT, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
                }
            }
        }
        CK(cudaLaunchCooperativeKernel(kfn, dim3(h->nsm), dim3(MGSP_THREADS), args, smem,
                                       h->stream));
        acct.launches[GMRES_K_ORTHO] += 1;
        h->timer.end(GMRES_K_ORTHO, e);
        return GMRES_OK;
    } else {
        if (c.pv & PV_ORTHO) {  // the per-variable study's instantiations
            for (int i = 0; i < ncols; ++i)
                k_mgs_step<T, VT, true><<<g, b, 0, h->stream>>>(c, i);
            k_mgs_last<T, VT, true><<<g, b, 0, h->stream>>>(c, ncols);
        } else {
            for (int i = 0; i < ncols; ++i)
                k_mgs_step<T, VT><<<g, b, 0, h->stream>>>(c, i);
            k_mgs_last<T, VT><<<g, b, 0, h->stream>>>(c, ncols);
        }
        acct.launches[GMRES_K_ORTHO] += ncols + 1;
    }
    CKL();
    h->timer.end(GMRES_K_ORTHO, e);
    e = h->timer.begin();
    k_normalize<T, VT><<<g, b, 0, h->stream>>>(c, col + 1, h->opts.orth_norm != GMRES_ORTH_OFF);
    CKL();
    h->timer.end(GMRES_K_NORMALIZE, e);
    acct.launches[GMRES_K_NORMALIZE]++;
    return GMRES_OK;
}

// The inner step plus, when enabled, the loss-of-orthogonality test (Sec. 3,
// fourth strategy): u = V^T v_{col+2} by the Gram pass of the rows kernel,
// then the S column, its norm and the restart decision in one block.
template <class T, class VT>
gmres_status enqueue_step(gmres_handle *h, GridCtx<T, VT> &c, int col, gmres_ortho ortho,
                          Acct &acct) {
    gmres_status st = enqueue_step_core(h, c, col, ortho, acct);
    if (st != GMRES_OK || h->opts.orth_norm == GMRES_ORTH_OFF)
        return st;
    const int k = col + 2;  // stored vectors v_1 .. v_{col+2}
    const int ncols = k - 1;
    cudaEvent_t e = h->timer.begin();
    static int per_sm = 0;
    if (per_sm == 0) {
        int bpsm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_cgs_rows<T, VT, 3>,
                                                         ROWS_THREADS, 0));
        per_sm = std::max(1, std::min(bpsm, h->rows_blocks_per_sm));
    }
    const int64_t nsl = h->ldv / (ROWS_WARPS * 32 * (16 / (int64_t)sizeof(VT)));
    const int64_t cap = (int64_t)h->nsm * per_sm;
    const int64_t kpb = (nsl + cap - 1) / cap;
    const int gsz = (int)((nsl + kpb - 1) / kpb);
    k_cgs_rows<T, VT, 3><<<gsz, ROWS_THREADS, 0, h->stream>>>(c, ncols, c.part, kpb,
                                                              h->opts.l2_prefetch);
    k_reduce_cols<T><<<ncols, 256, 0, h->stream>>>(c.part, gsz, ncols, c.h2, c.ctl, 2);
    OrthMon M;
    M.U = h->mon.as<double>() + 2 * (MMAX + 2);
    M.S = M.U + (size_t)ORTH_LD * ORTH_LD;
    M.hist = mon_hist(h);
    M.threshold = h->opts.orth_threshold;
    M.norm = h->opts.orth_norm;
    M.iters = h->opts.orth_iters > 0 ? h->opts.orth_iters : 10;
    k_orth_monitor<T><<<1, ORTH_THREADS, 0, h->stream>>>(c.ctl, c.h2, k, M);
    CKL();
    h->timer.end(GMRES_K_ORTHO, e);
    acct.launches[GMRES_K_ORTHO] += 3;
    return GMRES_OK;
}

// Algorithmic bytes of a finished cycle of length j (what each step must
// move: basis read once per pass, vectors once, gathers of x counted once).
template <class T, class VT>
void account_cycle(gmres_handle *h, int j, gmres_ortho ortho, Acct &acct) {
    const double n = h->n, nnz = (double)h->nnz;
    const double sT = sizeof(T), sV = sizeof(VT);
    // matrix value bytes the Krylov step reads
    const double sA = h->split ? ((sizeof(T) == 8 && !h->limited) ? 8.0 : 4.0)
                               : (h->limited ? 4.0 : sT);
    const bool pre = spai_on(h);
    const bool ilu = ilu_on(h);
    // ILU(0) factor bytes one triangular solve pair reads (values, indices,
    // row pointers, diagonal positions) plus its vectors and ready flags
    const double sL = (sizeof(T) == 8 && !h->limited && !h->opts.ilu_binary32) ? 8.0 : 4.0;
    const double ilu_bytes = nnz * (sL + 4) + 2.0 * (n + 1) * 4 + n * 4 + 4.0 * n * sT + 8.0 * n;
    // A's bytes per product: CSR values, column indices and row pointers, or
    // the sliced copy's values, indices, row lengths and slice offsets
    const int sf = sell_fmt_for<T>(h, true);
    const double nsl = (double)((h->n + SELL_C - 1) / SELL_C);
    const double a_bytes = sf ? nnz * (sA + (sf == 1 ? 2 : 4)) + nsl * SELL_C * 2 + (nsl + 1) * 4
                              : nnz * (sA + 4) + (n + 1) * 4;
    for (int it = 0; it < j; ++it) {
        const double c = it + 1;
        acct.bytes[GMRES_K_SPMV] += a_bytes + n * (pre ? sT : sV) + n * sT;
        if (pre)
            acct.bytes[GMRES_K_PRECOND] += nnz * (sA + 4) + (n + 1) * 4 + n * sV + n * sT;
        if (ilu)
            acct.bytes[GMRES_K_PRECOND] += ilu_bytes;
        if (ortho == GMRES_ORTHO_CGSR)
            acct.bytes[GMRES_K_ORTHO] += 3 * c * n * sV + 5 * n * sT;
        else
            acct.bytes[GMRES_K_ORTHO] += c * n * sV + 2 * n * sT;
        if (h->opts.orth_norm != GMRES_ORTH_OFF)
            acct.bytes[GMRES_K_ORTHO] += (c + 1) * n * sV;  // u = V^T v_{j+1}
        if (it + 1 < j)
            acct.bytes[GMRES_K_NORMALIZE] += n * sT + n * sV;
    }
    acct.bytes[GMRES_K_NORMALIZE] += n * sT + n * sV;  // v_1 = r / beta
    acct.bytes[GMRES_K_UPDATE] += j * n * sV + 2 * n * 8 + (pre ? 2 * n * sT : 0);
}

template <class T, class VT>
void account_residual(gmres_handle *h, Acct &acct) {
    const double n = h->n, nnz = (double)h->nnz;
    acct.bytes[GMRES_K_RESIDUAL] += nnz * 12 + (n + 1) * 4 + n * 8 * 2 + n * sizeof(T);
    acct.launches[GMRES_K_RESIDUAL]++;
}

gmres_status read_ctl(gmres_handle *h) {
    CK(cudaMemcpyAsync(h->hctl, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

template <class T, class VT>
gmres_status solve_grid(gmres_handle *h, const double *b, double *x, int m, double tol,
                        gmres_ortho ortho, gmres_precision prec, int maxiter, gmres_info *info) {
    gmres_status st = ensure_workspace(h, m, prec);
    if (st != GMRES_OK)
        return st;
    GridCtx<T, VT> c = make_ctx<T, VT>(h, m);
    const double tau = h->opts.tau >= 0 ? h->opts.tau : default_tau(prec);
    const int repeat_first = h->opts.repeat_first >= 0 ? h->opts.repeat_first
                                                       : (prec == GMRES_FP64 ? 0 : 1);
    Acct acct;
    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
    k_bnorm<T, VT><<<h->grid, kThreads, 0, h->stream>>>(c, b);
    CKL();
    acct.launches[GMRES_K_RESIDUAL]++;
    st = read_ctl(h);
    if (st != GMRES_OK)
        return st;
    const double bnorm = h->hctl->bnorm;
    info->bnorm = bnorm;
    if (h->hctl->nonfinite || !std::isfinite(bnorm))
        return GMRES_ERR_NONFINITE;
    if (bnorm == 0) {
        CK(cudaMemsetAsync(x, 0, sizeof(double) * h->n, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        info->converged = 1;
        info->relres = 0;
        return GMRES_OK;
    }
    c.tol_abs = tol * bnorm;
    c.inner_abs = h->opts.inner_factor * tol * bnorm;
    if (c.pv & PV_X) {
        // the solution as the study stores it from the start
        k_round32<double><<<h->grid, kThreads, 0, h->stream>>>(h->n, x, nullptr);
        CKL();
    }
    cudaEvent_t e = h->timer.begin();
    CK(launch_residual(h, c, b, x, nullptr, 1));
    h->timer.end(GMRES_K_RESIDUAL, e);
    account_residual<T, VT>(h, acct);
    st = left_start<T, VT>(h, c, acct);
    if (st != GMRES_OK)
        return st;
    st = read_ctl(h);
    if (st != GMRES_OK)
        return st;
    int cycle_len = m;
    int stall = 0;
    double prev_rn = h->hctl->rnorm;
    gmres_status result = GMRES_MAXITER;
    for (;;) {
        const Ctl &k = *h->hctl;
        info->relres = k.rnorm / bnorm;
        if (k.nonfinite) {
            result = GMRES_ERR_NONFINITE;
            break;
        }
        if (k.timeout) {
            result = GMRES_ERR_TIMEOUT;
            break;
        }
        if (k.converged) {
            result = GMRES_OK;
            info->converged = 1;
            break;
        }
        if (info->iters >= maxiter) {
            result = GMRES_MAXITER;
            break;
        }
        if (!k.active) {
            result = GMRES_ERR_BREAKDOWN;  // beta == 0 in the working precision
            break;
        }
        const int kmax = std::min(cycle_len, maxiter - info->iters);
        c.kmax = kmax;
        c.tau = (repeat_first && info->restarts > 0) ? 0.0 : tau;
        if (h->opts.orth_norm != GMRES_ORTH_OFF)
            CK(cudaMemsetAsync(mon_hist(h), 0, (MMAX + 2) * sizeof(double), h->stream));
        e = h->timer.begin();
        {
            int gi = 0;
            const GridCtx<T, VT> ci = stream_ctx(h, c, &gi);
            k_init<T, VT><<<gi, kThreads, 0, h->stream>>>(ci);
        }
        CKL();
        h->timer.end(GMRES_K_NORMALIZE, e);
        acct.launches[GMRES_K_NORMALIZE]++;
        for (int it = 0; it < kmax; ++it) {
            st = enqueue_step(h, c, it, ortho, acct);
            if (st != GMRES_OK)
                return st;
        }
        e = h->timer.begin();
        size_t sm = (size_t)m * m * sizeof(T) + (size_t)(m + 1) * sizeof(T);
        CK(cudaFuncSetAttribute(k_backsolve<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm));
        k_backsolve<T, VT><<<1, 32, sm, h->stream>>>(c);
        CKL();
        const bool pre = c.pvals != nullptr;
        int gu = 0;
        const GridCtx<T, VT> cu = stream_ctx(h, c, &gu);
        if (c.pv & PV_X)  // the per-variable study's instantiation
            k_update<T, VT, true><<<gu, kThreads, 0, h->stream>>>(cu, x, pre ? 1 : 0);
        else
            k_update<T, VT><<<gu, kThreads, 0, h->stream>>>(cu, x, pre ? 1 : 0);
        CKL();
        acct.launches[GMRES_K_UPDATE] += 2;
        if (pre) {
            // u = M t with t = V_j y, then x += u (right preconditioning)
            if (c.pvals_lim)
                CK((launch_spmv_plain<T, float>(h, lanes_for<T, VT>(h), c.pvals_lim, c.t, c.w)));
            else
                CK(launch_spmv_plain<T>(h, lanes_for<T, VT>(h), c.pvals, c.t, c.w));
            k_axpy_x<T><<<h->grid, kThreads, 0, h->stream>>>(h->n, c.w, x, c.ctl, c.pv);
            CKL();
            acct.launches[GMRES_K_UPDATE] += 2;
        }
        h->timer.end(GMRES_K_UPDATE, e);
        e = h->timer.begin();
        CK(launch_residual(h, c, b, x, nullptr, 1));
        h->timer.end(GMRES_K_RESIDUAL, e);
        account_residual<T, VT>(h, acct);
        st = left_start<T, VT>(h, c, acct);
        if (st != GMRES_OK)
            return st;
        st = read_ctl(h);
        if (st != GMRES_OK)
            return st;
        h->timer.harvest(info->kernel_ms);
        const int j = h->hctl->last_j;
        account_cycle<T, VT>(h, j, ortho, acct);
        if (h->hctl->timeout) {
            result = GMRES_ERR_TIMEOUT;
            info->iters += j;
            break;
        }
        info->iters += j;
        info->restarts += 1;
        if (info->restarts == 1) {
            info->first_len = j;
            if (repeat_first)
                cycle_len = std::max(1, j);
        }
        const double rn = h->hctl->rnorm;
        const bool no_progress =
            j == 0 || (h->hctl->breakdown && rn >= prev_rn && !h->hctl->converged);
        if (c.pvals) {
            // Stagnation fallback for the learned preconditioner: a cycle that
            // produced non-finite values, made no progress, or two cycles in a
            // row that cut the binary64 residual by less than 10 % switch the
            // solve to unpreconditioned mixed GMRES (the residual decides).
            stall = (rn > 0.9 * prev_rn) ? stall + 1 : 0;
            if (h->opts.fallback && (h->hctl->nonfinite || no_progress || stall >= 2)) {
                c.pvals = nullptr;
                info->fell_back = 1;
                stall = 0;
                if (h->hctl->nonfinite) {
                    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
                    CK(launch_residual(h, c, b, x, nullptr, 1));
                    st = read_ctl(h);
                    if (st != GMRES_OK)
                        return st;
                }
                prev_rn = h->hctl->rnorm;
                continue;
            }
        }
        if (no_progress) {
            info->relres = rn / bnorm;
            result = GMRES_ERR_BREAKDOWN;
            break;
        }
        prev_rn = rn;
    }
    if (c.pv & (PV_A_RESID | PV_B | PV_X | PV_AX)) {
        // the solver tested its own residual (A, b, x or A x stored in
        // binary32); report the binary64 residual of the x it returns, and
        // count the solve as converged only if that met tol
        GridCtx<T, VT> ct = c;
        ct.pv = 0;
        CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
        CK(launch_residual(h, ct, b, x, nullptr, 0));
        acct.launches[GMRES_K_RESIDUAL]++;
        st = read_ctl(h);
        if (st != GMRES_OK)
            return st;
        info->relres = h->hctl->rnorm / bnorm;
        info->converged = h->hctl->converged;
        if (result == GMRES_OK && !info->converged)
            result = GMRES_MAXITER;
    }
    h->timer.harvest(info->kernel_ms);
    for (int k = 0; k < GMRES_K_COUNT; ++k) {
        info->kernel_bytes[k] += acct.bytes[k];
        info->kernel_launches[k] += acct.launches[k];
        info->launches += acct.launches[k];
    }
    return result;
}

template <class T, class VT>
gmres_status solve_block(gmres_handle *h, const double *b, double *x, int m, double tol,
                         gmres_ortho ortho, gmres_precision prec, int maxiter, gmres_info *info) {
    gmres_status st = ensure_workspace(h, m, prec);
    if (st != GMRES_OK)
        return st;
    BlockSys<T, VT> S;
    S.n = h->n;
    S.ldv = h->ldv;
    S.rowptr = h->rowptr.as<int>();
    S.colind = h->colind.as<int>();
    S.a = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->vals64.p)
                                         : reinterpret_cast<const T *>(h->vals32.p);
    S.a64 = h->vals64.as<double>();
    S.b = b;
    S.x = x;
    S.V = h->V.as<VT>();
    S.w = h->w.as<T>();
    S.r = h->r.as<T>();
    S.vscale = std::is_same<VT, __half>::value ? fp16_scale(h->n) : 1.0f;
    S.vinv = 1.0f / S.vscale;
    CK(h->bsys.ensure(sizeof(S) + sizeof(unsigned) * 4));
    CK(h->bres.ensure(sizeof(BlockResult)));
    CK(cudaMemcpyAsync(h->bsys.p, &S, sizeof(S), cudaMemcpyHostToDevice, h->stream));
    unsigned *queue = reinterpret_cast<unsigned *>(h->bsys.as<unsigned char>() + sizeof(S));
    CK(cudaMemsetAsync(queue, 0, sizeof(unsigned), h->stream));
    BlockParams P;
    P.m = m;
    P.maxiter = maxiter;
    P.ortho = (int)ortho;
    P.repeat_first = h->opts.repeat_first >= 0 ? h->opts.repeat_first
                                               : (prec == GMRES_FP64 ? 0 : 1);
    P.tol = tol;
    P.tau = h->opts.tau >= 0 ? h->opts.tau : default_tau(prec);
    P.inner_factor = h->opts.inner_factor;
    P.brk = std::is_same<T, double>::value ? 1e-14 : 1e-6;
    P.stall_factor = h->opts.stall_factor;
    P.stall_w = h->opts.stall_window > 0 ? h->opts.stall_window : (m + 19) / 20;
    P.nsys = 1;
    P.queue = queue;
    P.order = nullptr;
    size_t smem = block_smem_bytes<T>(m);
    int L = lanes_for<T, VT>(h);
    // one block, or one cluster: binary64 arithmetic is slow on one SM, so a
    // binary64 system of 2048+ rows spreads over a cluster by default
    int cs = h->opts.block_cluster;
    if (cs == 0)
        cs = (std::is_same<T, double>::value && h->n >= 2048) ? TEAM_SINGLE_CTAS : 1;
    if (cs == TEAM_SINGLE_CTAS) {
        const int64_t chunk = (h->n + cs - 1) / cs;
        const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(64, round_up(chunk / 2, 32)));
        cudaEvent_t e = h->timer.begin();
        CK((launch_team_single<T, VT>(h->bsys.as<BlockSys<T, VT>>(), P, h->bres.as<BlockResult>(),
                                      L, threads, smem, h->stream)));
        h->timer.end(GMRES_K_BLOCK, e);
    } else {
    int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(64, round_up(h->n / 4, 32)));
    auto *kfn = &k_block_solve<T, VT, 4>;
    switch (L) {
    case 1: kfn = &k_block_solve<T, VT, 1>; break;
    case 2: kfn = &k_block_solve<T, VT, 2>; break;
    case 4: kfn = &k_block_solve<T, VT, 4>; break;
    case 8: kfn = &k_block_solve<T, VT, 8>; break;
    case 16: kfn = &k_block_solve<T, VT, 16>; break;
    default: kfn = &k_block_solve<T, VT, 32>; break;
    }
    CK(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaEvent_t e = h->timer.begin();
    kfn<<<1, threads, smem, h->stream>>>(h->bsys.as<BlockSys<T, VT>>(), P,
                                          h->bres.as<BlockResult>());
    CKL();
    h->timer.end(GMRES_K_BLOCK, e);
    }
    BlockResult R;
    CK(cudaMemcpyAsync(&R, h->bres.p, sizeof(R), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->timer.harvest(info->kernel_ms);
    info->iters = R.iters;
    info->restarts = R.restarts;
    info->converged = R.converged;
    info->first_len = R.first_len;
    info->relres = R.relres;
    info->bnorm = R.bnorm;
    info->launches += 1;
    info->kernel_launches[GMRES_K_BLOCK] += 1;
    {
        // algorithmic bytes of the solve (SpMV + orthogonalisation per inner
        // step, binary64 residual per cycle), counted as the batched solver does
        const double n = (double)h->n, nz = (double)h->nnz;
        const double sv = sizeof(VT), st = sizeof(T);
        const double cycles = R.restarts, it = R.iters;
        const double avgc = cycles > 0 ? (it / cycles + 1) / 2 : 0;  // mean basis size
        const double orth = ortho == GMRES_ORTHO_CGSR ? 3 * avgc * n * sv + 5 * n * st
                                                      : avgc * n * sv + 2 * n * st;
        info->kernel_bytes[GMRES_K_BLOCK] +=
            it * (nz * (st + 4) + 4 * n + n * sv + n * st + orth + n * st + n * sv) +
            (cycles + 1) * (12 * nz + 4 * n + 24 * n);
    }
    return (gmres_status)R.status;
}

template <class T, class VT>
gmres_status solve_dispatch_path(gmres_handle *h, const double *b, double *x, int m, double tol,
                                 gmres_ortho ortho, gmres_precision prec, int maxiter,
                                 gmres_info *info) {
    int path = h->opts.path;
    const bool grid_only = h->opts.orth_norm != GMRES_ORTH_OFF || h->limited || h->split ||
                           ilu_on(h) || h->opts.pv_mask != 0;
    if (path == GMRES_PATH_AUTO)
        path = (h->n <= 16384 && !spai_on(h) && !grid_only)
                   ? GMRES_PATH_BLOCK
                   : GMRES_PATH_GRID;
    if (path == GMRES_PATH_BLOCK && grid_only)
        return GMRES_ERR_ARG;  // the orthogonality test, limited mixed and split storage
                               // run on the grid path
    info->path = path;
    if (path == GMRES_PATH_BLOCK)
        return solve_block<T, VT>(h, b, x, m, tol, ortho, prec, maxiter, info);
    return solve_grid<T, VT>(h, b, x, m, tol, ortho, prec, maxiter, info);
}

gmres_status validate_opts(const gmres_opts *o) {
    if (!o)
        return GMRES_ERR_ARG;
    if (!(o->inner_factor >= 0) || o->path < 0 || o->path > 2 || o->spin_limit < 0 ||
        (o->spmv_lanes != 0 && (o->spmv_lanes < 1 || o->spmv_lanes > 32 ||
                                (o->spmv_lanes & (o->spmv_lanes - 1)))) ||
        o->cgs_kernel < 0 || o->cgs_kernel > 3 || o->mgs_kernel < 0 || o->mgs_kernel > 2 ||
        o->cgs_kernel == 1 || o->cgs_kernel == 3 || o->l2_prefetch < 0 || o->l2_prefetch > 4 ||
        !(o->stall_factor >= 0) ||
        (o->block_cluster != 0 && o->block_cluster != 1 && o->block_cluster != TEAM_SINGLE_CTAS) ||
        o->stall_window < 0 || o->stall_window > MMAX || o->orth_norm < GMRES_ORTH_OFF ||
        o->orth_norm > GMRES_ORTH_FROBENIUS || o->orth_iters < 0 ||
        (o->orth_norm != GMRES_ORTH_OFF && !(o->orth_threshold > 0)) ||
        o->repeat_first < -1 || o->repeat_first > 1 || o->precond < 0 || o->precond > 2 ||
        o->ilu_binary32 < 0 || o->ilu_binary32 > 1 || o->trsv_kernel < 0 || o->trsv_kernel > 3 ||
        o->pv_mask < 0 || o->pv_mask > (int32_t)PV_ALL || o->spmv_format < GMRES_SPMV_AUTO ||
        o->spmv_format > GMRES_SPMV_SLICED)
        return GMRES_ERR_ARG;
    return GMRES_OK;
}

}  // namespace

extern "C" {

void gmres_default_opts(gmres_opts *o) {
    if (!o)
        return;
    memset(o, 0, sizeof(*o));
    o->tau = -1.0;
    o->inner_factor = 0.5;
    o->repeat_first = -1;
    o->path = GMRES_PATH_AUTO;
    o->profile = 0;
    o->spin_limit = 0;
    o->precond = 0;
    o->fallback = 1;
    o->spmv_lanes = 0;
    o->stall_factor = 0.0;
    o->stall_window = 0;
    o->orth_norm = GMRES_ORTH_OFF;
    o->orth_threshold = 1.0;
    o->orth_iters = 10;
    o->trsv_kernel = 0;
}

const char *gmres_status_str(gmres_status s) {
    switch (s) {
    case GMRES_OK: return "converged";
    case GMRES_MAXITER: return "iteration limit reached";
    case GMRES_ERR_ARG: return "invalid argument";
    case GMRES_ERR_CUDA: return "CUDA error";
    case GMRES_ERR_NONFINITE: return "non-finite value";
    case GMRES_ERR_BREAKDOWN: return "breakdown without progress";
    case GMRES_ERR_TIMEOUT: return "device wait timed out";
    case GMRES_ERR_OOM: return "out of device memory";
    case GMRES_ERR_INDEX: return "column index outside its system (checked build)";
    }
    return "unknown status";
}

const char *gmres_version(void) { return "gmres_gb300 0.1 (sm_103a)"; }

gmres_status gmres_create(gmres_t *out, int32_t n, const int32_t *rowptr, const int32_t *colind,
                          const double *vals, int32_t flags, void *stream) {
    if (!out)
        return GMRES_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || !rowptr ||
        (flags & ~(GMRES_CREATE_DEVICE_PTRS | GMRES_CREATE_TRANSPOSE | GMRES_CREATE_SPLIT)) ||
        ((flags & GMRES_CREATE_SPLIT) && (flags & GMRES_CREATE_TRANSPOSE)))
        return GMRES_ERR_ARG;
    const bool dev = (flags & GMRES_CREATE_DEVICE_PTRS) != 0;
    // Validate the structure on the host (device arrays are copied down).
    std::vector<int32_t> rp(n + 1);
    if (dev) {
        if (cudaMemcpy(rp.data(), rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            cudaGetLastError();
            return GMRES_ERR_ARG;
        }
    } else {
        memcpy(rp.data(), rowptr, sizeof(int32_t) * (n + 1));
    }
    const int64_t nnz = rp[n];
    if (nnz < 0 || (nnz > 0 && (!colind || !vals)))
        return GMRES_ERR_ARG;
    std::vector<int32_t> ci(nnz);
    std::vector<double> va(nnz);
    if (nnz > 0) {
        if (dev) {
            if (cudaMemcpy(ci.data(), colind, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) !=
                    cudaSuccess ||
                cudaMemcpy(va.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost) !=
                    cudaSuccess) {
                cudaGetLastError();
                return GMRES_ERR_ARG;
            }
        } else {
            memcpy(ci.data(), colind, sizeof(int32_t) * nnz);
            memcpy(va.data(), vals, sizeof(double) * nnz);
        }
    }
    gmres_status st = check_csr_host(n, rp.data(), ci.data(), nnz, n);
    if (st != GMRES_OK)
        return st;
    for (int64_t k = 0; k < nnz; ++k)
        if (!std::isfinite(va[k]))
            return GMRES_ERR_NONFINITE;

    gmres_handle *h = new (std::nothrow) gmres_handle();
    if (!h)
        return GMRES_ERR_OOM;
    gmres_default_opts(&h->opts);
    h->n = n;
    h->nnz = nnz;
    h->ldv = round_up(n, LDV_ALIGN);  // every row slice of the streaming kernels divides it
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    h->timer.st = h->stream;
    auto fail = [&](gmres_status s) {
        gmres_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    h->grid = 2 * h->nsm;
    h->rows_blocks_per_sm = 16;
    h->chunk = round_up((h->ldv + h->grid - 1) / h->grid, 4);
    const double avg = (double)nnz / n;
    h->lanes32 = h->lanes64 = pow2_lanes(avg / 2.0);
    h->split = (flags & GMRES_CREATE_SPLIT) != 0;
    // vals64 holds the binary64 values, or with split storage hi[nnz] then
    // lo[nnz] (the same 8 bytes per nonzero); vals32 the binary32 copy (not
    // kept with split storage)
    if (h->rowptr.ensure(sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        h->colind.ensure(sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        h->vals64.ensure(sizeof(double) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        (!h->split && h->vals32.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)) != cudaSuccess))
        return fail(GMRES_ERR_OOM);
    ScopedBuf staging;  // binary64 values on the device before the split
    if (h->split && nnz > 0 && staging.ensure(sizeof(double) * nnz) != cudaSuccess)
        return fail(GMRES_ERR_OOM);
    if (cudaMemcpyAsync(h->rowptr.p, rp.data(), sizeof(int32_t) * (n + 1),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        (nnz > 0 && (cudaMemcpyAsync(h->colind.p, ci.data(), sizeof(int32_t) * nnz,
                                     cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                     cudaMemcpyAsync(h->split ? staging.p : h->vals64.p, va.data(),
                                     sizeof(double) * nnz, cudaMemcpyHostToDevice,
                                     h->stream) != cudaSuccess)))
        return fail(GMRES_ERR_CUDA);
    if (nnz > 0) {
        if (h->split)
            k_split_vals<<<h->nsm * 4, 256, 0, h->stream>>>(
                nnz, staging.as<double>(), h->vals64.as<unsigned>(),
                h->vals64.as<unsigned>() + nnz);
        else
            k_cast_vals<<<h->nsm * 4, 256, 0, h->stream>>>(nnz, h->vals64.as<double>(),
                                                            h->vals32.as<float>());
        if (cudaGetLastError() != cudaSuccess)
            return fail(GMRES_ERR_CUDA);
    }
    if (flags & GMRES_CREATE_TRANSPOSE) {
        // CSR of A^T built on the host from the validated arrays.
        std::vector<int32_t> trp(n + 1, 0), tci(nnz);
        std::vector<double> tva(nnz);
        for (int64_t k = 0; k < nnz; ++k)
            trp[ci[k] + 1]++;
        for (int i = 0; i < n; ++i)
            trp[i + 1] += trp[i];
        std::vector<int32_t> pos(trp.begin(), trp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                int32_t d = pos[ci[k]]++;
                tci[d] = i;
                tva[d] = va[k];
            }
        if (h->trowptr.ensure(sizeof(int32_t) * (n + 1)) != cudaSuccess ||
            h->tcolind.ensure(sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
            h->tvals64.ensure(sizeof(double) * std::max<int64_t>(nnz, 1)) != cudaSuccess)
            return fail(GMRES_ERR_OOM);
        if (cudaMemcpyAsync(h->trowptr.p, trp.data(), sizeof(int32_t) * (n + 1),
                            cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            (nnz > 0 && (cudaMemcpyAsync(h->tcolind.p, tci.data(), sizeof(int32_t) * nnz,
                                         cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                         cudaMemcpyAsync(h->tvals64.p, tva.data(), sizeof(double) * nnz,
                                         cudaMemcpyHostToDevice, h->stream) != cudaSuccess)))
            return fail(GMRES_ERR_CUDA);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    *out = h;
    return GMRES_OK;
}

void gmres_destroy(gmres_t h) {
    if (!h)
        return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    else
        cudaDeviceSynchronize();
    for (DevBuf *b : {&h->rowptr, &h->colind, &h->vals64, &h->vals32, &h->trowptr, &h->tcolind,
                      &h->tvals64, &h->V, &h->w, &h->r, &h->t, &h->z, &h->xb, &h->bb, &h->small,
                      &h->part, &h->part64, &h->ctl, &h->bsys, &h->bres, &h->pvals64,
                      &h->pvals32, &h->spai_feat, &h->spai_rowv, &h->tvals32, &h->spai_params,
                      &h->spai_m, &h->spai_gm, &h->spai_H, &h->spai_vec, &h->spai_part,
                      &h->spai_Z, &h->spai_grad, &h->mgs_seq, &h->mon, &h->ilu64, &h->ilu32,
                      &h->ilu_dpos, &h->ilu_flags, &h->t2, &h->ilu_order, &h->ilu_lptr,
                      &h->sptr, &h->slen, &h->scol, &h->sval32, &h->sval64})
        b->release();
    if (h->hctl)
        cudaFreeHost(h->hctl);
    h->timer.destroy();
    delete h;
}

gmres_status gmres_set_values(gmres_t h, const double *vals) {
    if (!h || (h->nnz > 0 && !vals))
        return GMRES_ERR_ARG;
    if (h->nnz == 0)
        return GMRES_OK;
    const bool dev = is_device_ptr(vals);
    if (!dev) {
        for (int64_t k = 0; k < h->nnz; ++k)
            if (!std::isfinite(vals[k]))
                return GMRES_ERR_NONFINITE;
    }
    if (h->split) {
        ScopedBuf staging;
        CK(staging.ensure(sizeof(double) * h->nnz));
        CK(cudaMemcpyAsync(staging.p, vals, sizeof(double) * h->nnz,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        k_split_vals<<<h->nsm * 4, 256, 0, h->stream>>>(h->nnz, staging.as<double>(),
                                                         h->vals64.as<unsigned>(),
                                                         h->vals64.as<unsigned>() + h->nnz);
        CKL();
        CK(cudaStreamSynchronize(h->stream));
    } else {
        CK(cudaMemcpyAsync(h->vals64.p, vals, sizeof(double) * h->nnz,
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        k_cast_vals<<<h->nsm * 4, 256, 0, h->stream>>>(h->nnz, h->vals64.as<double>(),
                                                        h->vals32.as<float>());
        CKL();
        CK(cudaStreamSynchronize(h->stream));
    }
    // derived data of the old values is stale
    h->trowptr.release();
    h->tcolind.release();
    h->tvals64.release();
    h->spai_feat_ok = 0;
    h->has_precond = 0;
    h->ilu_ok = 0;
    return sell_refill(h);  // the sliced copy takes the new values
}

gmres_status gmres_set_stream(gmres_t h, void *stream) {
    if (!h)
        return GMRES_ERR_ARG;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    h->timer.st = h->stream;
    return GMRES_OK;
}

gmres_status gmres_set_opts(gmres_t h, const gmres_opts *o) {
    if (!h)
        return GMRES_ERR_ARG;
    gmres_status st = validate_opts(o);
    if (st != GMRES_OK)
        return st;
    if (o->spmv_format == GMRES_SPMV_SLICED) {
        st = sell_build(h);  // the sliced copy must exist before a solve reads it
        if (st != GMRES_OK)
            return st;
    }
    h->opts = *o;
    return GMRES_OK;
}

gmres_status gmres_spmv_format(gmres_t h, int32_t *fmt32, int32_t *fmt64) {
    if (!h)
        return GMRES_ERR_ARG;
    if (fmt32)
        *fmt32 = sell_fmt_for<float>(h, false) ? GMRES_SPMV_SLICED : GMRES_SPMV_CSR;
    if (fmt64)
        *fmt64 = sell_fmt_for<double>(h, false) ? GMRES_SPMV_SLICED : GMRES_SPMV_CSR;
    return GMRES_OK;
}

gmres_status gmres_get_opts(gmres_t h, gmres_opts *o) {
    if (!h || !o)
        return GMRES_ERR_ARG;
    *o = h->opts;
    return GMRES_OK;
}

gmres_status gmres_solve(gmres_t h, const double *b, double *x, int32_t m, double tol,
                         gmres_ortho ortho, gmres_precision prec, int32_t maxiter,
                         gmres_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    gmres_info local;
    if (!info)
        info = &local;
    memset(info, 0, sizeof(*info));
    if (!h || !b || !x || m < 1 || m > MMAX || !(tol > 0) || maxiter < 0 ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_LIMITED)
        return GMRES_ERR_ARG;
    if (h->opts.precond == 2 && !h->ilu_ok)
        return GMRES_ERR_ARG;  // ILU(0) selected but not factored (gmres_ilu0)
    h->timer.on = h->opts.profile != 0;
    // Host buffers go through library-owned device copies.
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    const double *db = b;
    double *dx = x;
    if (!bdev || !xdev) {
        CK(h->xb.ensure((size_t)h->ldv * 8));
        CK(h->bb.ensure((size_t)h->ldv * 8));
    }
    if (!bdev) {
        CK(cudaMemcpyAsync(h->bb.p, b, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->stream));
        db = h->bb.as<double>();
    }
    if (!xdev) {
        CK(cudaMemcpyAsync(h->xb.p, x, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->stream));
        dx = h->xb.as<double>();
    }
    gmres_status st;
    if (h->opts.pv_mask != 0 &&
        (prec != GMRES_FP64 || h->split ||
         h->opts.path == GMRES_PATH_BLOCK)) {
        st = GMRES_ERR_ARG;  // the per-variable study: binary64 solves on the grid path
    } else switch (prec) {
    case GMRES_FP64:
        // the basis switch stores V as binary32 values
        if (h->opts.pv_mask & PV_V)
            st = solve_dispatch_path<double, float>(h, db, dx, m, tol, ortho, prec, maxiter,
                                                    info);
        else
            st = solve_dispatch_path<double, double>(h, db, dx, m, tol, ortho, prec, maxiter,
                                                     info);
        break;
    case GMRES_MIXED:
        st = solve_dispatch_path<float, float>(h, db, dx, m, tol, ortho, prec, maxiter, info);
        break;
    case GMRES_MIXED_BF16:
        st = solve_dispatch_path<float, __nv_bfloat16>(h, db, dx, m, tol, ortho, prec, maxiter,
                                                       info);
        break;
    case GMRES_MIXED_LIMITED:
        h->limited = true;
        st = solve_dispatch_path<double, float>(h, db, dx, m, tol, ortho, prec, maxiter, info);
        h->limited = false;
        break;
    default:
        st = solve_dispatch_path<float, __half>(h, db, dx, m, tol, ortho, prec, maxiter, info);
        break;
    }
    if (!xdev) {
        CK(cudaMemcpyAsync(x, dx, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->timer.on = false;
#ifdef GMRES_CHECKS
    if (check_word_take(h->stream) != 0)
        st = GMRES_ERR_INDEX;
#endif
    info->time_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

gmres_status gmres_spmv(gmres_t h, const void *x, void *y, gmres_precision prec) {
    if (!h || !x || !y || prec < GMRES_FP64 || prec > GMRES_MIXED_FP16)
        return GMRES_ERR_ARG;
    if (prec == GMRES_FP64 && sell_fmt_for<double>(h, false))
        CK(sell_spmv_plain<double>(h, (const double *)x, (double *)y));
    else if (prec != GMRES_FP64 && sell_fmt_for<float>(h, false))
        CK(sell_spmv_plain<float>(h, (const float *)x, (float *)y));
    else if (prec == GMRES_FP64)
        CK(launch_spmv_any<double>(h, h->opts.spmv_lanes ? h->opts.spmv_lanes : h->lanes64,
                                   (const double *)x, (double *)y));
    else
        CK(launch_spmv_any<float>(h, h->opts.spmv_lanes ? h->opts.spmv_lanes : h->lanes32,
                                  (const float *)x, (float *)y));
    CK(cudaStreamSynchronize(h->stream));
#ifdef GMRES_CHECKS
    if (check_word_take(h->stream) + sell_check_take(h->stream) != 0)
        return GMRES_ERR_INDEX;
#endif
    return GMRES_OK;
}

int32_t gmres_checks_enabled(void) {
#ifdef GMRES_CHECKS
    return 1;
#else
    return 0;
#endif
}

gmres_status gmres_residual(gmres_t h, const double *b, const double *x, double *z,
                            double *znorm) {
    if (!h || !b || !x)
        return GMRES_ERR_ARG;
    gmres_status st = ensure_workspace(h, 1, GMRES_FP64);
    if (st != GMRES_OK)
        return st;
    GridCtx<double, double> c = make_ctx<double, double>(h, 1);
    c.tol_abs = -1.0;
    c.pv = 0;  // plain binary64, whatever the per-variable switches
    CK(launch_residual(h, c, b, x, z, 0));
    st = read_ctl(h);
    if (st != GMRES_OK)
        return st;
    if (znorm)
        *znorm = h->hctl->rnorm;
    return GMRES_OK;
}

gmres_status gmres_backward_error(gmres_t h, const double *b, const double *x, double *eta) {
    if (!h || !b || !x || !eta || !is_device_ptr(b) || !is_device_ptr(x))
        return GMRES_ERR_ARG;
    gmres_status st = ensure_workspace(h, 1, GMRES_FP64);
    if (st != GMRES_OK)
        return st;
    GridCtx<double, double> c = make_ctx<double, double>(h, 1);
    c.tol_abs = -1.0;
    c.pv = 0;  // plain binary64, whatever the per-variable switches
    double *z = h->z.as<double>();
    CK(launch_residual(h, c, b, x, z, 0));
    ScopedBuf mx;
    CK(mx.ensure(4 * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(mx.p, 0, mx.bytes, h->stream));
    unsigned long long *m = mx.as<unsigned long long>();
    const int g = h->nsm * 4;
    const unsigned *hi = h->split ? split_hi(h) : nullptr, *lo = h->split ? split_lo(h) : nullptr;
    k_absmax<<<g, 256, 0, h->stream>>>(h->n, h->split ? nullptr : h->vals64.as<double>(),
                                        h->rowptr.as<int>(), hi, lo, m + 0);
    k_absmax<<<g, 256, 0, h->stream>>>(h->n, x, nullptr, nullptr, nullptr, m + 1);
    k_absmax<<<g, 256, 0, h->stream>>>(h->n, b, nullptr, nullptr, nullptr, m + 2);
    k_absmax<<<g, 256, 0, h->stream>>>(h->n, z, nullptr, nullptr, nullptr, m + 3);
    CKL();
    unsigned long long r[4];
    CK(cudaMemcpyAsync(r, m, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double v[4];
    memcpy(v, r, sizeof(v));
    const double den = v[0] * v[1] + v[2];
    *eta = den > 0 ? v[3] / den : 0.0;
    return GMRES_OK;
}

}  // extern "C"

namespace {

template <class T>
void export_small(const T *dev, double *host, size_t count, cudaStream_t st,
                  std::vector<T> &tmp) {
    tmp.resize(count);
    cudaMemcpyAsync(tmp.data(), dev, sizeof(T) * count, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    for (size_t i = 0; i < count; ++i)
        host[i] = (double)tmp[i];
}

template <class T, class VT>
gmres_status arnoldi_impl(gmres_handle *h, const double *r0, int m, int kmax, gmres_ortho ortho,
                          gmres_precision prec, double tau, double inner_abs, double *V,
                          double *Hbar, double *H, double *s, double *cs, double *sn, double *y,
                          double *u, double *arn, int32_t *jout, int32_t *breakdown) {
    gmres_status st = ensure_workspace(h, m, prec);
    if (st != GMRES_OK)
        return st;
    GridCtx<T, VT> c = make_ctx<T, VT>(h, m);
    c.tol_abs = -1.0;
    c.tau = tau;
    c.inner_abs = inner_abs;
    c.kmax = kmax;
    // one cycle from r0: only the per-variable switches inside the cycle act
    c.pv &= ~(unsigned)(PV_A_RESID | PV_B | PV_X | PV_AX);
    Acct acct;
    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
    // small arrays start at zero so unused entries export as zero
    CK(cudaMemsetAsync(h->small.p, 0, h->small.bytes, h->stream));
    // r = fl(r0): the residual kernel with x = 0 gives z = r0 exactly
    CK(cudaMemsetAsync(h->xb.p, 0, sizeof(double) * h->ldv, h->stream));
    CK(launch_residual(h, c, r0, h->xb.as<double>(), nullptr, 1));
    st = left_start<T, VT>(h, c, acct);
    if (st != GMRES_OK)
        return st;
    CK(cudaMemsetAsync(mon_hist(h), 0, (MMAX + 2) * sizeof(double), h->stream));
    k_init<T, VT><<<h->grid, kThreads, 0, h->stream>>>(c);
    CKL();
    std::vector<double> arnv;
    arnv.reserve(kmax);
    int j = 0;
    for (int it = 0; it < kmax; ++it) {
        st = enqueue_step(h, c, it, ortho, acct);
        if (st != GMRES_OK)
            return st;
        st = read_ctl(h);
        if (st != GMRES_OK)
            return st;
        if (h->hctl->j == it + 1) {
            arnv.push_back(h->hctl->arn);
            j = it + 1;
        }
        if (!h->hctl->active)
            break;
    }
    size_t sm = (size_t)m * m * sizeof(T) + (size_t)(m + 1) * sizeof(T);
    CK(cudaFuncSetAttribute(k_backsolve<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sm));
    k_backsolve<T, VT><<<1, 32, sm, h->stream>>>(c);
    CKL();
    k_update<T, VT><<<h->grid, kThreads, 0, h->stream>>>(c, h->z.as<double>(), 1);
    CKL();
    st = read_ctl(h);
    if (st != GMRES_OK)
        return st;
    std::vector<T> tmp;
    SmallPtrs<T> sp = small_ptrs<T>(h);
    const int ld = m + 1;
    if (Hbar)
        export_small(sp.Hb, Hbar, (size_t)ld * m, h->stream, tmp);
    if (H)
        export_small(sp.H, H, (size_t)ld * m, h->stream, tmp);
    if (s)
        export_small(sp.s, s, (size_t)m + 1, h->stream, tmp);
    if (cs)
        export_small(sp.cs, cs, (size_t)m, h->stream, tmp);
    if (sn)
        export_small(sp.sn, sn, (size_t)m, h->stream, tmp);
    if (y)
        export_small(sp.y, y, (size_t)m, h->stream, tmp);
    if (u) {
        if (c.pvals) {
            if (c.pvals_lim)
                CK((launch_spmv_plain<T, float>(h, lanes_for<T, VT>(h), c.pvals_lim, c.t, c.w)));
            else
                CK(launch_spmv_plain<T>(h, lanes_for<T, VT>(h), c.pvals, c.t, c.w));
            export_small(c.w, u, (size_t)h->n, h->stream, tmp);
        } else {
            export_small(c.t, u, (size_t)h->n, h->stream, tmp);
        }
    }
    if (arn) {
        for (int i = 0; i < m; ++i)
            arn[i] = i < (int)arnv.size() ? arnv[i] : 0.0;
    }
    if (V) {
        CK(h->z.ensure((size_t)h->n * (m + 1) * 8));
        CK(cudaMemsetAsync(h->z.p, 0, (size_t)h->n * (m + 1) * 8, h->stream));
        k_export_basis<T, VT><<<h->nsm * 4, 256, 0, h->stream>>>(c, std::min(j + 1, m + 1),
                                                                 h->z.as<double>());
        CKL();
        CK(cudaMemcpyAsync(V, h->z.p, (size_t)h->n * (m + 1) * 8, cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (jout)
        *jout = j;
    if (breakdown)
        *breakdown = h->hctl->breakdown;
    if (h->hctl->nonfinite)
        return GMRES_ERR_NONFINITE;
    return GMRES_OK;
}

// One inner iteration from a caller-given basis (gmres_arnoldi_step): the
// basis is loaded into the workspace, the control block says "cycle running,
// column ncols-1", and the same enqueue_step_core a solve uses runs once.
template <class T, class VT>
gmres_status arnoldi_step_impl(gmres_handle *h, const double *V, int ncols, gmres_ortho ortho,
                               gmres_precision prec, double *hcol, double *vnext) {
    const int m = ncols;  // the basis holds m + 1 = ncols + 1 vectors
    gmres_status st = ensure_workspace(h, m, prec);
    if (st != GMRES_OK)
        return st;
    GridCtx<T, VT> c = make_ctx<T, VT>(h, m);
    c.tol_abs = -1.0;
    c.tau = 0.0;
    c.inner_abs = -1.0;
    c.stall_factor = 0.0;
    c.kmax = m + 1;  // the Givens step must not end the cycle
    Acct acct;
    CK(cudaMemsetAsync(h->small.p, 0, h->small.bytes, h->stream));
    Ctl k0;
    memset(&k0, 0, sizeof(k0));
    k0.active = 1;
    k0.j = ncols - 1;
    k0.beta = 1.0;
    k0.arn = 1.0;
    CK(cudaMemcpyAsync(h->ctl.p, &k0, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
    const size_t vbytes = (size_t)h->n * (ncols + 1) * sizeof(double);
    CK(h->z.ensure(vbytes));
    CK(cudaMemcpyAsync(h->z.p, V, (size_t)h->n * ncols * sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    k_import_basis<T, VT><<<h->nsm * 4, 256, 0, h->stream>>>(c, ncols, h->z.as<double>());
    CKL();
    st = enqueue_step_core(h, c, ncols - 1, ortho, acct);
    if (st != GMRES_OK)
        return st;
    st = read_ctl(h);
    if (st != GMRES_OK)
        return st;
    std::vector<T> tmp;
    SmallPtrs<T> sp = small_ptrs<T>(h);
    export_small(sp.Hb + (size_t)(ncols - 1) * (m + 1), hcol, (size_t)ncols + 1, h->stream, tmp);
    if (vnext) {
        k_export_basis<T, VT><<<h->nsm * 4, 256, 0, h->stream>>>(c, ncols + 1, h->z.as<double>());
        CKL();
        CK(cudaMemcpyAsync(vnext, h->z.as<double>() + (size_t)ncols * h->n,
                           (size_t)h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (h->hctl->nonfinite)
        return GMRES_ERR_NONFINITE;
    if (h->hctl->breakdown)
        return GMRES_ERR_BREAKDOWN;
    return GMRES_OK;
}

}  // namespace

extern "C" {

gmres_status gmres_arnoldi(gmres_t h, const double *r0, int32_t m, int32_t kmax, gmres_ortho ortho,
                           gmres_precision prec, double tau, double inner_abs, double *V,
                           double *Hbar, double *H, double *s, double *cs, double *sn, double *y,
                           double *u, double *arn, int32_t *jout, int32_t *breakdown) {
    if (!h || !r0 || m < 1 || m > MMAX || kmax < 1 || kmax > m ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_LIMITED)
        return GMRES_ERR_ARG;
    h->timer.on = false;
    if (h->opts.pv_mask != 0 && (prec != GMRES_FP64 || h->split))
        return GMRES_ERR_ARG;
    switch (prec) {
    case GMRES_FP64:
        if (h->opts.pv_mask & PV_V)
            return arnoldi_impl<double, float>(h, r0, m, kmax, ortho, prec, tau, inner_abs, V,
                                               Hbar, H, s, cs, sn, y, u, arn, jout, breakdown);
        return arnoldi_impl<double, double>(h, r0, m, kmax, ortho, prec, tau, inner_abs, V, Hbar,
                                            H, s, cs, sn, y, u, arn, jout, breakdown);
    case GMRES_MIXED:
        return arnoldi_impl<float, float>(h, r0, m, kmax, ortho, prec, tau, inner_abs, V, Hbar, H,
                                          s, cs, sn, y, u, arn, jout, breakdown);
    case GMRES_MIXED_BF16:
        return arnoldi_impl<float, __nv_bfloat16>(h, r0, m, kmax, ortho, prec, tau, inner_abs, V,
                                                  Hbar, H, s, cs, sn, y, u, arn, jout, breakdown);
    case GMRES_MIXED_LIMITED: {
        h->limited = true;
        gmres_status st = arnoldi_impl<double, float>(h, r0, m, kmax, ortho, prec, tau, inner_abs,
                                                      V, Hbar, H, s, cs, sn, y, u, arn, jout,
                                                      breakdown);
        h->limited = false;
        return st;
    }
    default:
        return arnoldi_impl<float, __half>(h, r0, m, kmax, ortho, prec, tau, inner_abs, V, Hbar,
                                           H, s, cs, sn, y, u, arn, jout, breakdown);
    }
}

gmres_status gmres_arnoldi_step(gmres_t h, const double *V, int32_t ncols, gmres_ortho ortho,
                                gmres_precision prec, double *hcol, double *vnext) {
    if (!h || !V || !hcol || ncols < 1 || ncols > MMAX ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_LIMITED || h->split || h->opts.precond != 0 ||
        h->opts.pv_mask != 0)
        return GMRES_ERR_ARG;
    h->timer.on = false;
    switch (prec) {
    case GMRES_FP64:
        return arnoldi_step_impl<double, double>(h, V, ncols, ortho, prec, hcol, vnext);
    case GMRES_MIXED:
        return arnoldi_step_impl<float, float>(h, V, ncols, ortho, prec, hcol, vnext);
    case GMRES_MIXED_BF16:
        return arnoldi_step_impl<float, __nv_bfloat16>(h, V, ncols, ortho, prec, hcol, vnext);
    case GMRES_MIXED_LIMITED: {
        h->limited = true;
        gmres_status st = arnoldi_step_impl<double, float>(h, V, ncols, ortho, prec, hcol, vnext);
        h->limited = false;
        return st;
    }
    default:
        return arnoldi_step_impl<float, __half>(h, V, ncols, ortho, prec, hcol, vnext);
    }
}

gmres_status gmres_autotune(gmres_t h, int32_t *lanes32, int32_t *lanes64) {
    if (!h)
        return GMRES_ERR_ARG;
    gmres_status st = ensure_workspace(h, 1, GMRES_FP64);
    if (st != GMRES_OK)
        return st;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    const int cand[6] = {1, 2, 4, 8, 16, 32};
    float best32 = 1e30f, best64 = 1e30f;
    int L32 = h->lanes32, L64 = h->lanes64;
    double *x64 = h->r.as<double>(), *y64 = h->w.as<double>();
    float *x32 = h->r.as<float>(), *y32 = h->w.as<float>();
    for (int prec = 0; prec < 2; ++prec) {
        for (int ci = 0; ci < 6; ++ci) {
            const int L = cand[ci];
            for (int rep = 0; rep < 2; ++rep) {  // warm-up
                if (prec)
                    CK(launch_spmv_any<float>(h, L, x32, y32));
                else
                    CK(launch_spmv_any<double>(h, L, x64, y64));
            }
            CK(cudaEventRecord(a, h->stream));
            const int reps = 5;
            for (int rep = 0; rep < reps; ++rep) {
                if (prec)
                    CK(launch_spmv_any<float>(h, L, x32, y32));
                else
                    CK(launch_spmv_any<double>(h, L, x64, y64));
            }
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (prec && ms < best32) {
                best32 = ms;
                L32 = L;
            }
            if (!prec && ms < best64) {
                best64 = ms;
                L64 = L;
            }
        }
    }
    // the sliced copy of A, where it can be built: kept when it beats the
    // best CSR variant in either precision
    bool s32 = false, s64 = false;
    const bool had = h->sell_fmt != 0;
    if (!h->split && sell_build(h) == GMRES_OK) {
        for (int prec = 0; prec < 2; ++prec) {
            for (int rep = 0; rep < 2; ++rep) {  // warm-up
                if (prec)
                    CK(sell_spmv_plain<float>(h, x32, y32));
                else
                    CK(sell_spmv_plain<double>(h, x64, y64));
            }
            CK(cudaEventRecord(a, h->stream));
            const int reps = 5;
            for (int rep = 0; rep < reps; ++rep) {
                if (prec)
                    CK(sell_spmv_plain<float>(h, x32, y32));
                else
                    CK(sell_spmv_plain<double>(h, x64, y64));
            }
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (prec)
                s32 = ms < best32;
            else
                s64 = ms < best64;
        }
        // an explicitly requested copy stays; an unused one is released
        if (!s32 && !s64 && !(had && h->opts.spmv_format == GMRES_SPMV_SLICED))
            sell_free(h);
    }
    cudaGetLastError();  // a copy that did not fit is not an error here
    h->sell32 = s32;
    h->sell64 = s64;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->lanes32 = L32;
    h->lanes64 = L64;
    if (lanes32)
        *lanes32 = L32;
    if (lanes64)
        *lanes64 = L64;
    return GMRES_OK;
}

gmres_status gmres_memory_bytes(gmres_t h, int32_t m, gmres_precision prec, int64_t *matrix_bytes,
                                int64_t *workspace_bytes) {
    if (!h || m < 1 || m > MMAX || prec < GMRES_FP64 || prec > GMRES_MIXED_LIMITED)
        return GMRES_ERR_ARG;
    const int64_t n = h->n, nnz = h->nnz;
    // indices shared by both copies; binary64 + binary32 values (Sec. 4)
    if (matrix_bytes)
        *matrix_bytes =
            4 * (n + 1) + 4 * nnz + 8 * nnz + (h->split ? 0 : 4 * nnz) + sell_bytes(h);
    if (workspace_bytes) {
        const int64_t sT = (prec == GMRES_FP64 || prec == GMRES_MIXED_LIMITED) ? 8 : 4;
        *workspace_bytes = h->ldv * (m + 1) * elem_bytes(prec)  // basis
                           + 3 * h->ldv * sT                   // w, r, t
                           + 2 * (int64_t)(m + 1) * m * sT      // H, Hbar
                           + 6 * (int64_t)(m + 2) * sT;         // s, cs, sn, y, h1, h2
    }
    return GMRES_OK;
}

gmres_status gmres_ilu0(gmres_t h) {
    if (!h || h->split)
        return GMRES_ERR_ARG;
    if (h->nnz == 0)
        return GMRES_ERR_ARG;
    return ilu_factor(h);
}

gmres_status gmres_ilu_levels(gmres_t h, int32_t *lower, int32_t *upper) {
    if (!h || !lower || !upper || !h->ilu_ok)
        return GMRES_ERR_ARG;
    *lower = h->ilu_levels;
    *upper = h->ilu_ulevels;
    return GMRES_OK;
}

gmres_status gmres_ilu_factors(gmres_t h, double *lu) {
    if (!h || !lu || !h->ilu_ok)
        return GMRES_ERR_ARG;
    CK(cudaMemcpyAsync(lu, h->ilu64.p, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

gmres_status gmres_ilu_apply(gmres_t h, const void *z, void *out, gmres_precision prec) {
    if (!h || !z || !out || !h->ilu_ok || prec < GMRES_FP64 || prec > GMRES_MIXED_LIMITED)
        return GMRES_ERR_ARG;
    CK(h->ctl.ensure(sizeof(Ctl)));
    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
    ScopedBuf tmp;
    CK(tmp.ensure(sizeof(double) * h->n));
    int *err = &h->ctl.as<Ctl>()->timeout;
    if (prec == GMRES_FP64)
        CK((ilu_apply<double, double>(h, h->ilu64.as<double>(), (const double *)z,
                                      tmp.as<double>(), (double *)out, err)));
    else
        CK((ilu_apply<float, float>(h, h->ilu32.as<float>(), (const float *)z, tmp.as<float>(),
                                    (float *)out, err)));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return bad ? GMRES_ERR_TIMEOUT : GMRES_OK;
}

gmres_status gmres_orth_norms(gmres_t h, double *out, int32_t count) {
    if (!h || !out || count < 0 || count > MMAX)
        return GMRES_ERR_ARG;
    if (count == 0)
        return GMRES_OK;
    if (h->mon.bytes < MON_DOUBLES * sizeof(double)) {
        memset(out, 0, sizeof(double) * (size_t)count);
        return GMRES_OK;
    }
    CK(cudaMemcpyAsync(out, mon_hist(h), sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

}  // extern "C"
