// batch.cu -- batched restarted GMRES(m): many independent systems of uneven
// size solved in one persistent launch (C-ABI gmres_batch_*, declared in
// include/gmres_gb300.h).
//
// The systems are the diagonal blocks of one CSR matrix.  Each thread block
// of a persistent grid takes the next system from a device work queue
// (largest first, so the long solves start early) and runs the whole
// restarted solve of Algorithm 1 for it with block-wide reductions
// (block_solver.cuh).  Converged systems leave the queue for good, so the
// grid's remaining blocks keep working on the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "block_solver.cuh"
#include "team_launch.hpp"
#include "host_util.hpp"

using namespace gmres;
using namespace gmres_host;

// Systems of at least this many rows are solved by a cluster of CLUSTER_CTAS
// thread blocks (distributed-shared-memory reductions); smaller ones by one
// block.  Both launches run concurrently, each over its own work queue.
constexpr int CLUSTER_MIN_ROWS = 8192;
constexpr int CLUSTER_CTAS = 8;
// Threads per block of the cluster launch (the one-block launch uses 256).
// More threads give the large systems' clusters fewer rows per thread (a
// shorter latency chain per inner iteration) but fewer clusters at once;
// measured on 2048 uneven systems, 256 is fastest.
constexpr int CLUSTER_THREADS = 256;

struct gmres_batch {
    int nsys = 0;
    int64_t nrows = 0, nnz = 0;
    cudaStream_t stream = nullptr;
    int nsm = 0;
    double avg_row = 1.0;
    std::vector<int64_t> sys_ptr;   // host copy
    std::vector<int64_t> ws_ofs;    // padded row offset of each system's workspace
    int64_t ws_rows = 0;            // total padded rows
    std::vector<int> order;         // largest system first
    int nlarge = 0;                 // systems solved by clusters (the first nlarge of order)
    int tuned_lanes = 0;            // lanes per row chosen by gmres_batch_autotune (0: none)
    int cluster_threads = CLUSTER_THREADS;  // threads per block of the cluster launch
    cudaStream_t aux = nullptr;     // stream of the cluster launch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DevBuf rowptr, colind, vals64, vals32;
    DevBuf V, w, r, xb, bb, sys, res, ord, queue;
};


// The systems of at least min_rows rows (0: none) go to clusters: they are
// the first nlarge entries of the largest-first order.
void set_nlarge(gmres_batch *B, int64_t min_rows) {
    B->nlarge = 0;
    if (min_rows <= 0)
        return;
    for (int i = 0; i < B->nsys; ++i) {
        const int s = B->order[i];
        if (B->sys_ptr[s + 1] - B->sys_ptr[s] >= min_rows)
            B->nlarge = i + 1;
    }
}

namespace {

__global__ void k_batch_cast(int64_t nnz, const double *a, float *b) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}



template <class T, class VT>
gmres_status batch_run(gmres_batch *B, const double *db, double *dx, int m, double tol,
                       gmres_ortho ortho, gmres_precision prec, int maxiter, int lanes,
                       gmres_batch_result *results, gmres_info *info) {
    const double sv = sizeof(VT), st = sizeof(T);
    CK(B->V.ensure((size_t)B->ws_rows * (m + 1) * sizeof(VT)));
    CK(B->w.ensure((size_t)B->ws_rows * 8));
    CK(B->r.ensure((size_t)B->ws_rows * 8));
    std::vector<BlockSys<T, VT>> S(B->nsys);
    const int *rp = B->rowptr.as<int>();
    for (int i = 0; i < B->nsys; ++i) {
        const int64_t r0 = B->sys_ptr[i];
        BlockSys<T, VT> &s = S[i];
        s.n = (int)(B->sys_ptr[i + 1] - r0);
        s.ldv = round_up(s.n, 32);
        s.rowptr = rp + r0;
        s.colind = B->colind.as<int>();
        s.a = std::is_same<T, double>::value ? reinterpret_cast<const T *>(B->vals64.p)
                                             : reinterpret_cast<const T *>(B->vals32.p);
        s.a64 = B->vals64.as<double>();
        s.b = db + r0;
        s.x = dx + r0;
        s.V = B->V.as<VT>() + (size_t)B->ws_ofs[i] * (m + 1);
        s.w = B->w.as<T>() + B->ws_ofs[i];
        s.r = B->r.as<T>() + B->ws_ofs[i];
        s.vscale = std::is_same<VT, __half>::value ? fp16_scale(s.n) : 1.0f;
        s.vinv = 1.0f / s.vscale;
    }
    CK(B->sys.ensure(sizeof(BlockSys<T, VT>) * B->nsys));
    CK(B->res.ensure(sizeof(BlockResult) * B->nsys));
    CK(cudaMemcpyAsync(B->sys.p, S.data(), sizeof(BlockSys<T, VT>) * B->nsys,
                       cudaMemcpyHostToDevice, B->stream));
    BlockParams P;
    P.m = m;
    P.maxiter = maxiter;
    P.ortho = (int)ortho;
    P.repeat_first = prec == GMRES_FP64 ? 0 : 1;
    P.tol = tol;
    P.tau = default_tau(prec);
    P.inner_factor = 0.5;
    P.brk = std::is_same<T, double>::value ? 1e-14 : 1e-6;
    P.nsys = B->nsys;
    P.queue = nullptr;
    P.order = nullptr;
    const int L = lanes > 0 ? lanes
                  : (B->tuned_lanes > 0 ? B->tuned_lanes : pow2_lanes(B->avg_row / 2.0));
    using KFn = void (*)(const BlockSys<T, VT> *, BlockParams, BlockResult *);
    KFn kfn = nullptr, kcl = nullptr;
    // 256-thread launches: the instantiations bounded for several resident
    // blocks per SM; other cluster widths: the plain bound
    const bool c256 = B->cluster_threads == 256;
    switch (L) {
    case 1:
        kfn = &k_block_solve<T, VT, 1, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 1, CLUSTER_CTAS, 256> : &k_team_solve<T, VT, 1, CLUSTER_CTAS>;
        break;
    case 2:
        kfn = &k_block_solve<T, VT, 2, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 2, CLUSTER_CTAS, 256> : &k_team_solve<T, VT, 2, CLUSTER_CTAS>;
        break;
    case 4:
        kfn = &k_block_solve<T, VT, 4, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 4, CLUSTER_CTAS, 256> : &k_team_solve<T, VT, 4, CLUSTER_CTAS>;
        break;
    case 8:
        kfn = &k_block_solve<T, VT, 8, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 8, CLUSTER_CTAS, 256> : &k_team_solve<T, VT, 8, CLUSTER_CTAS>;
        break;
    case 16:
        kfn = &k_block_solve<T, VT, 16, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 16, CLUSTER_CTAS, 256>
                   : &k_team_solve<T, VT, 16, CLUSTER_CTAS>;
        break;
    default:
        kfn = &k_block_solve<T, VT, 32, 256>;
        kcl = c256 ? &k_team_solve<T, VT, 32, CLUSTER_CTAS, 256>
                   : &k_team_solve<T, VT, 32, CLUSTER_CTAS>;
        break;
    }
    const size_t smem = block_smem_bytes<T>(m);
    CK(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CK(cudaFuncSetAttribute(kcl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = 256;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
    per_sm = std::max(1, per_sm);
    const int nsmall = B->nsys - B->nlarge;
    unsigned *q = B->queue.as<unsigned>();
    const int *ord = B->ord.as<int>();
    // cluster launch for the large systems (the first nlarge entries of order)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    int ncl = 0;
    if (B->nlarge > 0) {
        cfg.blockDim = dim3(B->cluster_threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = B->aux;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CLUSTER_CTAS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(CLUSTER_CTAS * B->nsm);
        CK(cudaOccupancyMaxActiveClusters(&ncl, kcl, &cfg));
        ncl = std::max(1, std::min(ncl, B->nlarge));
        cfg.gridDim = dim3(CLUSTER_CTAS * ncl);
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaMemsetAsync(q, 0, 2 * sizeof(unsigned), B->stream));
    CK(cudaEventRecord(e0, B->stream));
    if (B->nlarge > 0) {
        BlockParams PL = P;
        PL.nsys = B->nlarge;
        PL.queue = q + 1;
        PL.order = ord;
        CK(cudaEventRecord(B->ev_fork, B->stream));
        CK(cudaStreamWaitEvent(B->aux, B->ev_fork, 0));
        CK(cudaLaunchKernelEx(&cfg, kcl, (const BlockSys<T, VT> *)B->sys.as<BlockSys<T, VT>>(),
                              PL, B->res.as<BlockResult>()));
        CK(cudaEventRecord(B->ev_join, B->aux));
    }
    if (nsmall > 0) {
        BlockParams PS = P;
        PS.nsys = nsmall;
        PS.queue = q;
        PS.order = ord + B->nlarge;
        const int grid = std::min<int64_t>(nsmall, (int64_t)B->nsm * per_sm);
        kfn<<<grid, threads, smem, B->stream>>>(B->sys.as<BlockSys<T, VT>>(), PS,
                                                 B->res.as<BlockResult>());
        CKL();
    }
    if (B->nlarge > 0)
        CK(cudaStreamWaitEvent(B->stream, B->ev_join, 0));
    CK(cudaEventRecord(e1, B->stream));
    std::vector<BlockResult> R(B->nsys);
    CK(cudaMemcpyAsync(R.data(), B->res.p, sizeof(BlockResult) * B->nsys,
                       cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gmres_status worst = GMRES_OK;
    int all_conv = 1;
    int64_t iters = 0, restarts = 0;
    double bytes = 0;
    for (int i = 0; i < B->nsys; ++i) {
        if (results) {
            results[i].iters = R[i].iters;
            results[i].restarts = R[i].restarts;
            results[i].converged = R[i].converged;
            results[i].status = R[i].status;
            results[i].relres = R[i].relres;
        }
        iters += R[i].iters;
        restarts += R[i].restarts;
        all_conv &= R[i].converged;
        const gmres_status s = (gmres_status)R[i].status;
        if (s < 0 && (worst >= 0))
            worst = s;
        else if (s == GMRES_MAXITER && worst == GMRES_OK)
            worst = GMRES_MAXITER;
        // algorithmic bytes of this system's solve (SpMV + orthogonalisation
        // per inner step, residual per cycle), for the aggregate GB/s
        const double n = (double)(B->sys_ptr[i + 1] - B->sys_ptr[i]);
        const double nz = n * B->avg_row;
        const double cycles = R[i].restarts, it = R[i].iters;
        const double avgc = cycles > 0 ? (it / cycles + 1) / 2 : 0;  // mean basis size
        const double orth = ortho == GMRES_ORTHO_CGSR ? 3 * avgc * n * sv + 5 * n * st
                                                      : avgc * n * sv + 2 * n * st;
        bytes += it * (nz * (st + 4) + 4 * n + n * sv + n * st + orth + n * st + n * sv) +
                 (cycles + 1) * (12 * nz + 4 * n + 24 * n);
    }
    if (info) {
        info->iters = (int32_t)std::min<int64_t>(iters, INT32_MAX);
        info->restarts = (int32_t)std::min<int64_t>(restarts, INT32_MAX);
        info->converged = all_conv;
        info->kernel_ms[GMRES_K_BLOCK] = ms;
        info->kernel_bytes[GMRES_K_BLOCK] = bytes;
        info->kernel_launches[GMRES_K_BLOCK] = (B->nlarge > 0) + (B->nsys - B->nlarge > 0);
        info->launches = info->kernel_launches[GMRES_K_BLOCK];
        info->path = GMRES_PATH_BLOCK;
    }
    return worst;
}

}  // namespace

namespace gmres {

template <class T, class VT>
cudaError_t launch_team_single(const BlockSys<T, VT> *sys, const BlockParams &P,
                               BlockResult *res, int L, int threads, size_t smem,
                               cudaStream_t stream) {
    using KFn = void (*)(const BlockSys<T, VT> *, BlockParams, BlockResult *);
    KFn k = nullptr;
    switch (L) {
    case 1: k = &k_team_solve<T, VT, 1, TEAM_SINGLE_CTAS>; break;
    case 2: k = &k_team_solve<T, VT, 2, TEAM_SINGLE_CTAS>; break;
    case 4: k = &k_team_solve<T, VT, 4, TEAM_SINGLE_CTAS>; break;
    case 8: k = &k_team_solve<T, VT, 8, TEAM_SINGLE_CTAS>; break;
    case 16: k = &k_team_solve<T, VT, 16, TEAM_SINGLE_CTAS>; break;
    default: k = &k_team_solve<T, VT, 32, TEAM_SINGLE_CTAS>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = TEAM_SINGLE_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(TEAM_SINGLE_CTAS);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, sys, P, res);
}

template cudaError_t launch_team_single<double, double>(const BlockSys<double, double> *,
                                                        const BlockParams &, BlockResult *, int,
                                                        int, size_t, cudaStream_t);
template cudaError_t launch_team_single<double, float>(const BlockSys<double, float> *,
                                                       const BlockParams &, BlockResult *, int,
                                                       int, size_t, cudaStream_t);
template cudaError_t launch_team_single<float, float>(const BlockSys<float, float> *,
                                                      const BlockParams &, BlockResult *, int, int,
                                                      size_t, cudaStream_t);
template cudaError_t launch_team_single<float, __nv_bfloat16>(
    const BlockSys<float, __nv_bfloat16> *, const BlockParams &, BlockResult *, int, int, size_t,
    cudaStream_t);
template cudaError_t launch_team_single<float, __half>(const BlockSys<float, __half> *,
                                                       const BlockParams &, BlockResult *, int,
                                                       int, size_t, cudaStream_t);

}  // namespace gmres

extern "C" {

gmres_status gmres_batch_create(gmres_batch_t *out, int32_t nsys, const int64_t *sys_ptr,
                                const int32_t *rowptr, const int32_t *colind, const double *vals,
                                void *stream) {
    if (!out)
        return GMRES_ERR_ARG;
    *out = nullptr;
    if (nsys <= 0 || !sys_ptr || !rowptr)
        return GMRES_ERR_ARG;
    if (sys_ptr[0] != 0)
        return GMRES_ERR_ARG;
    for (int i = 0; i < nsys; ++i)
        if (sys_ptr[i + 1] <= sys_ptr[i] || sys_ptr[i + 1] - sys_ptr[i] > INT32_MAX)
            return GMRES_ERR_ARG;
    const int64_t nrows = sys_ptr[nsys];
    const int64_t nnz = rowptr[nrows];
    if (nnz < 0 || (nnz > 0 && (!colind || !vals)))
        return GMRES_ERR_ARG;
    gmres_status stc = check_csr_host(nrows, rowptr, colind, nnz, nrows);
    if (stc != GMRES_OK)
        return stc;
    // columns must stay inside their system; store them system-local
    std::vector<int32_t> local(nnz);
    for (int i = 0; i < nsys; ++i) {
        const int64_t r0 = sys_ptr[i], r1 = sys_ptr[i + 1];
        for (int64_t r = r0; r < r1; ++r)
            for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
                if (colind[k] < r0 || colind[k] >= r1)
                    return GMRES_ERR_ARG;
                local[k] = (int32_t)(colind[k] - r0);
            }
    }
    for (int64_t k = 0; k < nnz; ++k)
        if (!std::isfinite(vals[k]))
            return GMRES_ERR_NONFINITE;
    gmres_batch *B = new (std::nothrow) gmres_batch();
    if (!B)
        return GMRES_ERR_OOM;
    auto fail = [&](gmres_status s) {
        gmres_batch_destroy(B);
        return s;
    };
    B->nsys = nsys;
    B->nrows = nrows;
    B->nnz = nnz;
    B->stream = reinterpret_cast<cudaStream_t>(stream);
    B->avg_row = nrows > 0 ? (double)nnz / nrows : 1.0;
    B->sys_ptr.assign(sys_ptr, sys_ptr + nsys + 1);
    B->ws_ofs.resize(nsys);
    int64_t ofs = 0;
    for (int i = 0; i < nsys; ++i) {
        B->ws_ofs[i] = ofs;
        ofs += round_up(sys_ptr[i + 1] - sys_ptr[i], 32);
    }
    B->ws_rows = ofs;
    B->order.resize(nsys);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) {
        return (sys_ptr[a + 1] - sys_ptr[a]) > (sys_ptr[b + 1] - sys_ptr[b]);
    });
    set_nlarge(B, CLUSTER_MIN_ROWS);
    if (cudaStreamCreateWithFlags(&B->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    if (B->rowptr.ensure(sizeof(int32_t) * (nrows + 1)) != cudaSuccess ||
        B->colind.ensure(sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        B->vals64.ensure(sizeof(double) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        B->vals32.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)) != cudaSuccess ||
        B->ord.ensure(sizeof(int) * nsys) != cudaSuccess ||
        B->queue.ensure(sizeof(unsigned) * 4) != cudaSuccess)
        return fail(GMRES_ERR_OOM);
    if (cudaMemcpyAsync(B->rowptr.p, rowptr, sizeof(int32_t) * (nrows + 1),
                        cudaMemcpyHostToDevice, B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->colind.p, local.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->vals64.p, vals, sizeof(double) * nnz, cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess ||
        cudaMemcpyAsync(B->ord.p, B->order.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice,
                        B->stream) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    k_batch_cast<<<B->nsm * 4, 256, 0, B->stream>>>(nnz, B->vals64.as<double>(),
                                                     B->vals32.as<float>());
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(B->stream) != cudaSuccess)
        return fail(GMRES_ERR_CUDA);
    *out = B;
    return GMRES_OK;
}

void gmres_batch_destroy(gmres_batch_t B) {
    if (!B)
        return;
    if (B->stream)
        cudaStreamSynchronize(B->stream);
    else
        cudaDeviceSynchronize();
    if (B->aux)
        cudaStreamSynchronize(B->aux);
    for (DevBuf *b : {&B->rowptr, &B->colind, &B->vals64, &B->vals32, &B->V, &B->w, &B->r,
                      &B->xb, &B->bb, &B->sys, &B->res, &B->ord, &B->queue})
        b->release();
    if (B->ev_fork)
        cudaEventDestroy(B->ev_fork);
    if (B->ev_join)
        cudaEventDestroy(B->ev_join);
    if (B->aux)
        cudaStreamDestroy(B->aux);
    delete B;
}

gmres_status gmres_batch_solve(gmres_batch_t B, const double *rhs, double *x, int32_t m,
                               double tol, gmres_ortho ortho, gmres_precision prec,
                               int32_t maxiter, int32_t lanes, gmres_batch_result *results,
                               gmres_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    if (info)
        memset(info, 0, sizeof(*info));
    if (!B || !rhs || !x || m < 1 || m > MMAX || !(tol > 0) || maxiter < 0 ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_FP16 || lanes < 0 || lanes > 32 || (lanes & (lanes - 1)))
        return GMRES_ERR_ARG;
    const bool bdev = is_device_ptr(rhs), xdev = is_device_ptr(x);
    const double *db = rhs;
    double *dx = x;
    if (!bdev) {
        CK(B->bb.ensure(sizeof(double) * B->nrows));
        CK(cudaMemcpyAsync(B->bb.p, rhs, sizeof(double) * B->nrows, cudaMemcpyHostToDevice,
                           B->stream));
        db = B->bb.as<double>();
    }
    if (!xdev) {
        CK(B->xb.ensure(sizeof(double) * B->nrows));
        CK(cudaMemcpyAsync(B->xb.p, x, sizeof(double) * B->nrows, cudaMemcpyHostToDevice,
                           B->stream));
        dx = B->xb.as<double>();
    }
    gmres_status st;
    switch (prec) {
    case GMRES_FP64:
        st = batch_run<double, double>(B, db, dx, m, tol, ortho, prec, maxiter, lanes, results,
                                       info);
        break;
    case GMRES_MIXED:
        st = batch_run<float, float>(B, db, dx, m, tol, ortho, prec, maxiter, lanes, results,
                                     info);
        break;
    case GMRES_MIXED_BF16:
        st = batch_run<float, __nv_bfloat16>(B, db, dx, m, tol, ortho, prec, maxiter, lanes,
                                             results, info);
        break;
    default:
        st = batch_run<float, __half>(B, db, dx, m, tol, ortho, prec, maxiter, lanes, results,
                                      info);
        break;
    }
    if (!xdev) {
        CK(cudaMemcpyAsync(x, dx, sizeof(double) * B->nrows, cudaMemcpyDeviceToHost, B->stream));
        CK(cudaStreamSynchronize(B->stream));
    }
#ifdef GMRES_CHECKS
    if (st != GMRES_ERR_CUDA && check_word_take(B->stream) != 0)
        st = GMRES_ERR_INDEX;
#endif
    if (info)
        info->time_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
    return st;
}

gmres_status gmres_batch_set_cluster_rows(gmres_batch_t B, int32_t min_rows) {
    if (!B || min_rows < 0)
        return GMRES_ERR_ARG;
    set_nlarge(B, min_rows);
    return GMRES_OK;
}

gmres_status gmres_batch_set_cluster_threads(gmres_batch_t B, int32_t threads) {
    if (!B || (threads != 128 && threads != 256 && threads != 512 && threads != 1024))
        return GMRES_ERR_ARG;
    B->cluster_threads = threads;
    return GMRES_OK;
}

gmres_status gmres_batch_autotune(gmres_batch_t B, const double *rhs, int32_t m,
                                  gmres_ortho ortho, gmres_precision prec, int32_t iters,
                                  int32_t *lanes_out) {
    if (!B || !rhs || m < 1 || m > MMAX || iters < 1 ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_FP16)
        return GMRES_ERR_ARG;
    // every candidate runs the same capped solve from x0 = 0 on a scratch x
    DevBuf xs;
    CK(xs.ensure(sizeof(double) * B->nrows));
    const double *db = rhs;
    if (!is_device_ptr(rhs)) {
        CK(B->bb.ensure(sizeof(double) * B->nrows));
        CK(cudaMemcpyAsync(B->bb.p, rhs, sizeof(double) * B->nrows, cudaMemcpyHostToDevice,
                           B->stream));
        db = B->bb.as<double>();
    }
    int best = 0;
    double best_ms = 0;
    for (int L = 1; L <= 16; L *= 2) {
        CK(cudaMemsetAsync(xs.p, 0, sizeof(double) * B->nrows, B->stream));
        gmres_info inf;
        memset(&inf, 0, sizeof(inf));
        gmres_status st;
        double *dx = xs.as<double>();
        // tol below reach: every system runs the full iteration budget
        switch (prec) {
        case GMRES_FP64:
            st = batch_run<double, double>(B, db, dx, m, 1e-300, ortho, prec, iters, L, nullptr,
                                           &inf);
            break;
        case GMRES_MIXED:
            st = batch_run<float, float>(B, db, dx, m, 1e-300, ortho, prec, iters, L, nullptr,
                                         &inf);
            break;
        case GMRES_MIXED_BF16:
            st = batch_run<float, __nv_bfloat16>(B, db, dx, m, 1e-300, ortho, prec, iters, L,
                                                 nullptr, &inf);
            break;
        default:
            st = batch_run<float, __half>(B, db, dx, m, 1e-300, ortho, prec, iters, L, nullptr,
                                          &inf);
            break;
        }
        if (st != GMRES_OK && st != GMRES_MAXITER && st != GMRES_ERR_BREAKDOWN)
            return st;
        const double ms = inf.kernel_ms[GMRES_K_BLOCK];
        if (best == 0 || ms < best_ms) {
            best = L;
            best_ms = ms;
        }
    }
    B->tuned_lanes = best;
    if (lanes_out)
        *lanes_out = best;
    return GMRES_OK;
}

}  // extern "C"
