// noalloc.cu -- a GMRES solve that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: cudaMalloc and cudaFree may synchronise the whole device (stalling
// every other stream of a time-stepping code), and some frameworks own the
// entire device budget through their own allocator.  gmres_solve_noalloc
// serves them: it runs the single-block whole-solve kernel of the block path
// on the caller's device arrays, and takes every byte of workspace -- the
// Krylov basis, the work vectors, the binary32 copy of A's values, the result
// record -- from one file-scope device array of GMRES_NOALLOC_SCRATCH_BYTES.
// That array exists on every GPU that loads the library, for the life of the
// process.  All calls share it, so calls that overlap on the GPU (different
// streams, different host threads) race on it and must be serialised by the
// caller; each call overwrites what the previous one left there.  Every call
// waits for its stream to finish before it returns: it reads rowptr's end
// points and the result record back to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/gmres_gb300.h"
#include "block_solver.cuh"
#include "host_util.hpp"

using namespace gmres;
using namespace gmres_host;

namespace {

constexpr size_t kScratchBytes = GMRES_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in).
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {nullptr};

gmres_status scratch_address(void **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return GMRES_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "gmres_solve_noalloc: cudaGetSymbolAddress failed: %s\n",
                    cudaGetErrorString(e));
            return GMRES_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GMRES_OK;
}

__global__ void k_noalloc_cast(int64_t nnz, const double *a, float *b) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

// The block-path solver for one system passed by value (no descriptor array).
template <class T, class VT, int L>
__global__ void __launch_bounds__(1024) k_noalloc_solve(BlockSys<T, VT> S, BlockParams P,
                                                        BlockResult *res) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    block_solve_one<T, VT, L>(S, P, res, smem_raw);
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

template <class T, class VT>
gmres_status run(int n, int64_t nnz, const int32_t *rowptr, const int32_t *colind,
                 const double *vals, const double *b, double *x, int m, double tol,
                 gmres_ortho ortho, gmres_precision prec, int maxiter, cudaStream_t stream,
                 gmres_info *info) {
    const int64_t ldv = round_up(n, 64);
    const bool narrow = !std::is_same<T, double>::value;
    const size_t off_a = 256;
    const size_t off_v = off_a + (narrow ? up256((size_t)nnz * sizeof(float)) : 0);
    const size_t off_w = off_v + up256((size_t)ldv * (m + 1) * sizeof(VT));
    const size_t off_r = off_w + up256((size_t)ldv * sizeof(T));
    const size_t need = off_r + up256((size_t)ldv * sizeof(T));
    if (need > kScratchBytes) {
        fprintf(stderr,
                "gmres_solve_noalloc: system needs %zu bytes of workspace, more than the "
                "%zu-byte scratch (n = %d, nnz = %lld, m = %d)\n",
                need, kScratchBytes, n, (long long)nnz, m);
        return GMRES_ERR_ARG;
    }
    unsigned char *base = nullptr;
    gmres_status st = scratch_address(reinterpret_cast<void **>(&base));
    if (st != GMRES_OK)
        return st;
    BlockResult *res = reinterpret_cast<BlockResult *>(base);
    CK(cudaMemsetAsync(res, 0, sizeof(BlockResult), stream));
    BlockSys<T, VT> S;
    S.n = n;
    S.ldv = ldv;
    S.rowptr = rowptr;
    S.colind = colind;
    if (narrow) {
        float *a32 = reinterpret_cast<float *>(base + off_a);
        k_noalloc_cast<<<64, 256, 0, stream>>>(nnz, vals, a32);
        CKL();
        S.a = reinterpret_cast<const T *>(a32);
    } else {
        S.a = reinterpret_cast<const T *>(vals);
    }
    S.a64 = vals;
    S.b = b;
    S.x = x;
    S.V = reinterpret_cast<VT *>(base + off_v);
    S.w = reinterpret_cast<T *>(base + off_w);
    S.r = reinterpret_cast<T *>(base + off_r);
    S.vscale = std::is_same<VT, __half>::value ? fp16_scale(n) : 1.0f;
    S.vinv = 1.0f / S.vscale;
    BlockParams P;
    P.m = m;
    P.maxiter = maxiter;
    P.ortho = (int)ortho;
    P.repeat_first = prec == GMRES_FP64 ? 0 : 1;
    P.tol = tol;
    P.tau = default_tau(prec);
    P.inner_factor = 0.5;
    P.brk = narrow ? 1e-6 : 1e-14;
    P.nsys = 1;
    P.queue = nullptr;
    P.order = nullptr;
    const int L = pow2_lanes((double)nnz / n / 2.0);
    void (*kfn)(BlockSys<T, VT>, BlockParams, BlockResult *) = nullptr;
    switch (L) {
    case 1: kfn = &k_noalloc_solve<T, VT, 1>; break;
    case 2: kfn = &k_noalloc_solve<T, VT, 2>; break;
    case 4: kfn = &k_noalloc_solve<T, VT, 4>; break;
    case 8: kfn = &k_noalloc_solve<T, VT, 8>; break;
    case 16: kfn = &k_noalloc_solve<T, VT, 16>; break;
    default: kfn = &k_noalloc_solve<T, VT, 32>; break;
    }
    const size_t smem = block_smem_bytes<T>(m);
    CK(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(64, round_up(n / 4, 32)));
    kfn<<<1, threads, smem, stream>>>(S, P, res);
    CKL();
    BlockResult R;
    CK(cudaMemcpyAsync(&R, res, sizeof(R), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (info) {
        info->iters = R.iters;
        info->restarts = R.restarts;
        info->converged = R.converged;
        info->first_len = R.first_len;
        info->relres = R.relres;
        info->bnorm = R.bnorm;
        info->path = GMRES_PATH_BLOCK;
        info->launches = narrow ? 2 : 1;
        info->kernel_launches[GMRES_K_BLOCK] = 1;
    }
    return (gmres_status)R.status;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gmres_status gmres_solve_noalloc(int32_t n, const int32_t *rowptr,
                                            const int32_t *colind, const double *vals,
                                            int64_t nnz, const double *b, double *x, int32_t m,
                                            double tol, gmres_ortho ortho, gmres_precision prec,
                                            int32_t maxiter, void *stream, gmres_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    if (info)
        memset(info, 0, sizeof(*info));
    if (n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colind || !vals)) || !b || !x || m < 1 ||
        m > MMAX || !(tol > 0) || maxiter < 0 ||
        (ortho != GMRES_ORTHO_MGS && ortho != GMRES_ORTHO_CGSR) || prec < GMRES_FP64 ||
        prec > GMRES_MIXED_FP16)
        return GMRES_ERR_ARG;
    if (!on_device(rowptr) || (nnz > 0 && (!on_device(colind) || !on_device(vals))) ||
        !on_device(b) || !on_device(x))
        return GMRES_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // rowptr[0] and rowptr[n] against the stated nonzero count: the kernels
    // read rowptr[n] entries of colind and vals, and the binary32 copy in the
    // scratch holds nnz of them (two 4-byte reads; the call synchronises its
    // stream at the end anyway)
    int32_t ends[2] = {-1, -1};
    if (cudaMemcpyAsync(&ends[0], rowptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&ends[1], rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GMRES_ERR_CUDA;
    }
    if (ends[0] != 0 || (int64_t)ends[1] != nnz) {
        fprintf(stderr, "gmres_solve_noalloc: rowptr[0] = %d, rowptr[n] = %d, nnz = %lld\n",
                ends[0], ends[1], (long long)nnz);
        return GMRES_ERR_ARG;
    }
    gmres_status st;
    switch (prec) {
    case GMRES_FP64:
        st = run<double, double>(n, nnz, rowptr, colind, vals, b, x, m, tol, ortho, prec, maxiter,
                                 s, info);
        break;
    case GMRES_MIXED:
        st = run<float, float>(n, nnz, rowptr, colind, vals, b, x, m, tol, ortho, prec, maxiter,
                               s, info);
        break;
    case GMRES_MIXED_BF16:
        st = run<float, __nv_bfloat16>(n, nnz, rowptr, colind, vals, b, x, m, tol, ortho, prec,
                                       maxiter, s, info);
        break;
    default:
        st = run<float, __half>(n, nnz, rowptr, colind, vals, b, x, m, tol, ortho, prec, maxiter,
                                s, info);
        break;
    }
#ifdef GMRES_CHECKS
    if (st != GMRES_ERR_CUDA && check_word_take(s) != 0)
        st = GMRES_ERR_INDEX;
#endif
    if (info)
        info->time_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
    return st;
}
