// sell.cu -- A's sliced storage (SELL-32, sell.cuh): built on the device
// from the CSR arrays the handle holds, and the plain product in it.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "../../include/gmres_gb300.h"
#include "grid_kernels.cuh"
#include "handle.hpp"
#include "host_util.hpp"
#include "sell.hpp"

using namespace gmres;
using namespace gmres_host;

namespace {

constexpr int kThreads = 256;

// Largest |col - row| over A's entries: one atomicMax per warp.
__global__ void __launch_bounds__(kThreads) k_sell_maxoff(int n, const int *__restrict__ rowptr,
                                                          const int *__restrict__ colind,
                                                          unsigned *out) {
    unsigned m = 0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int e = rowptr[row + 1];
        for (int k = rowptr[row]; k < e; ++k) {
            const long long d = (long long)colind[k] - row;
            m = max(m, (unsigned)(d < 0 ? -d : d));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, m);
}

// Row `row`'s entries into their slice positions: entry j of the slice's row
// l at sptr[s] + 32 j + l; columns as offsets from the row (rel) or as they are.
template <class IT>
__global__ void __launch_bounds__(kThreads)
    k_sell_fill(int n, const int *__restrict__ rowptr, const int *__restrict__ colind,
                const float *__restrict__ v32, const double *__restrict__ v64,
                const int *__restrict__ sptr, IT *col, float *s32, double *s64, int rel) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int b = rowptr[row], e = rowptr[row + 1];
        const int base = sptr[row / SELL_C] + row % SELL_C;
        for (int k = b; k < e; ++k) {
            const int i = base + SELL_C * (k - b);
            col[i] = rel ? (IT)(colind[k] - row) : (IT)colind[k];
            s32[i] = v32[k];
            s64[i] = v64[k];
        }
    }
}

template <class T, class CV>
__global__ void __launch_bounds__(kThreads)
    k_spmv_plain_sell(int n, const int *sptr, const unsigned short *slen, CV col, const T *sval,
                      const T *x, T *y) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nsl = (n + SELL_C - 1) / SELL_C;
    for (int s = warp; s < nsl; s += nwarps) {
        const int row = s * SELL_C + lane;
        const T v = sell_row<T>(sptr, slen, col, ValPlain<T>{sval}, XPlain<T, T>{x, 1.f}, s, lane,
                                row, n);
        if (row < n)
            y[row] = v;
    }
}

void release_all(gmres_handle *h) {
    for (DevBuf *b : {&h->sptr, &h->slen, &h->scol, &h->sval32, &h->sval64})
        b->release();
    h->sell_fmt = 0;
    h->sell_entries = 0;
}

gmres_status fill(gmres_handle *h) {
    const int grid = h->nsm * 8;
    if (h->sell_fmt == 1)
        k_sell_fill<short><<<grid, kThreads, 0, h->stream>>>(
            h->n, h->rowptr.as<int>(), h->colind.as<int>(), h->vals32.as<float>(),
            h->vals64.as<double>(), h->sptr.as<int>(), h->scol.as<short>(), h->sval32.as<float>(),
            h->sval64.as<double>(), 1);
    else
        k_sell_fill<int><<<grid, kThreads, 0, h->stream>>>(
            h->n, h->rowptr.as<int>(), h->colind.as<int>(), h->vals32.as<float>(),
            h->vals64.as<double>(), h->sptr.as<int>(), h->scol.as<int>(), h->sval32.as<float>(),
            h->sval64.as<double>(), 0);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess)
        return GMRES_ERR_CUDA;
    return GMRES_OK;
}

}  // namespace

gmres_status sell_build(gmres_handle *h) {
    if (h->sell_fmt)
        return GMRES_OK;
    if (h->split || h->n < 1)
        return GMRES_ERR_ARG;
    const int n = h->n;
    const int nsl = (n + SELL_C - 1) / SELL_C;
    std::vector<int> rp((size_t)n + 1);
    if (cudaMemcpyAsync(rp.data(), h->rowptr.p, sizeof(int) * ((size_t)n + 1),
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return GMRES_ERR_CUDA;
    // slice offsets (entries, padding included) and row lengths
    std::vector<int> sp((size_t)nsl + 1);
    std::vector<unsigned short> len((size_t)nsl * SELL_C, 0);
    int64_t tot = 0;
    for (int s = 0; s < nsl; ++s) {
        int w = 0;
        for (int r = s * SELL_C; r < std::min(n, (s + 1) * SELL_C); ++r) {
            const int l = rp[r + 1] - rp[r];
            if (l > 65535)
                return GMRES_ERR_ARG;
            len[r] = (unsigned short)l;
            w = std::max(w, l);
        }
        sp[s] = (int)tot;
        tot += (int64_t)SELL_C * w;
        if (tot > (int64_t)INT_MAX - 256)
            return GMRES_ERR_ARG;
    }
    sp[nsl] = (int)tot;
    // 16-bit column offsets when every |col - row| fits
    ScopedBuf dmax;
    if (dmax.ensure(sizeof(unsigned)) != cudaSuccess)
        return GMRES_ERR_OOM;
    unsigned maxoff = 0;
    if (cudaMemsetAsync(dmax.p, 0, sizeof(unsigned), h->stream) != cudaSuccess)
        return GMRES_ERR_CUDA;
    k_sell_maxoff<<<h->nsm * 8, kThreads, 0, h->stream>>>(n, h->rowptr.as<int>(),
                                                          h->colind.as<int>(), dmax.as<unsigned>());
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&maxoff, dmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return GMRES_ERR_CUDA;
    const bool rel = maxoff <= 32767u;
    const size_t ent = (size_t)std::max<int64_t>(tot, 1);
    if (h->sptr.ensure(sizeof(int) * sp.size()) != cudaSuccess ||
        h->slen.ensure(sizeof(unsigned short) * len.size()) != cudaSuccess ||
        h->scol.ensure(ent * (rel ? sizeof(short) : sizeof(int))) != cudaSuccess ||
        h->sval32.ensure(ent * sizeof(float)) != cudaSuccess ||
        h->sval64.ensure(ent * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        release_all(h);
        return GMRES_ERR_OOM;
    }
    h->sell_fmt = rel ? 1 : 2;
    h->sell_entries = tot;
    if (cudaMemcpyAsync(h->sptr.p, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->slen.p, len.data(), sizeof(unsigned short) * len.size(),
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->scol.p, 0, ent * (rel ? sizeof(short) : sizeof(int)), h->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(h->sval32.p, 0, ent * sizeof(float), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->sval64.p, 0, ent * sizeof(double), h->stream) != cudaSuccess) {
        release_all(h);
        return GMRES_ERR_CUDA;
    }
    const gmres_status st = fill(h);
    if (st != GMRES_OK)
        release_all(h);
    return st;
}

gmres_status sell_refill(gmres_handle *h) {
    if (!h->sell_fmt)
        return GMRES_OK;
    return fill(h);
}

void sell_free(gmres_handle *h) {
    release_all(h);
    h->sell32 = h->sell64 = false;
}

template <class T>
cudaError_t sell_spmv_plain(gmres_handle *h, const T *x, T *y) {
    const T *sval = std::is_same<T, double>::value ? reinterpret_cast<const T *>(h->sval64.p)
                                                   : reinterpret_cast<const T *>(h->sval32.p);
    const dim3 g(h->nsm * 8), b(kThreads);
    if (h->sell_fmt == 1)
        k_spmv_plain_sell<T, SellCol16><<<g, b, 0, h->stream>>>(
            h->n, h->sptr.as<int>(), h->slen.as<unsigned short>(),
            sell_cols<SellCol16>(h->scol.p), sval, x, y);
    else
        k_spmv_plain_sell<T, SellCol32><<<g, b, 0, h->stream>>>(
            h->n, h->sptr.as<int>(), h->slen.as<unsigned short>(),
            sell_cols<SellCol32>(h->scol.p), sval, x, y);
    return cudaGetLastError();
}

#ifdef GMRES_CHECKS
unsigned sell_check_take(cudaStream_t st) { return check_word_take(st); }
#endif

template cudaError_t sell_spmv_plain<float>(gmres_handle *, const float *, float *);
template cudaError_t sell_spmv_plain<double>(gmres_handle *, const double *, double *);

int64_t sell_bytes(const gmres_handle *h) {
    if (!h->sell_fmt)
        return 0;
    const int64_t nsl = ((int64_t)h->n + SELL_C - 1) / SELL_C;
    return 4 * (nsl + 1) + 2 * nsl * SELL_C +
           h->sell_entries * ((h->sell_fmt == 1 ? 2 : 4) + 4 + 8);
}
