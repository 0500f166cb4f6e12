// host_util.hpp -- host-side helpers shared by the library's translation
// units: owned device buffers, CUDA error checks that map to gmres_status,
// pointer classification and small numeric helpers.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/gmres_gb300.h"

namespace gmres_host {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want) {
        if (want <= bytes)
            return cudaSuccess;
        if (p)
            cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = want;
        return cudaSuccess;
    }
    void release() {
        if (p)
            cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// A device buffer freed when it goes out of scope (temporary staging).
struct ScopedBuf : DevBuf {
    ScopedBuf() = default;
    ScopedBuf(const ScopedBuf &) = delete;
    ScopedBuf &operator=(const ScopedBuf &) = delete;
    ~ScopedBuf() { release(); }
};


#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            fprintf(stderr, "gmres_gb300: %s failed: %s (%s:%d)\n", #call,            \
                    cudaGetErrorString(e_), __FILE__, __LINE__);                      \
            return e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;  \
        }                                                                             \
    } while (0)

#define CKL()                                                                         \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) {                                                      \
            fprintf(stderr, "gmres_gb300: launch failed: %s (%s:%d)\n",               \
                    cudaGetErrorString(e_), __FILE__, __LINE__);                      \
            return GMRES_ERR_CUDA;                                                    \
        }                                                                             \
    } while (0)

inline bool is_device_ptr(const void *p) {
    if (!p)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

inline int elem_bytes(gmres_precision p) {
    switch (p) {
    case GMRES_FP64: return 8;
    case GMRES_MIXED: return 4;
    case GMRES_MIXED_LIMITED: return 4;
    default: return 2;
    }
}

inline double default_tau(gmres_precision p) {
    switch (p) {
    case GMRES_FP64: return 0.0;
    case GMRES_MIXED: return 1e-6;
    case GMRES_MIXED_LIMITED: return 1e-6;
    case GMRES_MIXED_BF16: return 0.00390625;     // 2^-8, the bfloat16 unit roundoff
    default: return 0.00048828125;                // 2^-11, the binary16 unit roundoff
    }
}

// Power-of-two binary16 scale 2^floor(log2(n)/2).
inline float fp16_scale(int n) {
    int lg = 0;
    while (lg < 31 && ((int64_t)1 << (lg + 1)) <= (int64_t)n)
        ++lg;
    return std::ldexp(1.0f, lg / 2);
}


inline int pow2_lanes(double avg) {
    int L = 1;
    while (L < 32 && L * 2 <= avg)
        L *= 2;
    return L;
}

// CSR structure check: rowptr[0] = 0, monotone, rowptr[n] = nnz, columns in
// [0, ncols).
inline gmres_status check_csr_host(int64_t n, const int32_t *rp, const int32_t *ci, int64_t nnz,
                                   int64_t ncols) {
    if (rp[0] != 0)
        return GMRES_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i])
            return GMRES_ERR_ARG;
    if ((int64_t)rp[n] != nnz)
        return GMRES_ERR_ARG;
    for (int64_t k = 0; k < nnz; ++k)
        if (ci[k] < 0 || ci[k] >= ncols)
            return GMRES_ERR_ARG;
    return GMRES_OK;
}

}  // namespace gmres_host
