// common.cuh -- device helpers shared by the GB300 GMRES kernels.
//
// Basis storage types, deterministic block and grid reductions, and the
// device-resident control block of a restart cycle.  Everything here is device
// code for sm_103a; no host fallback exists.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gmres {

// Largest restart length m supported by the kernels (the Hessenberg column has
// at most MMAX+1 entries).
constexpr int MMAX = 128;
constexpr int WARP = 32;

// Device-resident control block of one solve.  Written by the "last block" of
// grid reductions and read by every later kernel on the stream; the host reads
// it once per restart cycle.
struct Ctl {
    int active;      // the restart cycle is still running
    int j;           // inner iterations done in the current cycle
    int last_j;      // length of the cycle that just finished
    int breakdown;   // h_{j+1,j} vanished in the current cycle
    int converged;   // binary64 residual met the tolerance at the last check
    int nonfinite;   // NaN/Inf seen
    int timeout;     // a bounded wait gave up
    int pad;
    unsigned counter[8];  // last-block arrival counters (reset by the last block)
    double rnorm;    // ||b - A x||_2, binary64
    double bnorm;    // ||b||_2, binary64
    double beta;     // ||r||_2 in the working precision (value of type T)
    double arn;      // |s_{j+1}| after the last inner step
    double hnext;    // h_{j+1,j} of the last inner step (value of type T)
    double wnorm0;   // ||A v_j|| of the current step (breakdown reference)
};

// ---------------------------------------------------------------------------
// Krylov-basis storage: load/store one element of the basis in its storage
// type, widening to / rounding from the working type T (round-to-nearest-
// even for every narrowing).  The binary16 basis holds v * scale with scale a
// power of two, so scaling is exact.
// ---------------------------------------------------------------------------
template <class VT>
struct Basis;

template <>
struct Basis<double> {
    static constexpr int bytes = 8;
    __device__ __forceinline__ static double ld(const double *p, float) { return *p; }
    __device__ __forceinline__ static void st(double *p, double v, float) { *p = v; }
    // the value a store followed by a load gives (rt = round trip)
    __device__ __forceinline__ static double rt(double v, float, float) { return v; }
};

template <>
struct Basis<float> {
    static constexpr int bytes = 4;
    __device__ __forceinline__ static float ld(const float *p, float) { return *p; }
    __device__ __forceinline__ static void st(float *p, float v, float) { *p = v; }
    __device__ __forceinline__ static float rt(float v, float, float) { return v; }
    __device__ __forceinline__ static double rt(double v, float, float) {
        return (double)(float)v;
    }
};

template <>
struct Basis<__nv_bfloat16> {
    static constexpr int bytes = 2;
    __device__ __forceinline__ static float ld(const __nv_bfloat16 *p, float) {
        return __bfloat162float(*p);
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, float v, float) {
        *p = __float2bfloat16_rn(v);
    }
    __device__ __forceinline__ static float rt(float v, float, float) {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
};

template <>
struct Basis<__half> {
    static constexpr int bytes = 2;
    // scale = 2^floor(log2(n)/2); loads divide by it (multiply by the exact
    // reciprocal), stores multiply before rounding.
    __device__ __forceinline__ static float ld(const __half *p, float inv_scale) {
        return __half2float(*p) * inv_scale;
    }
    __device__ __forceinline__ static void st(__half *p, float v, float scale) {
        *p = __float2half_rn(v * scale);
    }
    __device__ __forceinline__ static float rt(float v, float scale, float inv_scale) {
        return __half2float(__float2half_rn(v * scale)) * inv_scale;
    }
};

// Square root in the working type.
__device__ __forceinline__ double wsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float wsqrt(float v) { return sqrtf(v); }

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// The checked build (compiled with -DGMRES_CHECKS, in place of a memory
// sanitizer): every column index a gather kernel reads x with is tested
// against the system's columns [0, ncol) before the load.  A column outside
// is counted in this translation unit's check word and replaced by column 0,
// so the load stays inside x.  The entry points that launch these kernels
// read and clear the word after their last synchronize and return
// GMRES_ERR_INDEX when it was set.  Without the flag the check is the
// identity and costs nothing.
// ---------------------------------------------------------------------------
#ifdef GMRES_CHECKS
static __device__ unsigned gmres_check_word;

__device__ __forceinline__ int chk_col(int c, int ncol) {
    if ((unsigned)c >= (unsigned)ncol) {
        atomicAdd(&gmres_check_word, 1u);
        return 0;
    }
    return c;
}

// Host side: the number of bad columns this translation unit's kernels met
// since the last call, then cleared (synchronizes st).
static inline unsigned check_word_take(cudaStream_t st) {
    unsigned v = 0;
    const unsigned z = 0;
    if (cudaMemcpyFromSymbolAsync(&v, gmres_check_word, sizeof(v), 0, cudaMemcpyDeviceToHost,
                                  st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(gmres_check_word, &z, sizeof(z), 0, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return ~0u;  // the check itself failed: report it as a violation
    return v;
}
#else
__device__ __forceinline__ int chk_col(int c, int) { return c; }
#endif

// ---------------------------------------------------------------------------
// Deterministic reductions.  The xor-butterfly gives the same association
// order on every run, so repeated solves are bitwise reproducible.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum K values per thread over the block; every thread receives the K sums.
// smem must hold K * 32 values of T.  Contains __syncthreads.
template <class T, int K>
__device__ __forceinline__ void block_sum(T (&v)[K], T *smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            smem[k * 32 + wid] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        T t = (lane < nw) ? smem[k * 32 + lane] : T(0);
        v[k] = warp_sum(t);
    }
    __syncthreads();
}

template <class T>
__device__ __forceinline__ T block_sum1(T v, T *smem) {
    T a[1] = {v};
    block_sum<T, 1>(a, smem);
    return a[0];
}

// "Last block" of a grid reduction: every block has written its partials;
// returns true in exactly one block (the last to arrive), which then sees all
// partials.  The counter is reset by that block for the next launch.
__device__ __forceinline__ bool arrive_last(unsigned *counter) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    int last = s_last;
    if (last) {
        __threadfence();
        if (threadIdx.x == 0)
            atomicExch(counter, 0u);
    }
    return last != 0;
}

// Load bypassing L1 (values written by other blocks of the same grid).
template <class T>
__device__ __forceinline__ T ldcg(const T *p) {
    return __ldcg(p);
}

}  // namespace gmres
