// sell.cuh -- A in sliced storage (SELL-32) for w <- A v_j of the Arnoldi
// step (Alg. 1 of arXiv 2011.01850) and for the library's plain SpMV.
//
// Rows go in slices of 32 consecutive rows.  A slice's entries are stored
// column-major: entry k of the slice's row l sits at sptr[s] + 32 k + l, and
// the slice is padded to its longest row (the padding is never read: every
// row's length is in slen).  One warp takes one slice, so every load of
// values, indices and row lengths is one contiguous 32-wide access, where the
// CSR kernel with one lane per row strides by the row length.  For banded
// matrices the gathers of x are contiguous too (entry k of neighbouring rows
// lies on one diagonal).  Columns are kept as 16-bit offsets from the row
// when every |col - row| fits (half the index bytes), else as 32-bit column
// indices.  A row's products are summed in the order of its columns, the
// same additions as the one-lane-per-row CSR kernel makes, so the two formats
// give the same result bit for bit.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace gmres {

constexpr int SELL_C = 32;  // rows per slice (one warp)

// column of entry i of row `row`: 16-bit offsets from the row, or 32-bit
// column indices
struct SellCol16 {
    const short *c;
    __device__ __forceinline__ int operator()(int i, int row) const {
        return row + (int)__ldg(c + i);
    }
};
struct SellCol32 {
    const int *c;
    __device__ __forceinline__ int operator()(int i, int) const { return __ldg(c + i); }
};

template <class CV>
__host__ __device__ __forceinline__ CV sell_cols(const void *p);
template <>
__host__ __device__ __forceinline__ SellCol16 sell_cols<SellCol16>(const void *p) {
    return SellCol16{static_cast<const short *>(p)};
}
template <>
__host__ __device__ __forceinline__ SellCol32 sell_cols<SellCol32>(const void *p) {
    return SellCol32{static_cast<const int *>(p)};
}

// Row `row` (= 32 s + lane) of slice s: sum of a_k x_{col_k} over the row's
// entries in column order, the same sequence of additions as the CSR kernel at
// one lane per row.  The loads go in groups of SELL_G entries: all of a
// group's indices and values, then all its gathers, then the sums in order,
// so a row of up to SELL_G entries costs one dependent round trip.  The loop
// runs to the slice's width, uniform over the warp; entries past the row's
// length are predicated off.
constexpr int SELL_G = 8;

template <class T, class AV, class XV, class CV>
__device__ __forceinline__ T sell_row(const int *__restrict__ sptr,
                                      const unsigned short *__restrict__ slen, CV col, AV a, XV xv,
                                      int s, int lane, int row, int n) {
    const int beg = __ldg(sptr + s);
    const int W = (__ldg(sptr + s + 1) - beg) / SELL_C;
    const int len = row < n ? (int)__ldg(slen + row) : 0;
    T acc = 0;
    for (int k = 0; k < W; k += SELL_G) {
        const int i = beg + SELL_C * k + lane;
        int c[SELL_G];
        T av[SELL_G], xw[SELL_G];
#pragma unroll
        for (int g = 0; g < SELL_G; ++g) {
            const bool p = k + g < len;
            c[g] = p ? chk_col(col(i + g * SELL_C, row), n) : row;
            av[g] = p ? (T)a(i + g * SELL_C) : T(0);
        }
#pragma unroll
        for (int g = 0; g < SELL_G; ++g)
            xw[g] = k + g < len ? xv(c[g]) : T(0);
#pragma unroll
        for (int g = 0; g < SELL_G; ++g)
            if (k + g < len)
                acc += av[g] * xw[g];
    }
    return acc;
}

}  // namespace gmres
