// team_launch.hpp -- launch of the whole-solve kernel for one system on a
// thread-block cluster (the kernels are compiled once, in batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "block_solver.cuh"

namespace gmres {

// Cluster size of the single-system team launch.
constexpr int TEAM_SINGLE_CTAS = 8;

// Solve system sys[0] (device array) with one cluster of TEAM_SINGLE_CTAS
// blocks of `threads` threads, L lanes per CSR row (1..32, power of two),
// `smem` dynamic shared memory bytes per block, on `stream`.
template <class T, class VT>
cudaError_t launch_team_single(const BlockSys<T, VT> *sys, const BlockParams &P,
                               BlockResult *res, int L, int threads, size_t smem,
                               cudaStream_t stream);

}  // namespace gmres
