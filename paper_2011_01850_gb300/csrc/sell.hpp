// sell.hpp -- host side of A's sliced storage (sell.cuh): building it from
// the device CSR arrays, refilling its values, releasing it, and the plain
// product y = A x in it.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gmres_gb300.h"
#include "handle.hpp"

// Build A's sliced copy (no-op when it exists).  GMRES_ERR_ARG when A is
// stored split, a row has more than 65535 entries or the padded copy has
// 2^31 - 256 entries or more; GMRES_ERR_OOM when it does not fit (nothing is
// kept then); GMRES_ERR_CUDA on a failed launch or copy.  Synchronizes the
// handle's stream.
gmres_status sell_build(gmres_handle *h);

// Copy A's current values into the sliced copy (after gmres_set_values);
// no-op when there is none.  Synchronizes the handle's stream.
gmres_status sell_refill(gmres_handle *h);

// Release the sliced copy and forget the autotuner's choice of it.
void sell_free(gmres_handle *h);

// y = A x with the sliced copy (which must exist), on the handle's stream.
template <class T>
cudaError_t sell_spmv_plain(gmres_handle *h, const T *x, T *y);

// Device bytes the sliced copy holds (0 when there is none).
int64_t sell_bytes(const gmres_handle *h);

#ifdef GMRES_CHECKS
// Checked build: bad columns met by this file's kernels since the last call
// (then cleared; synchronizes st).
unsigned sell_check_take(cudaStream_t st);
#endif
