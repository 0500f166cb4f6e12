// ilu.hpp -- ILU(0) left preconditioning (ilu.cu): factorization and the
// two triangular solves.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gmres_gb300.h"
#include "handle.hpp"

namespace gmres {

// Factor the handle's A (binary64 values) into ILU(0) on its pattern: level
// analysis on the host, one launch per level; also a binary32 copy.
// GMRES_ERR_ARG for unsorted rows or a missing diagonal entry,
// GMRES_ERR_BREAKDOWN for a zero or non-finite pivot.
gmres_status ilu_factor(gmres_handle *h);

// out = (L U)^-1 z on the device: L y = z into tmp, then U out = tmp (T
// arithmetic, factors of type AT); a wait that runs out sets *err.
// Kernel of one triangular solve: opts.trsv_kernel when set, else 3 (no
// barrier) for a triangle whose rows hold at most four entries and whose
// levels fit the grid, 2 (level barrier) otherwise.
int trsv_kind(const gmres_handle *h, bool lower);

template <class T, class AT>
cudaError_t ilu_apply(gmres_handle *h, const AT *lu, const T *z, T *tmp, T *out, int *err);

}  // namespace gmres
