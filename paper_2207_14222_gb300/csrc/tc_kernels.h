// tc_kernels.h -- 256-point transforms along a strided axis on the 5th
// generation tensor cores (tc_kernels.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace usp {

// Uploads the DFT-16 operand tables and sets the kernel's shared-memory
// limit (once per device).
cudaError_t tc_cols_init();

// The strided-axis pass of ColsTmaArgs (COL_FWD, COL_INV or COL_FWD_MUL_INV
// with MUL_LINV) for axis length 256, single problem, tiles of 8 columns
// (map: box {8, 256, 1}).  Two CTAs of 128 threads per SM.
cudaError_t launch_cols_tc(const CUtensorMap& map, const ColsTmaArgs& a, int grid, cudaStream_t s);

}  // namespace usp
