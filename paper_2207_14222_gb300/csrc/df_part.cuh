// df_part.cuh -- one part of the double-float pencil passes (the refinement
// residual, df_kernels.cu).  The passes are split over several translation
// units by line length so that they compile in parallel; each unit holds
// its own copy of the twiddle tables (device variables are per unit).
#pragma once

#include "pencil_core.cuh"

namespace usp {
namespace {

__device__ dfl2 g_twdf[256];        // W_256^m
__device__ dfl2 g_twxdf[TWX_LEN];   // W_1536^m

}  // namespace

template <>
__device__ __forceinline__ dfl2 tw_entry<dfl>(int m) { return g_twdf[m]; }
template <>
__device__ __forceinline__ dfl2 twx_entry<dfl>(int m) { return g_twxdf[m]; }

// The FP64 passes' grid arithmetic (rows per block, rows_per_block_f64)
// serves these passes too.
template <int... Ns>
constexpr bool df_rows_match_f64() {
  return ((RowsShape<dfl, Ns>::F == RowsShape<double, Ns>::F &&
           RowsShape<dfl, Ns>::THREADS == RowsShape<double, Ns>::THREADS) && ...);
}
static_assert(df_rows_match_f64<2, 4, 8, 16, 32, 64, 96, 128, 192, 256, 384, 512>(),
              "double-float rows blocks must match the FP64 ones");

// This unit's tables and the shared-memory limits of its kernels.
template <int... Ns>
static cudaError_t df_part_init(const dfl2* tw256, const dfl2* tw1536) {
  cudaError_t e = cudaMemcpyToSymbol(g_twdf, tw256, sizeof(dfl2) * 256);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_twxdf, tw1536, sizeof(dfl2) * TWX_LEN);
  if (e != cudaSuccess) return e;
  ((e == cudaSuccess ? (e = attrs_one<dfl, Ns>(), 0) : 0), ...);
  return e;
}

template <int... Ns>
static cudaError_t df_part_rows(int n, const RowsArgs<dfl>& a, int64_t grid, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  ((n == Ns ? (e = rows_go<dfl, Ns>(a, grid, s), 0) : 0), ...);
  return e;
}

template <int... Ns>
static cudaError_t df_part_cols(int n, const ColsArgs<dfl>& a, cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  ((n == Ns ? (e = cols_go<dfl, Ns>(a, s), 0) : 0), ...);
  return e;
}

}  // namespace usp

// Defines the part's entry points df_{init,rows,cols}_<name> for line
// lengths __VA_ARGS__.
#define USP_DF_PART(name, ...)                                                                   \
  namespace usp {                                                                                \
  cudaError_t df_init_##name(const dfl2* tw256, const dfl2* tw1536) {                            \
    return df_part_init<__VA_ARGS__>(tw256, tw1536);                                             \
  }                                                                                              \
  cudaError_t df_rows_##name(int n, const RowsArgs<dfl>& a, int64_t grid, cudaStream_t s) {      \
    return df_part_rows<__VA_ARGS__>(n, a, grid, s);                                             \
  }                                                                                              \
  cudaError_t df_cols_##name(int n, const ColsArgs<dfl>& a, cudaStream_t s) {                    \
    return df_part_cols<__VA_ARGS__>(n, a, s);                                                   \
  }                                                                                              \
  }
