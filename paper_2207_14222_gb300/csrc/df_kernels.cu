// df_kernels.cu -- the pencil passes (pencil_core.cuh) in double-float for
// the refinement residual y - A x: forward FFT of x, the multiplier
// Lhat(p)/N, inverse FFT, then r = y - (L x + V x) with the products V x
// exact in two words (Sec. 2.1's A = L + V).  The kernels live in the
// df_part_*.cu units (one per group of line lengths); this unit dispatches
// on the line length and fills every part's twiddle tables.
#include "dfloat.cuh"
#include "kernels.h"

namespace usp {

#define USP_DF_DECLARE(name)                                                                \
  cudaError_t df_init_##name(const dfl2* tw256, const dfl2* tw1536);                        \
  cudaError_t df_rows_##name(int n, const RowsArgs<dfl>& a, int64_t grid, cudaStream_t s); \
  cudaError_t df_cols_##name(int n, const ColsArgs<dfl>& a, cudaStream_t s);
USP_DF_DECLARE(small)
USP_DF_DECLARE(p128)
USP_DF_DECLARE(p256)
USP_DF_DECLARE(p384)
USP_DF_DECLARE(p512)
#undef USP_DF_DECLARE

cudaError_t launch_rows_df(int n, const RowsArgs<dfl>& a, int64_t grid, cudaStream_t s) {
  switch (n) {
    case 2: case 4: case 8: case 16: case 32: case 64: return df_rows_small(n, a, grid, s);
    case 96: case 128: return df_rows_p128(n, a, grid, s);
    case 192: case 256: return df_rows_p256(n, a, grid, s);
    case 384: return df_rows_p384(n, a, grid, s);
    case 512: return df_rows_p512(n, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cols_df(int n, const ColsArgs<dfl>& a, cudaStream_t s) {
  switch (n) {
    case 2: case 4: case 8: case 16: case 32: case 64: return df_cols_small(n, a, s);
    case 96: case 128: return df_cols_p128(n, a, s);
    case 192: case 256: return df_cols_p256(n, a, s);
    case 384: return df_cols_p384(n, a, s);
    case 512: return df_cols_p512(n, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t init_twiddles_df(const double2* tw256, const double2* tw1536) {
  static dfl2 h[256], x[1536];
  for (int m = 0; m < 256; ++m) h[m] = dfl2{dfl(tw256[m].x), dfl(tw256[m].y)};
  for (int m = 0; m < 1536; ++m) x[m] = dfl2{dfl(tw1536[m].x), dfl(tw1536[m].y)};
  cudaError_t e;
  if ((e = df_init_small(h, x)) != cudaSuccess) return e;
  if ((e = df_init_p128(h, x)) != cudaSuccess) return e;
  if ((e = df_init_p256(h, x)) != cudaSuccess) return e;
  if ((e = df_init_p384(h, x)) != cudaSuccess) return e;
  return df_init_p512(h, x);
}

}  // namespace usp
