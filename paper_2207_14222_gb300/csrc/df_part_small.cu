// Double-float pencil passes for line lengths 2, 4, 8, 16, 32, 64 (df_part.cuh).
#include "df_part.cuh"

USP_DF_PART(small, 2, 4, 8, 16, 32, 64)
