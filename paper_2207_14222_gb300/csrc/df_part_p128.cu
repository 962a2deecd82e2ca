// Double-float pencil passes for line lengths 128, 96 (df_part.cuh).
#include "df_part.cuh"

USP_DF_PART(p128, 128, 96)
