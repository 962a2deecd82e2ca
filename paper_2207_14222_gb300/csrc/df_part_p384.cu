// Double-float pencil passes for line lengths 384 (df_part.cuh).
#include "df_part.cuh"

USP_DF_PART(p384, 384)
