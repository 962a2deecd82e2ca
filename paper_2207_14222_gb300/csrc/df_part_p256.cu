// Double-float pencil passes for line lengths 256, 192 (df_part.cuh).
#include "df_part.cuh"

USP_DF_PART(p256, 256, 192)
