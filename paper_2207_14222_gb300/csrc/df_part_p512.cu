// Double-float pencil passes for line lengths 512 (df_part.cuh).
#include "df_part.cuh"

USP_DF_PART(p512, 512)
