// FP32-pair BK5/BK6 kernels for p1 in {13, 14} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(13) X(14)
#define CEEDBP_DF_NAME(f) f##_f
#include "elem_df_group.cuh"
