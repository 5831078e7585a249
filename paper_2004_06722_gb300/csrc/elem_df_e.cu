// FP32-pair BK5/BK6 kernels for p1 in {12} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(12)
#define CEEDBP_DF_NAME(f) f##_e
#include "elem_df_group.cuh"
