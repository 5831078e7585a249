// FP32-pair BK5/BK6 kernels for p1 in {9, 10} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(9) X(10)
#define CEEDBP_DF_NAME(f) f##_c
#include "elem_df_group.cuh"
