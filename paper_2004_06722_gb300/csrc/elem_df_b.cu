// FP32-pair BK5/BK6 kernels for p1 in {7, 8} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(7) X(8)
#define CEEDBP_DF_NAME(f) f##_b
#include "elem_df_group.cuh"
