// FP32-pair BK5/BK6 kernels for p1 in {11} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(11)
#define CEEDBP_DF_NAME(f) f##_d
#include "elem_df_group.cuh"
