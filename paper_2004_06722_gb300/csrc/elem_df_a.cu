// FP32-pair BK5/BK6 kernels for p1 in {2, 3, 4, 5, 6} (see elem_df_group.cuh).
#define CEEDBP_DF_ORDERS(X) X(2) X(3) X(4) X(5) X(6)
#define CEEDBP_DF_NAME(f) f##_a
#include "elem_df_group.cuh"
