// Low-precision element kernel instantiations (orders 1..15; FP32 or BF16
// storage; one or three components), see elem_lp.cuh; FP32 storage runs the
// pipelined schedule of elem_lpp.cuh where its shape fits.
#include "elem_lpp.cuh"

namespace ceedbp {

template <int P1>
static cudaError_t launch_lp_p(const DeviceMesh& m, const ElemLpArgs& a, int bf16, cudaStream_t s) {
  if (m.ncomp == 3)
    return bf16 ? launch_elem_lp_t<P1, 3, __nv_bfloat16>(m, a, s) : launch_elem_lpp_t<P1, 3>(m, a, s);
  return bf16 ? launch_elem_lp_t<P1, 1, __nv_bfloat16>(m, a, s) : launch_elem_lpp_t<P1, 1>(m, a, s);
}

#define CEEDBP_LP_CASE(P) \
  case P: return launch_lp_p<P>(m, a, bf16, s);
#define CEEDBP_LP_BLOCKS(P) \
  case P: return m.ncomp == 3 ? elem_lp_blocks_t<P, 3>(m.nelem) : elem_lp_blocks_t<P, 1>(m.nelem);

cudaError_t launch_elem_lp(const DeviceMesh& m, const ElemLpArgs& a, int bf16, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_LP_CASE(2) CEEDBP_LP_CASE(3) CEEDBP_LP_CASE(4) CEEDBP_LP_CASE(5) CEEDBP_LP_CASE(6)
    CEEDBP_LP_CASE(7) CEEDBP_LP_CASE(8) CEEDBP_LP_CASE(9) CEEDBP_LP_CASE(10) CEEDBP_LP_CASE(11)
    CEEDBP_LP_CASE(12) CEEDBP_LP_CASE(13) CEEDBP_LP_CASE(14) CEEDBP_LP_CASE(15) CEEDBP_LP_CASE(16)
    default: return cudaErrorInvalidValue;
  }
}

int elem_lp_blocks(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_LP_BLOCKS(2) CEEDBP_LP_BLOCKS(3) CEEDBP_LP_BLOCKS(4) CEEDBP_LP_BLOCKS(5) CEEDBP_LP_BLOCKS(6)
    CEEDBP_LP_BLOCKS(7) CEEDBP_LP_BLOCKS(8) CEEDBP_LP_BLOCKS(9) CEEDBP_LP_BLOCKS(10) CEEDBP_LP_BLOCKS(11)
    CEEDBP_LP_BLOCKS(12) CEEDBP_LP_BLOCKS(13) CEEDBP_LP_BLOCKS(14) CEEDBP_LP_BLOCKS(15) CEEDBP_LP_BLOCKS(16)
    default: return 0;
  }
}

}  // namespace ceedbp
