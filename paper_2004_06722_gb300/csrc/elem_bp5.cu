// Element kernel instantiations for BP5 (orders 1..15), see elem.cuh.
#include "elem.cuh"

namespace ceedbp {

#define CEEDBP_ELEM_CASE(P) \
  case P: return launch_elem_t<P, P + 0, true, kStiff, 1>(m, a, s);
#define CEEDBP_BLOCKS_CASE(P) \
  case P: return elem_blocks_t<P, P + 0, true, 1>(m.nelem);
#define CEEDBP_EB_CASE(P) \
  case P: return elem_per_block<P, P + 0, true, 1>();

cudaError_t launch_elem_bp5(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_ELEM_CASE(2) CEEDBP_ELEM_CASE(3) CEEDBP_ELEM_CASE(4) CEEDBP_ELEM_CASE(5) CEEDBP_ELEM_CASE(6)
    CEEDBP_ELEM_CASE(7) CEEDBP_ELEM_CASE(8) CEEDBP_ELEM_CASE(9) CEEDBP_ELEM_CASE(10) CEEDBP_ELEM_CASE(11)
    CEEDBP_ELEM_CASE(12) CEEDBP_ELEM_CASE(13) CEEDBP_ELEM_CASE(14) CEEDBP_ELEM_CASE(15) CEEDBP_ELEM_CASE(16)
    default: return cudaErrorInvalidValue;
  }
}

int elem_blocks_bp5(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_BLOCKS_CASE(2) CEEDBP_BLOCKS_CASE(3) CEEDBP_BLOCKS_CASE(4) CEEDBP_BLOCKS_CASE(5) CEEDBP_BLOCKS_CASE(6)
    CEEDBP_BLOCKS_CASE(7) CEEDBP_BLOCKS_CASE(8) CEEDBP_BLOCKS_CASE(9) CEEDBP_BLOCKS_CASE(10) CEEDBP_BLOCKS_CASE(11)
    CEEDBP_BLOCKS_CASE(12) CEEDBP_BLOCKS_CASE(13) CEEDBP_BLOCKS_CASE(14) CEEDBP_BLOCKS_CASE(15) CEEDBP_BLOCKS_CASE(16)
    default: return 0;
  }
}

// elements per block of the BP5 kernel (block tables of batched solves)
int elem_per_block_bp5(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_EB_CASE(2) CEEDBP_EB_CASE(3) CEEDBP_EB_CASE(4) CEEDBP_EB_CASE(5) CEEDBP_EB_CASE(6)
    CEEDBP_EB_CASE(7) CEEDBP_EB_CASE(8) CEEDBP_EB_CASE(9) CEEDBP_EB_CASE(10) CEEDBP_EB_CASE(11)
    CEEDBP_EB_CASE(12) CEEDBP_EB_CASE(13) CEEDBP_EB_CASE(14) CEEDBP_EB_CASE(15) CEEDBP_EB_CASE(16)
    default: return 0;
  }
}

}  // namespace ceedbp
