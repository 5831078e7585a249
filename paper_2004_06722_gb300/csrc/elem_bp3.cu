// Element kernel instantiations for BP3 (orders 1..15): the even-odd kernel of
// elem_gl.cuh (every 1D contraction in even-odd form); at order 14, where that
// kernel runs out of registers, the column kernel of elem.cuh.
#include "elem_gl.cuh"

namespace ceedbp {

#define CEEDBP_ELEM_CASE(P) \
  case P: return launch_elem_gl_t<P, P + 1, kStiff>(m, a, s);
#define CEEDBP_BLOCKS_CASE(P) \
  case P: return elem_gl_blocks_t<P, P + 1>(m.nelem);

cudaError_t launch_elem_bp3(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_ELEM_CASE(2) CEEDBP_ELEM_CASE(3) CEEDBP_ELEM_CASE(4) CEEDBP_ELEM_CASE(5) CEEDBP_ELEM_CASE(6)
    CEEDBP_ELEM_CASE(7) CEEDBP_ELEM_CASE(8) CEEDBP_ELEM_CASE(9) CEEDBP_ELEM_CASE(10) CEEDBP_ELEM_CASE(11)
    CEEDBP_ELEM_CASE(12) CEEDBP_ELEM_CASE(13) CEEDBP_ELEM_CASE(14) CEEDBP_ELEM_CASE(16)
    case 15: return launch_elem_t<15, 16, false, kStiff, 1>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

int elem_blocks_bp3(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_BLOCKS_CASE(2) CEEDBP_BLOCKS_CASE(3) CEEDBP_BLOCKS_CASE(4) CEEDBP_BLOCKS_CASE(5) CEEDBP_BLOCKS_CASE(6)
    CEEDBP_BLOCKS_CASE(7) CEEDBP_BLOCKS_CASE(8) CEEDBP_BLOCKS_CASE(9) CEEDBP_BLOCKS_CASE(10) CEEDBP_BLOCKS_CASE(11)
    CEEDBP_BLOCKS_CASE(12) CEEDBP_BLOCKS_CASE(13) CEEDBP_BLOCKS_CASE(14) CEEDBP_BLOCKS_CASE(16)
    case 15: return elem_blocks_t<15, 16, false, 1>(m.nelem);
    default: return 0;
  }
}

}  // namespace ceedbp
