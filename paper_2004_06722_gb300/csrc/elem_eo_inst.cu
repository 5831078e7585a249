// Even-odd FP64 BK5/BK6 instantiations for even p1 (odd orders 1..15), see elem_eo.cuh.
#include "elem_eo.cuh"

namespace ceedbp {

#define CEEDBP_EO_CASE(P) \
  case P: return m.ncomp == 3 ? launch_elem_eo_t<P, 3>(m, a, s) : launch_elem_eo_t<P, 1>(m, a, s);
#define CEEDBP_EO_BLOCKS(P) \
  case P: return m.ncomp == 3 ? elem_eo_blocks_t<P, 3>(m.nelem) : elem_eo_blocks_t<P, 1>(m.nelem);

cudaError_t launch_elem_eo(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_EO_CASE(2) CEEDBP_EO_CASE(4) CEEDBP_EO_CASE(6) CEEDBP_EO_CASE(8)
    CEEDBP_EO_CASE(10) CEEDBP_EO_CASE(12) CEEDBP_EO_CASE(14) CEEDBP_EO_CASE(16)
    default: return cudaErrorInvalidValue;
  }
}

int elem_eo_blocks(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_EO_BLOCKS(2) CEEDBP_EO_BLOCKS(4) CEEDBP_EO_BLOCKS(6) CEEDBP_EO_BLOCKS(8)
    CEEDBP_EO_BLOCKS(10) CEEDBP_EO_BLOCKS(12) CEEDBP_EO_BLOCKS(14) CEEDBP_EO_BLOCKS(16)
    default: return 0;
  }
}

#define CEEDBP_EO_EB(P) \
  case P: return m.ncomp == 3 ? elem_eo_per_block<P, 3>() : elem_eo_per_block<P, 1>();

int elem_eo_per_block_rt(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_EO_EB(2) CEEDBP_EO_EB(4) CEEDBP_EO_EB(6) CEEDBP_EO_EB(8)
    CEEDBP_EO_EB(10) CEEDBP_EO_EB(12) CEEDBP_EO_EB(14) CEEDBP_EO_EB(16)
    default: return 0;
  }
}

#define CEEDBP_EO_OK(P) \
  case P: return m.ncomp == 3 ? elem_eo_launchable<P, 3>() : elem_eo_launchable<P, 1>();

bool elem_eo_available(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_EO_OK(2) CEEDBP_EO_OK(4) CEEDBP_EO_OK(6) CEEDBP_EO_OK(8)
    CEEDBP_EO_OK(10) CEEDBP_EO_OK(12) CEEDBP_EO_OK(14) CEEDBP_EO_OK(16)
    default: return false;
  }
}

}  // namespace ceedbp
