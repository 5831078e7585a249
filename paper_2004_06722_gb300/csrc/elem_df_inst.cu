// FP32-pair BK5/BK6 element kernel instantiations (orders 1..15), see elem_df.cuh.
#include "elem_df.cuh"

namespace ceedbp {

cudaError_t set_df_dconst(int p1, const dfloat* host, cudaStream_t s) {
  if (p1 < 2 || p1 > kMaxP1) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbolAsync(c_Ddf, host, sizeof(dfloat) * p1 * p1,
                                 sizeof(dfloat) * size_t(p1 - 2) * kMaxP1 * kMaxP1, cudaMemcpyHostToDevice, s);
}

#define CEEDBP_DF_CASE(P)                                                                \
  case P:                                                                                \
    return m.ncomp == 3 ? launch_elem_df_t<P, 3>(m, a, s) : launch_elem_df_t<P, 1>(m, a, s);
#define CEEDBP_DF_BLOCKS(P) \
  case P:                   \
    return m.ncomp == 3 ? elem_df_blocks_t<P, 3>(m) : elem_df_blocks_t<P, 1>(m);
#define CEEDBP_DF_CAND(P) \
  case P:                 \
    return m.ncomp == 3 ? elem_df_candidates<P, 3>(eb, stage, cap) : elem_df_candidates<P, 1>(eb, stage, cap);

cudaError_t launch_elem_df(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_DF_CASE(2) CEEDBP_DF_CASE(3) CEEDBP_DF_CASE(4) CEEDBP_DF_CASE(5) CEEDBP_DF_CASE(6)
    CEEDBP_DF_CASE(7) CEEDBP_DF_CASE(8) CEEDBP_DF_CASE(9) CEEDBP_DF_CASE(10) CEEDBP_DF_CASE(11)
    CEEDBP_DF_CASE(12) CEEDBP_DF_CASE(13) CEEDBP_DF_CASE(14) CEEDBP_DF_CASE(15) CEEDBP_DF_CASE(16)
    default: return cudaErrorInvalidValue;
  }
}

int elem_df_blocks(const DeviceMesh& m) {
  switch (m.p1) {
    CEEDBP_DF_BLOCKS(2) CEEDBP_DF_BLOCKS(3) CEEDBP_DF_BLOCKS(4) CEEDBP_DF_BLOCKS(5) CEEDBP_DF_BLOCKS(6)
    CEEDBP_DF_BLOCKS(7) CEEDBP_DF_BLOCKS(8) CEEDBP_DF_BLOCKS(9) CEEDBP_DF_BLOCKS(10) CEEDBP_DF_BLOCKS(11)
    CEEDBP_DF_BLOCKS(12) CEEDBP_DF_BLOCKS(13) CEEDBP_DF_BLOCKS(14) CEEDBP_DF_BLOCKS(15) CEEDBP_DF_BLOCKS(16)
    default: return 0;
  }
}

int elem_df_tile_candidates(const DeviceMesh& m, int* eb, int* stage, int cap) {
  switch (m.p1) {
    CEEDBP_DF_CAND(2) CEEDBP_DF_CAND(3) CEEDBP_DF_CAND(4) CEEDBP_DF_CAND(5) CEEDBP_DF_CAND(6)
    CEEDBP_DF_CAND(7) CEEDBP_DF_CAND(8) CEEDBP_DF_CAND(9) CEEDBP_DF_CAND(10) CEEDBP_DF_CAND(11)
    CEEDBP_DF_CAND(12) CEEDBP_DF_CAND(13) CEEDBP_DF_CAND(14) CEEDBP_DF_CAND(15) CEEDBP_DF_CAND(16)
    default: return 0;
  }
}

}  // namespace ceedbp
