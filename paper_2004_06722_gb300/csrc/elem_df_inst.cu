// FP32-pair BK5/BK6 element kernel instantiations (orders 1..15), see
// elem_df.cuh, and of its software-pipelined schedule (orders 1..7), see
// elem_dfp.cuh.
#include "elem_dfp.cuh"

namespace ceedbp {

namespace {

constexpr int kDfpMaxP1 = 8;

template <int P1, int NC>
cudaError_t launch_df_any(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if constexpr (P1 <= kDfpMaxP1) {
    if (m.tune_stage == 2 && a.blk_prob == nullptr) return launch_elem_dfp_t<P1, NC>(m, a, s);
  }
  return launch_elem_df_t<P1, NC>(m, a, s);
}

// (eb, stage, ns) shapes the autotuner times: the per-element schedules of
// elem_df_kernel, then the pipelined schedule with 1..2 slots of 4..16 elements
template <int P1, int NC>
int df_candidates(int* eb, int* stage, int* ns, int cap, bool pipelined) {
  int n = elem_df_candidates<P1, NC>(eb, stage, cap);
  for (int k = 0; k < n; ++k) ns[k] = 1;
  if constexpr (P1 <= kDfpMaxP1) {
    if (pipelined) {
      for (int e = 1; e <= 2; ++e) {
        if (!elem_dfp_shape_ok<P1, NC>(e)) continue;
        for (int q = 4; q <= 16 && n < cap; q *= 2) {
          eb[n] = e;
          stage[n] = 2;
          ns[n++] = q;
        }
      }
    }
  }
  return n;
}

}  // namespace

cudaError_t set_df_dconst(int p1, const dfloat* host, cudaStream_t s) {
  if (p1 < 2 || p1 > kMaxP1) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbolAsync(c_Ddf, host, sizeof(dfloat) * p1 * p1,
                                 sizeof(dfloat) * size_t(p1 - 2) * kMaxP1 * kMaxP1, cudaMemcpyHostToDevice, s);
}

#define CEEDBP_DF_CASE(P)                                                                \
  case P:                                                                                \
    return m.ncomp == 3 ? launch_df_any<P, 3>(m, a, s) : launch_df_any<P, 1>(m, a, s);
#define CEEDBP_DF_BLOCKS(P) \
  case P:                   \
    return m.ncomp == 3 ? elem_df_blocks_t<P, 3>(m) : elem_df_blocks_t<P, 1>(m);
#define CEEDBP_DF_CAND(P) \
  case P:                 \
    return m.ncomp == 3 ? df_candidates<P, 3>(eb, stage, ns, cap, pipelined) \
                        : df_candidates<P, 1>(eb, stage, ns, cap, pipelined);

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

int elem_df_tile_candidates(const DeviceMesh& m, int* eb, int* stage, int* ns, int cap, bool pipelined) {
  switch (m.p1) {
    CEEDBP_DF_CAND(2) CEEDBP_DF_CAND(3) CEEDBP_DF_CAND(4) CEEDBP_DF_CAND(5) CEEDBP_DF_CAND(6)
    CEEDBP_DF_CAND(7) CEEDBP_DF_CAND(8) CEEDBP_DF_CAND(9) CEEDBP_DF_CAND(10) CEEDBP_DF_CAND(11)
    CEEDBP_DF_CAND(12) CEEDBP_DF_CAND(13) CEEDBP_DF_CAND(14) CEEDBP_DF_CAND(15) CEEDBP_DF_CAND(16)
    default: return 0;
  }
}

}  // namespace ceedbp
