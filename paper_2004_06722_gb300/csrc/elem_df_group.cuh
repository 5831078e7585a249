// One group of orders of the FP32-pair BK5/BK6 kernels (elem_df.cuh: per-element
// schedules; elem_dfp.cuh: pipelined sequences).  A translation unit defines
//   CEEDBP_DF_ORDERS(X)   X(p1) for every p1 of the group
//   CEEDBP_DF_NAME(f)     f##_<group tag>
// and includes this file, which defines the group's launcher,
// autotuner candidates and constant-bank setter; elem_df_inst.cu dispatches to
// the group that holds an order.  Splitting the orders over translation units
// lets nvcc compile them in parallel.
#include "elem_dfp.cuh"

namespace ceedbp {

namespace {

// The pipelined schedule is instantiated for one component up to p1 = 16 and
// for three components up to p1 = 8 (larger tiles do not fit shared memory).
template <int P1, int NC>
constexpr bool kDfpBuilt = (NC == 1) || (P1 <= 8);

template <int P1, int NC>
cudaError_t launch_df_any(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if constexpr (kDfpBuilt<P1, NC>) {
    if (m.tune_stage == 2) return launch_elem_dfp_t<P1, NC>(m, a, s);
  }
  return launch_elem_df_t<P1, NC>(m, a, s);
}

// (eb, stage, ns) shapes the autotuner times: the per-element schedules of
// elem_df_kernel, then the pipelined schedule with 1..2 slots of 4..16 elements
template <int P1, int NC>
int df_candidates(int* eb, int* stage, int* ns, int cap, bool pipelined) {
  int n = elem_df_candidates<P1, NC>(eb, stage, cap);
  for (int k = 0; k < n; ++k) ns[k] = 1;
  if constexpr (kDfpBuilt<P1, NC>) {
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

#define CEEDBP_DF_CASE(P) \
  case P:                 \
    return m.ncomp == 3 ? launch_df_any<P, 3>(m, a, s) : launch_df_any<P, 1>(m, a, s);
#define CEEDBP_DF_CAND(P)                                                      \
  case P:                                                                      \
    return m.ncomp == 3 ? df_candidates<P, 3>(eb, stage, ns, cap, pipelined) \
                        : df_candidates<P, 1>(eb, stage, ns, cap, pipelined);
#define CEEDBP_DF_HAS(P) \
  case P:                \
    return true;

cudaError_t CEEDBP_DF_NAME(set_df_dconst)(int p1, const dfloat* host, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(c_Ddf, host, sizeof(dfloat) * p1 * p1,
                                 sizeof(dfloat) * size_t(p1 - 2) * kMaxP1 * kMaxP1, cudaMemcpyHostToDevice, s);
}

bool CEEDBP_DF_NAME(df_has)(int p1) {
  switch (p1) {
    CEEDBP_DF_ORDERS(CEEDBP_DF_HAS)
    default: return false;
  }
}

cudaError_t CEEDBP_DF_NAME(launch_elem_df)(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  switch (m.p1) {
    CEEDBP_DF_ORDERS(CEEDBP_DF_CASE)
    default: return cudaErrorInvalidValue;
  }
}

int CEEDBP_DF_NAME(elem_df_tile_candidates)(const DeviceMesh& m, int* eb, int* stage, int* ns, int cap,
                                            bool pipelined) {
  switch (m.p1) {
    CEEDBP_DF_ORDERS(CEEDBP_DF_CAND)
    default: return 0;
  }
}

}  // namespace ceedbp
