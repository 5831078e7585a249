// Dispatch of the FP32-pair BK5/BK6 kernels to the translation unit that holds
// each order (elem_df_a.cu .. elem_df_h.cu, see elem_df_group.cuh).
#include <cuda_runtime.h>

#include "df.cuh"
#include "internal.h"
#include "kernel_args.h"

namespace ceedbp {

cudaError_t set_df_dconst_a(int, const dfloat*, cudaStream_t);
bool df_has_a(int);
cudaError_t launch_elem_df_a(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_a(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_b(int, const dfloat*, cudaStream_t);
bool df_has_b(int);
cudaError_t launch_elem_df_b(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_b(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_c(int, const dfloat*, cudaStream_t);
bool df_has_c(int);
cudaError_t launch_elem_df_c(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_c(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_d(int, const dfloat*, cudaStream_t);
bool df_has_d(int);
cudaError_t launch_elem_df_d(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_d(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_e(int, const dfloat*, cudaStream_t);
bool df_has_e(int);
cudaError_t launch_elem_df_e(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_e(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_f(int, const dfloat*, cudaStream_t);
bool df_has_f(int);
cudaError_t launch_elem_df_f(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_f(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_g(int, const dfloat*, cudaStream_t);
bool df_has_g(int);
cudaError_t launch_elem_df_g(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_g(const DeviceMesh&, int*, int*, int*, int, bool);
cudaError_t set_df_dconst_h(int, const dfloat*, cudaStream_t);
bool df_has_h(int);
cudaError_t launch_elem_df_h(const DeviceMesh&, const ElemDfArgs&, cudaStream_t);
int elem_df_tile_candidates_h(const DeviceMesh&, int*, int*, int*, int, bool);

cudaError_t set_df_dconst(int p1, const dfloat* host, cudaStream_t s) {
  if (p1 < 2 || p1 > kMaxP1) return cudaErrorInvalidValue;
  if (df_has_a(p1)) return set_df_dconst_a(p1, host, s);
  if (df_has_b(p1)) return set_df_dconst_b(p1, host, s);
  if (df_has_c(p1)) return set_df_dconst_c(p1, host, s);
  if (df_has_d(p1)) return set_df_dconst_d(p1, host, s);
  if (df_has_e(p1)) return set_df_dconst_e(p1, host, s);
  if (df_has_f(p1)) return set_df_dconst_f(p1, host, s);
  if (df_has_g(p1)) return set_df_dconst_g(p1, host, s);
  if (df_has_h(p1)) return set_df_dconst_h(p1, host, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_elem_df(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if (!m.colloc) return launch_elem_dfgl(m, a, s);  // BP1 / BP3 (Gauss quadrature)
  if (m.tune_stage == 3) return launch_elem_dfeo(m, a, s);  // even-odd BK5
  const int p1 = m.p1;
  if (df_has_a(p1)) return launch_elem_df_a(m, a, s);
  if (df_has_b(p1)) return launch_elem_df_b(m, a, s);
  if (df_has_c(p1)) return launch_elem_df_c(m, a, s);
  if (df_has_d(p1)) return launch_elem_df_d(m, a, s);
  if (df_has_e(p1)) return launch_elem_df_e(m, a, s);
  if (df_has_f(p1)) return launch_elem_df_f(m, a, s);
  if (df_has_g(p1)) return launch_elem_df_g(m, a, s);
  if (df_has_h(p1)) return launch_elem_df_h(m, a, s);
  return cudaErrorInvalidValue;
}

int elem_df_tile_candidates(const DeviceMesh& m, int* eb, int* stage, int* ns, int cap, bool pipelined) {
  const int p1 = m.p1;
  if (df_has_a(p1)) return elem_df_tile_candidates_a(m, eb, stage, ns, cap, pipelined);
  if (df_has_b(p1)) return elem_df_tile_candidates_b(m, eb, stage, ns, cap, pipelined);
  if (df_has_c(p1)) return elem_df_tile_candidates_c(m, eb, stage, ns, cap, pipelined);
  if (df_has_d(p1)) return elem_df_tile_candidates_d(m, eb, stage, ns, cap, pipelined);
  if (df_has_e(p1)) return elem_df_tile_candidates_e(m, eb, stage, ns, cap, pipelined);
  if (df_has_f(p1)) return elem_df_tile_candidates_f(m, eb, stage, ns, cap, pipelined);
  if (df_has_g(p1)) return elem_df_tile_candidates_g(m, eb, stage, ns, cap, pipelined);
  if (df_has_h(p1)) return elem_df_tile_candidates_h(m, eb, stage, ns, cap, pipelined);
  return 0;
}

}  // namespace ceedbp
