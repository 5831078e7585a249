// Definition of the opaque ceedbp context (shared by the C-ABI translation units).
#pragma once

#include <string>
#include <vector>

#include "df.cuh"
#include "internal.h"
#include "kernel_args.h"

struct GraphEntry {
  double* x;
  int n;
  int profile;
  int mode;  // 0: FP64 / pair iteration, else the CEEDBP_MIXED_* precision of the inner iterations
  cudaGraphExec_t exec;
};

struct ceedbp_ctx {
  ceedbp_params prm{};
  int ncomp = 1, p1 = 0, q = 0, op_kind = ceedbp::kStiff;
  bool colloc = false;
  cudaStream_t stream = nullptr;
  ceedbp::DeviceMesh mesh{};
  int* d_l2g = nullptr;
  int* d_off = nullptr;
  int* d_slots = nullptr;
  double* d_basis = nullptr;
  double* d_G = nullptr;
  double* d_X = nullptr;  // [E][3][p1^3] coordinates when the factors are recomputed
  int* d_l2g_id = nullptr;  // identity gather map of ceedbp_bk_apply (allocated on its first call)
  double* d_Mq = nullptr;
  double* d_dinv = nullptr;
  double* d_mdiag = nullptr;
  double* d_wl = nullptr;
  double* d_r = nullptr;
  double* d_p = nullptr;
  double* d_ax = nullptr;
  // FP32-pair path (arith == CEEDBP_ARITH_DF64): pair copies of G, D and the
  // Jacobi inverse; the CG pair vectors reuse d_r, d_p, d_ax and the local
  // scratch d_wl (a pair has the size of a double).
  int arith = 0;
  bool pipelined_only = false;  // batched groups: tune among the pipelined pair-kernel shapes only
  double beta = 0.0;  // Helmholtz coefficient of Eq. (17) (ceedbp_set_helmholtz)
  ceedbp::dfloat* d_Gdf = nullptr;
  ceedbp::dfloat* d_Ddf = nullptr;
  ceedbp::dfloat* d_dinvdf = nullptr;
  float dnorm_row = 0.0f, dnorm_col = 0.0f;
  int wait_polls = ceedbp::kDefaultWaitPolls;  // first bounded wait of the staged pair schedule
  // defect correction: low-precision G copies, FP32 inner vectors, outer norms
  float* d_G32 = nullptr;
  void* d_Gbf = nullptr;
  float* d_dinv32 = nullptr;
  float* d_xin = nullptr;
  float* d_rin = nullptr;
  void* d_pin = nullptr;  // n * ncomp * 4 bytes (FP32 or BF16 direction)
  double* d_outer = nullptr;
  double* h_outer = nullptr;
  bool tc_ready = false;  // the tensor-core inner operator was prepared (CEEDBP_MIXED_FP32_TC)
  // variable coefficient: coefficient-free factors (kept when kappa is used)
  double* d_Ghat = nullptr;
  double* d_scal = nullptr;  // small device outputs (misfit)
  double* h_scal = nullptr;
  double* d_part_apply = nullptr;
  double* d_part_vec = nullptr;
  ceedbp::SolveState* d_state = nullptr;
  ceedbp::SolveState* h_state = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> prof;  // 4 events per profiled iteration
  std::vector<GraphEntry> graphs;
  std::string err;
};

