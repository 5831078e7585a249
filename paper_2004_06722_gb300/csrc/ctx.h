// Definition of the opaque ceedbp context (shared by the C-ABI translation units).
#pragma once

#include <string>
#include <vector>

#include "internal.h"

struct GraphEntry {
  double* x;
  int n;
  int profile;
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
  double* d_Mq = nullptr;
  double* d_dinv = nullptr;
  double* d_mdiag = nullptr;
  double* d_wl = nullptr;
  double* d_r = nullptr;
  double* d_p = nullptr;
  double* d_ax = nullptr;
  double* d_part_apply = nullptr;
  double* d_part_vec = nullptr;
  ceedbp::SolveState* d_state = nullptr;
  ceedbp::SolveState* h_state = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> prof;  // 4 events per profiled iteration
  std::vector<GraphEntry> graphs;
  std::string err;
};

