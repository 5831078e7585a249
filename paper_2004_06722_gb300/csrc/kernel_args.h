// Argument blocks of the FP32-pair and low-precision element kernels (shared
// by the kernel translation units and the C-ABI implementation).
#pragma once

#include "df.cuh"
#include "internal.h"

namespace ceedbp {

// Polls of a bounded mbarrier wait before a kernel gives up on its staging copy.
constexpr int kDefaultWaitPolls = 1 << 22;

struct ElemDfArgs {
  const double* u_f64;   // global input in FP64 (apply), or nullptr
  const dfloat* u_df;    // global input as pairs (CG direction), or nullptr
  dfloat* wl;            // local output [E p1^3][ncomp] pairs
  const dfloat* G;       // [E][6][p1^3] pairs
  const dfloat* D;       // [p1][p1] pairs of the GLL derivative matrix
  float dnorm_row;       // max_i sum_n |D_in| (rounded up)
  float dnorm_col;       // max_i sum_n |D_ni| (rounded up)
  double* partials;      // [ncomp][nblocks] or nullptr
  SolveState* state;     // CG scalars (alpha from the fused dot) or nullptr
  int mask_in;
  int skip_dirichlet_out;
  int* fault;            // set to 1 if the staging copy of G does not complete (bounded wait)
  int first_wait = kDefaultWaitPolls;  // polls of the wait for the staged G (0: give up at once);
                                       // the draining wait before exit always keeps the default
  // batched solves (one scalar problem per segment of blocks); nullptr otherwise
  const int* blk_prob;   // [nblocks] problem of each block
  const int* blk_e0;     // [nblocks] first element of the block
  const int* blk_n;      // [nblocks] elements in the block (<= elements per block)
  const int* prob_blk0;  // [nprob] first block of each problem
  const int* prob_nblk;  // [nprob] number of blocks of each problem
  BatchScalars* bst;     // [nprob] per-problem CG scalars
  int batch_blocks;      // grid size of a batched launch (entries of blk_prob)
};

struct ElemLpArgs {
  const void* u;        // direction p [nglobal][ncomp] in the storage type
  float* wl;            // [E p1^3][ncomp]
  const void* G;        // [E][6][p1^3] in the storage type
  double* partials;     // [ncomp][nblocks] or nullptr
  SolveState* state;    // inner CG scalars or nullptr
};

}  // namespace ceedbp
