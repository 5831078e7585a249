// Device helpers shared by the ceedbp kernels: deterministic block and grid
// reductions (fixed summation order, no floating-point atomics).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace ceedbp {

// Sum of v over the block, valid in thread 0.  The order of additions depends
// only on the block shape, so repeated launches give identical bits.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red /* >= 32*NV doubles */) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5, nwarps = (nthreads + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nwarps ? red[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
}

// Grid reduction by the last block to finish: every block stores its NV
// partial sums at partials[k * nblocks + block]; the last block to take a
// ticket re-reads all partials in index order and returns true in every one
// of its threads with the totals in v (valid in thread 0).  Requires blockDim
// to be a multiple of 32.  The ticket is reset for the next launch.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partials, int nblocks, int block,
                                              unsigned int* ticket, double* red) {
  __shared__ bool s_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  block_sum<NV>(v, red);
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[size_t(k) * nblocks + block] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == unsigned(nblocks) - 1u);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = 0.0;
    for (int i = tid; i < nblocks; i += nthreads) x += __ldcg(partials + size_t(k) * nblocks + i);
    v[k] = x;
  }
  block_sum<NV>(v, red);
  if (tid == 0) *ticket = 0u;
  return true;
}

// Batched solves: the blocks of one problem form a contiguous range starting at
// prob_blk0[prob]; that problem's (p, A p) is summed over its own blocks by the
// last of them to finish (fixed order), which writes the problem's alpha.
__device__ __forceinline__ void batch_alpha(double (&dot)[1], double* partials, const int* prob_blk0,
                                            const int* prob_nblk, BatchScalars* bst, int prob, double* red) {
  const int b0 = prob_blk0[prob];
  if (grid_sum_last<1>(dot, partials + b0, prob_nblk[prob], int(blockIdx.x) - b0, &bst[prob].ticket[kTicketApply],
                       red)) {
    if (threadIdx.x == 0) {
      CompScalars& cs = bst[prob].c;
      const double pAp = dot[0];
      cs.pAp = pAp;
      if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(cs.rz)) {
        cs.status = CEEDBP_EBREAKDOWN;
        cs.alpha = 0.0;
      } else {
        cs.alpha = cs.rz / pAp;
      }
    }
  }
}

}  // namespace ceedbp
