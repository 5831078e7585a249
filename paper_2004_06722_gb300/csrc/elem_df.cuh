// FP64-accurate BK5/BK6 element kernel on the FP32 pipe (pairs of floats).
//
// Same operator as elem_kernel with GLL collocation (Eq. (22) with J = I):
//   u_r = D_1 u, u_s = D_2 u, u_t = D_3 u           (3 x p1 pair products per node)
//   (w_r, w_s, w_t) = G (u_r, u_s, u_t)              (Eq. (23) factors, stored as pairs)
//   w = D_1^T w_r + D_2^T w_s + D_3^T w_t            (3 x p1 pair products per node)
// and the fused (u, w) of Algorithm 1.  Every sum of pair products uses the
// splitter accumulation of df.cuh with a power-of-two splitter derived from an
// element-wide bound (|D|_inf max|u| for the gradient; |D^T|_inf max|w_r| etc.
// for each of the three transpose sums, added afterwards as pairs) or a
// per-point bound (the G product), so a pair product costs 6 FP32
// instructions and no FP64 instruction is issued.
//
// Shared-memory tiles use rows of p1+1 pairs so that the row (u_r) and column
// (u_s) reads of a warp hit distinct banks.
#pragma once

#include "common.cuh"
#include "df.cuh"
#include "kernel_args.h"

namespace ceedbp {

// GLL derivative matrices as pairs, one slot of kMaxP1^2 per order (p1 - 2):
// the t-direction operands D[k][n] are read straight from the constant bank.
// Internal linkage: every translation unit that instantiates the kernels (one
// per group of orders, compiled in parallel) has its own copy and its own
// setter (elem_df_group.cuh).
static __constant__ dfloat c_Ddf[kMaxP1 - 1][kMaxP1 * kMaxP1];

template <int P1, int NC, bool STAGE>
struct ElemDfShape {
  static constexpr int PP = P1 * P1, P3 = PP * P1;
  static constexpr int ROW = P1 + 1;            // padded row length (pairs)
  static constexpr int SLAB = P1 * ROW;         // padded slab (pairs)
  static constexpr int TILE = P1 * SLAB;        // padded tile (pairs)
  // G of an element (6 p1^3 pairs, contiguous in memory) is staged in shared
  // memory by one bulk asynchronous copy when it fits next to the tiles.
  static constexpr bool STAGE_G = STAGE && P1 <= 10;
  // staged: the whole element's G; otherwise a ring of 3 slabs filled by
  // per-thread cp.async two slabs ahead of use
  static constexpr int GSTAGE = STAGE_G ? 6 * P3 : 3 * 6 * PP;  // pairs per element
};

template <int P1, int NC>
inline int elem_df_per_block() {
  int eb = 128 / (P1 * P1 * NC);
  return eb < 1 ? 1 : eb;
}

// layout: [mbarrier 16 B][red 32 NC doubles][smax 128 u32][sD p1 x (p1+1) pairs, padded to 16 B]
//         then per element: [G stage][sX][sR][sS]
template <int P1, int NC, bool STAGE>
__host__ __device__ inline size_t elem_df_head_bytes() {
  using S = ElemDfShape<P1, NC, STAGE>;
  const size_t h = 16 + sizeof(double) * 32 * NC + sizeof(unsigned) * 128 + sizeof(dfloat) * P1 * S::ROW;
  return (h + 15) / 16 * 16;
}

template <int P1, int NC, bool STAGE>
__host__ __device__ inline size_t elem_df_slot_pairs() {
  using S = ElemDfShape<P1, NC, STAGE>;
  return size_t(S::GSTAGE) + 3 * NC * S::TILE + 1;  // +1 pair keeps every slot 16-byte aligned
}

template <int P1, int NC, bool STAGE>
inline size_t elem_df_smem_bytes(int eb) {
  size_t slot = elem_df_slot_pairs<P1, NC, STAGE>();
  slot = (slot + 1) / 2 * 2;
  return elem_df_head_bytes<P1, NC, STAGE>() + sizeof(dfloat) * size_t(eb) * slot;
}

__device__ __forceinline__ float row_abs_sum3(dfloat a, dfloat b, dfloat c) {
  return fabsf(a.hi) + fabsf(b.hi) + fabsf(c.hi);
}

// max of v over the lanes of one element; lanes of an element are whole warps when p1^2 % 32 == 0
template <int PP>
__device__ __forceinline__ void slot_max(unsigned* dst, float v, bool active) {
  if constexpr (PP % 32 == 0) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (active && (threadIdx.x & 31) == 0) atomicMax(dst, m);
  } else {
    if (active) atomicMax(dst, __float_as_uint(v));
  }
}

constexpr int kMbarPolls = kDefaultWaitPolls;

// Register cap: for p1 <= 8 (one component) keep two 256-thread (or four 128-thread) blocks per SM.
template <int P1, int NC, bool STAGE>
__global__ void __launch_bounds__(P1 <= 8 ? 256 : 1024, (P1 <= 8 && NC == 1) ? 2 : 1)
    elem_df_kernel(const DeviceMesh m, const ElemDfArgs a, const int eb) {
  using S = ElemDfShape<P1, NC, STAGE>;
  constexpr int PP = S::PP, P3 = S::P3, ROW = S::ROW, SLAB = S::SLAB, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.state != nullptr && a.state->stop) return;

  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + 16);                 // 32 * NC
  unsigned* smax = reinterpret_cast<unsigned*>(red + 32 * NC);            // [4][32]
  dfloat* sD = reinterpret_cast<dfloat*>(smax + 128);                     // [P1][ROW]
  dfloat* ebuf = reinterpret_cast<dfloat*>(smem_raw + elem_df_head_bytes<P1, NC, STAGE>());
  size_t slot_pairs = elem_df_slot_pairs<P1, NC, STAGE>();
  slot_pairs = (slot_pairs + 1) / 2 * 2;

  const int tid = threadIdx.x;
  const int slot = tid / PP, t = tid - slot * PP;
  const int i = t % P1, j = t / P1;
  int64_t e0;
  int nact;
  int prob = 0;
  if (a.blk_prob != nullptr) {  // batched: this block holds elements of one problem
    prob = a.blk_prob[blockIdx.x];
    if (!a.bst[prob].c.active) return;
    e0 = a.blk_e0[blockIdx.x];
    nact = a.blk_n[blockIdx.x];
  } else {
    e0 = int64_t(blockIdx.x) * eb;
    const int64_t nact64 = m.nelem - e0;
    nact = nact64 < eb ? int(nact64) : eb;
  }
  const int64_t e = e0 + slot;
  const bool active = slot < nact;

  if constexpr (S::STAGE_G) {
    if (tid == 0) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  for (int q = tid; q < P1 * P1; q += blockDim.x) sD[(q / P1) * ROW + (q % P1)] = a.D[q];
  for (int q = tid; q < 128; q += blockDim.x) smax[q] = 0u;
  __syncthreads();
  if constexpr (S::STAGE_G) {
    if (tid == 0) {
      const unsigned bytes = unsigned(sizeof(dfloat)) * 6u * P3;
      mbar_expect_tx(bar, bytes * unsigned(nact));
      for (int sl = 0; sl < nact; ++sl)
        bulk_copy_g2s(ebuf + size_t(sl) * slot_pairs, a.G + (e0 + sl) * 6 * P3, bytes, bar);
    }
  }

  dfloat* sG = ebuf + size_t(active ? slot : 0) * slot_pairs;
  dfloat* sX = sG + S::GSTAGE;
  dfloat* sR = sX + NC * TILE;
  dfloat* sS = sR + NC * TILE;
  const int* l2g = m.l2g + e * P3;
  const int my = j * ROW + i;  // position of (i, j) inside a padded slab
  if constexpr (!S::STAGE_G) {
    if (active) {  // first two slabs of G in flight during the gather
      const dfloat* Gg0 = a.G + size_t(e) * 6 * P3;
#pragma unroll
      for (int s2 = 0; s2 < 2 && s2 < P1; ++s2) {
#pragma unroll
        for (int q = 0; q < 6; ++q) cp_async8(sG + s2 * 6 * PP + q * PP + t, Gg0 + q * P3 + s2 * PP + t);
        cp_async_commit();
      }
    }
  }

  // ---- gather the column (i, j, 0..p1-1) of u^e = Q u
  dfloat xc[NC][P1];
  unsigned dmask = 0u;  // bit k: node (i, j, k) is a Dirichlet node
  float mx = 0.0f;
  if (active) {
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int g = __ldg(l2g + t + PP * k);
      const bool dir = g < 0;
      dmask |= unsigned(dir) << k;
      const int gg = dir ? -g - 1 : g;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        dfloat v{0.0f, 0.0f};
        if (!(dir && a.mask_in)) {
          if (a.u_f64 != nullptr) v = f64_to_df(__ldg(a.u_f64 + size_t(gg) * NC + c));
          else v = a.u_df[size_t(gg) * NC + c];
        }
        xc[c][k] = v;
        sX[c * TILE + k * SLAB + my] = v;
        mx = fmaxf(mx, fabsf(v.hi));
      }
    }
  }
  slot_max<PP>(&smax[slot], mx, active);
  bool staged = true;
  if constexpr (S::STAGE_G) staged = mbar_wait(bar, 0, a.first_wait);
  __syncthreads();
  const float sig1 = splitter(a.dnorm_row * __uint_as_float(smax[slot]));

  // ---- gradient and geometric factors
  dfloat wt[NC][P1];
  float mr = 0.0f, ms = 0.0f, mt = 0.0f;
  if (active) {
    dfloat Di[P1], Dj[P1];
#pragma unroll
    for (int n = 0; n < P1; ++n) {
      Di[n] = sD[i * ROW + n];
      Dj[n] = sD[j * ROW + n];
    }
    const dfloat* Gg = a.G + size_t(e) * 6 * P3;
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int pt = k * PP + t;
      dfloat g[6];
      if constexpr (S::STAGE_G) {
#pragma unroll
        for (int q = 0; q < 6; ++q) g[q] = sG[q * P3 + pt];
      } else {
        if (k + 2 < P1) {
          dfloat* ring = sG + ((k + 2) % 3) * 6 * PP;
#pragma unroll
          for (int q = 0; q < 6; ++q) cp_async8(ring + q * PP + t, Gg + q * P3 + pt + 2 * PP);
        }
        cp_async_commit();
        cp_async_wait<2>();  // this thread's copies of slab k have landed
        const dfloat* ring = sG + (k % 3) * 6 * PP;
#pragma unroll
        for (int q = 0; q < 6; ++q) g[q] = ring[q * PP + t];
      }
      const float gb = fmaxf(fmaxf(row_abs_sum3(g[0], g[1], g[2]), row_abs_sum3(g[1], g[3], g[4])),
                             row_abs_sum3(g[2], g[4], g[5]));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        SplitAcc ar(sig1), as(sig1), at(sig1);
        const dfloat* xs = sX + c * TILE + k * SLAB;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          const dfloat xr = xs[j * ROW + n];
          const dfloat xq = xs[n * ROW + i];
          const dfloat dk = c_Ddf[P1 - 2][k * P1 + n];
          ar.add(Di[n].hi, Di[n].lo, xr.hi, xr.lo);
          as.add(Dj[n].hi, Dj[n].lo, xq.hi, xq.lo);
          at.add(dk.hi, dk.lo, xc[c][n].hi, xc[c][n].lo);
        }
        const dfloat ur = ar.result(sig1), us = as.result(sig1), ut = at.result(sig1);
        const float um = fmaxf(fmaxf(fabsf(ur.hi), fabsf(us.hi)), fabsf(ut.hi));
        const float sg = splitter(gb * um);
        SplitAcc wr(sg), ws(sg), wq(sg);
        wr.add(g[0].hi, g[0].lo, ur.hi, ur.lo);
        wr.add(g[1].hi, g[1].lo, us.hi, us.lo);
        wr.add(g[2].hi, g[2].lo, ut.hi, ut.lo);
        ws.add(g[1].hi, g[1].lo, ur.hi, ur.lo);
        ws.add(g[3].hi, g[3].lo, us.hi, us.lo);
        ws.add(g[4].hi, g[4].lo, ut.hi, ut.lo);
        wq.add(g[2].hi, g[2].lo, ur.hi, ur.lo);
        wq.add(g[4].hi, g[4].lo, us.hi, us.lo);
        wq.add(g[5].hi, g[5].lo, ut.hi, ut.lo);
        const dfloat vr = wr.result(sg), vs = ws.result(sg), vt = wq.result(sg);
        sR[c * TILE + k * SLAB + my] = vr;
        sS[c * TILE + k * SLAB + my] = vs;
        wt[c][k] = vt;
        mr = fmaxf(mr, fabsf(vr.hi));
        ms = fmaxf(ms, fabsf(vs.hi));
        mt = fmaxf(mt, fabsf(vt.hi));
      }
    }
  }
  slot_max<PP>(&smax[32 + slot], mr, active);
  slot_max<PP>(&smax[64 + slot], ms, active);
  slot_max<PP>(&smax[96 + slot], mt, active);
  __syncthreads();
  // one accumulator per direction, each with its own element-wide splitter
  const float sig_r = splitter(a.dnorm_col * __uint_as_float(smax[32 + slot]));
  const float sig_s = splitter(a.dnorm_col * __uint_as_float(smax[64 + slot]));
  const float sig_t = splitter(a.dnorm_col * __uint_as_float(smax[96 + slot]));

  // ---- transpose gradient, output, fused dot
  double dot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dot[c] = 0.0;
  if (active) {
    dfloat Dni[P1], Dnj[P1];
#pragma unroll
    for (int n = 0; n < P1; ++n) {
      Dni[n] = sD[n * ROW + i];
      Dnj[n] = sD[n * ROW + j];
    }
    dfloat* wl = a.wl + size_t(e) * P3 * NC;
    dfloat acc_dot[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc_dot[c] = dfloat{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int idx = k * PP + t;
      const bool skip = a.skip_dirichlet_out && ((dmask >> k) & 1u);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        SplitAcc acr(sig_r), acs(sig_s), act(sig_t);
        const dfloat* rs = sR + c * TILE + k * SLAB;
        const dfloat* ss = sS + c * TILE + k * SLAB;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          const dfloat vr = rs[j * ROW + n];
          const dfloat vs = ss[n * ROW + i];
          const dfloat dk = c_Ddf[P1 - 2][n * P1 + k];
          acr.add(Dni[n].hi, Dni[n].lo, vr.hi, vr.lo);
          acs.add(Dnj[n].hi, Dnj[n].lo, vs.hi, vs.lo);
          act.add(dk.hi, dk.lo, wt[c][n].hi, wt[c][n].lo);
        }
        const dfloat w = dw_add(dw_add(acr.result(sig_r), acs.result(sig_s)), act.result(sig_t));
        if (!skip) {
          dfloat wn;
          two_sum(w.hi, w.lo, wn.hi, wn.lo);
          wl[size_t(idx) * NC + c] = wn;
        }
        acc_dot[c] = dw_add(acc_dot[c], dw_mul(w, xc[c][k]));
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) dot[c] = df_to_f64(acc_dot[c]);
  }
  if constexpr (S::STAGE_G) {
    // a copy that did not land in time: flag it, give it a second bounded wait
    // before the block's shared memory is released
    if (__syncthreads_or(!staged)) {
      if (tid == 0) {
        if (a.fault) atomicExch(a.fault, 1);
        mbar_wait(bar, 0, kMbarPolls);
      }
      __syncthreads();
    }
  }

  if constexpr (NC == 1) {
    if (a.blk_prob != nullptr) {  // per-problem alpha from a segmented last-block reduction
      const int b0 = a.prob_blk0[prob];
      if (grid_sum_last<1>(dot, a.partials + b0, a.prob_nblk[prob], int(blockIdx.x) - b0,
                           &a.bst[prob].ticket[kTicketApply], red)) {
        if (threadIdx.x == 0) {
          CompScalars& cs = a.bst[prob].c;
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
      return;
    }
  }
  if (a.partials != nullptr) {
    if (grid_sum_last<NC>(dot, a.partials, gridDim.x, blockIdx.x, &a.state->ticket[kTicketApply], red)) {
      if (threadIdx.x == 0) {
        SolveState* st = a.state;
        int any = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          CompScalars& cs = st->c[c];
          if (!cs.active) continue;
          const double pAp = dot[c];
          cs.pAp = pAp;
          if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(cs.rz)) {
            cs.status = CEEDBP_EBREAKDOWN;
            cs.alpha = 0.0;
            if (!st->fixed) cs.active = 0;
          } else {
            cs.alpha = cs.rz / pAp;
          }
          any |= cs.active;
        }
        if (!any) st->stop = 1;
      }
    }
  }
}

constexpr size_t kMaxSmemPerBlock = 220 * 1024;  // below the 227 KB opt-in limit with room for static shared memory

template <int P1, int NC, bool STAGE>
cudaError_t elem_df_attr() {
  static const cudaError_t attr = cudaFuncSetAttribute(elem_df_kernel<P1, NC, STAGE>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       int(kMaxSmemPerBlock));
  return attr;
}

// elements per block: the tuned value when set, else the default
template <int P1, int NC>
inline int elem_df_eb(const DeviceMesh& m) {
  return m.tune_eb > 0 ? m.tune_eb : elem_df_per_block<P1, NC>();
}

// Whether a shape (elements per block, staging) can run: shared memory within
// the limit and at least one block resident per SM (registers included).
template <int P1, int NC, bool STAGE>
inline bool elem_df_shape_ok(int eb) {
  const size_t smem = elem_df_smem_bytes<P1, NC, STAGE>(eb);
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  if (smem > kMaxSmemPerBlock || nthreads > 1024) return false;
  if (elem_df_attr<P1, NC, STAGE>() != cudaSuccess) return false;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, elem_df_kernel<P1, NC, STAGE>) != cudaSuccess || nthreads > fa.maxThreadsPerBlock)
    return false;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, elem_df_kernel<P1, NC, STAGE>, nthreads, smem) !=
      cudaSuccess)
    return false;
  return nb >= 1;
}

template <int P1, int NC, bool STAGE>
cudaError_t launch_elem_df_s(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  const int eb = elem_df_eb<P1, NC>(m);
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  const size_t smem = elem_df_smem_bytes<P1, NC, STAGE>(eb);
  if (smem > kMaxSmemPerBlock) return cudaErrorInvalidConfiguration;
  const cudaError_t attr = elem_df_attr<P1, NC, STAGE>();
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = a.blk_prob != nullptr ? int64_t(a.batch_blocks) : (m.nelem + eb - 1) / eb;
  elem_df_kernel<P1, NC, STAGE><<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

template <int P1, int NC>
cudaError_t launch_elem_df_t(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if constexpr (P1 <= 10) {
    if (m.tune_stage) return launch_elem_df_s<P1, NC, true>(m, a, s);
  }
  return launch_elem_df_s<P1, NC, false>(m, a, s);
}

// candidate shapes for the autotuner: (elements per block, staged) pairs that can run
template <int P1, int NC>
inline int elem_df_candidates(int* eb_out, int* stage_out, int cap) {
  int n = 0;
  for (int eb = 1; eb <= 4 && n < cap; ++eb) {
    if (elem_df_shape_ok<P1, NC, false>(eb)) {
      eb_out[n] = eb;
      stage_out[n++] = 0;
    }
    if constexpr (P1 <= 10) {
      if (n < cap && elem_df_shape_ok<P1, NC, true>(eb)) {
        eb_out[n] = eb;
        stage_out[n++] = 1;
      }
    }
  }
  return n;
}

}  // namespace ceedbp
