// Software-pipelined variant of the FP32-pair BK5/BK6 element kernel
// (instantiated for p1 <= 16 with one component, p1 <= 8 with three).
//
// Same arithmetic as elem_df_kernel (splitter accumulation, per-direction
// transpose accumulators, fused (u, w) and alpha), different schedule: each
// group of p1*p1 threads (a slot) works through a sequence of `ns` elements and
// fetches the next element's data while it computes the current one, so the
// dependent l2g -> u gather no longer stalls the warps:
//
//   top of element i:  plain loads of l2g of element i+1 (used an element phase later)
//   end of the gradient phase of element i:
//       cp.async  u of element i+1 (addresses from those l2g registers)
//   all along:  cp.async  G two slabs ahead, continuing into element i+1
//   top of element i+1: wait for this thread's copies; convert u to pairs in
//                 place; one barrier; compute
//
// Every thread copies and converts only its own column (i, j, 0..p1-1) of u
// and G, so each element needs only the two barriers of the contraction (after
// the gather and after the gradient phase).  The u tile in
// shared memory doubles as the pair tile of the r and s derivatives (rows of
// p1+1 pairs, no bank conflicts between row and column reads).
//
// The slab loops are not unrolled (the unrolled element body, ~75 KB of
// code, thrashed the instruction cache); the t-direction values therefore go
// through a private shared tile, and the fused (u, w) takes x_k from the front
// of the column registers, shifted down once per slab.
//
// Shared memory per slot: 3-slab G ring, u tile, r and s gradient tiles (rows
// padded to p1+1 pairs), the private t tile; for p1 = 8 and one component
// 26.5 KB, so four two-slot blocks fit on an SM.  Batched solves pass block
// tables (one problem's range of elements per block) and get a per-problem
// alpha from a segmented reduction, as in elem_df_kernel.
#pragma once

#include "elem_df.cuh"

namespace ceedbp {

template <int P1, int NC>
struct ElemDfpShape {
  static constexpr int PP = P1 * P1, P3 = PP * P1;
  static constexpr int ROW = P1 + 1, SLAB = P1 * ROW, TILE = P1 * SLAB;
  static constexpr int RING = 3 * 6 * PP;  // pairs
};

// layout: [red 32 NC doubles][smax 2 x 4 x 32 u32][sD p1 x (p1+1) pairs] then per slot:
//         [G ring][sU NC tiles][sR NC tiles][sS NC tiles][sT NC x p1^3 pairs]
template <int P1, int NC>
__host__ __device__ inline size_t elem_dfp_head_bytes() {
  const size_t h = sizeof(double) * 32 * NC + sizeof(unsigned) * 256 + sizeof(dfloat) * P1 * (P1 + 1);
  return (h + 15) / 16 * 16;
}

template <int P1, int NC>
__host__ __device__ inline size_t elem_dfp_slot_bytes() {
  using S = ElemDfpShape<P1, NC>;
  const size_t b = sizeof(dfloat) * (size_t(S::RING) + 3 * NC * size_t(S::TILE) + size_t(NC) * S::P3);
  return (b + 15) / 16 * 16;
}

template <int P1, int NC>
inline size_t elem_dfp_smem_bytes(int eb) {
  return elem_dfp_head_bytes<P1, NC>() + size_t(eb) * elem_dfp_slot_bytes<P1, NC>();
}

// Register cap: for p1 <= 8 (one component) two 256-thread blocks per SM; above p1 = 8 one
// slot per block (p1^2 threads), so a thread may use up to 255 registers.
template <int P1, int NC>
__global__ void __launch_bounds__(P1 <= 8 ? 256 : ((P1 * P1 + 31) / 32) * 32, (P1 <= 8 && NC == 1) ? 2 : 1)
    elem_dfp_kernel(const DeviceMesh m, const ElemDfArgs a, const int eb, const int ns) {
  using S = ElemDfpShape<P1, NC>;
  constexpr int PP = S::PP, P3 = S::P3, ROW = S::ROW, SLAB = S::SLAB, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.state != nullptr && a.state->stop) return;

  double* red = reinterpret_cast<double*>(smem_raw);                   // 32 * NC
  unsigned* smax = reinterpret_cast<unsigned*>(red + 32 * NC);        // [2][4][32]
  dfloat* sD = reinterpret_cast<dfloat*>(smax + 256);                 // [P1][ROW]
  const int tid = threadIdx.x;
  const int slot = tid / PP, t = tid - slot * PP;
  const int i = t % P1, j = t / P1;
  const bool in_slot = slot < eb;  // threads past eb slots (rounding to whole warps) only join barriers
  unsigned char* sbase = smem_raw + elem_dfp_head_bytes<P1, NC>() +
                         size_t(in_slot ? slot : 0) * elem_dfp_slot_bytes<P1, NC>();
  dfloat* ring = reinterpret_cast<dfloat*>(sbase);
  dfloat* sU = ring + S::RING;
  dfloat* sR = sU + NC * TILE;
  dfloat* sS = sR + NC * TILE;
  dfloat* sT = sS + NC * TILE;  // [NC][P3] private columns of the t components (unpadded)
  const int my = j * ROW + i;

  for (int q = tid; q < PP; q += blockDim.x) sD[(q / P1) * ROW + (q % P1)] = a.D[q];
  for (int q = tid; q < 256; q += blockDim.x) smax[q] = 0u;
  __syncthreads();

  // elements of this slot: e(s) = first + s * eb + slot, s = 0 .. ns-1, the first `count`
  // elements from `first` (batched solves: one problem's range per block, from the block tables)
  int64_t first = int64_t(blockIdx.x) * eb * ns;
  int64_t count = int64_t(eb) * ns;
  int prob = 0;
  if (a.blk_prob != nullptr) {
    prob = a.blk_prob[blockIdx.x];
    if (!a.bst[prob].c.active) return;  // the whole block belongs to one problem
    first = a.blk_e0[blockIdx.x];
    count = a.blk_n[blockIdx.x];
  }
  auto elem_of = [&](int s) -> int64_t { return first + int64_t(s) * eb + slot; };
  auto live = [&](int s) -> bool {
    return in_slot && s < ns && int64_t(s) * eb + slot < count && elem_of(s) < m.nelem;
  };

  // this thread's column of l2g of sequence entry s (plain loads, consumed an element later)
  auto load_l2g = [&](int s, int (&lg)[P1]) {
    const int* src = m.l2g + elem_of(s) * P3 + t;
#pragma unroll
    for (int k = 0; k < P1; ++k) lg[k] = __ldg(src + k * PP);
  };
  auto dir_mask = [&](const int (&lg)[P1]) -> unsigned {
    unsigned dm = 0u;
#pragma unroll
    for (int k = 0; k < P1; ++k) dm |= unsigned(lg[k] < 0) << k;
    return dm;
  };
  // copy this thread's column of u (8 bytes per value: a double or a pair) to the u tile
  auto fetch_u = [&](const int (&lg)[P1]) {
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int g = lg[k];
      const int64_t gg = g < 0 ? -int64_t(g) - 1 : int64_t(g);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const void* src = a.u_f64 != nullptr ? static_cast<const void*>(a.u_f64 + gg * NC + c)
                                             : static_cast<const void*>(a.u_df + gg * NC + c);
        cp_async8(sU + c * TILE + k * SLAB + my, src);
      }
    }
  };
  // copy this thread's entries of G slab `sl` of sequence entry s into ring position rp
  auto fetch_g = [&](int s, int sl, int rp) {
    const dfloat* src = a.G + elem_of(s) * 6 * P3 + sl * PP + t;
#pragma unroll
    for (int q = 0; q < 6; ++q) cp_async8(ring + rp * 6 * PP + q * PP + t, src + q * P3);
  };

  // ---- prologue: l2g and u of entry 0 and its first two G slabs
  unsigned dmask = 0u;  // bit k: node (i, j, k) of the current entry is a Dirichlet node
  if (live(0)) {
    int lg[P1];
    load_l2g(0, lg);
    dmask = dir_mask(lg);
    fetch_u(lg);
    fetch_g(0, 0, 0);
    if (P1 > 1) fetch_g(0, 1, 1);
  }
  cp_async_commit();

  double dot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dot[c] = 0.0;
  int rp = 0;  // ring position of the current G slab

  for (int s = 0; s < ns; ++s) {
    const bool active = live(s);
    const int b = s & 1;
    unsigned* mx_s = smax + b * 128;        // [4][32] maxima of this entry
    unsigned* mx_o = smax + (b ^ 1) * 128;  // the other entry's, reset during this one
    cp_async_wait_all();
    // l2g of the next entry: its loads fly during this entry's gather and gradient
    int lg_next[P1];
    const bool next_live = live(s + 1);
    if (next_live) load_l2g(s + 1, lg_next);

    // ---- gather: own column of u to pairs (in place) and to registers
    dfloat xc[NC][P1];
    float mx = 0.0f;
    if (active) {
#pragma unroll
      for (int k = 0; k < P1; ++k) {
        const bool dir = (dmask >> k) & 1u;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          dfloat* cell = sU + c * TILE + k * SLAB + my;
          dfloat v;
          if (a.u_f64 != nullptr) v = f64_to_df(*reinterpret_cast<const double*>(cell));
          else v = *cell;
          if (dir && a.mask_in) v = dfloat{0.0f, 0.0f};
          *cell = v;
          xc[c][k] = v;
          mx = fmaxf(mx, fabsf(v.hi));
        }
      }
    }
    slot_max<PP>(&mx_s[slot], mx, active);
    __syncthreads();
    if (in_slot && t == 0) {
      mx_o[slot] = 0u;
      mx_o[32 + slot] = 0u;
      mx_o[64 + slot] = 0u;
      mx_o[96 + slot] = 0u;
    }
    const float sig1 = splitter(a.dnorm_row * __uint_as_float(mx_s[slot]));

    // ---- gradient and geometric factors; slab loop kept rolled (a fully unrolled element
    //      body overflows the instruction cache), so the t components live in the private tile sT
    float mr = 0.0f, ms = 0.0f, mt = 0.0f;
    {
      dfloat Di[P1], Dj[P1];
#pragma unroll
      for (int n = 0; n < P1; ++n) {
        Di[n] = sD[i * ROW + n];
        Dj[n] = sD[j * ROW + n];
      }
#pragma unroll 1
      for (int k = 0; k < P1; ++k) {
        // prefetch the slab two ahead: this element's, or the next element's first two
        const int rp2 = rp + 2 >= 3 ? rp - 1 : rp + 2;
        if (k + 2 < P1) {
          if (active) fetch_g(s, k + 2, rp2);
        } else if (next_live) {
          fetch_g(s + 1, k + 2 - P1, rp2);
        }
        cp_async_commit();
        cp_async_wait<2>();  // this thread's copies of slab k have landed
        const dfloat* gs = ring + rp * 6 * PP + t;
        rp = rp + 1 == 3 ? 0 : rp + 1;
        if (!active) continue;
        dfloat g[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) g[q] = gs[q * PP];
        const float gb = fmaxf(fmaxf(row_abs_sum3(g[0], g[1], g[2]), row_abs_sum3(g[1], g[3], g[4])),
                               row_abs_sum3(g[2], g[4], g[5]));
        const dfloat* dkrow = c_Ddf[P1 - 2] + k * P1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          SplitAcc ar(sig1), as(sig1), at(sig1);
          const dfloat* xs = sU + c * TILE + k * SLAB;
#pragma unroll
          for (int n = 0; n < P1; ++n) {
            const dfloat xr = xs[j * ROW + n];
            const dfloat xq = xs[n * ROW + i];
            const dfloat dk = dkrow[n];
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
          sT[c * P3 + k * PP + t] = vt;
          mr = fmaxf(mr, fabsf(vr.hi));
          ms = fmaxf(ms, fabsf(vs.hi));
          mt = fmaxf(mt, fabsf(vt.hi));
        }
      }
    }
    slot_max<PP>(&mx_s[32 + slot], mr, active);
    slot_max<PP>(&mx_s[64 + slot], ms, active);
    slot_max<PP>(&mx_s[96 + slot], mt, active);
    __syncthreads();
    // every thread of the block is past its reads of this entry's u tile: fetch the next one
    unsigned dmask_next = 0u;
    if (next_live) {
      fetch_u(lg_next);
      dmask_next = dir_mask(lg_next);
    }
    cp_async_commit();
    const float sig_r = splitter(a.dnorm_col * __uint_as_float(mx_s[32 + slot]));
    const float sig_s = splitter(a.dnorm_col * __uint_as_float(mx_s[64 + slot]));
    const float sig_t = splitter(a.dnorm_col * __uint_as_float(mx_s[96 + slot]));

    // ---- transpose gradient, output and the fused (p^e, w^e) of Algorithm 1; the rolled slab
    //      loop takes x_k from the front of the column registers and shifts the column down
    if (active) {
      dfloat acc_dot[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc_dot[c] = dfloat{0.0f, 0.0f};
      dfloat Dni[P1], Dnj[P1];
#pragma unroll
      for (int n = 0; n < P1; ++n) {
        Dni[n] = sD[n * ROW + i];
        Dnj[n] = sD[n * ROW + j];
      }
      dfloat* wl = a.wl + size_t(elem_of(s)) * P3 * NC;
#pragma unroll 1
      for (int k = 0; k < P1; ++k) {
        const int idx = k * PP + t;
        const bool skip = a.skip_dirichlet_out && ((dmask >> k) & 1u);
        const dfloat* dkcol = c_Ddf[P1 - 2] + k;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          SplitAcc acr(sig_r), acs(sig_s), act(sig_t);
          const dfloat* rs = sR + c * TILE + k * SLAB;
          const dfloat* ss = sS + c * TILE + k * SLAB;
          const dfloat* ts = sT + c * P3 + t;
#pragma unroll
          for (int n = 0; n < P1; ++n) {
            const dfloat vr = rs[j * ROW + n];
            const dfloat vs = ss[n * ROW + i];
            const dfloat vt = ts[n * PP];
            const dfloat dk = dkcol[n * P1];
            acr.add(Dni[n].hi, Dni[n].lo, vr.hi, vr.lo);
            acs.add(Dnj[n].hi, Dnj[n].lo, vs.hi, vs.lo);
            act.add(dk.hi, dk.lo, vt.hi, vt.lo);
          }
          const dfloat w = dw_add(dw_add(acr.result(sig_r), acs.result(sig_s)), act.result(sig_t));
          if (!skip) {
            dfloat wn;
            two_sum(w.hi, w.lo, wn.hi, wn.lo);
            wl[size_t(idx) * NC + c] = wn;
          }
          acc_dot[c] = dw_add(acc_dot[c], dw_mul(w, xc[c][0]));
#pragma unroll
          for (int n = 0; n + 1 < P1; ++n) xc[c][n] = xc[c][n + 1];
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) dot[c] += df_to_f64(acc_dot[c]);
    }
    dmask = dmask_next;
    // the next entry's gather rewrites the u tile only after its own copies land, and the
    // gradient tiles only after its first barrier, by which time every thread is done here
  }
  cp_async_wait_all();

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

template <int P1, int NC>
cudaError_t elem_dfp_attr() {
  static const cudaError_t attr = cudaFuncSetAttribute(elem_dfp_kernel<P1, NC>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       int(kMaxSmemPerBlock));
  return attr;
}

template <int P1, int NC>
inline bool elem_dfp_shape_ok(int eb) {
  const size_t smem = elem_dfp_smem_bytes<P1, NC>(eb);
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  if (smem > kMaxSmemPerBlock || nthreads > 1024) return false;
  if (elem_dfp_attr<P1, NC>() != cudaSuccess) return false;
  // the launch bound caps the block size (the occupancy query alone does not reject larger blocks)
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, elem_dfp_kernel<P1, NC>) != cudaSuccess || nthreads > fa.maxThreadsPerBlock)
    return false;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, elem_dfp_kernel<P1, NC>, nthreads, smem) != cudaSuccess)
    return false;
  return nb >= 1;
}

template <int P1, int NC>
cudaError_t launch_elem_dfp_t(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  const int eb = m.tune_eb > 0 ? m.tune_eb : 1;
  const int ns = m.tune_ns > 0 ? m.tune_ns : 8;
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  const size_t smem = elem_dfp_smem_bytes<P1, NC>(eb);
  if (smem > kMaxSmemPerBlock) return cudaErrorInvalidConfiguration;
  const cudaError_t attr = elem_dfp_attr<P1, NC>();
  if (attr != cudaSuccess) return attr;
  const int64_t per_block = int64_t(eb) * ns;
  const int64_t blocks = a.blk_prob != nullptr ? int64_t(a.batch_blocks) : (m.nelem + per_block - 1) / per_block;
  elem_dfp_kernel<P1, NC><<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb, ns);
  return cudaGetLastError();
}

}  // namespace ceedbp
