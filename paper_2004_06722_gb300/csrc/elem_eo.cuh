// FP64 BK5/BK6 element kernel with the even-odd decomposition of the 1D
// contractions (the symmetry of Eq. (37); Solomonoff 1992, Kopriva 2009).
//
// The GLL derivative matrix D and its transpose are centro-antisymmetric:
// D[p1-1-i][p1-1-j] = -D[i][j].  With h = p1/2 (even p1), x+_j = x_j + x_{p1-1-j},
// x-_j = x_j - x_{p1-1-j} and E_ij = (D_ij + D_{i,p1-1-j})/2, O_ij = (D_ij - D_{i,p1-1-j})/2
// (i, j < h), one 1D product y = D x is
//   y_i = S_E + S_O,   y_{p1-1-i} = S_O - S_E,   S_E = sum_j E_ij x+_j,  S_O = sum_j O_ij x-_j,
// i.e. p1^2/2 multiply-adds instead of p1^2.  On GB300 the FP64 pipe bounds this
// kernel, so the saved FP64 instructions are saved time.
//
// Thread mapping: one thread per mirror octet of nodes {i, p1-1-i} x {j, p1-1-j}
// x {k, p1-1-k} (i, j, k < h), so both outputs of every 1D pair product in all
// three directions belong to the same thread.  The decomposed input lines are
// exchanged through shared memory; G, the transpose and the output stay per
// thread.  Same operator, layout and fused (u, w) dot as elem_kernel.
#pragma once

#include "common.cuh"

namespace ceedbp {

template <int P1>
struct EoShape {
  static constexpr int H = P1 / 2, H3 = H * H * H, PP = P1 * P1, P3 = PP * P1;
  static constexpr int HALF = P1 * P1 * H;  // one sign of one direction's decomposed tile
  static constexpr int TILE = 6 * HALF;     // r+, r-, s+, s-, t+, t- (doubles)
};

template <int P1, int NC>
inline int elem_eo_per_block() {
  constexpr int H3 = EoShape<P1>::H3;
  int eb = 128 / (H3 * NC);
  return eb < 1 ? 1 : eb;
}

template <int P1, int NC>
inline size_t elem_eo_smem_bytes(int eb) {
  using S = EoShape<P1>;
  return sizeof(double) * (4 * S::H * S::H + 32 * NC + size_t(eb) * NC * S::TILE);
}

// node index of octet corner (bi, bj, bk) in {0,1}^3 of octet (i, j, k)
template <int P1>
__device__ __forceinline__ int eo_node(int i, int j, int k, int bi, int bj, int bk) {
  const int ii = bi ? P1 - 1 - i : i, jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
  return ii + P1 * (jj + P1 * kk);
}

// One folded line product: S_E = sum_n E_n x+_n, then S_O accumulated on top of it, so that
// y0 = S_E + S_O comes out of the chain and y1 = S_O - S_E = (S_E + S_O) - 2 S_E is one fma --
// one FP64 operation fewer per output pair than summing S_E and S_O apart and combining them.
template <int H>
__device__ __forceinline__ void eo_pair(const double* E, const double* O, const double* xp, const double* xm,
                                        double& y0, double& y1) {
  double se = __dmul_rn(E[0], xp[0]);
#pragma unroll
  for (int n = 1; n < H; ++n) se = __fma_rn(E[n], xp[n], se);
  double s = se;
#pragma unroll
  for (int n = 0; n < H; ++n) s = __fma_rn(O[n], xm[n], s);
  y0 = s;
  y1 = __fma_rn(-2.0, se, s);
}

// HELM: the Helmholtz term beta B u of Eq. (17) is compiled in only for beta != 0, so the plain
// stiffness kernel carries no extra registers or branches.  BATCH: the block tables and per-problem
// reductions of batched solves (one component), likewise compiled in only where used.
template <int P1, int NC, bool HELM, bool BATCH = false>
__global__ void elem_eo_kernel(const DeviceMesh m, const ElemArgs a, const int eb) {
  using S = EoShape<P1>;
  constexpr int H = S::H, H3 = S::H3, P3 = S::P3, HALF = S::HALF;
  extern __shared__ double smem_eo[];
  if (a.state != nullptr && a.state->stop) return;
  double* sE = smem_eo;          // [H][H] even part of D (gradient)
  double* sO = sE + H * H;       // [H][H] odd part of D
  double* sEt = sO + H * H;      // [H][H] even part of D^T (transpose)
  double* sOt = sEt + H * H;     // [H][H] odd part of D^T
  double* red = sOt + H * H;     // 32 * NC
  double* tiles = red + 32 * NC;

  const int tid = threadIdx.x;
  const int slot = tid / H3, o = tid - slot * H3;
  const int i = o % H, j = (o / H) % H, k = o / (H * H);
  int64_t e0 = int64_t(blockIdx.x) * eb;
  int nact = m.nelem - e0 < eb ? int(m.nelem - e0) : eb;
  int prob = 0;
  if constexpr (BATCH) {  // batched: this block holds elements of one problem
    prob = a.blk_prob[blockIdx.x];
    if (!a.bst[prob].c.active) return;
    e0 = a.blk_e0[blockIdx.x];
    nact = a.blk_n[blockIdx.x];
  }
  const int64_t e = e0 + slot;
  const bool active = slot < nact;

  // E, O of D and of D^T from the FP64 derivative table Dq [P1][P1]
  const double* D = m.basis + 2 * P1 * P1;
  for (int q = tid; q < H * H; q += blockDim.x) {
    const int r = q / H, c = q % H;
    const double d0 = D[r * P1 + c], d1 = D[r * P1 + (P1 - 1 - c)];
    sE[q] = 0.5 * (d0 + d1);
    sO[q] = 0.5 * (d0 - d1);
    const double t0 = D[c * P1 + r], t1 = D[(P1 - 1 - c) * P1 + r];  // D^T[r][c], D^T[r][p1-1-c]
    sEt[q] = 0.5 * (t0 + t1);
    sOt[q] = 0.5 * (t0 - t1);
  }

  double* T = tiles + size_t(active ? slot : 0) * NC * S::TILE;
  // decomposed tile layout for direction d (0 r, 1 s, 2 t), sign s (0 +, 1 -):
  //   T[(2d + s) * HALF + line * H + pos], line = the two other indices, pos < H
  auto rpos = [&](int jj, int kk) { return (kk * P1 + jj) * H; };  // r: line (j, k), pos along i
  auto spos = [&](int ii, int kk) { return (kk * P1 + ii) * H; };  // s: line (i, k), pos along j
  auto tpos = [&](int ii, int jj) { return (jj * P1 + ii) * H; };  // t: line (i, j), pos along k

  const int* l2g = m.l2g + e * P3;
  double u[NC][8];
  int dmask = 0;
  if (active) {
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int node = eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2);
      const int g = __ldg(l2g + node);
      dmask |= int(g < 0) << c8;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double v;
        if (g >= 0) v = __ldg(a.u + size_t(g) * NC + c);
        else v = a.mask_in ? 0.0 : __ldg(a.u + size_t(-g - 1) * NC + c);
        u[c][c8] = v;
      }
    }
    // decompose the octet's values in all three directions (corner bits: bit0 i, bit1 j, bit2 k)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double* Tc = T + c * S::TILE;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // r: pairs (bit0 = 0, 1) at fixed (bj, bk) = q
        const int bj = q & 1, bk = q >> 1;
        const int jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
        const double a0 = u[c][(bk << 2) | (bj << 1)], a1 = u[c][(bk << 2) | (bj << 1) | 1];
        Tc[0 * HALF + rpos(jj, kk) + i] = a0 + a1;
        Tc[1 * HALF + rpos(jj, kk) + i] = a0 - a1;
        // s: pairs over bit1 at fixed (bi, bk)
        const int bi = q & 1;
        const int ii = bi ? P1 - 1 - i : i;
        const double s0 = u[c][(bk << 2) | bi], s1 = u[c][(bk << 2) | 2 | bi];
        Tc[2 * HALF + spos(ii, kk) + j] = s0 + s1;
        Tc[3 * HALF + spos(ii, kk) + j] = s0 - s1;
        // t: pairs over bit2 at fixed (bi, bj) = (q & 1, q >> 1)
        const int ti = q & 1, tj = q >> 1;
        const int iii = ti ? P1 - 1 - i : i, jjj = tj ? P1 - 1 - j : j;
        const double t0 = u[c][(tj << 1) | ti], t1 = u[c][4 | (tj << 1) | ti];
        Tc[4 * HALF + tpos(iii, jjj) + k] = t0 + t1;
        Tc[5 * HALF + tpos(iii, jjj) + k] = t0 - t1;
      }
    }
  }
  __syncthreads();

  // gradient: 12 pair products per octet -> (u_r, u_s, u_t) at its 8 nodes
  double gr[NC][8], gs[NC][8], gt[NC][8];
  if (active) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double* Tc = T + c * S::TILE;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        {  // r: line (j', k'), output pair (i, p1-1-i)
          const int bj = q & 1, bk = q >> 1;
          const int jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
          const double* xp = Tc + 0 * HALF + rpos(jj, kk);
          const double* xm = Tc + 1 * HALF + rpos(jj, kk);
          double y0, y1;
          eo_pair<H>(sE + i * H, sO + i * H, xp, xm, y0, y1);
          gr[c][(bk << 2) | (bj << 1)] = y0;
          gr[c][(bk << 2) | (bj << 1) | 1] = y1;
        }
        {  // s: line (i', k'), output pair (j, p1-1-j)
          const int bi = q & 1, bk = q >> 1;
          const int ii = bi ? P1 - 1 - i : i, kk = bk ? P1 - 1 - k : k;
          const double* xp = Tc + 2 * HALF + spos(ii, kk);
          const double* xm = Tc + 3 * HALF + spos(ii, kk);
          double y0, y1;
          eo_pair<H>(sE + j * H, sO + j * H, xp, xm, y0, y1);
          gs[c][(bk << 2) | bi] = y0;
          gs[c][(bk << 2) | 2 | bi] = y1;
        }
        {  // t: line (i', j'), output pair (k, p1-1-k)
          const int bi = q & 1, bj = q >> 1;
          const int ii = bi ? P1 - 1 - i : i, jj = bj ? P1 - 1 - j : j;
          const double* xp = Tc + 4 * HALF + tpos(ii, jj);
          const double* xm = Tc + 5 * HALF + tpos(ii, jj);
          double y0, y1;
          eo_pair<H>(sE + k * H, sO + k * H, xp, xm, y0, y1);
          gt[c][(bj << 1) | bi] = y0;
          gt[c][4 | (bj << 1) | bi] = y1;
        }
      }
    }
  }
  __syncthreads();  // every thread is done reading the u tiles

  // geometric factors at the 8 nodes, then decompose (w_r, w_s, w_t) for the transpose
  if (active) {
    const double* G = a.G + e * 6 * P3;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int node = eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2);
      const double g00 = __ldcs(G + 0 * P3 + node), g01 = __ldcs(G + 1 * P3 + node), g02 = __ldcs(G + 2 * P3 + node);
      const double g11 = __ldcs(G + 3 * P3 + node), g12 = __ldcs(G + 4 * P3 + node), g22 = __ldcs(G + 5 * P3 + node);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double ur = gr[c][c8], us = gs[c][c8], ut = gt[c][c8];
        gr[c][c8] = g00 * ur + g01 * us + g02 * ut;
        gs[c][c8] = g01 * ur + g11 * us + g12 * ut;
        gt[c][c8] = g02 * ur + g12 * us + g22 * ut;
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double* Tc = T + c * S::TILE;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bj = q & 1, bk = q >> 1;
        const int jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
        const double a0 = gr[c][(bk << 2) | (bj << 1)], a1 = gr[c][(bk << 2) | (bj << 1) | 1];
        Tc[0 * HALF + rpos(jj, kk) + i] = a0 + a1;
        Tc[1 * HALF + rpos(jj, kk) + i] = a0 - a1;
        const int bi = q & 1;
        const int ii = bi ? P1 - 1 - i : i;
        const double s0 = gs[c][(bk << 2) | bi], s1 = gs[c][(bk << 2) | 2 | bi];
        Tc[2 * HALF + spos(ii, kk) + j] = s0 + s1;
        Tc[3 * HALF + spos(ii, kk) + j] = s0 - s1;
        const int ti = q & 1, tj = q >> 1;
        const int iii = ti ? P1 - 1 - i : i, jjj = tj ? P1 - 1 - j : j;
        const double t0 = gt[c][(tj << 1) | ti], t1 = gt[c][4 | (tj << 1) | ti];
        Tc[4 * HALF + tpos(iii, jjj) + k] = t0 + t1;
        Tc[5 * HALF + tpos(iii, jjj) + k] = t0 - t1;
      }
    }
  }
  __syncthreads();

  // transpose: the three directions' pair products summed at the octet's 8 nodes
  double dot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dot[c] = 0.0;
  if (active) {
    double* wl = a.wl + size_t(e) * P3 * NC;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double* Tc = T + c * S::TILE;
      double w[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bj = q & 1, bk = q >> 1;
        const int jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
        const double* xp = Tc + 0 * HALF + rpos(jj, kk);
        const double* xm = Tc + 1 * HALF + rpos(jj, kk);
        double y0, y1;
        eo_pair<H>(sEt + i * H, sOt + i * H, xp, xm, y0, y1);
        w[(bk << 2) | (bj << 1)] = y0;
        w[(bk << 2) | (bj << 1) | 1] = y1;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bi = q & 1, bk = q >> 1;
        const int ii = bi ? P1 - 1 - i : i, kk = bk ? P1 - 1 - k : k;
        const double* xp = Tc + 2 * HALF + spos(ii, kk);
        const double* xm = Tc + 3 * HALF + spos(ii, kk);
        double y0, y1;
        eo_pair<H>(sEt + j * H, sOt + j * H, xp, xm, y0, y1);
        w[(bk << 2) | bi] += y0;
        w[(bk << 2) | 2 | bi] += y1;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bi = q & 1, bj = q >> 1;
        const int ii = bi ? P1 - 1 - i : i, jj = bj ? P1 - 1 - j : j;
        const double* xp = Tc + 4 * HALF + tpos(ii, jj);
        const double* xm = Tc + 5 * HALF + tpos(ii, jj);
        double y0, y1;
        eo_pair<H>(sEt + k * H, sOt + k * H, xp, xm, y0, y1);
        w[(bj << 1) | bi] += y0;
        w[4 | (bj << 1) | bi] += y1;
      }
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        const int node = eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2);
        if constexpr (HELM) w[c8] += a.beta * __ldg(a.Mq + e * P3 + node) * u[c][c8];  // Eq. (17)
        if (!(a.skip_dirichlet_out && ((dmask >> c8) & 1))) wl[size_t(node) * NC + c] = w[c8];
        dot[c] += w[c8] * u[c][c8];
      }
    }
  }

  if constexpr (BATCH && NC == 1) {  // per-problem alpha from a segmented last-block reduction
    batch_alpha(dot, a.partials, a.prob_blk0, a.prob_nblk, a.bst, prob, red);
    return;
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

template <int P1, int NC, bool HELM, bool BATCH = false>
cudaError_t launch_elem_eo_h(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  const int eb = elem_eo_per_block<P1, NC>();
  const int nthreads = ((eb * EoShape<P1>::H3 + 31) / 32) * 32;
  const size_t smem = elem_eo_smem_bytes<P1, NC>(eb);
  auto kern = elem_eo_kernel<P1, NC, HELM, BATCH>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = BATCH ? int64_t(a.batch_blocks) : (m.nelem + eb - 1) / eb;
  kern<<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

template <int P1, int NC>
cudaError_t launch_elem_eo_t(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  if constexpr (NC == 1) {
    if (a.blk_prob != nullptr) return launch_elem_eo_h<P1, 1, false, true>(m, a, s);
  }
  return a.beta != 0.0 ? launch_elem_eo_h<P1, NC, true>(m, a, s) : launch_elem_eo_h<P1, NC, false>(m, a, s);
}

// whether the kernel can be resident (its registers and threads fit an SM)
template <int P1, int NC>
inline bool elem_eo_launchable() {
  static const bool ok = [] {
    const int eb = elem_eo_per_block<P1, NC>();
    const int nthreads = ((eb * EoShape<P1>::H3 + 31) / 32) * 32;
    const size_t smem = elem_eo_smem_bytes<P1, NC>(eb);
    int nb0 = 0, nb1 = 0;
    if (cudaFuncSetAttribute(elem_eo_kernel<P1, NC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem)) != cudaSuccess ||
        cudaFuncSetAttribute(elem_eo_kernel<P1, NC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem)) != cudaSuccess)
      return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb0, elem_eo_kernel<P1, NC, false>, nthreads, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, elem_eo_kernel<P1, NC, true>, nthreads, smem) !=
            cudaSuccess)
      return false;
    return nb0 >= 1 && nb1 >= 1;
  }();
  return ok;
}

template <int P1, int NC>
inline int elem_eo_blocks_t(int64_t nelem) {
  const int eb = elem_eo_per_block<P1, NC>();
  return int((nelem + eb - 1) / eb);
}

}  // namespace ceedbp
