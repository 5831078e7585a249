// Software-pipelined FP32 BK5/BK6 element kernel for the inner solve of
// defect correction (FP32 storage of G and the direction p).
//
// Same operator and arithmetic as elem_lp_kernel with TS = float (Eq. (22)
// with J = I and the factors of Eq. (23), FMAs in FP32, the fused (p, A p) of
// Algorithm 1 accumulated as an FP32 pair), scheduled like the pipelined pair
// kernel (elem_dfp.cuh): each group of p1*p1 threads (a slot) works through a
// sequence of `ns` elements; the next element's l2g column is loaded into
// registers at the top of the current element, its p column is copied into
// the p tile by cp.async after the current element's gradient phase, and G
// streams through a three-slab ring two slabs ahead across element
// boundaries.  Each thread copies only its own column, so the only barriers
// are the two the contraction needs.  Slab loops stay rolled; the t components
// go through a private tile.
#pragma once

#include "elem_lp.cuh"

namespace ceedbp {

template <int P1, int NC>
struct ElemLppShape {
  static constexpr int PP = P1 * P1, P3 = PP * P1;
  static constexpr int ROW = P1 + 1, SLAB = P1 * ROW, TILE = P1 * SLAB;
  static constexpr int RING = 3 * 6 * PP;  // floats
};

// layout: [red 32 NC doubles][sD p1 x p1 floats] then per slot:
//         [G ring][sU NC tiles][sR NC tiles][sS NC tiles][sT NC x p1^3]  (floats)
template <int P1, int NC>
__host__ __device__ inline size_t elem_lpp_head_bytes() {
  const size_t h = sizeof(double) * 32 * NC + sizeof(float) * P1 * P1;
  return (h + 15) / 16 * 16;
}

template <int P1, int NC>
__host__ __device__ inline size_t elem_lpp_slot_bytes() {
  using S = ElemLppShape<P1, NC>;
  const size_t b = sizeof(float) * (size_t(S::RING) + 3 * NC * size_t(S::TILE) + size_t(NC) * S::P3);
  return (b + 15) / 16 * 16;
}

template <int P1, int NC>
inline size_t elem_lpp_smem_bytes(int eb) {
  return elem_lpp_head_bytes<P1, NC>() + size_t(eb) * elem_lpp_slot_bytes<P1, NC>();
}

template <int P1, int NC>
__global__ void __launch_bounds__(256) elem_lpp_kernel(const DeviceMesh m, const ElemLpArgs a, const int eb,
                                                       const int ns) {
  using S = ElemLppShape<P1, NC>;
  constexpr int PP = S::PP, P3 = S::P3, ROW = S::ROW, SLAB = S::SLAB, TILE = S::TILE;
  extern __shared__ __align__(16) unsigned char smem_lpp[];
  if (a.state != nullptr && a.state->stop) return;

  double* red = reinterpret_cast<double*>(smem_lpp);        // 32 * NC
  float* sD = reinterpret_cast<float*>(red + 32 * NC);     // [P1][P1]
  const int tid = threadIdx.x;
  const int slot = tid / PP, t = tid - slot * PP;
  const int i = t % P1, j = t / P1;
  const bool in_slot = slot < eb;
  float* ring = reinterpret_cast<float*>(smem_lpp + elem_lpp_head_bytes<P1, NC>() +
                                         size_t(in_slot ? slot : 0) * elem_lpp_slot_bytes<P1, NC>());
  float* sU = ring + S::RING;
  float* sR = sU + NC * TILE;
  float* sS = sR + NC * TILE;
  float* sT = sS + NC * TILE;  // [NC][P3] private columns
  const int my = j * ROW + i;
  const float* u = static_cast<const float*>(a.u);
  const float* Gp = static_cast<const float*>(a.G);

  for (int q = tid; q < PP; q += blockDim.x) sD[q] = float(m.basis[2 * PP + q]);  // Dq of the FP64 tables
  __syncthreads();

  const int64_t first = int64_t(blockIdx.x) * eb * ns;
  auto elem_of = [&](int s) -> int64_t { return first + int64_t(s) * eb + slot; };
  auto live = [&](int s) -> bool { return in_slot && s < ns && elem_of(s) < m.nelem; };
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
  auto fetch_u = [&](const int (&lg)[P1]) {
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int g = lg[k];
      const int64_t gg = g < 0 ? -int64_t(g) - 1 : int64_t(g);
#pragma unroll
      for (int c = 0; c < NC; ++c) cp_async4(sU + c * TILE + k * SLAB + my, u + gg * NC + c);
    }
  };
  auto fetch_g = [&](int s, int sl, int rp) {
    const float* src = Gp + elem_of(s) * 6 * P3 + sl * PP + t;
#pragma unroll
    for (int q = 0; q < 6; ++q) cp_async4(ring + rp * 6 * PP + q * PP + t, src + q * P3);
  };

  unsigned dmask = 0u;
  if (live(0)) {
    int lg[P1];
    load_l2g(0, lg);
    dmask = dir_mask(lg);
    fetch_u(lg);
    fetch_g(0, 0, 0);
    if (P1 > 1) fetch_g(0, 1, 1);
  }
  cp_async_commit();

  dfloat dacc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dacc[c] = dfloat{0.0f, 0.0f};
  int rp = 0;

  for (int s = 0; s < ns; ++s) {
    const bool active = live(s);
    cp_async_wait_all();
    int lg_next[P1];
    const bool next_live = live(s + 1);
    if (next_live) load_l2g(s + 1, lg_next);

    // own column of p (zero on Dirichlet nodes: p is masked) to registers and the tile
    float xc[NC][P1];
    if (active) {
#pragma unroll
      for (int k = 0; k < P1; ++k) {
        const bool dir = (dmask >> k) & 1u;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float* cell = sU + c * TILE + k * SLAB + my;
          const float v = dir ? 0.0f : *cell;
          *cell = v;
          xc[c][k] = v;
        }
      }
    }
    __syncthreads();

    // gradient and geometric factors (rolled slab loop)
    {
      float Di[P1], Dj[P1];
#pragma unroll
      for (int n = 0; n < P1; ++n) {
        Di[n] = sD[i * P1 + n];
        Dj[n] = sD[j * P1 + n];
      }
#pragma unroll 1
      for (int k = 0; k < P1; ++k) {
        const int rp2 = rp + 2 >= 3 ? rp - 1 : rp + 2;
        if (k + 2 < P1) {
          if (active) fetch_g(s, k + 2, rp2);
        } else if (next_live) {
          fetch_g(s + 1, k + 2 - P1, rp2);
        }
        cp_async_commit();
        cp_async_wait<2>();
        const float* gs = ring + rp * 6 * PP + t;
        rp = rp + 1 == 3 ? 0 : rp + 1;
        if (!active) continue;
        const float g00 = gs[0], g01 = gs[PP], g02 = gs[2 * PP], g11 = gs[3 * PP], g12 = gs[4 * PP],
                    g22 = gs[5 * PP];
        const float* dk = sD + k * P1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float* xs = sU + c * TILE + k * SLAB;
          float ur = 0.0f, us = 0.0f, ut = 0.0f;
#pragma unroll
          for (int n = 0; n < P1; ++n) {
            ur = fmaf(Di[n], xs[j * ROW + n], ur);
            us = fmaf(Dj[n], xs[n * ROW + i], us);
            ut = fmaf(dk[n], xc[c][n], ut);
          }
          sR[c * TILE + k * SLAB + my] = g00 * ur + g01 * us + g02 * ut;
          sS[c * TILE + k * SLAB + my] = g01 * ur + g11 * us + g12 * ut;
          sT[c * P3 + k * PP + t] = g02 * ur + g12 * us + g22 * ut;
        }
      }
    }
    __syncthreads();
    if (next_live) fetch_u(lg_next);
    cp_async_commit();
    const unsigned dmask_next = next_live ? dir_mask(lg_next) : 0u;

    // transpose, output, fused dot (x_k from the front of the shifted column)
    if (active) {
      float Dni[P1], Dnj[P1];
#pragma unroll
      for (int n = 0; n < P1; ++n) {
        Dni[n] = sD[n * P1 + i];
        Dnj[n] = sD[n * P1 + j];
      }
      float* wl = a.wl + size_t(elem_of(s)) * P3 * NC;
#pragma unroll 1
      for (int k = 0; k < P1; ++k) {
        const int idx = k * PP + t;
        const bool skip = (dmask >> k) & 1u;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float* rs = sR + c * TILE + k * SLAB;
          const float* ss = sS + c * TILE + k * SLAB;
          const float* ts = sT + c * P3 + t;
          float v = 0.0f;
#pragma unroll
          for (int n = 0; n < P1; ++n) {
            v = fmaf(Dni[n], rs[j * ROW + n], v);
            v = fmaf(Dnj[n], ss[n * ROW + i], v);
            v = fmaf(sD[n * P1 + k], ts[n * PP], v);
          }
          if (!skip) wl[size_t(idx) * NC + c] = v;
          const float ph = __fmul_rn(v, xc[c][0]);
          dacc[c] = dw_add(dacc[c], dfloat{ph, __fmaf_rn(v, xc[c][0], -ph)});
#pragma unroll
          for (int n = 0; n + 1 < P1; ++n) xc[c][n] = xc[c][n + 1];
        }
      }
    }
    dmask = dmask_next;
  }
  cp_async_wait_all();

  if (a.partials != nullptr) {
    double dot[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) dot[c] = df_to_f64(dacc[c]);
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

// The shape: two slots per block (one where two do not fit), sequences of 8 elements.
template <int P1, int NC>
struct ElemLppPlan {
  int eb = 0;  // 0: not launchable, use elem_lp_kernel
  int ns = 8;
};

template <int P1, int NC>
inline ElemLppPlan<P1, NC> elem_lpp_plan() {
  static const ElemLppPlan<P1, NC> plan = [] {
    ElemLppPlan<P1, NC> p;
    if (cudaFuncSetAttribute(elem_lpp_kernel<P1, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) !=
        cudaSuccess)
      return p;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, elem_lpp_kernel<P1, NC>) != cudaSuccess) return p;
    for (int eb = 2; eb >= 1; --eb) {
      const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
      const size_t smem = elem_lpp_smem_bytes<P1, NC>(eb);
      int nb = 0;
      if (nthreads > fa.maxThreadsPerBlock || smem > 220 * 1024) continue;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, elem_lpp_kernel<P1, NC>, nthreads, smem) !=
              cudaSuccess ||
          nb < 1)
        continue;
      p.eb = eb;
      break;
    }
    return p;
  }();
  return plan;
}

template <int P1, int NC>
cudaError_t launch_elem_lpp_t(const DeviceMesh& m, const ElemLpArgs& a, cudaStream_t s) {
  const ElemLppPlan<P1, NC> p = elem_lpp_plan<P1, NC>();
  if (p.eb == 0) return launch_elem_lp_t<P1, NC, float>(m, a, s);
  const int nthreads = ((p.eb * P1 * P1 + 31) / 32) * 32;
  const size_t smem = elem_lpp_smem_bytes<P1, NC>(p.eb);
  const int64_t per_block = int64_t(p.eb) * p.ns;
  const int64_t blocks = (m.nelem + per_block - 1) / per_block;
  elem_lpp_kernel<P1, NC><<<unsigned(blocks), nthreads, smem, s>>>(m, a, p.eb, p.ns);
  return cudaGetLastError();
}

}  // namespace ceedbp
