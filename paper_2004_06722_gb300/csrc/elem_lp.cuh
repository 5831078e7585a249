// Low-precision BK5/BK6 element kernel for the inner solve of FP64 defect
// correction: FP32 arithmetic, with the geometric factors and the input
// direction stored in FP32 or in BF16 (TS).  Same operator and layout as the
// collocated elem_kernel (Eq. (22) with J = I, factors of Eq. (23)); the local
// output w_L is FP32.  The fused (p, A p) of Algorithm 1 is accumulated as an
// FP32 pair per thread (two_prod + dw_add) and reduced in FP64, so the CG
// inner products keep FP64 accuracy while the operator runs in FP32.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "df.cuh"
#include "kernel_args.h"

namespace ceedbp {

__device__ __forceinline__ float lp_load(const float* p) { return __ldg(p); }
// BF16 -> FP32 is exact: the BF16 bits are the top half of the FP32 encoding.
__device__ __forceinline__ float lp_load(const __nv_bfloat16* p) {
  return __uint_as_float(unsigned(__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
}
__device__ __forceinline__ float lp_load_cs(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float lp_load_cs(const __nv_bfloat16* p) {
  return __uint_as_float(unsigned(__ldcs(reinterpret_cast<const unsigned short*>(p))) << 16);
}


template <int P1, int NC>
inline int elem_lp_per_block() {
  int eb = 256 / (P1 * P1 * NC);
  return eb < 1 ? 1 : eb;
}

template <int P1, int NC>
inline size_t elem_lp_smem_bytes(int eb) {
  return sizeof(float) * (size_t(P1) * P1 + size_t(eb) * 3 * NC * P1 * P1 * P1) + sizeof(double) * 32 * NC;
}

template <int P1, int NC, typename TS>
__global__ void elem_lp_kernel(const DeviceMesh m, const ElemLpArgs a, const int eb) {
  constexpr int PP = P1 * P1, P3 = PP * P1;
  extern __shared__ double smem_lp[];
  if (a.state != nullptr && a.state->stop) return;
  double* red = smem_lp;                            // 32 * NC
  float* sD = reinterpret_cast<float*>(red + 32 * NC);  // [P1][P1]
  float* ebuf = sD + PP;
  const int tid = threadIdx.x;
  const int slot = tid / PP, t = tid - slot * PP;
  const int tx = t % P1, ty = t / P1;
  const int64_t e = int64_t(blockIdx.x) * eb + slot;
  const bool active = slot < eb && e < m.nelem;
  for (int i = tid; i < PP; i += blockDim.x) sD[i] = float(m.basis[2 * P1 * P1 + i]);  // Dq of the FP64 tables
  float* sU = ebuf + size_t(active ? slot : 0) * 3 * NC * P3;
  float* sR = sU + NC * P3;
  float* sS = sR + NC * P3;
  const int* l2g = m.l2g + e * P3;
  const TS* u = static_cast<const TS*>(a.u);
  float uq[NC][P1];
  if (active) {
#pragma unroll
    for (int k = 0; k < P1; ++k) {
      const int g = __ldg(l2g + t + PP * k);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float v = g >= 0 ? lp_load(u + size_t(g) * NC + c) : 0.0f;
        uq[c][k] = v;
        sU[c * P3 + k * PP + t] = v;
      }
    }
  }
  __syncthreads();
  float tq[NC][P1];
  if (active) {
    const TS* G = static_cast<const TS*>(a.G) + size_t(e) * 6 * P3;
#pragma unroll
    for (int z = 0; z < P1; ++z) {
      const int pt = z * PP + t;
      const float g00 = lp_load_cs(G + 0 * P3 + pt), g01 = lp_load_cs(G + 1 * P3 + pt), g02 = lp_load_cs(G + 2 * P3 + pt);
      const float g11 = lp_load_cs(G + 3 * P3 + pt), g12 = lp_load_cs(G + 4 * P3 + pt), g22 = lp_load_cs(G + 5 * P3 + pt);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float ur = 0.0f, us = 0.0f, ut = 0.0f;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          ur = fmaf(sD[tx * P1 + n], sU[c * P3 + z * PP + ty * P1 + n], ur);
          us = fmaf(sD[ty * P1 + n], sU[c * P3 + z * PP + n * P1 + tx], us);
          ut = fmaf(sD[z * P1 + n], uq[c][n], ut);
        }
        sR[c * P3 + pt] = g00 * ur + g01 * us + g02 * ut;
        sS[c * P3 + pt] = g01 * ur + g11 * us + g12 * ut;
        tq[c][z] = g02 * ur + g12 * us + g22 * ut;
      }
    }
  }
  __syncthreads();
  dfloat dacc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dacc[c] = dfloat{0.0f, 0.0f};
  if (active) {
    float* wl = a.wl + size_t(e) * P3 * NC;
#pragma unroll
    for (int z = 0; z < P1; ++z) {
      const int idx = z * PP + t;
      const bool skip = __ldg(l2g + idx) < 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float v = 0.0f;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          v = fmaf(sD[n * P1 + tx], sR[c * P3 + z * PP + ty * P1 + n], v);
          v = fmaf(sD[n * P1 + ty], sS[c * P3 + z * PP + n * P1 + tx], v);
          v = fmaf(sD[n * P1 + z], tq[c][n], v);
        }
        if (!skip) wl[size_t(idx) * NC + c] = v;
        const float ph = __fmul_rn(v, uq[c][z]);
        dacc[c] = dw_add(dacc[c], dfloat{ph, __fmaf_rn(v, uq[c][z], -ph)});
      }
    }
  }
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

template <int P1, int NC, typename TS>
cudaError_t launch_elem_lp_t(const DeviceMesh& m, const ElemLpArgs& a, cudaStream_t s) {
  const int eb = elem_lp_per_block<P1, NC>();
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  const size_t smem = elem_lp_smem_bytes<P1, NC>(eb);
  auto kern = elem_lp_kernel<P1, NC, TS>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + eb - 1) / eb;
  kern<<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

template <int P1, int NC>
inline int elem_lp_blocks_t(int64_t nelem) {
  const int eb = elem_lp_per_block<P1, NC>();
  return int((nelem + eb - 1) / eb);
}

}  // namespace ceedbp
