// FP64 BK1/BK3 element kernel (Gauss quadrature, q = N + 2 > p1) with every
// 1D contraction in even-odd form (Eq. (37)).
//
// The interpolation J (q x p1) from the GLL nodes to the GL points is
// centro-symmetric and the GL derivative matrix Dq (q x q) centro-
// antisymmetric, so each 1D product of a line costs about half the multiply-
// adds when one thread computes all outputs of that line from the line's
// even and odd halves.  Each stage therefore maps one thread to one line:
//
//   x:  u (p1^3)        -> X (q p1^2)  lines (j, k),    J along i
//   y:  X               -> Y (q^2 p1)  lines (qx, k),   J along j
//   z:  Y               -> u at the q^3 points, column (qx, qy) in registers
//   BK3: u_r, u_s along lines (qy, z) and (qx, z), u_t in the column; the
//        factors G of Eq. (23) per column; the transposes Dq^T in place on
//        the same lines; the three parts summed per column
//   BK1: the mass factors of Eq. (34) per column
//   z^T, y^T, x^T: J^T on the same line families back to the nodes.
//
// The interpolate-then-differentiate form of Eqs. (31)-(33) is kept (the
// cheaper of the paper's two forms at q = p1 + 1), with the same operator,
// layout, masking and fused (u, w) dot as elem_kernel, which this kernel
// replaces for one component.  Tiles live in shared memory; a q x q group of
// threads holds one element, several elements share a block.
#pragma once

#include "elem.cuh"

namespace ceedbp {

template <int P1, int Q>
struct GlShape {
  static constexpr int QQ = Q * Q, Q3 = QQ * Q, P3 = P1 * P1 * P1;
  static constexpr int SLOT = P3 + 3 * Q3;  // doubles per element: u, then three q^3 work tiles
};

template <int P1, int Q>
__host__ __device__ constexpr int elem_gl_per_block() {
  return 256 / (Q * Q) < 1 ? 1 : 256 / (Q * Q);
}

template <int P1, int Q>
__host__ __device__ constexpr int elem_gl_threads() {
  return ((elem_gl_per_block<P1, Q>() * Q * Q + 31) / 32) * 32;
}

template <int P1, int Q>
inline size_t elem_gl_smem_bytes() {
  return sizeof(double) * (32 + elem_eo_tab_doubles<P1, Q>() +
                           size_t(elem_gl_per_block<P1, Q>()) * GlShape<P1, Q>::SLOT);
}

template <int P1, int Q, int KIND, bool HELM>
__global__ void __launch_bounds__(elem_gl_threads<P1, Q>()) elem_gl_kernel(const DeviceMesh m, const ElemArgs a) {
  using S = GlShape<P1, Q>;
  constexpr int QQ = S::QQ, Q3 = S::Q3, P3 = S::P3;
  constexpr int EB = elem_gl_per_block<P1, Q>();
  extern __shared__ double smem_gl[];
  if (a.state != nullptr && a.state->stop) return;
  double* red = smem_gl;       // 32
  double* tJ = red + 32;       // even-odd tables of J, J^T, Dq, Dq^T
  double* tJT = tJ + EoTab<Q, P1>::SIZE;
  double* tD = tJT + EoTab<P1, Q>::SIZE;
  double* tDT = tD + EoTab<Q, Q>::SIZE;
  double* ebuf = tDT + EoTab<Q, Q>::SIZE;

  const int tid = threadIdx.x;
  const int slot = tid / QQ, t = tid - slot * QQ;
  const int64_t e0 = int64_t(blockIdx.x) * EB;
  const int nact = m.nelem - e0 < EB ? int(m.nelem - e0) : EB;
  const int64_t e = e0 + slot;
  const bool active = slot < nact;

  eo_build<Q, P1, false>(m.basis, P1, tJ, tid, blockDim.x);
  eo_build<P1, Q, true>(m.basis, P1, tJT, tid, blockDim.x);
  eo_build<Q, Q, false>(m.basis + 2 * Q * P1, Q, tD, tid, blockDim.x);
  eo_build<Q, Q, true>(m.basis + 2 * Q * P1, Q, tDT, tid, blockDim.x);

  double* sU = ebuf + size_t(active ? slot : 0) * S::SLOT;  // [P3] nodes, i fastest
  double* sA = sU + P3;                                     // X, then u_r / w_r, then the y^T output
  double* sB = sA + Q3;                                     // Y, then u_s / w_s, then the nodal result
  double* sC = sB + Q3;                                     // u at the points, then the z^T output
  const int* l2g = m.l2g + e * P3;

  // ---- gather u^e = Q u (Eq. (21)); Dirichlet nodes read as 0 when masking
  if (active) {
    for (int idx = t; idx < P3; idx += QQ) {
      const int g = __ldg(l2g + idx);
      double v;
      if (g >= 0) v = __ldg(a.u + g);
      else v = a.mask_in ? 0.0 : __ldg(a.u + (-g - 1));
      sU[idx] = v;
    }
  }
  __syncthreads();
  // ---- x: X[qx + Q (j + P1 k)] = sum_i J[qx][i] u[i + P1 (j + P1 k)], line (j, k) = t
  if (active && t < P1 * P1) {
    double x[P1], y[Q];
#pragma unroll
    for (int i = 0; i < P1; ++i) x[i] = sU[t * P1 + i];
    eo_mul<Q, P1, 1>(tJ, x, y);
#pragma unroll
    for (int q = 0; q < Q; ++q) sA[t * Q + q] = y[q];
  }
  __syncthreads();
  // ---- y: Y[qx + Q (qy + Q k)] = sum_j J[qy][j] X[qx + Q (j + P1 k)], line (qx, k): qx = t % Q, k = t / Q
  if (active && t < Q * P1) {
    const int qx = t % Q, k = t / Q;
    double x[P1], y[Q];
#pragma unroll
    for (int j = 0; j < P1; ++j) x[j] = sA[qx + Q * (j + P1 * k)];
    eo_mul<Q, P1, 1>(tJ, x, y);
#pragma unroll
    for (int q = 0; q < Q; ++q) sB[qx + Q * (q + Q * k)] = y[q];
  }
  __syncthreads();
  // ---- z: the column (qx, qy) = t of u at the points, kept in registers and in sC
  double uq[Q];
  if (active) {
    double x[P1];
#pragma unroll
    for (int k = 0; k < P1; ++k) x[k] = sB[t + QQ * k];
    eo_mul<Q, P1, 1>(tJ, x, uq);
    if constexpr (KIND == kStiff) {
#pragma unroll
      for (int z = 0; z < Q; ++z) sC[t + QQ * z] = uq[z];
    }
  }

  double vq[Q];
  if constexpr (KIND == kMass) {
    if (active) {
      const double* M = a.G + e * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) vq[z] = __ldcs(M + t + QQ * z) * uq[z];
    }
  } else {
    __syncthreads();
    // ---- u_r along lines (qy, z) and u_s along lines (qx, z): both line families are indexed by t
    if (active) {
      const int lo = t % Q, hi = t / Q;
      double x[Q], y[Q];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sC[n + Q * lo + QQ * hi];  // r: qy = lo, z = hi
      eo_mul<Q, Q, -1>(tD, x, y);
#pragma unroll
      for (int n = 0; n < Q; ++n) sA[n + Q * lo + QQ * hi] = y[n];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sC[lo + Q * n + QQ * hi];  // s: qx = lo, z = hi
      eo_mul<Q, Q, -1>(tD, x, y);
#pragma unroll
      for (int n = 0; n < Q; ++n) sB[lo + Q * n + QQ * hi] = y[n];
    }
    __syncthreads();
    // ---- u_t in the column, then G grad u per point (Eq. (23)); w_r, w_s in place, w_t in registers
    double wt[Q];
    if (active) {
      double ut[Q];
      eo_mul<Q, Q, -1>(tD, uq, ut);
      const double* G = a.G + e * 6 * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const int pt = t + QQ * z;
        const double g00 = __ldcs(G + 0 * Q3 + pt), g01 = __ldcs(G + 1 * Q3 + pt), g02 = __ldcs(G + 2 * Q3 + pt);
        const double g11 = __ldcs(G + 3 * Q3 + pt), g12 = __ldcs(G + 4 * Q3 + pt), g22 = __ldcs(G + 5 * Q3 + pt);
        const double ur = sA[pt], us = sB[pt];
        sA[pt] = g00 * ur + g01 * us + g02 * ut[z];
        sB[pt] = g01 * ur + g11 * us + g12 * ut[z];
        wt[z] = g02 * ur + g12 * us + g22 * ut[z];
      }
    }
    __syncthreads();
    // ---- transposes Dq^T: r and s on their lines, in place (each line belongs to one thread)
    if (active) {
      const int lo = t % Q, hi = t / Q;
      double x[Q], y[Q];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sA[n + Q * lo + QQ * hi];
      eo_mul<Q, Q, -1>(tDT, x, y);
#pragma unroll
      for (int n = 0; n < Q; ++n) sA[n + Q * lo + QQ * hi] = y[n];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sB[lo + Q * n + QQ * hi];
      eo_mul<Q, Q, -1>(tDT, x, y);
#pragma unroll
      for (int n = 0; n < Q; ++n) sB[lo + Q * n + QQ * hi] = y[n];
      eo_mul<Q, Q, -1>(tDT, wt, vq);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int z = 0; z < Q; ++z) vq[z] += sA[t + QQ * z] + sB[t + QQ * z];
      if constexpr (HELM) {  // + beta B u at the quadrature points (Eq. (17))
        const double* M = a.Mq + e * Q3;
#pragma unroll
        for (int z = 0; z < Q; ++z) vq[z] += a.beta * __ldg(M + t + QQ * z) * uq[z];
      }
    }
  }
  __syncthreads();  // every read of sA, sB, sC above is done
  // ---- z^T: T2[t + QQ k] = sum_z J[z][k] v(t, z), into sC
  if (active) {
    double wk[P1];
    eo_mul<P1, Q, 1>(tJT, vq, wk);
#pragma unroll
    for (int k = 0; k < P1; ++k) sC[t + QQ * k] = wk[k];
  }
  __syncthreads();
  // ---- y^T: T1[qx + Q (j + P1 k)] = sum_qy J[qy][j] T2[qx + Q (qy + Q k)], line (qx, k), into sA
  if (active && t < Q * P1) {
    const int qx = t % Q, k = t / Q;
    double x[Q], y[P1];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = sC[qx + Q * (q + Q * k)];
    eo_mul<P1, Q, 1>(tJT, x, y);
#pragma unroll
    for (int j = 0; j < P1; ++j) sA[qx + Q * (j + P1 * k)] = y[j];
  }
  __syncthreads();
  // ---- x^T: w[i + P1 (j + P1 k)] = sum_qx J[qx][i] T1[qx + Q (j + P1 k)], line (j, k), into sB
  if (active && t < P1 * P1) {
    double x[Q], y[P1];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = sA[q + Q * t];
    eo_mul<P1, Q, 1>(tJT, x, y);
#pragma unroll
    for (int i = 0; i < P1; ++i) sB[t * P1 + i] = y[i];
  }
  __syncthreads();
  // ---- w^e to the local output (coalesced), (u^e, w^e)
  double dot[1] = {0.0};
  if (active) {
    double* wl = a.wl + size_t(e) * P3;
    for (int idx = t; idx < P3; idx += QQ) {
      const double w = sB[idx];
      if (!(a.skip_dirichlet_out && __ldg(l2g + idx) < 0)) wl[idx] = w;
      dot[0] += w * sU[idx];
    }
  }

  if (a.partials != nullptr) {
    if (grid_sum_last<1>(dot, a.partials, gridDim.x, blockIdx.x, &a.state->ticket[kTicketApply], red)) {
      if (threadIdx.x == 0) {
        SolveState* st = a.state;
        CompScalars& cs = st->c[0];
        if (cs.active) {
          const double pAp = dot[0];
          cs.pAp = pAp;
          if (!(pAp > 0.0) || !isfinite(pAp) || !isfinite(cs.rz)) {
            cs.status = CEEDBP_EBREAKDOWN;
            cs.alpha = 0.0;
            if (!st->fixed) cs.active = 0;
          } else {
            cs.alpha = cs.rz / pAp;
          }
        }
        if (!cs.active) st->stop = 1;
      }
    }
  }
}

template <int P1, int Q, int KIND, bool HELM>
cudaError_t launch_elem_gl_h(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  constexpr int EB = elem_gl_per_block<P1, Q>();
  const size_t smem = elem_gl_smem_bytes<P1, Q>();
  auto kern = elem_gl_kernel<P1, Q, KIND, HELM>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + EB - 1) / EB;
  kern<<<unsigned(blocks), elem_gl_threads<P1, Q>(), smem, s>>>(m, a);
  return cudaGetLastError();
}

template <int P1, int Q, int KIND>
cudaError_t launch_elem_gl_t(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  if constexpr (KIND == kStiff) {
    if (a.beta != 0.0) return launch_elem_gl_h<P1, Q, KIND, true>(m, a, s);
  }
  return launch_elem_gl_h<P1, Q, KIND, false>(m, a, s);
}

template <int P1, int Q>
constexpr int elem_gl_blocks_t(int64_t nelem) {
  return int((nelem + elem_gl_per_block<P1, Q>() - 1) / elem_gl_per_block<P1, Q>());
}

}  // namespace ceedbp
