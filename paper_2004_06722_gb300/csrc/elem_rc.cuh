// BK5/BK6 element kernel that recomputes the geometric factors from the nodal
// coordinates instead of reading them (the bytes-for-flops variant of the
// stored-factor kernels).
//
// With GLL collocation the Jacobian at node (i, j, k) is the derivative of the
// iso-parametric map of Eq. (18) taken with the same 1D matrix D as the
// operator: dx_d/dr_m = (D_m x_d)(i, j, k), nine contractions of length p1.
// From it, Eq. (23): G = rho_i rho_j rho_k adj(J) adj(J)^T / |J| (adj(J) =
// |J| J^{-1}), six symmetric components, and then the operator of Eq. (22)
// exactly as in elem_kernel.  The element reads 3 coordinates per node
// (stored [E][3][p1^3]) instead of 6 factors: 24 fewer bytes per node for
// about 9 p1 + 40 more FMAs per node.
//
// Layout: one element per p1*p1 thread group; thread (i, j) owns the column
// of nodes (i, j, 0..p1-1).  Shared memory per element: the coordinate tile,
// the u tile and two gradient tiles.
#pragma once

#include "common.cuh"

namespace ceedbp {

template <int P1, int NC>
inline int elem_rc_per_block() {
  int eb = 256 / (P1 * P1 * NC);
  return eb < 1 ? 1 : eb;
}

template <int P1, int NC>
inline size_t elem_rc_smem_bytes(int eb) {
  constexpr size_t P3 = size_t(P1) * P1 * P1;
  return sizeof(double) * (size_t(P1) * P1 + P1 + size_t(eb) * (3 + 3 * NC) * P3 + 32 * NC);
}

template <int P1, int NC>
__global__ void elem_rc_kernel(const DeviceMesh m, const ElemArgs a, const int eb) {
  constexpr int PP = P1 * P1, P3 = PP * P1;
  extern __shared__ double smem[];
  if (a.state != nullptr && a.state->stop) return;

  double* sD = smem;           // [P1][P1] GLL derivative matrix
  double* sw = sD + PP;        // [P1] GLL weights
  double* red = sw + P1;       // 32 * NC reduction scratch
  double* ebuf = red + 32 * NC;

  const int tid = threadIdx.x;
  const int slot = tid / PP, t = tid - slot * PP;
  const int tx = t % P1, ty = t / P1;
  const int64_t e = int64_t(blockIdx.x) * eb + slot;
  const bool active = slot < eb && e < m.nelem;

  // basis layout: [J q x p1][Dh q x p1][Dq q x q][w q] with q = p1 (collocated)
  for (int i = tid; i < PP; i += blockDim.x) sD[i] = m.basis[2 * PP + i];
  for (int i = tid; i < P1; i += blockDim.x) sw[i] = m.basis[3 * PP + i];

  double* sX = ebuf + size_t(active ? slot : 0) * (3 + 3 * NC) * P3;  // [3][P3] coordinates
  double* sU = sX + 3 * P3;                                           // [NC][P3]
  double* sR = sU + NC * P3;
  double* sS = sR + NC * P3;

  const int* l2g = m.l2g + e * P3;
  if (active) {
    const double* X = m.X + e * 3 * P3;
    for (int idx = t; idx < 3 * P3; idx += PP) sX[idx] = __ldcs(X + idx);
    for (int idx = t; idx < P3; idx += PP) {
      const int g = __ldg(l2g + idx);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double v;
        if (g >= 0) v = __ldg(a.u + size_t(g) * NC + c);
        else v = a.mask_in ? 0.0 : __ldg(a.u + size_t(-g - 1) * NC + c);
        sU[c * P3 + idx] = v;
      }
    }
  }
  __syncthreads();

  double uq[NC][P1];
  double tq[NC][P1];
  if (active) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int z = 0; z < P1; ++z) uq[c][z] = sU[c * P3 + z * PP + t];
    const double wxy = sw[tx] * sw[ty];
#pragma unroll
    for (int z = 0; z < P1; ++z) {
      const int pt = z * PP + t;
      // Jacobian A[d][mm] = dx_d / dr_mm at node (tx, ty, z)
      double A[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double* xd = sX + d * P3;
        double jr = 0.0, js = 0.0, jt = 0.0;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          jr += sD[tx * P1 + n] * xd[z * PP + ty * P1 + n];
          js += sD[ty * P1 + n] * xd[z * PP + n * P1 + tx];
          jt += sD[z * P1 + n] * xd[n * PP + t];
        }
        A[d][0] = jr;
        A[d][1] = js;
        A[d][2] = jt;
      }
      // adj[mm][d] = |J| dr_mm / dx_d
      double adj[3][3];
      adj[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
      adj[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
      adj[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
      adj[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
      adj[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
      adj[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
      adj[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
      adj[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
      adj[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      const double det = A[0][0] * adj[0][0] + A[0][1] * adj[1][0] + A[0][2] * adj[2][0];
      const double sc = wxy * sw[z] / det;
      const double g00 = sc * (adj[0][0] * adj[0][0] + adj[0][1] * adj[0][1] + adj[0][2] * adj[0][2]);
      const double g01 = sc * (adj[0][0] * adj[1][0] + adj[0][1] * adj[1][1] + adj[0][2] * adj[1][2]);
      const double g02 = sc * (adj[0][0] * adj[2][0] + adj[0][1] * adj[2][1] + adj[0][2] * adj[2][2]);
      const double g11 = sc * (adj[1][0] * adj[1][0] + adj[1][1] * adj[1][1] + adj[1][2] * adj[1][2]);
      const double g12 = sc * (adj[1][0] * adj[2][0] + adj[1][1] * adj[2][1] + adj[1][2] * adj[2][2]);
      const double g22 = sc * (adj[2][0] * adj[2][0] + adj[2][1] * adj[2][1] + adj[2][2] * adj[2][2]);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          ur += sD[tx * P1 + n] * sU[c * P3 + z * PP + ty * P1 + n];
          us += sD[ty * P1 + n] * sU[c * P3 + z * PP + n * P1 + tx];
          ut += sD[z * P1 + n] * uq[c][n];
        }
        sR[c * P3 + pt] = g00 * ur + g01 * us + g02 * ut;
        sS[c * P3 + pt] = g01 * ur + g11 * us + g12 * ut;
        tq[c][z] = g02 * ur + g12 * us + g22 * ut;
      }
    }
  }
  __syncthreads();

  double dot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dot[c] = 0.0;
  if (active) {
    double* wl = a.wl + size_t(e) * P3 * NC;
#pragma unroll
    for (int z = 0; z < P1; ++z) {
      const int idx = z * PP + t;
      const bool skip = a.skip_dirichlet_out && __ldg(l2g + idx) < 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double v = 0.0;
#pragma unroll
        for (int n = 0; n < P1; ++n) {
          v += sD[n * P1 + tx] * sR[c * P3 + z * PP + ty * P1 + n];
          v += sD[n * P1 + ty] * sS[c * P3 + z * PP + n * P1 + tx];
          v += sD[n * P1 + z] * tq[c][n];
        }
        if (a.beta != 0.0) v += a.beta * __ldg(a.Mq + e * P3 + idx) * uq[c][z];  // Eq. (17)
        if (!skip) wl[size_t(idx) * NC + c] = v;
        dot[c] += v * uq[c][z];
      }
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
cudaError_t launch_elem_rc_t(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  const int eb = elem_rc_per_block<P1, NC>();
  const int nthreads = ((eb * P1 * P1 + 31) / 32) * 32;
  const size_t smem = elem_rc_smem_bytes<P1, NC>(eb);
  auto kern = elem_rc_kernel<P1, NC>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + eb - 1) / eb;
  kern<<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

template <int P1, int NC>
inline int elem_rc_blocks_t(int64_t nelem) {
  const int eb = elem_rc_per_block<P1, NC>();
  return int((nelem + eb - 1) / eb);
}

}  // namespace ceedbp
