// Element operator kernels (BK1, BK3, BK5, BK6): w^e = A^e u^e or B^e u^e for
// every element, the unassembled product A_L Q u of Eq. (21).
//
// Stiffness, Eq. (22): w^e = sum_{m,m'} D_m^T G_mm' D_m' u^e with the
// geometric factors G of Eq. (23) (six symmetric components per quadrature
// point, stored [E][6][q^3]).  Mass, Eq. (34): w^e = J^T Btilde J u^e with one
// factor rho_i rho_j rho_k |J| per quadrature point.
//
// The gradient is taken in the interpolate-then-differentiate form of
// Eqs. (31)-(33): u is interpolated to the q^3 points with J (x, y, z
// contractions), differentiated there with the q x q matrix Dq, multiplied by G,
// and carried back with Dq^T and J^T.  With GLL quadrature (BP5/BP6) J is the
// identity and the interpolation stages are compiled out (Eq. (22) with
// J = I, 12 p1^4 + 15 p1^3 flops per element).
//
// Layout: one element per q*q thread group, thread (qx, qy) owns the column of
// points (qx, qy, 0..q-1); the element's q^3 tiles live in shared memory; the
// t-direction column stays in registers.  Several elements share a block when
// q*q is small.  The per-block dot (Q u, w^e) needed by CG is reduced in a
// fixed order (no float atomics); the last block turns it into alpha = rz / pAp.
#pragma once

#include "common.cuh"

namespace ceedbp {

template <int P1, int Q, bool COLLOC>
struct ElemShape {
  static constexpr int QQ = Q * Q;
  static constexpr int Q3 = Q * Q * Q;
  static constexpr int P3 = P1 * P1 * P1;
  static constexpr int NBUF = COLLOC ? 3 : 4;
};

template <int P1, int Q, bool COLLOC, int NC>
inline int elem_per_block() {
  constexpr int QQ = Q * Q;
  int eb = 256 / (QQ * NC);
  return eb < 1 ? 1 : eb;
}

template <int P1, int Q, bool COLLOC, int NC>
inline size_t elem_smem_bytes(int eb) {
  using S = ElemShape<P1, Q, COLLOC>;
  return sizeof(double) * (size_t(Q) * P1 + size_t(Q) * Q + size_t(eb) * S::NBUF * NC * S::Q3 + 32 * NC);
}

// Threads of one block (whole warps); the launch bound below lets the compiler
// size registers for exactly this block.
template <int Q, int NC>
constexpr int elem_threads() {
  return (((256 / (Q * Q * NC) < 1 ? 1 : 256 / (Q * Q * NC)) * Q * Q + 31) / 32) * 32;
}

template <int P1, int Q, bool COLLOC, int KIND, int NC>
__global__ void __launch_bounds__(elem_threads<Q, NC>()) elem_kernel(const DeviceMesh m, const ElemArgs a,
                                                                     const int eb) {
  using S = ElemShape<P1, Q, COLLOC>;
  constexpr int QQ = S::QQ, Q3 = S::Q3, P3 = S::P3;
  extern __shared__ double smem[];
  if (a.state != nullptr && a.state->stop) return;

  double* sJ = smem;            // [Q][P1]
  double* sD = sJ + Q * P1;     // [Q][Q]
  double* red = sD + Q * Q;     // 32 * NC reduction scratch
  double* ebuf = red + 32 * NC;

  const int tid = threadIdx.x;
  const int slot = tid / QQ, t = tid - (tid / QQ) * QQ;
  const int tx = t % Q, ty = t / Q;
  const int64_t e = int64_t(blockIdx.x) * eb + slot;
  const bool active = slot < eb && e < m.nelem;

  for (int i = tid; i < Q * P1; i += blockDim.x) sJ[i] = m.basis[i];
  for (int i = tid; i < Q * Q; i += blockDim.x) sD[i] = m.basis[2 * Q * P1 + i];

  double* sU = ebuf + size_t(active ? slot : 0) * S::NBUF * NC * Q3;
  double* sA = sU + NC * Q3;
  double* sB = sA + NC * Q3;
  double* sC = sB + NC * Q3;

  const int* l2g = m.l2g + e * P3;
  // ---- gather u^e = Q u (Eq. (21)); Dirichlet nodes read as 0 when masking
  if (active) {
    for (int idx = t; idx < P3; idx += QQ) {
      const int g = __ldg(l2g + idx);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double v;
        if (g >= 0) v = __ldg(a.u + size_t(g) * NC + c);
        else v = a.mask_in ? 0.0 : __ldg(a.u + size_t(-g - 1) * NC + c);
        sU[c * Q3 + idx] = v;
      }
    }
  }
  __syncthreads();

  double uq[NC][Q];
  if constexpr (COLLOC) {
    if (active) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int z = 0; z < Q; ++z) uq[c][z] = sU[c * Q3 + z * QQ + t];
    }
  } else {
    // stage x: T1[k][j][qx] = sum_i J[qx][i] U[k][j][i]
    if (active && ty < P1) {
#pragma unroll 1
      for (int k = 0; k < P1; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = 0.0;
#pragma unroll
          for (int i = 0; i < P1; ++i) s += sJ[tx * P1 + i] * sU[c * Q3 + k * P1 * P1 + ty * P1 + i];
          sA[c * Q3 + k * P1 * Q + ty * Q + tx] = s;
        }
    }
    __syncthreads();
    // stage y: T2[k][qy][qx] = sum_j J[qy][j] T1[k][j][qx]
    if (active) {
#pragma unroll 1
      for (int k = 0; k < P1; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = 0.0;
#pragma unroll
          for (int j = 0; j < P1; ++j) s += sJ[ty * P1 + j] * sA[c * Q3 + k * P1 * Q + j * Q + tx];
          sB[c * Q3 + k * QQ + t] = s;
        }
    }
    __syncthreads();
    // stage z: u(qx, qy, qz) = sum_k J[qz][k] T2[k][qy][qx], kept in registers
    if (active) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double col[P1];
#pragma unroll
        for (int k = 0; k < P1; ++k) col[k] = sB[c * Q3 + k * QQ + t];
#pragma unroll
        for (int z = 0; z < Q; ++z) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < P1; ++k) s += sJ[z * P1 + k] * col[k];
          uq[c][z] = s;
          if constexpr (KIND == kStiff) sA[c * Q3 + z * QQ + t] = s;
        }
      }
    }
    __syncthreads();
  }

  // ---- quadrature-point operator
  double vq[NC][Q];
  if constexpr (KIND == kMass) {
    if (active) {
      const double* M = a.G + e * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const double mz = __ldcs(M + z * QQ + t);
#pragma unroll
        for (int c = 0; c < NC; ++c) vq[c][z] = mz * uq[c][z];
      }
    }
  } else {
    double* sUQ = COLLOC ? sU : sA;
    double* sR = COLLOC ? sA : sB;
    double* sS = COLLOC ? sB : sC;
    double tq[NC][Q];
    if (active) {
      const double* G = a.G + e * 6 * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const int pt = z * QQ + t;
        const double g00 = __ldcs(G + 0 * Q3 + pt), g01 = __ldcs(G + 1 * Q3 + pt), g02 = __ldcs(G + 2 * Q3 + pt);
        const double g11 = __ldcs(G + 3 * Q3 + pt), g12 = __ldcs(G + 4 * Q3 + pt), g22 = __ldcs(G + 5 * Q3 + pt);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
          for (int n = 0; n < Q; ++n) {
            ur += sD[tx * Q + n] * sUQ[c * Q3 + z * QQ + ty * Q + n];
            us += sD[ty * Q + n] * sUQ[c * Q3 + z * QQ + n * Q + tx];
            ut += sD[z * Q + n] * uq[c][n];
          }
          sR[c * Q3 + pt] = g00 * ur + g01 * us + g02 * ut;
          sS[c * Q3 + pt] = g01 * ur + g11 * us + g12 * ut;
          tq[c][z] = g02 * ur + g12 * us + g22 * ut;
        }
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int z = 0; z < Q; ++z) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double v = 0.0;
#pragma unroll
          for (int n = 0; n < Q; ++n) {
            v += sD[n * Q + tx] * sR[c * Q3 + z * QQ + ty * Q + n];
            v += sD[n * Q + ty] * sS[c * Q3 + z * QQ + n * Q + tx];
            v += sD[n * Q + z] * tq[c][n];
          }
          vq[c][z] = v;
        }
      }
      if (a.beta != 0.0) {  // Helmholtz: + beta B u at the quadrature points (Eq. (17))
        const double* M = a.Mq + e * Q3;
#pragma unroll
        for (int z = 0; z < Q; ++z) {
          const double bm = a.beta * __ldg(M + z * QQ + t);
#pragma unroll
          for (int c = 0; c < NC; ++c) vq[c][z] += bm * uq[c][z];
        }
      }
    }
  }

  // ---- carry back to the nodes, write w^e, accumulate (u^e, w^e)
  double dot[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dot[c] = 0.0;
  double* wl = a.wl + size_t(e) * P3 * NC;
  if constexpr (COLLOC) {
    if (active) {
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const int idx = z * QQ + t;
        const bool skip = a.skip_dirichlet_out && __ldg(l2g + idx) < 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (!skip) wl[size_t(idx) * NC + c] = vq[c][z];
          dot[c] += vq[c][z] * uq[c][z];
        }
      }
    }
  } else {
    __syncthreads();
    // stage z^T: T2[k][qy][qx] = sum_qz J[qz][k] v(qx, qy, qz)
    if (active) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < P1; ++k) {
          double s = 0.0;
#pragma unroll
          for (int z = 0; z < Q; ++z) s += sJ[z * P1 + k] * vq[c][z];
          sA[c * Q3 + k * QQ + t] = s;
        }
    }
    __syncthreads();
    // stage y^T: T1[k][j][qx] = sum_qy J[qy][j] T2[k][qy][qx]
    if (active && ty < P1) {
#pragma unroll 1
      for (int k = 0; k < P1; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = 0.0;
#pragma unroll
          for (int y = 0; y < Q; ++y) s += sJ[y * P1 + ty] * sA[c * Q3 + k * QQ + y * Q + tx];
          sB[c * Q3 + k * P1 * Q + ty * Q + tx] = s;
        }
    }
    __syncthreads();
    // stage x^T: w[k][j][i] = sum_qx J[qx][i] T1[k][j][qx]
    if (active && tx < P1 && ty < P1) {
#pragma unroll 1
      for (int k = 0; k < P1; ++k) {
        const int idx = k * P1 * P1 + ty * P1 + tx;
        const bool skip = a.skip_dirichlet_out && __ldg(l2g + idx) < 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double s = 0.0;
#pragma unroll
          for (int x = 0; x < Q; ++x) s += sJ[x * P1 + tx] * sB[c * Q3 + k * P1 * Q + ty * Q + x];
          if (!skip) wl[size_t(idx) * NC + c] = s;
          dot[c] += s * sU[c * Q3 + idx];
        }
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

// Launch one instantiation.
template <int P1, int Q, bool COLLOC, int KIND, int NC>
cudaError_t launch_elem_t(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  const int eb = elem_per_block<P1, Q, COLLOC, NC>();
  const int nthreads = ((eb * Q * Q + 31) / 32) * 32;
  const size_t smem = elem_smem_bytes<P1, Q, COLLOC, NC>(eb);
  auto kern = elem_kernel<P1, Q, COLLOC, KIND, NC>;
  // set once per instantiation (not a stream operation; kept out of graph capture)
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + eb - 1) / eb;
  kern<<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

template <int P1, int Q, bool COLLOC, int NC>
inline int elem_blocks_t(int64_t nelem) {
  const int eb = elem_per_block<P1, Q, COLLOC, NC>();
  return int((nelem + eb - 1) / eb);
}

}  // namespace ceedbp
