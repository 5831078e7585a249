// Element operator kernels (the column kernel): w^e = A^e u^e or B^e u^e for
// every element, the unassembled product A_L Q u of Eq. (21).  It serves BK5/BK6
// at even orders, BK2/BK4, and BK3 at order 14; BK1/BK3 otherwise run the
// even-odd kernel of elem_gl.cuh, and BK5/BK6 at odd orders that of elem_eo.cuh.
// The even-odd tables and products (EoTab, eo_build, eo_mul) defined here are
// shared by those kernels.
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

// Even-odd form (Eq. (37)) of a product y = M x with M centro-symmetric
// (SIGN = +1: M[A-1-a][B-1-b] = M[a][b], the interpolation J and J^T) or
// centro-antisymmetric (SIGN = -1: the derivative D and D^T).  With
// x+_b = x_b + x_{B-1-b}, x-_b = x_b - x_{B-1-b} (b < B/2) and the half tables
// E = (M[a][b] + M[a][B-1-b]) / 2, O = (M[a][b] - M[a][B-1-b]) / 2 of the top
// rows (a < (A+1)/2), plus the middle column M[a][B/2] when B is odd:
//   y_a = S_E + S_O,  y_{A-1-a} = SIGN (S_E - S_O),
// and for odd A the middle row is S_E (SIGN = +1) or S_O (SIGN = -1).  About
// half the multiply-adds of the direct product; used for the contractions
// that stay in a thread's registers.
template <int A, int B>
struct EoTab {
  static constexpr int HA = (A + 1) / 2, HB = B / 2;
  static constexpr int SIZE = 2 * HA * HB + HA;  // [E HA x HB][O HA x HB][middle column HA]
};

// tables of row-major M (A x B, leading dimension ld, element (a, b) at M[a * ld + b],
// or M[b * ld + a] when TRANS) into T
template <int A, int B, bool TRANS>
__device__ __forceinline__ void eo_build(const double* M, int ld, double* T, int tid, int nthr) {
  using E = EoTab<A, B>;
  for (int q = tid; q < E::HA * E::HB; q += nthr) {
    const int ra = q / E::HB, cb = q % E::HB;
    const double m0 = TRANS ? M[cb * ld + ra] : M[ra * ld + cb];
    const double m1 = TRANS ? M[(B - 1 - cb) * ld + ra] : M[ra * ld + B - 1 - cb];
    T[q] = 0.5 * (m0 + m1);
    T[E::HA * E::HB + q] = 0.5 * (m0 - m1);
  }
  if constexpr (B % 2 == 1)
    for (int ra = tid; ra < E::HA; ra += nthr) T[2 * E::HA * E::HB + ra] = TRANS ? M[(B / 2) * ld + ra] : M[ra * ld + B / 2];
}

template <int A, int B, int SIGN>
__device__ __forceinline__ void eo_mul(const double* T, const double (&x)[B], double (&y)[A]) {
  using E = EoTab<A, B>;
  constexpr int HA = E::HA, HB = E::HB;
  const double* TE = T;
  const double* TO = T + HA * HB;
  const double* TM = T + 2 * HA * HB;
  double xe[HB > 0 ? HB : 1], xo[HB > 0 ? HB : 1];
#pragma unroll
  for (int b = 0; b < HB; ++b) {
    xe[b] = x[b] + x[B - 1 - b];
    xo[b] = x[b] - x[B - 1 - b];
  }
  // the odd half-sum accumulates on top of the even one: y[ra] = S_E + S_O leaves the chain and
  // the mirror output is one fma of it (one FP64 operation fewer per output pair)
#pragma unroll
  for (int ra = 0; ra < A / 2; ++ra) {
    double se = 0.0;
#pragma unroll
    for (int b = 0; b < HB; ++b) se += TE[ra * HB + b] * xe[b];
    if constexpr (B % 2 == 1) se += TM[ra] * x[B / 2];
    double s = se;
#pragma unroll
    for (int b = 0; b < HB; ++b) s = __fma_rn(TO[ra * HB + b], xo[b], s);
    y[ra] = s;                                                               // S_E + S_O
    y[A - 1 - ra] = SIGN > 0 ? __fma_rn(2.0, se, -s) : __fma_rn(-2.0, se, s);  // S_E - S_O or S_O - S_E
  }
  if constexpr (A % 2 == 1) {
    constexpr int ra = A / 2;
    double sm = 0.0;
#pragma unroll
    for (int b = 0; b < HB; ++b) sm += SIGN > 0 ? TE[ra * HB + b] * xe[b] : TO[ra * HB + b] * xo[b];
    if constexpr (SIGN > 0 && B % 2 == 1) sm += TM[ra] * x[B / 2];
    y[ra] = sm;
  }
}

// EO tables of the generic kernel: J (Q x P1), J^T (P1 x Q), D (Q x Q), D^T (Q x Q)
template <int P1, int Q>
constexpr int elem_eo_tab_doubles() {
  return EoTab<Q, P1>::SIZE + EoTab<P1, Q>::SIZE + 2 * EoTab<Q, Q>::SIZE;
}

template <int P1, int Q, bool COLLOC, int NC>
inline int elem_per_block() {
  constexpr int QQ = Q * Q;
  int eb = 256 / (QQ * NC);
  return eb < 1 ? 1 : eb;
}

template <int P1, int Q, bool COLLOC, int NC>
inline size_t elem_smem_bytes(int eb) {
  using S = ElemShape<P1, Q, COLLOC>;
  return sizeof(double) * (size_t(Q) * P1 + size_t(Q) * Q + elem_eo_tab_doubles<P1, Q>() +
                           size_t(eb) * S::NBUF * NC * S::Q3 + 32 * NC);
}

// Threads of one block (whole warps); the launch bound below lets the compiler
// size registers for exactly this block.
template <int Q, int NC>
constexpr int elem_threads() {
  return (((256 / (Q * Q * NC) < 1 ? 1 : 256 / (Q * Q * NC)) * Q * Q + 31) / 32) * 32;
}

template <int P1, int Q, bool COLLOC, int KIND, int NC, bool BATCH = false>
__global__ void __launch_bounds__(elem_threads<Q, NC>()) elem_kernel(const DeviceMesh m, const ElemArgs a,
                                                                     const int eb) {
  using S = ElemShape<P1, Q, COLLOC>;
  constexpr int QQ = S::QQ, Q3 = S::Q3, P3 = S::P3;
  extern __shared__ double smem[];
  if (a.state != nullptr && a.state->stop) return;

  double* sJ = smem;            // [Q][P1]
  double* sD = sJ + Q * P1;     // [Q][Q]
  double* red = sD + Q * Q;     // 32 * NC reduction scratch
  double* tJ = red + 32 * NC;   // even-odd tables of J, J^T, D, D^T (register contractions)
  double* tJT = tJ + EoTab<Q, P1>::SIZE;
  double* tD = tJT + EoTab<P1, Q>::SIZE;
  double* tDT = tD + EoTab<Q, Q>::SIZE;
  double* ebuf = tDT + EoTab<Q, Q>::SIZE;

  const int tid = threadIdx.x;
  const int slot = tid / QQ, t = tid - (tid / QQ) * QQ;
  const int tx = t % Q, ty = t / Q;
  int64_t e0 = int64_t(blockIdx.x) * eb;
  int nact = m.nelem - e0 < eb ? int(m.nelem - e0) : eb;
  int prob = 0;
  if constexpr (BATCH) {  // batched: this block holds elements of one problem (block tables)
    prob = a.blk_prob[blockIdx.x];
    if (!a.bst[prob].c.active) return;
    e0 = a.blk_e0[blockIdx.x];
    nact = a.blk_n[blockIdx.x];
  }
  const int64_t e = e0 + slot;
  const bool active = slot < nact;

  for (int i = tid; i < Q * P1; i += blockDim.x) sJ[i] = m.basis[i];
  for (int i = tid; i < Q * Q; i += blockDim.x) sD[i] = m.basis[2 * Q * P1 + i];
  // read by every thread only after the barrier that follows the gather
  eo_build<Q, P1, false>(m.basis, P1, tJ, tid, blockDim.x);
  eo_build<P1, Q, true>(m.basis, P1, tJT, tid, blockDim.x);
  eo_build<Q, Q, false>(m.basis + 2 * Q * P1, Q, tD, tid, blockDim.x);
  eo_build<Q, Q, true>(m.basis + 2 * Q * P1, Q, tDT, tid, blockDim.x);

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
        double col[P1], uz[Q];
#pragma unroll
        for (int k = 0; k < P1; ++k) col[k] = sB[c * Q3 + k * QQ + t];
        eo_mul<Q, P1, 1>(tJ, col, uz);
#pragma unroll
        for (int z = 0; z < Q; ++z) {
          uq[c][z] = uz[z];
          if constexpr (KIND == kStiff) sA[c * Q3 + z * QQ + t] = uz[z];
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
      // t derivatives of the whole column first (even-odd, in registers); tq[c][z] holds u_t
      // until the loop below overwrites it with the t component of G grad u
#pragma unroll
      for (int c = 0; c < NC; ++c) eo_mul<Q, Q, -1>(tD, uq[c], tq[c]);
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const int pt = z * QQ + t;
        const double g00 = __ldcs(G + 0 * Q3 + pt), g01 = __ldcs(G + 1 * Q3 + pt), g02 = __ldcs(G + 2 * Q3 + pt);
        const double g11 = __ldcs(G + 3 * Q3 + pt), g12 = __ldcs(G + 4 * Q3 + pt), g22 = __ldcs(G + 5 * Q3 + pt);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double ur = 0.0, us = 0.0;
          const double ut = tq[c][z];
#pragma unroll
          for (int n = 0; n < Q; ++n) {
            ur += sD[tx * Q + n] * sUQ[c * Q3 + z * QQ + ty * Q + n];
            us += sD[ty * Q + n] * sUQ[c * Q3 + z * QQ + n * Q + tx];
          }
          sR[c * Q3 + pt] = g00 * ur + g01 * us + g02 * ut;
          sS[c * Q3 + pt] = g01 * ur + g11 * us + g12 * ut;
          tq[c][z] = g02 * ur + g12 * us + g22 * ut;
        }
      }
    }
    __syncthreads();
    if (active) {
      // t part of the transpose for the whole column (even-odd, in registers)
#pragma unroll
      for (int c = 0; c < NC; ++c) eo_mul<Q, Q, -1>(tDT, tq[c], vq[c]);
#pragma unroll
      for (int z = 0; z < Q; ++z) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double v = vq[c][z];
#pragma unroll
          for (int n = 0; n < Q; ++n) {
            v += sD[n * Q + tx] * sR[c * Q3 + z * QQ + ty * Q + n];
            v += sD[n * Q + ty] * sS[c * Q3 + z * QQ + n * Q + tx];
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
      for (int c = 0; c < NC; ++c) {
        double wk[P1];
        eo_mul<P1, Q, 1>(tJT, vq[c], wk);
#pragma unroll
        for (int k = 0; k < P1; ++k) sA[c * Q3 + k * QQ + t] = wk[k];
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

// Launch one instantiation of the kernel.
template <int P1, int Q, bool COLLOC, int KIND, int NC, bool BATCH>
cudaError_t launch_elem_b(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  const int eb = elem_per_block<P1, Q, COLLOC, NC>();
  const int nthreads = ((eb * Q * Q + 31) / 32) * 32;
  const size_t smem = elem_smem_bytes<P1, Q, COLLOC, NC>(eb);
  auto kern = elem_kernel<P1, Q, COLLOC, KIND, NC, BATCH>;
  // set once per instantiation (not a stream operation; kept out of graph capture)
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = BATCH ? int64_t(a.batch_blocks) : (m.nelem + eb - 1) / eb;
  kern<<<unsigned(blocks), nthreads, smem, s>>>(m, a, eb);
  return cudaGetLastError();
}

// Launch one instantiation (batched solves take the block-table variant: collocated stiffness,
// one component).
template <int P1, int Q, bool COLLOC, int KIND, int NC>
cudaError_t launch_elem_t(const DeviceMesh& m, const ElemArgs& a, cudaStream_t s) {
  if constexpr (COLLOC && KIND == kStiff && NC == 1) {
    if (a.blk_prob != nullptr) return launch_elem_b<P1, Q, COLLOC, KIND, NC, true>(m, a, s);
  }
  return launch_elem_b<P1, Q, COLLOC, KIND, NC, false>(m, a, s);
}

template <int P1, int Q, bool COLLOC, int NC>
inline int elem_blocks_t(int64_t nelem) {
  const int eb = elem_per_block<P1, Q, COLLOC, NC>();
  return int((nelem + eb - 1) / eb);
}

}  // namespace ceedbp
