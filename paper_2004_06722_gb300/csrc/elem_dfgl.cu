// BK1/BK3 element operator (Gauss quadrature, q = N + 2) on FP32 pairs: the
// FP64-accurate arithmetic of df.cuh for the bake-off problems with
// interpolation stages (Table 1: BP1 mass, BP3 Poisson; one component).
//
// Stages as in the FP64 kernel of elem_gl.cuh, one thread per line:
// interpolation J (q x p1) along x, y, z; for BK3 the GL derivative Dq along
// the r and s lines and the t column, the factors G of Eq. (23) per point, the
// transposes Dq^T, and for BK1 the mass factors of Eq. (34); then J^T back
// along z, y, x.  Every 1D output is a sum of pair products accumulated with a
// power-of-two splitter (SplitAcc of df.cuh): the splitter of a line is set by
// the line's own largest input times the largest absolute row sum of the
// matrix applied, which bounds every partial sum of every output of that line;
// the G products take a splitter per point and row.  Pair results are
// normalised (two_sum) before they feed the next stage.  Direct products (not
// the even-odd halves): a pair addition costs about two pair products, so the
// even-odd split saves nothing here.
#include <cuda_runtime.h>

#include "common.cuh"
#include "df.cuh"
#include "kernel_args.h"

namespace ceedbp {
namespace {

template <int P1, int Q>
struct DfGlShape {
  static constexpr int QQ = Q * Q, Q3 = QQ * Q, P3 = P1 * P1 * P1;
  static constexpr int EB = 256 / QQ < 1 ? 1 : 256 / QQ;
  static constexpr int THREADS = ((EB * QQ + 31) / 32) * 32;
  static constexpr int SLOT = P3 + 3 * Q3;  // pairs per element
  static constexpr int TAB = Q * P1 + Q * Q;  // J then Dq, pairs
};

// Bound factor on the splitter: the hi parts used for the bounds miss the lo
// parts (2^-24 relative) and the rounded row sums (a few ulps).
constexpr float kBoundSlack = 1.0001f;

__device__ __forceinline__ dfloat norm_pair(dfloat v) {
  dfloat r;
  two_sum(v.hi, v.lo, r.hi, r.lo);
  return r;
}

// y[a] = sum_n M[a * lda + n * ldn] x[n], a < A, n < B, with one splitter from max|x| and the
// largest absolute row sum R of M
template <int A, int B>
__device__ __forceinline__ void line_mul(const dfloat* M, int lda, int ldn, float R, const dfloat (&x)[B],
                                         dfloat (&y)[A]) {
  float mx = 0.0f;
#pragma unroll
  for (int n = 0; n < B; ++n) mx = fmaxf(mx, fabsf(x[n].hi));
  const float sig = splitter(__fmul_rn(__fmul_rn(mx, R), kBoundSlack));
#pragma unroll
  for (int a = 0; a < A; ++a) {
    SplitAcc acc(sig);
#pragma unroll
    for (int n = 0; n < B; ++n) {
      const dfloat m = M[a * lda + n * ldn];
      acc.add(m.hi, m.lo, x[n].hi, x[n].lo);
    }
    y[a] = norm_pair(acc.result(sig));
  }
}

// The same with the outputs stored to shared memory, out[a * ostride], one output at a time
// (a rolled loop keeps the code of the many line stages small enough for the instruction cache)
template <int A, int B>
__device__ __forceinline__ void line_mul_to(const dfloat* M, int lda, int ldn, float R, const dfloat (&x)[B],
                                            dfloat* out, int ostride) {
  float mx = 0.0f;
#pragma unroll
  for (int n = 0; n < B; ++n) mx = fmaxf(mx, fabsf(x[n].hi));
  const float sig = splitter(__fmul_rn(__fmul_rn(mx, R), kBoundSlack));
#pragma unroll 1
  for (int a = 0; a < A; ++a) {
    SplitAcc acc(sig);
    const dfloat* Ma = M + a * lda;
#pragma unroll
    for (int n = 0; n < B; ++n) {
      const dfloat m = Ma[n * ldn];
      acc.add(m.hi, m.lo, x[n].hi, x[n].lo);
    }
    out[a * ostride] = norm_pair(acc.result(sig));
  }
}

// (g_k0 ur + g_k1 us + g_k2 ut) with a splitter from this point's values
__device__ __forceinline__ dfloat grow(dfloat g0, dfloat g1, dfloat g2, dfloat ur, dfloat us, dfloat ut, float mx) {
  const float rs = fabsf(g0.hi) + fabsf(g1.hi) + fabsf(g2.hi);
  const float sig = splitter(__fmul_rn(__fmul_rn(mx, rs), kBoundSlack));
  SplitAcc acc(sig);
  acc.add(g0.hi, g0.lo, ur.hi, ur.lo);
  acc.add(g1.hi, g1.lo, us.hi, us.lo);
  acc.add(g2.hi, g2.lo, ut.hi, ut.lo);
  return norm_pair(acc.result(sig));
}

template <int P1, int Q, int KIND>
__global__ void __launch_bounds__(DfGlShape<P1, Q>::THREADS) elem_dfgl_kernel(const DeviceMesh m, const ElemDfArgs a) {
  using S = DfGlShape<P1, Q>;
  constexpr int QQ = S::QQ, Q3 = S::Q3, P3 = S::P3, EB = S::EB;
  extern __shared__ __align__(16) unsigned char smem_dfgl[];
  if (a.state != nullptr && a.state->stop) return;
  double* red = reinterpret_cast<double*>(smem_dfgl);      // 32
  float* rows = reinterpret_cast<float*>(red + 32);        // 4 row-sum bounds (+ padding)
  dfloat* sJ = reinterpret_cast<dfloat*>(rows + 4);        // [Q][P1]
  dfloat* sD = sJ + Q * P1;                                // [Q][Q]
  dfloat* ebuf = sD + Q * Q;

  const int tid = threadIdx.x;
  const int slot = tid / QQ, t = tid - slot * QQ;
  const int64_t e0 = int64_t(blockIdx.x) * EB;
  const int nact = m.nelem - e0 < EB ? int(m.nelem - e0) : EB;
  const int64_t e = e0 + slot;
  const bool active = slot < nact;

  for (int i = tid; i < S::TAB; i += blockDim.x) sJ[i] = a.D[i];
  if (tid < 4) {
    // 0: rows of J, 1: rows of J^T (columns of J), 2: rows of Dq, 3: rows of Dq^T
    float best = 0.0f;
    const int na = tid == 0 ? Q : (tid == 1 ? P1 : Q), nb = tid == 1 ? Q : (tid == 0 ? P1 : Q);
    for (int r = 0; r < na; ++r) {
      float sum = 0.0f;
      for (int c = 0; c < nb; ++c) {
        dfloat v;
        if (tid == 0) v = a.D[r * P1 + c];
        else if (tid == 1) v = a.D[c * P1 + r];
        else if (tid == 2) v = a.D[Q * P1 + r * Q + c];
        else v = a.D[Q * P1 + c * Q + r];
        sum = __fadd_ru(sum, fabsf(v.hi));
      }
      best = fmaxf(best, sum);
    }
    rows[tid] = best;
  }

  dfloat* sU = ebuf + size_t(active ? slot : 0) * S::SLOT;
  dfloat* sA = sU + P3;
  dfloat* sB = sA + Q3;
  dfloat* sC = sB + Q3;
  const int* l2g = m.l2g + e * P3;
  if constexpr (KIND == kStiff) {
    // the element's G (48 q^3 bytes) into L2 now, in 128-byte lines: the factor stage reads it
    // after the gather and five line stages, from L2 instead of HBM
    if (active) {
      const char* gsrc = reinterpret_cast<const char*>(a.G + e * 6 * Q3);
      for (int q = t; q < (48 * Q3 + 127) / 128; q += QQ)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(gsrc + size_t(q) * 128));
    }
  }
  if (active) {
    for (int idx = t; idx < P3; idx += QQ) {
      const int g = __ldg(l2g + idx);
      const int gg = g < 0 ? -g - 1 : g;
      dfloat v{0.0f, 0.0f};
      if (!(g < 0 && a.mask_in)) v = a.u_f64 != nullptr ? f64_to_df(__ldg(a.u_f64 + gg)) : a.u_df[gg];
      sU[idx] = v;
    }
  }
  // BK1: the column's mass factors are loaded now, their latency hidden behind the x and y stages
  dfloat mq[KIND == kMass ? Q : 1];
  if constexpr (KIND == kMass) {
    if (active) {
      const dfloat* M = a.G + e * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) mq[z] = M[t + QQ * z];
    }
  }
  __syncthreads();
  const float RJ = rows[0], RJT = rows[1], RD = rows[2], RDT = rows[3];

  // ---- x: line (j, k) = t along i
  if (active && t < P1 * P1) {
    dfloat x[P1];
#pragma unroll
    for (int i = 0; i < P1; ++i) x[i] = sU[t * P1 + i];
    line_mul_to<Q, P1>(sJ, P1, 1, RJ, x, sA + t * Q, 1);
  }
  __syncthreads();
  // ---- y: line (qx, k) along j
  if (active && t < Q * P1) {
    const int qx = t % Q, k = t / Q;
    dfloat x[P1];
#pragma unroll
    for (int j = 0; j < P1; ++j) x[j] = sA[qx + Q * (j + P1 * k)];
    line_mul_to<Q, P1>(sJ, P1, 1, RJ, x, sB + qx + QQ * k, Q);
  }
  __syncthreads();
  // ---- z: column (qx, qy) = t
  dfloat uq[Q];
  if (active) {
    dfloat x[P1];
#pragma unroll
    for (int k = 0; k < P1; ++k) x[k] = sB[t + QQ * k];
    line_mul<Q, P1>(sJ, P1, 1, RJ, x, uq);
    if constexpr (KIND == kStiff) {
#pragma unroll
      for (int z = 0; z < Q; ++z) sC[t + QQ * z] = uq[z];
    }
  }

  dfloat vq[Q];
  if constexpr (KIND == kMass) {
    if (active) {
#pragma unroll
      for (int z = 0; z < Q; ++z) vq[z] = norm_pair(dw_mul(mq[z], uq[z]));
    }
  } else {
    __syncthreads();
    if (active) {  // u_r on line (qy, z) = (lo, hi), u_s on line (qx, z) = (lo, hi)
      const int lo = t % Q, hi = t / Q;
      dfloat x[Q];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sC[n + Q * lo + QQ * hi];
      line_mul_to<Q, Q>(sD, Q, 1, RD, x, sA + Q * lo + QQ * hi, 1);
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sC[lo + Q * n + QQ * hi];
      line_mul_to<Q, Q>(sD, Q, 1, RD, x, sB + lo + QQ * hi, Q);
    }
    __syncthreads();
    dfloat wt[Q];
    if (active) {
      dfloat ut[Q];
      line_mul<Q, Q>(sD, Q, 1, RD, uq, ut);
      const dfloat* G = a.G + e * 6 * Q3;
#pragma unroll
      for (int z = 0; z < Q; ++z) {
        const int pt = t + QQ * z;
        const dfloat g00 = G[0 * Q3 + pt], g01 = G[1 * Q3 + pt], g02 = G[2 * Q3 + pt];
        const dfloat g11 = G[3 * Q3 + pt], g12 = G[4 * Q3 + pt], g22 = G[5 * Q3 + pt];
        const dfloat ur = sA[pt], us = sB[pt];
        const float mx = fmaxf(fmaxf(fabsf(ur.hi), fabsf(us.hi)), fabsf(ut[z].hi));
        sA[pt] = grow(g00, g01, g02, ur, us, ut[z], mx);
        sB[pt] = grow(g01, g11, g12, ur, us, ut[z], mx);
        wt[z] = grow(g02, g12, g22, ur, us, ut[z], mx);
      }
    }
    __syncthreads();
    if (active) {  // transposes Dq^T (row a of Dq^T is column a of Dq), r and s in place
      const int lo = t % Q, hi = t / Q;
      dfloat x[Q];
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sA[n + Q * lo + QQ * hi];
      line_mul_to<Q, Q>(sD, 1, Q, RDT, x, sA + Q * lo + QQ * hi, 1);
#pragma unroll
      for (int n = 0; n < Q; ++n) x[n] = sB[lo + Q * n + QQ * hi];
      line_mul_to<Q, Q>(sD, 1, Q, RDT, x, sB + lo + QQ * hi, Q);
      line_mul<Q, Q>(sD, 1, Q, RDT, wt, vq);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int z = 0; z < Q; ++z) vq[z] = dw_add(dw_add(vq[z], sA[t + QQ * z]), sB[t + QQ * z]);
    }
  }
  __syncthreads();
  // ---- z^T: column t, rows of J^T
  if (active) {
    dfloat wk[P1];
    line_mul<P1, Q>(sJ, 1, P1, RJT, vq, wk);
#pragma unroll
    for (int k = 0; k < P1; ++k) sC[t + QQ * k] = wk[k];
  }
  __syncthreads();
  // ---- y^T: line (qx, k)
  if (active && t < Q * P1) {
    const int qx = t % Q, k = t / Q;
    dfloat x[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = sC[qx + Q * (q + Q * k)];
    line_mul_to<P1, Q>(sJ, 1, P1, RJT, x, sA + qx + Q * P1 * k, Q);
  }
  __syncthreads();
  // ---- x^T: line (j, k) = t
  if (active && t < P1 * P1) {
    dfloat x[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = sA[q + Q * t];
    line_mul_to<P1, Q>(sJ, 1, P1, RJT, x, sB + t * P1, 1);
  }
  __syncthreads();
  dfloat acc_dot{0.0f, 0.0f};
  if (active) {
    dfloat* wl = a.wl + size_t(e) * P3;
    for (int idx = t; idx < P3; idx += QQ) {
      const dfloat w = sB[idx];
      if (!(a.skip_dirichlet_out && __ldg(l2g + idx) < 0)) wl[idx] = w;
      acc_dot = dw_add(acc_dot, dw_mul(w, sU[idx]));
    }
  }
  if (a.partials != nullptr) {
    double dot[1] = {df_to_f64(acc_dot)};
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

template <int P1, int Q, int KIND>
cudaError_t launch_dfgl_t(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  using S = DfGlShape<P1, Q>;
  const size_t smem = sizeof(double) * 32 + sizeof(float) * 4 + sizeof(dfloat) * (S::TAB + size_t(S::EB) * S::SLOT);
  auto kern = elem_dfgl_kernel<P1, Q, KIND>;
  static const cudaError_t attr = [&] {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + S::EB - 1) / S::EB;
  kern<<<unsigned(blocks), S::THREADS, smem, s>>>(m, a);
  return cudaGetLastError();
}

template <int P1>
cudaError_t launch_dfgl_p(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  return m.bp == 1 ? launch_dfgl_t<P1, P1 + 1, kMass>(m, a, s) : launch_dfgl_t<P1, P1 + 1, kStiff>(m, a, s);
}

}  // namespace

// Orders 1..15 (at order 15 one element of q^3 pair tiles takes 150 KB of shared memory).
bool elem_dfgl_supported(const DeviceMesh& m) {
  return !m.colloc && m.ncomp == 1 && (m.bp == 1 || m.bp == 3) && m.p1 >= 2 && m.p1 <= 16;
}

int elem_dfgl_blocks(const DeviceMesh& m) {
  const int qq = (m.p1 + 1) * (m.p1 + 1);
  const int eb = 256 / qq < 1 ? 1 : 256 / qq;
  return int((m.nelem + eb - 1) / eb);
}

cudaError_t launch_elem_dfgl(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if (!elem_dfgl_supported(m)) return cudaErrorInvalidValue;
  switch (m.p1) {
    case 2: return launch_dfgl_p<2>(m, a, s);
    case 3: return launch_dfgl_p<3>(m, a, s);
    case 4: return launch_dfgl_p<4>(m, a, s);
    case 5: return launch_dfgl_p<5>(m, a, s);
    case 6: return launch_dfgl_p<6>(m, a, s);
    case 7: return launch_dfgl_p<7>(m, a, s);
    case 8: return launch_dfgl_p<8>(m, a, s);
    case 9: return launch_dfgl_p<9>(m, a, s);
    case 10: return launch_dfgl_p<10>(m, a, s);
    case 11: return launch_dfgl_p<11>(m, a, s);
    case 12: return launch_dfgl_p<12>(m, a, s);
    case 13: return launch_dfgl_p<13>(m, a, s);
    case 14: return launch_dfgl_p<14>(m, a, s);
    case 15: return launch_dfgl_p<15>(m, a, s);
    case 16: return launch_dfgl_p<16>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ceedbp
