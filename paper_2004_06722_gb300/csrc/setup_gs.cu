// Setup kernels (geometric factors, local Jacobi diagonals) and the
// deterministic gather-scatter sum of Q^T.
//
// Geometric factors, Eq. (23): at every quadrature point
//   G_mm' = rho_i rho_j rho_k |J| sum_l (d r_m / d x_l)(d r_m' / d x_l)
//         = w kappa adj(J) adj(J)^T / |J|,
// with J_dm = d x_d / d r_m of the iso-parametric map of Eq. (18), obtained
// by the sum-factorized contractions (J (x) J (x) Dh) x_d etc.  The mass
// factors rho_i rho_j rho_k |J| are those of Eq. (34).
//
// Gather-scatter: w_g = sum over the local slots s of node g (sorted by slot)
// of w_L[s] -- the action of Q^T in Eq. (21) in a fixed summation order, with
// no floating-point atomics.  Bit 31 of off[g] flags a Dirichlet node, whose
// output is zero when masking (the restriction of Algorithm 1).
#include "common.cuh"

namespace ceedbp {

namespace {

constexpr int kGeomBlocks = 1216;  // 8 x 152 SMs

template <int P1, int Q>
__global__ void geom_kernel(const DeviceMesh m, const double* __restrict__ coords, const double* __restrict__ kappa,
                            double* __restrict__ G, double* __restrict__ Mq, double* __restrict__ scratch) {
  constexpr int QQ = Q * Q, Q3 = QQ * Q, P3 = P1 * P1 * P1;
  extern __shared__ double smem[];
  double* sJ = smem;            // [Q][P1]
  double* sDh = sJ + Q * P1;    // [Q][P1]
  double* sw = sDh + Q * P1;    // [Q]
  double* sX = sw + Q;          // [3][P3]
  const double* basis = m.basis;
  for (int i = threadIdx.x; i < Q * P1; i += blockDim.x) {
    sJ[i] = basis[i];
    sDh[i] = basis[Q * P1 + i];
  }
  for (int i = threadIdx.x; i < Q; i += blockDim.x) sw[i] = basis[2 * Q * P1 + Q * Q + i];
  double* jac = scratch + size_t(blockIdx.x) * 9 * Q3;
  const int t = threadIdx.x, tx = t % Q, ty = t / Q;
  for (int64_t e = blockIdx.x; e < m.nelem; e += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * P3; i += blockDim.x) {
      const int a = i / 3, d = i - 3 * a;
      sX[d * P3 + a] = coords[(e * P3 + a) * 3 + d];
    }
    __syncthreads();
    if (t < QQ) {
      for (int d = 0; d < 3; ++d)
        for (int mm = 0; mm < 3; ++mm) {
          const double* Bx = mm == 0 ? sDh : sJ;
          const double* By = mm == 1 ? sDh : sJ;
          const double* Bz = mm == 2 ? sDh : sJ;
          double Ty[P1];
          for (int k = 0; k < P1; ++k) {
            double sy = 0.0;
            for (int j = 0; j < P1; ++j) {
              double sx = 0.0;
              for (int i = 0; i < P1; ++i) sx += Bx[tx * P1 + i] * sX[d * P3 + k * P1 * P1 + j * P1 + i];
              sy += By[ty * P1 + j] * sx;
            }
            Ty[k] = sy;
          }
          for (int z = 0; z < Q; ++z) {
            double v = 0.0;
            for (int k = 0; k < P1; ++k) v += Bz[z * P1 + k] * Ty[k];
            jac[(d * 3 + mm) * Q3 + z * QQ + t] = v;
          }
        }
    }
    __syncthreads();
    for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x) {
      double A[3][3];
      for (int d = 0; d < 3; ++d)
        for (int mm = 0; mm < 3; ++mm) A[d][mm] = jac[(d * 3 + mm) * Q3 + pt];
      // adj[m][d] = |J| (J^-1)[m][d] = |J| d r_m / d x_d
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
      const int qx = pt % Q, qy = (pt / Q) % Q, qz = pt / QQ;
      const double wq = sw[qx] * sw[qy] * sw[qz];
      if (Mq) Mq[e * Q3 + pt] = wq * det;
      if (G) {
        const double kap = kappa ? kappa[e * Q3 + pt] : 1.0;
        const double s = wq * kap / det;
        const int mi[6] = {0, 0, 0, 1, 1, 2}, mj[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; ++c) {
          const int a1 = mi[c], a2 = mj[c];
          G[(e * 6 + c) * Q3 + pt] =
              s * (adj[a1][0] * adj[a2][0] + adj[a1][1] * adj[a2][1] + adj[a1][2] * adj[a2][2]);
        }
      }
    }
  }
}

// diag(A^e) (stiffness: sum over the six G terms) or diag(B^e) (mass) per local node:
// diag(i,j,k) = sum_{mm'} c_mm' sum_Q F_mm'(Q) Mx[qx][i] My[qy][j] Mz[qz][k],
// M_d = A_d o B_d (elementwise), A_d = Dh if m == d else J, B_d = Dh if m' == d else J.
template <int P1, int Q>
__global__ void local_diag_kernel(const DeviceMesh m, int kind, const double* __restrict__ G,
                                  const double* __restrict__ Mq, double* __restrict__ wl) {
  constexpr int QQ = Q * Q, Q3 = QQ * Q, P3 = P1 * P1 * P1;
  extern __shared__ double smem[];
  double* sJ = smem;
  double* sDh = sJ + Q * P1;
  double* sM = sDh + Q * P1;   // [3][Q][P1]
  double* sF = sM + 3 * Q * P1;  // [Q3]
  double* sT1 = sF + Q3;       // [Q][Q][P1]
  double* sT2 = sT1 + QQ * P1;  // [Q][P1][P1]
  for (int i = threadIdx.x; i < Q * P1; i += blockDim.x) {
    sJ[i] = m.basis[i];
    sDh[i] = m.basis[Q * P1 + i];
  }
  const int64_t e = blockIdx.x;
  const int t = threadIdx.x, tx = t % Q, ty = t / Q;
  double acc[P1];
  for (int k = 0; k < P1; ++k) acc[k] = 0.0;
  const int nterms = kind == kStiff ? 6 : 1;
  const int mi[6] = {0, 0, 0, 1, 1, 2}, mj[6] = {0, 1, 2, 1, 2, 2};
  for (int term = 0; term < nterms; ++term) {
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * Q * P1; i += blockDim.x) {
      const int d = i / (Q * P1), r = i - d * Q * P1;
      double a1, a2;
      if (kind == kStiff) {
        a1 = (mi[term] == d ? sDh : sJ)[r];
        a2 = (mj[term] == d ? sDh : sJ)[r];
      } else {
        a1 = a2 = sJ[r];
      }
      sM[i] = a1 * a2;
    }
    const double scale = (kind == kStiff && mi[term] != mj[term]) ? 2.0 : 1.0;
    for (int pt = threadIdx.x; pt < Q3; pt += blockDim.x)
      sF[pt] = scale * (kind == kStiff ? G[(e * 6 + term) * Q3 + pt] : Mq[e * Q3 + pt]);
    __syncthreads();
    // x: T1[qz][qy][i] = sum_qx Mx[qx][i] F[qz][qy][qx]
    if (t < QQ && tx < P1)
      for (int z = 0; z < Q; ++z) {
        double s = 0.0;
        for (int x = 0; x < Q; ++x) s += sM[0 * Q * P1 + x * P1 + tx] * sF[z * QQ + ty * Q + x];
        sT1[z * Q * P1 + ty * P1 + tx] = s;
      }
    __syncthreads();
    // y: T2[qz][j][i] = sum_qy My[qy][j] T1[qz][qy][i]
    if (t < QQ && tx < P1 && ty < P1)
      for (int z = 0; z < Q; ++z) {
        double s = 0.0;
        for (int y = 0; y < Q; ++y) s += sM[1 * Q * P1 + y * P1 + ty] * sT1[z * Q * P1 + y * P1 + tx];
        sT2[z * P1 * P1 + ty * P1 + tx] = s;
      }
    __syncthreads();
    // z: diag[k][j][i] += sum_qz Mz[qz][k] T2[qz][j][i]
    if (t < QQ && tx < P1 && ty < P1)
      for (int k = 0; k < P1; ++k) {
        double s = 0.0;
        for (int z = 0; z < Q; ++z) s += sM[2 * Q * P1 + z * P1 + k] * sT2[z * P1 * P1 + ty * P1 + tx];
        acc[k] += s;
      }
  }
  if (t < QQ && tx < P1 && ty < P1)
    for (int k = 0; k < P1; ++k) wl[e * P3 + k * P1 * P1 + ty * P1 + tx] = acc[k];
}

template <int NC>
__global__ void gs_kernel(const int* __restrict__ off, const int* __restrict__ slots, const double* __restrict__ wl,
                          double* __restrict__ w, int64_t n, int mask_out) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const int o0 = __ldg(off + g), o1 = __ldg(off + g + 1) & 0x7fffffff;
    const bool dir = o0 < 0;
    double s[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = 0.0;
    if (!(dir && mask_out)) {
      for (int k = o0 & 0x7fffffff; k < o1; ++k) {
        const int sl = __ldg(slots + k);
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] += __ldg(wl + size_t(sl) * NC + c);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) w[g * NC + c] = s[c];
  }
}

__global__ void scale_kernel(const double* __restrict__ d, const double* __restrict__ u, double* __restrict__ w,
                             int64_t n, int nc) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * nc; i += int64_t(gridDim.x) * blockDim.x)
    w[i] = d[i / nc] * u[i];
}

__global__ void dinv_kernel(const int* __restrict__ off, const double* __restrict__ diag, double* __restrict__ dinv,
                            int64_t n) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const double d = diag[g];
    dinv[g] = (dir || d == 0.0) ? 0.0 : 1.0 / d;
  }
}

template <int P1, int Q>
cudaError_t geom_t(const DeviceMesh& m, const double* coords, const double* kappa, double* G, double* Mq,
                   double* scratch, cudaStream_t s) {
  const int threads = ((Q * Q + 31) / 32) * 32;
  const size_t smem = sizeof(double) * (2 * Q * P1 + Q + 3 * P1 * P1 * P1);
  auto k = geom_kernel<P1, Q>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  k<<<geom_blocks(m.nelem), threads, smem, s>>>(m, coords, kappa, G, Mq, scratch);
  return cudaGetLastError();
}

template <int P1, int Q>
cudaError_t diag_t(const DeviceMesh& m, int kind, const double* G, const double* Mq, double* wl, cudaStream_t s) {
  const int threads = ((Q * Q + 31) / 32) * 32;
  const size_t smem = sizeof(double) * (2 * Q * P1 + 3 * Q * P1 + Q * Q * Q + Q * Q * P1 + Q * P1 * P1);
  auto k = local_diag_kernel<P1, Q>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  k<<<unsigned(m.nelem), threads, smem, s>>>(m, kind, G, Mq, wl);
  return cudaGetLastError();
}

}  // namespace

int geom_blocks(int64_t nelem) { return int(nelem < kGeomBlocks ? nelem : kGeomBlocks); }
size_t geom_scratch_doubles(int blocks, int q) { return size_t(blocks) * 9 * q * q * q; }

#define CEEDBP_CASES_PQ(X)                                                                              \
  X(2, 2) X(3, 3) X(4, 4) X(5, 5) X(6, 6) X(7, 7) X(8, 8) X(9, 9) X(10, 10) X(11, 11) X(12, 12) X(13, 13) \
  X(14, 14) X(15, 15) X(16, 16) X(2, 3) X(3, 4) X(4, 5) X(5, 6) X(6, 7) X(7, 8) X(8, 9) X(9, 10)         \
  X(10, 11) X(11, 12) X(12, 13) X(13, 14) X(14, 15) X(15, 16) X(16, 17)

cudaError_t launch_geom(const DeviceMesh& m, const double* coords, const double* kappa, double* G, double* Mq,
                        double* scratch, cudaStream_t s) {
#define X(P, QV) \
  if (m.p1 == P && m.q == QV) return geom_t<P, QV>(m, coords, kappa, G, Mq, scratch, s);
  CEEDBP_CASES_PQ(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_local_diag(const DeviceMesh& m, int kind, const double* G, const double* Mq, double* wl,
                              cudaStream_t s) {
#define X(P, QV) \
  if (m.p1 == P && m.q == QV) return diag_t<P, QV>(m, kind, G, Mq, wl, s);
  CEEDBP_CASES_PQ(X)
#undef X
  return cudaErrorInvalidValue;
}

int vec_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > kGeomBlocks ? kGeomBlocks : b));
}

cudaError_t launch_gs(const DeviceMesh& m, const double* wl, double* w, int mask_out, cudaStream_t s) {
  if (m.ncomp == 3)
    gs_kernel<3><<<vec_blocks(m.nglobal), 256, 0, s>>>(m.off, m.slots, wl, w, m.nglobal, mask_out);
  else
    gs_kernel<1><<<vec_blocks(m.nglobal), 256, 0, s>>>(m.off, m.slots, wl, w, m.nglobal, mask_out);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* d, const double* u, double* w, int64_t n, int ncomp, cudaStream_t s) {
  scale_kernel<<<vec_blocks(n * ncomp), 256, 0, s>>>(d, u, w, n, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_dinv(const int* off, const double* diag, double* dinv, int64_t n, cudaStream_t s) {
  dinv_kernel<<<vec_blocks(n), 256, 0, s>>>(off, diag, dinv, n);
  return cudaGetLastError();
}

}  // namespace ceedbp
