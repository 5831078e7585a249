// Variable-coefficient Poisson and its adjoint gradient (BP5-type, collocated).
//
// Eq. (4) with mu = kappa(x): the stiffness factors of Eq. (23) become
// kappa_q Ghat_q with Ghat the coefficient-free factors.  For
// J = 1/2 (u - u*)^T B (u - u*) and A(kappa) u = b the gradient at quadrature
// point q of element e is
//   dJ/dkappa_{e,q} = -(grad lambda)_q^T Ghat_q (grad u)_q,   A lambda = M B (u - u*),
// with grad = (D_1, D_2, D_3) of Eq. (22) applied to the element's nodal values
// (one adjoint solve: A is symmetric).
#include "common.cuh"

namespace ceedbp {

namespace {

template <int P1>
__global__ void kappa_grad_kernel(const DeviceMesh m, const double* __restrict__ u, const double* __restrict__ lam,
                                  const double* __restrict__ Ghat, double* __restrict__ g) {
  constexpr int PP = P1 * P1, P3 = PP * P1;
  __shared__ double sD[P1 * P1];
  __shared__ double sU[P3], sL[P3];
  const int t = threadIdx.x, i = t % P1, j = t / P1;
  for (int q = t; q < PP; q += blockDim.x) sD[q] = m.basis[2 * P1 * P1 + q];
  const int64_t e = blockIdx.x;
  const int* l2g = m.l2g + e * P3;
  if (t < PP)
    for (int k = 0; k < P1; ++k) {
      const int gi = __ldg(l2g + t + PP * k);
      sU[t + PP * k] = gi >= 0 ? u[gi] : 0.0;
      sL[t + PP * k] = gi >= 0 ? lam[gi] : 0.0;
    }
  __syncthreads();
  if (t >= PP) return;
  const double* G = Ghat + e * 6 * P3;
  for (int k = 0; k < P1; ++k) {
    double ur = 0, us = 0, ut = 0, lr = 0, ls = 0, lt = 0;
#pragma unroll
    for (int n = 0; n < P1; ++n) {
      ur += sD[i * P1 + n] * sU[k * PP + j * P1 + n];
      us += sD[j * P1 + n] * sU[k * PP + n * P1 + i];
      ut += sD[k * P1 + n] * sU[n * PP + j * P1 + i];
      lr += sD[i * P1 + n] * sL[k * PP + j * P1 + n];
      ls += sD[j * P1 + n] * sL[k * PP + n * P1 + i];
      lt += sD[k * P1 + n] * sL[n * PP + j * P1 + i];
    }
    const int pt = k * PP + t;
    const double g00 = G[0 * P3 + pt], g01 = G[1 * P3 + pt], g02 = G[2 * P3 + pt];
    const double g11 = G[3 * P3 + pt], g12 = G[4 * P3 + pt], g22 = G[5 * P3 + pt];
    const double wr = g00 * ur + g01 * us + g02 * ut;
    const double ws = g01 * ur + g11 * us + g12 * ut;
    const double wt = g02 * ur + g12 * us + g22 * ut;
    g[e * P3 + pt] = -(lr * wr + ls * ws + lt * wt);
  }
}

__global__ void scale_factors_kernel(const double* __restrict__ Ghat, const double* __restrict__ kappa,
                                     double* __restrict__ G, int64_t nelem, int q3) {
  const int64_t total = nelem * 6 * q3;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = i / (6 * int64_t(q3));
    const int64_t pt = i % q3;
    G[i] = Ghat[i] * kappa[e * q3 + pt];
  }
}

// rhs = M B (u - u*) and J = 1/2 (u - u*)^T B (u - u*) with the assembled diagonal GLL mass.
__global__ void misfit_kernel(const int* __restrict__ off, const double* __restrict__ mdiag,
                              const double* __restrict__ u, const double* __restrict__ us, double* __restrict__ rhs,
                              int64_t n, double* partials, unsigned* ticket, double* out) {
  __shared__ double red[32];
  double acc[1] = {0.0};
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const double d = u[g] - us[g];
    const double bd = mdiag[g] * d;
    rhs[g] = __ldg(off + g) < 0 ? 0.0 : bd;
    acc[0] += d * bd;
  }
  if (grid_sum_last<1>(acc, partials, gridDim.x, blockIdx.x, ticket, red))
    if (threadIdx.x == 0) out[0] = 0.5 * acc[0];
}

}  // namespace

cudaError_t launch_kappa_grad(const DeviceMesh& m, const double* u, const double* lam, const double* Ghat, double* g,
                              cudaStream_t s) {
  const int threads = ((m.p1 * m.p1 + 31) / 32) * 32;
#define CEEDBP_KG(P) \
  case P: kappa_grad_kernel<P><<<unsigned(m.nelem), threads, 0, s>>>(m, u, lam, Ghat, g); break;
  switch (m.p1) {
    CEEDBP_KG(2) CEEDBP_KG(3) CEEDBP_KG(4) CEEDBP_KG(5) CEEDBP_KG(6) CEEDBP_KG(7) CEEDBP_KG(8) CEEDBP_KG(9)
    CEEDBP_KG(10) CEEDBP_KG(11) CEEDBP_KG(12)
    default: return cudaErrorInvalidValue;
  }
#undef CEEDBP_KG
  return cudaGetLastError();
}

cudaError_t launch_scale_factors(const double* Ghat, const double* kappa, double* G, int64_t nelem, int q3,
                                 cudaStream_t s) {
  scale_factors_kernel<<<vec_blocks(nelem * 6 * q3), 256, 0, s>>>(Ghat, kappa, G, nelem, q3);
  return cudaGetLastError();
}

cudaError_t launch_misfit(const DeviceMesh& m, const double* mdiag, const double* u, const double* us, double* rhs,
                          double* partials, unsigned* ticket, double* out, cudaStream_t s) {
  misfit_kernel<<<vec_blocks(m.nglobal), 256, 0, s>>>(m.off, mdiag, u, us, rhs, m.nglobal, partials, ticket, out);
  return cudaGetLastError();
}

}  // namespace ceedbp
