// Fused Jacobi-PCG kernels with device-resident scalars (Sec. 3: diagonally
// preconditioned CG around the bake-off kernels).
//
// One iteration = three launches:
//   elem   : w_L = A_L Q p and pAp = sum_e (p^e, w^e) (Algorithm 1 computes this
//            dot before the direct-stiffness sum: it needs no multiplicity
//            weighting); the last block forms alpha = rz / pAp.
//   update : w = Q^T w_L (deterministic gather-scatter, masked), then
//            x += alpha p, r -= alpha w, z = dinv r, and the sums (r, z), (r, r);
//            the last block forms beta = rz_new / rz and tests ||r|| <= tol ||b||.
//   dir    : p = dinv r + beta p.
// Independent components (BP6) carry their own scalars and stop separately.
#include "common.cuh"

namespace ceedbp {

namespace {

template <int NC>
__global__ void pcg_init_kernel(const int* __restrict__ off, const double* __restrict__ b,
                                const double* __restrict__ ax, double* __restrict__ x, double* __restrict__ r,
                                double* __restrict__ p,
                                const double* __restrict__ dinv, int64_t n, double* partials, SolveState* st,
                                double tol, int fixed) {
  __shared__ double red[32 * 3 * NC];
  double acc[3 * NC];
#pragma unroll
  for (int k = 0; k < 3 * NC; ++k) acc[k] = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const double di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double bv = dir ? 0.0 : b[g * NC + c];
      const double rv = dir ? 0.0 : bv - (ax ? ax[g * NC + c] : 0.0);
      const double zv = di * rv;
      if (dir) x[g * NC + c] = 0.0;
      r[g * NC + c] = rv;
      p[g * NC + c] = zv;
      acc[c] += rv * zv;
      acc[NC + c] += rv * rv;
      acc[2 * NC + c] += bv * bv;
    }
  }
  if (grid_sum_last<3 * NC>(acc, partials, gridDim.x, blockIdx.x, &st->ticket[kTicketInit], red)) {
    if (threadIdx.x == 0) {
      int any = 0;
      st->ncomp = NC;
      st->fixed = fixed;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        CompScalars& cs = st->c[c];
        cs.rz = acc[c];
        cs.rr = acc[NC + c];
        cs.bb = acc[2 * NC + c];
        cs.tol2 = tol * tol * cs.bb;
        cs.pAp = 0.0;
        cs.alpha = cs.beta = 0.0;
        cs.iters = 0;
        cs.status = isfinite(cs.rz) && isfinite(cs.rr) && isfinite(cs.bb) ? CEEDBP_OK : CEEDBP_EBREAKDOWN;
        cs.active = cs.status != CEEDBP_OK ? 0 : (fixed ? 1 : (cs.rr > cs.tol2 ? 1 : 0));
        any |= cs.active;
      }
      for (int c = NC; c < 3; ++c) st->c[c].active = 0;
      st->stop = any ? 0 : 1;
    }
  }
}

template <int NC>
__global__ void pcg_update_kernel(const int* __restrict__ off, const int* __restrict__ slots,
                                  const double* __restrict__ wl, double* __restrict__ x, double* __restrict__ r,
                                  const double* __restrict__ p, const double* __restrict__ dinv, int64_t n,
                                  double* partials, SolveState* st) {
  __shared__ double red[32 * 2 * NC];
  if (st->stop) return;
  double alpha[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    alpha[c] = st->c[c].alpha;
  }
  double acc[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; ++k) acc[k] = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const int o0 = __ldg(off + g);
    if (o0 < 0) continue;  // Dirichlet node: x, r, p stay zero
    const int o1 = __ldg(off + g + 1) & 0x7fffffff;
    // start from the first slot (one FP64 add fewer per node); a node no element touches sums to 0
    double w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = 0.0;
    if (o0 < o1) {
      const int sl = __ldg(slots + o0);
#pragma unroll
      for (int c = 0; c < NC; ++c) w[c] = __ldcs(wl + size_t(sl) * NC + c);
    }
    // the remaining slots two at a time (loads issued together, sums in slot order)
    int k = o0 + 1;
    for (; k + 1 < o1; k += 2) {
      const int s0 = __ldg(slots + k), s1 = __ldg(slots + k + 1);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double v0 = __ldcs(wl + size_t(s0) * NC + c), v1 = __ldcs(wl + size_t(s1) * NC + c);
        w[c] += v0;
        w[c] += v1;
      }
    }
    if (k < o1) {
      const int s0 = __ldg(slots + k);
#pragma unroll
      for (int c = 0; c < NC; ++c) w[c] += __ldcs(wl + size_t(s0) * NC + c);
    }
    const double di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const size_t i = size_t(g) * NC + c;
      const double rv = r[i] - alpha[c] * w[c];
      x[i] += alpha[c] * p[i];
      r[i] = rv;
      acc[c] += rv * (di * rv);
      acc[NC + c] += rv * rv;
    }
  }
  if (grid_sum_last<2 * NC>(acc, partials, gridDim.x, blockIdx.x, &st->ticket[kTicketUpdate], red)) {
    if (threadIdx.x == 0) {
      int any = 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        CompScalars& cs = st->c[c];
        if (!cs.active) continue;
        const double rz_new = acc[c];
        cs.beta = cs.rz != 0.0 ? rz_new / cs.rz : 0.0;
        cs.rz = rz_new;
        cs.rr = acc[NC + c];
        cs.iters += 1;
        if (!isfinite(rz_new)) {
          cs.status = CEEDBP_EBREAKDOWN;
          if (!st->fixed) cs.active = 0;
        }
        if (!st->fixed && cs.rr <= cs.tol2) cs.active = 0;
        any |= cs.active;
      }
      if (!any) st->stop = 1;
    }
  }
}

template <int NC>
__global__ void pcg_dir_kernel(const int* __restrict__ off, const double* __restrict__ r, double* __restrict__ p,
                               const double* __restrict__ dinv, int64_t n, const SolveState* st) {
  if (st->stop) return;
  double beta[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    beta[c] = st->c[c].beta;
  }
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    if (__ldg(off + g) < 0) continue;
    const double di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const size_t i = size_t(g) * NC + c;
      p[i] = di * r[i] + beta[c] * p[i];
    }
  }
}

}  // namespace

cudaError_t launch_pcg_init(const DeviceMesh& m, const double* b, const double* ax, double* x, double* r, double* p,
                            const double* dinv, double* partials, SolveState* st, double tol, int fixed,
                            cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    pcg_init_kernel<3><<<nb, 256, 0, s>>>(m.off, b, ax, x, r, p, dinv, m.nglobal, partials, st, tol, fixed);
  else
    pcg_init_kernel<1><<<nb, 256, 0, s>>>(m.off, b, ax, x, r, p, dinv, m.nglobal, partials, st, tol, fixed);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(const DeviceMesh& m, const double* wl, double* x, double* r, const double* p,
                              const double* dinv, double* partials, SolveState* st, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    pcg_update_kernel<3><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, p, dinv, m.nglobal, partials, st);
  else
    pcg_update_kernel<1><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, p, dinv, m.nglobal, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_pcg_dir(const DeviceMesh& m, const double* r, double* p, const double* dinv,
                           const SolveState* st, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    pcg_dir_kernel<3><<<nb, 256, 0, s>>>(m.off, r, p, dinv, m.nglobal, st);
  else
    pcg_dir_kernel<1><<<nb, 256, 0, s>>>(m.off, r, p, dinv, m.nglobal, st);
  return cudaGetLastError();
}

}  // namespace ceedbp
