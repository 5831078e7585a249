// Jacobi-PCG vector kernels on FP32 pairs (the FP64-accurate path that issues
// no FP64 arithmetic inside the iteration; see df.cuh).
//
// The CG vectors x, r, p and the Jacobi inverse are stored as pairs (8 bytes,
// the size of a double); b and the returned x stay FP64 at the interface.
// Per-thread sums are accumulated as pairs and handed to the FP64 block and
// grid reductions of common.cuh, so alpha and beta are formed in FP64 exactly
// as in the FP64 kernels (pcg.cu).
#include "common.cuh"
#include "df.cuh"
#include "internal.h"

namespace ceedbp {

namespace {

__device__ __forceinline__ dfloat df_from_f64_scalar(double v) { return f64_to_df(v); }

template <int NC>
__global__ void init_df_kernel(const int* __restrict__ off, const double* __restrict__ b,
                               const double* __restrict__ ax, double* __restrict__ x, dfloat* __restrict__ xd,
                               dfloat* __restrict__ r, dfloat* __restrict__ p, const dfloat* __restrict__ dinv,
                               int64_t n, int x0, double* partials, SolveState* st, double tol, int fixed) {
  __shared__ double red[32 * 3 * NC];
  double acc[3 * NC];
#pragma unroll
  for (int k = 0; k < 3 * NC; ++k) acc[k] = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const dfloat di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const size_t i = size_t(g) * NC + c;
      const double bv = dir ? 0.0 : b[i];
      const double rv64 = dir ? 0.0 : bv - (ax ? ax[i] : 0.0);
      const dfloat rv = f64_to_df(rv64);
      const dfloat zv = dw_mul(di, rv);
      if (dir) x[i] = 0.0;
      xd[i] = (x0 && !dir) ? f64_to_df(x[i]) : dfloat{0.0f, 0.0f};
      r[i] = rv;
      p[i] = zv;
      acc[c] += df_to_f64(dw_mul(rv, zv));
      acc[NC + c] += rv64 * rv64;
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
__global__ void update_df_kernel(const int* __restrict__ off, const int* __restrict__ slots,
                                 const dfloat* __restrict__ wl, dfloat* __restrict__ x, dfloat* __restrict__ r,
                                 const dfloat* __restrict__ p, const dfloat* __restrict__ dinv, int64_t n,
                                 double* partials, SolveState* st) {
  __shared__ double red[32 * 2 * NC];
  if (st->stop) return;
  dfloat alpha[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    alpha[c] = df_from_f64_scalar(st->c[c].alpha);
  }
  dfloat rz[NC], rr[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rz[c] = rr[c] = dfloat{0.0f, 0.0f};
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const int o0 = __ldg(off + g);
    if (o0 < 0) continue;
    const int o1 = __ldg(off + g + 1) & 0x7fffffff;
    // start from the first slot (the local values are normalised pairs, so this equals adding
    // them to zero); a node no element touches sums to 0
    dfloat w[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = dfloat{0.0f, 0.0f};
    if (o0 < o1) {
      const int sl = __ldg(slots + o0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(wl + size_t(sl) * NC + c));
        w[c] = dfloat{v.x, v.y};
      }
    }
    // the remaining slots two at a time (loads issued together, sums in slot order)
    int k = o0 + 1;
    for (; k + 1 < o1; k += 2) {
      const int s0 = __ldg(slots + k), s1 = __ldg(slots + k + 1);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 v0 = __ldcs(reinterpret_cast<const float2*>(wl + size_t(s0) * NC + c));
        const float2 v1 = __ldcs(reinterpret_cast<const float2*>(wl + size_t(s1) * NC + c));
        w[c] = dw_add(w[c], dfloat{v0.x, v0.y});
        w[c] = dw_add(w[c], dfloat{v1.x, v1.y});
      }
    }
    if (k < o1) {
      const int s0 = __ldg(slots + k);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(wl + size_t(s0) * NC + c));
        w[c] = dw_add(w[c], dfloat{v.x, v.y});
      }
    }
    const dfloat di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const size_t i = size_t(g) * NC + c;
      const dfloat rv = dw_add(r[i], dw_neg(dw_mul(alpha[c], w[c])));
      x[i] = dw_add(x[i], dw_mul(alpha[c], p[i]));
      r[i] = rv;
      rz[c] = dw_add(rz[c], dw_mul(rv, dw_mul(di, rv)));
      rr[c] = dw_add(rr[c], dw_mul(rv, rv));
    }
  }
  double acc[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    acc[c] = df_to_f64(rz[c]);
    acc[NC + c] = df_to_f64(rr[c]);
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
__global__ void dir_df_kernel(const int* __restrict__ off, const dfloat* __restrict__ r, dfloat* __restrict__ p,
                              const dfloat* __restrict__ dinv, int64_t n, const SolveState* st) {
  if (st->stop) return;
  dfloat beta[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    beta[c] = df_from_f64_scalar(st->c[c].beta);
  }
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    if (__ldg(off + g) < 0) continue;
    const dfloat di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const size_t i = size_t(g) * NC + c;
      p[i] = dw_add(dw_mul(di, r[i]), dw_mul(beta[c], p[i]));
    }
  }
}

__global__ void df_to_f64_kernel(const dfloat* __restrict__ src, double* __restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = df_to_f64(src[i]);
}

__global__ void f64_to_df_kernel(const double* __restrict__ src, dfloat* __restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = f64_to_df(src[i]);
}

template <int NC>
__global__ void gs_df_kernel(const int* __restrict__ off, const int* __restrict__ slots, const dfloat* __restrict__ wl,
                             double* __restrict__ w, int64_t n, int mask_out) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const int o0 = __ldg(off + g), o1 = __ldg(off + g + 1) & 0x7fffffff;
    dfloat s[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = dfloat{0.0f, 0.0f};
    if (!(o0 < 0 && mask_out)) {
      for (int k = o0 & 0x7fffffff; k < o1; ++k) {
        const int sl = __ldg(slots + k);
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = dw_add(s[c], wl[size_t(sl) * NC + c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) w[g * NC + c] = df_to_f64(s[c]);
  }
}

}  // namespace

cudaError_t launch_init_df(const DeviceMesh& m, const double* b, const double* ax, double* x, dfloat* xd, dfloat* r,
                           dfloat* p, const dfloat* dinv, int x0, double* partials, SolveState* st, double tol,
                           int fixed, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    init_df_kernel<3><<<nb, 256, 0, s>>>(m.off, b, ax, x, xd, r, p, dinv, m.nglobal, x0, partials, st, tol, fixed);
  else
    init_df_kernel<1><<<nb, 256, 0, s>>>(m.off, b, ax, x, xd, r, p, dinv, m.nglobal, x0, partials, st, tol, fixed);
  return cudaGetLastError();
}

cudaError_t launch_update_df(const DeviceMesh& m, const dfloat* wl, dfloat* x, dfloat* r, const dfloat* p,
                             const dfloat* dinv, double* partials, SolveState* st, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    update_df_kernel<3><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, p, dinv, m.nglobal, partials, st);
  else
    update_df_kernel<1><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, p, dinv, m.nglobal, partials, st);
  return cudaGetLastError();
}

cudaError_t launch_dir_df(const DeviceMesh& m, const dfloat* r, dfloat* p, const dfloat* dinv, const SolveState* st,
                          cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3)
    dir_df_kernel<3><<<nb, 256, 0, s>>>(m.off, r, p, dinv, m.nglobal, st);
  else
    dir_df_kernel<1><<<nb, 256, 0, s>>>(m.off, r, p, dinv, m.nglobal, st);
  return cudaGetLastError();
}

cudaError_t launch_df_to_f64(const dfloat* src, double* dst, int64_t n, cudaStream_t s) {
  df_to_f64_kernel<<<vec_blocks(n), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_f64_to_df(const double* src, dfloat* dst, int64_t n, cudaStream_t s) {
  f64_to_df_kernel<<<vec_blocks(n), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_gs_df(const DeviceMesh& m, const dfloat* wl, double* w, int mask_out, cudaStream_t s) {
  if (m.ncomp == 3)
    gs_df_kernel<3><<<vec_blocks(m.nglobal), 256, 0, s>>>(m.off, m.slots, wl, w, m.nglobal, mask_out);
  else
    gs_df_kernel<1><<<vec_blocks(m.nglobal), 256, 0, s>>>(m.off, m.slots, wl, w, m.nglobal, mask_out);
  return cudaGetLastError();
}

}  // namespace ceedbp
