// FP64 defect correction with a low-precision inner Jacobi-PCG.
//
// Outer loop (FP64): r = M (b - A x) with the FP64 operator, then the inner
// solve A_lp d = r / ||r|| with the operator in FP32 (geometric factors and
// the direction p stored in FP32 or BF16, FP32 arithmetic), and x += ||r|| d.
// FP64 accuracy is kept for the outer residual, the solution update and every
// CG inner product (FP32 products summed as FP32 pairs per thread, reduced in
// FP64).  The inner vectors x_in and r_in are FP32.
#include <cuda_bf16.h>

#include "common.cuh"
#include "df.cuh"
#include "internal.h"

namespace ceedbp {

namespace {

__device__ __forceinline__ float lp_get(const float* p) { return *p; }
__device__ __forceinline__ float lp_get(const __nv_bfloat16* p) {
  return __uint_as_float(unsigned(*reinterpret_cast<const unsigned short*>(p)) << 16);
}
__device__ __forceinline__ void lp_put(float* p, float v) { *p = v; }
__device__ __forceinline__ void lp_put(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// exact FP32 product as a pair, added to a pair accumulator
__device__ __forceinline__ void acc_prod(dfloat& acc, float a, float b) {
  const float ph = __fmul_rn(a, b);
  acc = dw_add(acc, dfloat{ph, __fmaf_rn(a, b, -ph)});
}

template <int NC>
__global__ void residual_kernel(const int* __restrict__ off, const double* __restrict__ b,
                                const double* __restrict__ ax, double* __restrict__ r, int64_t n, double* partials,
                                unsigned* ticket, double* out) {
  __shared__ double red[32 * NC];
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const size_t i = size_t(g) * NC + c;
      const double v = dir ? 0.0 : b[i] - (ax ? ax[i] : 0.0);
      r[i] = v;
      acc[c] += v * v;
    }
  }
  if (grid_sum_last<NC>(acc, partials, gridDim.x, blockIdx.x, ticket, red)) {
    if (threadIdx.x == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c) out[c] = acc[c];
  }
}

struct Scale3 {
  double s[3];
};

template <int NC, typename TS>
__global__ void inner_init_kernel(const int* __restrict__ off, const double* __restrict__ r64, Scale3 scale,
                                  const float* __restrict__ dinv, float* __restrict__ x, float* __restrict__ r,
                                  TS* __restrict__ p, int64_t n, double* partials, SolveState* st, double tol) {
  __shared__ double red[32 * 2 * NC];
  dfloat rz[NC], rr[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rz[c] = rr[c] = dfloat{0.0f, 0.0f};
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    const bool dir = __ldg(off + g) < 0;
    const float di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const size_t i = size_t(g) * NC + c;
      const float rv = dir ? 0.0f : float(r64[i] * scale.s[c]);
      const float zv = di * rv;
      x[i] = 0.0f;
      r[i] = rv;
      lp_put(p + i, zv);
      acc_prod(rz[c], rv, zv);
      acc_prod(rr[c], rv, rv);
    }
  }
  double acc[2 * NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    acc[c] = df_to_f64(rz[c]);
    acc[NC + c] = df_to_f64(rr[c]);
  }
  if (grid_sum_last<2 * NC>(acc, partials, gridDim.x, blockIdx.x, &st->ticket[kTicketInit], red)) {
    if (threadIdx.x == 0) {
      int any = 0;
      st->ncomp = NC;
      st->fixed = 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        CompScalars& cs = st->c[c];
        cs.rz = acc[c];
        cs.rr = acc[NC + c];
        cs.bb = acc[NC + c];
        cs.tol2 = tol * tol * cs.bb;
        cs.pAp = 0.0;
        cs.alpha = cs.beta = 0.0;
        cs.iters = 0;
        cs.status = isfinite(cs.rz) && isfinite(cs.rr) ? CEEDBP_OK : CEEDBP_EBREAKDOWN;
        cs.active = cs.status == CEEDBP_OK && cs.rr > cs.tol2 ? 1 : 0;
        any |= cs.active;
      }
      for (int c = NC; c < 3; ++c) st->c[c].active = 0;
      st->stop = any ? 0 : 1;
    }
  }
}

template <int NC, typename TS>
__global__ void inner_update_kernel(const int* __restrict__ off, const int* __restrict__ slots,
                                    const float* __restrict__ wl, float* __restrict__ x, float* __restrict__ r,
                                    const TS* __restrict__ p, const float* __restrict__ dinv, int64_t n,
                                    double* partials, SolveState* st) {
  __shared__ double red[32 * 2 * NC];
  if (st->stop) return;
  float alpha[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    alpha[c] = float(st->c[c].alpha);
  }
  dfloat rz[NC], rr[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rz[c] = rr[c] = dfloat{0.0f, 0.0f};
  // Two nodes per thread and step, g and g + stride: the offsets, the first local slot and its
  // values of both nodes are loaded before either is used (most nodes -- element interiors --
  // have exactly one slot), so two dependent load chains are in flight per thread.
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t g0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g0 < n; g0 += 2 * stride) {
    int64_t gs[2] = {g0, g0 + stride};
    int o0[2], o1[2];
    float w[2][NC];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool in = gs[h] < n;
      o0[h] = in ? __ldg(off + gs[h]) : -1;
      o1[h] = in ? (__ldg(off + gs[h] + 1) & 0x7fffffff) : 0;
    }
    int sl[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) sl[h] = (o0[h] >= 0 && o0[h] < o1[h]) ? __ldg(slots + o0[h]) : -1;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int c = 0; c < NC; ++c) w[h][c] = sl[h] >= 0 ? __ldcs(wl + size_t(sl[h]) * NC + c) : 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (o0[h] < 0) continue;  // Dirichlet node (or past the end)
      for (int k = o0[h] + 1; k < o1[h]; ++k) {
        const int s = __ldg(slots + k);
#pragma unroll
        for (int c = 0; c < NC; ++c) w[h][c] += __ldcs(wl + size_t(s) * NC + c);
      }
      const int64_t g = gs[h];
      const float di = dinv[g];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (!act[c]) continue;
        const size_t i = size_t(g) * NC + c;
        const float rv = fmaf(-alpha[c], w[h][c], r[i]);
        x[i] = fmaf(alpha[c], lp_get(p + i), x[i]);
        r[i] = rv;
        acc_prod(rz[c], rv, di * rv);
        acc_prod(rr[c], rv, rv);
      }
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
          cs.active = 0;
        }
        if (cs.rr <= cs.tol2) cs.active = 0;
        any |= cs.active;
      }
      if (!any) st->stop = 1;
    }
  }
}

template <int NC, typename TS>
__global__ void inner_dir_kernel(const int* __restrict__ off, const float* __restrict__ r, TS* __restrict__ p,
                                 const float* __restrict__ dinv, int64_t n, const SolveState* st) {
  if (st->stop) return;
  float beta[NC];
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    act[c] = st->c[c].active != 0;
    beta[c] = float(st->c[c].beta);
  }
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    if (__ldg(off + g) < 0) continue;
    const float di = dinv[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (!act[c]) continue;
      const size_t i = size_t(g) * NC + c;
      lp_put(p + i, fmaf(beta[c], lp_get(p + i), di * r[i]));
    }
  }
}

template <int NC>
__global__ void correct_kernel(const int* __restrict__ off, double* __restrict__ x, const float* __restrict__ d,
                               Scale3 norm, int64_t n) {
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    if (__ldg(off + g) < 0) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const size_t i = size_t(g) * NC + c;
      x[i] = fma(double(d[i]), norm.s[c], x[i]);
    }
  }
}

template <typename TO>
__global__ void narrow_kernel(const double* __restrict__ src, TO* __restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    lp_put(dst + i, float(src[i]));
}

}  // namespace

cudaError_t launch_residual(const DeviceMesh& m, const double* b, const double* ax, double* r, double* partials,
                            unsigned* ticket, double* out, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3) residual_kernel<3><<<nb, 256, 0, s>>>(m.off, b, ax, r, m.nglobal, partials, ticket, out);
  else residual_kernel<1><<<nb, 256, 0, s>>>(m.off, b, ax, r, m.nglobal, partials, ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_inner_init(const DeviceMesh& m, int bf16, const double* r64, const double* scale,
                              const float* dinv, float* x, float* r, void* p, double* partials, SolveState* st,
                              double tol, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  Scale3 sc{{scale[0], scale[1], scale[2]}};
  if (m.ncomp == 3) {
    if (bf16)
      inner_init_kernel<3, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, r64, sc, dinv, x, r, static_cast<__nv_bfloat16*>(p),
                                                             m.nglobal, partials, st, tol);
    else
      inner_init_kernel<3, float><<<nb, 256, 0, s>>>(m.off, r64, sc, dinv, x, r, static_cast<float*>(p), m.nglobal,
                                                     partials, st, tol);
  } else {
    if (bf16)
      inner_init_kernel<1, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, r64, sc, dinv, x, r, static_cast<__nv_bfloat16*>(p),
                                                             m.nglobal, partials, st, tol);
    else
      inner_init_kernel<1, float><<<nb, 256, 0, s>>>(m.off, r64, sc, dinv, x, r, static_cast<float*>(p), m.nglobal,
                                                     partials, st, tol);
  }
  return cudaGetLastError();
}

cudaError_t launch_inner_update(const DeviceMesh& m, int bf16, const float* wl, float* x, float* r, const void* p,
                                const float* dinv, double* partials, SolveState* st, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3) {
    if (bf16)
      inner_update_kernel<3, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r,
                                                               static_cast<const __nv_bfloat16*>(p), dinv, m.nglobal,
                                                               partials, st);
    else
      inner_update_kernel<3, float><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, static_cast<const float*>(p), dinv,
                                                       m.nglobal, partials, st);
  } else {
    if (bf16)
      inner_update_kernel<1, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r,
                                                               static_cast<const __nv_bfloat16*>(p), dinv, m.nglobal,
                                                               partials, st);
    else
      inner_update_kernel<1, float><<<nb, 256, 0, s>>>(m.off, m.slots, wl, x, r, static_cast<const float*>(p), dinv,
                                                       m.nglobal, partials, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_inner_dir(const DeviceMesh& m, int bf16, const float* r, void* p, const float* dinv,
                             const SolveState* st, cudaStream_t s) {
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3) {
    if (bf16)
      inner_dir_kernel<3, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, r, static_cast<__nv_bfloat16*>(p), dinv, m.nglobal, st);
    else
      inner_dir_kernel<3, float><<<nb, 256, 0, s>>>(m.off, r, static_cast<float*>(p), dinv, m.nglobal, st);
  } else {
    if (bf16)
      inner_dir_kernel<1, __nv_bfloat16><<<nb, 256, 0, s>>>(m.off, r, static_cast<__nv_bfloat16*>(p), dinv, m.nglobal, st);
    else
      inner_dir_kernel<1, float><<<nb, 256, 0, s>>>(m.off, r, static_cast<float*>(p), dinv, m.nglobal, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_correct(const DeviceMesh& m, double* x, const float* d, const double* norm, cudaStream_t s) {
  Scale3 sc{{norm[0], norm[1], norm[2]}};
  const int nb = vec_blocks(m.nglobal);
  if (m.ncomp == 3) correct_kernel<3><<<nb, 256, 0, s>>>(m.off, x, d, sc, m.nglobal);
  else correct_kernel<1><<<nb, 256, 0, s>>>(m.off, x, d, sc, m.nglobal);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const double* src, void* dst, int64_t n, int bf16, cudaStream_t s) {
  if (bf16) narrow_kernel<__nv_bfloat16><<<vec_blocks(n), 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), n);
  else narrow_kernel<float><<<vec_blocks(n), 256, 0, s>>>(src, static_cast<float*>(dst), n);
  return cudaGetLastError();
}

}  // namespace ceedbp
