// FP32 BK5/BK6 element operator for the inner solve of FP64 defect correction
// with the three 1D contraction stages on the tensor cores (order 7, p1 = 8).
//
// The contractions of Eq. (22) (J = I) are small dense products: along
// direction r, u_r(i, line) = sum_n D[i][n] u(n, line) for the 64 lines (j, k)
// of an element, i.e. the 64 x 8 matrix U_r^T times D^T; likewise for s and t,
// and the transposes w(n, line) = sum_i D[i][n] w_r(i, line) are U^T times D.
// Each is four m16n8k8 MMAs (16 lines x 8 outputs x 8 terms) on the warp-level
// tensor-core instruction.  TF32 keeps 11 significant bits, so every operand
// x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi) and the product is
// accumulated as a_hi b_hi + a_hi b_lo + a_lo b_hi in FP32 (the 3xTF32
// scheme; the dropped a_lo b_lo term is ~2^-22 of the product), which gives
// FP32-level contractions -- the same operator as elem_lp_kernel with FP32
// storage.  The geometric factors (Eq. (23)) multiply the gradient on the
// CUDA cores.
//
// One warp per element, four elements per block.  The element's tiles live in
// shared memory with planes padded to 72 floats (index i + 8 j + 72 k), which
// keeps the fragment loads of the three directions nearly free of bank
// conflicts.  The fused (p, A p) is accumulated as an FP32 pair per lane and
// reduced in FP64 with the last-block alpha of the other inner kernels.
#include <cuda_runtime.h>

#include "common.cuh"
#include "df.cuh"
#include "kernel_args.h"

namespace ceedbp {
namespace {

constexpr int kTcP1 = 8, kTcP3 = 512;
constexpr int kTcPlane = 72;                  // padded plane stride (floats)
constexpr int kTcTile = kTcP1 * kTcPlane;     // one component's padded tile
constexpr int kTcWarps = 4;                   // elements (warps) per block

__device__ __forceinline__ int tc_pad(int i, int j, int k) { return i + 8 * j + kTcPlane * k; }

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi, lo in TF32 (lo rounded too: the product error stays ~2^-22)
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C += A B in 3xTF32 (A given as the four FP32 fragment values, B pre-split)
__device__ __forceinline__ void mma3(float (&c)[4], const float (&a)[4], const unsigned (&bh)[2],
                                     const unsigned (&bl)[2]) {
  unsigned ah[4], al[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split_tf32(a[q], ah[q], al[q]);
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

// Padded tile position of entry (row = line in 0..63, col = index along the
// contracted direction) for direction d (0: r, lines (j, k); 1: s, lines (i, k);
// 2: t, lines (i, j)).
__device__ __forceinline__ int tc_pos(int d, int line, int col) {
  const int a = line & 7, b = line >> 3;
  if (d == 0) return tc_pad(col, a, b);
  if (d == 1) return tc_pad(a, col, b);
  return tc_pad(a, b, col);
}

template <int NC>
__global__ void __launch_bounds__(32 * kTcWarps) elem_tc_kernel(const DeviceMesh m, const ElemLpArgs a) {
  extern __shared__ double smem_tc[];
  if (a.state != nullptr && a.state->stop) return;
  double* red = smem_tc;  // 32 * NC
  float* base = reinterpret_cast<float*>(red + 32 * NC);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int64_t e = int64_t(blockIdx.x) * kTcWarps + warp;
  const bool active = e < m.nelem;
  float* sU = base + size_t(warp) * 4 * NC * kTcTile;  // u, then the three gradient tiles
  float* sW[3] = {sU + NC * kTcTile, sU + 2 * NC * kTcTile, sU + 3 * NC * kTcTile};

  // B operands from the FP64 derivative table Dq[i][n]: the gradient takes B[k = n][col = i] = D[i][n],
  // the transpose B[k = i][col = n] = D[i][n]; fragment b0 = B[t4][g], b1 = B[t4 + 4][g]
  const double* D = m.basis + 2 * kTcP1 * kTcP1;
  unsigned bgh[2], bgl[2], bth[2], btl[2];
  split_tf32(float(D[g * 8 + t4]), bgh[0], bgl[0]);
  split_tf32(float(D[g * 8 + t4 + 4]), bgh[1], bgl[1]);
  split_tf32(float(D[t4 * 8 + g]), bth[0], btl[0]);
  split_tf32(float(D[(t4 + 4) * 8 + g]), bth[1], btl[1]);

  const int* l2g = m.l2g + e * kTcP3;
  const float* u = static_cast<const float*>(a.u);
  if (active) {
    for (int idx = lane; idx < kTcP3; idx += 32) {
      const int gg = __ldg(l2g + idx);
      const int pos = tc_pad(idx & 7, (idx >> 3) & 7, idx >> 6);
#pragma unroll
      for (int c = 0; c < NC; ++c) sU[c * kTcTile + pos] = gg >= 0 ? __ldg(u + size_t(gg) * NC + c) : 0.0f;
    }
  }
  __syncwarp();

  // ---- gradient: three directions x four 16-line tiles per component
  if (active) {
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      const float* U = sU + c * kTcTile;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        float* W = sW[d] + c * kTcTile;
#pragma unroll
        for (int T = 0; T < 4; ++T) {
          const int l0 = 16 * T + g, l1 = l0 + 8;
          const float av[4] = {U[tc_pos(d, l0, t4)], U[tc_pos(d, l1, t4)], U[tc_pos(d, l0, t4 + 4)],
                               U[tc_pos(d, l1, t4 + 4)]};
          float cf[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          mma3(cf, av, bgh, bgl);
          // C[row][col]: c0 (g, 2t4), c1 (g, 2t4 + 1), c2 (g + 8, 2t4), c3 (g + 8, 2t4 + 1)
          W[tc_pos(d, l0, 2 * t4)] = cf[0];
          W[tc_pos(d, l0, 2 * t4 + 1)] = cf[1];
          W[tc_pos(d, l1, 2 * t4)] = cf[2];
          W[tc_pos(d, l1, 2 * t4 + 1)] = cf[3];
        }
      }
    }
  }
  __syncwarp();

  // ---- geometric factors at the 512 points (CUDA cores), in place
  if (active) {
    const float* G = static_cast<const float*>(a.G) + size_t(e) * 6 * kTcP3;
#pragma unroll 4
    for (int q = 0; q < kTcP3 / 32; ++q) {
      const int idx = q * 32 + lane;
      const int pos = tc_pad(idx & 7, (idx >> 3) & 7, idx >> 6);
      const float g00 = __ldcs(G + 0 * kTcP3 + idx), g01 = __ldcs(G + 1 * kTcP3 + idx);
      const float g02 = __ldcs(G + 2 * kTcP3 + idx), g11 = __ldcs(G + 3 * kTcP3 + idx);
      const float g12 = __ldcs(G + 4 * kTcP3 + idx), g22 = __ldcs(G + 5 * kTcP3 + idx);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float ur = sW[0][c * kTcTile + pos], us = sW[1][c * kTcTile + pos], ut = sW[2][c * kTcTile + pos];
        sW[0][c * kTcTile + pos] = g00 * ur + g01 * us + g02 * ut;
        sW[1][c * kTcTile + pos] = g01 * ur + g11 * us + g12 * ut;
        sW[2][c * kTcTile + pos] = g02 * ur + g12 * us + g22 * ut;
      }
    }
  }
  __syncwarp();

  // ---- transpose: w = sum_d D_d^T w_d; direction r writes its result over its own input tile
  // (after all four of its tiles are computed), s and t accumulate into it
  if (active) {
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      float* Out = sW[0] + c * kTcTile;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float* W = sW[d] + c * kTcTile;
        float cf[4][4];
#pragma unroll
        for (int T = 0; T < 4; ++T) {
          const int l0 = 16 * T + g, l1 = l0 + 8;
          if (d == 0) {
            cf[T][0] = cf[T][1] = cf[T][2] = cf[T][3] = 0.0f;
          } else {
            cf[T][0] = Out[tc_pos(d, l0, 2 * t4)];
            cf[T][1] = Out[tc_pos(d, l0, 2 * t4 + 1)];
            cf[T][2] = Out[tc_pos(d, l1, 2 * t4)];
            cf[T][3] = Out[tc_pos(d, l1, 2 * t4 + 1)];
          }
          const float av[4] = {W[tc_pos(d, l0, t4)], W[tc_pos(d, l1, t4)], W[tc_pos(d, l0, t4 + 4)],
                               W[tc_pos(d, l1, t4 + 4)]};
          mma3(cf[T], av, bth, btl);
        }
        __syncwarp();  // every lane has read its inputs before any result overwrites them
#pragma unroll
        for (int T = 0; T < 4; ++T) {
          const int l0 = 16 * T + g, l1 = l0 + 8;
          Out[tc_pos(d, l0, 2 * t4)] = cf[T][0];
          Out[tc_pos(d, l0, 2 * t4 + 1)] = cf[T][1];
          Out[tc_pos(d, l1, 2 * t4)] = cf[T][2];
          Out[tc_pos(d, l1, 2 * t4 + 1)] = cf[T][3];
        }
        __syncwarp();
      }
    }
  }

  // ---- w^e to the local output, (u^e, w^e) as an FP32 pair per lane
  dfloat dacc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) dacc[c] = dfloat{0.0f, 0.0f};
  if (active) {
    float* wl = a.wl + size_t(e) * kTcP3 * NC;
    for (int idx = lane; idx < kTcP3; idx += 32) {
      const int pos = tc_pad(idx & 7, (idx >> 3) & 7, idx >> 6);
      const bool skip = __ldg(l2g + idx) < 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float v = sW[0][c * kTcTile + pos];
        const float uv = sU[c * kTcTile + pos];
        if (!skip) wl[size_t(idx) * NC + c] = v;
        const float ph = __fmul_rn(v, uv);
        dacc[c] = dw_add(dacc[c], dfloat{ph, __fmaf_rn(v, uv, -ph)});
      }
    }
  }
  if (a.partials != nullptr) {
    double dot[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) dot[c] = df_to_f64(dacc[c]);
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

template <int NC>
size_t elem_tc_smem_bytes() {
  return sizeof(double) * 32 * NC + sizeof(float) * size_t(kTcWarps) * 4 * NC * kTcTile;
}

template <int NC>
cudaError_t launch_elem_tc_t(const DeviceMesh& m, const ElemLpArgs& a, cudaStream_t s) {
  const size_t smem = elem_tc_smem_bytes<NC>();
  static const cudaError_t attr =
      cudaFuncSetAttribute(elem_tc_kernel<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (attr != cudaSuccess) return attr;
  const int64_t blocks = (m.nelem + kTcWarps - 1) / kTcWarps;
  elem_tc_kernel<NC><<<unsigned(blocks), 32 * kTcWarps, smem, s>>>(m, a);
  return cudaGetLastError();
}

}  // namespace

bool elem_tc_supported(const DeviceMesh& m) { return m.colloc && m.p1 == kTcP1 && m.X == nullptr; }

cudaError_t launch_elem_tc(const DeviceMesh& m, const ElemLpArgs& a, cudaStream_t s) {
  if (!elem_tc_supported(m)) return cudaErrorInvalidValue;
  return m.ncomp == 3 ? launch_elem_tc_t<3>(m, a, s) : launch_elem_tc_t<1>(m, a, s);
}

}  // namespace ceedbp
