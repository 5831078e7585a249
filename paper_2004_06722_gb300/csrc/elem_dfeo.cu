// FP32-pair BK5 element kernel with the even-odd decomposition of the 1D
// contractions (the centro-antisymmetry of Eq. (37), as in the FP64 kernel of
// elem_eo.cuh): every 1D pair product y = D x of a line becomes, for each
// mirror pair of outputs (i, p1-1-i), two half-length sums
//   S_E = sum_n E_in x+_n,  S_O = sum_n O_in x-_n,  y_i = S_E + S_O,  y_{p1-1-i} = S_O - S_E,
// so a pair-arithmetic line costs p1^2/2 pair products instead of p1^2.
//
// What makes the folds and unfolds cheap on pairs: before a stage, every value
// of the element is put on the grid of an element-wide power of two tau >= 2 max|x|
// (hi' = (hi + tau) - tau, the remainder moved into lo).  Then x+ = x_a + x_b and
// x- = x_a - x_b are exact in their hi parts (multiples of 2^-24 tau, at most
// tau in size), so a fold is two float additions.  S_E and S_O accumulate with
// one splitter sigma (SplitAcc, df.cuh), so their grid parts A - sigma are
// multiples of 2^-24 sigma of at most sigma/2 and S_E + S_O is again exact in
// its hi part: an unfold is four float additions for two outputs.  The
// bounds: sum_n |E_in| <= (1/2) sum_n |D_in| and |x+| <= 2 max|x|, so the
// splitter of the direct kernel (dnorm_row max|x|) bounds both half sums.
//
// Thread mapping: one thread per mirror octet of nodes (i, j, k < p1/2), so
// both outputs of every folded line product belong to the same thread (the
// layout of elem_eo.cuh).  Schedule: each slot of p1^3/8 threads works through
// a sequence of elements and fetches the next element's l2g and u by
// asynchronous copies while it computes the current one (the dependent
// l2g -> u gather is off the critical path); the next element's G is
// prefetched into L2 and read from global memory in the geometric stage
// (p1 <= 10), or copied into shared memory with u (p1 = 12).  The folded tiles
// of the three directions go through shared memory, and one loop body serves
// the three directions; the fused (u, w) dot and alpha are those of the direct
// pair kernels.  One component, even p1 (odd N), p1 = 4 .. 12; not used for
// batched launches (block tables).
#include <cuda_runtime.h>

#include <type_traits>

#include "elem_df.cuh"
#include "internal.h"
#include "kernel_args.h"

namespace ceedbp {

namespace {

// G of the element staged in shared memory by asynchronous copies (p1 >= 12), or read from global
// memory in the geometric stage after an L2 prefetch one element ahead (p1 <= 10: less than half
// the shared memory per slot, so more warps per SM; measured faster at p1 = 8, slower at 12)
template <int P1>
constexpr bool kDfeoStageG = P1 >= 12;

template <int P1>
struct DfeoShape {
  static constexpr int H = P1 / 2, H3 = H * H * H, PP = P1 * P1, P3 = PP * P1;
  // one sign of one direction's folded tile: PP lines of H pairs, line L at L*H + L/P1 (the skew
  // of one pair per P1 lines spreads the lines a warp reads over distinct banks)
  static constexpr int HALF = (PP * H + P1 + 1) / 2 * 2;
  static constexpr int TILE = 6 * HALF;  // r+, r-, s+, s-, t+, t-
  static constexpr int GSZ = kDfeoStageG<P1> ? 6 * P3 : 0;  // staged G of one element (pairs)
  static constexpr int USZ = 8 * H3;     // staged u of one element, [corner][octet] (8-byte cells)
  static constexpr int LSZ = 8 * H3;     // staged l2g of the next element, [corner][octet] (int32)
  static constexpr size_t SLOT_BYTES = sizeof(dfloat) * (TILE + GSZ + USZ) + sizeof(int) * ((LSZ + 3) / 4 * 4);
};

// layout: [red 32 doubles][smax 2 x 4 x 32 u32][E, O, Et, Ot: H x H pairs each], padded to 16 bytes,
// then eb slots of SLOT_BYTES: [folded tiles][G][u][l2g]
template <int P1>
__host__ __device__ constexpr size_t dfeo_head_bytes() {
  using S = DfeoShape<P1>;
  return (sizeof(double) * 32 + sizeof(unsigned) * 256 + sizeof(dfloat) * 4 * S::H * S::H + 15) / 16 * 16;
}

template <int P1>
size_t dfeo_smem_bytes(int eb) {
  return dfeo_head_bytes<P1>() + size_t(eb) * DfeoShape<P1>::SLOT_BYTES;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// x on the grid of tau (|x.hi| <= tau / 2): the hi part becomes a multiple of 2^-24 tau,
// the (exact) remainder moves into lo
__device__ __forceinline__ dfloat grid_align(dfloat x, float tau) {
  const float h = __fsub_rn(__fadd_rn(x.hi, tau), tau);
  return dfloat{h, __fadd_rn(x.lo, __fsub_rn(x.hi, h))};
}

// the two outputs (i, p1-1-i) of one folded line product from the half sums S_E, S_O
// (both accumulated with splitter sig): y_i = S_E + S_O, y_{p1-1-i} = S_O - S_E
__device__ __forceinline__ void eo_unfold(const SplitAcc& ae, const SplitAcc& ao, float sig, dfloat& y0,
                                          dfloat& y1) {
  const float xe = __fsub_rn(ae.A, sig), xo = __fsub_rn(ao.A, sig);
  const float le = __fadd_rn(ae.s, ae.c), lo = __fadd_rn(ao.s, ao.c);
  y0 = dfloat{__fadd_rn(xe, xo), __fadd_rn(le, lo)};
  y1 = dfloat{__fsub_rn(xo, xe), __fsub_rn(lo, le)};
}

// S_E, S_O of one line: coefficient rows ce, co (H pairs each), folded line xp, xm
template <int H>
__device__ __forceinline__ void eo_line(const dfloat* ce, const dfloat* co, const dfloat* xp, const dfloat* xm,
                                        SplitAcc& ae, SplitAcc& ao) {
#pragma unroll
  for (int n = 0; n < H; ++n) {
    const dfloat e = ce[n], od = co[n], p = xp[n], q = xm[n];
    ae.add(e.hi, e.lo, p.hi, p.lo);
    ao.add(od.hi, od.lo, q.hi, q.lo);
  }
}

// w += y with the hi parts summed by two_sum (their error into lo)
__device__ __forceinline__ void pair_accumulate(dfloat& w, dfloat y) {
  float s, e;
  two_sum(w.hi, y.hi, s, e);
  w = dfloat{s, __fadd_rn(__fadd_rn(w.lo, y.lo), e)};
}

template <int P1>
__device__ __forceinline__ int eo_node(int i, int j, int k, int bi, int bj, int bk) {
  const int ii = bi ? P1 - 1 - i : i, jj = bj ? P1 - 1 - j : j, kk = bk ? P1 - 1 - k : k;
  return ii + P1 * (jj + P1 * kk);
}

// Each slot (H^3 threads) works through a sequence of ns elements e = first + s eb + slot.
// Schedule of entry s (four barriers):
//   top:  wait for this thread's copies (u and G of entry s); copy l2g of entry s+1 (async)
//   A     maxima of |u|                   -> align and fold u
//   B     folded u tiles                  -> gradient, geometric factors (staged G)
//   D     maxima of |v|; tiles and G read -> copy u and G of entry s+1 (async); align and fold v
//   E     folded v tiles                  -> transpose, w^e, fused (u, w)
// Register cap: 128 at p1 = 8 (no spills; up to four 64-thread blocks per SM fit the shared memory
// anyway), 168 elsewhere (the odd half lengths and longer lines need more to stay spill-free).
template <int P1>
constexpr int kDfeoRegs = P1 == 8 ? 128 : 168;

template <int P1>
__global__ void __launch_bounds__(256) __maxnreg__(kDfeoRegs<P1>) elem_dfeo_kernel(const DeviceMesh m, const ElemDfArgs a, const int eb,
                                                          const int ns) {
  using S = DfeoShape<P1>;
  constexpr int H = S::H, H3 = S::H3, HALF = S::HALF, P3 = S::P3;
  extern __shared__ __align__(16) unsigned char smem_dfeo[];
  if (a.state != nullptr && a.state->stop) return;
  double* red = reinterpret_cast<double*>(smem_dfeo);        // 32
  unsigned* smax = reinterpret_cast<unsigned*>(red + 32);    // [2][4][32]: |u|, |v_r|, |v_s|, |v_t|
  dfloat* sE = reinterpret_cast<dfloat*>(smax + 256);        // [H][H] even part of D
  dfloat* sO = sE + H * H;                                   // odd part of D
  dfloat* sEt = sO + H * H;                                  // even part of D^T
  dfloat* sOt = sEt + H * H;                                 // odd part of D^T

  const int tid = threadIdx.x;
  const int slot = tid / H3, o = tid - slot * H3;
  const int i = o % H, j = (o / H) % H, k = o / (H * H);
  const bool in_slot = slot < eb;
  unsigned char* base = smem_dfeo + dfeo_head_bytes<P1>() + size_t(in_slot ? slot : 0) * S::SLOT_BYTES;
  dfloat* T = reinterpret_cast<dfloat*>(base);
  dfloat* sG = T + S::TILE;
  dfloat* sU = sG + S::GSZ;
  int* sL = reinterpret_cast<int*>(sU + S::USZ);

  const int64_t first = int64_t(blockIdx.x) * eb * ns;
  const auto elem_of = [&](int s) -> int64_t { return first + int64_t(s) * eb + slot; };
  const auto live = [&](int s) -> bool { return in_slot && s < ns && elem_of(s) < m.nelem; };

  // E, O of D and of D^T from the FP64 derivative table, as pairs
  {
    const double* D = m.basis + 2 * P1 * P1;
    for (int q = tid; q < H * H; q += blockDim.x) {
      const int r = q / H, c = q % H;
      const double d0 = D[r * P1 + c], d1 = D[r * P1 + (P1 - 1 - c)];
      const double t0 = D[c * P1 + r], t1 = D[(P1 - 1 - c) * P1 + r];
      const double v[4] = {0.5 * (d0 + d1), 0.5 * (d0 - d1), 0.5 * (t0 + t1), 0.5 * (t0 - t1)};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float hi = __double2float_rn(v[t]);
        sE[t * H * H + q] = dfloat{hi, __double2float_rn(v[t] - double(hi))};
      }
    }
    for (int q = tid; q < 256; q += blockDim.x) smax[q] = 0u;
  }

  // asynchronous copies of one entry: its l2g (own corners), u (own corners, 8-byte cells holding a
  // double or a pair) and G (the slot's threads in 16-byte pieces)
  const auto fetch_l2g = [&](int s) {
    const int* src = m.l2g + elem_of(s) * P3;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8)
      cp_async4(sL + c8 * H3 + o, src + eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2));
  };
  const auto fetch_u_g = [&](int s) {
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int g = sL[c8 * H3 + o];
      const int64_t gg = g < 0 ? -int64_t(g) - 1 : int64_t(g);
      const void* src = a.u_f64 != nullptr ? static_cast<const void*>(a.u_f64 + gg)
                                           : static_cast<const void*>(a.u_df + gg);
      cp_async8(sU + c8 * H3 + o, src);
    }
    if constexpr (kDfeoStageG<P1>) {
      const float4* gsrc = reinterpret_cast<const float4*>(a.G + elem_of(s) * 6 * P3);
      float4* gdst = reinterpret_cast<float4*>(sG);
      for (int q = o; q < 3 * P3; q += H3) cp_async16(gdst + q, gsrc + q);
    }
  };
  // the element's G (48 p1^3 bytes) into L2 in 128-byte lines, issued after the geometric stage
  // of the element before it (an element earlier measured slower at p1 = 8)
  const auto prefetch_g = [&](int s) {
    if constexpr (!kDfeoStageG<P1>) {
      const char* gsrc = reinterpret_cast<const char*>(a.G + elem_of(s) * 6 * P3);
      for (int q = o; q < 6 * P3 / 16; q += H3)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(gsrc + size_t(q) * 128));
    }
  };
  const auto dir_bits = [&]() -> unsigned {
    unsigned dm = 0u;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) dm |= unsigned(sL[c8 * H3 + o] < 0) << c8;
    return dm;
  };

  // prologue: l2g of entry 0, then its u and G
  unsigned dmask = 0u;
  if (live(0)) {
    fetch_l2g(0);
    cp_async_commit();
    cp_async_wait_all();
    dmask = dir_bits();
    prefetch_g(0);
    fetch_u_g(0);
  }
  cp_async_commit();
  __syncthreads();  // tables and maxima initialised

  // Direction-generic indexing.  For direction d (0 r, 1 s, 2 t) the octet's 8 values are held in
  // the d-local corner order l = b_d | b_{d+1} << 1 | b_{d+2} << 2 (cyclic; the r-local order is the
  // natural one, bit0 i, bit1 j, bit2 k).  The folded tile of d holds PP lines indexed by the mirrored
  // coordinates (a1, a2) of directions d+1, d+2 (line a2 * P1 + a1, at L*H + L/P1), positions along d.
  // Quadrant q = (b_{d+1}, b_{d+2}) of the octet then reads line q and owns the outputs l = 2q, 2q+1,
  // so one loop body serves all three directions.
  const auto lineoff = [&](int L) { return L * H + L / P1; };
  const auto coords = [&](int d, int& c0, int& c1, int& c2) {
    c0 = d == 0 ? i : (d == 1 ? j : k);
    c1 = d == 0 ? j : (d == 1 ? k : i);
    c2 = d == 0 ? k : (d == 1 ? i : j);
  };
  // fold the values x (d-local order) into the tile of direction d (D static)
  const auto fold_dir = [&](auto dc, const dfloat (&x)[8]) {
    constexpr int D = decltype(dc)::value;
    int c0, c1, c2;
    coords(D, c0, c1, c2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a1 = (q & 1) ? P1 - 1 - c1 : c1, a2 = (q >> 1) ? P1 - 1 - c2 : c2;
      const int L = lineoff(a2 * P1 + a1) + c0;
      const dfloat x0 = x[2 * q], x1 = x[2 * q + 1];
      T[(2 * D) * HALF + L] = dfloat{__fadd_rn(x0.hi, x1.hi), __fadd_rn(x0.lo, x1.lo)};
      T[(2 * D + 1) * HALF + L] = dfloat{__fsub_rn(x0.hi, x1.hi), __fsub_rn(x0.lo, x1.lo)};
    }
  };
  // d-local index of natural corner c8 for d = 1 (bits j, k, i) and d = 2 (bits k, i, j)
  const auto loc_s = [](int c8) { return ((c8 >> 1) & 1) | (((c8 >> 2) & 1) << 1) | ((c8 & 1) << 2); };
  const auto loc_t = [](int c8) { return ((c8 >> 2) & 1) | ((c8 & 1) << 1) | (((c8 >> 1) & 1) << 2); };

  double dot = 0.0;
  for (int s = 0; s < ns; ++s) {
    const bool active = live(s);
    const bool next_live = live(s + 1);
    unsigned* mx_s = smax + (s & 1) * 128;        // this entry's maxima
    unsigned* mx_o = smax + ((s & 1) ^ 1) * 128;  // the next entry's, reset during this one
    cp_async_wait_all();  // this thread's copies of u and G of entry s
    if (next_live) fetch_l2g(s + 1);
    cp_async_commit();

    // ---- u of this entry as pairs (own staged cells)
    dfloat u[8];
    float mx = 0.0f;
    if (active) {
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        const dfloat* cell = sU + c8 * H3 + o;
        dfloat v = a.u_f64 != nullptr ? f64_to_df(*reinterpret_cast<const double*>(cell)) : *cell;
        if (((dmask >> c8) & 1u) && a.mask_in) v = dfloat{0.0f, 0.0f};
        u[c8] = v;
        mx = fmaxf(mx, fabsf(v.hi));
      }
    }
    slot_max<H3>(&mx_s[slot], mx, active);
    __syncthreads();  // A
    if (in_slot && o == 0) {
      mx_o[slot] = 0u;
      mx_o[32 + slot] = 0u;
      mx_o[64 + slot] = 0u;
      mx_o[96 + slot] = 0u;
    }
    const float mu = __uint_as_float(mx_s[slot]);
    const float sig1 = splitter(a.dnorm_row * mu);
    if (active) {
      const float tau = splitter(mu);
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) u[c8] = grid_align(u[c8], tau);
      dfloat us[8], ut[8];
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        us[loc_s(c8)] = u[c8];
        ut[loc_t(c8)] = u[c8];
      }
      fold_dir(std::integral_constant<int, 0>{}, u);
      fold_dir(std::integral_constant<int, 1>{}, us);
      fold_dir(std::integral_constant<int, 2>{}, ut);
    }
    __syncthreads();  // B

    // ---- gradient: per direction 4 folded line products -> the 8 derivatives in d-local order
    //      (X0: r, X1: s, X2: t after the loop), then the geometric factors at the 8 nodes
    dfloat X0[8], X1[8], X2[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) X1[l] = X2[l] = dfloat{0.0f, 0.0f};
    float mr = 0.0f, ms = 0.0f, mt = 0.0f;
    if (active) {
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          X0[l] = X1[l];
          X1[l] = X2[l];
        }
        int c0, c1, c2;
        coords(d, c0, c1, c2);
        const dfloat* Tp = T + 2 * d * HALF;
        dfloat ce[H], co[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
          ce[n] = sE[c0 * H + n];
          co[n] = sO[c0 * H + n];
        }
        const int o1[2] = {c1 * H, (P1 - 1 - c1) * H};
        const int o2[2] = {c2 * (P1 * H + 1), (P1 - 1 - c2) * (P1 * H + 1)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int L = o2[q >> 1] + o1[q & 1];  // lineoff(a2 * P1 + a1)
          const dfloat xp0 = Tp[L], xm0 = Tp[HALF + L];
          SplitAcc ae = SplitAcc::first(sig1, ce[0].hi, ce[0].lo, xp0.hi, xp0.lo);
          SplitAcc ao = SplitAcc::first(sig1, co[0].hi, co[0].lo, xm0.hi, xm0.lo);
#pragma unroll
          for (int n = 1; n < H; ++n) {
            const dfloat xp = Tp[L + n], xm = Tp[HALF + L + n];
            ae.add(ce[n].hi, ce[n].lo, xp.hi, xp.lo);
            ao.add(co[n].hi, co[n].lo, xm.hi, xm.lo);
          }
          eo_unfold(ae, ao, sig1, X2[2 * q], X2[2 * q + 1]);
        }
      }
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        const int node = eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2);
        const int ls = loc_s(c8), lt = loc_t(c8);
        dfloat g[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if constexpr (kDfeoStageG<P1>) {
            g[q] = sG[q * P3 + node];
          } else {
            const float2 v = __ldg(reinterpret_cast<const float2*>(a.G + elem_of(s) * 6 * P3 + q * P3 + node));
            g[q] = dfloat{v.x, v.y};
          }
        }
        const float gb = fmaxf(fmaxf(row_abs_sum3(g[0], g[1], g[2]), row_abs_sum3(g[1], g[3], g[4])),
                               row_abs_sum3(g[2], g[4], g[5]));
        const dfloat ur = X0[c8], us = X1[ls], ut = X2[lt];
        const float um = fmaxf(fmaxf(fabsf(ur.hi), fabsf(us.hi)), fabsf(ut.hi));
        const float sg = splitter(gb * um);
        SplitAcc wr = SplitAcc::first(sg, g[0].hi, g[0].lo, ur.hi, ur.lo);
        wr.add(g[1].hi, g[1].lo, us.hi, us.lo);
        wr.add(g[2].hi, g[2].lo, ut.hi, ut.lo);
        SplitAcc ws = SplitAcc::first(sg, g[1].hi, g[1].lo, ur.hi, ur.lo);
        ws.add(g[3].hi, g[3].lo, us.hi, us.lo);
        ws.add(g[4].hi, g[4].lo, ut.hi, ut.lo);
        SplitAcc wq = SplitAcc::first(sg, g[2].hi, g[2].lo, ur.hi, ur.lo);
        wq.add(g[4].hi, g[4].lo, us.hi, us.lo);
        wq.add(g[5].hi, g[5].lo, ut.hi, ut.lo);
        X0[c8] = wr.result(sg);
        X1[ls] = ws.result(sg);
        X2[lt] = wq.result(sg);
        mr = fmaxf(mr, fabsf(X0[c8].hi));
        ms = fmaxf(ms, fabsf(X1[ls].hi));
        mt = fmaxf(mt, fabsf(X2[lt].hi));
      }
    }
    slot_max<H3>(&mx_s[32 + slot], mr, active);
    slot_max<H3>(&mx_s[64 + slot], ms, active);
    slot_max<H3>(&mx_s[96 + slot], mt, active);
    __syncthreads();  // D

    // every thread is past its reads of this entry's tiles and G: copy the next entry's u and G
    unsigned dmask_next = 0u;
    if (next_live) {
      cp_async_wait_all();  // its l2g
      dmask_next = dir_bits();
      prefetch_g(s + 1);
      fetch_u_g(s + 1);
    }
    cp_async_commit();

    const float vr = __uint_as_float(mx_s[32 + slot]), vs = __uint_as_float(mx_s[64 + slot]),
                vt = __uint_as_float(mx_s[96 + slot]);
    if (active) {
      const float tr = splitter(vr), ts = splitter(vs), tt = splitter(vt);
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        X0[l] = grid_align(X0[l], tr);
        X1[l] = grid_align(X1[l], ts);
        X2[l] = grid_align(X2[l], tt);
      }
      fold_dir(std::integral_constant<int, 0>{}, X0);
      fold_dir(std::integral_constant<int, 1>{}, X1);
      fold_dir(std::integral_constant<int, 2>{}, X2);
    }
    __syncthreads();  // E

    // ---- transpose: per direction 4 folded line products accumulated into w (held in the d-local
    //      order of the direction being added, moved to the next direction's order after each)
    if (active) {
      dfloat w[8];
#pragma unroll
      for (int l = 0; l < 8; ++l) w[l] = dfloat{0.0f, 0.0f};
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        const float sig = splitter(a.dnorm_col * (d == 0 ? vr : (d == 1 ? vs : vt)));
        int c0, c1, c2;
        coords(d, c0, c1, c2);
        const dfloat* Tp = T + 2 * d * HALF;
        dfloat ce[H], co[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
          ce[n] = sEt[c0 * H + n];
          co[n] = sOt[c0 * H + n];
        }
        const int o1[2] = {c1 * H, (P1 - 1 - c1) * H};
        const int o2[2] = {c2 * (P1 * H + 1), (P1 - 1 - c2) * (P1 * H + 1)};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int L = o2[q >> 1] + o1[q & 1];  // lineoff(a2 * P1 + a1)
          const dfloat xp0 = Tp[L], xm0 = Tp[HALF + L];
          SplitAcc ae = SplitAcc::first(sig, ce[0].hi, ce[0].lo, xp0.hi, xp0.lo);
          SplitAcc ao = SplitAcc::first(sig, co[0].hi, co[0].lo, xm0.hi, xm0.lo);
#pragma unroll
          for (int n = 1; n < H; ++n) {
            const dfloat xp = Tp[L + n], xm = Tp[HALF + L + n];
            ae.add(ce[n].hi, ce[n].lo, xp.hi, xp.lo);
            ao.add(co[n].hi, co[n].lo, xm.hi, xm.lo);
          }
          dfloat y0, y1;
          eo_unfold(ae, ao, sig, y0, y1);
          pair_accumulate(w[2 * q], y0);
          pair_accumulate(w[2 * q + 1], y1);
        }
        // d-local -> (d+1)-local: index bits (x0, x1, x2) -> (x1, x2, x0)
        dfloat t8[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) t8[(l >> 1) | ((l & 1) << 2)] = w[l];
#pragma unroll
        for (int l = 0; l < 8; ++l) w[l] = t8[l];
      }
      // w^e out, and the fused (u, w) over the octet with one splitter: |sum| <= 8 max|w| max|u|
      // (9 leaves room for the alignment of u and the rounding of the bound)
      dfloat* wl = a.wl + elem_of(s) * P3;
      float mw = 0.0f;
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        dfloat wn;
        two_sum(w[c8].hi, w[c8].lo, wn.hi, wn.lo);
        if (!(a.skip_dirichlet_out && ((dmask >> c8) & 1u)))
          wl[eo_node<P1>(i, j, k, c8 & 1, (c8 >> 1) & 1, c8 >> 2)] = wn;
        w[c8] = wn;
        mw = fmaxf(mw, fabsf(wn.hi));
      }
      const float sd = splitter(9.0f * mw * mu);
      SplitAcc acc = SplitAcc::first(sd, w[0].hi, w[0].lo, u[0].hi, u[0].lo);
#pragma unroll
      for (int c8 = 1; c8 < 8; ++c8) acc.add(w[c8].hi, w[c8].lo, u[c8].hi, u[c8].lo);
      dot += df_to_f64(acc.result(sd));
    }
    dmask = dmask_next;
  }
  cp_async_wait_all();

  if (a.partials != nullptr) {
    double v[1] = {dot};
    if (grid_sum_last<1>(v, a.partials, gridDim.x, blockIdx.x, &a.state->ticket[kTicketApply], red)) {
      if (threadIdx.x == 0) {
        SolveState* st = a.state;
        CompScalars& cs = st->c[0];
        if (cs.active) {
          const double pAp = v[0];
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

template <int P1>
bool dfeo_shape_ok(int eb) {
  const int nthreads = (eb * DfeoShape<P1>::H3 + 31) / 32 * 32;
  return eb >= 1 && eb <= 32 && nthreads <= 256 && dfeo_smem_bytes<P1>(eb) <= kMaxSmemPerBlock;
}

template <int P1>
cudaError_t launch_dfeo_p(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  using S = DfeoShape<P1>;
  const int eb = m.tune_eb > 0 ? m.tune_eb : 1;
  const int ns = m.tune_ns > 0 ? m.tune_ns : 8;
  if (!dfeo_shape_ok<P1>(eb)) return cudaErrorInvalidConfiguration;
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(elem_dfeo_kernel<P1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kMaxSmemPerBlock));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(elem_dfeo_kernel<P1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  const int64_t per_block = int64_t(eb) * ns;
  const int64_t blocks = (m.nelem + per_block - 1) / per_block;
  const int nthreads = (eb * S::H3 + 31) / 32 * 32;
  elem_dfeo_kernel<P1><<<unsigned(blocks), nthreads, dfeo_smem_bytes<P1>(eb), s>>>(m, a, eb, ns);
  return cudaGetLastError();
}

// (eb, ns) shapes the autotuner times: blocks of at least two warps' worth of octets, up to four
// times that, each with sequences of 4, 8 or 16 elements per slot
template <int P1>
int dfeo_candidates(int* eb, int* ns, int cap) {
  constexpr int H3 = DfeoShape<P1>::H3;
  const int e0 = H3 >= 64 ? 1 : 64 / H3;
  int n = 0;
  for (int e = e0; e <= 4 * e0 && n < cap; e *= 2) {
    if (!dfeo_shape_ok<P1>(e)) continue;
    for (int q = 4; q <= 16 && n < cap; q *= 2) {
      eb[n] = e;
      ns[n++] = q;
    }
  }
  return n;
}

}  // namespace

bool elem_dfeo_supported(const DeviceMesh& m) {
  return m.colloc && m.ncomp == 1 && m.p1 % 2 == 0 && m.p1 >= 4 && m.p1 <= 12;
}

int elem_dfeo_candidates(const DeviceMesh& m, int* eb, int* ns, int cap) {
  if (!elem_dfeo_supported(m)) return 0;
  switch (m.p1) {
    case 4: return dfeo_candidates<4>(eb, ns, cap);
    case 6: return dfeo_candidates<6>(eb, ns, cap);
    case 8: return dfeo_candidates<8>(eb, ns, cap);
    case 10: return dfeo_candidates<10>(eb, ns, cap);
    case 12: return dfeo_candidates<12>(eb, ns, cap);
    default: return 0;
  }
}

cudaError_t launch_elem_dfeo(const DeviceMesh& m, const ElemDfArgs& a, cudaStream_t s) {
  if (!elem_dfeo_supported(m) || a.blk_prob != nullptr) return cudaErrorInvalidValue;
  switch (m.p1) {
    case 4: return launch_dfeo_p<4>(m, a, s);
    case 6: return launch_dfeo_p<6>(m, a, s);
    case 8: return launch_dfeo_p<8>(m, a, s);
    case 10: return launch_dfeo_p<10>(m, a, s);
    case 12: return launch_dfeo_p<12>(m, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ceedbp
