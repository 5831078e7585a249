// Double-float arithmetic: a value is an unevaluated pair (hi, lo) of FP32
// numbers, hi + lo.  The GB300 issues FP32 FMAs about 63 times faster than
// FP64 ones, so FP64-accurate contractions run on pairs of FP32 numbers.
//
// Building blocks (Dekker 1971; Knuth TAOCP vol. 2; Joldes, Muller and Popescu,
// ACM TOMS 44(2), 2017):
//   two_sum         exact sum of two floats as a pair (6 flops)
//   fast_two_sum    same when |a| >= |b| (3 flops)
//   dw_add          pair + pair (Joldes et al., Alg. 5; 11 flops)
//   dw_mul          pair x pair (Joldes et al., Alg. 12 without the lo*lo term; 8 flops)
//
// Splitter accumulation: for a sum s = sum_n D_n x_n whose partial sums are
// bounded by B, pick sigma = 2^k >= 2B.  Then A = sigma + partial stays in
// [sigma/2, 3 sigma/2] where every float is a multiple of 2^-24 sigma; each step
// A' = fl(D x + A) rounds on that grid, the step A - A' is exact (a multiple of
// the grid below sigma in size) and fl(D x + (A - A')) recovers its rounding
// error to 2^-24 of one grid unit.  The exact grid part accumulates in A and
// the small parts in a plain float, 6 FP32 instructions per pair product
// instead of 12 for a two_sum-based pair dot (same idea as the error-free
// splitting of Rump, Ogita and Oishi, SIAM J. Sci. Comput. 31(1), 2008).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ceedbp {

struct __align__(8) dfloat {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat dw_add(dfloat x, dfloat y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(e, v);
  dfloat r;
  fast_two_sum(s, w, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfloat dw_mul(dfloat x, dfloat y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  float cl = __fmaf_rn(x.hi, y.hi, -ch);
  cl = __fmaf_rn(x.hi, y.lo, cl);
  cl = __fmaf_rn(x.lo, y.hi, cl);
  dfloat r;
  fast_two_sum(ch, cl, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfloat dw_neg(dfloat x) { return dfloat{-x.hi, -x.lo}; }

// FP64 -> pair without FP64 instructions: hi = x truncated to 24 significant
// bits (bit manipulation of the IEEE encoding), lo = the next 23 bits.  The
// pair represents x to 2^-46 relative; |x| < 2^-100 maps to (0, 0) and values
// beyond the float range are not supported (the operators here stay far inside).
__device__ __forceinline__ dfloat f64_to_df(double x) {
  const unsigned hw = static_cast<unsigned>(__double2hiint(x));
  const unsigned lw = static_cast<unsigned>(__double2loint(x));
  const unsigned sign = hw & 0x80000000u;
  const int e = static_cast<int>((hw >> 20) & 0x7ffu);
  dfloat r{0.0f, 0.0f};
  if (e <= 923) return r;  // |x| < 2^-100 (and zero)
  const unsigned mant23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  r.hi = __uint_as_float(sign | (static_cast<unsigned>(e - 896) << 23) | mant23);
  // remaining 29 mantissa bits r29, weight 2^(e-1075) each; keep the top 23:
  // F = 2^K (1 + (r29 >> 6) 2^-23) with K = e - 1046, lo = F - 2^K exactly.
  const unsigned r23 = (lw & 0x1fffffffu) >> 6;
  const int K = e - 1046;
  const float base = __uint_as_float(static_cast<unsigned>(K + 127) << 23);
  const float F = __uint_as_float((static_cast<unsigned>(K + 127) << 23) | r23);
  const float lo = __fsub_rn(F, base);
  r.lo = sign ? -lo : lo;
  return r;
}

__device__ __forceinline__ double df_to_f64(dfloat v) {
  return __dadd_rn(static_cast<double>(v.hi), static_cast<double>(v.lo));
}

// Smallest power of two >= 2 b (b >= 0), at least 2^-100.
__device__ __forceinline__ float splitter(float b) {
  b = fmaxf(__fmul_rn(b, 2.0f), 7.8886091e-31f);
  const unsigned bits = (__float_as_uint(b) + 0x007fffffu) & 0x7f800000u;
  return __uint_as_float(bits);
}

// Accumulator of sum D x over pairs with a fixed splitter sigma.  The grid
// part accumulates in A, the rounding errors of the grid steps in s and the
// cross terms dh*xl + dl*xh in c (separate chains keep the dependency depth
// at two instructions per term).
struct SplitAcc {
  float A, s, c;
  __device__ __forceinline__ explicit SplitAcc(float sigma) : A(sigma), s(0.0f), c(0.0f) {}
  // += (dh + dl)(xh + xl), dropping dl*xl
  __device__ __forceinline__ void add(float dh, float dl, float xh, float xl) {
    const float an = __fmaf_rn(dh, xh, A);
    const float d = __fsub_rn(A, an);
    s = __fadd_rn(s, __fmaf_rn(dh, xh, d));
    c = __fmaf_rn(dh, xl, c);
    c = __fmaf_rn(dl, xh, c);
    A = an;
  }
  __device__ __forceinline__ dfloat result(float sigma) const {
    return dfloat{__fsub_rn(A, sigma), __fadd_rn(s, c)};
  }
  // The accumulator after its first term: the sums of SplitAcc(sigma) followed by add(), less the
  // additions of zero (which IEEE signed zeros keep the compiler from removing); equal results up
  // to the sign of a zero.
  __device__ __forceinline__ static SplitAcc first(float sigma, float dh, float dl, float xh, float xl) {
    SplitAcc r(sigma);
    const float an = __fmaf_rn(dh, xh, sigma);
    r.s = __fmaf_rn(dh, xh, __fsub_rn(sigma, an));
    r.c = __fmaf_rn(dl, xh, __fmul_rn(dh, xl));
    r.A = an;
    return r;
  }
};

// ---- bulk asynchronous copy global -> shared with an mbarrier (Blackwell TMA unit)
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// bytes: multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ---- per-thread asynchronous copies global -> shared (no registers in flight)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bounded wait on phase `parity` of an mbarrier: returns false after `limit`
// polls (each try_wait may itself suspend the thread for a short while).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace ceedbp
