// Device helpers shared by the GB300 kernels: compensated (float-float)
// arithmetic, bounded mbarrier waits, 1D TMA bulk copies, binomials.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gw {

// Bits of the device status word (one 32-bit word in the context workspace).
enum : unsigned {
  ERR_TIMEOUT = 1u,    // a bounded wait gave up
  ERR_NONFINITE = 2u,  // a non-finite value reached an output
};

// Upper bound on the polls of one bounded wait before it gives up.  A healthy
// wait ends within a few thousand polls; 2^22 polls with a short sleep is
// about half a second.
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ void set_status(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// --------------------------------------------------------------------------
// Float-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2).  Used for the
// long carries across row bands, where plain float would lose digits in
// proportion to the number of bands.  Double precision uses plain double.
// --------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ ff ff_from_double(double d) {
  float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff ff_norm(float hi, float lo) {
  float s = __fadd_rn(hi, lo);
  return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_add(ff a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  return ff_norm(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// a * c with c a float (exact product error through fma).
__device__ __forceinline__ ff ff_mul(ff a, float c) {
  float p = __fmul_rn(a.hi, c);
  float e = __fmaf_rn(a.hi, c, -p);
  e = __fmaf_rn(a.lo, c, e);
  return ff_norm(p, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_norm(p, e);
}

__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Accumulator type for band carries: float-float for float data, double for
// double data.  acc_* give both the same interface.
template <typename Real> struct AccT;
template <> struct AccT<float> { using type = ff; };
template <> struct AccT<double> { using type = double; };

__device__ __forceinline__ ff acc_zero(ff*) { return {0.0f, 0.0f}; }
__device__ __forceinline__ double acc_zero(double*) { return 0.0; }
__device__ __forceinline__ ff acc_add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ double acc_sub(double a, double b) { return a - b; }
__device__ __forceinline__ ff acc_scale(ff a, float c) { return ff_mul(a, c); }
__device__ __forceinline__ double acc_scale(double a, double c) { return a * c; }
__device__ __forceinline__ ff acc_of(float x) { return ff_make(x); }
__device__ __forceinline__ ff acc_of(float hi, float lo) { return ff_norm(hi, lo); }
__device__ __forceinline__ double acc_of(double x) { return x; }
__device__ __forceinline__ double acc_of(double hi, double lo) { return hi + lo; }
__device__ __forceinline__ ff acc_shfl_down(ff a, int d) {
  return {__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ double acc_shfl_down(double a, int d) { return __shfl_down_sync(0xffffffffu, a, d); }
__device__ __forceinline__ ff acc_neg_of(ff a) { return ff_neg(a); }
__device__ __forceinline__ double acc_neg_of(double a) { return -a; }
__device__ __forceinline__ float acc_round(ff a) { return ff_to_float(a); }
__device__ __forceinline__ double acc_round(double a) { return a; }

// exp2 on the special-function unit (relative error about 2 ulp, subnormal
// results flushed to zero, which only drops terms below 2^-126 of a sum of
// terms bounded by 1).  The plan T = 2^(F_i + G_p - c Pi_ip) is formed with
// it wherever T is made from the potentials (the plan pass and the gradient
// kernels that read the plan from Pi), so every form gives the same values.
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double ex2(double x) { return exp2(x); }

// Binomial coefficient C(r, s) for small r (compile-time friendly).
__host__ __device__ constexpr int binom(int r, int s) {
  if (s < 0 || s > r) return 0;
  int v = 1;
  for (int i = 1; i <= s; ++i) v = v * (r - s + i) / i;
  return v;
}

__host__ __device__ constexpr int ipow(int b, int e) {
  int v = 1;
  for (int i = 0; i < e; ++i) v *= b;
  return v;
}

// --------------------------------------------------------------------------
// mbarrier + 1D bulk copy (TMA, non-tensor form) helpers.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and sets ERR_TIMEOUT)
// if the phase did not complete within kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* status) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    // Once any wait has given up, the results are already invalid: later
    // waits give up too (checked every 256 polls, so that short waits never
    // pay a global load) and the launch finishes quickly and reports.
    if ((it & 255u) == 255u && status && (*(volatile unsigned*)status & ERR_TIMEOUT)) return false;
    if (it >= 1024) __nanosleep(64);
  }
  set_status(status, ERR_TIMEOUT);
  return false;
}

// Global -> shared bulk copy completing on an mbarrier.  dst, src 16-byte
// aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// L2 prefetch of a global range (bulk, no shared memory involved).  addr and
// bytes 16-byte aligned.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src_gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src_gmem), "r"(bytes) : "memory");
}

}  // namespace gw
