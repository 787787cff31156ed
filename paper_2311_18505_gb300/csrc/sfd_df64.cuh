// Double-float arithmetic for the adjoint sweep (sfd_adjoint.cu): a value is
// the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about
// 48 significant bits.  On this GPU FP64 runs at a small fraction of the
// FP32 rate, so the adjoint recursion, which needs more than FP32 but not
// all of FP64, runs on the FP32 pipes instead: sums by Knuth's TwoSum and
// Dekker's FastTwoSum, products by the fused multiply-add error term
// (a b - fl(a b) exactly), reciprocals by one Newton step from the FP32
// reciprocal.  Every primitive uses the _rn intrinsics, so the compiler
// neither fuses nor reorders the error terms.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace sfd {
// In a namespace of its own, so that its fabs / fmax / shuffles are found by
// argument-dependent lookup for double-floats only and hide nothing that the
// FP32 kernels call unqualified.
namespace dfl {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(int v) : hi(static_cast<float>(v)), lo(0.f) {}
};

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// a + b = s + e exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return df64(s, e);
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator+(df64 a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  fast_two_sum(s, e, s, e);
  return df64(s, e);
}
__device__ __forceinline__ df64 operator+(float a, df64 b) { return b + a; }
__device__ __forceinline__ df64 operator-(df64 a, float b) { return a + (-b); }
__device__ __forceinline__ df64 operator-(float a, df64 b) { return (-b) + a; }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df64(s, e);
}

__device__ __forceinline__ df64 operator*(df64 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df64(s, e);
}
__device__ __forceinline__ df64 operator*(float a, df64 b) { return b * a; }

// The exact product of two floats as a double-float.
__device__ __forceinline__ df64 mul_ff(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df64(p, __fmaf_rn(a, b, -p));
}

// 1 / b: x0 ~ 1 / b.hi (the MUFU reciprocal, about 1 ulp; b is a normal
// float), then x0 + x0 (1 - b x0), relative error ~2^-46.
__device__ __forceinline__ df64 rcp_df(df64 b) {
  float x0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x0) : "f"(b.hi));
  const df64 r = 1.f - b * x0;
  return df64(x0) + r * x0;
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return a * rcp_df(b); }
__device__ __forceinline__ df64 operator/(df64 a, float b) { return a * rcp_df(df64(b)); }
__device__ __forceinline__ df64 operator/(float a, df64 b) { return rcp_df(b) * a; }

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// comparisons: by hi, then lo (both parts normalised)
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f) ? -a : a; }
__device__ __forceinline__ df64 fmax(df64 a, df64 b) { return a < b ? b : a; }
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }

// conversions with FP64 (segment boundaries and the host-facing results only)
__device__ __forceinline__ df64 df_from_double(double d) {
  const float h = static_cast<float>(d);
  return df64(h, static_cast<float>(d - static_cast<double>(h)));
}
__device__ __forceinline__ double to_double(df64 a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

// warp shuffles of both parts
__device__ __forceinline__ df64 shfl_up(df64 v, int s) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, s), __shfl_up_sync(0xffffffffu, v.lo, s));
}
__device__ __forceinline__ df64 shfl_down(df64 v, int s) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, s), __shfl_down_sync(0xffffffffu, v.lo, s));
}
__device__ __forceinline__ df64 shfl_xor(df64 v, int s) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, s), __shfl_xor_sync(0xffffffffu, v.lo, s));
}

}  // namespace dfl

using dfl::df64;
using dfl::df_from_double;

}  // namespace sfd
