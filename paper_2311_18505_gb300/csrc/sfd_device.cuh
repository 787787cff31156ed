// Device helpers shared by the step kernels: warp tridiagonal partition
// solver on shared-memory rows, reductions, point interpolation and the bow
// friction root.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sfd_df64.cuh"
#include "sfd_types.h"

namespace sfd {

#define SFD_FULL 0xffffffffu

// whole-warp shuffles by precision (the templated solvers below; df64 in
// sfd_df64.cuh)
__device__ __forceinline__ float shfl_up(float v, int s) { return __shfl_up_sync(SFD_FULL, v, s); }
__device__ __forceinline__ float shfl_down(float v, int s) { return __shfl_down_sync(SFD_FULL, v, s); }
__device__ __forceinline__ double shfl_up(double v, int s) { return __shfl_up_sync(SFD_FULL, v, s); }
__device__ __forceinline__ double shfl_down(double v, int s) { return __shfl_down_sync(SFD_FULL, v, s); }

template <class T>
struct RedT {          // per-lane factors of the reduced (lane-boundary) system
  T k1[5], k2[5];
  T binv, cl;
  int nlev;            // cyclic-reduction levels kept (warp-uniform)
};
using Red = RedT<float>;

// Reciprocal for the eliminations: one MUFU instruction (rcp.approx.ftz,
// about 1 ulp) instead of the IEEE sequence with its slow-path branch.  The
// pivots are O(1) (the systems are strictly diagonally dominant), so
// flushing subnormals never applies; the solves then carry FP32-rounding
// sized errors, which scale with the small accelerations being solved for.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Cyclic reduction stops once every lane's remaining off-diagonal coupling
// is below this fraction of its diagonal: the reduced system is then
// diagonal to FP32 precision (a strictly diagonally dominant tridiagonal
// squares its coupling ratio at every level).
constexpr float kPcrDrop = 7.4505806e-9f;   // 2^-27

// reciprocal and reduction cut-off per precision (the FP64 instances serve
// the adjoint sweep)
__device__ __forceinline__ float rcp_of(float x) { return fast_rcp(x); }
__device__ __forceinline__ double rcp_of(double x) { return 1.0 / x; }
__device__ __forceinline__ df64 rcp_of(df64 x) { return rcp_df(x); }
__device__ __forceinline__ float pcr_drop(float) { return kPcrDrop; }
__device__ __forceinline__ double pcr_drop(double) { return 8.673617379884035e-19; }   // 2^-60
__device__ __forceinline__ float pcr_drop(df64) { return 7.105427357601002e-15f; }     // 2^-47

// ----------------------------------------------------------------------------
// Tridiagonal partition solver on a warp.  Row i: a_i x_{i-1} + b_i x_i +
// c_i x_{i+1} = d_i.  On entry SUB = a, INV = b, CP = c for the lane's rows;
// on exit INV = 1/pivot, CP = c', AL = coefficient of the previous lane's last
// unknown, FF/GG = back-substitution weights of the lane's last unknown and
// the previous lane's last unknown.
// ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void tri_factor(const T* __restrict__ SUB, T* __restrict__ INV, T* __restrict__ CP,
                                           T* __restrict__ AL, T* __restrict__ FF, T* __restrict__ GG, int m,
                                           int lane, RedT<T>& rd) {
  const int base = lane * m;
  T cprev = 0, alprev = 0;
  for (int r = 0; r < m; ++r) {
    const int i = base + r;
    const T a = SUB[i], b = INV[i], c = CP[i];
    T inv, al;
    if (r == 0) {
      inv = rcp_of(b);
      al = a * inv;
    } else {
      inv = rcp_of(b - a * cprev);
      al = -a * alprev * inv;
    }
    const T cp = c * inv;
    INV[i] = inv;
    CP[i] = cp;
    AL[i] = al;
    cprev = cp;
    alprev = al;
  }
  T f = 1, g = 0;
  FF[base + m - 1] = 1;
  GG[base + m - 1] = 0;
  for (int r = m - 2; r >= 0; --r) {
    const int i = base + r;
    const T cp = CP[i];
    f = -cp * f;
    g = -AL[i] - cp * g;
    FF[i] = f;
    GG[i] = g;
  }
  T f0n = shfl_down(FF[base], 1);
  T g0n = shfl_down(GG[base], 1);
  if (lane == kWarp - 1) { f0n = 0; g0n = 0; }
  const T cl = CP[base + m - 1];
  T A = AL[base + m - 1];
  T B = 1 + cl * g0n;
  T C = cl * f0n;
  rd.cl = cl;
  rd.nlev = 5;
#pragma unroll
  for (int l = 0; l < 5; ++l) { rd.k1[l] = 0; rd.k2[l] = 0; }
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    if (__all_sync(SFD_FULL, fabs(A) + fabs(C) <= pcr_drop(T(0)) * fabs(B))) { rd.nlev = l; break; }
    const int s = 1 << l;
    T Am = shfl_up(A, s), Bm = shfl_up(B, s);
    T Cm = shfl_up(C, s);
    T Ap = shfl_down(A, s), Bp = shfl_down(B, s);
    T Cp = shfl_down(C, s);
    if (lane < s) { Am = 0; Bm = 1; Cm = 0; }
    if (lane + s >= kWarp) { Ap = 0; Bp = 1; Cp = 0; }
    const T k1 = A * rcp_of(Bm), k2 = C * rcp_of(Bp);
    A = -Am * k1;
    C = -Cp * k2;
    B = B - Cm * k1 - Ap * k2;
    rd.k1[l] = k1;
    rd.k2[l] = k2;
  }
  rd.binv = rcp_of(B);
}

// Solve in place: E holds d for the lane's rows on entry and x on exit.
template <class T>
__device__ __forceinline__ void tri_solve(const T* __restrict__ SUB, const T* __restrict__ INV,
                                          const T* __restrict__ CP, const T* __restrict__ FF,
                                          const T* __restrict__ GG, T* __restrict__ E, int m, int lane,
                                          const RedT<T>& rd) {
  const int base = lane * m;
  T dp = 0;
  for (int r = 0; r < m; ++r) {
    const int i = base + r;
    const T v = (r == 0) ? E[i] : E[i] - SUB[i] * dp;
    dp = v * INV[i];
    E[i] = dp;
  }
  const T dlast = dp;
  T e = 0;
  E[base + m - 1] = 0;
  for (int r = m - 2; r >= 0; --r) {
    const int i = base + r;
    e = E[i] - CP[i] * e;
    E[i] = e;
  }
  T e0n = shfl_down(E[base], 1);
  if (lane == kWarp - 1) e0n = 0;
  T D = dlast - rd.cl * e0n;
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    if (l >= rd.nlev) break;      // the factorisation dropped the remaining levels (warp-uniform)
    const int s = 1 << l;
    T Dm = shfl_up(D, s);
    T Dp = shfl_down(D, s);
    if (lane < s) Dm = 0;
    if (lane + s >= kWarp) Dp = 0;
    D = D - rd.k1[l] * Dm - rd.k2[l] * Dp;
  }
  const T X = D * rd.binv;
  T Xp = shfl_up(X, 1);
  if (lane == 0) Xp = 0;
  for (int r = 0; r < m; ++r) {
    const int i = base + r;
    E[i] = E[i] + FF[i] * X + GG[i] * Xp;
  }
}

// Stopping rule of the coupled Gauss-Seidel solve, from the largest
// relative change e of the latest sweep and e_prev of the one before:
// converged when e is below the tolerance, when the change predicted for
// the next sweep (e^2 / e_prev for a linear contraction) is, or when the
// change has stopped shrinking at the FP32 noise floor.
__device__ __forceinline__ bool sweep_converged(float e, float e_prev, int sweep) {
  if (e <= kSweepTol) return true;
  if (sweep >= 2 && e < e_prev && e * e <= kSweepTol * e_prev) return true;
  if (sweep >= 3 && e >= 0.5f * e_prev && e <= 64.f * kSweepTol) return true;
  return false;
}

__device__ __forceinline__ float warp_max_nonneg(float v) {
  // non-negative floats order like their bit patterns
  return __uint_as_float(__reduce_max_sync(SFD_FULL, __float_as_uint(v)));
}

// Value of a transverse-node field at nodes `node` and `node + 1` with weight w
// on the second (linear interpolation I(x), Sec. 3.3); rows are node - 1 and the
// fixed ends read the zero guard cells.
__device__ __forceinline__ float interp2(const float* __restrict__ A, int node, float w) {
  return (1.f - w) * A[node - 1] + w * A[node];
}

// The same interpolation on the longitudinal grid (nodes 0..N_l, rows
// node - 1): the fixed ends and rows past n_z read zero.
__device__ __forceinline__ float zinterp(const float* __restrict__ A, int node, float w, int n_z) {
  const float a = (node >= 1 && node - 1 < n_z) ? A[node - 1] : 0.f;
  const float b = (node >= 0 && node < n_z) ? A[node] : 0.f;
  return (1.f - w) * a + w * b;
}

// Wave-speed factor rm = (gamma^n / gamma)^2 of the step from level n
// (reading A14), which scales every gamma^2 term.  Vibrato: 2^{(2c/1200)
// sin(2 pi t)} with the phase t = frac(n f_v k + phi / 2 pi) kept as a 64-bit
// fixed-point fraction, where the integer product's wrap-around is the
// fractional part (exact for any n, and no FP64 arithmetic, which runs at a
// small fraction of the FP32 rate on this GPU, enters the step); glissando:
// 2^{2 D min(n k, T) / T}, i.e. held at 2^{2D} from step n_end on.
__device__ __forceinline__ float mod_factor(int kind, uint64_t inc_fx, uint64_t phase_fx, float depth2,
                                            float inc, float hold, int64_t n_end, int64_t n) {
  if (kind == 1) {
    const uint64_t t_fx = static_cast<uint64_t>(n) * inc_fx + phase_fx;
    const float t = static_cast<float>(static_cast<uint32_t>(t_fx >> 40)) * 5.9604644775390625e-8f;   // 2^-24
    // sin(2 pi t) = -sin(2 pi (t - 1/2)), whose argument lies in [-pi, pi):
    // there the hardware sine's absolute error is ~2^-21, i.e. ~1e-8 in rm
    return exp2f(-depth2 * __sinf(6.28318530717958647f * (t - 0.5f)));
  }
  if (kind == 2) return exp2f(n < n_end ? inc * static_cast<float>(n) : hold);
  return 1.f;
}

// Bow controls of step n from the descriptor's breakpoint envelopes
// (breakpoints in steps): linear between breakpoints, the first or last
// value outside them; x is the bow position, from which the step's
// interpolation node and weight (node, w) follow as for a fixed point.
__device__ __forceinline__ void bow_env_eval(const Desc* __restrict__ D, int64_t n, float& v, float& f, int& node,
                                             float& w) {
  const int m = D->bow_env_n;
  const double t = static_cast<double>(n);
  double x;
  if (m == 1 || t <= D->bow_env_t[0]) {
    v = D->bow_env_v[0]; f = D->bow_env_f[0]; x = D->bow_env_x[0];
  } else if (t >= D->bow_env_t[m - 1]) {
    v = D->bow_env_v[m - 1]; f = D->bow_env_f[m - 1]; x = D->bow_env_x[m - 1];
  } else {
    int j = 0;
    while (j + 1 < m - 1 && t >= D->bow_env_t[j + 1]) ++j;
    const double r = (t - D->bow_env_t[j]) / (D->bow_env_t[j + 1] - D->bow_env_t[j]);
    v = static_cast<float>(D->bow_env_v[j] + r * (static_cast<double>(D->bow_env_v[j + 1]) - D->bow_env_v[j]));
    f = static_cast<float>(D->bow_env_f[j] + r * (static_cast<double>(D->bow_env_f[j + 1]) - D->bow_env_f[j]));
    x = D->bow_env_x[j] + r * (static_cast<double>(D->bow_env_x[j + 1]) - D->bow_env_x[j]);
  }
  const double pos = x * D->n_t;
  int l = static_cast<int>(floor(pos));
  l = l < 0 ? 0 : (l > D->n_t - 1 ? D->n_t - 1 : l);
  node = l;
  w = static_cast<float>(pos - l);
}

// Bow friction: solve v + c phi(v) = b with phi(v) = sign(v)(eps + (1-eps)
// e^{-a|v|}) (Sec. 3.3.1, Eq. 5).  Sticking (v = 0, phi = b/c) whenever
// |b| <= c; otherwise the root of the convex g(w) = w + c phi(w) - |b| on
// (0, |b|).  Newton from a point right of the root decreases monotonically
// for a convex g increasing there, so it stops as soon as an iterate fails
// to decrease (the root within FP32 rounding).  The start is the previous
// slip speed w_warm when it lies right of the root, its tangent root when it
// lies left (right of the root by convexity), else |b|; w_warm is updated.
__device__ __forceinline__ float bow_phi(float b, float c, float a, float eps, float& w_warm) {
  if (!(c > 0.f)) {
    const float w = fabsf(b);
    return b == 0.f ? 0.f : copysignf(eps + (1.f - eps) * expf(-a * w), b);
  }
  if (fabsf(b) <= c) return __fdividef(b, c);   // |b| <= c, c > 0: within 2 ulp
  const float B = fabsf(b);
  const float a2 = a * 1.44269504088896341f;   // e^{-a w} = 2^{-a2 w}
  const float ce = c * (1.f - eps), c0 = c * eps - B;
  float w = B;
  if (w_warm > 0.f && w_warm < B) {
    const float ex = exp2f(-a2 * w_warm);
    const float g = w_warm + c0 + ce * ex;
    const float dg = 1.f - ce * a * ex;
    if (g >= 0.f) w = w_warm;
    else if (dg > 0.f) w = fminf(w_warm - __fdividef(g, dg), B);
  }
  for (int it = 0; it < 32; ++it) {
    const float ex = exp2f(-a2 * w);
    const float g = w + c0 + ce * ex;
    const float dg = 1.f - ce * a * ex;
    if (!(g > 0.f) || !(dg > 0.f)) break;
    const float wn = fmaxf(w - __fdividef(g, dg), 0.f);
    if (!(wn < w)) break;
    w = wn;
  }
  w_warm = w;
  return copysignf(eps + (1.f - eps) * expf(-a * w), b);
}

}  // namespace sfd
