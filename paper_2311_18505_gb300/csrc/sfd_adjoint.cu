// Discrete adjoint of the string time-stepping (gradients of a waveform loss;
// the paper has no counterpart: its synthesizer only renders).
//
// One step n -> n+1 of the scheme of Eq. 4 (as stepped by the forward kernel,
// transverse line scaled by beta, see fill_desc) solves the linear system
//   R(x, w) = 0,  w = (a, az, s):
//   R1 = RHS_u(x) + cb B az + J s - A_u(g) a
//   R2 = RHS_z(x) + cz C a      - A_z az
//   R3 = M G eta - (M G / 2) I a - (1 + G / 2) s               (hammer, Eq. 6)
// with x = (u, D, z, Dz, u_H, D_H) at level n, g = d_- u, e = d_- P z,
//   RHS_u = lam2 d2 u - mu2 d4 u - 2 s0u D + 2 s1 d2 D + d_+[2 ca g^3 + 4 cb g e]
//   RHS_z = lam2l d2 z - 2 s0 Dz + 2 s1l d2 Dz + 2 cz P^T d_+[g^2]
//   A_u(g) = dg I + og (shifts) - d_+[ca g^2 d_-],  A_z = (1 + s0) I - s1l d2,
//   B = d_+ g d_- P,  C = P^T d_+ g d_- = B^T,  G = k^2 w_H^{1+a_H} [eta]_+^{a_H-1},
//   eta = u_H - I u, and advances D+ = D + a, u+ = u + D+, likewise z, and
//   D_H+ = D_H - s / M, u_H+ = u_H + D_H+.
//
// Reverse step, given the adjoint L of level n+1 (plus dJ/dy of that level's
// output sample):
//   mu = (L_D + L_u, L_Dz + L_z, -(L_DH + L_uH) / M)   (adjoint of w)
//   M^T nu = mu        (M = -dR/dw, the step's matrix)
//   L_n = (dx+/dx)^T L + (dR/dx)^T nu,   dJ/dc += (dR/dc)^T nu
// M^T is M with cb and cz exchanged and the hammer row and column scaled, so
// nu is found by the forward block Gauss-Seidel solve of M (nu_a, nz, st) =
// (mu_a, (cz/cb) mu_z, -(M G / (2 js)) mu_s), nu_z = (cb/cz) nz,
// nu_s = -(2 js / (M G)) st  (js: the spreading scale of J).
//
// The states of the segment's levels come from a replay of the forward
// kernel from a checkpoint (Job::traj), so the adjoint is that of the FP32
// trajectory the forward produced.  One block of four warps per string
// (one per SM sub-partition), every per-row array in shared memory: the row
// loops are spread over the block's threads, the partitioned tridiagonal
// solves run on warp 0 (lane partitions and cyclic reduction over its
// shuffles) between block barriers.
//
// The adjoint recursion runs in double-float arithmetic (sfd_df64.cuh,
// ~48 bits; the trajectory stays FP32): nu carries a large smooth part, and
// its FP32 representation noise, amplified by the second and fourth
// differences, enters L_u every step; after a few hundred steps that noise
// dominates the adjoint's high-wavenumber content, which is exactly what the
// kappa and sigma1 gradients weight (measured: 2-15 % errors against the
// oracle's gradient in FP32, none in FP64).  FP64 itself, at a small
// fraction of the FP32 rate on this GPU, left each string's warp waiting on
// the FP64 pipe; double-floats run on the FP32 pipes, and converting the
// FP32 trajectory to them is free.  FP64 remains only at the segment
// boundaries (the adjoint state kept between launches, the gradients) and
// in the hammer's power law and the bow's friction exponential.
#include <cuda_runtime.h>

#include <mutex>

#include "sfd_device.cuh"

namespace sfd {

namespace {

using R = df64;
constexpr float kAdjTol = 1e-13f;   // relative change that ends an adjoint block Gauss-Seidel solve
constexpr int kAdjSweeps = 40;
constexpr int kAdjWarps = 4;          // warps per string (one per SM sub-partition)
constexpr int kAdjThreads = kAdjWarps * kWarp;

// (the change measures e are float: they only decide when to stop)
__device__ __forceinline__ bool adj_converged(float e, float e_prev, int sweep) {
  if (e <= kAdjTol) return true;
  if (sweep >= 2 && e < e_prev && e * e <= kAdjTol * e_prev) return true;
  if (sweep >= 3 && e >= 0.5f * e_prev && e <= 64.f * kAdjTol) return true;
  return sweep >= kAdjSweeps;
}

}  // namespace

__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_kernel(const AdjJob* __restrict__ jobs, int n_jobs) {
  extern __shared__ double smem_d[];
  __shared__ float red[2][2][kAdjWarps];   // block maxima of the sweep's change measures (two buffers)
  __shared__ R gsum[kAdjWarps][kGradSlots];   // per-warp gradient sums
  const int tid = threadIdx.x, lane = tid & (kWarp - 1), warp = tid >> 5;
  if (static_cast<int>(blockIdx.x) >= n_jobs) return;
  const AdjJob J = jobs[blockIdx.x];
  const Desc* __restrict__ Dp = J.desc;
  const int n_t = Dp->n_t, n_l = Dp->n_l, n_u = Dp->n_u, n_z = Dp->n_z;
  const int m_u = Dp->m_u, m_z = Dp->m_z;
  const bool has_z = m_z > 0;
  const bool linear = Dp->linear != 0;
  const bool hammer = Dp->exc == kHammer;
  const int RU = kWarp * m_u + 4, RZ = has_z ? kWarp * m_z + 4 : 0;
  const R dg = Dp->dg, og = Dp->og, s0 = Dp->s0, s0u = Dp->s0u, s1 = Dp->s1, s1l = Dp->s1l;
  const R mu2 = Dp->mu2;
  // the gamma^2 coefficients of the step being reversed: with f0 modulation
  // the forward scales them by rm = (gamma^n / gamma)^2 each step, and they
  // are formed here from the same FP32 expressions (so the adjoint is that
  // of the forward's own arithmetic); rmd carries rm into the gradients of
  // the unscaled coefficients
  const float lam2_0f = Dp->lam2, lam2lo_0f = Dp->lam2_lo, lam2l_0f = Dp->lam2l;
  const float ca_0f = Dp->ca, cb_0f = Dp->cb, cz_0f = Dp->cz;
  const int mod_kind = Dp->mod_kind;
  const float mod_depth2 = Dp->mod_depth2;
  R lam2 = static_cast<R>(lam2_0f) + static_cast<R>(lam2lo_0f), lam2l = lam2l_0f;
  R ca = ca_0f, cb = cb_0f, cz = cz_0f, rmd = 1.0f;
  const R bsgn = Dp->boundary == 1 ? -1.0f : 1.0f;
  const int en = Dp->e_node, on = Dp->o_node;
  const R ew = Dp->e_w, js = Dp->jscale, ow = Dp->o_w, oscale = Dp->out_scale;
  const bool zout = Dp->out_ch == 1;   // output reads zeta on the longitudinal grid
  const int oln = Dp->ol_node;
  const R olw = Dp->ol_w;
  const R hM = Dp->ham_M, hk2w = Dp->ham_k2w, hexpo = Dp->ham_expo;
  const bool bow = Dp->exc == kBow;
  const R bF = Dp->bow_F, ba = Dp->bow_a, beps = Dp->bow_eps, kk = Dp->k;
  const int64_t brel = Dp->bow_release_n;

  // ---- shared memory: FP64 adjoint arrays, then the FP32 trajectory ----
  R* const rbase = reinterpret_cast<R*>(smem_d);   // double-floats: 8 bytes, as the FP64 slots
  R* pd = rbase;
  auto DU_ = [&]() { R* a = pd + 2; pd += RU; return a; };
  R *LU = DU_(), *LD = DU_(), *NA = DU_(), *RA = DU_(), *SUB = DU_(), *INV = DU_(), *CP = DU_(), *AL = DU_();
  R *FF = DU_(), *GG = DU_(), *XP = DU_(), *FT = DU_(), *PNZ = DU_(), *GAM = DU_(), *PSG = DU_(), *XZT = DU_();
  R* T1 = DU_();
  R *LZ = nullptr, *LDZ = nullptr, *NZ = nullptr, *RZ_ = nullptr, *SUBZ = nullptr, *INVZ = nullptr, *CPZ = nullptr;
  R *ALZ = nullptr, *FFZ = nullptr, *GGZ = nullptr, *E1Z = nullptr, *XZ = nullptr, *T2 = nullptr;
  if (has_z) {
    auto DZ_ = [&]() { R* a = pd + 2; pd += RZ; return a; };
    LZ = DZ_(); LDZ = DZ_(); NZ = DZ_(); RZ_ = DZ_(); SUBZ = DZ_(); INVZ = DZ_(); CPZ = DZ_(); ALZ = DZ_();
    FFZ = DZ_(); GGZ = DZ_(); E1Z = DZ_(); XZ = DZ_(); T2 = DZ_();
  }
  float* pf = reinterpret_cast<float*>(pd);
  auto FU_ = [&]() { float* a = pf + 2; pf += RU; return a; };
  float *U = FU_(), *DU = FU_(), *DN1 = FU_(), *A = FU_(), *G = FU_(), *ZT = FU_(), *AZT = FU_();
  int* TMI = reinterpret_cast<int*>(FU_());
  float* TMW = FU_();
  float *Z = nullptr, *DZ = nullptr, *DZN1 = nullptr, *AZ = nullptr;
  int *ZLO = nullptr, *ZHI = nullptr;
  if (has_z) {
    auto FZ_ = [&]() { float* a = pf + 2; pf += RZ; return a; };
    Z = FZ_(); DZ = FZ_(); DZN1 = FZ_(); AZ = FZ_();
    ZLO = reinterpret_cast<int*>(FZ_());
    ZHI = reinterpret_cast<int*>(FZ_());
  }
  {
    const int nd = static_cast<int>(pd - rbase);
    for (int k = tid; k < nd; k += kAdjThreads) smem_d[k] = 0.0f;
    float* f0 = reinterpret_cast<float*>(smem_d + nd);
    const int nf = static_cast<int>(pf - f0);
    for (int k = tid; k < nf; k += kAdjThreads) f0[k] = 0.f;
  }
  __syncthreads();

  // grid transfer P (longitudinal -> transverse nodes) and P^T, as the forward
  if (has_z) {
    for (int i = tid; i < n_u; i += kAdjThreads) {
      const int pos = (i + 1) * n_l;
      const int mm = pos / n_t;
      TMI[i] = mm;
      TMW[i] = static_cast<float>(pos - mm * n_t) / static_cast<float>(n_t);
    }
    for (int i = tid; i < n_z; i += kAdjThreads) {
      const int mm = i + 1;
      const int lo = ((mm - 1) * n_t) / n_l + 1;
      const int hi = ((mm + 1) * n_t + n_l - 1) / n_l - 1;
      ZLO[i] = lo < 1 ? 1 : lo;
      ZHI[i] = hi > n_t - 1 ? n_t - 1 : hi;
    }
  }
  __syncthreads();
  const R inv_nt = 1.0f / static_cast<R>(n_t);
  auto interp_z = [&](const auto* X, int i) -> R {
    const int mm = TMI[i];
    const R w = TMW[i];
    return (1.0f - w) * static_cast<R>(X[mm - 1]) + w * static_cast<R>(X[mm]);
  };
  auto spread = [&](const R* F, int i) -> R {
    const int mm = i + 1, lo = ZLO[i], hi = ZHI[i];
    R acc = 0.0f;
    for (int l = lo; l <= hi; ++l) {
      const int dd = l * n_l - mm * n_t;
      const R w = 1.0f - static_cast<R>(dd < 0 ? -dd : dd) * inv_nt;
      acc = fma(fmax(w, 0.0f), F[l - 1], acc);
    }
    return acc;
  };
  // second and fourth differences (the fourth with the boundary ghost)
  auto d2_of = [&](const auto* X, int i) -> R {
    return (static_cast<R>(X[i + 1]) - X[i]) - (static_cast<R>(X[i]) - X[i - 1]);
  };
  auto d4_of = [&](const R* X, int i) -> R {
    const R gl = X[i] - X[i - 1], gr = X[i + 1] - X[i];
    R d4 = ((X[i + 2] - X[i + 1]) - gr) - 2.0f * (gr - gl) + (gl - (X[i - 1] - X[i - 2]));
    if (i == 0) d4 += bsgn * X[i];
    if (i == n_u - 1) d4 += bsgn * X[i];
    return d4;
  };

  // ---- the partitioned tridiagonal solves: warp 0 (rows lane m .. lane m + m - 1,
  // cyclic reduction across its lanes), between block barriers; the other
  // warps take part in the row loops around them ----
  RedT<R> rdu, rdz;   // (valid in warp 0)
  auto factor_u = [&]() {
    __syncthreads();
    if (warp == 0) tri_factor(SUB, INV, CP, AL, FF, GG, m_u, lane, rdu);
    __syncthreads();
  };
  auto solve_u = [&](R* X) {
    __syncthreads();
    if (warp == 0) tri_solve(SUB, INV, CP, FF, GG, X, m_u, lane, rdu);
    __syncthreads();
  };
  auto solve_z = [&](R* X) {
    __syncthreads();
    if (warp == 0) tri_solve(SUBZ, INVZ, CPZ, FFZ, GGZ, X, m_z, lane, rdz);
    __syncthreads();
  };
  // block-wide maxima of two non-negative floats (double-buffered slots)
  int rbuf = 0;
  auto block_max2 = [&](float& a, float& b) {
    a = warp_max_nonneg(a);
    b = warp_max_nonneg(b);
    if (lane == 0) { red[rbuf][0][warp] = a; red[rbuf][1][warp] = b; }
    __syncthreads();
    a = red[rbuf][0][0];
    b = red[rbuf][1][0];
#pragma unroll
    for (int w = 1; w < kAdjWarps; ++w) { a = fmaxf(a, red[rbuf][0][w]); b = fmaxf(b, red[rbuf][1][w]); }
    rbuf ^= 1;
  };

  // ---- constant matrices ----
  if (has_z) {
    const R dzd = 1.0f + s0 + 2.0f * s1l;
    for (int i = tid; i < kWarp * m_z; i += kAdjThreads) {
      const bool real = i < n_z;
      SUBZ[i] = real && i > 0 ? -s1l : 0.0f;
      INVZ[i] = real ? dzd : 1.0f;
      CPZ[i] = real && i < n_z - 1 ? -s1l : 0.0f;
    }
    __syncthreads();
    if (warp == 0) tri_factor(SUBZ, INVZ, CPZ, ALZ, FFZ, GGZ, m_z, lane, rdz);
    __syncthreads();
  }
  auto assemble_u = [&]() {   // A_u(g) at the current level
    for (int i = tid; i < kWarp * m_u; i += kAdjThreads) {
      if (i < n_u) {
        const R gl = G[i], gr = G[i + 1];
        const R gl2 = linear ? 0.0f : gl * gl, gr2 = linear ? 0.0f : gr * gr;
        SUB[i] = i > 0 ? og - ca * gl2 : 0.0f;
        INV[i] = dg + ca * (gl2 + gr2);
        CP[i] = i < n_u - 1 ? og - ca * gr2 : 0.0f;
      } else {
        SUB[i] = 0.0f; INV[i] = 1.0f; CP[i] = 0.0f;
      }
    }
    factor_u();
  };
  if (linear) assemble_u();
  __syncthreads();

  // Solve M (X, XZ) = (ra, rz) (forward form; rz null: zero), block
  // Gauss-Seidel from the warm start in XZw, as the forward kernel.
  auto coupled = [&](const R* ra, const R* rz, R* X, R* XZw) {
    if (!has_z) {
      for (int i = tid; i < kWarp * m_u; i += kAdjThreads) X[i] = ra[i];
      solve_u(X);
      return;
    }
    float e_prev = 0.f;
    for (int sweep = 1;; ++sweep) {
      for (int i = tid; i < n_u; i += kAdjThreads) XZT[i] = interp_z(XZw, i);
      __syncthreads();
      for (int i = tid; i < kWarp * m_u; i += kAdjThreads) {
        X[i] = i < n_u ? ra[i] + cb * (static_cast<R>(G[i + 1]) * (XZT[i + 1] - XZT[i]) -
                                       static_cast<R>(G[i]) * (XZT[i] - XZT[i - 1]))
                       : 0.0f;
      }
      solve_u(X);
      for (int i = tid; i < n_u; i += kAdjThreads)
        FT[i] = static_cast<R>(G[i + 1]) * (X[i + 1] - X[i]) - static_cast<R>(G[i]) * (X[i] - X[i - 1]);
      __syncthreads();
      for (int i = tid; i < kWarp * m_z; i += kAdjThreads)
        E1Z[i] = i < n_z ? (rz ? rz[i] : 0.0f) + cz * spread(FT, i) : 0.0f;
      solve_z(E1Z);
      float chg = 0.f, mag = 0.f;
      for (int i = tid; i < kWarp * m_z; i += kAdjThreads) {
        const R v = E1Z[i];
        chg = fmaxf(chg, fabsf((v - XZw[i]).hi));
        mag = fmaxf(mag, fabsf(v.hi));
        XZw[i] = v;
      }
      block_max2(chg, mag);   // (its barrier also orders the XZw updates)
      const float e = chg > 0.f ? __fdividef(chg, mag) : 0.f;
      if (adj_converged(e, e_prev, sweep)) break;
      e_prev = e;
    }
  };

  // ---- adjoint state at level m_end, warm starts of the longitudinal solves ----
  double* adj = J.adj;
  // (kept in FP64 between segments)
  for (int i = tid; i < n_u; i += kAdjThreads) { LU[i] = df_from_double(adj[i]); LD[i] = df_from_double(adj[n_u + i]); }
  for (int i = tid; i < n_z; i += kAdjThreads) {
    LZ[i] = df_from_double(adj[2 * n_u + i]); LDZ[i] = df_from_double(adj[2 * n_u + n_z + i]);
    NZ[i] = df_from_double(adj[2 * n_u + 2 * n_z + 2 + i]); XZ[i] = df_from_double(adj[2 * n_u + 3 * n_z + 2 + i]);
  }
  R luh = df_from_double(adj[2 * n_u + 2 * n_z]), ldh = df_from_double(adj[2 * n_u + 2 * n_z + 1]);
  R acc[kGradSlots];
#pragma unroll
  for (int k = 0; k < kGradSlots; ++k) acc[k] = 0.0f;

  // level loaders: m_start from the checkpoint, later levels from the replay
  auto level_ptr = [&](int64_t lev, const float*& pu, const float*& pdu, const float*& pz, const float*& pdz,
                       float& uh, float& dh) {
    if (lev == J.m_start) {
      pu = J.u0; pdu = J.du0; pz = J.z0; pdz = J.dz0;
      uh = J.sc0->uh; dh = J.sc0->duh;
    } else {
      const float* rec = J.traj + (lev - J.m_start - 1) * J.traj_stride;
      pu = rec; pdu = rec + n_u; pz = rec + 2 * n_u; pdz = pz + n_z;
      uh = rec[2 * n_u + 2 * n_z]; dh = rec[2 * n_u + 2 * n_z + 1];
    }
  };
  // dJ/du of an output sample y = L I(x_o) u, or dJ/dz of y = L I_l(x_o) z
  // (LD, LDZ also take -c w for the first sample, which reads level 1 - D)
  auto add_output = [&](R dyv, bool first_level) {
    const R c = dyv * oscale;
    if (tid != 0) return;
    if (zout) {
      if (!has_z) return;   // zeta is identically zero
      if (oln - 1 >= 0 && oln - 1 < n_z) {
        LZ[oln - 1] += c * (1.0f - olw);
        if (first_level) LDZ[oln - 1] -= c * (1.0f - olw);
      }
      if (oln >= 0 && oln < n_z) {
        LZ[oln] += c * olw;
        if (first_level) LDZ[oln] -= c * olw;
      }
    } else {
      if (on - 1 >= 0 && on - 1 < n_u) {
        LU[on - 1] += c * (1.0f - ow);
        if (first_level) LD[on - 1] -= c * (1.0f - ow);
      }
      if (on >= 0 && on < n_u) {
        LU[on] += c * ow;
        if (first_level) LD[on] -= c * ow;
      }
    }
  };

  // D at level m_end (the first step's "next" level); for a bowed string the
  // level's u_H slot holds the bow velocity of the step that produced it
  float uh1, dh1;
  {
    const float *pu, *pdu, *pz, *pdz;
    level_ptr(J.m_end, pu, pdu, pz, pdz, uh1, dh1);
    for (int i = tid; i < n_u; i += kAdjThreads) DN1[i] = pdu[i];
    for (int i = tid; i < n_z; i += kAdjThreads) DZN1[i] = pdz[i];
  }
  __syncthreads();

  for (int64_t m = J.m_end; m > J.m_start; --m) {
    const int64_t n = m - 1;
    if (mod_kind != 0) {   // the step n -> n + 1 as the forward took it
      const float rm = mod_factor(mod_kind, Dp->mod_inc_fx, Dp->mod_phase_fx, mod_depth2, Dp->mod_inc, Dp->mod_hold,
                                  Dp->mod_n_end, n);
      const float l2 = lam2_0f * rm;
      lam2 = static_cast<R>(l2) + static_cast<R>(fmaf(lam2_0f, rm, -l2) + lam2lo_0f * rm);
      lam2l = static_cast<R>(lam2l_0f * rm);
      ca = static_cast<R>(ca_0f * rm);
      cb = static_cast<R>(cb_0f * rm);
      cz = static_cast<R>(cz_0f * rm);
      rmd = static_cast<R>(rm);
    }
    add_output(J.dy[m], false);
    // ---- level n state; a = D(n+1) - D(n) etc. ----
    float uh, dh;
    {
      const float *pu, *pdu, *pz, *pdz;
      level_ptr(n, pu, pdu, pz, pdz, uh, dh);
      for (int i = tid; i < n_u; i += kAdjThreads) {
        U[i] = pu[i];
        const float d = pdu[i];
        DU[i] = d;
        A[i] = DN1[i] - d;
      }
      for (int i = tid; i < n_z; i += kAdjThreads) {
        Z[i] = pz[i];
        const float d = pdz[i];
        DZ[i] = d;
        AZ[i] = DZN1[i] - d;
      }
    }
    const R s_h = -hM * (static_cast<R>(dh1) - dh);   // hammer force of the step (k^2-scaled)
    __syncthreads();
    for (int i = tid; i <= n_u; i += kAdjThreads) G[i] = U[i] - U[i - 1];
    if (has_z) {
      for (int i = tid; i < n_u; i += kAdjThreads) {
        ZT[i] = interp_z(Z, i).hi;   // the nearest float
        AZT[i] = interp_z(AZ, i).hi;
      }
    }
    __syncthreads();
    if (!linear) assemble_u();
    R eta = 0.0f, k2G = 0.0f;
    if (hammer) {
      eta = static_cast<R>(uh) - ((1.0f - ew) * static_cast<R>(U[en - 1]) + ew * static_cast<R>(U[en]));
      if (eta > 0.0f) k2G = hk2w * df_from_double(pow(to_double(eta), to_double(hexpo)));   // (FP64: contact only)
    }
    // ---- transposed solve ----
    const R mus = hammer ? -(ldh + luh) / hM : 0.0f;
    for (int i = tid; i < kWarp * m_u; i += kAdjThreads) RA[i] = i < n_u ? LD[i] + LU[i] : 0.0f;
    const R zs = has_z ? cz / cb : 0.0f;
    for (int i = tid; i < kWarp * m_z; i += kAdjThreads) RZ_[i] = i < n_z ? zs * (LDZ[i] + LZ[i]) : 0.0f;
    __syncthreads();
    coupled(RA, RZ_, NA, NZ);
    R nus = mus;
    // bow (Eq. 5) with force on: sliding, R3 = s + k^2 F phi(v) with
    // v = I(a + 2D) / 2k - v_B; sticking (v = 0), R3 = v.  Either way M^T
    // adds a rank-one term along the unit-force response.
    const bool bow_on = bow && n < brel && bF > 0.0f;
    const R vb = uh1;
    R phid = 0.0f;
    if (bow_on) phid = -ba * (1.0f - beps) * df_from_double(exp(-to_double(ba) * ::fabs(static_cast<double>(uh1))));
    if (hammer && k2G > 0.0f) {
      const R rs = -(hM * k2G / (2.0f * js)) * mus;
      for (int i = tid; i < kWarp * m_u; i += kAdjThreads) {
        R v = 0.0f;
        if (i == en - 1) v += (1.0f - ew) * js;
        if (i == en) v += ew * js;
        T1[i] = i < n_u ? v : 0.0f;
      }
      __syncthreads();
      coupled(T1, nullptr, XP, XZ);
      const R cm = 0.5f * hM * k2G;
      const R ia = (1.0f - ew) * NA[en - 1] + ew * NA[en], ix = (1.0f - ew) * XP[en - 1] + ew * XP[en];
      const R st = (rs - cm * ia) / (1.0f + 0.5f * k2G + cm * ix);
      __syncthreads();   // every thread has read NA at the contact point
      for (int i = tid; i < n_u; i += kAdjThreads) NA[i] = fma(st, XP[i], NA[i]);
      for (int i = tid; i < n_z; i += kAdjThreads) NZ[i] = fma(st, XZ[i], NZ[i]);
      nus = -(2.0f * js / (hM * k2G)) * st;
      __syncthreads();
    } else if (bow_on) {
      for (int i = tid; i < kWarp * m_u; i += kAdjThreads) {
        R v = 0.0f;
        if (i == en - 1) v += (1.0f - ew) * js;
        if (i == en) v += ew * js;
        T1[i] = i < n_u ? v : 0.0f;
      }
      __syncthreads();
      coupled(T1, nullptr, XP, XZ);
      const R ia = (1.0f - ew) * NA[en - 1] + ew * NA[en], ix = (1.0f - ew) * XP[en - 1] + ew * XP[en];
      R st;
      if (vb == 0.0f) {   // sticking: I nu_a = 0
        st = -ia / ix;
        nus = 2.0f * kk * js * st;
      } else {           // sliding
        const R bj = 0.5f * kk * bF * phid;
        st = -bj * ia / (1.0f + bj * ix);
        nus = -js * (ia + st * ix);
      }
      __syncthreads();   // every thread has read NA at the bow
      for (int i = tid; i < n_u; i += kAdjThreads) NA[i] = fma(st, XP[i], NA[i]);
      for (int i = tid; i < n_z; i += kAdjThreads) NZ[i] = fma(st, XZ[i], NZ[i]);
      __syncthreads();
    }
    // nu_z = (cb / cz) nz; the warm start of the next step keeps nz
    const R zr = has_z ? cb / cz : 0.0f;
    for (int i = tid; i < n_z; i += kAdjThreads) T2[i] = zr * NZ[i];
    __syncthreads();
    const R* NUZ = T2;

    // ---- (dR/dx)^T nu and (dR/dc)^T nu ----
    R pg[kGradSlots];
#pragma unroll
    for (int k = 0; k < kGradSlots; ++k) pg[k] = 0.0f;
    if (has_z) {
      for (int i = tid; i < n_u; i += kAdjThreads) PNZ[i] = interp_z(NUZ, i);
      __syncthreads();
    }
    // intervals (for a linear string, alpha = 1, only the c_a term is first
    // order in alpha: the longitudinal field and its adjoint stay zero)
    for (int i = tid; i <= n_u; i += kAdjThreads) {
      const R g = G[i], psi = NA[i] - NA[i - 1];
      const R sa = static_cast<R>(A[i]) - A[i - 1];
      R e = 0.0f, q = 0.0f, chi = 0.0f;
      if (has_z) {
        e = static_cast<R>(ZT[i]) - ZT[i - 1];
        q = static_cast<R>(AZT[i]) - AZT[i - 1];
        chi = PNZ[i] - PNZ[i - 1];
      }
      GAM[i] = -psi * (6.0f * ca * g * g + 4.0f * cb * e + cb * q + 2.0f * ca * g * sa) - chi * (4.0f * cz * g + cz * sa);
      PSG[i] = psi * g;
      pg[kGCa] -= psi * (2.0f * g * g * g + g * g * sa);
      pg[kGCb] -= psi * (4.0f * g * e + g * q);
      pg[kGCz] -= chi * (2.0f * g * g + g * sa);
    }
    __syncthreads();
    for (int i = tid; i < n_u; i += kAdjThreads) {
      const R d2na = d2_of(NA, i), d4na = d4_of(NA, i);
      const R d2u = d2_of(U, i), d2du = d2_of(DU, i), d2a = d2_of(A, i);
      const R na = NA[i], lu = LU[i];
      R lun = lu + lam2 * d2na - mu2 * d4na;
      if (!linear) lun += GAM[i] - GAM[i + 1];
      LD[i] = LD[i] + lu - 2.0f * s0u * na + 2.0f * s1 * d2na;
      LU[i] = lun;
      pg[kGLam2] += na * d2u;
      // nu . d4 u summed by parts: (d2 nu) . (d2 u) plus the ghost's corner terms
      R nd4u = d2na * d2u;
      if (i == 0 || i == n_u - 1) nd4u += (1.0f + bsgn) * na * static_cast<R>(U[i]);
      pg[kGMu2] -= nd4u;
      pg[kGS0u] += na * (-2.0f * static_cast<R>(DU[i]) - static_cast<R>(A[i]));
      pg[kGS1] += na * (2.0f * d2du + d2a);
    }
    if (has_z) {
      for (int i = tid; i < n_u; i += kAdjThreads) FT[i] = PSG[i + 1] - PSG[i];   // d_+[psi g] at the rows
      __syncthreads();
      for (int i = tid; i < n_z; i += kAdjThreads) {
        const R nz = NUZ[i];
        const R d2n = d2_of(NUZ, i), d2z = d2_of(Z, i), d2dz = d2_of(DZ, i), d2az = d2_of(AZ, i);
        const R lz = LZ[i];
        LDZ[i] = LDZ[i] + lz - 2.0f * s0 * nz + 2.0f * s1l * d2n;
        LZ[i] = lz + lam2l * d2n + 4.0f * cb * spread(FT, i);
        pg[kGLam2l] += nz * d2z;
        pg[kGS0] += nz * (-2.0f * static_cast<R>(DZ[i]) - static_cast<R>(AZ[i]));
        pg[kGS1l] += nz * (2.0f * d2dz + d2az);
      }
    }
    __syncthreads();
    if (hammer) {
      R psi_eta = 0.0f;
      if (k2G > 0.0f) {
        const R dG = hexpo * k2G / eta;
        const R ia = (1.0f - ew) * static_cast<R>(A[en - 1]) + ew * static_cast<R>(A[en]);
        psi_eta = nus * (hM * k2G + (hM * eta - 0.5f * hM * ia - 0.5f * s_h) * dG);
      }
      if (tid == 0 && psi_eta != 0.0f) {
        if (en - 1 >= 0 && en - 1 < n_u) LU[en - 1] -= psi_eta * (1.0f - ew);
        if (en >= 0 && en < n_u) LU[en] -= psi_eta * ew;
      }
      ldh = ldh + luh;
      luh = luh + psi_eta;
    }
    if (bow_on && tid == 0) {
      // (dR3/dD)^T nu_s and dR3/dv_B (the amplitude slot of a bowed string)
      const R cd = vb == 0.0f ? 1.0f / kk : kk * bF * phid;
      if (en - 1 >= 0 && en - 1 < n_u) LD[en - 1] += cd * (1.0f - ew) * nus;
      if (en >= 0 && en < n_u) LD[en] += cd * ew * nus;
      pg[kGAmp] += vb == 0.0f ? -nus : -kk * kk * bF * phid * nus;
    }
    __syncthreads();
    if (mod_kind != 0) {   // d(coefficient of step n) / d(unscaled coefficient) = rm
      pg[kGLam2] *= rmd;
      pg[kGLam2l] *= rmd;
      pg[kGCa] *= rmd;
      pg[kGCb] *= rmd;
      pg[kGCz] *= rmd;
    }
#pragma unroll
    for (int k = 0; k < kGradSlots; ++k) acc[k] += pg[k];
    // the level-n D becomes the next step's D(n+1)
    { float* t = DN1; DN1 = DU; DU = t; }
    if (has_z) { float* t = DZN1; DZN1 = DZ; DZ = t; }
    dh1 = dh;
    uh1 = uh;
    __syncthreads();
  }

  if (J.first) {
    // level 1 output, level 0 output y^0 = L I(u^1 - D^1), initial-state terms
    add_output(J.dy[1], false);
    __syncthreads();
    add_output(J.dy[0], true);
    __syncthreads();
    R pa = 0.0f;
    if (J.pluck_pos >= 0.f) {   // u^0 = u^1 = c0 tri(x), D^1 = 0
      const R xp = J.pluck_pos;
      for (int i = tid; i < n_u; i += kAdjThreads) {
        const R x = static_cast<R>(i + 1) * inv_nt;
        const R tri = x <= xp ? x / xp : (1.0f - x) / (1.0f - xp);
        pa += LU[i] * tri;
      }
    } else if (hammer && tid == 0) {   // u_H^1 = D_H^1 = v k
      pa = static_cast<R>(Dp->k) * (luh + ldh);
    }
    acc[kGAmp] += pa;
  }

  // ---- store the adjoint state, the warm starts and the gradients ----
  for (int i = tid; i < n_u; i += kAdjThreads) { adj[i] = to_double(LU[i]); adj[n_u + i] = to_double(LD[i]); }
  for (int i = tid; i < n_z; i += kAdjThreads) {
    adj[2 * n_u + i] = to_double(LZ[i]); adj[2 * n_u + n_z + i] = to_double(LDZ[i]);
    adj[2 * n_u + 2 * n_z + 2 + i] = to_double(NZ[i]); adj[2 * n_u + 3 * n_z + 2 + i] = to_double(XZ[i]);
  }
  if (tid == 0) { adj[2 * n_u + 2 * n_z] = to_double(luh); adj[2 * n_u + 2 * n_z + 1] = to_double(ldh); }
#pragma unroll
  for (int k = 0; k < kGradSlots; ++k) {
    R v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    if (lane == 0) gsum[warp][k] = v;
  }
  __syncthreads();
  if (tid < kGradSlots) {
    R v = gsum[0][tid];
#pragma unroll
    for (int w = 1; w < kAdjWarps; ++w) v += gsum[w][tid];
    J.grad[tid] += to_double(v);
  }
}

namespace {
// The dynamic shared-memory limit is a process-wide attribute of the
// kernel: raised once per device to the opt-in maximum and never lowered,
// so concurrent launches from other threads cannot shrink it under a launch.
constexpr int kMaxAdjDevices = 64;
std::mutex g_adj_attr_mu;
bool g_adj_attr_done[kMaxAdjDevices] = {};

cudaError_t raise_adjoint_smem_limit() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxAdjDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_adj_attr_mu);
  if (g_adj_attr_done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, adjoint_kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - static_cast<int>(fa.sharedSizeBytes));
  if (e == cudaSuccess) g_adj_attr_done[dev] = true;
  return e;
}
}  // namespace

// Static shared memory of the adjoint kernel (its reduction cells), which a
// launch's dynamic shared memory must leave room for.
cudaError_t adjoint_static_smem(size_t* bytes) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, adjoint_kernel);
  if (e == cudaSuccess) *bytes = fa.sharedSizeBytes;
  return e;
}

// Host-side launcher (called by sfd_api.cu): one block of kAdjWarps warps per job.
cudaError_t launch_adjoint(const AdjJob* d_jobs, int n_jobs, int smem_bytes, cudaStream_t stream) {
  cudaError_t e = raise_adjoint_smem_limit();
  if (e != cudaSuccess) return e;
  adjoint_kernel<<<n_jobs, kAdjThreads, static_cast<size_t>(smem_bytes), stream>>>(d_jobs, n_jobs);
  return cudaGetLastError();
}

}  // namespace sfd
