// Shared-memory path of the step kernel (every per-row array in the warp's
// shared-memory region); used for grids with more than kMaxRegRows transverse
// rows per lane.
#pragma once

#include "sfd_device.cuh"

namespace sfd {

// ----------------------------------------------------------------------------
// One job: a string advanced by n_samples output samples.
//
// Unknowns per step are the accelerations a = D+ - D (transverse) and
// az = Dz+ - Dz (longitudinal).  Substituting D+ = D + a into the
// increment form cancels the Theta terms exactly:
//   A a - d_+[cb g de_a] = lam2 d2 u - mu2 d4 u - 2 s0 D + 2 s1 d2 D
//                          + d_+[2 ca g^3 + 4 cb g e]
//   (1 + s0 - s1l d2) az - cz P^T d_+[g dg_a]
//                        = lam2l d2 z - 2 s0 Dz + 2 s1l d2 Dz + 2 cz P^T d_+[g^2]
// so FP32 rounding in the solve scales with the acceleration, not the
// velocity, and no Theta mismatch between the two sides can act as a loss.
// ----------------------------------------------------------------------------
static __device__ void run_job(const Job& job, float* __restrict__ wbase, int lane) {
  const Desc* __restrict__ Dp = job.desc;
  const int n_t = Dp->n_t, n_l = Dp->n_l, n_u = Dp->n_u, n_z = Dp->n_z;
  const int m_u = Dp->m_u, m_z = Dp->m_z;
  const bool has_z = m_z > 0;
  const bool linear = Dp->linear != 0;
  const bool zjac = Dp->z_jacobi != 0;
  const int exc = Dp->exc;
  const int RU = kWarp * m_u + 4, RZ = has_z ? kWarp * m_z + 4 : 0;
  const float dg = Dp->dg, og = Dp->og, s0 = Dp->s0, s0u = Dp->s0u, s1 = Dp->s1, s1l = Dp->s1l;
  const float lam2_0 = Dp->lam2, mu2 = Dp->mu2, lam2l_0 = Dp->lam2l, lam2lo_0 = Dp->lam2_lo;
  const float ca_0 = Dp->ca, cb_0 = Dp->cb, cz_0 = Dp->cz;
  const float bsgn = Dp->boundary == 1 ? -1.f : 1.f;
  const int mod_kind = Dp->mod_kind;
  const int sweep_cap = job.sweep_cap > 0 ? job.sweep_cap : kMaxSweeps;

  // ---- carve the warp's shared-memory region (kArraysU + kArraysZ arrays) ----
  float* p = wbase;
  auto U_ = [&]() { float* a = p + 2; p += RU; return a; };
  float *U = U_(), *DU = U_(), *AC = U_(), *XP = U_(), *RA = U_(), *SUB = U_(), *INV = U_();
  float *CP = U_(), *AL = U_(), *FF = U_(), *GG = U_(), *FV = U_(), *XFC = U_();
  float *ZT = U_(), *AZT = U_(), *XZT = U_(), *G = U_();
  int* TMI = reinterpret_cast<int*>(U_());     // left longitudinal node of transverse node i+1
  float* TMW = U_();                           // its interpolation weight on the right node
  float *Z = nullptr, *DZ = nullptr, *AZ = nullptr, *XZ = nullptr, *RZ_ = nullptr, *SUBZ = nullptr;
  float *INVZ = nullptr, *CPZ = nullptr, *ALZ = nullptr, *FFZ = nullptr, *GGZ = nullptr, *E1Z = nullptr;
  float* E2Z = nullptr;
  int *ZLO = nullptr, *ZHI = nullptr;
  if (has_z) {
    auto Z_ = [&]() { float* a = p + 2; p += RZ; return a; };
    Z = Z_(); DZ = Z_(); AZ = Z_(); XZ = Z_(); RZ_ = Z_(); SUBZ = Z_(); INVZ = Z_(); CPZ = Z_();
    ALZ = Z_(); FFZ = Z_(); GGZ = Z_(); E1Z = Z_(); E2Z = Z_();
    ZLO = reinterpret_cast<int*>(Z_());
    ZHI = reinterpret_cast<int*>(Z_());
  }
  const int total = static_cast<int>(p - wbase);
  for (int k = lane; k < total; k += kWarp) wbase[k] = 0.f;
  __syncwarp();

  // ---- load the state ----
  for (int i = lane; i < n_u; i += kWarp) { U[i] = Dp->u[i]; DU[i] = Dp->du[i]; }
  for (int i = lane; i < n_z; i += kWarp) {
    Z[i] = Dp->z[i]; DZ[i] = Dp->dz[i]; XZ[i] = Dp->xz[i]; AZ[i] = Dp->az[i];
  }
  Scalars* scp = Dp->sc;
  int64_t n = scp->n, jnext = scp->next_out;
  const int64_t n_first = n;
  float uh = scp->uh, duh = scp->duh, bow_w = scp->bow_w;
  int status = scp->status;
  int max_sweeps = scp->max_sweeps;
  int64_t sweeps_total = scp->sweeps_total;

  const int ub = lane * m_u, zb = lane * m_z;
  // grid transfer maps from exact integer positions: transverse node l sits at
  // longitudinal coordinate l N_l / N_t; longitudinal node mm's hat function
  // covers the transverse nodes with |l N_l - mm N_t| < N_t
  if (has_z) {
    for (int r = 0; r < m_u; ++r) {
      const int i = ub + r;
      if (i < n_u) {
        const int pos = (i + 1) * n_l;
        const int mm = pos / n_t;
        TMI[i] = mm;
        TMW[i] = static_cast<float>(pos - mm * n_t) / static_cast<float>(n_t);
      }
    }
    for (int r = 0; r < m_z; ++r) {
      const int i = zb + r;
      if (i < n_z) {
        const int mm = i + 1;
        const int lo = ((mm - 1) * n_t) / n_l + 1;
        const int hi = ((mm + 1) * n_t + n_l - 1) / n_l - 1;
        ZLO[i] = lo < 1 ? 1 : lo;
        ZHI[i] = hi > n_t - 1 ? n_t - 1 : hi;
      }
    }
  }
  const float inv_nt = 1.f / static_cast<float>(n_t);
  auto interp_z = [&](const float* A, int i) {   // z field at transverse row i
    const int mm = TMI[i];
    const float w = TMW[i];
    return (1.f - w) * A[mm - 1] + w * A[mm];
  };
  auto spread = [&](const float* F, int i) {     // (P^T F) at longitudinal row i
    const int mm = i + 1, lo = ZLO[i], hi = ZHI[i];
    float acc = 0.f;
    for (int l = lo; l <= hi; ++l) {
      const int dd = l * n_l - mm * n_t;
      const float w = 1.f - static_cast<float>(dd < 0 ? -dd : dd) * inv_nt;
      acc = fmaf(fmaxf(w, 0.f), F[l - 1], acc);
    }
    return acc;
  };

  // ---- constant matrices ----
  Red rdu, rdz;
  const float dz_diag = 1.f + s0 + 2.f * s1l;
  const float dz_inv = 1.f / dz_diag;
  if (has_z && !zjac) {
    for (int r = 0; r < m_z; ++r) {
      const int i = zb + r;
      if (i < n_z) {
        SUBZ[i] = i > 0 ? -s1l : 0.f;
        INVZ[i] = dz_diag;
        CPZ[i] = i < n_z - 1 ? -s1l : 0.f;
      } else {
        SUBZ[i] = 0.f; INVZ[i] = 1.f; CPZ[i] = 0.f;
      }
    }
    tri_factor(SUBZ, INVZ, CPZ, ALZ, FFZ, GGZ, m_z, lane, rdz);
  }
  for (int r = 0; r < m_u; ++r) {
    const int i = ub + r;
    if (i < n_u) {
      SUB[i] = i > 0 ? og : 0.f;
      INV[i] = dg;
      CP[i] = i < n_u - 1 ? og : 0.f;
    } else {
      SUB[i] = 0.f; INV[i] = 1.f; CP[i] = 0.f;
    }
  }
  const bool forced = exc != kPluck;
  int en = Dp->e_node;              // excitation point (a bow envelope moves it per step)
  float ew = Dp->e_w;
  const float js = Dp->jscale;
  const int benv = exc == kBow ? Dp->bow_env_n : 0;
  float bv = Dp->bow_v;             // the step's bow velocity
  auto load_J = [&](float* E) {      // E[i] = J_i for the lane's rows
    for (int r = 0; r < m_u; ++r) {
      const int i = ub + r;
      float v = 0.f;
      if (i == en - 1) v += (1.f - ew) * js;
      if (i == en) v += ew * js;
      E[i] = (i < n_u) ? v : 0.f;
    }
  };
  if (linear) {
    tri_factor(SUB, INV, CP, AL, FF, GG, m_u, lane, rdu);
    if (forced) {
      load_J(XP);
      tri_solve(SUB, INV, CP, FF, GG, XP, m_u, lane, rdu);
    }
  }
  __syncwarp();

  // One longitudinal half-sweep: new values of the field X (AZ or XZ) from
  // the right-hand side held in E1Z; returns the largest change and magnitude
  // (lane-local).  Exact tridiagonal solve, or one Jacobi update of the tiny
  // off-diagonal when it is folded into the sweeps.
  auto z_update = [&](float* X, float& chg, float& mag) {
    if (zjac) {
      for (int r = 0; r < m_z; ++r) {
        const int i = zb + r;
        E2Z[i] = i < n_z ? (E1Z[i] + s1l * (X[i - 1] + X[i + 1])) * dz_inv : 0.f;
      }
      __syncwarp();
      for (int r = 0; r < m_z; ++r) {
        const int i = zb + r;
        const float v = E2Z[i];
        chg = fmaxf(chg, fabsf(v - X[i]));
        mag = fmaxf(mag, fabsf(v));
        X[i] = v;
      }
    } else {
      tri_solve(SUBZ, INVZ, CPZ, FFZ, GGZ, E1Z, m_z, lane, rdz);
      for (int r = 0; r < m_z; ++r) {
        const int i = zb + r;
        const float v = E1Z[i];
        chg = fmaxf(chg, fabsf(v - X[i]));
        mag = fmaxf(mag, fmaxf(fabsf(v), X == AZ ? fabsf(DZ[i]) : 0.f));
        X[i] = v;
      }
    }
  };

  const int on = Dp->o_node, oln = Dp->ol_node;
  const float ow = Dp->o_w, olw = Dp->ol_w, oscale = Dp->out_scale;
  const bool zout = Dp->out_ch == 1;
  const int64_t j_end = jnext + job.n_samples;
  float outbuf = 0.f;
  int64_t opos = 0;

  while (jnext < j_end) {
    if (jnext > n && !(status & kStUnstable)) {
      // ======================= one step n -> n+1 =======================
      const float rm = mod_factor(mod_kind, Dp->mod_inc_fx, Dp->mod_phase_fx, Dp->mod_depth2, Dp->mod_inc,
                                  Dp->mod_hold, Dp->mod_n_end, n);
      const float lam2 = lam2_0 * rm, lam2l = lam2l_0 * rm;
      // low part of lam2_0 * rm (exact product residual plus the stored low part)
      const float lam2_lo = fmaf(lam2_0, rm, -lam2) + lam2lo_0 * rm;
      const float ca = ca_0 * rm, cb = cb_0 * rm, cz = cz_0 * rm;

      // excitation scalars at time level n
      float eta = 0.f, k2G = 0.f, FB = 0.f;
      float vrec = 0.f;   // bow: relative velocity of the step (0 while sticking), for the adjoint
      if (exc == kHammer) {
        eta = uh - interp2(U, en, ew);
        if (eta > 0.f) k2G = Dp->ham_k2w * powf(eta, Dp->ham_expo);
      } else if (exc == kBow) {
        float bf = Dp->bow_F;
        if (benv > 0) {
          const int en0 = en;
          const float ew0 = ew;
          bow_env_eval(Dp, n, bv, bf, en, ew);
          if (linear && (en != en0 || ew != ew0)) {   // the fixed-matrix response A^-1 J follows x_B
            __syncwarp();                             // the last step's reads of XP are done
            load_J(XP);
            tri_solve(SUB, INV, CP, FF, GG, XP, m_u, lane, rdu);
            __syncwarp();
          }
        }
        FB = (n < Dp->bow_release_n) ? bf : 0.f;
      }
      const bool need_resp = !linear && ((exc == kHammer && k2G > 0.f) || (exc == kBow && FB > 0.f));

      // ---- stage 0: longitudinal field and warm starts at the transverse nodes ----
      if (has_z) {
        for (int r = 0; r < m_u; ++r) {
          const int i = ub + r;
          if (i < n_u) {
            ZT[i] = interp_z(Z, i);
            AZT[i] = interp_z(AZ, i);
            if (need_resp) XZT[i] = interp_z(XZ, i);
          }
        }
        __syncwarp();
      }

      // ---- stage 1: transverse right-hand side and matrix ----
      for (int r = 0; r < m_u; ++r) {
        const int i = ub + r;
        if (i >= n_u) break;
        const float u0 = U[i], um1 = U[i - 1], up1 = U[i + 1], um2 = U[i - 2], up2 = U[i + 2];
        const float gl = u0 - um1, gr = up1 - u0;
        const float d2 = gr - gl;
        float d4 = ((up2 - up1) - gr) - 2.f * d2 + (gl - (um1 - um2));
        if (i == 0) d4 += bsgn * u0;
        if (i == n_u - 1) d4 += bsgn * u0;
        const float du0 = DU[i];
        const float d2du = (DU[i + 1] - du0) - (du0 - DU[i - 1]);
        float rhs = fmaf(lam2, d2, lam2_lo * d2) - mu2 * d4 - 2.f * s0u * du0 + 2.f * s1 * d2du;
        if (!linear) {
          const float gl2 = gl * gl, gr2 = gr * gr;
          float yl = 2.f * ca * gl2 * gl, yr = 2.f * ca * gr2 * gr;
          if (has_z) {
            yl += 4.f * cb * gl * (ZT[i] - ZT[i - 1]);
            yr += 4.f * cb * gr * (ZT[i + 1] - ZT[i]);
            FV[i] = gr2 - gl2;
          }
          rhs += yr - yl;
          SUB[i] = i > 0 ? og - ca * gl2 : 0.f;
          INV[i] = dg + ca * (gl2 + gr2);
          CP[i] = i < n_u - 1 ? og - ca * gr2 : 0.f;
          G[i] = gl;
          if (i == n_u - 1) G[i + 1] = gr;
        }
        RA[i] = rhs;
      }
      if (!linear) tri_factor(SUB, INV, CP, AL, FF, GG, m_u, lane, rdu);
      __syncwarp();

      if (!has_z) {
        // ---- single transverse solve ----
        for (int r = 0; r < m_u; ++r) AC[ub + r] = RA[ub + r];
        tri_solve(SUB, INV, CP, FF, GG, AC, m_u, lane, rdu);
        if (need_resp) {
          load_J(XP);
          tri_solve(SUB, INV, CP, FF, GG, XP, m_u, lane, rdu);
        }
        __syncwarp();
      } else {
        // ---- stage 2: longitudinal right-hand side ----
        for (int r = 0; r < m_z; ++r) {
          const int i = zb + r;
          if (i >= n_z) break;
          const float z0 = Z[i];
          const float d2z = (Z[i + 1] - z0) - (z0 - Z[i - 1]);
          const float dz0 = DZ[i];
          const float d2dz = (DZ[i + 1] - dz0) - (dz0 - DZ[i - 1]);
          RZ_[i] = lam2l * d2z - 2.f * s0 * dz0 + 2.f * s1l * d2dz + 2.f * cz * spread(FV, i);
        }
        __syncwarp();
        // ---- stage 3: block Gauss-Seidel on (a, az) [and the response] ----
        int sweep = 0;
        float e_prev = 0.f;
        for (;;) {
          if (sweep > 0) {
            for (int r = 0; r < m_u; ++r) {
              const int i = ub + r;
              if (i < n_u) {
                AZT[i] = interp_z(AZ, i);
                if (need_resp) XZT[i] = interp_z(XZ, i);
              }
            }
            __syncwarp();
          }
          for (int r = 0; r < m_u; ++r) {
            const int i = ub + r;
            float v = 0.f;
            if (i < n_u)
              v = RA[i] + cb * (G[i + 1] * (AZT[i + 1] - AZT[i]) - G[i] * (AZT[i] - AZT[i - 1]));
            AC[i] = v;
          }
          tri_solve(SUB, INV, CP, FF, GG, AC, m_u, lane, rdu);
          if (need_resp) {
            load_J(XP);
            for (int r = 0; r < m_u; ++r) {
              const int i = ub + r;
              if (i < n_u) XP[i] += cb * (G[i + 1] * (XZT[i + 1] - XZT[i]) - G[i] * (XZT[i] - XZT[i - 1]));
            }
            tri_solve(SUB, INV, CP, FF, GG, XP, m_u, lane, rdu);
          }
          __syncwarp();
          for (int r = 0; r < m_u; ++r) {
            const int i = ub + r;
            if (i < n_u) {
              FV[i] = G[i + 1] * (AC[i + 1] - AC[i]) - G[i] * (AC[i] - AC[i - 1]);
              if (need_resp) XFC[i] = G[i + 1] * (XP[i + 1] - XP[i]) - G[i] * (XP[i] - XP[i - 1]);
            }
          }
          __syncwarp();
          float chg = 0.f, mag = 0.f, chx = 0.f, mgx = 0.f;
          for (int r = 0; r < m_z; ++r) {
            const int i = zb + r;
            E1Z[i] = i < n_z ? RZ_[i] + cz * spread(FV, i) : 0.f;
          }
          z_update(AZ, chg, mag);
          if (need_resp) {
            __syncwarp();
            for (int r = 0; r < m_z; ++r) {
              const int i = zb + r;
              E1Z[i] = i < n_z ? cz * spread(XFC, i) : 0.f;
            }
            z_update(XZ, chx, mgx);
          }
          // converged when every field's largest change is below the
          // tolerance relative to that field's largest magnitude
          chg = warp_max_nonneg(chg);
          mag = warp_max_nonneg(mag);
          chx = warp_max_nonneg(chx);
          mgx = warp_max_nonneg(mgx);
          __syncwarp();
          ++sweep;
          const float e = fmaxf(chg > 0.f ? __fdividef(chg, mag) : 0.f, chx > 0.f ? __fdividef(chx, mgx) : 0.f);
          if (sweep_converged(e, e_prev, sweep)) break;
          if (sweep >= sweep_cap) { status |= kStNoConv; break; }
          e_prev = e;
        }
        sweeps_total += sweep;
        if (sweep > max_sweeps) max_sweeps = sweep;
      }

      // ---- stage 4: excitation force (scalar elimination) ----
      if (exc == kHammer) {
        float s = 0.f;
        if (k2G > 0.f) {
          const float M = Dp->ham_M;
          const float cm = 0.5f * M * k2G;
          s = cm * (2.f * eta - interp2(AC, en, ew)) / (1.f + 0.5f * k2G + cm * interp2(XP, en, ew));
          duh -= s / M;
        }
        uh += duh;
        if (s != 0.f) {
          for (int r = 0; r < m_u; ++r) AC[ub + r] = fmaf(s, XP[ub + r], AC[ub + r]);
          if (has_z)
            for (int r = 0; r < m_z; ++r) AZ[zb + r] = fmaf(s, XZ[zb + r], AZ[zb + r]);
        }
      } else if (exc == kBow && FB > 0.f) {
        const float k = Dp->k;
        const float b = (interp2(AC, en, ew) + 2.f * interp2(DU, en, ew)) * (0.5f / k) - bv;
        const float c = 0.5f * k * FB * interp2(XP, en, ew);
        const float phi = bow_phi(b, c, Dp->bow_a, Dp->bow_eps, bow_w);
        vrec = !(c > 0.f) ? b : (fabsf(b) <= c ? 0.f : b - c * phi);
        const float s = -Dp->k2 * FB * phi;
        for (int r = 0; r < m_u; ++r) AC[ub + r] = fmaf(s, XP[ub + r], AC[ub + r]);
        if (has_z)
          for (int r = 0; r < m_z; ++r) AZ[zb + r] = fmaf(s, XZ[zb + r], AZ[zb + r]);
      }

      // ---- stage 5: advance the time level ----
      bool bad = false;
      for (int r = 0; r < m_u; ++r) {
        const int i = ub + r;
        if (i < n_u) {
          const float d = DU[i] + AC[i];
          const float v = U[i] + d;
          DU[i] = d;
          U[i] = v;
          bad |= !isfinite(v);
        }
      }
      if (has_z) {
        for (int r = 0; r < m_z; ++r) {
          const int i = zb + r;
          if (i < n_z) {
            const float d = DZ[i] + AZ[i];
            DZ[i] = d;
            Z[i] += d;
          }
        }
      }
      if (__any_sync(SFD_FULL, bad)) status |= kStUnstable;
      __syncwarp();
      ++n;
      if (job.traj) {   // replay for the adjoint: record the new level
        float* rec = job.traj + (n - n_first - 1) * job.traj_stride;
        for (int i = lane; i < n_u; i += kWarp) { rec[i] = U[i]; rec[n_u + i] = DU[i]; }
        for (int i = lane; i < n_z; i += kWarp) { rec[2 * n_u + i] = Z[i]; rec[2 * n_u + n_z + i] = DZ[i]; }
        // (a bowed string has no hammer state: its slot holds the step's bow velocity)
        if (lane == 0) { rec[2 * n_u + 2 * n_z] = exc == kBow ? vrec : uh; rec[2 * n_u + 2 * n_z + 1] = duh; }
      }
    }
    // output sample j = jnext: u^n or u^{n-1}, or zeta (zeros once unstable)
    float y;
    if (zout) {
      y = 0.f;
      if (has_z) {
        y = zinterp(Z, oln, olw, n_z);
        if (jnext == n - 1) y -= zinterp(DZ, oln, olw, n_z);
      }
    } else if (jnext == n - 1) {
      y = interp2(U, on, ow) - interp2(DU, on, ow);
    } else {
      y = interp2(U, on, ow);
    }
    y *= oscale;
    if (status & kStUnstable) y = 0.f;
    if ((opos & (kWarp - 1)) == lane) outbuf = y;
    ++opos;
    if ((opos & (kWarp - 1)) == 0) job.out[opos - kWarp + lane] = outbuf;
    ++jnext;
  }
  {
    const int rem = static_cast<int>(opos & (kWarp - 1));
    if (lane < rem) job.out[opos - rem + lane] = outbuf;
  }

  // ---- store the state ----
  __syncwarp();
  for (int i = lane; i < n_u; i += kWarp) { Dp->u[i] = U[i]; Dp->du[i] = DU[i]; }
  for (int i = lane; i < n_z; i += kWarp) {
    Dp->z[i] = Z[i]; Dp->dz[i] = DZ[i]; Dp->xz[i] = XZ[i]; Dp->az[i] = AZ[i];
  }
  if (lane == 0) {
    scp->n = n;
    scp->next_out = jnext;
    scp->uh = uh;
    scp->duh = duh;
    scp->bow_w = bow_w;
    scp->status = status;
    scp->max_sweeps = max_sweeps;
    scp->sweeps_total = sweeps_total;
  }
  __syncwarp();
}

}  // namespace sfd
