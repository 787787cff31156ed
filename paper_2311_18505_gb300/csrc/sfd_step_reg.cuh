// Register-resident transverse path of the step kernel (included by
// sfd_kernel.cu).  Same scheme and stages as the shared-memory path
// (acceleration form of Eq. 4, partitioned tridiagonal solve, block
// Gauss-Seidel with the longitudinal grid, scalar hammer / bow
// elimination); the MU transverse rows of each lane live in registers with
// fully unrolled loops, neighbours come from shuffles, and only the grid
// transfer arrays and the longitudinal field stay in shared memory.
#pragma once

#include "sfd_device.cuh"

namespace sfd {

// Row values of x at offsets -2..+2 around the lane's chunk:
// e[0] = row base-2, e[1] = base-1, e[2 + r] = x[r], e[MU+2] = base+MU, e[MU+3].
template <int MU>
__device__ __forceinline__ void extend(const float (&x)[MU], float (&e)[MU + 4], int lane) {
  float l1 = __shfl_up_sync(SFD_FULL, x[MU - 1], 1);
  float r1 = __shfl_down_sync(SFD_FULL, x[0], 1);
  float l2, r2;
  if (MU >= 2) {
    l2 = __shfl_up_sync(SFD_FULL, x[MU >= 2 ? MU - 2 : 0], 1);
    r2 = __shfl_down_sync(SFD_FULL, x[MU >= 2 ? 1 : 0], 1);
    if (lane == 0) l2 = 0.f;
    if (lane == kWarp - 1) r2 = 0.f;
  } else {
    l2 = __shfl_up_sync(SFD_FULL, x[0], 2);
    r2 = __shfl_down_sync(SFD_FULL, x[0], 2);
    if (lane < 2) l2 = 0.f;
    if (lane >= kWarp - 2) r2 = 0.f;
  }
  if (lane == 0) l1 = 0.f;
  if (lane == kWarp - 1) r1 = 0.f;
  e[0] = l2;
  e[1] = l1;
#pragma unroll
  for (int r = 0; r < MU; ++r) e[r + 2] = x[r];
  e[MU + 2] = r1;
  e[MU + 3] = r2;
}

// Left/right neighbours only.
template <int MU>
__device__ __forceinline__ void extend1(const float (&x)[MU], float (&e)[MU + 2], int lane) {
  float l1 = __shfl_up_sync(SFD_FULL, x[MU - 1], 1);
  float r1 = __shfl_down_sync(SFD_FULL, x[0], 1);
  if (lane == 0) l1 = 0.f;
  if (lane == kWarp - 1) r1 = 0.f;
  e[0] = l1;
#pragma unroll
  for (int r = 0; r < MU; ++r) e[r + 1] = x[r];
  e[MU + 1] = r1;
}

// Value of row q (uniform across the warp); 0 outside [0, n_u).
template <int MU>
__device__ __forceinline__ float row_value(const float (&x)[MU], int q, int n_u) {
  const int qq = (q < 0 || q >= n_u) ? 0 : q;
  const int r = qq % MU, src = qq / MU;
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < MU; ++k)
    if (k == r) t = x[k];
  const float v = __shfl_sync(SFD_FULL, t, src);
  return (q < 0 || q >= n_u) ? 0.f : v;
}

template <int MU>
__device__ __forceinline__ float node_interp(const float (&x)[MU], int node, float w, int n_u) {
  return (1.f - w) * row_value<MU>(x, node - 1, n_u) + w * row_value<MU>(x, node, n_u);
}

// Partition factorisation of the lane's MU rows (register version of
// tri_factor): on entry iv = diagonal, cp = super-diagonal, sb = sub-diagonal;
// on exit iv = 1/pivot, cp = c', ff/gg = back-substitution weights.
template <int MU>
__device__ __forceinline__ void tri_factor_r(const float (&sb)[MU], float (&iv)[MU], float (&cp)[MU],
                                             float (&ff)[MU], float (&gg)[MU], int lane, Red& rd) {
  float al[MU];
  float cprev = 0.f, alprev = 0.f;
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    float inv;
    if (r == 0) {
      inv = fast_rcp(iv[r]);
      al[r] = sb[r] * inv;
    } else {
      inv = fast_rcp(iv[r] - sb[r] * cprev);
      al[r] = -sb[r] * alprev * inv;
    }
    cp[r] = cp[r] * inv;
    iv[r] = inv;
    cprev = cp[r];
    alprev = al[r];
  }
  ff[MU - 1] = 1.f;
  gg[MU - 1] = 0.f;
#pragma unroll
  for (int r = MU - 2; r >= 0; --r) {
    ff[r] = -cp[r] * ff[r + 1];
    gg[r] = -al[r] - cp[r] * gg[r + 1];
  }
  float f0n, g0n;
  if (MU == 1) {   // one row per lane: every lane's ff = 1, gg = 0
    f0n = lane == kWarp - 1 ? 0.f : 1.f;
    g0n = 0.f;
  } else {
    f0n = __shfl_down_sync(SFD_FULL, ff[0], 1);
    g0n = __shfl_down_sync(SFD_FULL, gg[0], 1);
    if (lane == kWarp - 1) { f0n = 0.f; g0n = 0.f; }
  }
  const float cl = cp[MU - 1];
  float A = al[MU - 1], B = 1.f + cl * g0n, C = cl * f0n;
  rd.cl = cl;
  rd.nlev = 5;
#pragma unroll
  for (int l = 0; l < 5; ++l) { rd.k1[l] = 0.f; rd.k2[l] = 0.f; }
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    if (__all_sync(SFD_FULL, fabsf(A) + fabsf(C) <= kPcrDrop * fabsf(B))) { rd.nlev = l; break; }
    const int s = 1 << l;
    float Am = __shfl_up_sync(SFD_FULL, A, s), Bm = __shfl_up_sync(SFD_FULL, B, s);
    float Cm = __shfl_up_sync(SFD_FULL, C, s);
    float Ap = __shfl_down_sync(SFD_FULL, A, s), Bp = __shfl_down_sync(SFD_FULL, B, s);
    float Cp = __shfl_down_sync(SFD_FULL, C, s);
    if (lane < s) { Am = 0.f; Bm = 1.f; Cm = 0.f; }
    if (lane + s >= kWarp) { Ap = 0.f; Bp = 1.f; Cp = 0.f; }
    const float k1 = A * fast_rcp(Bm), k2 = C * fast_rcp(Bp);
    A = -Am * k1;
    C = -Cp * k2;
    B = B - Cm * k1 - Ap * k2;
    rd.k1[l] = k1;
    rd.k2[l] = k2;
  }
  rd.binv = fast_rcp(B);
}

// Solve one (NR = 1) or two (NR = 2) right-hand sides in place, interleaved.
template <int MU, int NR>
__device__ __forceinline__ void tri_solve_r(const float (&sb)[MU], const float (&iv)[MU], const float (&cp)[MU],
                                            const float (&ff)[MU], const float (&gg)[MU], float (&x1)[MU],
                                            float (&x2)[MU], int lane, const Red& rd) {
  float p1 = 0.f, p2 = 0.f;
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    if (r == 0) {
      p1 = x1[r] * iv[r];
      if (NR == 2) p2 = x2[r] * iv[r];
    } else {
      p1 = (x1[r] - sb[r] * p1) * iv[r];
      if (NR == 2) p2 = (x2[r] - sb[r] * p2) * iv[r];
    }
    x1[r] = p1;
    if (NR == 2) x2[r] = p2;
  }
  const float dl1 = p1, dl2 = p2;
  x1[MU - 1] = 0.f;
  if (NR == 2) x2[MU - 1] = 0.f;
#pragma unroll
  for (int r = MU - 2; r >= 0; --r) {
    x1[r] = x1[r] - cp[r] * x1[r + 1];
    if (NR == 2) x2[r] = x2[r] - cp[r] * x2[r + 1];
  }
  // (one row per lane: the row just cleared is the neighbour's first, so
  // e1 = e2 = 0 and the shuffles are skipped)
  float e1 = 0.f, e2 = 0.f;
  if (MU > 1) {
    e1 = __shfl_down_sync(SFD_FULL, x1[0], 1);
    e2 = NR == 2 ? __shfl_down_sync(SFD_FULL, x2[0], 1) : 0.f;
    if (lane == kWarp - 1) { e1 = 0.f; e2 = 0.f; }
  }
  float D1 = dl1 - rd.cl * e1, D2 = dl2 - rd.cl * e2;
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    if (l >= rd.nlev) break;      // the factorisation dropped the remaining levels (warp-uniform)
    const int s = 1 << l;
    float m1 = __shfl_up_sync(SFD_FULL, D1, s), q1 = __shfl_down_sync(SFD_FULL, D1, s);
    float m2 = 0.f, q2 = 0.f;
    if (NR == 2) {
      m2 = __shfl_up_sync(SFD_FULL, D2, s);
      q2 = __shfl_down_sync(SFD_FULL, D2, s);
    }
    if (lane < s) { m1 = 0.f; m2 = 0.f; }
    if (lane + s >= kWarp) { q1 = 0.f; q2 = 0.f; }
    D1 = D1 - rd.k1[l] * m1 - rd.k2[l] * q1;
    if (NR == 2) D2 = D2 - rd.k1[l] * m2 - rd.k2[l] * q2;
  }
  const float X1 = D1 * rd.binv, X2 = D2 * rd.binv;
  // (one row per lane: gg = 0, so the previous lane's unknown is not needed)
  float Xp1 = 0.f, Xp2 = 0.f;
  if (MU > 1) {
    Xp1 = __shfl_up_sync(SFD_FULL, X1, 1);
    Xp2 = NR == 2 ? __shfl_up_sync(SFD_FULL, X2, 1) : 0.f;
    if (lane == 0) { Xp1 = 0.f; Xp2 = 0.f; }
  }
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    x1[r] = x1[r] + ff[r] * X1 + gg[r] * Xp1;
    if (NR == 2) x2[r] = x2[r] + ff[r] * X2 + gg[r] * Xp2;
  }
}

// Visit the lane's longitudinal rows i = lane + 32 k for k = k0, k0 + ks, ...
// < m_z (k0 = 0, ks = 1: all of them; a warp pair splits them by k parity):
// full groups of 4 rows compute all four results before any store (so the
// loads of the group overlap), the remainder row by row.  fn(i, v, x)
// computes, st(i, v, x) stores.
template <class Fn, class St>
__device__ __forceinline__ void z_rows(int m_z, int lane, Fn fn, St st, int k0 = 0, int ks = 1) {
  int k = k0;
  for (; k + 3 * ks < m_z; k += 4 * ks) {
    float v[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) fn(lane + kWarp * (k + q * ks), v[q], x[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) st(lane + kWarp * (k + q * ks), v[q], x[q]);
  }
  for (; k < m_z; k += ks) {
    float v, x;
    fn(lane + kWarp * k, v, x);
    st(lane + kWarp * k, v, x);
  }
}

// Barrier of the ng warps stepping one string together (named barrier id
// 1-3, 32 ng threads).  Ids and counts are immediates, so the kernel
// reserves only those barriers.
__device__ __forceinline__ void group_sync(int id, int ng) {
  if (ng == 4) {
    if (id == 3) asm volatile("bar.sync 3, 128;" ::: "memory");
    else asm volatile("bar.sync 1, 128;" ::: "memory");
  } else {
    if (id == 1) asm volatile("bar.sync 1, 64;" ::: "memory");
    else if (id == 2) asm volatile("bar.sync 2, 64;" ::: "memory");
    else asm volatile("bar.sync 3, 64;" ::: "memory");
  }
}

// A string may be stepped by one warp or by a group of ng = 2 or 4 warps of
// one CTA (warp pw of the group; the group launched with npw warps shares
// the string's shared-memory region, named barrier bar_id and exchange
// cells xcell[1024]).  Every warp of a group does the whole transverse side
// identically (same data, same operations, so the same bits), and the
// group splits the longitudinal rows by k mod ng; the warps meet at a
// barrier once the state is loaded, once per Gauss-Seidel sweep (where they
// also take the maximum of each lane's convergence measures, so all see
// exactly what one warp over all rows would) and once per step after the
// longitudinal update.  Every barrier sits in control flow that depends
// only on that shared data.  Only strings whose longitudinal grid is folded
// into the sweeps (z_jacobi) with at least 3 rows per lane take a group (4
// warps from 7 rows per lane); the launch's other warps return at once.
// Warp 0 of a group writes the output, the trajectory record and the state.
template <int MU>
__device__ void run_job_reg(const Job& job, float* __restrict__ wbase, int lane, int pw = 0, int npw = 1,
                            int bar_id = 1, float* xcell = nullptr) {
  const Desc* __restrict__ Dp = job.desc;
  const int n_t = Dp->n_t, n_l = Dp->n_l, n_u = Dp->n_u, n_z = Dp->n_z;
  const int m_z = Dp->m_z;
  const bool has_z = m_z > 0;
  const bool linear = Dp->linear != 0;
  const bool zjac = Dp->z_jacobi != 0;
  int ng = 1;                                  // warps stepping this string
  if (npw >= 2 && has_z && zjac && m_z >= 3) ng = 2;
  if (npw == 4 && has_z && zjac && m_z >= 7) ng = 4;
  if (pw >= ng) return;                       // the group's other warps step it
  const bool paired = ng > 1;
  const int kz0 = pw, kzs = ng;               // this warp's longitudinal rows: k = pw, pw + ng, ...
  const bool writer = pw == 0;
  int xpar = 0;                                             // exchange buffer in use
  const int exc = Dp->exc;
  const int RU = kWarp * MU + 4, RZ = has_z ? kWarp * m_z + 4 : 0;
  const float dg = Dp->dg, og = Dp->og, s0 = Dp->s0, s0u = Dp->s0u, s1 = Dp->s1, s1l = Dp->s1l;
  const float lam2_0 = Dp->lam2, mu2 = Dp->mu2, lam2l_0 = Dp->lam2l, lam2lo_0 = Dp->lam2_lo;
  const float ca_0 = Dp->ca, cb_0 = Dp->cb, cz_0 = Dp->cz;
  const float bsgn = Dp->boundary == 1 ? -1.f : 1.f;
  const int mod_kind = Dp->mod_kind;
  const uint64_t mod_inc_fx = Dp->mod_inc_fx, mod_phase_fx = Dp->mod_phase_fx;
  const int64_t mod_n_end = Dp->mod_n_end;
  const float mod_depth2 = Dp->mod_depth2, mod_inc = Dp->mod_inc, mod_hold = Dp->mod_hold;
  const float ham_k2w = Dp->ham_k2w, ham_expo = Dp->ham_expo, ham_M = Dp->ham_M;
  const float bow_F = Dp->bow_F, bow_v = Dp->bow_v, bow_a = Dp->bow_a, bow_eps = Dp->bow_eps;
  const float kk = Dp->k, k2 = Dp->k2;
  const float inv2k = 0.5f / kk;   // 1 / 2k: the bow's velocity I(a + 2D) / 2k without a divide per step
  const int64_t bow_release_n = Dp->bow_release_n;
  const int sweep_cap = job.sweep_cap > 0 ? job.sweep_cap : kMaxSweeps;

  // ---- shared memory: transverse transfer arrays, then the longitudinal grid ----
  float* p = wbase;
  auto U_ = [&]() { float* a = p + 2; p += RU; return a; };
  float* TMWs = U_();
  int* TMIs = reinterpret_cast<int*>(U_());
  float *Z = nullptr, *DZ = nullptr, *AZ = nullptr, *XZ = nullptr, *RZ_ = nullptr, *E1Z = nullptr;
  float *E2Z = nullptr, *E3Z = nullptr, *SUBZ = nullptr, *INVZ = nullptr, *CPZ = nullptr, *ALZ = nullptr;
  float *FFZ = nullptr, *GGZ = nullptr;
  float *SF0 = nullptr, *SF1 = nullptr, *SX0 = nullptr, *SX1 = nullptr;   // scatter slots
  if (has_z) {
    auto Z_ = [&]() { float* a = p + 2; p += RZ; return a; };
    Z = Z_(); DZ = Z_(); AZ = Z_(); XZ = Z_(); RZ_ = Z_(); E1Z = Z_(); E2Z = Z_(); E3Z = Z_();
    SF0 = Z_(); SF1 = Z_(); SX0 = Z_(); SX1 = Z_();
    if (!zjac) {
      SUBZ = Z_(); INVZ = Z_(); CPZ = Z_(); ALZ = Z_(); FFZ = Z_(); GGZ = Z_();
    }
  }
  const int total = static_cast<int>(p - wbase);
  for (int k = lane + kWarp * kz0; k < total; k += kWarp * kzs) wbase[k] = 0.f;
  __syncwarp();
  if (paired) group_sync(bar_id, ng);   // the region is zero before either warp writes to it

  // ---- registers: the lane's transverse rows i = lane*MU + r ----
  const int ub = lane * MU;
  float U[MU], DU[MU];
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    const int i = ub + r;
    U[r] = i < n_u ? Dp->u[i] : 0.f;
    DU[r] = i < n_u ? Dp->du[i] : 0.f;
  }
  for (int i = lane + kWarp * kz0; i < n_z; i += kWarp * kzs) {
    Z[i] = Dp->z[i]; DZ[i] = Dp->dz[i]; XZ[i] = Dp->xz[i]; AZ[i] = Dp->az[i];
  }
  Scalars* scp = Dp->sc;
  int64_t n = scp->n, jnext = scp->next_out;
  const int64_t n_first = n;
  float uh = scp->uh, duh = scp->duh, bow_w = scp->bow_w, scz = scp->scale_z, scx = scp->scale_x;
  int status = scp->status;
  int max_sweeps = scp->max_sweeps;
  int64_t sweeps_total = scp->sweeps_total;

  // grid transfer maps (exact integer positions)
  if (has_z) {
    // pad rows (i >= n_u) point at longitudinal node N_l + 1 (a zero cell)
    // with weight 0, so every lane can interpolate and scatter
    // unconditionally (no divergent branches)
#pragma unroll
    for (int r = 0; r < MU; ++r) {
      const int i = ub + r;
      const int pos = (i + 1) * n_l;
      const int mm = i < n_u ? pos / n_t : n_l + 1;
      TMIs[i] = mm;
      TMWs[i] = i < n_u ? static_cast<float>(pos - mm * n_t) / static_cast<float>(n_t) : 0.f;
    }
  }
  __syncwarp();
  if (paired) group_sync(bar_id, ng);   // both halves of the longitudinal state are loaded
  // (P^T F) at longitudinal node m = sum over the transverse nodes l of
  // P[l, m] F_l, P the linear interpolation from the longitudinal to the
  // transverse nodes.  Transverse node l (row l - 1) lies in the longitudinal
  // interval [m_l, m_l + 1) and gives (1 - w_l) F_l to node m_l and w_l F_l
  // to node m_l + 1.  The rows of one interval are consecutive, and each
  // lane owns consecutive rows, so emit() sums every interval by a segmented
  // scan (within the lane's rows, then across lanes by shuffles) and the
  // interval's last row stores the two sums: S0[m] = sum of (1 - w) F over
  // interval m, S1[m + 1] = sum of w F over it.  Node m then reads
  // S0[m] + S1[m] (spreadS).  Which slots are written is fixed by the grid,
  // so the others keep the zeros they were given; pad rows form their own
  // interval N_l + 1 with weight 0.
  int mmr[MU];
  float wr[MU];
  unsigned lastm = 0;          // bit r: row r is the last row of its interval
  bool carry_ok = false;       // the lane's first interval began in an earlier lane
  bool scan_flag = true;       // the lane's last interval begins in this lane
  int scan_lv = 0;             // shuffle levels that close every interval
  unsigned scan_add = 0;       // bit l: the lane adds the sum from lane - 2^l at scan level l
  if (has_z) {
#pragma unroll
    for (int r = 0; r < MU; ++r) { mmr[r] = TMIs[ub + r]; wr[r] = TMWs[ub + r]; }
    const int nxt = __shfl_down_sync(SFD_FULL, mmr[0], 1);
    const int prv = __shfl_up_sync(SFD_FULL, mmr[MU - 1], 1);
#pragma unroll
    for (int r = 0; r < MU - 1; ++r)
      if (mmr[r + 1] != mmr[r]) lastm |= 1u << r;
    if (lane == kWarp - 1 || nxt != mmr[MU - 1]) lastm |= 1u << (MU - 1);
#pragma unroll
    for (int r = 0; r < MU; ++r)
      if (ub + r >= n_u) lastm &= ~(1u << r);   // pad rows store nothing
    carry_ok = lane > 0 && prv == mmr[0];
    scan_flag = !(lane > 0 && prv == mmr[MU - 1]);
    bool f = scan_flag;
    for (int l = 0; l < 5 && !__all_sync(SFD_FULL, f); ++l) {
      const int sh = 1 << l;
      const bool fu = __shfl_up_sync(SFD_FULL, f ? 1 : 0, sh) != 0;
      if (lane >= sh) {
        if (!f) scan_add |= 1u << l;
        f = f || fu;
      }
      scan_lv = l + 1;
    }
  }
  // A longitudinal field interpolated to the lane's transverse row r (the
  // row's transfer map is held in registers; pad rows read the zero cell).
  auto interp_zr = [&](const float* A, int r) {
    const int mm = mmr[r];
    const float w = wr[r];
    return (1.f - w) * A[mm - 1] + w * A[mm];
  };
  // Interval sums of (1 - w) f and w f for NF fields at once (independent
  // chains interleaved), stored into their slot pairs.
  auto emit2 = [&](const float (&f)[MU], float* S0, float* S1, const float (&g)[MU], float* T0, float* T1,
                   bool two) {
    float a0[MU], a1[MU], b0[MU], b1[MU];
#pragma unroll
    for (int r = 0; r < MU; ++r) {
      const float p0 = (1.f - wr[r]) * f[r], p1 = wr[r] * f[r];
      const float q0 = (1.f - wr[r]) * g[r], q1 = wr[r] * g[r];
      const bool cont = r > 0 && mmr[r] == mmr[r > 0 ? r - 1 : 0];
      a0[r] = cont ? a0[r > 0 ? r - 1 : 0] + p0 : p0;
      a1[r] = cont ? a1[r > 0 ? r - 1 : 0] + p1 : p1;
      b0[r] = cont ? b0[r > 0 ? r - 1 : 0] + q0 : q0;
      b1[r] = cont ? b1[r > 0 ? r - 1 : 0] + q1 : q1;
    }
    float v0 = a0[MU - 1], v1 = a1[MU - 1], x0 = b0[MU - 1], x1 = b1[MU - 1];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      if (l >= scan_lv) break;
      const int sh = 1 << l;
      const float u0 = __shfl_up_sync(SFD_FULL, v0, sh), u1 = __shfl_up_sync(SFD_FULL, v1, sh);
      float y0 = 0.f, y1 = 0.f;
      if (two) {
        y0 = __shfl_up_sync(SFD_FULL, x0, sh);
        y1 = __shfl_up_sync(SFD_FULL, x1, sh);
      }
      if ((scan_add >> l) & 1u) { v0 += u0; v1 += u1; x0 += y0; x1 += y1; }
    }
    float c0 = __shfl_up_sync(SFD_FULL, v0, 1), c1 = __shfl_up_sync(SFD_FULL, v1, 1);
    float d0 = 0.f, d1 = 0.f;
    if (two) {
      d0 = __shfl_up_sync(SFD_FULL, x0, 1);
      d1 = __shfl_up_sync(SFD_FULL, x1, 1);
    }
#pragma unroll
    for (int r = 0; r < MU; ++r) {
      if (!((lastm >> r) & 1u)) continue;
      const bool add = carry_ok && mmr[r] == mmr[0];
      S0[mmr[r]] = add ? a0[r] + c0 : a0[r];
      S1[mmr[r] + 1] = add ? a1[r] + c1 : a1[r];
      if (two) {
        T0[mmr[r]] = add ? b0[r] + d0 : b0[r];
        T1[mmr[r] + 1] = add ? b1[r] + d1 : b1[r];
      }
    }
  };
  auto emit = [&](const float (&f)[MU], float* S0, float* S1) { emit2(f, S0, S1, f, S0, S1, false); };
  auto spreadS = [&](const float* S0, const float* S1, int i) { return S0[i + 1] + S1[i + 1]; };

  // ---- constant matrices ----
  Red rdu, rdz;
  const float dz_diag = 1.f + s0 + 2.f * s1l;
  const float dz_inv = fast_rcp(dz_diag);
  auto z_axpy = [&](float a) {        // AZ += a XZ over the lane's longitudinal rows
    z_rows(m_z, lane, [&](int i, float& v, float&) { v = fmaf(a, XZ[i], AZ[i]); },
           [&](int i, float v, float) { AZ[i] = v; }, kz0, kzs);
  };
  if (has_z && !zjac) {
    for (int r = 0; r < m_z; ++r) {
      const int i = lane * m_z + r;
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
  float SB[MU], IV[MU], CPr[MU], FFr[MU], GGr[MU];
  // unfactored diagonal and superdiagonal, kept for the refinement residual
  // (single-row lanes only: the strings that refine have at most 31 rows)
  float DG0[MU], CP0[MU];
  const bool refine = MU == 1 && Dp->refine != 0;
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    const int i = ub + r;
    if (i < n_u) {
      SB[r] = i > 0 ? og : 0.f;
      IV[r] = dg;
      CPr[r] = i < n_u - 1 ? og : 0.f;
    } else {
      SB[r] = 0.f; IV[r] = 1.f; CPr[r] = 0.f;
    }
    DG0[r] = IV[r];
    CP0[r] = CPr[r];
  }
  const bool forced = exc != kPluck;
  int en = Dp->e_node;              // excitation point (a bow envelope moves it per step)
  float ew = Dp->e_w;
  const float js = Dp->jscale;
  const int benv = exc == kBow ? Dp->bow_env_n : 0;
  float bv = bow_v;                 // the step's bow velocity
  float XP[MU];
  auto load_J = [&](float (&E)[MU]) {
#pragma unroll
    for (int r = 0; r < MU; ++r) {
      const int i = ub + r;
      float v = 0.f;
      if (i == en - 1) v += (1.f - ew) * js;
      if (i == en) v += ew * js;
      E[r] = (i < n_u) ? v : 0.f;
    }
  };
#pragma unroll
  for (int r = 0; r < MU; ++r) XP[r] = 0.f;
  if (linear) {
    tri_factor_r<MU>(SB, IV, CPr, FFr, GGr, lane, rdu);
    if (forced) {
      load_J(XP);
      tri_solve_r<MU, 1>(SB, IV, CPr, FFr, GGr, XP, XP, lane, rdu);
    }
  }
  __syncwarp();

  // One step of iterative refinement of the transverse solve A x = b: the
  // residual against the unfactored entries (exact floats for a linear
  // string) is solved with the same factors and added, which removes the
  // lasting error of the FP32 factorisation from the solution.
  auto refine_solve = [&](const float (&b)[MU], float (&x)[MU]) {
    float xe[MU + 2], rr[MU];
    extend1<MU>(x, xe, lane);
#pragma unroll
    for (int r = 0; r < MU; ++r) rr[r] = b[r] - (SB[r] * xe[r] + DG0[r] * xe[r + 1] + CP0[r] * xe[r + 2]);
    tri_solve_r<MU, 1>(SB, IV, CPr, FFr, GGr, rr, rr, lane, rdu);
#pragma unroll
    for (int r = 0; r < MU; ++r) x[r] += rr[r];
  };

  const int on = Dp->o_node, oln = Dp->ol_node;
  const float ow = Dp->o_w, olw = Dp->ol_w, oscale = Dp->out_scale;
  const bool zout = Dp->out_ch == 1;
  const int64_t j_end = jnext + job.n_samples;
  float outbuf = 0.f;
  int64_t opos = 0;
  float AC[MU];

  while (jnext < j_end) {
    if (jnext > n && !(status & kStUnstable)) {
      // ======================= one step n -> n+1 =======================
      const float rm = mod_factor(mod_kind, mod_inc_fx, mod_phase_fx, mod_depth2, mod_inc, mod_hold, mod_n_end, n);
      const float lam2 = lam2_0 * rm, lam2l = lam2l_0 * rm;
      // low part of lam2_0 * rm (exact product residual plus the stored low part)
      const float lam2_lo = fmaf(lam2_0, rm, -lam2) + lam2lo_0 * rm;
      const float ca = ca_0 * rm, cb = cb_0 * rm, cz = cz_0 * rm;

      float eta = 0.f, k2G = 0.f, FB = 0.f;
      float vrec = 0.f;   // bow: relative velocity of the step (0 while sticking), for the adjoint
      if (exc == kHammer) {
        eta = uh - node_interp<MU>(U, en, ew, n_u);
        if (eta > 0.f) k2G = ham_k2w * powf(eta, ham_expo);
      } else if (exc == kBow) {
        float bf = bow_F;
        if (benv > 0) {
          const int en0 = en;
          const float ew0 = ew;
          bow_env_eval(Dp, n, bv, bf, en, ew);
          if (linear && (en != en0 || ew != ew0)) {   // the fixed-matrix response A^-1 J follows x_B
            load_J(XP);
            tri_solve_r<MU, 1>(SB, IV, CPr, FFr, GGr, XP, XP, lane, rdu);
          }
        }
        FB = (n < bow_release_n) ? bf : 0.f;
      }
      const bool need_resp = !linear && ((exc == kHammer && k2G > 0.f) || (exc == kBow && FB > 0.f));

      // ---- stage 1: transverse right-hand side and matrix (registers) ----
      float Ue[MU + 4], DUe[MU + 2], GL[MU], GR[MU];
      extend<MU>(U, Ue, lane);
      extend1<MU>(DU, DUe, lane);
#pragma unroll
      for (int r = 0; r < MU; ++r) {   // interval differences; zero on pad rows
        const bool real = ub + r < n_u;
        GL[r] = real ? Ue[r + 2] - Ue[r + 1] : 0.f;
        GR[r] = real ? Ue[r + 3] - Ue[r + 2] : 0.f;
      }
      float ZTe[MU + 2];
      if (has_z) {
        float zt[MU];
#pragma unroll
        for (int r = 0; r < MU; ++r) zt[r] = interp_zr(Z, r);
        extend1<MU>(zt, ZTe, lane);
      }
      float RA[MU], fv[MU];
#pragma unroll
      for (int r = 0; r < MU; ++r) {
        const int i = ub + r;
        fv[r] = 0.f;
        const float u0 = Ue[r + 2], um1 = Ue[r + 1], up1 = Ue[r + 3], um2 = Ue[r], up2 = Ue[r + 4];
        const float gl = GL[r], gr = GR[r];
        const float d2 = gr - gl;
        float d4 = ((up2 - up1) - gr) - 2.f * d2 + (gl - (um1 - um2));
        if (i == 0) d4 += bsgn * u0;
        if (i == n_u - 1) d4 += bsgn * u0;
        const float du0 = DUe[r + 1];
        const float d2du = (DUe[r + 2] - du0) - (du0 - DUe[r]);
        float rhs = fmaf(lam2, d2, lam2_lo * d2) - mu2 * d4 - 2.f * s0u * du0 + 2.f * s1 * d2du;
        if (!linear) {
          const float gl2 = gl * gl, gr2 = gr * gr;
          float yl = 2.f * ca * gl2 * gl, yr = 2.f * ca * gr2 * gr;
          if (has_z) {
            yl += 4.f * cb * gl * (ZTe[r + 1] - ZTe[r]);
            yr += 4.f * cb * gr * (ZTe[r + 2] - ZTe[r + 1]);
            fv[r] = gr2 - gl2;   // zero on pad rows
          }
          rhs += yr - yl;
          const bool real = i < n_u;
          SB[r] = (real && i > 0) ? og - ca * gl2 : 0.f;
          IV[r] = real ? dg + ca * (gl2 + gr2) : 1.f;
          CPr[r] = i < n_u - 1 ? og - ca * gr2 : 0.f;
          DG0[r] = IV[r];
          CP0[r] = CPr[r];
        }
        RA[r] = i < n_u ? rhs : 0.f;
      }
      if (has_z) emit(fv, SF0, SF1);
      if (!linear) tri_factor_r<MU>(SB, IV, CPr, FFr, GGr, lane, rdu);
      __syncwarp();

      if (!has_z) {
#pragma unroll
        for (int r = 0; r < MU; ++r) AC[r] = RA[r];
        if (need_resp) {
          load_J(XP);
          tri_solve_r<MU, 2>(SB, IV, CPr, FFr, GGr, AC, XP, lane, rdu);
        } else {
          tri_solve_r<MU, 1>(SB, IV, CPr, FFr, GGr, AC, AC, lane, rdu);
        }
        if (refine) refine_solve(RA, AC);
      } else {
        // ---- stage 2: longitudinal right-hand side ----
        float dzmax = 0.f;   // lane's largest |Dz|: scale of the longitudinal increments
        {
          auto rhs_row = [&](int i) {
            const float z0 = Z[i], dz0 = DZ[i];
            const float d2z = (Z[i + 1] - z0) - (z0 - Z[i - 1]);
            const float d2dz = (DZ[i + 1] - dz0) - (dz0 - DZ[i - 1]);
            dzmax = fmaxf(dzmax, fabsf(dz0));
            const float v = lam2l * d2z - 2.f * s0 * dz0 + 2.f * s1l * d2dz + 2.f * cz * spreadS(SF0, SF1, i);
            return i < n_z ? v : 0.f;
          };
          auto st = [&](int i, float v, float) { RZ_[i] = v; };
          z_rows(m_z, lane, [&](int i, float& v, float&) { v = rhs_row(i); }, st, kz0, kzs);
        }
        __syncwarp();
        // ---- stage 3: block Gauss-Seidel on (a, az) [and the response] ----
        int sweep = 0;
        float e_prev = 0.f, mag_all = 0.f, mgx_all = 0.f;
        for (;;) {
          float az[MU], AZe[MU + 2];
#pragma unroll
          for (int r = 0; r < MU; ++r) az[r] = interp_zr(AZ, r);
          extend1<MU>(az, AZe, lane);
#pragma unroll
          for (int r = 0; r < MU; ++r)
            AC[r] = RA[r] + cb * (GR[r] * (AZe[r + 2] - AZe[r + 1]) - GL[r] * (AZe[r + 1] - AZe[r]));
          float BC[MU];
#pragma unroll
          for (int r = 0; r < MU; ++r) BC[r] = AC[r];
          if (need_resp) {
            float xz[MU], XZe[MU + 2];
#pragma unroll
            for (int r = 0; r < MU; ++r) xz[r] = interp_zr(XZ, r);
            extend1<MU>(xz, XZe, lane);
            load_J(XP);
#pragma unroll
            for (int r = 0; r < MU; ++r)
              XP[r] += cb * (GR[r] * (XZe[r + 2] - XZe[r + 1]) - GL[r] * (XZe[r + 1] - XZe[r]));
            tri_solve_r<MU, 2>(SB, IV, CPr, FFr, GGr, AC, XP, lane, rdu);
          } else {
            tri_solve_r<MU, 1>(SB, IV, CPr, FFr, GGr, AC, AC, lane, rdu);
          }
          if (refine) refine_solve(BC, AC);
          // nodal d_+[g d(.)] of the new accelerations for the longitudinal rows
          {
            float ACe[MU + 2], fc[MU], fx[MU];
            extend1<MU>(AC, ACe, lane);
#pragma unroll
            for (int r = 0; r < MU; ++r)
              fc[r] = GR[r] * (ACe[r + 2] - ACe[r + 1]) - GL[r] * (ACe[r + 1] - ACe[r]);
            if (need_resp) {
              float XPe[MU + 2];
              extend1<MU>(XP, XPe, lane);
#pragma unroll
              for (int r = 0; r < MU; ++r)
                fx[r] = GR[r] * (XPe[r + 2] - XPe[r + 1]) - GL[r] * (XPe[r + 1] - XPe[r]);
              emit2(fc, SF0, SF1, fx, SX0, SX1, true);
            } else {
              emit(fc, SF0, SF1);
            }
          }
          __syncwarp();
          float chg = 0.f, mag = 0.f, chx = 0.f, mgx = 0.f;
          if (zjac) {
            // one Jacobi update of each field into the spare buffer, then swap
            auto jac = [&](int i, float& v, float& x) {
              const bool real = i < n_z;
              v = (RZ_[i] + cz * spreadS(SF0, SF1, i) + s1l * (AZ[i - 1] + AZ[i + 1])) * dz_inv;
              v = real ? v : 0.f;
              chg = fmaxf(chg, fabsf(v - AZ[i]));
              mag = fmaxf(mag, fabsf(v));
              if (need_resp) {
                x = (cz * spreadS(SX0, SX1, i) + s1l * (XZ[i - 1] + XZ[i + 1])) * dz_inv;
                x = real ? x : 0.f;
                chx = fmaxf(chx, fabsf(x - XZ[i]));
                mgx = fmaxf(mgx, fabsf(x));
              }
            };
            auto st = [&](int i, float v, float x) {
              E2Z[i] = v;
              if (need_resp) E3Z[i] = x;
            };
            z_rows(m_z, lane, jac, st, kz0, kzs);
            __syncwarp();
            { float* t = AZ; AZ = E2Z; E2Z = t; }
            if (need_resp) { float* t = XZ; XZ = E3Z; E3Z = t; }
          } else {
            for (int r = 0; r < m_z; ++r) {
              const int i = lane * m_z + r;
              E1Z[i] = i < n_z ? RZ_[i] + cz * spreadS(SF0, SF1, i) : 0.f;
            }
            tri_solve(SUBZ, INVZ, CPZ, FFZ, GGZ, E1Z, m_z, lane, rdz);
            for (int r = 0; r < m_z; ++r) {
              const int i = lane * m_z + r;
              const float v = E1Z[i];
              chg = fmaxf(chg, fabsf(v - AZ[i]));
              mag = fmaxf(mag, fmaxf(fabsf(v), fabsf(DZ[i])));
              AZ[i] = v;
            }
            if (need_resp) {
              for (int r = 0; r < m_z; ++r) {
                const int i = lane * m_z + r;
                E1Z[i] = i < n_z ? cz * spreadS(SX0, SX1, i) : 0.f;
              }
              tri_solve(SUBZ, INVZ, CPZ, FFZ, GGZ, E1Z, m_z, lane, rdz);
              for (int r = 0; r < m_z; ++r) {
                const int i = lane * m_z + r;
                const float v = E1Z[i];
                chx = fmaxf(chx, fabsf(v - XZ[i]));
                mgx = fmaxf(mgx, fabsf(v));
                XZ[i] = v;
              }
            }
          }
          // relative change: each field against the larger of its magnitude
          // in this lane and its string-wide scale from the previous step,
          // so one warp reduction per sweep suffices
          mag = fmaxf(mag, dzmax);
          if (paired) {
            // each lane's maxima over the group's rows: the other warps'
            // updates are in shared memory once all pass the barrier
            float* xc = xcell + xpar * 512;
            xc[pw * 128 + lane] = chg;
            xc[pw * 128 + 32 + lane] = mag;
            xc[pw * 128 + 64 + lane] = chx;
            xc[pw * 128 + 96 + lane] = mgx;
            group_sync(bar_id, ng);
            for (int w = 0; w < ng; ++w) {
              const float* xo = xc + w * 128;
              chg = fmaxf(chg, xo[lane]);
              mag = fmaxf(mag, xo[32 + lane]);
              chx = fmaxf(chx, xo[64 + lane]);
              mgx = fmaxf(mgx, xo[96 + lane]);
            }
            xpar ^= 1;
          }
          // (a measure compared with thresholds: the fast divide suffices)
          float el = chg > 0.f ? __fdividef(chg, fmaxf(mag, scz)) : 0.f;
          if (need_resp) el = fmaxf(el, chx > 0.f ? __fdividef(chx, fmaxf(mgx, scx)) : 0.f);
          mag_all = fmaxf(mag_all, mag);
          mgx_all = fmaxf(mgx_all, mgx);
          const float e = warp_max_nonneg(el);
          ++sweep;
          if (sweep_converged(e, e_prev, sweep)) break;
          if (sweep >= sweep_cap) { status |= kStNoConv; break; }
          e_prev = e;
        }
        sweeps_total += sweep;
        if (sweep > max_sweeps) max_sweeps = sweep;
        // string-wide scales for the next step's convergence test
        scz = warp_max_nonneg(mag_all);
        if (need_resp) scx = warp_max_nonneg(mgx_all);
      }

      // ---- stage 4: excitation force (scalar elimination) ----
      if (exc == kHammer) {
        float s = 0.f;
        if (k2G > 0.f) {
          const float cm = 0.5f * ham_M * k2G;
          s = cm * (2.f * eta - node_interp<MU>(AC, en, ew, n_u)) /
              (1.f + 0.5f * k2G + cm * node_interp<MU>(XP, en, ew, n_u));
          duh -= s / ham_M;
        }
        uh += duh;
        if (s != 0.f) {
#pragma unroll
          for (int r = 0; r < MU; ++r) AC[r] = fmaf(s, XP[r], AC[r]);
          if (has_z) z_axpy(s);
        }
      } else if (exc == kBow && FB > 0.f) {
        const float b = (node_interp<MU>(AC, en, ew, n_u) + 2.f * node_interp<MU>(DU, en, ew, n_u)) * inv2k -
                        bv;
        const float c = 0.5f * kk * FB * node_interp<MU>(XP, en, ew, n_u);
        const float phi = bow_phi(b, c, bow_a, bow_eps, bow_w);
        vrec = !(c > 0.f) ? b : (fabsf(b) <= c ? 0.f : b - c * phi);
        const float s = -k2 * FB * phi;
#pragma unroll
        for (int r = 0; r < MU; ++r) AC[r] = fmaf(s, XP[r], AC[r]);
        if (has_z) z_axpy(s);
      }

      // ---- stage 5: advance the time level ----
      bool bad = false;
#pragma unroll
      for (int r = 0; r < MU; ++r) {   // pad rows stay zero (their accelerations are zero)
        DU[r] = DU[r] + AC[r];
        U[r] = U[r] + DU[r];
        bad |= !isfinite(U[r]);
      }
      if (has_z) {
        z_rows(m_z, lane, [&](int i, float& d, float& z) { d = DZ[i] + AZ[i]; z = Z[i] + d; },
               [&](int i, float d, float z) { DZ[i] = d; Z[i] = z; }, kz0, kzs);
      }
      if (__any_sync(SFD_FULL, bad)) status |= kStUnstable;
      __syncwarp();
      if (paired) group_sync(bar_id, ng);   // the new level is complete in shared memory
      ++n;
      if (job.traj && writer) {   // replay for the adjoint: record the new level
        float* rec = job.traj + (n - n_first - 1) * job.traj_stride;
#pragma unroll
        for (int r = 0; r < MU; ++r) {
          const int i = ub + r;
          if (i < n_u) { rec[i] = U[r]; rec[n_u + i] = DU[r]; }
        }
        for (int i = lane; i < n_z; i += kWarp) { rec[2 * n_u + i] = Z[i]; rec[2 * n_u + n_z + i] = DZ[i]; }
        // (a bowed string has no hammer state: its slot holds the step's bow velocity)
        if (lane == 0) { rec[2 * n_u + 2 * n_z] = exc == kBow ? vrec : uh; rec[2 * n_u + 2 * n_z + 1] = duh; }
      }
    }
    float y;
    if (zout) {   // L zeta^j at the pickup (zero without a longitudinal grid)
      y = 0.f;
      if (has_z) {
        y = zinterp(Z, oln, olw, n_z);
        if (jnext == n - 1) y -= zinterp(DZ, oln, olw, n_z);
      }
    } else if (jnext == n - 1) {
      y = node_interp<MU>(U, on, ow, n_u) - node_interp<MU>(DU, on, ow, n_u);
    } else {
      y = node_interp<MU>(U, on, ow, n_u);
    }
    y *= oscale;
    if (status & kStUnstable) y = 0.f;
    if ((opos & (kWarp - 1)) == lane) outbuf = y;
    ++opos;
    if ((opos & (kWarp - 1)) == 0 && writer) job.out[opos - kWarp + lane] = outbuf;
    ++jnext;
  }
  {
    const int rem = static_cast<int>(opos & (kWarp - 1));
    if (lane < rem && writer) job.out[opos - rem + lane] = outbuf;
  }

  // ---- store the state ----
  __syncwarp();
  if (!writer) return;
#pragma unroll
  for (int r = 0; r < MU; ++r) {
    const int i = ub + r;
    if (i < n_u) { Dp->u[i] = U[r]; Dp->du[i] = DU[r]; }
  }
  for (int i = lane; i < n_z; i += kWarp) {
    Dp->z[i] = Z[i]; Dp->dz[i] = DZ[i]; Dp->xz[i] = XZ[i]; Dp->az[i] = AZ[i];
  }
  if (lane == 0) {
    scp->n = n;
    scp->next_out = jnext;
    scp->uh = uh;
    scp->duh = duh;
    scp->bow_w = bow_w;
    scp->scale_z = scz;
    scp->scale_x = scx;
    scp->status = status;
    scp->max_sweeps = max_sweeps;
    scp->sweeps_total = sweeps_total;
  }
  __syncwarp();
}

}  // namespace sfd
