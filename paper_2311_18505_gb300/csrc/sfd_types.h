// Internal layout shared by the host runtime (sfd_api.cu) and the step
// kernel (sfd_kernel.cu).  All coefficients are computed on the host in
// FP64 from the string parameters and rounded once to FP32.
#pragma once

#include <stdint.h>

namespace sfd {

constexpr int kWarp = 32;
constexpr int kMaxSweeps = 24;       // default cap of the coupled block Gauss-Seidel solve
constexpr int kMaxSweepCap = 64;     // largest cap a context may set
constexpr float kSweepTol = 5e-7f;   // relative change that ends the solve

enum ExcKind : int32_t { kPluck = 0, kHammer = 1, kBow = 2 };
enum StatusBits : int32_t { kStUnstable = 1, kStNoConv = 2 };

// Per-string mutable scalars (device memory).
struct Scalars {
  float uh, duh;          // hammer u_H^n and u_H^n - u_H^{n-1} (normalised)
  int64_t n;              // time level (state holds w^{n-1}, w^n)
  int64_t next_out;       // index of the next output sample
  int32_t status;         // StatusBits
  int32_t max_sweeps;     // largest sweep count seen (diagnostic)
  int64_t sweeps_total;   // total coupled-solve sweeps (diagnostic)
  float bow_w;            // last bow slip speed |v_rel| (Newton warm start)
  float scale_z;          // string-wide scale of the longitudinal increment (solver test)
  float scale_x;          // string-wide scale of the unit-force response (solver test)
  float pad_;
};

// Per-string descriptor (device memory, read-only in the kernel).
struct Desc {
  // grid: N_t, N_l intervals; n_u = N_t - 1, n_z = N_l - 1 unknowns;
  // m_u, m_z rows per lane (odd, 32 m >= n + 1; m_z = 0 without z).
  int32_t n_t, n_l, n_u, n_z, m_u, m_z;
  int32_t boundary;       // 0 clamped, 1 simply supported
  int32_t exc;            // ExcKind
  int32_t linear;         // alpha == 1: z stays zero, matrix constant
  int32_t mod_kind;       // 0 none, 1 vibrato, 2 glissando
  int32_t z_jacobi;       // longitudinal off-diagonal folded into the sweeps
  int32_t refine;         // one step of iterative refinement per transverse solve
  // delta-form coefficients (k^2-scaled Eq. 4), see the kernel.  The
  // transverse equation (dg, og, s0u, s1, lam2, mu2, ca, cb, jscale) is
  // multiplied by a scale beta that makes dg and og exact floats.
  float dg, og;           // beta (theta + s0 + 2 s1), beta ((1 - theta)/2 - s1)
  float s0, s1, s1l;      // sigma0 k (longitudinal), beta sigma1 k / h_t^2, sigma1 k / h_l^2
  float s0u;              // beta sigma0 k (transverse)
  float lam2, mu2, lam2l; // g^2 k^2 / h_t^2, kappa^2 k^2 / h_t^4, g^2 alpha^2 k^2 / h_l^2
  float ca, cb, cz;       // phi' k^2 / (2 h_t^4), phi' k^2 / (2 h_t^3), phi' k^2 / (2 h_t^2 h_l)
  float out_scale;        // L (output in metres)
  int32_t o_node;         // pickup: nodes o_node, o_node + 1 (0..N_t)
  float o_w;              //   weight of o_node + 1
  int32_t out_ch;         // 0: L u at the pickup, 1: L zeta at the pickup
  int32_t ol_node;        // pickup on the longitudinal grid: nodes ol_node, ol_node + 1 (0..N_l)
  float ol_w;             //   weight of ol_node + 1
  int32_t e_node;         // excitation point, same convention
  float e_w;
  float jscale;           // J = I / h_t
  // hammer (Eq. 6)
  float ham_M;            // mass ratio M
  float ham_k2w;          // k^2 omega_H^{1 + alpha_H}
  float ham_expo;         // alpha_H - 1
  // bow (Eq. 5)
  float bow_F;            // F_B / (rho A L^2)
  float bow_v;            // v_B / L
  float bow_a;            // a L
  float bow_eps;
  float k;                // time step
  float k2;               // k^2
  int64_t bow_release_n;  // first step index with F_B = 0 (INT64_MAX: never)
  // modulation: factor (gamma^n / gamma)^2 per step (mod_factor)
  uint64_t mod_inc_fx;    // vibrato: f_v k cycles per step, as a 64-bit fixed-point fraction
  uint64_t mod_phase_fx;  // vibrato: phase / (2 pi), the same
  int64_t mod_n_end;      // glissando: first step n with n k >= T (held from there on)
  float mod_depth2;       // vibrato: 2 c / 1200
  float mod_inc;          // glissando: 2 D k / T per step
  float mod_hold;         // glissando: 2 D
  float lam2_lo;          // lam2 + lam2_lo: wave coefficient to ~1e-15 (see fill_desc)
  // time-varying bow controls (Sec. 3.3.1): bow_env_n breakpoints (0: the
  // constant bow_v, bow_F, e_node / e_w), at steps bow_env_t (t fs) with
  // v_B / L, F_B / (rho A L^2) and x_B; linear between, held outside
  int32_t bow_env_n;
  int32_t pad_env_;
  double bow_env_t[16];
  float bow_env_v[16], bow_env_f[16], bow_env_x[16];
  // state (device pointers into the string's pool block)
  float* u;               // u^n            [n_u]
  float* du;              // u^n - u^{n-1}  [n_u]
  float* z;               // z^n            [n_z]
  float* dz;              // z^n - z^{n-1}  [n_z]
  float* xz;              // z-part of the unit-force response (warm start) [n_z]
  float* az;              // last longitudinal acceleration (warm start) [n_z]
  Scalars* sc;
};

// One unit of work for the persistent kernel.
struct Job {
  const Desc* desc;
  float* out;             // first output sample of this job
  int64_t n_samples;
  // optional trajectory record (gradient replay): after each step of the
  // job, the new level's [u | D | z | Dz | u_H | D_H] at traj + k stride
  // for the job's k-th step; nullptr: not recorded
  float* traj;
  int64_t traj_stride;
  int32_t sweep_cap;      // largest Gauss-Seidel sweep count per step (0: kMaxSweeps)
  int32_t pad_;
};

// One string's part of a reverse sweep of the discrete adjoint over the
// levels (m_start, m_end] of a replayed segment (sfd_adjoint.cu).
enum GradSlot : int {
  kGLam2 = 0, kGMu2, kGS0u, kGS1, kGCa, kGCb, kGCz, kGLam2l, kGS0, kGS1l, kGAmp, kGradSlots
};
struct AdjJob {
  const Desc* desc;            // coefficients and grid (the replayed string)
  const float* u0;             // state at level m_start (a checkpoint): u, D, z, Dz
  const float* du0;
  const float* z0;
  const float* dz0;
  const Scalars* sc0;          // ... and u_H, D_H
  const float* traj;           // levels m_start + 1 .. m_end (Job::traj layout)
  int64_t traj_stride;
  int64_t m_start, m_end;
  const float* dy;             // dJ/dy for the string's samples (index = level)
  double* adj;                 // adjoint of [u | D | z | Dz | u_H | D_H], level m_end in, m_start
                               // out; then the warm starts of the two longitudinal solves (2 n_z)
  double* grad;                // kGradSlots accumulators (raw coefficient gradients)
  int32_t first;               // m_start == 1: add the level-1 and level-0 outputs, initial-state terms
  float pluck_pos;             // peak of the pluck triangle (amplitude gradient), < 0: none
};

// Shared-memory words one warp needs for a string with row counts m_u, m_z.
// Up to kMaxRegRows transverse rows per lane live in registers (2 transverse
// transfer arrays in shared memory); larger grids use the shared-memory path.
constexpr int kMaxRegRows = 9;
// static shared memory of the register-path kernels (the warp pairs'
// exchange cells and job index cells); dynamic regions get the rest
constexpr int kStaticSmemBytes = 2 * 1024 * 4 + 4 * 4;
constexpr int kArraysU = 19;
constexpr int kArraysZ = 15;
inline __host__ __device__ int warp_smem_floats(int m_u, int m_z, int z_jacobi) {
  const int ru = kWarp * m_u + 4, rz = m_z > 0 ? kWarp * m_z + 4 : 0;
  if (m_u <= kMaxRegRows && (m_u & 1)) return 2 * ru + (z_jacobi ? 12 : 18) * rz;
  return kArraysU * ru + kArraysZ * rz;
}

// ... and the shared-memory bytes of the adjoint sweep: 17 FP64 and 9 FP32
// (or int) transverse arrays, 13 FP64 and 6 FP32 longitudinal ones.
inline __host__ __device__ int adj_smem_bytes(int m_u, int m_z) {
  const int ru = kWarp * m_u + 4, rz = m_z > 0 ? kWarp * m_z + 4 : 0;
  return (17 * 8 + 9 * 4) * ru + (13 * 8 + 6 * 4) * rz;
}

}  // namespace sfd
