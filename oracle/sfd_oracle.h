/*
 * FP64 CPU oracle for the nonlinear planar stiff-string finite-difference
 * scheme of "String Sound Synthesizer on GPU-Accelerated Finite Difference
 * Scheme" (Lee, Choi, Lee; arXiv 2311.18505).
 *
 * TEST INFRASTRUCTURE. This library is a plain, slow, step-by-step FP64
 * restatement of the scheme (Sec. 3, Eqs. 4-9) used only to check the CUDA
 * path: the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does. It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Conventions (all readings are listed in the design notes):
 *  - x is normalised to [0,1]; u and zeta are displacements divided by the
 *    length L (Table 1 defines gamma = L^-1 sqrt(T0/rho A), so f0 = gamma/2).
 *  - transverse grid: N_t intervals, h_t = 1/N_t, unknowns u_1..u_{N_t-1};
 *    longitudinal grid: N_l intervals, h_l = 1/N_l, unknowns z_1..z_{N_l-1}
 *    (Sec. 3.4, the state vector w = [u; z]).
 *  - the nonlinear term carries the "+" sign of Eq. 4.
 *  - loss enters as 2 sigma0 delta_t. and 2 sigma1 delta_t. delta_xx (Eq. 4).
 *  - the transverse-to-longitudinal transfer is S = (h_t/h_l) R^T where R is
 *    the overlap-weight form of D_x- I_(l->t) with a linear interpolant.
 *  - time-varying bow controls (Sec. 3.3.1) are piecewise linear in time;
 *    the step n -> n+1 takes them at t = n k, and I, J sit at x_B(t).
 *
 * Parity status: pinned (modal closed forms, energy invariant, stability
 * bound, dense brute force on tiny grids, special cases). The bowed string
 * is pinned at every step by its exact power budget and friction law and
 * by the brute force over the steps that covers; a bowed note near a
 * bifurcation that FP32-sized rounding crosses cannot be followed by an
 * FP32 run beyond it, so there only its level is compared.
 */
#ifndef SFD_ORACLE_H
#define SFD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SFDO_EXC_PLUCK = 0, SFDO_EXC_HAMMER = 1, SFDO_EXC_BOW = 2 };
enum { SFDO_MOD_NONE = 0, SFDO_MOD_VIBRATO = 1, SFDO_MOD_GLISS = 2 };

/* One string and its excitation, SI units at this boundary.
 * Field order and types are mirrored by the Python ctypes structure. */
typedef struct {
  double gamma;           /* wave speed [1/s] (f0 = gamma/2, Sec. 4.1)          */
  double kappa;           /* stiffness [1/s] (Table 1)                          */
  double alpha;           /* stiffness-to-tension ratio (Table 1)               */
  double sigma0;          /* frequency-independent loss [1/s] (Eq. 4)           */
  double sigma1;          /* frequency-dependent loss (Eq. 4)                   */
  double theta;           /* implicit-scheme free parameter (Sec. 3.2)          */
  double fs;              /* sample rate [Hz]; k = 1/fs (Sec. 3)                */
  double length;          /* L [m]                                              */
  double rho_a;           /* linear density rho*A [kg/m]                        */
  int32_t boundary;       /* 0 clamped (Sec. 4.1), 1 simply supported           */
  int32_t grid_rule;      /* 0 theta-consistent bound, 1 Sec. 3.2 literal       */
  int32_t n_t_override;   /* >0: use this N_t instead of the derived one        */
  int32_t n_l_override;   /* >0: use this N_l instead of the derived one        */
  double gamma_max_ratio; /* >=1: grid sized for gamma*ratio (modulation peak)  */
  double pickup;          /* output position, fraction of L                     */
  int32_t exc_kind;       /* SFDO_EXC_*                                         */
  int32_t pad0;
  double pluck_amp;       /* peak displacement [m] (c0 = amp/L, Table 1)        */
  double pluck_pos;       /* x_P, fraction of L                                 */
  double ham_mass;        /* hammer mass [kg]; M = mass/(rho A L)               */
  double ham_vel;         /* initial hammer velocity [m/s]                      */
  double ham_pos;         /* x_H, fraction of L                                 */
  double ham_omega;       /* omega_H [1/s] (Eq. 6)                              */
  double ham_alpha;       /* alpha_H (Eq. 6)                                    */
  double bow_vel;         /* v_B [m/s] (Eq. 5)                                  */
  double bow_force;       /* F_B [N] (Eq. 5)                                    */
  double bow_pos;         /* x_B, fraction of L                                 */
  double bow_a;           /* friction-curve a [s/m] (Sec. 3.3.1)                */
  double bow_eps;         /* friction-curve epsilon (Sec. 3.3.1)                */
  double bow_release;     /* time [s] from which F_B = 0; <0: never             */
  int32_t mod_kind;       /* SFDO_MOD_* (f0 modulation, abstract)               */
  int32_t pad1;
  double mod_rate;        /* vibrato rate [Hz]                                  */
  double mod_depth;       /* vibrato depth [cents] / glissando span [octaves]   */
  double mod_phase;       /* vibrato phase [rad]                                */
  double mod_duration;    /* glissando duration [s]                             */
  int32_t out_channel;    /* 0: transverse u, 1: longitudinal zeta (Sec. 4.2)   */
  int32_t bow_env_n;      /* bow: breakpoints of the control envelopes (0: none) */
  /* Time-varying bow controls (Sec. 3.3.1): breakpoint times [s] and v_B
   * [m/s], F_B [N], x_B at them; the step n -> n+1 takes the values at
   * t = n k, linear between breakpoints and held outside them. */
  double bow_env_t[16], bow_env_v[16], bow_env_f[16], bow_env_x[16];
} sfdo_spec;

typedef struct sfdo_string sfdo_string;

/* Grid sizes N_t, N_l for a spec (Sec. 3.2 spacing rules). 0 on success. */
int sfdo_grid(const sfdo_spec* s, int32_t* n_t, int32_t* n_l);

/* Create a string at time level n = 1 with w^0, w^1 set by the excitation.
 * Returns NULL on invalid input. */
sfdo_string* sfdo_create(const sfdo_spec* s);
void sfdo_destroy(sfdo_string* st);

/* Append n output samples y^j = L * I(x_o) u^j (out_channel 1: the
 * longitudinal L * I_l(x_o) zeta^j on the longitudinal grid), j = next
 * index ... to y.
 * Returns 0, or a negative code if the state became non-finite. */
int sfdo_run(sfdo_string* st, int64_t n, double* y);

/* Current time level n (state holds w^{n-1}, w^n). */
int64_t sfdo_time_level(const sfdo_string* st);

/* Copy the state: u^{n-1}, u^n (N_t-1 each), z^{n-1}, z^n (N_l-1 each) and
 * exc[6] = {u_H^{n-1}, u_H^n, P_last, G_last, v_last, F_last} where P_last is
 * the excitation power of the last step (Eq. 5/6 coupling, normalised units),
 * G_last the hammer stiffness coefficient used, v_last the bow relative
 * velocity and F_last the normalised force.  Any pointer may be NULL. */
int sfdo_get_state(const sfdo_string* st, double* u_prev, double* u,
                   double* z_prev, double* z, double* exc);

/* Overwrite u^{n-1}, u^n, z^{n-1}, z^n (NULL leaves a field unchanged). */
int sfdo_set_state(sfdo_string* st, const double* u_prev, const double* u,
                   const double* z_prev, const double* z);

/* Max relative residual |A w - b|/|b| of the last linear solve. */
double sfdo_last_residual(const sfdo_string* st);

/* Run n_str independent strings for n_samples[i] samples each into
 * y + offsets[i], using up to n_threads OpenMP threads (<=0: all).
 * Returns the number of threads used, or a negative code. */
int sfdo_run_batch(const sfdo_spec* specs, int32_t n_str,
                   const int64_t* n_samples, const int64_t* offsets,
                   double* y, int32_t n_threads);

/* Complex-step derivative (a second build of the same source with
 * -DSFDO_COMPLEX, where the scalar is a complex double; this function exists
 * only in that build).  Runs string s for n samples with parameter `which`
 * (0 kappa, 1 alpha, 2 sigma0, 3 sigma1, 4 the pluck amplitude, hammer
 * velocity or bow velocity) given the imaginary part h, and writes y (the
 * output) and dy = dy/d(parameter) = Im(y)/h, exact to rounding wherever the
 * path is smooth in the parameter (no hammer contact starting or ending, no
 * stick/slip switch, within the perturbation).  Use n_t_override and
 * n_l_override to hold the grid fixed.  0, or a negative code. */
int sfdo_cs_run(const sfdo_spec* s, int which, double h, int64_t n, double* y, double* dy);

#ifdef __cplusplus
}
#endif
#endif
