/*
 * FP64 CPU oracle of the nonlinear planar stiff-string scheme
 * (arXiv 2311.18505, Sec. 3, Eqs. 4-9).  TEST INFRASTRUCTURE ONLY: used by
 * the tests, the smoke check and the CPU-baseline leg of the benchmark,
 * never by the product path.  See sfd_oracle.h for the conventions.
 *
 * Each time step assembles the linearly-implicit system of Eq. 4 (the
 * matrix-vector form of Eqs. 7-9 written out entry by entry) for the
 * unknowns w^{n+1} = [u^{n+1}; z^{n+1}] (plus the hammer displacement when a
 * hammer is present, Eq. 6), stores it as a band matrix in position order
 * and solves it exactly by banded Gaussian elimination.  Nothing is blocked,
 * fused or iterated beyond what the scheme states.
 */
#include "sfd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_D 3.14159265358979323846

/* The scalar of the state, the system and the differentiable parameters.
 * Built a second time with -DSFDO_COMPLEX it is a complex double: a
 * parameter given an imaginary part i h then carries its derivative along
 * every operation (complex step: dy/dp = Im y / h, exact to rounding for a
 * smooth path).  Branches test real parts; |x| is continued analytically as
 * sign(Re x) x.  With plain doubles the macros are the usual functions. */
#ifdef SFDO_COMPLEX
#include <complex.h>
typedef double complex num_t;
#define RE(x) creal(x)
#define NEXP(x) cexp(x)
#define NPOW(x, y) cpow((x), (y))
#define NABS(x) (creal(x) < 0 ? -(x) : (x))
#define NMAG(x) cabs(x)
#else
typedef double num_t;
#define RE(x) (x)
#define NEXP(x) exp(x)
#define NPOW(x, y) pow((x), (y))
#define NABS(x) fabs(x)
#define NMAG(x) fabs(x)
#endif

struct sfdo_string {
  sfdo_spec p;
  int nt, nl;            /* intervals N_t, N_l (Sec. 3, Eq. 3 notation)      */
  int nu, nz;            /* unknowns N_t-1, N_l-1 (Sec. 3.4)                 */
  double ht, hl, k;      /* spacings and time step                           */
  num_t kappa, alpha, sigma0, sigma1;   /* the differentiable parameters     */
  num_t amp;             /* pluck amplitude, hammer or bow velocity           */
  num_t *u, *up;         /* u^n, u^{n-1}, index l-1 for node l               */
  num_t *z, *zp;         /* z^n, z^{n-1}, index m-1 for node m               */
  num_t uh, uhp;         /* hammer u_H^n, u_H^{n-1} (Eq. 6)                  */
  int64_t n;             /* time level: state holds w^{n-1}, w^n             */
  int64_t next_out;      /* index of the next output sample                  */
  /* linear system, position ordered */
  int ntot, hrow, bw, pattern;
  int *urow, *zrow;      /* node -> row, -1 at the fixed ends                */
  num_t *band, *band0, *rhs, *sol, *rhs0;
  num_t *zsol;           /* second solution (unit force) for the bow         */
  num_t *tmp, *tmpx;     /* residual workspace                               */
  /* interval quantities, index 1..N (entry 0 unused)                        */
  num_t *q, *qp, *pt, *ptp;
  /* overlap weights R_ij = |T_i cap L_j| / h_t, both directions (A6)      */
  int *t_ptr, *t_j; double *t_w;   /* for t-interval i: list of (j, R_ij)   */
  int *l_ptr, *l_i; double *l_w;   /* for l-interval j: list of (i, R_ij)   */
  /* excitation point interpolation (Sec. 3.3: I_p, J_p with p = 1)          */
  int e_node[2]; double e_w[2];
  int o_node[2]; double o_w[2];
  int ol_node[2]; double ol_w[2];   /* pickup on the longitudinal grid */
  num_t last_power, last_G, last_v, last_F;
  double last_resid;
};

/* ------------------------------------------------------------------ grid */

/* Spacing rules of Sec. 3.2.  Rule 1 is the printed transverse spacing
 * h_t = sqrt((g^2 k^2 + sqrt(g^4 k^4 + 16 kappa^2 k^2))/2), which is the
 * von Neumann bound of the theta-scheme for theta = 1.  Rule 0 (default)
 * is the same bound for the theta actually used:
 *   g^2 k^2/h^2 + 4 kappa^2 k^2/h^4 <= 2 theta - 1.
 * The longitudinal rule is h_l = g alpha k (CFL of the z wave equation).
 * N = floor(1/h_min) so that h = 1/N >= h_min (a relative slack of 1e-12
 * keeps exact ratios such as 1/h_min = 100 from rounding down). */
int sfdo_grid(const sfdo_spec* s, int32_t* n_t, int32_t* n_l) {
  if (!s || !(s->fs > 0) || !(s->gamma > 0) || !(s->kappa >= 0) ||
      !(s->alpha >= 1) || !(s->theta > 0.5) || !(s->theta <= 1))
    return -1;
  const double k = 1.0 / s->fs;
  const double ratio = s->gamma_max_ratio >= 1 ? s->gamma_max_ratio : 1.0;
  const double g = s->gamma * ratio;
  const double g2k2 = g * g * k * k;
  const double kk2 = s->kappa * s->kappa * k * k;
  double h2;
  if (s->grid_rule == 1) {
    h2 = 0.5 * (g2k2 + sqrt(g2k2 * g2k2 + 16.0 * kk2));
  } else {
    const double d = 2.0 * s->theta - 1.0;
    h2 = (g2k2 + sqrt(g2k2 * g2k2 + 16.0 * d * kk2)) / (2.0 * d);
  }
  int32_t nt = (int32_t)floor((1.0 / sqrt(h2)) * (1.0 + 1e-12));
  int32_t nl = (int32_t)floor((1.0 / (g * s->alpha * k)) * (1.0 + 1e-12));
  if (nl < 1) nl = 1;
  if (s->n_t_override > 0) nt = s->n_t_override;
  if (s->n_l_override > 0) nl = s->n_l_override;
  if (nt < 2) return -2;
  if (n_t) *n_t = nt;
  if (n_l) *n_l = nl;
  return 0;
}

/* ------------------------------------------------------------ helpers */

static num_t U(const sfdo_string* S, const num_t* u, int l) {
  /* node value with the fixed ends u_0 = u_N = 0 (Sec. 3.4: N-1 unknowns) */
  if (l <= 0 || l >= S->nt) return 0.0;
  return u[l - 1];
}

static num_t Ughost(const sfdo_string* S, const num_t* u, int l) {
  /* ghost nodes for the fourth difference: clamped u_{-1} = u_1,
   * simply supported u_{-1} = -u_1 (and mirrored at x = 1). */
  const double sgn = S->p.boundary == 1 ? -1.0 : 1.0;
  if (l == -1) return sgn * U(S, u, 1);
  if (l == S->nt + 1) return sgn * U(S, u, S->nt - 1);
  return U(S, u, l);
}

static num_t Z(const sfdo_string* S, const num_t* z, int m) {
  if (m <= 0 || m >= S->nl) return 0.0;
  return z[m - 1];
}

/* delta_xx u at node l (Sec. 3.1) */
static num_t dxx(const sfdo_string* S, const num_t* u, int l) {
  return (U(S, u, l + 1) - 2.0 * U(S, u, l) + U(S, u, l - 1)) / (S->ht * S->ht);
}

/* delta_xxxx u at node l with the boundary ghosts (Sec. 3.2) */
static num_t dxxxx(const sfdo_string* S, const num_t* u, int l) {
  const double h4 = S->ht * S->ht * S->ht * S->ht;
  return (Ughost(S, u, l + 2) - 4.0 * Ughost(S, u, l + 1) + 6.0 * Ughost(S, u, l) -
          4.0 * Ughost(S, u, l - 1) + Ughost(S, u, l - 2)) / h4;
}

static num_t dzz(const sfdo_string* S, const num_t* z, int m) {
  return (Z(S, z, m + 1) - 2.0 * Z(S, z, m) + Z(S, z, m - 1)) / (S->hl * S->hl);
}

/* linear interpolation weights I(x) on the transverse nodes (Sec. 3.3). */
static void interp_weights(const sfdo_string* S, double x, int node[2], double w[2]) {
  double pos = x * S->nt;
  int l = (int)floor(pos);
  if (l < 0) l = 0;
  if (l > S->nt - 1) l = S->nt - 1;
  double a = pos - l;
  node[0] = l; w[0] = 1.0 - a;
  node[1] = l + 1; w[1] = a;
}

static num_t interp(const sfdo_string* S, const num_t* u, const int node[2], const double w[2]) {
  return w[0] * U(S, u, node[0]) + w[1] * U(S, u, node[1]);
}

/* Bow controls at time t from the breakpoint envelopes (Sec. 3.3.1 makes
 * v_B, F_B and x_B time-varying): linear between breakpoints, the first or
 * last value outside them. */
static void bow_controls(const sfdo_spec* P, double t, double* v, double* f, double* x) {
  const int m = P->bow_env_n;
  if (t <= P->bow_env_t[0] || m == 1) {
    *v = P->bow_env_v[0]; *f = P->bow_env_f[0]; *x = P->bow_env_x[0];
    return;
  }
  if (t >= P->bow_env_t[m - 1]) {
    *v = P->bow_env_v[m - 1]; *f = P->bow_env_f[m - 1]; *x = P->bow_env_x[m - 1];
    return;
  }
  int j = 0;
  while (j + 1 < m - 1 && t >= P->bow_env_t[j + 1]) ++j;
  const double r = (t - P->bow_env_t[j]) / (P->bow_env_t[j + 1] - P->bow_env_t[j]);
  *v = P->bow_env_v[j] + r * (P->bow_env_v[j + 1] - P->bow_env_v[j]);
  *f = P->bow_env_f[j] + r * (P->bow_env_f[j + 1] - P->bow_env_f[j]);
  *x = P->bow_env_x[j] + r * (P->bow_env_x[j + 1] - P->bow_env_x[j]);
}

/* f0 modulation (abstract; Sec. 1 lists f0 modulation among the
 * stochastic parameters).  gamma^n for the step n -> n+1, t = n k: vibrato
 * gamma 2^{(c/1200) sin(2 pi f_v t + phi)}; glissando gamma 2^{D min(t, T) / T},
 * a glide over T that then holds at 2^D (the peak the grid is sized for). */
static double gamma_at(const sfdo_string* S, int64_t n) {
  const double t = (double)n * S->k;
  const sfdo_spec* p = &S->p;
  if (p->mod_kind == SFDO_MOD_VIBRATO)
    return p->gamma * pow(2.0, (p->mod_depth / 1200.0) * sin(2.0 * PI_D * p->mod_rate * t + p->mod_phase));
  if (p->mod_kind == SFDO_MOD_GLISS && p->mod_duration > 0) {
    const double tg = t < p->mod_duration ? t : p->mod_duration;
    return p->gamma * pow(2.0, p->mod_depth * tg / p->mod_duration);
  }
  return p->gamma;
}

/* ------------------------------------------------------- band storage */

static void add(sfdo_string* S, int r, int c, num_t v) {
  if (r < 0 || c < 0) return;
  if (S->pattern) {
    int d = abs(r - c);
    if (d > S->bw) S->bw = d;
    return;
  }
  S->band[(size_t)r * (2 * S->bw + 1) + (c - r + S->bw)] += v;
}

/* Banded Gaussian elimination without pivoting.  After weighting the u rows
 * by h_t and the z rows by h_l the matrix of Eqs. 7-8 is symmetric positive
 * definite (the coupling blocks are adjoint, A6), so all leading minors are
 * positive and no pivoting is needed. */
static int band_solve(sfdo_string* S, num_t* b) {
  const int n = S->ntot, bw = S->bw, ld = 2 * bw + 1;
  num_t* A = S->band;
  for (int kk = 0; kk < n; ++kk) {
    const num_t piv = A[(size_t)kk * ld + bw];
    if (piv == 0.0 || !isfinite(RE(piv))) return -4;
    const int iend = kk + bw < n - 1 ? kk + bw : n - 1;
    for (int i = kk + 1; i <= iend; ++i) {
      num_t* ai = A + (size_t)i * ld;
      const num_t l = ai[kk - i + bw] / piv;
      if (l == 0.0) continue;
      ai[kk - i + bw] = l;
      const num_t* ak = A + (size_t)kk * ld;
      for (int j = kk + 1; j <= kk + bw && j < n; ++j) ai[j - i + bw] -= l * ak[j - kk + bw];
      b[i] -= l * b[kk];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    const num_t* ai = A + (size_t)i * ld;
    num_t s = b[i];
    for (int j = i + 1; j <= i + bw && j < n; ++j) s -= ai[j - i + bw] * b[j];
    b[i] = s / ai[bw];
  }
  return 0;
}

static void band_mul(const sfdo_string* S, const num_t* A, const num_t* x, num_t* y) {
  const int n = S->ntot, bw = S->bw, ld = 2 * bw + 1;
  for (int i = 0; i < n; ++i) {
    num_t s = 0;
    for (int j = i - bw; j <= i + bw; ++j)
      if (j >= 0 && j < n) s += A[(size_t)i * ld + (j - i + bw)] * x[j];
    y[i] = s;
  }
}

/* ------------------------------------------------------ construction */

/* Overlap weights R_ij = |[(i-1)h_t, i h_t] cap [(j-1)h_l, j h_l]| / h_t.
 * R p is D_x- of the piecewise-linear interpolant of z on the transverse
 * grid, i.e. D_x- I_(l->t) with p = 1 (Sec. 3.1, reading A6). */
static int build_overlaps(sfdo_string* S) {
  const int nt = S->nt, nl = S->nl;
  int cap = 2 * (nt + nl) + 4;
  int* ti = malloc(sizeof(int) * cap);
  int* tj = malloc(sizeof(int) * cap);
  double* tw = malloc(sizeof(double) * cap);
  int cnt = 0;
  const double tol = 1e-12 * (S->ht < S->hl ? S->ht : S->hl);
  for (int i = 1; i <= nt; ++i) {
    const double a = (double)(i - 1) / nt, b = (double)i / nt;
    int j0 = (int)floor(a * nl) - 1, j1 = (int)ceil(b * nl) + 1;
    if (j0 < 1) j0 = 1;
    if (j1 > nl) j1 = nl;
    for (int j = j0; j <= j1; ++j) {
      const double c = (double)(j - 1) / nl, d = (double)j / nl;
      const double lo = a > c ? a : c, hi = b < d ? b : d;
      if (hi - lo > tol) {
        if (cnt == cap) {
          cap *= 2;
          ti = realloc(ti, sizeof(int) * cap);
          tj = realloc(tj, sizeof(int) * cap);
          tw = realloc(tw, sizeof(double) * cap);
        }
        ti[cnt] = i; tj[cnt] = j; tw[cnt] = (hi - lo) / S->ht; ++cnt;
      }
    }
  }
  S->t_ptr = calloc(nt + 2, sizeof(int));
  S->l_ptr = calloc(nl + 2, sizeof(int));
  S->t_j = malloc(sizeof(int) * (cnt + 1));
  S->t_w = malloc(sizeof(double) * (cnt + 1));
  S->l_i = malloc(sizeof(int) * (cnt + 1));
  S->l_w = malloc(sizeof(double) * (cnt + 1));
  for (int e = 0; e < cnt; ++e) { S->t_ptr[ti[e] + 1]++; S->l_ptr[tj[e] + 1]++; }
  for (int i = 1; i <= nt + 1; ++i) S->t_ptr[i] += S->t_ptr[i - 1];
  for (int j = 1; j <= nl + 1; ++j) S->l_ptr[j] += S->l_ptr[j - 1];
  int* fillt = calloc(nt + 2, sizeof(int));
  int* filll = calloc(nl + 2, sizeof(int));
  for (int e = 0; e < cnt; ++e) {
    int pt = S->t_ptr[ti[e]] + fillt[ti[e]]++;
    S->t_j[pt] = tj[e]; S->t_w[pt] = tw[e];
    int pl = S->l_ptr[tj[e]] + filll[tj[e]]++;
    S->l_i[pl] = ti[e]; S->l_w[pl] = tw[e];
  }
  free(ti); free(tj); free(tw); free(fillt); free(filll);
  return 0;
}

typedef struct { double x; int kind; int idx; } node_pos;

static int cmp_pos(const void* a, const void* b) {
  const node_pos* p = a; const node_pos* q = b;
  if (p->x < q->x) return -1;
  if (p->x > q->x) return 1;
  if (p->kind != q->kind) return p->kind - q->kind;
  return p->idx - q->idx;
}

/* Unknowns ordered by position along the string (u nodes, the hammer and
 * z nodes interleaved) so that Eqs. 7-9 form a band matrix. */
static void build_ordering(sfdo_string* S) {
  const int nn = S->nu + S->nz + (S->p.exc_kind == SFDO_EXC_HAMMER ? 1 : 0);
  node_pos* v = malloc(sizeof(node_pos) * (nn > 0 ? nn : 1));
  int c = 0;
  for (int l = 1; l < S->nt; ++l) { v[c].x = (double)l / S->nt; v[c].kind = 0; v[c].idx = l; ++c; }
  if (S->p.exc_kind == SFDO_EXC_HAMMER) { v[c].x = S->p.ham_pos; v[c].kind = 1; v[c].idx = 0; ++c; }
  for (int m = 1; m < S->nl; ++m) { v[c].x = (double)m / S->nl; v[c].kind = 2; v[c].idx = m; ++c; }
  qsort(v, nn, sizeof(node_pos), cmp_pos);
  S->urow = malloc(sizeof(int) * (S->nt + 1));
  S->zrow = malloc(sizeof(int) * (S->nl + 1));
  for (int l = 0; l <= S->nt; ++l) S->urow[l] = -1;
  for (int m = 0; m <= S->nl; ++m) S->zrow[m] = -1;
  S->hrow = -1;
  for (int r = 0; r < nn; ++r) {
    if (v[r].kind == 0) S->urow[v[r].idx] = r;
    else if (v[r].kind == 1) S->hrow = r;
    else S->zrow[v[r].idx] = r;
  }
  S->ntot = nn;
  free(v);
}

static void assemble(sfdo_string* S, double gam, num_t hamG);

/* A string at time level 1; `which` >= 0 (complex build only) gives that
 * parameter (0 kappa, 1 alpha, 2 sigma0, 3 sigma1, 4 the pluck amplitude,
 * hammer velocity or bow velocity) the imaginary part h. */
static sfdo_string* create_string(const sfdo_spec* s, int which, double h) {
  int32_t nt, nl;
  if (sfdo_grid(s, &nt, &nl) != 0) return NULL;
  if (!(s->pickup > 0 && s->pickup < 1) || !(s->length > 0) || !(s->rho_a > 0)) return NULL;
  if (!(s->sigma0 >= 0) || !(s->sigma1 >= 0)) return NULL;
  if (s->exc_kind == SFDO_EXC_HAMMER &&
      !(s->ham_pos > 0 && s->ham_pos < 1 && s->ham_mass > 0 && s->ham_alpha >= 1 && s->ham_omega > 0))
    return NULL;
  if (s->exc_kind == SFDO_EXC_BOW &&
      !(s->bow_pos > 0 && s->bow_pos < 1 && s->bow_force >= 0 && s->bow_eps >= 0 && s->bow_eps <= 1 &&
        s->bow_a >= 0))
    return NULL;
  if (s->exc_kind == SFDO_EXC_PLUCK && !(s->pluck_pos > 0 && s->pluck_pos < 1)) return NULL;
  if (s->bow_env_n < 0 || s->bow_env_n > 16) return NULL;
  for (int j = 0; j < s->bow_env_n; ++j) {
    if (!(s->bow_env_x[j] > 0 && s->bow_env_x[j] < 1 && s->bow_env_f[j] >= 0)) return NULL;
    if (j > 0 && !(s->bow_env_t[j] > s->bow_env_t[j - 1])) return NULL;
  }
  sfdo_string* S = calloc(1, sizeof(sfdo_string));
  S->p = *s;
  S->nt = nt; S->nl = nl;
  S->nu = nt - 1; S->nz = nl > 1 ? nl - 1 : 0;
  S->ht = 1.0 / nt; S->hl = 1.0 / nl; S->k = 1.0 / s->fs;
  S->kappa = s->kappa; S->alpha = s->alpha; S->sigma0 = s->sigma0; S->sigma1 = s->sigma1;
  S->amp = s->exc_kind == SFDO_EXC_PLUCK ? s->pluck_amp : (s->exc_kind == SFDO_EXC_HAMMER ? s->ham_vel : s->bow_vel);
#ifdef SFDO_COMPLEX
  num_t* pick[5] = {&S->kappa, &S->alpha, &S->sigma0, &S->sigma1, &S->amp};
  if (which >= 0 && which < 5) *pick[which] += I * h;
#else
  (void)which; (void)h;
#endif
  S->u = calloc(S->nu + 1, sizeof(num_t));
  S->up = calloc(S->nu + 1, sizeof(num_t));
  S->z = calloc(S->nz + 1, sizeof(num_t));
  S->zp = calloc(S->nz + 1, sizeof(num_t));
  S->q = calloc(nt + 2, sizeof(num_t));
  S->qp = calloc(nt + 2, sizeof(num_t));
  S->pt = calloc(nt + 2, sizeof(num_t));
  S->ptp = calloc(nt + 2, sizeof(num_t));
  build_overlaps(S);
  build_ordering(S);
  interp_weights(S, s->pickup, S->o_node, S->o_w);
  {   /* the same linear interpolation on the longitudinal nodes */
    double pos = s->pickup * nl;
    int m = (int)floor(pos);
    if (m < 0) m = 0;
    if (m > nl - 1) m = nl - 1;
    S->ol_node[0] = m; S->ol_w[0] = 1.0 - (pos - m);
    S->ol_node[1] = m + 1; S->ol_w[1] = pos - m;
  }
  if (s->exc_kind == SFDO_EXC_HAMMER) interp_weights(S, s->ham_pos, S->e_node, S->e_w);
  else if (s->exc_kind == SFDO_EXC_BOW) interp_weights(S, s->bow_pos, S->e_node, S->e_w);
  /* band width from the sparsity of the assembled system (all strains set
   * to one so that no coupling entry is structurally absent) */
  for (int i = 0; i <= nt; ++i) S->q[i] = 1.0;
  S->pattern = 1; S->bw = 0;
  assemble(S, s->gamma, 1.0);
  S->pattern = 0;
  if (S->bw < 1) S->bw = 1;
  const size_t bsz = (size_t)(S->ntot > 0 ? S->ntot : 1) * (2 * S->bw + 1);
  S->band = calloc(bsz, sizeof(num_t));
  S->band0 = calloc(bsz, sizeof(num_t));
  S->rhs = calloc(S->ntot + 1, sizeof(num_t));
  S->rhs0 = calloc(S->ntot + 1, sizeof(num_t));
  S->sol = calloc(S->ntot + 1, sizeof(num_t));
  S->zsol = calloc(S->ntot + 1, sizeof(num_t));
  S->tmp = calloc(S->ntot + 1, sizeof(num_t));
  S->tmpx = calloc(S->ntot + 1, sizeof(num_t));
  memset(S->q, 0, sizeof(num_t) * (nt + 2));
  /* initial conditions w^0, w^1 (Sec. 3.3 and 3.4) */
  if (s->exc_kind == SFDO_EXC_PLUCK) {
    /* triangle with peak c0 = amp/L at x_P, zero initial velocity (A9) */
    const num_t c0 = S->amp / s->length;
    const double xp = s->pluck_pos;
    for (int l = 1; l < nt; ++l) {
      const double x = (double)l / nt;
      const num_t v = x <= xp ? c0 * x / xp : c0 * (1.0 - x) / (1.0 - xp);
      S->u[l - 1] = v; S->up[l - 1] = v;
    }
  } else if (s->exc_kind == SFDO_EXC_HAMMER) {
    /* hammer starts at the string with velocity v_H: u_H^0 = 0, u_H^1 = v_H k */
    S->uhp = 0.0;
    S->uh = (S->amp / s->length) * S->k;
  }
  S->n = 1;
  S->next_out = 0;
  return S;
}

sfdo_string* sfdo_create(const sfdo_spec* s) { return create_string(s, -1, 0.0); }

void sfdo_destroy(sfdo_string* S) {
  if (!S) return;
  free(S->u); free(S->up); free(S->z); free(S->zp);
  free(S->q); free(S->qp); free(S->pt); free(S->ptp);
  free(S->t_ptr); free(S->t_j); free(S->t_w);
  free(S->l_ptr); free(S->l_i); free(S->l_w);
  free(S->urow); free(S->zrow);
  free(S->band); free(S->band0); free(S->rhs); free(S->rhs0); free(S->sol); free(S->zsol); free(S->tmp); free(S->tmpx);
  free(S);
}

/* ------------------------------------------------------------ a step */

/* Assemble A^n (band) and the right-hand side -(B^n w^n + C w^{n-1}) of
 * Eq. 7 from the stencil form of Eq. 4 (k^2-scaled), with
 *   q = D_x- u^n,  ptilde = R D_x- z^n,  phi' = gamma^2 (alpha^2-1)/2,
 *   Theta = theta I + (1-theta) M_x. (Sec. 3.2),
 * mu_t. q = (q^{n+1}+q^{n-1})/2 and mu_tt p = (p^{n+1}+2p^n+p^{n-1})/4.
 * hamG is the hammer stiffness coefficient of Eq. 6 (0 without contact). */
static void assemble(sfdo_string* S, double gam, num_t hamG) {
  const sfdo_spec* P = &S->p;
  const int nt = S->nt, nl = S->nl;
  const double k = S->k, ht = S->ht, hl = S->hl;
  const double th = P->theta;
  const double g2k2 = gam * gam * k * k;
  const num_t kk2 = S->kappa * S->kappa * k * k;
  const num_t s0k = S->sigma0 * k, s1k = S->sigma1 * k;
  const num_t cnl = 0.5 * gam * gam * (S->alpha * S->alpha - 1.0) * k * k; /* phi' k^2 */
  const num_t* q = S->q;

  if (!S->pattern) {
    memset(S->band, 0, sizeof(num_t) * (size_t)S->ntot * (2 * S->bw + 1));
    memset(S->rhs, 0, sizeof(num_t) * S->ntot);
  }

  /* ---- transverse rows, Eq. 4 (first line) ---- */
  for (int l = 1; l < nt; ++l) {
    const int r = S->urow[l];
    /* Theta u^{n+1} + sigma0 k u^{n+1} - sigma1 k delta_xx u^{n+1} */
    add(S, r, S->urow[l], th + s0k + 2.0 * s1k / (ht * ht));
    add(S, r, S->urow[l - 1], 0.5 * (1.0 - th) - s1k / (ht * ht));
    add(S, r, S->urow[l + 1], 0.5 * (1.0 - th) - s1k / (ht * ht));
    /* -(phi'k^2/2) delta_x+ [ q^2 q^{n+1} + q ptilde^{n+1} ]  (V and K^(tl)) */
    for (int side = 0; side < 2; ++side) {
      const int i = side == 0 ? l : l + 1;          /* intervals l and l+1 */
      const double sg = side == 0 ? 1.0 : -1.0;
      const num_t coef = sg * cnl / (2.0 * ht);
      add(S, r, S->urow[i], coef * q[i] * q[i] / ht);
      add(S, r, S->urow[i - 1], -coef * q[i] * q[i] / ht);
      for (int e = S->t_ptr[i]; e < S->t_ptr[i + 1]; ++e) {
        const int j = S->t_j[e];
        const num_t w = coef * q[i] * S->t_w[e] / hl;
        add(S, r, S->zrow[j], w);
        add(S, r, S->zrow[j - 1], -w);
      }
    }
    if (S->pattern) continue;
    const num_t* u = S->u;
    const num_t* up = S->up;
    num_t b = th * (2.0 * U(S, u, l) - U(S, up, l)) +
               0.5 * (1.0 - th) * (2.0 * U(S, u, l - 1) - U(S, up, l - 1) + 2.0 * U(S, u, l + 1) - U(S, up, l + 1));
    b += g2k2 * dxx(S, u, l);
    b -= kk2 * dxxxx(S, u, l);
    b += s0k * U(S, up, l);
    b -= s1k * dxx(S, up, l);
    /* (phi'k^2/2) delta_x+ [ q^2 q^{n-1} + q (2 ptilde^n + ptilde^{n-1}) ] */
    {
      const int i1 = l + 1, i0 = l;
      const num_t y1 = q[i1] * q[i1] * S->qp[i1] + q[i1] * (2.0 * S->pt[i1] + S->ptp[i1]);
      const num_t y0 = q[i0] * q[i0] * S->qp[i0] + q[i0] * (2.0 * S->pt[i0] + S->ptp[i0]);
      b += cnl / (2.0 * ht) * (y1 - y0);
    }
    S->rhs[r] = b;
  }

  /* ---- longitudinal rows, Eq. 4 (second line) ---- */
  for (int m = 1; m < nl; ++m) {
    const int r = S->zrow[m];
    add(S, r, S->zrow[m], 1.0 + s0k + 2.0 * s1k / (hl * hl));
    add(S, r, S->zrow[m - 1], -s1k / (hl * hl));
    add(S, r, S->zrow[m + 1], -s1k / (hl * hl));
    /* -(phi'k^2/2) delta_x+^(l) S [ q q^{n+1} ],  S = (h_t/h_l) R^T  (K^(lt)) */
    for (int side = 0; side < 2; ++side) {
      const int j = side == 0 ? m : m + 1;
      const double sg = side == 0 ? 1.0 : -1.0;
      const num_t coef = sg * cnl / (2.0 * hl) * (ht / hl);
      for (int e = S->l_ptr[j]; e < S->l_ptr[j + 1]; ++e) {
        const int i = S->l_i[e];
        const num_t w = coef * S->l_w[e] * q[i] / ht;
        add(S, r, S->urow[i], w);
        add(S, r, S->urow[i - 1], -w);
      }
    }
    if (S->pattern) continue;
    const num_t* z = S->z;
    const num_t* zp = S->zp;
    num_t b = 2.0 * Z(S, z, m) - Z(S, zp, m);
    b += g2k2 * S->alpha * S->alpha * dzz(S, z, m);
    b += s0k * Z(S, zp, m);
    b -= s1k * dzz(S, zp, m);
    num_t sz1 = 0, sz0 = 0;   /* (S [q q^{n-1}])_{m+1}, (S [q q^{n-1}])_m */
    for (int e = S->l_ptr[m + 1]; e < S->l_ptr[m + 2]; ++e) {
      const int i = S->l_i[e];
      sz1 += S->l_w[e] * q[i] * S->qp[i];
    }
    for (int e = S->l_ptr[m]; e < S->l_ptr[m + 1]; ++e) {
      const int i = S->l_i[e];
      sz0 += S->l_w[e] * q[i] * S->qp[i];
    }
    b += cnl / (2.0 * hl) * (ht / hl) * (sz1 - sz0);
    S->rhs[r] = b;
  }

  /* ---- hammer (Eq. 6): F_H = G mu_t. eta, eta = u_H - I u, the string
   * receives k^2 M F_H J and the hammer obeys delta_tt u_H = -F_H.  With G
   * taken at time n the pair is linear in (u^{n+1}, u_H^{n+1}) and is
   * solved jointly here as one extra unknown.  M = m_H / (rho A L). ---- */
  if (P->exc_kind == SFDO_EXC_HAMMER) {
    const double M = P->ham_mass / (P->rho_a * P->length);
    const num_t cg = 0.5 * k * k * hamG;
    const int hr = S->hrow;
    num_t etap = 0.0;
    if (!S->pattern) etap = S->uhp - interp(S, S->up, S->e_node, S->e_w);
    for (int a = 0; a < 2; ++a) {
      const int la = S->e_node[a];
      if (la <= 0 || la >= nt) continue;
      const double Ja = S->e_w[a] / ht;
      const int r = S->urow[la];
      add(S, r, hr, -M * cg * Ja);
      for (int bnd = 0; bnd < 2; ++bnd) {
        const int lb = S->e_node[bnd];
        if (lb <= 0 || lb >= nt) continue;
        add(S, r, S->urow[lb], M * cg * Ja * S->e_w[bnd]);
      }
      if (!S->pattern) S->rhs[r] += M * cg * Ja * etap;
    }
    add(S, hr, hr, 1.0 + cg);
    for (int bnd = 0; bnd < 2; ++bnd) {
      const int lb = S->e_node[bnd];
      if (lb <= 0 || lb >= nt) continue;
      add(S, hr, S->urow[lb], -cg * S->e_w[bnd]);
    }
    if (!S->pattern) S->rhs[hr] = 2.0 * S->uh - S->uhp - cg * etap;
  }
}

/* Bow friction characteristic of Sec. 3.3.1 with the argument read as the
 * relative velocity (reading A11): phi(v) = sign(v)(eps + (1-eps)e^{-a|v|}). */
static num_t friction_mag(double a, double eps, num_t w) { return eps + (1.0 - eps) * NEXP(-a * w); }

/* Solve v + c phi(v) = b (Eq. 5 after eliminating u^{n+1}; reading A11):
 * |b| <= c -> sticking, v = 0 and phi = b/c; otherwise the unique root of
 * the convex g(w) = w + c phi(w) - |b| on (0, |b|) with sign(v) = sign(b),
 * found by Newton from w = |b| guarded by bisection. Returns phi(v). */
static num_t bow_solve(num_t b, num_t c, double a, double eps, num_t* v_out) {
  if (!(RE(c) > 0)) { *v_out = b; return b == 0 ? 0.0 : (RE(b) > 0 ? 1.0 : -1.0) * friction_mag(a, eps, NABS(b)); }
  if (RE(NABS(b)) <= RE(c)) { *v_out = 0.0; return b / c; }
  const num_t B = NABS(b);
  const double sg = RE(b) > 0 ? 1.0 : -1.0;
  double lo = 0.0, hi = RE(B);
  num_t w = B;
  for (int it = 0; it < 200; ++it) {
    const num_t e = NEXP(-a * w);
    const num_t g = w + c * (eps + (1.0 - eps) * e) - B;
    if (RE(g) > 0) hi = RE(w); else lo = RE(w);
    const num_t dg = 1.0 - c * (1.0 - eps) * a * e;
    num_t wn = RE(dg) > 0 ? w - g / dg : 0.5 * (lo + hi);
    if (!(RE(wn) > lo && RE(wn) < hi)) wn = 0.5 * (lo + hi);
    if (NMAG(wn - w) <= 1e-16 * (1.0 + RE(w))) { w = wn; break; }
    w = wn;
  }
  *v_out = sg * w;
  return sg * friction_mag(a, eps, w);
}

static int step(sfdo_string* S) {
  const sfdo_spec* P = &S->p;
  const int nt = S->nt, nl = S->nl;
  const double k = S->k;
  const double gam = gamma_at(S, S->n);
  /* strains q^n, q^{n-1} and ptilde^n, ptilde^{n-1} on the intervals */
  for (int i = 1; i <= nt; ++i) {
    S->q[i] = (U(S, S->u, i) - U(S, S->u, i - 1)) / S->ht;
    S->qp[i] = (U(S, S->up, i) - U(S, S->up, i - 1)) / S->ht;
    num_t s = 0, sp = 0;
    for (int e = S->t_ptr[i]; e < S->t_ptr[i + 1]; ++e) {
      const int j = S->t_j[e];
      s += S->t_w[e] * (Z(S, S->z, j) - Z(S, S->z, j - 1)) / S->hl;
      sp += S->t_w[e] * (Z(S, S->zp, j) - Z(S, S->zp, j - 1)) / S->hl;
    }
    S->pt[i] = s; S->ptp[i] = sp;
  }
  num_t hamG = 0.0;
  if (P->exc_kind == SFDO_EXC_HAMMER) {
    const num_t eta = S->uh - interp(S, S->u, S->e_node, S->e_w);
    hamG = RE(eta) > 0 ? pow(P->ham_omega, 1.0 + P->ham_alpha) * NPOW(eta, P->ham_alpha - 1.0) : 0.0;
  }
  assemble(S, gam, hamG);
  const size_t bsz = (size_t)S->ntot * (2 * S->bw + 1);
  memcpy(S->band0, S->band, sizeof(num_t) * bsz);
  memcpy(S->rhs0, S->rhs, sizeof(num_t) * S->ntot);
  memcpy(S->sol, S->rhs, sizeof(num_t) * S->ntot);
  int rc = band_solve(S, S->sol);   /* band now holds the LU factors */
  if (rc) return rc;
  num_t force = 0.0;                /* normalised force on the string      */
  if (P->exc_kind == SFDO_EXC_BOW) {
    const double t = (double)S->n * k;
    num_t bv = S->amp;
    double bf = P->bow_force;
    if (P->bow_env_n > 0) {   /* time-varying controls: the step's values, and I, J at x_B(t) */
      double bx = P->bow_pos, ev = 0.0;
      bow_controls(P, t, &ev, &bf, &bx);
      bv = ev;
      interp_weights(S, bx, S->e_node, S->e_w);
    }
    const double FB = (P->bow_release >= 0 && t >= P->bow_release) ? 0.0
                      : bf / (P->rho_a * P->length * P->length);
    const num_t vB = bv / P->length;
    const double aN = P->bow_a * P->length;
    /* unit-force response A z = J (same factors) */
    memset(S->zsol, 0, sizeof(num_t) * S->ntot);
    for (int a = 0; a < 2; ++a) {
      const int la = S->e_node[a];
      if (la > 0 && la < nt) S->zsol[S->urow[la]] += S->e_w[a] / S->ht;
    }
    /* re-solve with the stored LU factors: forward (unit lower) + backward */
    {
      const int n = S->ntot, bw = S->bw, ld = 2 * bw + 1;
      const num_t* A = S->band;
      num_t* x = S->zsol;
      for (int kk = 0; kk < n; ++kk)
        for (int i = kk + 1; i <= kk + bw && i < n; ++i) x[i] -= A[(size_t)i * ld + (kk - i + bw)] * x[kk];
      for (int i = n - 1; i >= 0; --i) {
        num_t s = x[i];
        for (int j = i + 1; j <= i + bw && j < n; ++j) s -= A[(size_t)i * ld + (j - i + bw)] * x[j];
        x[i] = s / A[(size_t)i * ld + bw];
      }
    }
    num_t Iu = 0, Iz = 0, Iup = 0;
    for (int a = 0; a < 2; ++a) {
      const int la = S->e_node[a];
      if (la <= 0 || la >= nt) continue;
      Iu += S->e_w[a] * S->sol[S->urow[la]];
      Iz += S->e_w[a] * S->zsol[S->urow[la]];
      Iup += S->e_w[a] * S->up[la - 1];
    }
    const num_t b = (Iu - Iup) / (2.0 * k) - vB;
    const num_t c = 0.5 * k * FB * Iz;
    num_t v;
    const num_t ph = bow_solve(b, c, aN, P->bow_eps, &v);
    force = -FB * ph;
    for (int r = 0; r < S->ntot; ++r) S->sol[r] += k * k * force * S->zsol[r];
    S->last_v = v;
  }
  /* residual of the assembled system (without the bow term, which is added
   * through the exact unit-force response) */
  {
    num_t* tmp = S->tmp;
    num_t* x = S->tmpx;
    memcpy(x, S->sol, sizeof(num_t) * S->ntot);
    if (P->exc_kind == SFDO_EXC_BOW)
      for (int r = 0; r < S->ntot; ++r) x[r] -= k * k * force * S->zsol[r];
    band_mul(S, S->band0, x, tmp);
    double num = 0, den = 0;
    for (int r = 0; r < S->ntot; ++r) {
      num = fmax(num, NMAG(tmp[r] - S->rhs0[r]));
      den = fmax(den, NMAG(S->rhs0[r]));
    }
    S->last_resid = den > 0 ? num / den : num;
  }
  /* excitation power delivered to the string, F I(delta_t. u) (Eqs. 5, 6) */
  num_t unew_e = 0, uold_e = 0;
  for (int a = 0; a < 2; ++a) {
    const int la = S->e_node[a];
    if (P->exc_kind == SFDO_EXC_PLUCK || la <= 0 || la >= nt) continue;
    unew_e += S->e_w[a] * S->sol[S->urow[la]];
    uold_e += S->e_w[a] * S->up[la - 1];
  }
  if (P->exc_kind == SFDO_EXC_HAMMER) {
    const double M = P->ham_mass / (P->rho_a * P->length);
    const num_t eta_new = S->sol[S->hrow] - unew_e;
    const num_t eta_old = S->uhp - uold_e;
    force = M * hamG * 0.5 * (eta_new + eta_old);
  }
  S->last_F = force;
  S->last_G = hamG;
  S->last_power = force * (unew_e - uold_e) / (2.0 * k);
  /* rotate the time levels */
  for (int l = 1; l < nt; ++l) { S->up[l - 1] = S->u[l - 1]; S->u[l - 1] = S->sol[S->urow[l]]; }
  for (int m = 1; m < nl; ++m) { S->zp[m - 1] = S->z[m - 1]; S->z[m - 1] = S->sol[S->zrow[m]]; }
  if (P->exc_kind == SFDO_EXC_HAMMER) { S->uhp = S->uh; S->uh = S->sol[S->hrow]; }
  S->n += 1;
  for (int l = 0; l < S->nu; ++l)
    if (!isfinite(RE(S->u[l]))) return -3;
  return 0;
}

/* Output sample y^j = L I(x_o) u^j, j = 0, 1, 2, ... (reading A10), or the
 * longitudinal displacement at the pickup (out_channel 1). */
static int run_samples(sfdo_string* S, int64_t n, num_t* y) {
  if (!S || n < 0) return -1;
  for (int64_t s = 0; s < n; ++s) {
    const int64_t j = S->next_out;
    while (S->n < j) {
      int rc = step(S);
      if (rc) return rc;
    }
    if (S->p.out_channel == 1) {   /* longitudinal displacement at the pickup (Sec. 4.2) */
      const num_t* zs = (j == S->n) ? S->z : S->zp;
      y[s] = S->p.length * (S->ol_w[0] * Z(S, zs, S->ol_node[0]) + S->ol_w[1] * Z(S, zs, S->ol_node[1]));
    } else {
      const num_t* src = (j == S->n) ? S->u : S->up;
      y[s] = S->p.length * interp(S, src, S->o_node, S->o_w);
    }
    S->next_out++;
  }
  return 0;
}

#ifndef SFDO_COMPLEX
int sfdo_run(sfdo_string* S, int64_t n, double* y) { return run_samples(S, n, y); }

int64_t sfdo_time_level(const sfdo_string* S) { return S ? S->n : -1; }

int sfdo_get_state(const sfdo_string* S, double* u_prev, double* u, double* z_prev, double* z, double* exc) {
  if (!S) return -1;
  if (u_prev) memcpy(u_prev, S->up, sizeof(double) * S->nu);
  if (u) memcpy(u, S->u, sizeof(double) * S->nu);
  if (z_prev && S->nz) memcpy(z_prev, S->zp, sizeof(double) * S->nz);
  if (z && S->nz) memcpy(z, S->z, sizeof(double) * S->nz);
  if (exc) {
    exc[0] = S->uhp; exc[1] = S->uh; exc[2] = S->last_power;
    exc[3] = S->last_G; exc[4] = S->last_v; exc[5] = S->last_F;
  }
  return 0;
}

int sfdo_set_state(sfdo_string* S, const double* u_prev, const double* u, const double* z_prev, const double* z) {
  if (!S) return -1;
  if (u_prev) memcpy(S->up, u_prev, sizeof(double) * S->nu);
  if (u) memcpy(S->u, u, sizeof(double) * S->nu);
  if (z_prev && S->nz) memcpy(S->zp, z_prev, sizeof(double) * S->nz);
  if (z && S->nz) memcpy(S->z, z, sizeof(double) * S->nz);
  return 0;
}

double sfdo_last_residual(const sfdo_string* S) { return S ? S->last_resid : -1.0; }

int sfdo_run_batch(const sfdo_spec* specs, int32_t n_str, const int64_t* n_samples, const int64_t* offsets,
                   double* y, int32_t n_threads) {
  if (!specs || n_str < 0 || !n_samples || !offsets || !y) return -1;
  int used = 1;
#ifdef _OPENMP
  int nth = n_threads > 0 ? n_threads : omp_get_max_threads();
  if (nth > n_str && n_str > 0) nth = n_str;
  used = nth;
#endif
  int err = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth) reduction(| : err)
#endif
  for (int i = 0; i < n_str; ++i) {
    sfdo_string* S = sfdo_create(&specs[i]);
    if (!S) { err |= 1; continue; }
    if (sfdo_run(S, n_samples[i], y + offsets[i]) != 0) err |= 2;
    sfdo_destroy(S);
  }
  return err ? -err : used;
}
#else
/* Complex-step derivative of the output with respect to one parameter
 * (declared in sfd_oracle.h; built with -DSFDO_COMPLEX only). */
int sfdo_cs_run(const sfdo_spec* s, int which, double h, int64_t n, double* y, double* dy) {
  if (!s || which < 0 || which > 4 || !(h > 0) || n < 0 || !y || !dy) return -1;
  sfdo_string* S = create_string(s, which, h);
  if (!S) return -1;
  num_t* yc = malloc(sizeof(num_t) * (size_t)(n > 0 ? n : 1));
  int rc = yc ? run_samples(S, n, yc) : -5;
  if (rc == 0)
    for (int64_t j = 0; j < n; ++j) { y[j] = creal(yc[j]); dy[j] = cimag(yc[j]) / h; }
  free(yc);
  sfdo_destroy(S);
  return rc;
}
#endif
