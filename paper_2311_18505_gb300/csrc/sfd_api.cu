// C-ABI runtime of the string synthesizer (include/sfd.h): contexts with a
// device-memory pool, strings (grid + coefficient derivation in FP64, state
// in the pool), excitations, batches and the launch of the step kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sfd.h"
#include "sfd_types.h"

namespace sfd {
#define SFD_DECLARE_LAUNCHER(name)                                                                   \
  cudaError_t name(const Job* d_jobs, int n_jobs, int* d_counter, int warp_floats, int warps_per_cta, \
                   int n_ctas, int group, cudaStream_t stream);
SFD_DECLARE_LAUNCHER(launch_synth_reg1)
SFD_DECLARE_LAUNCHER(launch_synth_reg3)
SFD_DECLARE_LAUNCHER(launch_synth_reg5)
SFD_DECLARE_LAUNCHER(launch_synth_reg7)
SFD_DECLARE_LAUNCHER(launch_synth_reg9)
SFD_DECLARE_LAUNCHER(launch_synth_smem)
#undef SFD_DECLARE_LAUNCHER
}

using namespace sfd;

namespace {

thread_local std::string g_err;

sfd_status fail(sfd_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

sfd_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SFD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SFD_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

constexpr size_t kAlign = 256;
constexpr double kPi = 3.14159265358979323846;

// First-fit allocator over one device allocation.
class Pool {
 public:
  sfd_status init(size_t bytes) {
    size_ = (bytes + kAlign - 1) / kAlign * kAlign;
    cudaError_t e = cudaMalloc(&base_, size_);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(pool)");
    free_[0] = size_;
    return SFD_OK;
  }
  void release() {
    if (base_) cudaFree(base_);
    base_ = nullptr;
  }
  char* alloc(size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        used_ += bytes;
        live_[off] = bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void dealloc(char* p) {
    if (!p) return;
    const size_t off = static_cast<size_t>(p - base_);
    auto lit = live_.find(off);
    if (lit == live_.end()) return;
    size_t sz = lit->second;
    live_.erase(lit);
    used_ -= sz;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {
      sz += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        start = pv->first;
        sz += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = sz;
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  char* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_, live_;
};

}  // namespace

constexpr int kClasses = 6;   // rows per lane 1, 3, 5, 7, 9 (registers), larger (shared memory)

struct sfd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side[kClasses] = {};      // one per kernel class, forked from `stream`
  cudaEvent_t fork = nullptr, join[kClasses] = {};
  cudaStream_t copy = nullptr;           // host-output copies of classes already ended
  cudaEvent_t copied = nullptr;          // end of those copies, joined back to `stream`
  bool timing = false;                   // record per-class kernel times
  cudaEvent_t t0[kClasses] = {}, t1[kClasses] = {};
  int timed_jobs[kClasses] = {};         // jobs of each class in the last launch
  Pool pool;
  int sm_count = 0;
  size_t smem_optin = 0;
  int warp_pairs = 1;                      // 0: every string on one warp (sfd_ctx_set_warp_pairs)
  int sweep_cap = 0;                       // coupled-solve sweep cap of every launch (0: kMaxSweeps)
  Job* d_jobs = nullptr;
  int job_cap = 0;
  int* d_counter = nullptr;                // kClasses work-queue counters
  int last_launches = 0;
  uint64_t h2d_bytes = 0, d2h_bytes = 0;   // all host<->device copies made
  // pinned staging of strings' initial blocks (flush_strings); the event
  // marks the last flush's copies, after which the buffer may be rewritten
  char* stage = nullptr;
  size_t stage_cap = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
};

struct sfd_string {
  sfd_ctx* ctx = nullptr;
  sfd_string_params p{};
  double gamma = 0, k = 0;
  int n_t = 0, n_l = 0;
  Desc h{};                 // host copy of the descriptor
  char* block = nullptr;    // pool block: Desc | Scalars | u du z dz xz az
  Desc* d_desc = nullptr;
  Scalars* d_sc = nullptr;
  bool started = false;     // first synthesize done
  mutable bool dirty = false;   // host image newer than the device block (flush_strings)
  int batch_refs = 0;
  // excitation (kept to rebuild the initial state)
  int exc = kPluck;
  double pluck_amp = 0, pluck_pos = 0.5;
  double hammer_uh1 = 0;    // u_H^1 = v_H k (normalised), u_H^0 = 0
  double bow_pos = 0.5;     // x_B of sfd_excite_bow (constant position of an envelope)
  double exc_pos = 0.5;     // hammer or bow position (excitation node after a regrid)
  // The set-up calls as last made, which a checkpoint replays (sfd_string_load):
  // the excitation (pluck: amp, pos; hammer: mass, vel, pos, omega, alpha;
  // bow: vel, force, pos, a, eps, release), the bow envelope (t, vel, force,
  // pos; bit c of rec_env_mask: control c + 1 given) and the modulation
  // (rate, depth, phase, duration).
  int32_t rec_exc = kPluck;
  double rec_exc_args[6] = {0.0, 0.5, 0.0, 0.0, 0.0, 0.0};
  int32_t rec_env_n = 0, rec_env_mask = 0;
  double rec_env[4][16] = {};
  int32_t rec_mod = SFD_MOD_NONE;
  double rec_mod_args[4] = {};
};

struct sfd_batch {
  sfd_ctx* ctx = nullptr;
  std::vector<sfd_string*> strings;
  int wpc = 0;                 // warps per CTA (0: automatic)
  int groups = -1;             // warp groups: -1 the context's setting, 0 off, 1 on (autotune)
  // prepared launch (sfd_batch_prepare / sfd_batch_launch)
  void* plan = nullptr;        // Plan*
  char* d_jobs = nullptr;      // pool block holding the plan's job table
  size_t d_jobs_bytes = 0;
};

namespace {

sfd_status set_device(const sfd_ctx* c) {
  SFD_CUDA(cudaSetDevice(c->device));
  return SFD_OK;
}

cudaError_t h2d(sfd_ctx* c, void* dst, const void* src, size_t n) {
  c->h2d_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream);
}

cudaError_t d2h(sfd_ctx* c, void* dst, const void* src, size_t n, cudaStream_t st = nullptr) {
  c->d2h_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, st ? st : c->stream);
}

// Transverse and longitudinal grids from the spacing rules (Sec. 3.2).
// Rule 0 keeps g^2 k^2 / h^2 + 4 kappa^2 k^2 / h^4 <= 2 theta - 1 (von
// Neumann bound of the theta-scheme); rule 1 is the printed h_t, i.e. the
// same bound with theta = 1.  h_l >= g alpha k.  N = floor(1 / h_min), with
// a 1e-12 relative slack so exact ratios do not round down.
sfd_status derive_grid(const sfd_string_params& p, double gamma_max, int* n_t, int* n_l) {
  const double k = 1.0 / p.fs;
  const double a = gamma_max * gamma_max * k * k;
  const double b = p.kappa * p.kappa * k * k;
  double h2;
  if (p.grid_rule == SFD_GRID_PRINTED) {
    h2 = 0.5 * (a + std::sqrt(a * a + 16.0 * b));
  } else {
    const double d = 2.0 * p.theta - 1.0;
    h2 = (a + std::sqrt(a * a + 16.0 * d * b)) / (2.0 * d);
  }
  const double nt = std::floor((1.0 / std::sqrt(h2)) * (1.0 + 1e-12));
  const double nl = std::floor((1.0 / (gamma_max * p.alpha * k)) * (1.0 + 1e-12));
  if (!(nt >= 2.0)) return fail(SFD_EINVAL, "transverse grid has fewer than 2 intervals (f0 too high for fs)");
  if (nt > 4000.0) return fail(SFD_EINVAL, "transverse grid too fine (N_t = %.0f > 4000)", nt);
  if (nl > 16000.0) return fail(SFD_EINVAL, "longitudinal grid too fine (N_l = %.0f > 16000)", nl);
  *n_t = static_cast<int>(nt);
  *n_l = nl < 1.0 ? 1 : static_cast<int>(nl);
  return SFD_OK;
}

int rows_per_lane(int n) {  // odd m with 32 m >= n + 1
  int m = (n + 1 + kWarp - 1) / kWarp;
  if (m < 1) m = 1;
  if ((m & 1) == 0) ++m;
  return m;
}

void point_weights(int n_t, double x, int32_t* node, float* w) {
  double pos = x * n_t;
  int l = static_cast<int>(std::floor(pos));
  if (l < 0) l = 0;
  if (l > n_t - 1) l = n_t - 1;
  *node = l;
  *w = static_cast<float>(pos - l);
}

double n_l_sq(const sfd_string* s) { return static_cast<double>(s->n_l) * s->n_l; }

// Coefficients of the acceleration-form update (see sfd_kernel.cu), FP64 -> FP32.
// Best rational approximation num/den of x > 0 with num, den < 2^24
// (continued-fraction convergents and the last semiconvergent).
static void rational24(double x, double* num, double* den) {
  const double lim = 16777216.0;   // 2^24
  double p0 = 0, q0 = 1, p1 = 1, q1 = 0, y = x;
  double bp = std::max(1.0, std::min(lim - 1, std::round(x))), bq = 1;
  auto consider = [&](double p, double q) {
    if (p > 0 && q > 0 && p < lim && q < lim && std::fabs(p / q - x) < std::fabs(bp / bq - x)) { bp = p; bq = q; }
  };
  for (int it = 0; it < 64; ++it) {
    const double a = std::floor(y);
    const double p2 = a * p1 + p0, q2 = a * q1 + q0;
    if (p2 >= lim || q2 >= lim) {
      double t = std::floor((lim - 1 - p0) / p1);
      if (q1 > 0) t = std::min(t, std::floor((lim - 1 - q0) / q1));
      if (t >= 1) consider(t * p1 + p0, t * q1 + q0);
      break;
    }
    consider(p2, q2);
    p0 = p1; q0 = q1; p1 = p2; q1 = q2;
    const double f = y - a;
    if (f < 1e-300) break;
    y = 1.0 / f;
  }
  *num = bp;
  *den = bq;
}

// Scale beta of the transverse equation such that beta dg and beta og are
// floats: with dg/og ~ P/Q (P, Q < 2^24), dg' = P 2^e and og' = Q 2^e are
// exact, and beta = og'/og is within a factor 2^(1/2) of 1.  The ratio
// dg'/og' = P/Q matches dg/og to ~1e-14.  Falls back to plain rounding when
// og is zero or the ratio is out of range.
static void exact_matrix_scale(double dg, double og, float* dg_s, float* og_s) {
  *dg_s = static_cast<float>(dg);
  *og_s = static_cast<float>(og);
  if (!(og != 0.0) || !(dg > 0.0)) return;
  const double r = dg / std::fabs(og);
  if (!(r > 1e-6 && r < 1e6)) return;
  double P, Q;
  rational24(r, &P, &Q);
  const int e = static_cast<int>(std::lround(std::log2(std::fabs(og) / Q)));
  *dg_s = static_cast<float>(std::ldexp(P, e));
  *og_s = static_cast<float>(std::copysign(std::ldexp(Q, e), og));
}

void fill_desc(sfd_string* s) {
  const sfd_string_params& p = s->p;
  Desc& D = s->h;
  const double k = s->k, g = s->gamma;
  const double ht = 1.0 / s->n_t, hl = 1.0 / s->n_l;
  D.n_t = s->n_t;
  D.n_l = s->n_l;
  D.n_u = s->n_t - 1;
  D.linear = (p.alpha == 1.0) ? 1 : 0;
  D.n_z = (!D.linear && s->n_l > 1) ? s->n_l - 1 : 0;
  D.m_u = rows_per_lane(D.n_u);
  D.m_z = D.n_z > 0 ? rows_per_lane(D.n_z) : 0;
  // The longitudinal block (1 + s0) I - s1l d2 is nearly diagonal for string
  // losses: fold its off-diagonal into the Gauss-Seidel sweeps (Jacobi
  // contraction 2 s1l / (1 + s0 + 2 s1l)) when that ratio is small.
  {
    const double s1l = p.sigma1 * k * n_l_sq(s);
    D.z_jacobi = (2.0 * s1l / (1.0 + p.sigma0 * k + 2.0 * s1l) <= 0.01) ? 1 : 0;
  }
  D.boundary = p.boundary;
  const double s0 = p.sigma0 * k, s1 = p.sigma1 * k / (ht * ht);
  D.dg = static_cast<float>(p.theta + s0 + 2.0 * s1);
  D.og = static_cast<float>(0.5 * (1.0 - p.theta) - s1);
  // A constant matrix entry rounded to FP32 is a perturbation of the scheme
  // that lasts the whole run: an error of ~3e-8 in dg or og shifts mode
  // frequencies by about as much, a phase error growing with f0 * t that
  // reaches the 1e-4 tolerance over 0.25 s near 2 kHz.  Multiplying the
  // transverse equation by beta (exact_matrix_scale) makes dg and og exact;
  // every other transverse coefficient takes the same factor, computed from
  // the stored entries so that the rows sum to exactly beta (1 + s0).
  exact_matrix_scale(p.theta + s0 + 2.0 * s1, 0.5 * (1.0 - p.theta) - s1, &D.dg, &D.og);
  const double rho = (static_cast<double>(D.dg) + 2.0 * static_cast<double>(D.og)) / (1.0 + s0);
  D.s0 = static_cast<float>(s0);
  D.s0u = static_cast<float>(s0 * rho);
  D.s1 = static_cast<float>(s1 * rho);
  D.s1l = static_cast<float>(p.sigma1 * k / (hl * hl));
  const double lam2 = g * g * k * k / (ht * ht) * rho;   // carried as a float pair
  D.lam2 = static_cast<float>(lam2);
  D.lam2_lo = static_cast<float>(lam2 - static_cast<double>(D.lam2));
  D.mu2 = static_cast<float>(p.kappa * p.kappa * k * k / (ht * ht * ht * ht) * rho);
  D.lam2l = static_cast<float>(g * g * p.alpha * p.alpha * k * k / (hl * hl));
  const double phi = 0.5 * g * g * (p.alpha * p.alpha - 1.0);   // phi' of Eq. 4
  D.ca = static_cast<float>(phi * k * k / (2.0 * ht * ht * ht * ht) * rho);
  D.cb = static_cast<float>(phi * k * k / (2.0 * ht * ht * ht) * rho);
  D.cz = static_cast<float>(phi * k * k / (2.0 * ht * ht * hl));
  D.out_scale = static_cast<float>(p.length_m);
  point_weights(s->n_t, p.pickup_pos, &D.o_node, &D.o_w);
  D.out_ch = p.output;
  point_weights(s->n_l, p.pickup_pos, &D.ol_node, &D.ol_w);
  D.jscale = static_cast<float>(s->n_t * rho);
  // The FP32 factorisation of the transverse matrix is itself a lasting
  // perturbation of the same size.  Strings of at most 31 unknowns (f0
  // above ~450 Hz, the most cycles in a given time) correct each solve once
  // against the exact matrix.
  D.refine = D.m_u == 1 ? 1 : 0;
  D.k = static_cast<float>(k);
  D.k2 = static_cast<float>(k * k);
  D.exc = s->exc;
}

size_t block_bytes(const Desc& D) {
  size_t b = 0;
  auto take = [&](size_t n) { b = (b + kAlign - 1) / kAlign * kAlign + n; };
  take(sizeof(Desc));
  take(sizeof(Scalars));
  take(sizeof(float) * D.n_u);
  take(sizeof(float) * D.n_u);
  for (int a = 0; a < 4; ++a) take(sizeof(float) * (D.n_z > 0 ? D.n_z : 1));
  return (b + kAlign - 1) / kAlign * kAlign;
}

void carve(sfd_string* s) {
  size_t b = 0;
  auto take = [&](size_t n) {
    b = (b + kAlign - 1) / kAlign * kAlign;
    char* p = s->block + b;
    b += n;
    return p;
  };
  Desc& D = s->h;
  s->d_desc = reinterpret_cast<Desc*>(take(sizeof(Desc)));
  s->d_sc = reinterpret_cast<Scalars*>(take(sizeof(Scalars)));
  const size_t nz = D.n_z > 0 ? D.n_z : 1;
  D.u = reinterpret_cast<float*>(take(sizeof(float) * D.n_u));
  D.du = reinterpret_cast<float*>(take(sizeof(float) * D.n_u));
  D.z = reinterpret_cast<float*>(take(sizeof(float) * nz));
  D.dz = reinterpret_cast<float*>(take(sizeof(float) * nz));
  D.xz = reinterpret_cast<float*>(take(sizeof(float) * nz));
  D.az = reinterpret_cast<float*>(take(sizeof(float) * nz));
  D.sc = s->d_sc;
}

// Host image of a carved string's whole pool block (block_bytes(s->h)
// bytes at img): the descriptor, the scalars and the initial state w^0, w^1
// of Sec. 3.4 (pluck triangle or rest; the hammer at the rest position
// moving with v_H), zero elsewhere.
void write_image(const sfd_string* s, char* img) {
  const Desc& D = s->h;
  const size_t bytes = block_bytes(D);
  std::memset(img, 0, bytes);
  auto at = [&](const void* dev) { return img + (static_cast<const char*>(dev) - s->block); };
  std::memcpy(at(s->d_desc), &D, sizeof(Desc));
  Scalars sc{};
  sc.n = 1;
  sc.next_out = 0;
  if (s->exc == kHammer) {
    sc.uh = static_cast<float>(s->hammer_uh1);
    sc.duh = static_cast<float>(s->hammer_uh1);
  }
  std::memcpy(at(s->d_sc), &sc, sizeof(Scalars));
  if (s->exc == kPluck && s->pluck_amp != 0.0) {
    float* u = reinterpret_cast<float*>(at(D.u));
    const double c0 = s->pluck_amp / s->p.length_m, xp = s->pluck_pos;
    for (int l = 1; l < s->n_t; ++l) {
      const double x = static_cast<double>(l) / s->n_t;
      u[l - 1] = static_cast<float>(x <= xp ? c0 * x / xp : c0 * (1.0 - x) / (1.0 - xp));
    }
  }
}

// A string's device block (descriptor, scalars, initial state) is written
// on first use: creation, excitation, modulation and envelope calls only
// update the host descriptor and mark the string, and every call that runs
// or reads a string first flushes the marked ones, each with one
// asynchronous copy from the context's pinned staging buffer, ordered on the
// stream before the call's own work (no synchronisation per string).
void stage_initial(sfd_string* s) { s->dirty = true; }

sfd_status flush_strings(sfd_ctx* c, const sfd_string* const* ss, size_t n) {
  constexpr size_t kA = 256;
  size_t bytes = 0;
  for (size_t i = 0; i < n; ++i)
    if (ss[i]->dirty) bytes += (block_bytes(ss[i]->h) + kA - 1) / kA * kA;
  if (bytes == 0) return SFD_OK;
  if (c->stage_pending) {   // the previous flush's copies still read the buffer
    SFD_CUDA(cudaEventSynchronize(c->stage_done));
    c->stage_pending = false;
  }
  if (bytes > c->stage_cap) {
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    const size_t cap = std::max(bytes, size_t{1} << 20);
    SFD_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&c->stage), cap, cudaHostAllocDefault));
    c->stage_cap = cap;
  }
  if (!c->stage_done) SFD_CUDA(cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming));
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    const sfd_string* s = ss[i];
    if (!s->dirty) continue;
    const size_t bb = block_bytes(s->h);
    write_image(s, c->stage + off);
    e = h2d(c, s->block, c->stage + off, bb);
    if (e == cudaSuccess) s->dirty = false;
    off += (bb + kA - 1) / kA * kA;
  }
  // copies already enqueued read the buffer until this event, even after an error
  const cudaError_t er = cudaEventRecord(c->stage_done, c->stream);
  c->stage_pending = er == cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "upload of initial blocks");
  if (er != cudaSuccess) {
    cudaStreamSynchronize(c->stream);
    return cuda_fail(er, "cudaEventRecord");
  }
  return SFD_OK;
}

sfd_status flush_string(const sfd_string* s) { return flush_strings(s->ctx, &s, 1); }

// Upload the descriptor and the initial state now (one copy of the block image).
sfd_status upload_initial(sfd_string* s) {
  std::vector<char> img(block_bytes(s->h));
  write_image(s, img.data());
  sfd_ctx* c = s->ctx;
  SFD_CUDA(h2d(c, s->block, img.data(), img.size()));
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  return SFD_OK;
}

// Defaults and validation of string parameters (SI units, Table 1 ranges
// are not enforced, only what the scheme needs); gamma = 2 f0 unless given.
sfd_status normalize_params(sfd_string_params& q, double* gamma_out) {
  if (q.length_m == 0) q.length_m = 1.0;
  if (q.fs == 0) q.fs = 48000.0;
  if (q.linear_density == 0) q.linear_density = 5e-3;
  if (q.theta == 0) q.theta = 0.5 * (1.0 + 4.0 / (kPi * kPi));
  if (q.pickup_pos == 0) q.pickup_pos = 0.7;
  if (q.f0_max_ratio < 1.0) q.f0_max_ratio = 1.0;
  const double gamma = q.gamma > 0 ? q.gamma : 2.0 * q.f0;
  if (!(gamma > 0) || !std::isfinite(gamma)) return fail(SFD_EINVAL, "f0/gamma must be > 0");
  if (!(q.fs > 0)) return fail(SFD_EINVAL, "fs must be > 0");
  if (!(q.kappa >= 0)) return fail(SFD_EINVAL, "kappa must be >= 0");
  if (!(q.alpha >= 1.0)) return fail(SFD_EINVAL, "alpha must be >= 1");
  if (!(q.sigma0 >= 0) || !(q.sigma1 >= 0)) return fail(SFD_EINVAL, "losses must be >= 0");
  if (!(q.theta > 0.5 && q.theta <= 1.0)) return fail(SFD_EINVAL, "theta must be in (1/2, 1]");
  if (!(q.pickup_pos > 0 && q.pickup_pos < 1)) return fail(SFD_EINVAL, "pickup must be in (0, 1)");
  if (!(q.length_m > 0) || !(q.linear_density > 0)) return fail(SFD_EINVAL, "length and density must be > 0");
  if (q.boundary != 0 && q.boundary != 1) return fail(SFD_EINVAL, "bad boundary");
  if (q.grid_rule != 0 && q.grid_rule != 1) return fail(SFD_EINVAL, "bad grid rule");
  if (q.output != SFD_OUTPUT_TRANSVERSE && q.output != SFD_OUTPUT_LONGITUDINAL)
    return fail(SFD_EINVAL, "bad output channel");
  *gamma_out = gamma;
  return SFD_OK;
}

// Host part of sfd_string_create: parameters, grid and descriptor (no
// device access; s->ctx, block and device pointers are left unset).
sfd_status init_host_string(const sfd_string_params& p, sfd_string* s) {
  s->p = p;
  double gamma = 0;
  sfd_status rc = normalize_params(s->p, &gamma);
  if (rc) return rc;
  int n_t = 0, n_l = 0;
  if ((rc = derive_grid(s->p, gamma * s->p.f0_max_ratio, &n_t, &n_l))) return rc;
  s->gamma = gamma;
  s->k = 1.0 / s->p.fs;
  s->n_t = n_t;
  s->n_l = n_l;
  s->exc = kPluck;
  s->h.bow_release_n = INT64_MAX;
  fill_desc(s);
  return SFD_OK;
}

// Excitation fields of the descriptor at their values for a string that has
// none (every excitation call starts from here, so the descriptor depends
// only on the last excitation set, not on the ones before it).
void clear_excitation(Desc& D) {
  D.e_node = 0;
  D.e_w = 0.f;
  D.ham_M = D.ham_k2w = D.ham_expo = 0.f;
  D.bow_F = D.bow_v = D.bow_a = D.bow_eps = 0.f;
  D.bow_release_n = INT64_MAX;
  D.bow_env_n = 0;
  for (int j = 0; j < 16; ++j) {
    D.bow_env_t[j] = 0.0;
    D.bow_env_v[j] = D.bow_env_f[j] = D.bow_env_x[j] = 0.f;
  }
}

// Record of the last excitation call (a new excitation drops the envelope,
// as sfd_excite_bow does).
void record_excitation(sfd_string* s, int32_t kind, std::initializer_list<double> args) {
  s->rec_exc = kind;
  int j = 0;
  for (double a : args) s->rec_exc_args[j++] = a;
  s->rec_env_n = 0;
  s->rec_env_mask = 0;
  for (auto& row : s->rec_env)
    for (double& v : row) v = 0.0;
}

void record_modulation(sfd_string* s, int32_t kind, double rate_hz, double depth, double phase_rad,
                       double duration_s) {
  s->rec_mod = kind;
  s->rec_mod_args[0] = rate_hz;
  s->rec_mod_args[1] = depth;
  s->rec_mod_args[2] = phase_rad;
  s->rec_mod_args[3] = duration_s;
}

// Excitation of Sec. 3.3 / Eqs. 5-6 set on the host copy (as the
// sfd_excite_* calls do; the pluck is the initial condition).
sfd_status apply_excitation(sfd_string* s, const sfd_excitation& ex) {
  const sfd_string_params& q = s->p;
  const double pos = ex.pos;
  if (!(pos > 0 && pos < 1)) return fail(SFD_EINVAL, "excitation position must be in (0, 1)");
  if (ex.kind == kPluck) {
    if (!std::isfinite(ex.amp_m)) return fail(SFD_EINVAL, "bad pluck amplitude");
    s->exc = kPluck;
    s->pluck_amp = ex.amp_m;
    s->pluck_pos = pos;
    fill_desc(s);
    clear_excitation(s->h);
  } else if (ex.kind == kHammer) {
    if (!(ex.mass_kg > 0) || !(ex.omega_h > 0) || !(ex.alpha_h >= 1) || !std::isfinite(ex.vel_mps))
      return fail(SFD_EINVAL, "bad hammer parameters");
    s->exc = kHammer;
    s->pluck_amp = 0;
    fill_desc(s);
    clear_excitation(s->h);
    point_weights(s->n_t, pos, &s->h.e_node, &s->h.e_w);
    s->exc_pos = pos;
    s->h.ham_M = static_cast<float>(ex.mass_kg / (q.linear_density * q.length_m));
    s->h.ham_k2w = static_cast<float>(s->k * s->k * std::pow(ex.omega_h, 1.0 + ex.alpha_h));
    s->h.ham_expo = static_cast<float>(ex.alpha_h - 1.0);
    s->hammer_uh1 = (ex.vel_mps / q.length_m) * s->k;
  } else if (ex.kind == kBow) {
    if (!(ex.force_n >= 0) || !(ex.eps >= 0 && ex.eps <= 1) || !(ex.a_s_per_m >= 0) || !std::isfinite(ex.vel_mps))
      return fail(SFD_EINVAL, "bad bow parameters");
    s->exc = kBow;
    s->pluck_amp = 0;
    fill_desc(s);
    clear_excitation(s->h);
    point_weights(s->n_t, pos, &s->h.e_node, &s->h.e_w);
    s->exc_pos = pos;
    s->h.bow_F = static_cast<float>(ex.force_n / (q.linear_density * q.length_m * q.length_m));
    s->h.bow_v = static_cast<float>(ex.vel_mps / q.length_m);
    s->h.bow_a = static_cast<float>(ex.a_s_per_m * q.length_m);
    s->h.bow_eps = static_cast<float>(ex.eps);
    s->h.bow_env_n = 0;
    s->bow_pos = pos;
    s->h.bow_release_n = INT64_MAX;
    if (ex.release_time_s >= 0) {
      // first step n with n k >= release
      int64_t n = static_cast<int64_t>(std::ceil(ex.release_time_s * q.fs));
      while (n > 0 && static_cast<double>(n - 1) * s->k >= ex.release_time_s) --n;
      while (static_cast<double>(n) * s->k < ex.release_time_s) ++n;
      s->h.bow_release_n = n;
    }
  } else {
    return fail(SFD_EINVAL, "bad excitation kind %d", ex.kind);
  }
  return SFD_OK;
}

// Largest wave-speed ratio gamma^n / gamma a modulation reaches (reading
// A14): vibrato 2^{|c| / 1200}, glissando 2^{max(D, 0)}; 1 without one.
double modulation_peak(int32_t kind, double depth) {
  if (kind == SFD_MOD_VIBRATO) return std::pow(2.0, std::fabs(depth) / 1200.0);
  if (kind == SFD_MOD_GLISS) return std::pow(2.0, std::max(0.0, depth));
  return 1.0;
}

// Re-derive the grid of a string (host copy) for the peak wave speed
// gamma * ratio (reading A14: the grid of a modulated note is the one of its
// largest gamma): N_t, N_l, the descriptor and the excitation point.  The
// excitation's other fields, a bow envelope and the pluck (sampled on the
// grid when the block is written) carry over.
sfd_status regrid_host(sfd_string* s, double ratio) {
  sfd_string_params q = s->p;
  q.f0_max_ratio = ratio;
  int n_t = 0, n_l = 0;
  sfd_status rc = derive_grid(q, s->gamma * ratio, &n_t, &n_l);
  if (rc) return rc;
  s->p = q;
  s->n_t = n_t;
  s->n_l = n_l;
  fill_desc(s);
  if (s->exc != kPluck) point_weights(s->n_t, s->exc_pos, &s->h.e_node, &s->h.e_w);
  return SFD_OK;
}

// Fractional part of x as a 64-bit fixed-point fraction (x 2^64 mod 2^64).
uint64_t frac_fx(double x) {
  const double f = x - std::floor(x);             // [0, 1]: 1 only by rounding, taken as 0
  const double p = std::ldexp(f, 64);
  return p >= 18446744073709551616.0 ? 0 : static_cast<uint64_t>(p);
}

// f0 modulation on the host copy of the descriptor (reading A14).  Every
// modulation field is rewritten, so the descriptor depends only on the last
// modulation set.
sfd_status apply_modulation(sfd_string* s, int32_t kind, double rate_hz, double depth, double phase_rad,
                            double duration_s) {
  Desc& D = s->h;
  if (kind == SFD_MOD_VIBRATO) {
    if (!std::isfinite(rate_hz) || !std::isfinite(depth) || !std::isfinite(phase_rad))
      return fail(SFD_EINVAL, "bad vibrato");
    if (std::pow(2.0, std::fabs(depth) / 1200.0) > s->p.f0_max_ratio * (1.0 + 1e-12))
      return fail(SFD_EINVAL, "vibrato peak exceeds the grid's f0_max_ratio");
  } else if (kind == SFD_MOD_GLISS) {
    if (!(duration_s > 0) || !std::isfinite(duration_s) || !std::isfinite(depth))
      return fail(SFD_EINVAL, "bad glissando");
    if (std::pow(2.0, std::max(0.0, depth)) > s->p.f0_max_ratio * (1.0 + 1e-12))
      return fail(SFD_EINVAL, "glissando peak exceeds the grid's f0_max_ratio");
  } else if (kind != SFD_MOD_NONE) {
    return fail(SFD_EINVAL, "bad modulation kind");
  }
  D.mod_kind = 0;
  D.mod_inc_fx = 0;
  D.mod_phase_fx = 0;
  D.mod_depth2 = 0.f;
  D.mod_inc = 0.f;
  D.mod_hold = 0.f;
  D.mod_n_end = 0;
  if (kind == SFD_MOD_VIBRATO) {
    D.mod_kind = 1;
    D.mod_inc_fx = frac_fx(rate_hz * s->k);
    D.mod_phase_fx = frac_fx(phase_rad / (2.0 * kPi));
    D.mod_depth2 = static_cast<float>(2.0 * depth / 1200.0);
  } else if (kind == SFD_MOD_GLISS) {
    D.mod_kind = 2;
    D.mod_inc = static_cast<float>(2.0 * depth * s->k / duration_s);
    D.mod_hold = static_cast<float>(2.0 * depth);
    // first step n with n k >= T (the same comparison as a bow release)
    const double nt = std::ceil(duration_s * s->p.fs);
    int64_t n = nt < 9.0e18 ? static_cast<int64_t>(nt) : INT64_MAX;
    if (n != INT64_MAX) {
      while (n > 0 && static_cast<double>(n - 1) * s->k >= duration_s) --n;
      while (static_cast<double>(n) * s->k < duration_s) ++n;
    }
    D.mod_n_end = n;
  }
  return SFD_OK;
}

sfd_status ensure_jobs(sfd_ctx* c, int n) {
  if (n <= c->job_cap) return SFD_OK;
  if (c->d_jobs) cudaFree(c->d_jobs);
  c->d_jobs = nullptr;
  int cap = std::max(n, 64);
  SFD_CUDA(cudaMalloc(&c->d_jobs, sizeof(Job) * cap));
  c->job_cap = cap;
  return SFD_OK;
}

double job_cost(const sfd_string* s, int64_t n) {
  const Desc& D = s->h;
  double per = D.m_u * 3.0 + 40.0;
  if (D.n_z > 0) per += 4.0 * (D.m_u + D.m_z + 40.0);
  if (s->exc != kPluck) per *= 1.5;
  return per * static_cast<double>(n);
}

int job_class(const Desc& D) {
  if (D.m_u <= kMaxRegRows && (D.m_u & 1)) return D.m_u / 2;
  return kClasses - 1;
}

using Launcher = cudaError_t (*)(const Job*, int, int*, int, int, int, int, cudaStream_t);
const Launcher kLaunch[kClasses] = {launch_synth_reg1, launch_synth_reg3, launch_synth_reg5,
                                    launch_synth_reg7, launch_synth_reg9, launch_synth_smem};

// A launch plan: jobs grouped by kernel class (transverse rows per lane),
// each class sorted longest first (the order its work queue hands them
// out), with each class's shared-memory need and the warps per CTA.
struct Plan {
  std::vector<Job> jobs;
  int first[kClasses + 1] = {};
  int wf[kClasses] = {};
  int group[kClasses] = {};  // warps per string of the class's launch (1, 2 or 4)
  int order[kClasses] = {};  // launch order of the classes: heaviest step first
  int wpc = 1;
};

sfd_status make_plan(const sfd_ctx* c, const std::vector<Job>& jobs, const std::vector<const sfd_string*>& owners,
                     int wpc_override, Plan& P, int groups_override = -1) {
  const int nj = static_cast<int>(jobs.size());
  std::vector<int> order(nj), cls(nj);
  std::vector<double> cost(nj);
  for (int i = 0; i < nj; ++i) {
    order[i] = i;
    cls[i] = job_class(owners[i]->h);
    cost[i] = job_cost(owners[i], jobs[i].n_samples);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (cls[a] != cls[b]) return cls[a] < cls[b];
    return cost[a] > cost[b];
  });
  P.jobs.assign(nj, Job{});
  for (int k = 0; k <= kClasses; ++k) P.first[k] = 0;
  for (int k = 0; k < kClasses; ++k) P.wf[k] = 0;
  for (int i = 0; i < nj; ++i) {
    P.jobs[i] = jobs[order[i]];
    P.jobs[i].sweep_cap = c->sweep_cap;
  }
  for (int i = 0; i < nj; ++i) {
    const int k = cls[order[i]];
    P.first[k + 1]++;
    const Desc& D = owners[order[i]]->h;
    P.wf[k] = std::max(P.wf[k], warp_smem_floats(D.m_u, D.m_z, D.z_jacobi));
  }
  for (int k = 0; k < kClasses; ++k) P.first[k + 1] += P.first[k];
  for (int k = 0; k < kClasses; ++k) {
    if (static_cast<size_t>(P.wf[k]) * sizeof(float) > c->smem_optin)
      return fail(SFD_EINVAL, "string too large for one warp's shared memory");
  }
  // Classes are launched heaviest step first (shared-memory grids, then 9,
  // 7, 5, 3, 1 rows per lane).  The block scheduler starts CTAs in launch
  // order, and a class's persistent CTAs keep taking its jobs until its
  // queue is empty, so when the batch does not fit on the GPU at once the
  // class launched first holds the SMs; launched last, the slowest strings
  // would start only when a lighter class drains and finish last (measured
  // on the 4096-string batch: 5.3 s per step heaviest first against 6.7 s
  // lightest first; ordering by the host's cost estimate of each class's
  // longest job put the three 7-row strings behind the 3-row class, which
  // alone has more CTAs than the GPU holds, and gave 6.2 s).
  for (int k = 0; k < kClasses; ++k) P.order[k] = kClasses - 1 - k;
  // warps per CTA: ceil(jobs / SMs), 1..4.  Warps of one CTA sit on
  // different SM sub-partitions, so pairing jobs in a CTA keeps each string
  // on a scheduler of its own (measured on the 256-string batch: 2 warps per
  // CTA 27.3 M samples/s vs 19.9 M with single-warp CTAs).
  int wpc = std::max(1, std::min(4, (nj + c->sm_count - 1) / std::max(c->sm_count, 1)));
  if (const char* env = getenv("SFD_WARPS_PER_CTA")) {
    const int v = atoi(env);
    if (v >= 1 && v <= 4) wpc = v;
  }
  if (wpc_override >= 1 && wpc_override <= 4) wpc = wpc_override;
  P.wpc = wpc;
  // Warp groups: a string stepped by 2 or 4 warps of one SM (each does the
  // transverse side, each a share of the longitudinal rows) finishes its
  // steps sooner when its longitudinal grid is large.  Classes whose strings
  // have such grids (folded into the sweeps; >= 3 rows per lane for pairs,
  // >= 7 for groups of 4) get groups, heaviest class first, while the
  // launch's warps stay within one per SM sub-partition, so groups only use
  // schedulers that would otherwise idle.
  for (int k = 0; k < kClasses; ++k) P.group[k] = 1;
  if (groups_override < 0 ? c->warp_pairs : groups_override) {
    int warps = nj;
    for (int k = kClasses - 2; k >= 0; --k) {
      const int n_k = P.first[k + 1] - P.first[k];
      int max_mz = 0;
      for (int i = P.first[k]; i < P.first[k + 1]; ++i) {
        const Desc& D = owners[order[i]]->h;
        if (D.z_jacobi) max_mz = std::max(max_mz, D.m_z);
      }
      if (max_mz >= 7 && warps + 3 * n_k <= 4 * c->sm_count) {
        P.group[k] = 4;
        warps += 3 * n_k;
      } else if (max_mz >= 3 && warps + n_k <= 4 * c->sm_count) {
        P.group[k] = 2;
        warps += n_k;
      }
    }
  }
  return SFD_OK;
}

// Issue the plan's kernels on the context stream (job table already in
// device memory at d_jobs).  Classes run concurrently on side streams forked
// from and joined back to the context stream.  No host<->device copies, so
// this can be captured into a CUDA graph.
sfd_status issue_plan(sfd_ctx* c, const Plan& P, const Job* d_jobs) {
  c->last_launches = 0;
  int active = 0;
  for (int k = 0; k < kClasses; ++k) active += P.first[k + 1] > P.first[k];
  if (active == 0) return SFD_OK;
  if (active > 1) SFD_CUDA(cudaEventRecord(c->fork, c->stream));
  for (int k = 0; k < kClasses; ++k) c->timed_jobs[k] = 0;
  for (int kk = 0; kk < kClasses; ++kk) {
    const int k = P.order[kk];
    const int n_k = P.first[k + 1] - P.first[k];
    if (n_k == 0) continue;
    const size_t wbytes = static_cast<size_t>(P.wf[k]) * sizeof(float);
    // strings (regions) per CTA, limited by shared memory; a group of warps
    // per string (at most 4 warps per CTA)
    const int g = P.group[k];
    int regions = static_cast<int>(std::min<size_t>(static_cast<size_t>(P.wpc), c->smem_optin / wbytes));
    regions = std::max(1, std::min(regions, 4 / g));
    const int wpc = regions * g;
    const int n_ctas = (n_k + regions - 1) / regions;
    cudaStream_t st = c->stream;
    if (active > 1) {
      st = c->side[k];
      SFD_CUDA(cudaStreamWaitEvent(st, c->fork, 0));
    }
    if (c->timing) SFD_CUDA(cudaEventRecord(c->t0[k], st));
    cudaError_t e = kLaunch[k](d_jobs + P.first[k], n_k, c->d_counter + k, P.wf[k], wpc, n_ctas, P.group[k], st);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (c->timing) {
      SFD_CUDA(cudaEventRecord(c->t1[k], st));
      c->timed_jobs[k] = n_k;
    }
    c->last_launches++;
    if (active > 1) {
      SFD_CUDA(cudaEventRecord(c->join[k], st));
      SFD_CUDA(cudaStreamWaitEvent(c->stream, c->join[k], 0));
    }
  }
  return SFD_OK;
}

// Queue the persistent kernels for `jobs` on the context stream (job table
// uploaded into the context's table).
sfd_status launch_jobs(sfd_ctx* c, std::vector<Job>& jobs, const std::vector<const sfd_string*>& owners,
                       int wpc_override = 0, int groups_override = -1, Plan* keep = nullptr) {
  c->last_launches = 0;
  if (jobs.empty()) return SFD_OK;
  Plan P;
  sfd_status rc = make_plan(c, jobs, owners, wpc_override, P, groups_override);
  if (rc) return rc;
  rc = ensure_jobs(c, static_cast<int>(P.jobs.size()));
  if (rc) return rc;
  SFD_CUDA(h2d(c, c->d_jobs, P.jobs.data(), sizeof(Job) * P.jobs.size()));
  rc = issue_plan(c, P, c->d_jobs);
  if (keep) *keep = std::move(P);
  return rc;
}

// Copy every job's output from the device to out_host (the same offsets
// from dout), each class's jobs on the context's copy stream as soon as
// that class's kernel has ended (its join event), so that only the last
// class's copies follow the launch's end; the context stream then waits for
// them.  A plan with one class, whose kernel ran on the context stream,
// copies after it there.
sfd_status copy_out_by_class(sfd_ctx* c, const Plan& P, const float* dout, float* out_host) {
  int active = 0;
  for (int k = 0; k < kClasses; ++k) active += P.first[k + 1] > P.first[k];
  const cudaStream_t st = active > 1 ? c->copy : c->stream;
  for (int kk = 0; kk < kClasses; ++kk) {
    const int k = P.order[kk];
    if (P.first[k + 1] == P.first[k]) continue;
    if (active > 1) SFD_CUDA(cudaStreamWaitEvent(st, c->join[k], 0));
    for (int j = P.first[k]; j < P.first[k + 1]; ++j) {
      const Job& J = P.jobs[j];
      SFD_CUDA(d2h(c, out_host + (J.out - dout), J.out, sizeof(float) * static_cast<size_t>(J.n_samples), st));
    }
  }
  if (active > 1) {
    SFD_CUDA(cudaEventRecord(c->copied, st));
    SFD_CUDA(cudaStreamWaitEvent(c->stream, c->copied, 0));
  }
  return SFD_OK;
}

sfd_status read_status(const sfd_string* s, Scalars* out) {
  SFD_CUDA(d2h(s->ctx, out, s->d_sc, sizeof(Scalars)));
  SFD_CUDA(cudaStreamSynchronize(s->ctx->stream));
  return SFD_OK;
}

sfd_status status_code(const Scalars& sc) {
  if (sc.status & kStUnstable) return SFD_EUNSTABLE;
  if (sc.status & kStNoConv) return SFD_ENOCONV;
  return SFD_OK;
}

// ---- checkpoints (sfd_string_save / sfd_string_load) ----
// A checkpoint is [header | set-up record | descriptor | state]: the
// parameters and the set-up calls as last made, the descriptor the library
// derived from them (device pointers zeroed), and the string's device block
// from its scalars on (Scalars, u, D, z, Dz and the two longitudinal warm
// starts, in the block's own layout).  Loading replays the set-up calls
// through the public entry points, which validate them, and accepts the
// checkpoint only if the descriptor they give equals the saved one byte for
// byte; so the kernels only ever see a descriptor this library computed,
// and the resumed note continues bit for bit.
constexpr char kCkptMagic[8] = {'S', 'F', 'D', 'S', 'T', 'R', 'C', 'K'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  uint64_t total_bytes;
  uint32_t params_bytes, desc_bytes, scalars_bytes, record_bytes;
  uint64_t state_offset, state_bytes;   // the state's place in the device block and its size
  int32_t n_t, n_l, started, pad_;
};

struct CkptRecord {
  sfd_string_params p;
  int32_t exc, env_n, env_mask, mod;
  double exc_args[6];
  double env[4][16];
  double mod_args[4];
};

// The descriptor with its device pointers cleared (the part a checkpoint
// compares).
Desc portable_desc(const Desc& D) {
  Desc P;
  std::memcpy(&P, &D, sizeof(Desc));
  P.u = P.du = P.z = P.dz = P.xz = P.az = nullptr;
  P.sc = nullptr;
  return P;
}

size_t ckpt_state_offset(const sfd_string* s) {
  return static_cast<size_t>(reinterpret_cast<const char*>(s->d_sc) - s->block);
}

}  // namespace

extern "C" {

void sfd_params_default(sfd_string_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->f0 = 110.0;
  p->kappa = 1.0;
  p->alpha = 1.0;
  p->sigma0 = 0.5;
  p->sigma1 = 1e-5;
  p->length_m = 1.0;
  p->fs = 48000.0;
  p->linear_density = 5e-3;
  p->theta = 0.5 * (1.0 + 4.0 / (kPi * kPi));
  p->boundary = SFD_BOUNDARY_CLAMPED;
  p->grid_rule = SFD_GRID_THETA_BOUND;
  p->pickup_pos = 0.7;
  p->f0_max_ratio = 1.0;
}

const char* sfd_last_error(void) { return g_err.c_str(); }

sfd_status sfd_ctx_create(int device, void* cuda_stream, size_t mem_budget_bytes, sfd_ctx** out) {
  if (!out) return fail(SFD_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(SFD_ECUDA, "no CUDA device available");
  if (device < 0 || device >= ndev) return fail(SFD_EINVAL, "device %d out of range", device);
  sfd_ctx* c = new (std::nothrow) sfd_ctx();
  if (!c) return fail(SFD_ENOMEM, "host allocation failed");
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if ((e = cudaSetDevice(device)) != cudaSuccess) { delete c; return cuda_fail(e, "cudaSetDevice"); }
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) { delete c; return cuda_fail(e, "props"); }
  if (prop.major * 10 + prop.minor < 100) {
    delete c;
    return fail(SFD_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
                prop.minor);
  }
  c->sm_count = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin - kStaticSmemBytes;
  sfd_status rc = c->pool.init(mem_budget_bytes ? mem_budget_bytes : (size_t{256} << 20));
  if (rc) { delete c; return rc; }
  if ((e = cudaMalloc(&c->d_counter, sizeof(int) * kClasses)) != cudaSuccess) {
    c->pool.release();
    delete c;
    return cuda_fail(e, "cudaMalloc(counter)");
  }
  bool ok = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->copied, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < kClasses && ok; ++k) {
    ok = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->join[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreate(&c->t0[k]) == cudaSuccess && cudaEventCreate(&c->t1[k]) == cudaSuccess;
  }
  if (!ok) {
    sfd_ctx_destroy(c);
    return fail(SFD_ECUDA, "stream/event creation failed");
  }
  *out = c;
  return SFD_OK;
}

void sfd_ctx_destroy(sfd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (int k = 0; k < kClasses; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->join[k]) cudaEventDestroy(c->join[k]);
    if (c->t0[k]) cudaEventDestroy(c->t0[k]);
    if (c->t1[k]) cudaEventDestroy(c->t1[k]);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->copy) cudaStreamDestroy(c->copy);
  if (c->copied) cudaEventDestroy(c->copied);
  if (c->stage_done) cudaEventDestroy(c->stage_done);
  if (c->stage) cudaFreeHost(c->stage);
  c->pool.release();
  if (c->d_jobs) cudaFree(c->d_jobs);
  if (c->d_counter) cudaFree(c->d_counter);
  delete c;
}

sfd_status sfd_ctx_memory(const sfd_ctx* c, size_t* used, size_t* total) {
  if (!c) return fail(SFD_EINVAL, "ctx is NULL");
  if (used) *used = c->pool.used();
  if (total) *total = c->pool.size();
  return SFD_OK;
}

int32_t sfd_last_launch_count(const sfd_ctx* c) { return c ? c->last_launches : 0; }

sfd_status sfd_ctx_set_timing(sfd_ctx* c, int32_t enable) {
  if (!c) return fail(SFD_EINVAL, "ctx is NULL");
  c->timing = enable != 0;
  return SFD_OK;
}

sfd_status sfd_grid(const sfd_string_params* p, int32_t* n_t, int32_t* n_l) {
  if (!p || !n_t || !n_l) return fail(SFD_EINVAL, "NULL argument");
  sfd_string_params q = *p;
  double gamma = 0;
  sfd_status rc = normalize_params(q, &gamma);
  if (rc) return rc;
  int nt = 0, nl = 0;
  if ((rc = derive_grid(q, gamma * q.f0_max_ratio, &nt, &nl))) return rc;
  *n_t = nt;
  *n_l = nl;
  return SFD_OK;
}

sfd_status sfd_ctx_set_sweep_cap(sfd_ctx* c, int32_t cap) {
  if (!c) return fail(SFD_EINVAL, "ctx is NULL");
  if (cap < 0 || cap > kMaxSweepCap) return fail(SFD_EINVAL, "sweep cap must be 0 (default %d) or 1..%d", kMaxSweeps,
                                                 kMaxSweepCap);
  c->sweep_cap = cap;
  return SFD_OK;
}

sfd_status sfd_modulation_peak(int32_t kind, double depth, double* ratio) {
  if (!ratio) return fail(SFD_EINVAL, "ratio is NULL");
  if (kind != SFD_MOD_NONE && kind != SFD_MOD_VIBRATO && kind != SFD_MOD_GLISS)
    return fail(SFD_EINVAL, "bad modulation kind");
  if (!std::isfinite(depth)) return fail(SFD_EINVAL, "bad modulation depth");
  *ratio = modulation_peak(kind, depth);
  return SFD_OK;
}

sfd_status sfd_ctx_set_warp_pairs(sfd_ctx* c, int32_t enable) {
  if (!c) return fail(SFD_EINVAL, "ctx is NULL");
  c->warp_pairs = enable != 0;
  return SFD_OK;
}

sfd_status sfd_ctx_kernel_times(sfd_ctx* c, float* ms, int32_t* n_jobs) {
  if (!c || !ms || !n_jobs) return fail(SFD_EINVAL, "NULL argument");
  sfd_status rc = set_device(c);
  if (rc) return rc;
  for (int k = 0; k < kClasses; ++k) {
    ms[k] = 0.f;
    n_jobs[k] = c->timing ? c->timed_jobs[k] : 0;
    if (n_jobs[k] == 0) continue;
    SFD_CUDA(cudaEventSynchronize(c->t1[k]));
    SFD_CUDA(cudaEventElapsedTime(&ms[k], c->t0[k], c->t1[k]));
  }
  return SFD_OK;
}

sfd_status sfd_string_kernel_class(const sfd_string* s, int32_t* cls) {
  if (!s || !cls) return fail(SFD_EINVAL, "NULL argument");
  *cls = job_class(s->h);
  return SFD_OK;
}

sfd_status sfd_ctx_transfer_bytes(const sfd_ctx* c, uint64_t* h2d_total, uint64_t* d2h_total) {
  if (!c) return fail(SFD_EINVAL, "ctx is NULL");
  if (h2d_total) *h2d_total = c->h2d_bytes;
  if (d2h_total) *d2h_total = c->d2h_bytes;
  return SFD_OK;
}

sfd_status sfd_string_create(sfd_ctx* c, const sfd_string_params* p, sfd_string** out) {
  if (!c || !p || !out) return fail(SFD_EINVAL, "NULL argument");
  *out = nullptr;
  sfd_string* s = new (std::nothrow) sfd_string();
  if (!s) return fail(SFD_ENOMEM, "host allocation failed");
  sfd_status rc = init_host_string(*p, s);
  if (rc) { delete s; return rc; }
  s->ctx = c;
  const int n_t = s->n_t, n_l = s->n_l;
  const size_t wbytes = static_cast<size_t>(warp_smem_floats(s->h.m_u, s->h.m_z, s->h.z_jacobi)) * sizeof(float);
  if (wbytes > c->smem_optin) {
    delete s;
    return fail(SFD_EINVAL, "grid (N_t=%d, N_l=%d) exceeds one warp's shared memory", n_t, n_l);
  }
  if ((rc = set_device(c))) { delete s; return rc; }
  s->block = c->pool.alloc(block_bytes(s->h));
  if (!s->block) {
    delete s;
    return fail(SFD_ENOMEM, "device pool exhausted (%zu of %zu bytes used)", c->pool.used(), c->pool.size());
  }
  carve(s);
  stage_initial(s);
  *out = s;
  return SFD_OK;
}

sfd_status sfd_string_info(const sfd_string* s, int32_t* n_t, int32_t* n_l, double* h_t, double* h_l) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (n_t) *n_t = s->n_t;
  if (n_l) *n_l = s->n_l;
  if (h_t) *h_t = 1.0 / s->n_t;
  if (h_l) *h_l = 1.0 / s->n_l;
  return SFD_OK;
}

sfd_status sfd_excite_pluck(sfd_string* s, double amp_m, double pos) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (s->started) return fail(SFD_ESTATE, "pluck is an initial condition: excite before synthesizing");
  if (!(pos > 0 && pos < 1) || !std::isfinite(amp_m)) return fail(SFD_EINVAL, "bad pluck");
  s->exc = kPluck;
  s->pluck_amp = amp_m;
  s->pluck_pos = pos;
  fill_desc(s);
  clear_excitation(s->h);
  record_excitation(s, kPluck, {amp_m, pos, 0.0, 0.0, 0.0, 0.0});
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  stage_initial(s);
  return SFD_OK;
}

sfd_status sfd_excite_hammer(sfd_string* s, double mass_kg, double vel_mps, double pos, double omega_h,
                             double alpha_h) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (s->started) return fail(SFD_ESTATE, "excite before synthesizing");
  if (!(pos > 0 && pos < 1) || !(mass_kg > 0) || !(omega_h > 0) || !(alpha_h >= 1) || !std::isfinite(vel_mps))
    return fail(SFD_EINVAL, "bad hammer parameters");
  const sfd_string_params& p = s->p;
  s->exc = kHammer;
  fill_desc(s);
  clear_excitation(s->h);
  record_excitation(s, kHammer, {mass_kg, vel_mps, pos, omega_h, alpha_h, 0.0});
  point_weights(s->n_t, pos, &s->h.e_node, &s->h.e_w);
  s->exc_pos = pos;
  s->h.ham_M = static_cast<float>(mass_kg / (p.linear_density * p.length_m));
  s->h.ham_k2w = static_cast<float>(s->k * s->k * std::pow(omega_h, 1.0 + alpha_h));
  s->h.ham_expo = static_cast<float>(alpha_h - 1.0);
  s->pluck_amp = 0;
  s->hammer_uh1 = (vel_mps / p.length_m) * s->k;
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  stage_initial(s);
  return SFD_OK;
}

sfd_status sfd_excite_bow(sfd_string* s, double vel_mps, double force_n, double pos, double a_s_per_m, double eps,
                          double release_time_s) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (s->started) return fail(SFD_ESTATE, "excite before synthesizing");
  if (!(pos > 0 && pos < 1) || !(force_n >= 0) || !(eps >= 0 && eps <= 1) || !(a_s_per_m >= 0) ||
      !std::isfinite(vel_mps))
    return fail(SFD_EINVAL, "bad bow parameters");
  const sfd_string_params& p = s->p;
  s->exc = kBow;
  s->pluck_amp = 0;
  fill_desc(s);
  clear_excitation(s->h);
  record_excitation(s, kBow, {vel_mps, force_n, pos, a_s_per_m, eps, release_time_s});
  point_weights(s->n_t, pos, &s->h.e_node, &s->h.e_w);
  s->exc_pos = pos;
  s->h.bow_F = static_cast<float>(force_n / (p.linear_density * p.length_m * p.length_m));
  s->h.bow_v = static_cast<float>(vel_mps / p.length_m);
  s->h.bow_a = static_cast<float>(a_s_per_m * p.length_m);
  s->h.bow_eps = static_cast<float>(eps);
  s->h.bow_env_n = 0;   // constant controls until sfd_bow_envelope
  s->bow_pos = pos;
  if (release_time_s >= 0) {
    // first step n with n k >= release (same comparison as stated in Eq. 5's use)
    int64_t n = static_cast<int64_t>(std::ceil(release_time_s * p.fs));
    while (n > 0 && static_cast<double>(n - 1) * s->k >= release_time_s) --n;
    while (static_cast<double>(n) * s->k < release_time_s) ++n;
    s->h.bow_release_n = n;
  } else {
    s->h.bow_release_n = INT64_MAX;
  }
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  stage_initial(s);
  return SFD_OK;
}

// Breakpoint envelopes of the bow controls into the host descriptor (times
// in steps, velocity and force in normalised units); NULL arrays keep the
// constant controls.
sfd_status apply_bow_envelope(sfd_string* s, int32_t n_points, const double* t_s, const double* vel_mps,
                              const double* force_n, const double* pos) {
  if (!t_s) return fail(SFD_EINVAL, "NULL breakpoint times");
  if (s->exc != kBow) return fail(SFD_EINVAL, "the string is not bowed (call sfd_excite_bow first)");
  if (n_points < 1 || n_points > 16) return fail(SFD_EINVAL, "1 to 16 breakpoints");
  const sfd_string_params& p = s->p;
  Desc& D = s->h;
  for (int j = 0; j < n_points; ++j) {
    if (!std::isfinite(t_s[j]) || (j > 0 && !(t_s[j] > t_s[j - 1])))
      return fail(SFD_EINVAL, "breakpoint times must increase");
    if (vel_mps && !std::isfinite(vel_mps[j])) return fail(SFD_EINVAL, "bad bow velocity");
    if (force_n && !(force_n[j] >= 0)) return fail(SFD_EINVAL, "bow force must be >= 0");
    if (pos && !(pos[j] > 0 && pos[j] < 1)) return fail(SFD_EINVAL, "bow position must be in (0, 1)");
  }
  // constant controls where an array is NULL: the values of sfd_excite_bow
  const double x0 = s->bow_pos;
  for (int j = 0; j < n_points; ++j) {
    D.bow_env_t[j] = t_s[j] * p.fs;
    D.bow_env_v[j] = vel_mps ? static_cast<float>(vel_mps[j] / p.length_m) : D.bow_v;
    D.bow_env_f[j] = force_n ? static_cast<float>(force_n[j] / (p.linear_density * p.length_m * p.length_m)) : D.bow_F;
    D.bow_env_x[j] = pos ? static_cast<float>(pos[j]) : static_cast<float>(x0);
  }
  D.bow_env_n = n_points;
  return SFD_OK;
}

sfd_status sfd_bow_envelope(sfd_string* s, int32_t n_points, const double* t_s, const double* vel_mps,
                            const double* force_n, const double* pos) {
  if (!s) return fail(SFD_EINVAL, "NULL argument");
  if (s->started) return fail(SFD_ESTATE, "set the bow envelope before synthesizing");
  sfd_status rc = apply_bow_envelope(s, n_points, t_s, vel_mps, force_n, pos);
  if (rc) return rc;
  s->rec_env_n = n_points;
  s->rec_env_mask = (vel_mps ? 1 : 0) | (force_n ? 2 : 0) | (pos ? 4 : 0);
  const double* src[4] = {t_s, vel_mps, force_n, pos};
  for (int c = 0; c < 4; ++c)
    for (int j = 0; j < 16; ++j) s->rec_env[c][j] = (src[c] && j < n_points) ? src[c][j] : 0.0;
  stage_initial(s);
  return SFD_OK;
}

sfd_status sfd_set_modulation(sfd_string* s, int32_t kind, double rate_hz, double depth, double phase_rad,
                              double duration_s) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (s->started) return fail(SFD_ESTATE, "set modulation before synthesizing");
  const double peak = std::isfinite(depth) ? modulation_peak(kind, depth) : 1.0;
  if (!(peak > s->p.f0_max_ratio * (1.0 + 1e-12))) {
    sfd_status rc = apply_modulation(s, kind, rate_hz, depth, phase_rad, duration_s);
    if (rc) return rc;
    record_modulation(s, kind, rate_hz, depth, phase_rad, duration_s);
    stage_initial(s);
    return SFD_OK;
  }
  // The grid is re-derived for the modulation's peak (coarser: a faster wave)
  // in a new pool block; the string keeps its old grid and block unless the
  // modulation is accepted (nothing has run on the old block).
  if (s->batch_refs > 0)
    return fail(SFD_EBUSY, "the grid must change for this modulation's peak: set it before adding the string to a batch");
  sfd_ctx* c = s->ctx;
  const sfd_string saved = *s;
  sfd_status rc = regrid_host(s, peak);
  if (rc == SFD_OK &&
      static_cast<size_t>(warp_smem_floats(s->h.m_u, s->h.m_z, s->h.z_jacobi)) * sizeof(float) > c->smem_optin)
    rc = fail(SFD_EINVAL, "grid (N_t=%d, N_l=%d) exceeds one warp's shared memory", s->n_t, s->n_l);
  if (rc == SFD_OK) rc = apply_modulation(s, kind, rate_hz, depth, phase_rad, duration_s);
  char* nb = nullptr;
  if (rc == SFD_OK && !(nb = c->pool.alloc(block_bytes(s->h))))
    rc = fail(SFD_ENOMEM, "device pool exhausted (%zu of %zu bytes used)", c->pool.used(), c->pool.size());
  if (rc) {
    *s = saved;
    return rc;
  }
  c->pool.dealloc(saved.block);
  s->block = nb;
  carve(s);
  record_modulation(s, kind, rate_hz, depth, phase_rad, duration_s);
  stage_initial(s);
  return SFD_OK;
}

sfd_status sfd_synthesize(sfd_string* s, int64_t n_samples, float* out, int32_t out_on_device) {
  if (!s || (!out && n_samples > 0)) return fail(SFD_EINVAL, "NULL argument");
  if (n_samples < 0) return fail(SFD_EINVAL, "n_samples < 0");
  if (n_samples == 0) return SFD_OK;
  sfd_ctx* c = s->ctx;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  if ((rc = flush_string(s))) return rc;
  float* dout = out;
  char* tmp = nullptr;
  if (!out_on_device) {
    tmp = c->pool.alloc(sizeof(float) * n_samples);
    if (!tmp) return fail(SFD_ENOMEM, "device pool exhausted for the output buffer");
    dout = reinterpret_cast<float*>(tmp);
  }
  std::vector<Job> jobs{Job{s->d_desc, dout, n_samples}};
  std::vector<const sfd_string*> owners{s};
  rc = launch_jobs(c, jobs, owners);
  s->started = true;
  if (rc == SFD_OK && !out_on_device) {
    cudaError_t e = d2h(c, out, dout, sizeof(float) * n_samples);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy out");
  }
  Scalars sc{};
  if (rc == SFD_OK) rc = read_status(s, &sc);
  if (tmp) c->pool.dealloc(tmp);
  if (rc) return rc;
  rc = status_code(sc);
  if (rc == SFD_EUNSTABLE) return fail(rc, "string state became non-finite");
  if (rc == SFD_ENOCONV) return fail(rc, "coupled solve reached its sweep cap (result kept)");
  return SFD_OK;
}

sfd_status sfd_string_position(const sfd_string* s, int64_t* time_level, int64_t* next_sample) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  Scalars sc{};
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  if ((rc = flush_string(s))) return rc;
  if ((rc = read_status(s, &sc))) return rc;
  if (time_level) *time_level = sc.n;
  if (next_sample) *next_sample = sc.next_out;
  return SFD_OK;
}

sfd_status sfd_string_state(const sfd_string* s, float* u_prev, float* u, float* z_prev, float* z) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  if ((rc = flush_string(s))) return rc;
  const Desc& D = s->h;
  const int nz_full = s->n_l - 1;
  std::vector<float> hu(D.n_u), hdu(D.n_u), hz(std::max(D.n_z, 1)), hdz(std::max(D.n_z, 1));
  sfd_ctx* c = s->ctx;
  SFD_CUDA(d2h(c, hu.data(), D.u, sizeof(float) * D.n_u));
  SFD_CUDA(d2h(c, hdu.data(), D.du, sizeof(float) * D.n_u));
  if (D.n_z > 0) {
    SFD_CUDA(d2h(c, hz.data(), D.z, sizeof(float) * D.n_z));
    SFD_CUDA(d2h(c, hdz.data(), D.dz, sizeof(float) * D.n_z));
  }
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < D.n_u; ++i) {
    if (u) u[i] = hu[i];
    if (u_prev) u_prev[i] = hu[i] - hdu[i];
  }
  for (int i = 0; i < nz_full; ++i) {
    const float zv = D.n_z > 0 ? hz[i] : 0.f, dzv = D.n_z > 0 ? hdz[i] : 0.f;
    if (z) z[i] = zv;
    if (z_prev) z_prev[i] = zv - dzv;
  }
  return SFD_OK;
}

sfd_status sfd_string_delta_state(const sfd_string* s, float* u, float* du, float* z, float* dz) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  if ((rc = flush_string(s))) return rc;
  const Desc& D = s->h;
  const int nz_full = s->n_l - 1;
  sfd_ctx* c = s->ctx;
  if (u) SFD_CUDA(d2h(c, u, D.u, sizeof(float) * D.n_u));
  if (du) SFD_CUDA(d2h(c, du, D.du, sizeof(float) * D.n_u));
  if (D.n_z > 0) {
    if (z) SFD_CUDA(d2h(c, z, D.z, sizeof(float) * D.n_z));
    if (dz) SFD_CUDA(d2h(c, dz, D.dz, sizeof(float) * D.n_z));
  }
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  for (int i = std::max(D.n_z, 0); i < nz_full; ++i) {   // no longitudinal grid: zero
    if (z) z[i] = 0.f;
    if (dz) dz[i] = 0.f;
  }
  return SFD_OK;
}

sfd_status sfd_string_hammer(const sfd_string* s, double* u_h_prev, double* u_h) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  if (s->exc != kHammer) return fail(SFD_EINVAL, "the string is not struck by a hammer");
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  Scalars sc{};
  if ((rc = flush_string(s))) return rc;
  if ((rc = read_status(s, &sc))) return rc;
  if (u_h) *u_h = sc.uh;
  if (u_h_prev) *u_h_prev = static_cast<double>(sc.uh) - static_cast<double>(sc.duh);
  return SFD_OK;
}

sfd_status sfd_string_stats(const sfd_string* s, int32_t* status, int32_t* max_sweeps, int64_t* total_sweeps) {
  if (!s) return fail(SFD_EINVAL, "string is NULL");
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  Scalars sc{};
  if ((rc = flush_string(s))) return rc;
  if ((rc = read_status(s, &sc))) return rc;
  if (status) *status = status_code(sc);
  if (max_sweeps) *max_sweeps = sc.max_sweeps;
  if (total_sweeps) *total_sweeps = sc.sweeps_total;
  return SFD_OK;
}

sfd_status sfd_string_destroy(sfd_string* s) {
  if (!s) return SFD_OK;
  if (s->batch_refs > 0) return fail(SFD_EBUSY, "string belongs to a live batch");
  sfd_ctx* c = s->ctx;
  if (set_device(c) == SFD_OK) cudaStreamSynchronize(c->stream);
  c->pool.dealloc(s->block);
  delete s;
  return SFD_OK;
}

sfd_status sfd_string_save(const sfd_string* s, void* buf, size_t* bytes) {
  if (!s || !bytes) return fail(SFD_EINVAL, "NULL argument");
  const size_t state_off = ckpt_state_offset(s);
  const size_t state_bytes = block_bytes(s->h) - state_off;
  const size_t fixed = sizeof(CkptHeader) + sizeof(CkptRecord) + sizeof(Desc);
  const size_t total = fixed + state_bytes;
  if (!buf) {
    *bytes = total;
    return SFD_OK;
  }
  if (*bytes < total) {
    const size_t have = *bytes;
    *bytes = total;
    return fail(SFD_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", have, total);
  }
  sfd_status rc = set_device(s->ctx);
  if (rc) return rc;
  if ((rc = flush_string(s))) return rc;
  char* out = static_cast<char*>(buf);
  SFD_CUDA(d2h(s->ctx, out + fixed, s->block + state_off, state_bytes));
  SFD_CUDA(cudaStreamSynchronize(s->ctx->stream));
  CkptHeader H{};
  std::memcpy(H.magic, kCkptMagic, sizeof(H.magic));
  H.version = kCkptVersion;
  H.header_bytes = sizeof(CkptHeader);
  H.total_bytes = total;
  H.params_bytes = sizeof(sfd_string_params);
  H.desc_bytes = sizeof(Desc);
  H.scalars_bytes = sizeof(Scalars);
  H.record_bytes = sizeof(CkptRecord);
  H.state_offset = state_off;
  H.state_bytes = state_bytes;
  H.n_t = s->n_t;
  H.n_l = s->n_l;
  H.started = s->started ? 1 : 0;
  CkptRecord R{};
  R.p = s->p;
  R.exc = s->rec_exc;
  R.env_n = s->rec_env_n;
  R.env_mask = s->rec_env_mask;
  R.mod = s->rec_mod;
  std::memcpy(R.exc_args, s->rec_exc_args, sizeof(R.exc_args));
  std::memcpy(R.env, s->rec_env, sizeof(R.env));
  std::memcpy(R.mod_args, s->rec_mod_args, sizeof(R.mod_args));
  const Desc P = portable_desc(s->h);
  std::memcpy(out, &H, sizeof(H));
  std::memcpy(out + sizeof(H), &R, sizeof(R));
  std::memcpy(out + sizeof(H) + sizeof(R), &P, sizeof(Desc));
  *bytes = total;
  return SFD_OK;
}

sfd_status sfd_string_load(sfd_ctx* c, const void* buf, size_t bytes, sfd_string** out) {
  if (!c || !buf || !out) return fail(SFD_EINVAL, "NULL argument");
  *out = nullptr;
  const size_t fixed = sizeof(CkptHeader) + sizeof(CkptRecord) + sizeof(Desc);
  if (bytes < fixed) return fail(SFD_EINVAL, "checkpoint truncated (%zu bytes)", bytes);
  const char* in = static_cast<const char*>(buf);
  CkptHeader H;
  std::memcpy(&H, in, sizeof(H));
  if (std::memcmp(H.magic, kCkptMagic, sizeof(H.magic)) != 0) return fail(SFD_EINVAL, "not a string checkpoint");
  if (H.version != kCkptVersion || H.header_bytes != sizeof(CkptHeader) || H.params_bytes != sizeof(sfd_string_params) ||
      H.desc_bytes != sizeof(Desc) || H.scalars_bytes != sizeof(Scalars) || H.record_bytes != sizeof(CkptRecord))
    return fail(SFD_EINVAL, "checkpoint written by another version of the library");
  if (H.total_bytes != bytes || H.state_bytes != bytes - fixed)
    return fail(SFD_EINVAL, "checkpoint size does not match its header");
  CkptRecord R;
  std::memcpy(&R, in + sizeof(H), sizeof(R));
  Desc saved;
  std::memcpy(&saved, in + sizeof(H) + sizeof(R), sizeof(Desc));
  Scalars sc;
  if (H.state_bytes < sizeof(Scalars)) return fail(SFD_EINVAL, "checkpoint state truncated");
  std::memcpy(&sc, in + fixed, sizeof(Scalars));
  if (sc.n < 1 || sc.next_out < sc.n - 1 || sc.next_out > sc.n + 1)
    return fail(SFD_EINVAL, "checkpoint time level %lld / next sample %lld inconsistent",
                static_cast<long long>(sc.n), static_cast<long long>(sc.next_out));
  if (R.env_n < 0 || R.env_n > 16) return fail(SFD_EINVAL, "checkpoint bow envelope has %d breakpoints", R.env_n);

  // replay the set-up calls (each validates its arguments)
  sfd_string* s = nullptr;
  sfd_status rc = sfd_string_create(c, &R.p, &s);
  if (rc) return rc;
  const double* a = R.exc_args;
  if (R.exc == kPluck) rc = sfd_excite_pluck(s, a[0], a[1]);
  else if (R.exc == kHammer) rc = sfd_excite_hammer(s, a[0], a[1], a[2], a[3], a[4]);
  else if (R.exc == kBow) rc = sfd_excite_bow(s, a[0], a[1], a[2], a[3], a[4], a[5]);
  else rc = fail(SFD_EINVAL, "checkpoint excitation kind %d", R.exc);
  if (rc == SFD_OK && R.env_n > 0)
    rc = sfd_bow_envelope(s, R.env_n, R.env[0], (R.env_mask & 1) ? R.env[1] : nullptr,
                          (R.env_mask & 2) ? R.env[2] : nullptr, (R.env_mask & 4) ? R.env[3] : nullptr);
  if (rc == SFD_OK && R.mod != SFD_MOD_NONE)
    rc = sfd_set_modulation(s, R.mod, R.mod_args[0], R.mod_args[1], R.mod_args[2], R.mod_args[3]);
  if (rc) {
    std::string why = sfd_last_error();
    sfd_string_destroy(s);
    return fail(SFD_EINVAL, "checkpoint set-up does not replay: %s", why.c_str());
  }
  const Desc rebuilt = portable_desc(s->h);
  if (s->n_t != H.n_t || s->n_l != H.n_l || std::memcmp(&rebuilt, &saved, sizeof(Desc)) != 0 ||
      ckpt_state_offset(s) != H.state_offset || block_bytes(s->h) - ckpt_state_offset(s) != H.state_bytes) {
    sfd_string_destroy(s);
    return fail(SFD_EINVAL,
                "checkpoint descriptor differs from the one its parameters give here (another build or host)");
  }
  // the descriptor as rebuilt (with this block's pointers) and the saved state
  if ((rc = set_device(c)) == SFD_OK) {
    cudaError_t e = h2d(c, s->d_desc, &s->h, sizeof(Desc));
    if (e == cudaSuccess) e = h2d(c, s->block + H.state_offset, in + fixed, H.state_bytes);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "checkpoint upload");
  }
  if (rc) {
    sfd_string_destroy(s);
    return rc;
  }
  s->dirty = false;
  s->started = H.started != 0;
  *out = s;
  return SFD_OK;
}

sfd_status sfd_batch_create(sfd_ctx* c, int32_t n, sfd_string* const* strings, sfd_batch** out) {
  if (!c || !out || (n > 0 && !strings) || n < 0) return fail(SFD_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!strings[i] || strings[i]->ctx != c) return fail(SFD_EINVAL, "string %d is NULL or from another ctx", i);
  {
    std::vector<sfd_string*> sorted(strings, strings + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(SFD_EINVAL, "a string appears twice in the batch");
  }
  sfd_batch* b = new (std::nothrow) sfd_batch();
  if (!b) return fail(SFD_ENOMEM, "host allocation failed");
  b->ctx = c;
  b->strings.assign(strings, strings + n);
  for (auto* s : b->strings) s->batch_refs++;
  *out = b;
  return SFD_OK;
}

static sfd_status batch_run(sfd_batch* b, const int64_t* n_samples, float* out_device, const int64_t* offsets,
                            int32_t* per_string_status, Plan* keep = nullptr) {
  sfd_ctx* c = b->ctx;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  if ((rc = flush_strings(c, b->strings.data(), b->strings.size()))) return rc;
  std::vector<Job> jobs;
  std::vector<const sfd_string*> owners;
  for (size_t i = 0; i < b->strings.size(); ++i) {
    if (n_samples[i] < 0) return fail(SFD_EINVAL, "n_samples[%zu] < 0", i);
    if (n_samples[i] == 0) continue;
    jobs.push_back(Job{b->strings[i]->d_desc, out_device + offsets[i], n_samples[i]});
    owners.push_back(b->strings[i]);
  }
  rc = launch_jobs(c, jobs, owners, b->wpc, b->groups, keep);
  for (auto* s : b->strings) s->started = true;
  if (rc) return rc;
  if (per_string_status) {
    for (size_t i = 0; i < b->strings.size(); ++i) {
      Scalars sc{};
      if ((rc = read_status(b->strings[i], &sc))) return rc;
      per_string_status[i] = status_code(sc);
    }
  }
  return SFD_OK;
}

sfd_status sfd_batch_synthesize(sfd_batch* b, const int64_t* n_samples, float* out_device,
                                const int64_t* out_offsets, int32_t* per_string_status) {
  if (!b || !n_samples || !out_offsets || !out_device) return fail(SFD_EINVAL, "NULL argument");
  return batch_run(b, n_samples, out_device, out_offsets, per_string_status);
}

// The current device's address of host memory [p, p + n floats) when it is
// pinned and mapped for this device, with both ends at the same offset;
// nullptr otherwise (pageable memory, device memory, an unknown pointer).
static float* device_view(float* p, int64_t n) {
  cudaPointerAttributes a{}, z{};
  const bool mapped = cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                      a.devicePointer && (n <= 1 ||
                      (cudaPointerGetAttributes(&z, p + (n - 1)) == cudaSuccess && z.type == cudaMemoryTypeHost &&
                       z.devicePointer == static_cast<void*>(static_cast<float*>(a.devicePointer) + (n - 1))));
  cudaGetLastError();   // a pointer the runtime does not know is not an error here
  return mapped ? static_cast<float*>(a.devicePointer) : nullptr;
}

sfd_status sfd_batch_synthesize_host(sfd_batch* b, const int64_t* n_samples, float* out_host,
                                     const int64_t* out_offsets, int32_t* per_string_status) {
  if (!b || !n_samples || !out_offsets || !out_host) return fail(SFD_EINVAL, "NULL argument");
  sfd_ctx* c = b->ctx;
  int64_t total = 0;
  for (size_t i = 0; i < b->strings.size(); ++i) total = std::max(total, out_offsets[i] + n_samples[i]);
  sfd_status rc = set_device(c);
  if (rc) return rc;
  auto statuses = [&]() -> sfd_status {
    if (!per_string_status) return SFD_OK;
    for (size_t i = 0; i < b->strings.size(); ++i) {
      Scalars sc{};
      if (sfd_status r = read_status(b->strings[i], &sc)) return r;
      per_string_status[i] = status_code(sc);
    }
    return SFD_OK;
  };
  // Pinned host memory that this device can address: the kernels write the
  // samples there themselves (each warp stores 32 consecutive samples at a
  // time, about 0.7 GB/s for the whole 4096-string batch), so no copy
  // follows the launch.  Both ends of the range must map to the device at
  // the same offset (one allocation, as a C array is).
  if (float* dv = device_view(out_host, total)) {
    rc = batch_run(b, n_samples, dv, out_offsets, nullptr);
    if (rc == SFD_OK) {   // device-to-host bytes, moved by the kernels' stores
      for (size_t i = 0; i < b->strings.size(); ++i) c->d2h_bytes += sizeof(float) * static_cast<uint64_t>(n_samples[i]);
    }
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (rc == SFD_OK && e != cudaSuccess) rc = cuda_fail(e, "sync");
    if (rc == SFD_OK) rc = statuses();
    return rc;
  }
  char* tmp = c->pool.alloc(sizeof(float) * std::max<int64_t>(total, 1));
  if (!tmp) return fail(SFD_ENOMEM, "device pool exhausted for the output buffer");
  float* dout = reinterpret_cast<float*>(tmp);
  Plan P;
  rc = batch_run(b, n_samples, dout, out_offsets, nullptr, &P);
  if (rc == SFD_OK) {
    rc = copy_out_by_class(c, P, dout, out_host);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    // the copy stream too: after a failed copy call the context stream was
    // not made to wait for the copies already queued there
    const cudaError_t e2 = cudaStreamSynchronize(c->copy);
    if (e == cudaSuccess) e = e2;
    if (rc == SFD_OK && e != cudaSuccess) rc = cuda_fail(e, "sync");
  }
  if (rc == SFD_OK) rc = statuses();
  c->pool.dealloc(tmp);
  return rc;
}

sfd_status sfd_batch_set_warps_per_cta(sfd_batch* b, int32_t warps_per_cta) {
  if (!b) return fail(SFD_EINVAL, "batch is NULL");
  if (warps_per_cta < 0 || warps_per_cta > 4) return fail(SFD_EINVAL, "warps per CTA must be 0 (automatic) or 1..4");
  b->wpc = warps_per_cta;
  return SFD_OK;
}

sfd_status sfd_batch_prepare(sfd_batch* b, const int64_t* n_samples, float* out_device, const int64_t* out_offsets) {
  if (!b || !n_samples || !out_device || !out_offsets) return fail(SFD_EINVAL, "NULL argument");
  sfd_ctx* c = b->ctx;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  if ((rc = flush_strings(c, b->strings.data(), b->strings.size()))) return rc;
  std::vector<Job> jobs;
  std::vector<const sfd_string*> owners;
  for (size_t i = 0; i < b->strings.size(); ++i) {
    if (n_samples[i] < 0) return fail(SFD_EINVAL, "n_samples[%zu] < 0", i);
    if (n_samples[i] == 0) continue;
    jobs.push_back(Job{b->strings[i]->d_desc, out_device + out_offsets[i], n_samples[i]});
    owners.push_back(b->strings[i]);
  }
  Plan* P = b->plan ? static_cast<Plan*>(b->plan) : new (std::nothrow) Plan();
  if (!P) return fail(SFD_ENOMEM, "host allocation failed");
  b->plan = P;
  if ((rc = make_plan(c, jobs, owners, b->wpc, *P, b->groups))) return rc;
  const size_t bytes = std::max<size_t>(sizeof(Job) * P->jobs.size(), sizeof(Job));
  if (bytes > b->d_jobs_bytes) {
    if (b->d_jobs) c->pool.dealloc(b->d_jobs);
    b->d_jobs = c->pool.alloc(bytes);
    b->d_jobs_bytes = b->d_jobs ? bytes : 0;
    if (!b->d_jobs) return fail(SFD_ENOMEM, "device pool exhausted for the job table");
  }
  if (!P->jobs.empty()) SFD_CUDA(h2d(c, b->d_jobs, P->jobs.data(), sizeof(Job) * P->jobs.size()));
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  return SFD_OK;
}

sfd_status sfd_batch_launch(sfd_batch* b) {
  if (!b) return fail(SFD_EINVAL, "batch is NULL");
  if (!b->plan) return fail(SFD_ESTATE, "sfd_batch_prepare must come first");
  sfd_ctx* c = b->ctx;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SFD_CUDA(cudaStreamIsCapturing(c->stream, &cap));
  // a string excited or modulated since sfd_batch_prepare is uploaded now;
  // a graph cannot hold that copy (the staging buffer is reused)
  bool dirty = false;
  for (auto* s : b->strings) dirty = dirty || s->dirty;
  if (dirty && cap != cudaStreamCaptureStatusNone)
    return fail(SFD_ESTATE, "a string changed after sfd_batch_prepare: prepare again before capturing");
  if (dirty && (rc = flush_strings(c, b->strings.data(), b->strings.size()))) return rc;
  for (auto* s : b->strings) s->started = true;
  // per-class timing events cannot be read back from a graph: off while capturing
  const bool timing = c->timing;
  if (cap != cudaStreamCaptureStatusNone) c->timing = false;
  rc = issue_plan(c, *static_cast<Plan*>(b->plan), reinterpret_cast<const Job*>(b->d_jobs));
  c->timing = timing;
  return rc;
}

// A string with the same parameters, excitation and current state (device
// copy of the state block); used to probe launch settings without touching
// the original.
static sfd_status clone_string(const sfd_string* s, sfd_string** out) {
  sfd_ctx* c = s->ctx;
  sfd_string* t = new (std::nothrow) sfd_string(*s);
  if (!t) return fail(SFD_ENOMEM, "host allocation failed");
  t->batch_refs = 0;
  t->block = c->pool.alloc(block_bytes(t->h));
  if (!t->block) {
    delete t;
    return fail(SFD_ENOMEM, "device pool exhausted");
  }
  carve(t);
  SFD_CUDA(h2d(c, t->d_desc, &t->h, sizeof(Desc)));
  const size_t nz = t->h.n_z > 0 ? t->h.n_z : 1;
  struct { void* d; const void* s; size_t n; } cp[] = {
      {t->d_sc, s->d_sc, sizeof(Scalars)},      {t->h.u, s->h.u, sizeof(float) * t->h.n_u},
      {t->h.du, s->h.du, sizeof(float) * t->h.n_u}, {t->h.z, s->h.z, sizeof(float) * nz},
      {t->h.dz, s->h.dz, sizeof(float) * nz},    {t->h.xz, s->h.xz, sizeof(float) * nz},
      {t->h.az, s->h.az, sizeof(float) * nz}};
  for (auto& x : cp) SFD_CUDA(cudaMemcpyAsync(x.d, x.s, x.n, cudaMemcpyDeviceToDevice, c->stream));
  *out = t;
  return SFD_OK;
}

sfd_status sfd_batch_autotune(sfd_batch* b, int64_t probe_samples, int32_t* best_warps_per_cta) {
  if (!b || probe_samples <= 0) return fail(SFD_EINVAL, "bad autotune arguments");
  sfd_ctx* c = b->ctx;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  const size_t n = b->strings.size();
  if (n == 0) return fail(SFD_EINVAL, "empty batch");
  if ((rc = flush_strings(c, b->strings.data(), n))) return rc;   // the clones copy the device blocks
  char* dout = c->pool.alloc(sizeof(float) * probe_samples * n);
  if (!dout) return fail(SFD_ENOMEM, "device pool exhausted for the probe output");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 0.f;
  int best = 0, best_groups = 0;
  const int candidates[3] = {1, 2, 4};
  // warp groups are a candidate only if they would form for this batch
  bool groups_form = false;
  {
    std::vector<Job> jobs(n);
    std::vector<const sfd_string*> owners(b->strings.begin(), b->strings.end());
    Plan P;
    if (make_plan(c, jobs, owners, 0, P, 1) == SFD_OK)
      for (int k = 0; k < kClasses; ++k) groups_form = groups_form || P.group[k] > 1;
  }
  for (int cj = 0; cj < 6 && rc == SFD_OK; ++cj) {
    const int ci = cj % 3, groups = cj / 3;   // warps per CTA x warp groups off / on
    if (groups && !groups_form) continue;
    // fresh clones of the current state for every candidate
    std::vector<sfd_string*> cl;
    for (size_t i = 0; i < n && rc == SFD_OK; ++i) {
      sfd_string* t = nullptr;
      rc = clone_string(b->strings[i], &t);
      if (t) cl.push_back(t);
    }
    if (rc == SFD_OK) {
      std::vector<Job> jobs;
      std::vector<const sfd_string*> owners;
      for (size_t i = 0; i < n; ++i) {
        jobs.push_back(Job{cl[i]->d_desc, reinterpret_cast<float*>(dout) + i * probe_samples, probe_samples});
        owners.push_back(cl[i]);
      }
      const bool timing = c->timing;
      c->timing = false;
      cudaEventRecord(e0, c->stream);
      rc = launch_jobs(c, jobs, owners, candidates[ci], groups);
      cudaEventRecord(e1, c->stream);
      c->timing = timing;
      if (rc == SFD_OK) {
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
        else if (best == 0 || ms < best_ms) { best_ms = ms; best = candidates[ci]; best_groups = groups; }
      }
    }
    cudaStreamSynchronize(c->stream);
    for (auto* t : cl) { c->pool.dealloc(t->block); delete t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->pool.dealloc(dout);
  if (rc) return rc;
  b->wpc = best;
  b->groups = best_groups;
  if (best_warps_per_cta) *best_warps_per_cta = best;
  return SFD_OK;
}

sfd_status sfd_batch_destroy(sfd_batch* b) {
  if (!b) return SFD_OK;
  for (auto* s : b->strings) s->batch_refs--;
  if (b->d_jobs) b->ctx->pool.dealloc(b->d_jobs);
  delete static_cast<Plan*>(b->plan);
  delete b;
  return SFD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Synthesis without device allocation.
//
// Callers that must not allocate device memory -- a real-time audio callback
// (cudaMalloc can synchronise the device and block for an unbounded time), or
// a host that fixes a library's device footprint up front -- use this one
// entry point instead of a context.  Everything the step kernel needs beyond
// the caller's output buffer (the string's descriptor and state, the job
// entry and the work-queue counter) lives in one file-scope device array of
// SFD_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library keeps
// until exit.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = SFD_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};      // device address of the array, per device
size_t g_noalloc_smem[kMaxDevices] = {};    // opt-in shared memory per block, per device

// Puts back the caller's current device on every return path.
struct DeviceRestore {
  int dev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  }
  ~DeviceRestore() {
    if (dev >= 0) cudaSetDevice(dev);
  }
};

}  // namespace

extern "C" sfd_status sfd_synthesize_noalloc(int device, void* cuda_stream, const sfd_string_params* params,
                                             const sfd_excitation* exc, int64_t n_samples, float* out_device) {
  if (!params || !exc) return fail(SFD_EINVAL, "params and excitation are required");
  if (n_samples < 0) return fail(SFD_EINVAL, "n_samples < 0");
  if (n_samples > 0 && !out_device) return fail(SFD_EINVAL, "out_device is NULL");
  if (device < 0 || device >= kMaxDevices) return fail(SFD_EINVAL, "device %d out of range", device);

  // the string, as sfd_string_create + sfd_excite_* would set it up (host
  // arithmetic only: invalid parameters are refused whatever n_samples is)
  sfd_string s;
  sfd_status rc = init_host_string(*params, &s);
  if (rc) return rc;
  if ((rc = apply_excitation(&s, *exc))) return rc;
  const int n_t = s.n_t, n_l = s.n_l;
  const Desc& D = s.h;
  // layout inside the array: Desc | Scalars | u du z dz xz az | Job | counters
  const size_t nz = D.n_z > 0 ? D.n_z : 1;
  size_t off = 0;
  auto place = [&](size_t n) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    const size_t at = off;
    off += n;
    return at;
  };
  const size_t o_desc = place(sizeof(Desc)), o_sc = place(sizeof(Scalars));
  const size_t o_u = place(sizeof(float) * D.n_u), o_du = place(sizeof(float) * D.n_u);
  const size_t o_z = place(sizeof(float) * nz), o_dz = place(sizeof(float) * nz);
  const size_t o_xz = place(sizeof(float) * nz), o_az = place(sizeof(float) * nz);
  const size_t o_job = place(sizeof(Job)), o_cnt = place(sizeof(int) * kClasses);
  if (off > kNoAllocBytes)
    return fail(SFD_EINVAL,
                "string needs %zu bytes of scratch (N_t=%d, N_l=%d); the no-allocation entry point holds %zu",
                off, n_t, n_l, kNoAllocBytes);

  DeviceRestore restore;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  // The call copies from host memory it frees on return and waits for its
  // stream, neither of which a captured graph can hold.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SFD_EINVAL, "the stream is capturing: the no-allocation entry point cannot be captured");
  void* base = nullptr;
  size_t smem_optin = 0;
  {
    // once per device, with that device current: the array's device address
    // (a host-side reference to it is only a stand-in, not usable by kernels)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
      int optin = 0;
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
      if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
      g_noalloc_ptr[device] = p;
      g_noalloc_smem[device] = static_cast<size_t>(optin) - kStaticSmemBytes;
    }
    base = g_noalloc_ptr[device];
    smem_optin = g_noalloc_smem[device];
  }
  const size_t wbytes = static_cast<size_t>(warp_smem_floats(D.m_u, D.m_z, D.z_jacobi)) * sizeof(float);
  if (wbytes > smem_optin) return fail(SFD_EINVAL, "grid (N_t=%d, N_l=%d) exceeds one warp's shared memory", n_t, n_l);
  if (n_samples == 0) return SFD_OK;

  char* b = static_cast<char*>(base);
  s.h.u = reinterpret_cast<float*>(b + o_u);
  s.h.du = reinterpret_cast<float*>(b + o_du);
  s.h.z = reinterpret_cast<float*>(b + o_z);
  s.h.dz = reinterpret_cast<float*>(b + o_dz);
  s.h.xz = reinterpret_cast<float*>(b + o_xz);
  s.h.az = reinterpret_cast<float*>(b + o_az);
  s.h.sc = reinterpret_cast<Scalars*>(b + o_sc);

  // initial levels w^0, w^1 (the array keeps the previous call's contents,
  // so every field the kernel reads is written here)
  std::vector<float> u(D.n_u, 0.f), zero(std::max<size_t>(nz, static_cast<size_t>(D.n_u)), 0.f);
  Scalars sc{};
  sc.n = 1;
  sc.next_out = 0;
  if (s.exc == kPluck && s.pluck_amp != 0.0) {
    const double c0 = s.pluck_amp / s.p.length_m, xp = s.pluck_pos;
    for (int l = 1; l < n_t; ++l) {
      const double x = static_cast<double>(l) / n_t;
      u[l - 1] = static_cast<float>(x <= xp ? c0 * x / xp : c0 * (1.0 - x) / (1.0 - xp));
    }
  }
  if (s.exc == kHammer) {
    sc.uh = static_cast<float>(s.hammer_uh1);
    sc.duh = static_cast<float>(s.hammer_uh1);
  }
  const Job job{reinterpret_cast<const Desc*>(b + o_desc), out_device, n_samples};
  struct Copy { size_t at; const void* src; size_t n; };
  const Copy copies[] = {{o_desc, &s.h, sizeof(Desc)}, {o_sc, &sc, sizeof(Scalars)},
                         {o_u, u.data(), sizeof(float) * D.n_u}, {o_du, zero.data(), sizeof(float) * D.n_u},
                         {o_z, zero.data(), sizeof(float) * nz}, {o_dz, zero.data(), sizeof(float) * nz},
                         {o_xz, zero.data(), sizeof(float) * nz}, {o_az, zero.data(), sizeof(float) * nz},
                         {o_job, &job, sizeof(Job)}};
  for (const Copy& cp : copies) {
    e = cudaMemcpyAsync(b + cp.at, cp.src, cp.n, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy into the no-allocation scratch");
  }
  const int k = job_class(D);
  int* counter = reinterpret_cast<int*>(b + o_cnt) + k;   // the launcher clears it on `stream`
  e = kLaunch[k](reinterpret_cast<const Job*>(b + o_job), 1, counter,
                 warp_smem_floats(D.m_u, D.m_z, D.z_jacobi), 1, 1, 1, stream);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  e = cudaMemcpyAsync(&sc, b + o_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  rc = status_code(sc);
  if (rc == SFD_EUNSTABLE) return fail(rc, "string state became non-finite");
  if (rc == SFD_ENOCONV) return fail(rc, "coupled solve reached its sweep cap (result kept)");
  return SFD_OK;
}

#include "sfd_server.cuh"
#include "sfd_tape.cuh"
