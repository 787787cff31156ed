/*
 * sfd.h - C-ABI of the GB300 (sm_103a) nonlinear planar stiff-string
 * synthesizer: batched FP32 time-stepping of the finite-difference scheme of
 * "String Sound Synthesizer on GPU-Accelerated Finite Difference Scheme"
 * (Lee, Choi, Lee, arXiv 2311.18505).
 *
 * What one step computes (Sec. 3.2, Eq. 4; matrix form Sec. 3.4, Eqs. 7-9):
 *   transverse u (N_t intervals) and longitudinal zeta (N_l intervals) are
 *   advanced from (w^{n-1}, w^n) to w^{n+1} by the linearly-implicit scheme
 *     Theta delta_tt u = g^2 d_xx u - kappa^2 d_xxxx u
 *                      + g^2 (alpha^2-1)/2 d_x+ (q^2 mu_t. q + 2 q mu_tt p)
 *                      - 2 sigma0 delta_t. u + 2 sigma1 delta_t. d_xx u + F J
 *     delta_tt z = g^2 alpha^2 d_xx z + g^2 (alpha^2-1)/2 d_x+ I_(t->l)(q mu_t. q)
 *                      - 2 sigma0 delta_t. z + 2 sigma1 delta_t. d_xx z
 *   with a pluck initial condition, a hammer (Sec. 3.3.2, Eq. 6) or a bow
 *   (Sec. 3.3.1, Eq. 5) force F at one point, and one output sample per step
 *   read at the pickup.  Grids follow the spacing rules of Sec. 3.2.
 *
 * Units.  Parameters are SI at this boundary.  Internally x is normalised
 * to [0,1] and displacements by the length L (Table 1: gamma =
 * L^-1 sqrt(T0 / rho A), so f0 = gamma / 2, Sec. 4.1).  Output samples are
 * transverse displacement at the pickup in metres, FP32.
 *
 * Ownership.  The library owns every ctx, string and batch object and all
 * device memory behind them (carved from the context's device-memory pool).
 * The caller owns its output buffers (host memory, or device memory on the
 * context's device, e.g. a torch tensor's data pointer).
 *
 * Errors.  Every call returns an sfd_status; nothing aborts.  On error the
 * thread-local message of sfd_last_error() says why.  A string whose state
 * became non-finite reports SFD_EUNSTABLE from then on.
 *
 * Threading.  Objects are not thread-safe; distinct contexts may be used
 * from distinct threads.  Calls on one context are ordered on its stream.
 */
#ifndef SFD_H
#define SFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sfd_status;
enum {
  SFD_OK = 0,
  SFD_EINVAL = -1,     /* invalid argument or parameter                     */
  SFD_ENOMEM = -2,     /* device-memory pool exhausted                      */
  SFD_EUNSTABLE = -3,  /* state became non-finite                           */
  SFD_ENOCONV = -4,    /* coupled solve hit its sweep cap (result kept)     */
  SFD_ECUDA = -5,      /* CUDA runtime error                                */
  SFD_ETIMEOUT = -6,   /* bounded wait expired                              */
  SFD_EBUSY = -7,      /* object in use (e.g. string inside a live batch)   */
  SFD_ESTATE = -8      /* call not valid in the current state               */
};

enum { SFD_BOUNDARY_CLAMPED = 0, SFD_BOUNDARY_SIMPLY_SUPPORTED = 1 };
enum { SFD_GRID_THETA_BOUND = 0, SFD_GRID_PRINTED = 1 };
enum { SFD_MOD_NONE = 0, SFD_MOD_VIBRATO = 1, SFD_MOD_GLISS = 2 };
/* What the output samples read at the pickup (Sec. 4.2, Fig. 2 shows the
 * spectra of both): the transverse displacement L u(x_o) or the
 * longitudinal displacement L zeta(x_o), each linearly interpolated on its
 * own grid.  Strings with alpha = 1 have zeta = 0. */
enum { SFD_OUTPUT_TRANSVERSE = 0, SFD_OUTPUT_LONGITUDINAL = 1 };

typedef struct sfd_ctx sfd_ctx;
typedef struct sfd_string sfd_string;
typedef struct sfd_batch sfd_batch;

/* String parameters (Table 1).  Zero-initialise and set what you need;
 * sfd_params_default() fills the defaults listed below. */
typedef struct {
  double f0;              /* Hz; gamma = 2 f0 (Sec. 4.1).  Ignored if gamma > 0 */
  double gamma;           /* wave speed [1/s]                                    */
  double kappa;           /* stiffness [1/s] (Table 1, Eq. 4)                    */
  double alpha;           /* stiffness-to-tension ratio, >= 1 (Table 1)          */
  double sigma0;          /* frequency-independent loss [1/s] (Eq. 4)            */
  double sigma1;          /* frequency-dependent loss (Eq. 4)                     */
  double length_m;        /* L [m], default 1                                     */
  double fs;              /* sample rate [Hz], default 48000; k = 1/fs (Sec. 3)   */
  double linear_density;  /* rho A [kg/m], default 5e-3; maps N and kg to the
                             normalised equations                                 */
  double theta;           /* theta-scheme parameter, default (1+4/pi^2)/2 (Sec. 3.2) */
  int32_t boundary;       /* SFD_BOUNDARY_*, default clamped (Sec. 4.1)           */
  int32_t grid_rule;      /* SFD_GRID_*: 0 (default) sizes N_t by the stability
                             bound of the theta actually used; 1 uses the printed
                             h_t of Sec. 3.2, which is that bound for theta = 1   */
  double pickup_pos;      /* output point, fraction of L, default 0.7             */
  double f0_max_ratio;    /* >= 1: grids sized for gamma * ratio (modulation peak) */
  int32_t output;         /* SFD_OUTPUT_*, default transverse; anything else:
                             SFD_EINVAL                                            */
  int32_t pad_;
} sfd_string_params;

/* Fill p with the defaults (f0 = 110, kappa = 1, alpha = 1, sigma0 = 0.5,
 * sigma1 = 1e-5, L = 1 m, fs = 48 kHz, rho A = 5e-3, theta = (1+4/pi^2)/2,
 * clamped, theta-bound grid, pickup 0.7, ratio 1, transverse output). */
void sfd_params_default(sfd_string_params* p);

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * (NULL: the legacy default stream).  mem_budget_bytes sizes the device pool
 * that holds every string's state (0: 256 MiB).  *out receives the ctx. */
sfd_status sfd_ctx_create(int device, void* cuda_stream, size_t mem_budget_bytes, sfd_ctx** out);
void sfd_ctx_destroy(sfd_ctx* ctx);

/* Pool accounting: bytes in use and total. */
sfd_status sfd_ctx_memory(const sfd_ctx* ctx, size_t* used, size_t* total);

/* Create a string from parameters: derives N_t from the transverse stability
 * bound and N_l = floor(1 / (gamma alpha k)) (Sec. 3.2), allocates its state
 * and sets it at rest at time level n = 1.  SFD_EINVAL on bad parameters,
 * SFD_ENOMEM when the pool is full. */
sfd_status sfd_string_create(sfd_ctx* ctx, const sfd_string_params* p, sfd_string** out);

/* Grid of a string: intervals N_t, N_l and spacings h_t = 1/N_t, h_l = 1/N_l. */
sfd_status sfd_string_info(const sfd_string* s, int32_t* n_t, int32_t* n_l, double* h_t, double* h_l);

/* The grid sfd_string_create would give parameters p, without a context or a
 * device (host arithmetic only): N_t from the stability bound of the theta
 * scheme at the peak wave speed gamma * f0_max_ratio (Sec. 3.2, reading of
 * the spacing rule), N_l = floor(1 / (gamma alpha k)) (h_l = gamma alpha k).
 * Errors as sfd_string_create's parameter checks. */
sfd_status sfd_grid(const sfd_string_params* p, int32_t* n_t, int32_t* n_l);

/* Grid-sizing ratio of an f0 modulation: the largest gamma^n / gamma it
 * reaches (vibrato 2^{|c| / 1200}, glissando 2^{max(D, 0)}, none 1), the
 * f0_max_ratio at which a grid holds the whole note (Sec. 1's varying f0
 * on the fixed grid of Sec. 3.2).  SFD_EINVAL for an unknown kind or a
 * non-finite depth. */
sfd_status sfd_modulation_peak(int32_t kind, double depth, double* ratio);

/* Pluck (Sec. 3.3): initial condition u^0 = u^1 = triangle of peak amp/L at
 * pos (fraction of L), zero initial velocity.  Valid only before the first
 * synthesize call (else SFD_ESTATE). */
sfd_status sfd_excite_pluck(sfd_string* s, double amp_m, double pos);

/* Hammer (Sec. 3.3.2, Eq. 6): lumped mass m_H hitting at pos with velocity
 * vel from the string's rest position; contact force
 *   F_H = omega_H^{1+alpha_H} [eta]_+^{alpha_H-1} mu_t. eta,  eta = u_H - I u,
 * mass ratio M = m_H / (rho A L).  Before the first synthesize call only. */
sfd_status sfd_excite_hammer(sfd_string* s, double mass_kg, double vel_mps, double pos,
                             double omega_h, double alpha_h);

/* Bow (Sec. 3.3.1, Eq. 5): force F_B [N] and speed v_B [m/s] at pos with
 * friction phi(v) = sign(v)(eps + (1-eps) e^{-a |v|}), a in s/m; the force
 * drops to zero from release_time_s on (< 0: never).  Sticking (|v_rel| = 0)
 * is taken whenever it is consistent.  Before the first synthesize call. */
sfd_status sfd_excite_bow(sfd_string* s, double vel_mps, double force_n, double pos,
                          double a_s_per_m, double eps, double release_time_s);

/* Time-varying bow controls (Sec. 3.3.1 makes the bow velocity, force and
 * position control parameters that vary in time): after sfd_excite_bow and
 * before the first synthesis, n_points (1..16) breakpoints at times t_s[j]
 * (seconds from the start, increasing) with vel_mps[j] [m/s], force_n[j]
 * [N] and pos[j] (fraction of L, in (0, 1)); a NULL array keeps that
 * control at its sfd_excite_bow value.  The step n -> n+1 takes the values
 * at t = n / fs: linear between breakpoints, the first or last value
 * outside them; the interpolation I and spreading J of the bow follow pos.
 * The release time of sfd_excite_bow still sets the force to zero.  Errors:
 * SFD_EINVAL (not bowed, bad values), SFD_ESTATE (already started). */
sfd_status sfd_bow_envelope(sfd_string* s, int32_t n_points, const double* t_s, const double* vel_mps,
                            const double* force_n, const double* pos);

/* f0 modulation (Sec. 1): kind SFD_MOD_VIBRATO, gamma^n = gamma 2^{(c/1200)
 * sin(2 pi rate t + phase)} with depth c in cents; SFD_MOD_GLISS, gamma^n =
 * gamma 2^{D min(t, duration) / duration} with depth D in octaves (a glide
 * that holds at 2^D once t reaches the duration).  t = n k for the step from
 * level n.  SFD_MOD_NONE removes a modulation.  The grid must be stable
 * at the modulation's peak wave speed (sfd_modulation_peak): when the string
 * was created with a smaller f0_max_ratio, its grid is derived again for the
 * peak (a faster wave needs a coarser grid, so N_t and N_l shrink; the
 * excitation keeps its parameters and position; a new pool block holds the
 * state), SFD_ENOMEM if the pool has no room, SFD_EBUSY for a string already
 * in a batch.  Before the first synthesize call only (else SFD_ESTATE). */
sfd_status sfd_set_modulation(sfd_string* s, int32_t kind, double rate_hz, double depth,
                              double phase_rad, double duration_s);

/* Produce the next n_samples output samples y^j = L I(x_o) u^j (j counts
 * from 0, so the first two samples are the initial levels).  out is host
 * memory (out_on_device = 0) or device memory on the context's device.
 * Calls are resumable: synthesize(a) then synthesize(b) equals
 * synthesize(a + b).  Blocks until the samples are in `out`. */
sfd_status sfd_synthesize(sfd_string* s, int64_t n_samples, float* out, int32_t out_on_device);

/* Time level n and next output index of a string. */
sfd_status sfd_string_position(const sfd_string* s, int64_t* time_level, int64_t* next_sample);

/* Copy the state to host FP32 arrays: u^{n-1}, u^n (N_t - 1 each),
 * z^{n-1}, z^n (N_l - 1 each, may be NULL) in normalised units. */
sfd_status sfd_string_state(const sfd_string* s, float* u_prev, float* u, float* z_prev, float* z);

/* The state as the step kernel keeps it (Sec. 3.4's w^{n-1}, w^n in the
 * increment form): u^n, D = u^n - u^{n-1} (N_t - 1 each), z^n and
 * Dz = z^n - z^{n-1} (N_l - 1 each; zero without a longitudinal grid), FP32
 * in normalised units, so that w^{n-1} = w^n - D is exact in FP64.  Any
 * pointer may be NULL. */
sfd_status sfd_string_delta_state(const sfd_string* s, float* u, float* du, float* z, float* dz);

/* Hammer position u_H / L at time levels n-1 and n (Sec. 3.3.2, Eq. 6;
 * FP32 as kept, widened).  SFD_EINVAL for a string not struck. */
sfd_status sfd_string_hammer(const sfd_string* s, double* u_h_prev, double* u_h);

/* Solver statistics of a string since creation: status (SFD_OK,
 * SFD_EUNSTABLE, SFD_ENOCONV), the largest and the total number of
 * Gauss-Seidel sweeps of the coupled transverse/longitudinal solve. */
sfd_status sfd_string_stats(const sfd_string* s, int32_t* status, int32_t* max_sweeps, int64_t* total_sweeps);

sfd_status sfd_string_destroy(sfd_string* s);

/* Checkpoint of a string: its full state (Sec. 3.4's two time levels w^{n-1},
 * w^n as u, D, z, Dz; the hammer u_H^{n-1}, u_H^n of Eq. 6; the bow's slip
 * speed kept as the friction root's warm start; the coupled solve's warm
 * starts; the time level n, which also fixes the modulation phase and the
 * bow envelope's position; status and solver statistics) together with its
 * parameters and the excitation, bow envelope and modulation calls as last
 * made, so that a note can be moved to another context, device or process
 * and continue there.  Host memory, owned by the caller.  With buf NULL,
 * *bytes receives the size needed; otherwise *bytes is buf's capacity on
 * entry (SFD_EINVAL and the size needed in *bytes when it is too small) and
 * the size written on return.  Pending work on the string's stream is
 * waited for.  The format is this library's own, for the same library
 * version and host byte order. */
sfd_status sfd_string_save(const sfd_string* s, void* buf, size_t* bytes);

/* A new string in ctx from a checkpoint of sfd_string_save: sfd_string_load
 * then sfd_synthesize(n) gives exactly the samples that the saved string's
 * next sfd_synthesize(n) would have given (bit for bit, on any device of
 * this kind).  The saved set-up calls are made again through the public
 * entry points, which check them, and the descriptor they give must equal
 * the saved one byte for byte.  SFD_EINVAL for a buffer that is not a
 * checkpoint of this format, is truncated, carries an inconsistent time
 * level, or whose set-up does not give the saved descriptor (another build
 * or host); SFD_ENOMEM when the pool has no room.  The checkpoint buffer is
 * only read. */
sfd_status sfd_string_load(sfd_ctx* ctx, const void* buf, size_t bytes, sfd_string** out);

/* Batched form: n strings advanced together by one launch of the persistent
 * step kernel.  Strings stay owned by the caller's handles; a string in a
 * live batch cannot be destroyed (SFD_EBUSY). */
sfd_status sfd_batch_create(sfd_ctx* ctx, int32_t n, sfd_string* const* strings, sfd_batch** out);

/* Advance string i by n_samples[i] samples into out_device + out_offsets[i]
 * (device memory, FP32).  One launch of the persistent step kernel on the
 * ctx's stream; the call returns once it is queued, unless
 * per_string_status (host, may be NULL) is given, in which case it waits
 * and writes each string's status (SFD_OK, SFD_EUNSTABLE, SFD_ENOCONV). */
sfd_status sfd_batch_synthesize(sfd_batch* b, const int64_t* n_samples, float* out_device,
                                const int64_t* out_offsets, int32_t* per_string_status);

/* Same, with host output, and returns once out_host holds every string's
 * samples (out_host + out_offsets[i], n_samples[i] floats each; elements
 * between the strings' ranges are not written).  Pinned host memory that
 * the ctx's device can address (cudaHostAlloc, cudaHostRegister, a pinned
 * torch tensor) is written by the kernels directly, with no copy after
 * them.  Other host memory receives device-side output copied class by
 * class: the kernel classes run concurrently, and each class's strings are
 * copied as soon as its kernel ends, while the other classes still run. */
sfd_status sfd_batch_synthesize_host(sfd_batch* b, const int64_t* n_samples, float* out_host,
                                     const int64_t* out_offsets, int32_t* per_string_status);

/* Number of kernel launches issued by the last batch/synthesize call. */
int32_t sfd_last_launch_count(const sfd_ctx* ctx);

/* Number of step-kernel classes: strings are grouped by transverse rows per
 * lane (1, 3, 5, 7, 9 held in registers; more in shared memory) and each
 * group runs as its own persistent kernel, concurrently with the others. */
#define SFD_KERNEL_CLASSES 6

/* Per-class kernel timing: when enabled, every launch records CUDA events
 * around each class kernel on the stream it runs on; sfd_ctx_kernel_times
 * waits for them and reports, for the last batch/synthesize call, each
 * class's kernel time [ms] and job count (ms[SFD_KERNEL_CLASSES],
 * n_jobs[SFD_KERNEL_CLASSES]; zeros for classes not launched). */
sfd_status sfd_ctx_set_timing(sfd_ctx* ctx, int32_t enable);
sfd_status sfd_ctx_kernel_times(sfd_ctx* ctx, float* ms, int32_t* n_jobs);

/* Warp groups (default on).  The time steps of one string are strictly
 * sequential (the recursion of Eq. 4), so a launch with fewer strings than
 * the GPU has warp schedulers leaves schedulers idle and its time is that of
 * its slowest string.  With groups enabled, strings whose longitudinal grid
 * is large (the longitudinal coupling folded into the Gauss-Seidel sweeps;
 * 3 or more longitudinal rows per lane for 2 warps, 7 or more for 4) are
 * each stepped by 2 or 4 warps of one SM, which split the longitudinal
 * rows, as long as the launch then still has at most one warp per
 * scheduler.  The samples are bit for bit the same with and without groups.
 * enable = 0 steps every string with one warp. */
sfd_status sfd_ctx_set_warp_pairs(sfd_ctx* ctx, int32_t enable);

/* Sweep cap of the coupled transverse/longitudinal Gauss-Seidel solve for
 * every later launch on this context (the joint solve of Sec. 3.4 is
 * iterative; its tolerance is fixed, the cap bounds the work per step):
 * 1..64, or 0 for the default 24.  A step that reaches the cap keeps its
 * last iterate and marks the string SFD_ENOCONV; strings that need fewer
 * sweeps give the same samples whatever the cap. */
sfd_status sfd_ctx_set_sweep_cap(sfd_ctx* ctx, int32_t cap);

/* Kernel class (0 .. SFD_KERNEL_CLASSES-1) a string runs in. */
sfd_status sfd_string_kernel_class(const sfd_string* s, int32_t* cls);

/* Cumulative bytes the library moved host->device and device->host on this
 * context (state uploads, job tables, outputs, status reads; outputs the
 * kernels wrote straight into pinned host memory count as device->host). */
sfd_status sfd_ctx_transfer_bytes(const sfd_ctx* ctx, uint64_t* h2d_total, uint64_t* d2h_total);

/* Warps per CTA for this batch's launches: 1..4, or 0 (default) for
 * automatic (jobs / SMs, clamped).  Warps of one CTA run on different SM
 * sub-partitions, so this sets how many strings share an SM. */
sfd_status sfd_batch_set_warps_per_cta(sfd_batch* b, int32_t warps_per_cta);

/* Choose warps per CTA and warp groups by measurement: runs probe_samples
 * samples of every string for each candidate (1, 2, 4 warps per CTA, each
 * with warp groups off and on; see sfd_ctx_set_warp_pairs) on throwaway
 * copies of the strings' current state (the batch's strings are not
 * advanced), keeps the fastest for the batch and returns its warps per CTA
 * in *best (may be NULL).  The samples do not depend on either choice. */
sfd_status sfd_batch_autotune(sfd_batch* b, int64_t probe_samples, int32_t* best_warps_per_cta);

/* Split form of sfd_batch_synthesize for CUDA-graph capture.  prepare
 * uploads the batch's job table (string i advances n_samples[i] samples into
 * out_device + out_offsets[i]) and waits for it; launch then only enqueues
 * the kernels on the context stream (no host<->device copies, no
 * allocation), so it may be captured into a CUDA graph and replayed: every
 * launch or replay advances each string by its n_samples and overwrites the
 * same output ranges.  Per-class kernel timing is skipped while the
 * context stream is capturing.  The kernel classes run concurrently,
 * launched heaviest first; on an idle device they start in that order, but
 * enqueued behind a running batch they become ready together and the
 * device may start a light class first, which can lengthen the batch by up
 * to ~20 %: for the best schedule, launch (or replay) after the previous
 * batch has ended. */
sfd_status sfd_batch_prepare(sfd_batch* b, const int64_t* n_samples, float* out_device, const int64_t* out_offsets);
sfd_status sfd_batch_launch(sfd_batch* b);

sfd_status sfd_batch_destroy(sfd_batch* b);

/* Excitation of a string for sfd_synthesize_noalloc and sfd_server_submit
 * (same meaning and units as the sfd_excite_* calls).  kind: 0 pluck (amp_m, pos), 1 hammer
 * (mass_kg, vel_mps, pos, omega_h, alpha_h), 2 bow (vel_mps, force_n, pos,
 * a_s_per_m, eps, release_time_s). */
typedef struct {
  int32_t kind;
  int32_t pad_;
  double amp_m, pos;
  double mass_kg, vel_mps, omega_h, alpha_h;
  double force_n, a_s_per_m, eps, release_time_s;
} sfd_excitation;

/* Largest scratch a string may need in sfd_synthesize_noalloc (descriptor,
 * state, job entry and counters, 256-byte aligned). */
#define SFD_NOALLOC_SCRATCH_BYTES (32u * 1024u)

/* Synthesize the first n_samples output samples of one string, set up from
 * `params` and `exc` exactly as sfd_string_create + sfd_excite_* would, into
 * out_device (device memory on `device`), without allocating any device
 * memory.  For callers that cannot call cudaMalloc: real-time audio threads
 * (cudaMalloc can synchronise the device and block for an unbounded time)
 * and hosts that fix a library's device footprint in advance.  There is no
 * counterpart in the paper.
 *
 * The string's descriptor, state, job entry and work-queue counter live in
 * one static device array of SFD_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library keeps until the process exits; strings that need
 * more, or more shared memory than one warp may have, get SFD_EINVAL.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  Every call shares the
 * array and overwrites it, so calls that overlap on the GPU (from several
 * threads or streams) race: serialise them.  The call copies from host
 * memory and waits for its stream before returning (it reads the string's
 * status), so it cannot be captured into a CUDA graph: on a capturing
 * stream it returns SFD_EINVAL and enqueues nothing.  Parameters are
 * validated whatever n_samples is; n_samples = 0 then returns SFD_OK and
 * writes nothing.  The caller's current device is the same on return.
 * f0 modulation is not available here. */
sfd_status sfd_synthesize_noalloc(int device, void* cuda_stream, const sfd_string_params* params,
                                  const sfd_excitation* exc, int64_t n_samples, float* out_device);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of note requests.  There is no counterpart
 * in the paper (its synthesizer renders one batch offline); the notes are
 * the same strings, stepped by the same kernels.
 *
 * A server owns a context's stream.  Requests (a note: string parameters,
 * excitation, optional f0 modulation, length in samples) are queued by
 * sfd_server_submit on the host.  Each sfd_server_pump
 *   1. admits queued requests in arrival order while the server has a free
 *      slot and the context's device pool a block for the note's state
 *      (admission by device memory; a request that does not fit waits,
 *      later ones wait behind it);
 *   2. enqueues the next chunk (chunk_samples, fewer at a note's end) of
 *      every live note as one persistent launch per kernel class, and the
 *      copy of the chunk's audio to pinned host memory; the kernels are
 *      launched once the previous pump's chunk has ended, so that they
 *      start in launch order on an idle device;
 *   3. returns the audio of the chunk enqueued by the previous pump, one
 *      sfd_chunk per live note (so a pump's host work overlaps the GPU's
 *      work on a chunk);
 *   4. frees the slots and blocks of the notes that ended in that chunk.
 * A note's audio is bitwise the audio of the same string synthesized alone
 * (chunking and batching do not change a string's arithmetic).  Not
 * thread-safe; one server per context.
 * --------------------------------------------------------------------- */
typedef struct sfd_server sfd_server;

typedef struct {
  sfd_string_params params;
  sfd_excitation exc;
  int32_t mod_kind;         /* SFD_MOD_NONE / VIBRATO / GLISS (sfd_set_modulation) */
  int32_t pad_;
  double mod_rate_hz, mod_depth, mod_phase_rad, mod_duration_s;
  int64_t n_samples;        /* note length (> 0) */
  double arrival_s;         /* arrival on the server clock; < 0: the submit time */
  uint64_t tag;             /* caller's id, returned with every chunk */
} sfd_request;

typedef struct {
  uint64_t tag;
  int64_t first_sample;     /* index of the chunk's first sample within the note */
  int32_t n;                /* samples in this chunk */
  int32_t last;             /* 1 on the note's final chunk */
  sfd_status status;        /* on the final chunk: SFD_OK, SFD_EUNSTABLE or SFD_ENOCONV */
  int32_t pad_;
  const float* samples;     /* n samples (metres), pinned host memory owned by the
                               server, valid until the next sfd_server_pump */
  double ready_s;           /* server clock when the chunk's audio was on the host */
  double arrival_s;         /* the request's arrival */
} sfd_chunk;

typedef struct {
  int64_t queued, live, submitted, admitted, completed, chunks, samples;
  int64_t in_flight;        /* 1 while a chunk is enqueued and not yet returned */
  uint64_t pool_used, pool_size;
} sfd_server_stats;

/* chunk_samples > 0, max_live > 0 slots.  The server's output and job
 * buffers (2 x max_live x chunk_samples floats on the device, the same in
 * pinned host memory) are taken from the context's pool and the host;
 * SFD_ENOMEM if they do not fit. */
sfd_status sfd_server_create(sfd_ctx* ctx, int32_t chunk_samples, int32_t max_live, sfd_server** out);
/* Validates and queues a request (host only).  SFD_EINVAL for invalid
 * parameters, SFD_ENOMEM for a note whose state can never fit the pool. */
sfd_status sfd_server_submit(sfd_server* sv, const sfd_request* req);
/* The same for a bowed request whose velocity, force and position vary in
 * time (Sec. 3.3.1): the breakpoints as in sfd_bow_envelope, copied before
 * the call returns (the caller keeps ownership of the arrays).  SFD_EINVAL
 * also when the request is not bowed or n_points is outside 1..16. */
sfd_status sfd_server_submit_bow_envelope(sfd_server* sv, const sfd_request* req, int32_t n_points,
                                          const double* t_s, const double* vel_mps, const double* force_n,
                                          const double* pos);
/* One admission + launch + delivery round (see above).  *chunks points to
 * *n_chunks records owned by the server, valid until the next pump. */
sfd_status sfd_server_pump(sfd_server* sv, const sfd_chunk** chunks, int32_t* n_chunks);
/* Seconds since the server was created (steady clock). */
double sfd_server_clock(const sfd_server* sv);
sfd_status sfd_server_stats_get(const sfd_server* sv, sfd_server_stats* st);
/* Waits for any chunk in flight, frees every note and the buffers. */
sfd_status sfd_server_destroy(sfd_server* sv);

/* ---------------------------------------------------------------------
 * Gradients of a waveform loss with respect to string parameters, by the
 * discrete adjoint of the time-stepping (no counterpart in the paper).
 *
 * A tape holds n strings (params[i], exc[i]: pluck, hammer or bow, mod[i]:
 * f0 modulation, or mod = NULL for none) synthesized for n_samples each.  sfd_tape_forward writes the
 * audio y (device, y[i * n_samples + j], metres) and keeps every string's
 * state every checkpoint_every samples.  sfd_tape_backward takes dJ/dy
 * (device, same layout) and writes, per string, dJ/d(kappa, alpha, sigma0,
 * sigma1, amplitude) to grad[i * SFD_GRAD_PARAMS + k] (host): amplitude is
 * the pluck amp_m, the hammer vel_mps, or the bow velocity vel_mps.  The
 * gradient is that of the discrete scheme on the string's grid (N_t, N_l
 * held fixed), through the FP32 trajectory the forward computed: each
 * segment between checkpoints is swept backwards by the adjoint kernel over
 * its levels, which the forward recorded (when the whole trajectory, the
 * sum over strings of n_samples x (2 (N_t - 1) + 2 (N_l - 1) + 2) floats,
 * each count rounded up, fits in 4 GiB and the device has room; see
 * sfd_tape_set_record_forward) or which
 * are replayed from the segment's checkpoint (the same values bit for
 * bit).  For a bowed string each step keeps the
 * regime (sliding or sticking, Sec. 3.3.1) the forward took: the loss is
 * piecewise smooth in the parameters, and this is its derivative between
 * regime switches.
 * The tape's own device memory (checkpoints, one segment's replay record,
 * the whole-trajectory record when it is kept, adjoint state) is allocated
 * at create; the strings come from the ctx pool.
 * --------------------------------------------------------------------- */
typedef struct sfd_tape sfd_tape;
#define SFD_GRAD_PARAMS 5
/* f0 modulation of a string, as sfd_set_modulation takes it. */
typedef struct {
  int32_t kind;             /* SFD_MOD_NONE / VIBRATO / GLISS */
  int32_t pad_;
  double rate_hz, depth, phase_rad, duration_s;
} sfd_modulation;
sfd_status sfd_tape_create(sfd_ctx* ctx, int32_t n, const sfd_string_params* params, const sfd_excitation* exc,
                           const sfd_modulation* mod, int64_t n_samples, int32_t checkpoint_every,
                           sfd_tape** out);
/* Runs from the initial state every time; returns SFD_EUNSTABLE / SFD_ENOCONV
 * (audio written) if a string's synthesis reported one. */
sfd_status sfd_tape_forward(sfd_tape* t, float* y_device);
/* SFD_ESTATE before a forward. */
sfd_status sfd_tape_backward(sfd_tape* t, const float* dy_device, double* grad);
/* Record every level on the forward pass (enable = 1: the backward replays
 * nothing; SFD_ENOMEM when the device has no room for the record, whatever
 * its size) or replay each segment from its checkpoint (enable = 0: the
 * record's device memory is freed).  Enabling invalidates an earlier forward
 * pass (sfd_tape_backward then returns SFD_ESTATE until the next forward).
 * The gradients are the same bit for bit either way. */
sfd_status sfd_tape_set_record_forward(sfd_tape* t, int32_t enable);
sfd_status sfd_tape_destroy(sfd_tape* t);

/* Throughput peaks of device `device`, measured by three short
 * microbenchmarks timed with CUDA events (best of five launches after a
 * warm-up; no counterpart in the paper): FP32 and FP64 fused multiply-add
 * throughput [TFLOP/s, 2 flops per FMA] and conflict-free 16-byte
 * shared-memory load bandwidth [TB/s] over all SMs.  These are the
 * denominators of the step kernels' roofline: they are bound by FP32
 * arithmetic, shared-memory traffic and per-step latency, not by HBM.
 * Allocates and frees a small device buffer; the caller's current device
 * is the same on return.  SFD_EINVAL for NULL outputs, SFD_ECUDA on a CUDA
 * error. */
sfd_status sfd_measure_peaks(int device, double* fp32_tflops, double* fp64_tflops, double* smem_tbs);

/* Thread-local message describing the last error. */
const char* sfd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
