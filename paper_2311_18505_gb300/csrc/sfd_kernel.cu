// Persistent step kernel for the nonlinear planar stiff string
// (arXiv 2311.18505, Sec. 3.2 Eq. 4; excitations Sec. 3.3 Eqs. 5-6).
//
// One warp owns one string at a time and advances it for a whole job
// (thousands of steps) without leaving the SM.  Lane j owns the contiguous
// rows [j m, j m + m) of each grid (m odd, so a warp-wide shared-memory
// access to row j m + r is free of bank conflicts).  Up to 9 transverse rows
// per lane are held in registers (sfd_step_reg.cuh); larger grids keep every
// per-row array in the warp's shared-memory region (sfd_step_smem.cuh).
//
// The state is kept as (u^n, D = u^n - u^{n-1}) and each step solves for the
// acceleration a = u^{n+1} - 2u^n + u^{n-1} (run_job states the equations).
// g = u_l - u_{l-1} are interval differences, e the interval differences of
// the longitudinal field interpolated to the transverse nodes (P, linear),
// A the tridiagonal Theta + s0 - s1 d2 - d_+[ca g^2 d(.)] of the k^2-scaled
// transverse line of Eq. 4.  Solving for the small accelerations keeps FP32
// rounding proportional to the motion per step rather than the displacement.
//
// The coupled system is solved by block Gauss-Seidel: a transverse
// tridiagonal solve (partitioned Thomas per lane + parallel cyclic
// reduction over the 32 lane-boundary unknowns by shuffles) alternating with
// a longitudinal one (constant matrix, factored once per job) until the
// longitudinal acceleration stops changing.  When the longitudinal
// off-diagonal (sigma1 k / h_l^2) is tiny it is folded into the sweeps as a
// Jacobi update instead.  Hammer and bow forces are scalar eliminations
// through the unit-force response A^{-1} J solved alongside.
#include <cuda_runtime.h>

#include <mutex>

#include "sfd_step_smem.cuh"
#include "sfd_step_reg.cuh"

// One translation unit per transverse rows-per-lane class: compiled with
// -DSFD_MU=<1|3|5|7|9> for the register path, or without SFD_MU for the
// shared-memory path, so each kernel gets the registers its class needs.
#define SFD_CAT2(a, b) a##b
#define SFD_CAT(a, b) SFD_CAT2(a, b)
#ifdef SFD_MU
#define SFD_LAUNCHER SFD_CAT(launch_synth_reg, SFD_MU)
#define SFD_KERNEL SFD_CAT(synth_kernel_reg, SFD_MU)
#else
#define SFD_LAUNCHER launch_synth_smem
#define SFD_KERNEL synth_kernel_smem
#endif

namespace sfd {

// One resident block of up to 4 warps per SM lets each class use up to 255
// registers.  Capping them at 168 or 128 (3 or 4 resident blocks) makes ptxas
// spill 0.1-3 KB per thread and, measured on the 4096-string modulated
// batch, lowers throughput from 124 M to 92 M / 88 M samples/s despite the
// extra warps.
//
// With group = 2 or 4 (register path only) the CTA's warps work in groups
// (warps g*group .. g*group + group - 1 share region g): the group's first
// warp takes the next job from the queue and passes it on through shared
// memory (named barrier 1 + g over the whole group), and the warps the job
// can use step it (run_job_reg, in-job barrier 1 + g for pairs, 3 for
// groups of 4, whose unused warps meanwhile wait at barrier 1).  The job
// index cells alternate so that a cell is rewritten only after every warp
// of the group has passed the next barrier, i.e. after all have read it.
__global__ void __launch_bounds__(128, 1) SFD_KERNEL(const Job* __restrict__ jobs, int n_jobs,
                                                    int* __restrict__ counter, int warp_floats, int group) {
  extern __shared__ float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & (kWarp - 1);
#ifdef SFD_MU
  __shared__ float xcells[2][1024];  // per group: [buffer][warp][chg, mag, chx, mgx][lane]
  __shared__ int jcell[2][2];        // per group: job index, alternating
  const int npw = group == 4 ? 4 : (group == 2 ? 2 : 1);
#else
  const int npw = 1;
  (void)group;
#endif
  const int pi = warp / npw, pw = warp - pi * npw;
  float* wbase = smem + static_cast<size_t>(pi) * warp_floats;
#ifdef SFD_MU
  int it = 0;
#endif
  for (;;) {
    int j = 0;
    if (lane == 0 && pw == 0) j = atomicAdd(counter, 1);
    j = __shfl_sync(SFD_FULL, j, 0);
#ifdef SFD_MU
    if (npw > 1) {
      if (pw == 0 && lane == 0) jcell[pi][it & 1] = j;
      group_sync(1 + pi, npw);
      j = jcell[pi][it & 1];
      ++it;
    }
#endif
    if (j >= n_jobs) break;
#ifdef SFD_MU
    run_job_reg<SFD_MU>(jobs[j], wbase, lane, pw, npw, npw == 4 ? 3 : 1 + pi, npw > 1 ? xcells[pi] : nullptr);
#else
    run_job(jobs[j], wbase, lane);
#endif
  }
}

// The kernel's dynamic shared-memory limit is a process-wide attribute of
// the function on each device.  It is raised once per device to everything
// a block may opt into (minus the kernel's static shared memory) and never
// lowered, so launches from several threads or contexts cannot undo one
// another's setting between setting and launching; each launch still asks
// for only the bytes its strings need.
namespace {
constexpr int kMaxAttrDevices = 64;
std::mutex g_attr_mu;
bool g_attr_done[kMaxAttrDevices] = {};

cudaError_t raise_smem_limit() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxAttrDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_attr_done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, SFD_KERNEL);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(SFD_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - static_cast<int>(fa.sharedSizeBytes));
  if (e == cudaSuccess) g_attr_done[dev] = true;
  return e;
}
}  // namespace

// Host-side launcher of this class (C++ linkage, called by sfd_api.cu).  The
// job counter is cleared on the same stream before the kernel starts.  With
// group = 2 or 4 (register classes; warps_per_cta a multiple of it, 4 for
// groups of 4) each string gets a group of warps and one shared-memory
// region per group.
cudaError_t SFD_LAUNCHER(const Job* d_jobs, int n_jobs, int* d_counter, int warp_floats, int warps_per_cta,
                         int n_ctas, int group, cudaStream_t stream) {
#ifndef SFD_MU
  group = 1;
#endif
  if (group != 1 && group != 2 && group != 4) return cudaErrorInvalidValue;
  if (warps_per_cta % group != 0 || (group == 4 && warps_per_cta != 4)) return cudaErrorInvalidValue;
  const int regions = warps_per_cta / group;
  const size_t smem = static_cast<size_t>(warp_floats) * regions * sizeof(float);
  cudaError_t e = raise_smem_limit();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  SFD_KERNEL<<<n_ctas, warps_per_cta * kWarp, smem, stream>>>(d_jobs, n_jobs, d_counter, warp_floats, group);
  return cudaGetLastError();
}

}  // namespace sfd
