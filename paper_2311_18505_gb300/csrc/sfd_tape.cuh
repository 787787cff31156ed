// Gradients of a waveform loss (sfd_tape_* in sfd.h): forward synthesis with
// a checkpoint of every string's state every K samples, then a reverse sweep
// that, segment by segment from the last, restores a replay copy of each
// string from the segment's checkpoint, re-runs the forward kernels over the
// segment recording every level (Job::traj), and runs the adjoint kernel
// (sfd_adjoint.cu) backwards over those levels.  When the whole trajectory
// fits (kRecordForwardBytes, or sfd_tape_set_record_forward), the forward
// kernels record every level as they go and the reverse sweep replays
// nothing: a replay re-runs the same kernel from the same state, so its
// record is the forward's, bit for bit.
//
// Included once, at the end of sfd_api.cu (uses its internal pieces).

namespace sfd {
cudaError_t launch_adjoint(const AdjJob* d_jobs, int n_jobs, int smem_bytes, cudaStream_t stream);
cudaError_t adjoint_static_smem(size_t* bytes);
}

namespace {

constexpr size_t kTapeAlign = 256;
// largest whole-trajectory record the tape allocates on its own
constexpr size_t kRecordForwardBytes = size_t{4} << 30;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct sfd_tape {
  sfd_ctx* c = nullptr;
  int n = 0;
  int64_t n_samples = 0;
  int K = 0, n_seg = 0;
  std::vector<sfd_string*> fw, rp;      // forward strings and their replay copies
  std::vector<size_t> st_off, st_bytes; // per string: state (Scalars onwards) offset in the block, bytes
  std::vector<int64_t> rec_stride;      // per string: floats per recorded level
  size_t ckpt_stride = 0;               // bytes per checkpoint slot
  size_t traj_stride = 0;               // floats per string in the replay record
  size_t adj_stride = 0;                // doubles per string of adjoint state
  int adj_smem = 0;                     // shared-memory bytes of the adjoint kernel
  char* d_ckpt = nullptr;
  float* d_traj = nullptr;
  double* d_adj = nullptr;
  double* d_grad = nullptr;
  float* d_scratch = nullptr;
  AdjJob* d_ajobs = nullptr;
  bool forward_done = false;
  float* d_traj_full = nullptr;         // every level of every segment (record-on-forward mode)
  std::vector<size_t> full_off;         // per string: its first float in d_traj_full
  size_t full_floats = 0;               // floats of the whole record
};

namespace {

void tape_free(sfd_tape* t) {
  if (t->c) cudaStreamSynchronize(t->c->stream);
  for (sfd_string* s : t->fw) if (s) sfd_string_destroy(s);
  for (sfd_string* s : t->rp) {
    if (!s) continue;
    t->c->pool.dealloc(s->block);
    delete s;
  }
  cudaFree(t->d_ckpt);
  cudaFree(t->d_traj);
  cudaFree(t->d_adj);
  cudaFree(t->d_grad);
  cudaFree(t->d_scratch);
  cudaFree(t->d_ajobs);
  cudaFree(t->d_traj_full);
  delete t;
}

size_t full_traj_bytes(const sfd_tape* t) { return sizeof(float) * t->full_floats; }

// segment seg of string i in the whole-trajectory record (each string's
// segments at its own record stride)
float* full_traj(const sfd_tape* t, int i, int seg) {
  return t->d_traj_full + t->full_off[i] + static_cast<size_t>(seg) * t->K * t->rec_stride[i];
}

char* ckpt_slot(const sfd_tape* t, int i, int c) {
  return t->d_ckpt + (static_cast<size_t>(i) * (t->n_seg + 1) + c) * t->ckpt_stride;
}

sfd_status tape_checkpoint(sfd_tape* t, const std::vector<sfd_string*>& strings, int c) {
  for (int i = 0; i < t->n; ++i) {
    sfd_string* s = strings[i];
    SFD_CUDA(cudaMemcpyAsync(ckpt_slot(t, i, c), s->block + t->st_off[i], t->st_bytes[i],
                             cudaMemcpyDeviceToDevice, t->c->stream));
  }
  return SFD_OK;
}

// level at which segment c's checkpoint (c = 0: the initial state) sits
int64_t seg_start_level(const sfd_tape* t, int c) { return c == 0 ? 1 : static_cast<int64_t>(c) * t->K - 1; }

}  // namespace

extern "C" {

sfd_status sfd_tape_create(sfd_ctx* c, int32_t n, const sfd_string_params* params, const sfd_excitation* exc,
                           const sfd_modulation* mod, int64_t n_samples, int32_t checkpoint_every,
                           sfd_tape** out) {
  if (!c || !params || !exc || !out) return fail(SFD_EINVAL, "NULL argument");
  *out = nullptr;
  if (n <= 0 || n_samples < 2 || checkpoint_every < 2)
    return fail(SFD_EINVAL, "need n > 0 strings, n_samples >= 2 and checkpoint_every >= 2");
  for (int i = 0; i < n; ++i)
    if (exc[i].kind != kPluck && exc[i].kind != kHammer && exc[i].kind != kBow)
      return fail(SFD_EINVAL, "string %d: unknown excitation", i);
  sfd_status rc = set_device(c);
  if (rc) return rc;
  sfd_tape* t = new (std::nothrow) sfd_tape();
  if (!t) return fail(SFD_ENOMEM, "host allocation failed");
  t->c = c;
  t->n = n;
  t->n_samples = n_samples;
  t->K = checkpoint_every;
  t->n_seg = static_cast<int>((n_samples + checkpoint_every - 1) / checkpoint_every);
  for (int i = 0; i < n && rc == SFD_OK; ++i) {
    sfd_string* s = nullptr;
    rc = sfd_string_create(c, &params[i], &s);
    if (rc) break;
    t->fw.push_back(s);
    const sfd_excitation& e = exc[i];
    rc = e.kind == kPluck    ? sfd_excite_pluck(s, e.amp_m, e.pos)
         : e.kind == kHammer ? sfd_excite_hammer(s, e.mass_kg, e.vel_mps, e.pos, e.omega_h, e.alpha_h)
                             : sfd_excite_bow(s, e.vel_mps, e.force_n, e.pos, e.a_s_per_m, e.eps, e.release_time_s);
    if (rc) break;
    if (mod && mod[i].kind != SFD_MOD_NONE) {
      rc = sfd_set_modulation(s, mod[i].kind, mod[i].rate_hz, mod[i].depth, mod[i].phase_rad, mod[i].duration_s);
      if (rc) break;
    }
    sfd_string* r = nullptr;
    rc = clone_string(s, &r);
    if (rc) break;
    t->rp.push_back(r);
    const Desc& D = s->h;
    t->st_off.push_back(static_cast<size_t>(reinterpret_cast<char*>(s->d_sc) - s->block));
    t->st_bytes.push_back(block_bytes(D) - t->st_off.back());
    t->rec_stride.push_back(static_cast<int64_t>(round_up(2 * D.n_u + 2 * D.n_z + 2, 4)));
    t->ckpt_stride = std::max(t->ckpt_stride, round_up(t->st_bytes.back(), kTapeAlign));
    t->traj_stride = std::max(t->traj_stride, static_cast<size_t>(t->rec_stride.back()) * t->K);
    t->adj_stride = std::max(t->adj_stride, round_up(2 * D.n_u + 4 * D.n_z + 2, 64));
    t->adj_smem = std::max(t->adj_smem, adj_smem_bytes(D.m_u, D.m_z));
  }
  size_t adj_static = 0;
  if (rc == SFD_OK) {
    const cudaError_t e = adjoint_static_smem(&adj_static);
    if (e != cudaSuccess) rc = cuda_fail(e, "adjoint kernel attributes");
  }
  if (rc == SFD_OK && static_cast<size_t>(t->adj_smem) + adj_static > c->smem_optin)
    rc = fail(SFD_EINVAL, "a string's grid exceeds the adjoint kernel's shared memory");
  if (rc == SFD_OK) {
    cudaError_t e = cudaMalloc(&t->d_ckpt, static_cast<size_t>(n) * (t->n_seg + 1) * t->ckpt_stride);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_traj, sizeof(float) * n * t->traj_stride);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_adj, sizeof(double) * n * t->adj_stride);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_grad, sizeof(double) * n * kGradSlots);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_scratch, sizeof(float) * n * static_cast<size_t>(t->K));
    if (e == cudaSuccess) e = cudaMalloc(&t->d_ajobs, sizeof(AdjJob) * n);
    if (e != cudaSuccess) rc = cuda_fail(e, "tape buffers");
  }
  for (int i = 0; rc == SFD_OK && i < n; ++i) {
    t->full_off.push_back(t->full_floats);
    t->full_floats += static_cast<size_t>(t->n_seg) * t->K * t->rec_stride[i];
  }
  if (rc == SFD_OK && full_traj_bytes(t) <= kRecordForwardBytes) {
    // record on the forward pass when the device has room; else replay
    if (cudaMalloc(&t->d_traj_full, full_traj_bytes(t)) != cudaSuccess) {
      t->d_traj_full = nullptr;
      cudaGetLastError();   // an allocation failure is not sticky: clear it
    }
  }
  if (rc) {
    tape_free(t);
    return rc;
  }
  *out = t;
  return SFD_OK;
}

sfd_status sfd_tape_set_record_forward(sfd_tape* t, int32_t enable) {
  if (!t) return fail(SFD_EINVAL, "NULL argument");
  sfd_status rc = set_device(t->c);
  if (rc) return rc;
  if (!enable) {
    if (t->d_traj_full) {
      SFD_CUDA(cudaStreamSynchronize(t->c->stream));
      cudaFree(t->d_traj_full);
      t->d_traj_full = nullptr;
    }
    return SFD_OK;
  }
  if (t->d_traj_full) return SFD_OK;
  if (cudaMalloc(&t->d_traj_full, full_traj_bytes(t)) != cudaSuccess) {
    t->d_traj_full = nullptr;
    cudaGetLastError();
    return fail(SFD_ENOMEM, "no device room for the %zu-byte trajectory record", full_traj_bytes(t));
  }
  t->forward_done = false;   // the next forward pass records
  return SFD_OK;
}

sfd_status sfd_tape_forward(sfd_tape* t, float* y_device) {
  if (!t || !y_device) return fail(SFD_EINVAL, "NULL argument");
  sfd_ctx* c = t->c;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  for (sfd_string* s : t->fw) {   // every forward starts from the initial state
    if ((rc = upload_initial(s))) return rc;
    s->started = false;
  }
  if ((rc = tape_checkpoint(t, t->fw, 0))) return rc;
  std::vector<const sfd_string*> owners(t->fw.begin(), t->fw.end());
  for (int seg = 0; seg < t->n_seg; ++seg) {
    const int64_t first = static_cast<int64_t>(seg) * t->K;
    const int64_t ns = std::min<int64_t>(t->K, t->n_samples - first);
    std::vector<Job> jobs;
    for (int i = 0; i < t->n; ++i) {
      Job j{t->fw[i]->d_desc, y_device + i * t->n_samples + first, ns};
      if (t->d_traj_full) {
        j.traj = full_traj(t, i, seg);
        j.traj_stride = t->rec_stride[i];
      }
      jobs.push_back(j);
    }
    if ((rc = launch_jobs(c, jobs, owners))) return rc;
    for (sfd_string* s : t->fw) s->started = true;
    if ((rc = tape_checkpoint(t, t->fw, seg + 1))) return rc;
  }
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  int worst = SFD_OK;
  for (sfd_string* s : t->fw) {
    Scalars sc{};
    if ((rc = read_status(s, &sc))) return rc;
    const sfd_status st = status_code(sc);
    if (st == SFD_EUNSTABLE || (st == SFD_ENOCONV && worst == SFD_OK)) worst = st;
  }
  t->forward_done = true;
  if (worst == SFD_EUNSTABLE) return fail(worst, "a string's state became non-finite");
  if (worst == SFD_ENOCONV) return fail(worst, "a coupled solve reached its sweep cap (result kept)");
  return SFD_OK;
}

sfd_status sfd_tape_backward(sfd_tape* t, const float* dy_device, double* grad) {
  if (!t || !dy_device || !grad) return fail(SFD_EINVAL, "NULL argument");
  if (!t->forward_done) return fail(SFD_ESTATE, "sfd_tape_forward must come first");
  sfd_ctx* c = t->c;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  SFD_CUDA(cudaMemsetAsync(t->d_adj, 0, sizeof(double) * t->n * t->adj_stride, c->stream));
  SFD_CUDA(cudaMemsetAsync(t->d_grad, 0, sizeof(double) * t->n * kGradSlots, c->stream));
  std::vector<const sfd_string*> owners(t->rp.begin(), t->rp.end());
  std::vector<AdjJob> aj(t->n);
  for (int seg = t->n_seg - 1; seg >= 0; --seg) {
    const int64_t first = static_cast<int64_t>(seg) * t->K;
    const int64_t ns = std::min<int64_t>(t->K, t->n_samples - first);
    const int64_t m0 = seg_start_level(t, seg), m1 = first + ns - 1;
    // the segment's levels: recorded by the forward pass, or replayed now
    // from the segment's checkpoint
    std::vector<Job> jobs;
    for (int i = 0; i < t->n; ++i) {
      Job j{t->rp[i]->d_desc, t->d_scratch + static_cast<size_t>(i) * t->K, ns};
      j.traj = t->d_traj_full ? full_traj(t, i, seg) : t->d_traj + static_cast<size_t>(i) * t->traj_stride;
      j.traj_stride = t->rec_stride[i];
      jobs.push_back(j);
      if (!t->d_traj_full)
        SFD_CUDA(cudaMemcpyAsync(t->rp[i]->block + t->st_off[i], ckpt_slot(t, i, seg), t->st_bytes[i],
                                 cudaMemcpyDeviceToDevice, c->stream));
    }
    if (!t->d_traj_full && (rc = launch_jobs(c, jobs, owners))) return rc;
    // reverse sweep over the segment's levels (m0, m1]
    for (int i = 0; i < t->n; ++i) {
      const sfd_string* s = t->rp[i];
      const Desc& D = s->h;
      char* slot = ckpt_slot(t, i, seg);
      auto at = [&](const void* dev) {
        return reinterpret_cast<const float*>(slot + (static_cast<const char*>(dev) - s->block - t->st_off[i]));
      };
      AdjJob& a = aj[i];
      a.desc = s->d_desc;
      a.u0 = at(D.u);
      a.du0 = at(D.du);
      a.z0 = at(D.z);
      a.dz0 = at(D.dz);
      a.sc0 = reinterpret_cast<const Scalars*>(slot);
      a.traj = jobs[i].traj;
      a.traj_stride = t->rec_stride[i];
      a.m_start = m0;
      a.m_end = m1;
      a.dy = dy_device + static_cast<size_t>(i) * t->n_samples;
      a.adj = t->d_adj + static_cast<size_t>(i) * t->adj_stride;
      a.grad = t->d_grad + static_cast<size_t>(i) * kGradSlots;
      a.first = seg == 0 ? 1 : 0;
      a.pluck_pos = s->exc == kPluck ? static_cast<float>(s->pluck_pos) : -1.f;
    }
    SFD_CUDA(h2d(c, t->d_ajobs, aj.data(), sizeof(AdjJob) * t->n));
    SFD_CUDA(launch_adjoint(t->d_ajobs, t->n, t->adj_smem, c->stream));
    // (the next segment's replay and job table follow in stream order)
  }
  std::vector<double> g(static_cast<size_t>(t->n) * kGradSlots);
  // on the context stream, after the last sweep (a plain cudaMemcpy would not
  // wait for a non-blocking context stream)
  SFD_CUDA(cudaMemcpyAsync(g.data(), t->d_grad, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, c->stream));
  SFD_CUDA(cudaStreamSynchronize(c->stream));
  c->d2h_bytes += sizeof(double) * g.size();
  // chain rule from the step's coefficients to the physical parameters
  // (grid held fixed; the transverse line carries the scale rho)
  for (int i = 0; i < t->n; ++i) {
    const sfd_string* s = t->fw[i];
    const sfd_string_params& p = s->p;
    const Desc& D = s->h;
    const double* gi = &g[static_cast<size_t>(i) * kGradSlots];
    const double k = s->k, gm = s->gamma, ht = 1.0 / s->n_t, hl = 1.0 / s->n_l;
    const double s0 = p.sigma0 * k;
    const double rho = (static_cast<double>(D.dg) + 2.0 * static_cast<double>(D.og)) / (1.0 + s0);
    const double k2 = k * k, ht2 = ht * ht, ht3 = ht2 * ht, ht4 = ht2 * ht2, hl2 = hl * hl;
    double* o = grad + static_cast<size_t>(i) * SFD_GRAD_PARAMS;
    o[0] = gi[kGMu2] * 2.0 * rho * p.kappa * k2 / ht4;
    const double dphi = gm * gm * p.alpha;   // d phi' / d alpha
    o[1] = gi[kGLam2l] * 2.0 * gm * gm * p.alpha * k2 / hl2 +
           dphi * (gi[kGCa] * rho * k2 / (2.0 * ht4) + gi[kGCb] * rho * k2 / (2.0 * ht3) +
                   gi[kGCz] * k2 / (2.0 * ht2 * hl));
    o[2] = k * (rho * gi[kGS0u] + gi[kGS0]);
    o[3] = k * (rho * gi[kGS1] / ht2 + gi[kGS1l] / hl2);
    o[4] = gi[kGAmp] / p.length_m;   // c0 = amp / L; v_hat = v / L
  }
  return SFD_OK;
}

sfd_status sfd_tape_destroy(sfd_tape* t) {
  if (!t) return SFD_OK;
  sfd_status rc = set_device(t->c);
  if (rc) return rc;
  tape_free(t);
  return SFD_OK;
}

}  // extern "C"
