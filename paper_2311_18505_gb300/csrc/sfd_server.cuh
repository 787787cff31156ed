// Serving: continuous batching of note requests (sfd_server_* in sfd.h).
//
// Included once, at the end of sfd_api.cu: it uses that file's internal
// pieces (pool, string setup, block image, launch plan).
//
// Every pump prepares chunk p (ping-pong buffer p & 1: admission, uploads,
// job table) while chunk p - 1 runs, waits for chunk p - 1, then launches
// chunk p's kernels on the idle device and delivers chunk p - 1, so the
// host's admission and delivery work overlaps the GPU's work and the class
// kernels start in launch order.  All host<->device copies go through
// pinned buffers, so nothing in a pump waits for the stream except the one
// event of the previous chunk.  Buffer p & 1 (output, job table, staging
// of admitted notes' initial blocks, status scalars) is written again two
// pumps later, after chunk p has been waited for.

#include <chrono>
#include <deque>

namespace {

struct SvNote {
  sfd_string* s = nullptr;
  uint64_t tag = 0;
  int64_t total = 0;     // samples requested
  int64_t issued = 0;    // samples enqueued so far
  double arrival = 0;    // server clock
};

struct SvEntry {         // one note's part of an enqueued chunk
  SvNote* note;
  int64_t first;
  int32_t n;
  bool last;
};

struct SvChunk {
  bool active = false;
  std::vector<SvEntry> entries;   // row j of the chunk's output = entries[j]
};

template <class T>
struct Pinned {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    release();
    void* q = nullptr;
    cudaError_t e = cudaHostAlloc(&q, std::max<size_t>(count, 1) * sizeof(T), cudaHostAllocDefault);
    if (e != cudaSuccess) return e;
    p = static_cast<T*>(q);
    n = count;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    n = 0;
  }
};

constexpr size_t kStageInitial = 4u << 20;   // bytes of initial blocks staged per pump (grows)

}  // namespace

struct sfd_server {
  sfd_ctx* c = nullptr;
  int chunk = 0, max_live = 0;
  std::chrono::steady_clock::time_point t0;
  std::deque<SvNote*> queue;
  std::vector<SvNote*> live;
  char* d_out[2] = {};
  char* d_jobs[2] = {};
  size_t reserved = 0;                 // pool bytes held by the buffers above
  Pinned<float> h_out[2];
  Pinned<Job> h_jobs[2];
  Pinned<Scalars> h_sc[2];
  Pinned<char> stage[2];
  cudaEvent_t done[2] = {};
  SvChunk fl[2];
  int64_t seq = 0;
  std::vector<sfd_chunk> ready;
  sfd_server_stats st{};

  double clock() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void server_free(sfd_server* sv) {
  sfd_ctx* c = sv->c;
  for (int b = 0; b < 2; ++b) {
    if (sv->fl[b].active && sv->done[b]) cudaEventSynchronize(sv->done[b]);
  }
  cudaStreamSynchronize(c->stream);
  auto drop = [&](SvNote* nt) {
    if (nt->s) {
      if (nt->s->block) c->pool.dealloc(nt->s->block);
      delete nt->s;
    }
    delete nt;
  };
  for (SvNote* nt : sv->live) drop(nt);
  for (SvNote* nt : sv->queue) drop(nt);
  sv->live.clear();
  sv->queue.clear();
  for (int b = 0; b < 2; ++b) {
    c->pool.dealloc(sv->d_out[b]);
    c->pool.dealloc(sv->d_jobs[b]);
    sv->h_out[b].release();
    sv->h_jobs[b].release();
    sv->h_sc[b].release();
    sv->stage[b].release();
    if (sv->done[b]) cudaEventDestroy(sv->done[b]);
  }
  delete sv;
}

}  // namespace

extern "C" {

sfd_status sfd_server_create(sfd_ctx* c, int32_t chunk_samples, int32_t max_live, sfd_server** out) {
  if (!c || !out) return fail(SFD_EINVAL, "NULL argument");
  *out = nullptr;
  if (chunk_samples <= 0 || max_live <= 0) return fail(SFD_EINVAL, "chunk_samples and max_live must be > 0");
  sfd_status rc = set_device(c);
  if (rc) return rc;
  sfd_server* sv = new (std::nothrow) sfd_server();
  if (!sv) return fail(SFD_ENOMEM, "host allocation failed");
  sv->c = c;
  sv->chunk = chunk_samples;
  sv->max_live = max_live;
  sv->t0 = std::chrono::steady_clock::now();
  const size_t out_n = static_cast<size_t>(max_live) * chunk_samples;
  for (int b = 0; b < 2; ++b) {
    const size_t ob = sizeof(float) * out_n, jb = sizeof(Job) * max_live;
    sv->d_out[b] = c->pool.alloc(ob);
    sv->d_jobs[b] = c->pool.alloc(jb);
    if (!sv->d_out[b] || !sv->d_jobs[b]) {
      server_free(sv);
      return fail(SFD_ENOMEM, "device pool too small for the server's buffers");
    }
    sv->reserved += (ob + kAlign - 1) / kAlign * kAlign + (jb + kAlign - 1) / kAlign * kAlign;
    cudaError_t e = sv->h_out[b].alloc(out_n);
    if (e == cudaSuccess) e = sv->h_jobs[b].alloc(max_live);
    if (e == cudaSuccess) e = sv->h_sc[b].alloc(max_live);
    if (e == cudaSuccess) e = sv->stage[b].alloc(kStageInitial);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->done[b], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      server_free(sv);
      return cuda_fail(e, "server host buffers");
    }
  }
  *out = sv;
  return SFD_OK;
}

static sfd_status submit_note(sfd_server* sv, const sfd_request* r, int32_t env_n, const double* env_t,
                              const double* env_v, const double* env_f, const double* env_x) {
  if (!sv || !r) return fail(SFD_EINVAL, "NULL argument");
  if (r->n_samples <= 0) return fail(SFD_EINVAL, "n_samples must be > 0");
  sfd_string* s = new (std::nothrow) sfd_string();
  if (!s) return fail(SFD_ENOMEM, "host allocation failed");
  // the grid is sized for the modulation's peak wave speed (reading A14)
  sfd_string_params q = r->params;
  if (std::isfinite(r->mod_depth)) q.f0_max_ratio = std::max(q.f0_max_ratio, modulation_peak(r->mod_kind, r->mod_depth));
  sfd_status rc = init_host_string(q, s);
  if (rc == SFD_OK) rc = apply_excitation(s, r->exc);
  if (rc == SFD_OK && env_n > 0) rc = apply_bow_envelope(s, env_n, env_t, env_v, env_f, env_x);
  if (rc == SFD_OK) rc = apply_modulation(s, r->mod_kind, r->mod_rate_hz, r->mod_depth, r->mod_phase_rad,
                                          r->mod_duration_s);
  if (rc == SFD_OK) {
    const size_t wbytes = static_cast<size_t>(warp_smem_floats(s->h.m_u, s->h.m_z, s->h.z_jacobi)) * sizeof(float);
    if (wbytes > sv->c->smem_optin)
      rc = fail(SFD_EINVAL, "grid (N_t=%d, N_l=%d) exceeds one warp's shared memory", s->n_t, s->n_l);
  }
  if (rc == SFD_OK && block_bytes(s->h) > sv->c->pool.size() - sv->reserved)
    rc = fail(SFD_ENOMEM, "the note's state (%zu bytes) can never fit the device pool", block_bytes(s->h));
  if (rc) {
    delete s;
    return rc;
  }
  s->ctx = sv->c;
  SvNote* nt = new (std::nothrow) SvNote();
  if (!nt) {
    delete s;
    return fail(SFD_ENOMEM, "host allocation failed");
  }
  nt->s = s;
  nt->tag = r->tag;
  nt->total = r->n_samples;
  nt->arrival = r->arrival_s >= 0 ? r->arrival_s : sv->clock();
  sv->queue.push_back(nt);
  sv->st.submitted++;
  return SFD_OK;
}

sfd_status sfd_server_submit(sfd_server* sv, const sfd_request* r) {
  return submit_note(sv, r, 0, nullptr, nullptr, nullptr, nullptr);
}

sfd_status sfd_server_submit_bow_envelope(sfd_server* sv, const sfd_request* r, int32_t n_points, const double* t_s,
                                          const double* vel_mps, const double* force_n, const double* pos) {
  if (n_points <= 0) return fail(SFD_EINVAL, "1 to 16 breakpoints");
  return submit_note(sv, r, n_points, t_s, vel_mps, force_n, pos);
}

sfd_status sfd_server_pump(sfd_server* sv, const sfd_chunk** chunks, int32_t* n_chunks) {
  if (!sv || !chunks || !n_chunks) return fail(SFD_EINVAL, "NULL argument");
  *chunks = nullptr;
  *n_chunks = 0;
  sfd_ctx* c = sv->c;
  sfd_status rc = set_device(c);
  if (rc) return rc;
  const int b = static_cast<int>(sv->seq & 1), q = b ^ 1;

  // 1. admission, in arrival order, by free slot and device memory
  size_t staged = 0;
  while (!sv->queue.empty() && static_cast<int>(sv->live.size()) < sv->max_live) {
    SvNote* nt = sv->queue.front();
    sfd_string* s = nt->s;
    const size_t bytes = block_bytes(s->h);
    if (staged + bytes > sv->stage[b].n) {
      if (staged > 0) break;   // the rest next pump
      // nothing staged in this buffer since its last chunk completed
      cudaError_t e = sv->stage[b].alloc(std::max(bytes, 2 * sv->stage[b].n));
      if (e != cudaSuccess) return cuda_fail(e, "server staging buffer");
    }
    s->block = c->pool.alloc(bytes);
    if (!s->block) break;      // waits for memory (and later requests behind it)
    carve(s);
    write_image(s, sv->stage[b].p + staged);
    cudaError_t e = cudaMemcpyAsync(s->block, sv->stage[b].p + staged, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
      c->pool.dealloc(s->block);
      s->block = nullptr;
      return cuda_fail(e, "upload of an admitted note");
    }
    c->h2d_bytes += bytes;
    staged += bytes;
    sv->live.push_back(nt);
    sv->queue.pop_front();
    sv->st.admitted++;
  }

  // 2. the next chunk of every live note
  SvChunk& ch = sv->fl[b];
  ch.entries.clear();
  std::vector<Job> jobs;
  std::vector<const sfd_string*> owners;
  float* dout = reinterpret_cast<float*>(sv->d_out[b]);
  for (SvNote* nt : sv->live) {
    const int64_t rem = nt->total - nt->issued;
    if (rem <= 0) continue;
    const int32_t n = static_cast<int32_t>(std::min<int64_t>(rem, sv->chunk));
    jobs.push_back(Job{nt->s->d_desc, dout + ch.entries.size() * sv->chunk, n});
    owners.push_back(nt->s);
    ch.entries.push_back(SvEntry{nt, nt->issued, n, nt->issued + n == nt->total});
    nt->issued += n;
    nt->s->started = true;
  }
  if (!jobs.empty()) {
    Plan P;
    if ((rc = make_plan(c, jobs, owners, 0, P))) return rc;
    std::memcpy(sv->h_jobs[b].p, P.jobs.data(), sizeof(Job) * P.jobs.size());
    SFD_CUDA(cudaMemcpyAsync(sv->d_jobs[b], sv->h_jobs[b].p, sizeof(Job) * P.jobs.size(), cudaMemcpyHostToDevice,
                             c->stream));
    c->h2d_bytes += sizeof(Job) * P.jobs.size();
    // launched on an idle device the classes start in launch order, heaviest
    // first; enqueued behind the previous chunk they would become ready
    // together and start in no fixed order (measured on a 20 s trace at
    // 2000 notes/s: 151.9 and 151.8 M delivered samples/s this way against
    // 150.3 M, alternating runs).  The host's admission and job-table work
    // for this chunk has already overlapped the previous one.
    if (sv->fl[q].active) SFD_CUDA(cudaEventSynchronize(sv->done[q]));
    if ((rc = issue_plan(c, P, reinterpret_cast<const Job*>(sv->d_jobs[b])))) return rc;
    const size_t ob = sizeof(float) * ch.entries.size() * sv->chunk;
    SFD_CUDA(cudaMemcpyAsync(sv->h_out[b].p, dout, ob, cudaMemcpyDeviceToHost, c->stream));
    c->d2h_bytes += ob;
    int k = 0;
    for (const SvEntry& en : ch.entries) {
      if (!en.last) continue;
      SFD_CUDA(cudaMemcpyAsync(sv->h_sc[b].p + k++, en.note->s->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                               c->stream));
      c->d2h_bytes += sizeof(Scalars);
    }
    SFD_CUDA(cudaEventRecord(sv->done[b], c->stream));
    ch.active = true;
  }

  // 3. deliver the previous chunk, 4. retire the notes that ended in it
  sv->ready.clear();
  SvChunk& pv = sv->fl[q];
  if (pv.active) {
    SFD_CUDA(cudaEventSynchronize(sv->done[q]));
    const double t = sv->clock();
    int k = 0;
    for (size_t j = 0; j < pv.entries.size(); ++j) {
      const SvEntry& en = pv.entries[j];
      sfd_chunk r{};
      r.tag = en.note->tag;
      r.first_sample = en.first;
      r.n = en.n;
      r.last = en.last ? 1 : 0;
      r.status = en.last ? status_code(sv->h_sc[q].p[k++]) : SFD_OK;
      r.samples = sv->h_out[q].p + j * sv->chunk;
      r.ready_s = t;
      r.arrival_s = en.note->arrival;
      sv->ready.push_back(r);
      sv->st.samples += en.n;
      sv->st.chunks++;
    }
    for (const SvEntry& en : pv.entries) {
      if (!en.last) continue;
      auto it = std::find(sv->live.begin(), sv->live.end(), en.note);
      if (it != sv->live.end()) {
        *it = sv->live.back();
        sv->live.pop_back();
      }
      c->pool.dealloc(en.note->s->block);
      delete en.note->s;
      delete en.note;
      sv->st.completed++;
    }
    pv.active = false;
    pv.entries.clear();
  }
  sv->seq++;
  *chunks = sv->ready.data();
  *n_chunks = static_cast<int32_t>(sv->ready.size());
  return SFD_OK;
}

double sfd_server_clock(const sfd_server* sv) { return sv ? sv->clock() : 0.0; }

sfd_status sfd_server_stats_get(const sfd_server* sv, sfd_server_stats* st) {
  if (!sv || !st) return fail(SFD_EINVAL, "NULL argument");
  *st = sv->st;
  st->queued = static_cast<int64_t>(sv->queue.size());
  st->live = static_cast<int64_t>(sv->live.size());
  st->in_flight = (sv->fl[0].active || sv->fl[1].active) ? 1 : 0;
  st->pool_used = sv->c->pool.used();
  st->pool_size = sv->c->pool.size();
  return SFD_OK;
}

sfd_status sfd_server_destroy(sfd_server* sv) {
  if (!sv) return SFD_OK;
  sfd_status rc = set_device(sv->c);
  if (rc) return rc;
  server_free(sv);
  return SFD_OK;
}

}  // extern "C"
