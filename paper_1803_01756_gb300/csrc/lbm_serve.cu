// Serving: a request loop that advances many simulation jobs with continuous
// batching.  One server thread owns the device work; clients submit and poll
// from any thread.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lbm_handle.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  long id = 0;
  int nx = 0, ny = 0;
  lbm_params_t p{};
  long nsteps = 0, done_steps = 0;
  std::vector<double> rho0;
  size_t footprint = 0;
  lbm_h lat = nullptr;
  int state = LBM_JOB_QUEUED;  // LBM_JOB_* or a negative LBM_ERR_*
  std::vector<double> out[4];  // rho, ux, uy, T after the last step
  Clock::time_point t_submit, t_done;
};

// mode key: jobs with equal keys share one batched launch
int mode_key(const lbm_lattice *h) {
  return (h->dp.y_walls ? 1 : 0) | (h->dp.x_open ? 2 : 0) | (h->dp.thermal ? 4 : 0) |
         (h->dp.multiphase ? 8 : 0) | (h->p.storage << 4);
}

}  // namespace

struct lbm_server {
  lbm_server_config_t cfg{};
  std::mutex mu;
  std::condition_variable cv;
  std::map<long, std::shared_ptr<Job>> jobs;
  std::deque<std::shared_ptr<Job>> queue;       // submitted, not admitted (FIFO)
  std::vector<std::shared_ptr<Job>> active;     // owned by the server thread
  size_t bytes_in_use = 0, peak_bytes = 0;
  long n_active = 0;  // size of `active`, readable under the mutex
  long next_id = 1, completed = 0, failed = 0, rounds = 0, launches = 0;
  bool stop = false;
  std::thread worker;
  cudaStream_t stream = nullptr;
  // batched launch of each mode group, kept across rounds while the group's jobs (by id)
  // stay the same; rebuilt when a job joins or leaves
  struct Group {
    std::vector<long> ids;
    lbm_batch_h b = nullptr;
  };
  std::map<int, Group> groups;
  unsigned *h_status = nullptr;  // pinned, one status word per active job
};

namespace {

// device bytes lbm_create allocates for a lattice (populations x2, T x2, four scratch
// planes, reduction partials, staging, the boundary scalars of one graph chunk); used for
// admission before allocating
size_t footprint_of(int nx, int ny, int storage) {
  const size_t pitch = (size_t)((nx + 31) / 32 * 32);
  const size_t plane = pitch * (size_t)ny;
  const size_t es = storage == LBM_STORAGE_F32 ? 4 : 2;
  return 2 * 9 * plane * es + 6 * plane * sizeof(float) + (size_t)nx * ny * sizeof(double) +
         2 * 1216 * sizeof(double) + 64 + lbm_lattice::kChunk * sizeof(lbm::StepScalars);
}

void retire(lbm_server *s, const std::shared_ptr<Job> &j, int state) {
  if (j->lat) {
    if (state == LBM_JOB_DONE) {
      const size_t n = (size_t)j->nx * j->ny;
      for (auto &v : j->out) v.resize(n);
      int rc = lbm_read_fields(j->lat, j->out[0].data(), j->out[1].data(), j->out[2].data(),
                               j->out[3].data(), s->stream);
      if (rc != LBM_OK) state = rc;
    }
    lbm_destroy(j->lat);
    j->lat = nullptr;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  j->t_done = Clock::now();
  j->state = state;
  s->bytes_in_use -= j->footprint;
  if (state == LBM_JOB_DONE)
    s->completed++;
  else
    s->failed++;
  s->cv.notify_all();
}

// Move queued jobs into the active set while slots and the HBM budget allow
// (first come, first served; a job that does not fit blocks the ones behind it).
void admit(lbm_server *s) {
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->queue.empty() || (int)s->active.size() >= s->cfg.max_active) return;
      j = s->queue.front();
      if (s->bytes_in_use + j->footprint > s->cfg.hbm_budget) return;
      s->queue.pop_front();
      s->bytes_in_use += j->footprint;
      s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
      j->state = LBM_JOB_RUNNING;
    }
    lbm_params_t p = j->p;
    p.kernel = LBM_KERNEL_FUSED;
    int rc = lbm_create(j->nx, j->ny, &p, &j->lat);
    if (rc == LBM_OK && !j->rho0.empty())
      rc = lbm_write_fields(j->lat, j->rho0.data(), nullptr, s->stream);
    j->rho0.clear();
    j->rho0.shrink_to_fit();
    if (rc != LBM_OK) {
      retire(s, j, rc);
      continue;
    }
    s->active.push_back(j);
    std::lock_guard<std::mutex> lock(s->mu);
    s->n_active = (long)s->active.size();
  }
}

void drop_group(lbm_server::Group &g) {
  if (g.b) lbm_batch_destroy(g.b);
  g.b = nullptr;
  g.ids.clear();
}

// One scheduling round: every group of active jobs with equal modes advances by the
// same number of steps in one batched launch per step; then every job's status word is
// read with one synchronisation, and finished jobs are read back and freed.
// A lattice this large fills the GPU alone (about 4 tiles of the fused kernel per SM) and
// runs faster in the single-lattice kernel than in the batched one (69 against 102 us per
// update on 4096 x 512), so it is stepped alone.
constexpr long long kAloneNodes = 1LL << 20;

void round(lbm_server *s) {
  std::map<int, std::vector<std::shared_ptr<Job>>> groups;
  std::vector<std::shared_ptr<Job>> alone;
  for (auto &j : s->active) {
    if ((long long)j->nx * j->ny >= kAloneNodes)
      alone.push_back(j);
    else
      groups[mode_key(j->lat)].push_back(j);
  }
  for (auto &j : alone) {
    const long m = std::min(s->cfg.chunk_steps, j->nsteps - j->done_steps);
    if (m <= 0) continue;
    const int rc = lbm_step(j->lat, m, s->stream);
    s->launches += m;
    if (rc != LBM_OK)
      retire(s, j, rc);
    else
      j->done_steps += m;
  }
  // cached batches whose group changed or vanished go first
  for (auto it = s->groups.begin(); it != s->groups.end();) {
    auto g = groups.find(it->first);
    bool same = g != groups.end() && g->second.size() == it->second.ids.size();
    for (size_t k = 0; same && k < g->second.size(); k++) same = g->second[k]->id == it->second.ids[k];
    if (same) {
      ++it;
    } else {
      drop_group(it->second);
      it = s->groups.erase(it);
    }
  }
  for (auto &kv : groups) {
    auto &g = kv.second;
    long m = s->cfg.chunk_steps;
    for (auto &j : g) m = std::min(m, j->nsteps - j->done_steps);
    if (m <= 0) continue;
    lbm_server::Group &cached = s->groups[kv.first];
    int rc = LBM_OK;
    if (!cached.b) {
      std::vector<lbm_h> hs;
      for (auto &j : g) {
        hs.push_back(j->lat);
        cached.ids.push_back(j->id);
      }
      rc = lbm_batch_create(hs.data(), (int)hs.size(), &cached.b);
    }
    if (rc == LBM_OK) rc = lbm_batch_step(cached.b, m, s->stream);
    s->launches += m;
    if (rc != LBM_OK) drop_group(cached);
    for (auto &j : g) {
      if (rc != LBM_OK) {
        retire(s, j, rc);
        continue;
      }
      j->done_steps += m;
    }
  }
  // status words of the running jobs: one asynchronous copy each, one synchronisation
  std::vector<std::shared_ptr<Job>> run;
  for (auto &j : s->active)
    if (j->state == LBM_JOB_RUNNING) run.push_back(j);
  bool copied = true;
  for (size_t k = 0; k < run.size(); k++)
    copied = copied && cudaMemcpyAsync(&s->h_status[k], run[k]->lat->status, sizeof(unsigned),
                                       cudaMemcpyDeviceToHost, s->stream) == cudaSuccess;
  copied = cudaStreamSynchronize(s->stream) == cudaSuccess && copied;
  std::vector<std::shared_ptr<Job>> still;
  for (size_t k = 0; k < run.size(); k++) {
    auto &j = run[k];
    const unsigned bits = copied ? s->h_status[k] : ~0u;
    if (!copied) {
      retire(s, j, LBM_ERR_CUDA);
    } else if (bits) {
      retire(s, j, LBM_ERR_UNSTABLE);
    } else if (j->done_steps >= j->nsteps) {
      retire(s, j, LBM_JOB_DONE);
    } else {
      still.push_back(j);
    }
  }
  s->active.swap(still);
  std::lock_guard<std::mutex> lock(s->mu);
  s->n_active = (long)s->active.size();
  s->rounds++;
}

void serve(lbm_server *s) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv.wait(lock, [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
      if (s->stop) break;
    }
    admit(s);
    if (!s->active.empty()) round(s);
  }
  // stopped: jobs still running are cancelled
  for (auto &kv : s->groups) drop_group(kv.second);
  s->groups.clear();
  for (auto &j : s->active) retire(s, j, LBM_ERR_ARG);
  s->active.clear();
}

}  // namespace

extern "C" {

int lbm_server_create(const lbm_server_config_t *cfg, lbm_server_h *out) {
  if (!cfg || !out || cfg->max_active < 1 || cfg->chunk_steps < 1 || cfg->hbm_budget == 0)
    return LBM_ERR_ARG;
  *out = nullptr;
  lbm_server *s = new (std::nothrow) lbm_server();
  if (!s) return LBM_ERR_OOM;
  s->cfg = *cfg;
  if (cudaSetDevice(cfg->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return LBM_ERR_CUDA;
  }
  if (cudaMallocHost((void **)&s->h_status, sizeof(unsigned) * (size_t)cfg->max_active) !=
      cudaSuccess) {
    cudaStreamDestroy(s->stream);
    delete s;
    return LBM_ERR_OOM;
  }
  s->worker = std::thread(serve, s);
  *out = s;
  return LBM_OK;
}

int lbm_submit(lbm_server_h s, int nx, int ny, const lbm_params_t *p, const double *rho0,
               long nsteps, long *job_id) {
  if (!s || !p || nsteps < 0 || !job_id) return LBM_ERR_ARG;
  auto j = std::make_shared<Job>();
  j->nx = nx;
  j->ny = ny;
  j->p = *p;
  j->nsteps = nsteps;
  j->footprint = footprint_of(nx, ny, p->storage);
  if (j->footprint > s->cfg.hbm_budget) return LBM_ERR_BUSY;  // could never be admitted
  if (nx < 1 || ny < 1 || nx > (1 << 20) || ny > (1 << 20)) return LBM_ERR_ARG;
  if (rho0) j->rho0.assign(rho0, rho0 + (size_t)nx * ny);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return LBM_ERR_ARG;
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return LBM_OK;
}

int lbm_poll(lbm_server_h s, long job_id, int *state, double *rho, double *ux, double *uy,
             double *T, double *latency_s) {
  if (!s || !state) return LBM_ERR_ARG;
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return LBM_ERR_ARG;
    j = it->second;
    *state = j->state;
  }
  if (*state == LBM_JOB_DONE) {
    double *dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; k++)
      if (dst[k]) std::memcpy(dst[k], j->out[k].data(), j->out[k].size() * sizeof(double));
    if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  }
  return LBM_OK;
}

int lbm_wait(lbm_server_h s, long job_id, double timeout_s, int *state) {
  if (!s || !state) return LBM_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LBM_ERR_ARG;
  std::shared_ptr<Job> j = it->second;
  const bool ok = s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] {
    return j->state != LBM_JOB_QUEUED && j->state != LBM_JOB_RUNNING;
  });
  *state = j->state;
  return ok ? LBM_OK : LBM_ERR_TIMEOUT;
}

int lbm_server_stats(lbm_server_h s, lbm_server_stats_t *st) {
  if (!s || !st) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  st->queued = (long)s->queue.size();
  st->active = s->n_active;
  st->completed = s->completed;
  st->failed = s->failed;
  st->rounds = s->rounds;
  st->bytes_in_use = s->bytes_in_use;
  st->peak_bytes = s->peak_bytes;
  return LBM_OK;
}

void lbm_server_destroy(lbm_server_h s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (auto &j : s->queue) j->state = LBM_ERR_ARG;
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaStreamDestroy(s->stream);
  cudaFreeHost(s->h_status);
  delete s;
}

}  // extern "C"
