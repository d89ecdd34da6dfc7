// server.cpp -- serving loop of include/cdcc.h: continuous batching of
// gradient jobs of mixed sizes and point groups on one GPU.
//
// A dispatcher thread admits queued jobs (first come first served, look-ahead
// of four past the head) when a worker slot is free and the job's estimated
// peak device footprint fits the budget not yet promised to running jobs (or
// nothing else runs).  Each of the max_active workers owns a CUDA stream and
// drives one admitted job at a time to its gradient: the job's context keeps
// amplitudes, Lambda, DIIS histories and intermediates resident on the
// device, and the kernels of concurrently admitted jobs overlap on the GPU.
// A job whose device allocation fails is put back at the head of the queue
// and retried when it can run alone.  The ladder mode of a job is chosen
// from its size only, so its result is the same alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cdcc.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

int64_t pairs(const std::vector<int>& a, const std::vector<int>& b, int h,
              int gamma) {
  int64_t s = 0;
  for (int g = 0; g < h; ++g) s += (int64_t)a[g] * b[g ^ gamma];
  return s;
}

struct Job {
  uint64_t ticket = 0;
  // owned copies of the inputs
  int nirrep = 0, nocc = 0, nvir = 0, nchol = 0, nx = 0;
  std::vector<int32_t> orb_irrep, chol_irrep, x_irrep;
  std::vector<double> eps, L, dL;
  bool has_xirrep = false;
  // scheduling
  int state = CDCC_JOB_QUEUED;
  int status = CDCC_OK;
  int ladder = CDCC_LADDER_OTF;
  int retries = 0;
  size_t est_bytes = 0;
  Clock::time_point t_submit, t_admit;
  double t_wait = 0, t_run = 0;
  // results
  double e_corr = 0, err_dE = 0;
  std::vector<double> g;
  std::string message;

  cdcc_job_desc desc() const {
    cdcc_job_desc d;
    d.nirrep = nirrep;
    d.nocc = nocc;
    d.nvir = nvir;
    d.nchol = nchol;
    d.orb_irrep = orb_irrep.data();
    d.eps = eps.data();
    d.chol_irrep = chol_irrep.data();
    d.L = L.data();
    d.nx = nx;
    d.x_irrep = has_xirrep ? x_irrep.data() : nullptr;
    d.dL = dL.empty() ? nullptr : dL.data();
    return d;
  }
};

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
bool copy_in(std::vector<T>& dst, const T* src, size_t n) {
  dst.resize(n);
  if (n == 0) return true;
  if (is_device(src))
    return cudaMemcpy(dst.data(), src, n * sizeof(T),
                      cudaMemcpyDeviceToHost) == cudaSuccess;
  std::memcpy(dst.data(), src, n * sizeof(T));
  return true;
}

// per-irrep orbital and Cholesky counts of a job (labels validated)
bool counts(const cdcc_job_desc& j, std::vector<int>& o, std::vector<int>& v,
            std::vector<int>& q) {
  const int h = j.nirrep;
  if (!(h == 1 || h == 2 || h == 4 || h == 8)) return false;
  o.assign(h, 0);
  v.assign(h, 0);
  q.assign(h, 0);
  for (int p = 0; p < j.nocc + j.nvir; ++p) {
    const int g = j.orb_irrep[p];
    if (g < 0 || g >= h) return false;
    (p < j.nocc ? o : v)[g]++;
  }
  for (int P = 0; P < j.nchol; ++P) {
    const int g = j.chol_irrep[P];
    if (g < 0 || g >= h) return false;
    q[g]++;
  }
  return true;
}

size_t packed_size(const std::vector<int>& n, const std::vector<int>& q,
                   int h, int gx) {
  size_t s = 0;
  for (int gP = 0; gP < h; ++gP) s += (size_t)q[gP] * pairs(n, n, h, gP ^ gx);
  return s;
}

// Element counts of the large device arrays of one job and an upper
// estimate of its peak device memory.  About 64 doubles-sized arrays
// (amplitudes, residuals, multipliers, two DIIS histories, the recorded
// residual intermediates and their adjoints), (mc|bd) with its adjoint and
// slices, L in its blocks with adjoint and slices, the permuted copies of
// the constant tensors with their slices (about eight copies of o^2 v^2
// size, 20 bytes per element, at most 2.5 x the cache budget), plus the
// ladder: stored integrals with their adjoint and slices (16 / 28 / 36
// bytes per element for FP64 / MIXED / TC), or on the fly two batch
// buffers, the batch slices and the adjoint batch slices of the density
// sweep (measured peaks stay below five batches) plus the batch slices
// kept across applications (4 bytes per element, within their budget).
struct Footprint {
  int64_t t2 = 0, w = 0, ovvv = 0, nnz = 0;
  size_t bytes = 0, ladder_bytes = 0;
};

// canonical virtual pairs of pair irrep G (irrep(c) > irrep(d), or the same
// irrep and c >= d): the columns of the +/- packed ladder
int64_t canonical_pairs(const std::vector<int>& v, int h, int G) {
  int64_t s = 0;
  for (int g = 0; g < h; ++g) {
    const int g2 = g ^ G;
    if (g > g2) s += (int64_t)v[g] * v[g2];
    if (g == g2) s += (int64_t)v[g] * (v[g] + 1) / 2;
  }
  return s;
}

Footprint footprint(const cdcc_job_desc& j, int precision, int ladder,
                    double batch_gb, double perm_gb, double slices_gb,
                    bool pm) {
  Footprint f;
  std::vector<int> o, v, q;
  if (!counts(j, o, v, q)) return f;
  const int h = j.nirrep;
  std::vector<int> n(h);
  for (int g = 0; g < h; ++g) n[g] = o[g] + v[g];
  int64_t wpm = 0;   // W+ and W- elements of the +/- ladder
  for (int G = 0; G < h; ++G) {
    const int64_t u = canonical_pairs(v, h, G);
    wpm += 2 * u * u;
    f.t2 += pairs(o, o, h, G) * pairs(v, v, h, G);
    f.w += pairs(v, v, h, G) * pairs(v, v, h, G);
    f.ovvv += pairs(o, v, h, G) * pairs(v, v, h, G);
    f.nnz += (int64_t)q[G] * pairs(n, n, h, G);
  }
  const double perm =
      perm_gb > 0 ? std::min(8.0 * 20.0 * (double)f.t2, 2.5e9 * perm_gb)
                  : 0.0;
  const double base = 8.0 * (64.0 * f.t2 + 4.0 * f.ovvv + 10.0 * f.nnz) +
                      perm + (512 << 20);
  double lad;
  if (ladder == CDCC_LADDER_STORED) {
    const double k = precision == CDCC_PREC_TC      ? 4.5
                     : precision == CDCC_PREC_MIXED ? 3.5
                                                    : 2.0;
    lad = 8.0 * (double)f.w * k;
  } else {
    lad = 5.5 * batch_gb * 1e9;
    // BF16 batch slices kept across applications (two slices, float
    // schedules only): of the (ab|cd) rows, or of W+ and W- when packed
    if (precision != CDCC_PREC_FP64 && slices_gb > 0)
      lad += std::min(4.0 * (double)(pm ? wpm : f.w), slices_gb * 1e9);
  }
  f.ladder_bytes = (size_t)lad;
  f.bytes = (size_t)(base + lad);
  return f;
}

}  // namespace

struct cdcc_server {
  cdcc_options opt;
  cdcc_server_options sopt;
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_sched;   // dispatcher: something changed
  std::condition_variable cv_done;    // waiters: a job finished
  std::vector<std::condition_variable> cv_slot;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::deque<std::shared_ptr<Job>> queue;
  std::vector<std::shared_ptr<Job>> slot_job;   // job assigned to each slot
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  std::thread dispatcher;
  size_t committed = 0;
  int active = 0, max_seen = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  Clock::time_point t0 = Clock::now();

  explicit cdcc_server(int nslots) : cv_slot(nslots) {}

  void dispatch_loop();
  void worker_loop(int slot);
  int execute(Job& j, int slot);
};

namespace {

// Library executor: one gradient through the C ABI on the slot's stream,
// then the energy error report.
int library_execute(cdcc_server* s, Job& j, int slot) {
  cdcc_options o = s->opt;
  o.stream = (void*)s->streams[slot];
  o.dev_alloc = nullptr;
  o.dev_free = nullptr;
  o.alloc_user = nullptr;
  o.ladder = j.ladder;
  cdcc_ctx* ctx = nullptr;
  int st = cd_ccsd_init(&ctx, j.nirrep, j.nocc, j.nvir, j.nchol,
                        j.orb_irrep.data(), j.eps.data(), j.chol_irrep.data(),
                        j.L.data(), &o);
  if (st == CDCC_OK) {
    j.g.assign(j.nx, 0.0);
    st = gradient(ctx, j.nx, j.has_xirrep ? j.x_irrep.data() : nullptr,
                  j.dL.empty() ? nullptr : j.dL.data(), &j.e_corr,
                  j.g.data());
  }
  if (st == CDCC_OK && s->sopt.error_report)
    st = cdcc_energy_error(ctx, &j.err_dE);
  if (st != CDCC_OK && ctx) j.message = cdcc_last_error(ctx);
  if (ctx) cd_ccsd_free(ctx);
  return st;
}

}  // namespace

int cdcc_server::execute(Job& j, int slot) {
  if (sopt.executor) {
    const cdcc_job_desc d = j.desc();
    j.g.assign(j.nx, 0.0);
    return sopt.executor(j.ticket, &d, slot, &j.e_corr, j.g.data(),
                         &j.err_dE, sopt.executor_user);
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    (void)cudaGetLastError();
    j.message = "cudaSetDevice failed";
    return CDCC_ECUDA;
  }
  return library_execute(this, j, slot);
}

void cdcc_server::worker_loop(int slot) {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_slot[slot].wait(lk, [&] { return slot_job[slot] || stopping; });
    if (!slot_job[slot]) return;          // stopping with nothing assigned
    std::shared_ptr<Job> j = slot_job[slot];
    lk.unlock();
    int st;
    try {
      st = execute(*j, slot);
    } catch (...) {
      st = CDCC_EINVAL;
      j->message = "host exception in the executor";
    }
    lk.lock();
    slot_job[slot].reset();
    --active;
    committed -= std::min(committed, j->est_bytes);
    if (st == CDCC_ENOMEM && j->retries < 3 && !stopping) {
      // the estimate was low: retry alone, at the head of the queue
      ++j->retries;
      j->state = CDCC_JOB_QUEUED;
      queue.push_front(j);
    } else {
      j->status = st;
      j->state = st == CDCC_OK ? CDCC_JOB_DONE : CDCC_JOB_FAILED;
      if (st == CDCC_ENOMEM) j->message = "out of device memory";
      j->t_run = seconds_since(j->t_admit);
      // the inputs are no longer needed
      std::vector<double>().swap(j->L);
      std::vector<double>().swap(j->dL);
      cv_done.notify_all();
    }
    cv_sched.notify_all();
  }
}

void cdcc_server::dispatch_loop() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool admitted = true;
    while (admitted && !stopping && !queue.empty()) {
      admitted = false;
      int free_slot = -1;
      for (int s = 0; s < (int)slot_job.size(); ++s)
        if (!slot_job[s]) {
          free_slot = s;
          break;
        }
      if (free_slot < 0) break;
      const int look = std::min<int>((int)queue.size(), 4);
      for (int k = 0; k < look; ++k) {
        std::shared_ptr<Job> j = queue[k];
        if (j->retries > 0 && active > 0) break;   // a retry runs alone
        const bool fits = committed + j->est_bytes <= budget;
        if (!(fits || active == 0)) continue;
        queue.erase(queue.begin() + k);
        j->state = CDCC_JOB_RUNNING;
        j->t_admit = Clock::now();
        j->t_wait = std::chrono::duration<double>(j->t_admit - j->t_submit)
                        .count();
        committed += j->est_bytes;
        ++active;
        max_seen = std::max(max_seen, active);
        slot_job[free_slot] = j;
        cv_slot[free_slot].notify_one();
        admitted = true;
        break;
      }
    }
    if (stopping && active == 0) return;
    cv_sched.wait(lk);
  }
}

extern "C" {

void cdcc_server_default_options(cdcc_server_options* s) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->max_active = 4;
  s->budget_gb = 0.0;
  s->reserve_gb = 8.0;
  s->stored_max_gb = 24.0;
  s->error_report = 1;
}

size_t cdcc_job_footprint(const cdcc_job_desc* job, int precision, int ladder,
                          double batch_gb) {
  if (!job || !job->orb_irrep || !job->chol_irrep) return 0;
  cdcc_options d;
  cdcc_default_options(&d);
  return footprint(*job, precision, ladder, batch_gb, d.perm_cache_gb,
                   d.ladder_slices_gb, d.ladder_pm != 0)
      .bytes;
}

cdcc_status cdcc_server_create(cdcc_server** out, const cdcc_options* opt,
                               const cdcc_server_options* sopt) {
  if (!out) return CDCC_EINVAL;
  *out = nullptr;
  cdcc_server_options so;
  if (sopt)
    so = *sopt;
  else
    cdcc_server_default_options(&so);
  if (so.max_active < 1 || so.max_active > 64) return CDCC_EINVAL;
  std::unique_ptr<cdcc_server> s(new (std::nothrow)
                                     cdcc_server(so.max_active));
  if (!s) return CDCC_ENOMEM;
  if (opt)
    s->opt = *opt;
  else
    cdcc_default_options(&s->opt);
  s->sopt = so;
  s->device = s->opt.device;
  s->slot_job.resize(so.max_active);
  if (so.budget_gb > 0) {
    s->budget = (size_t)(so.budget_gb * 1e9);
  } else if (!so.executor) {
    size_t fre = 0, tot = 0;
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaMemGetInfo(&fre, &tot) != cudaSuccess) {
      (void)cudaGetLastError();
      return CDCC_ECUDA;
    }
    const size_t res = (size_t)(so.reserve_gb * 1e9);
    s->budget = fre > res ? fre - res : 0;
  } else {
    s->budget = (size_t)-1;
  }
  if (!so.executor) {
    if (cudaSetDevice(s->device) != cudaSuccess) {
      (void)cudaGetLastError();
      return CDCC_ECUDA;
    }
    for (int k = 0; k < so.max_active; ++k) {
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) !=
          cudaSuccess) {
        (void)cudaGetLastError();
        for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
        return CDCC_ECUDA;
      }
      s->streams.push_back(st);
    }
  }
  cdcc_server* raw = s.get();
  for (int k = 0; k < so.max_active; ++k)
    s->workers.emplace_back([raw, k] { raw->worker_loop(k); });
  s->dispatcher = std::thread([raw] { raw->dispatch_loop(); });
  *out = s.release();
  return CDCC_OK;
}

cdcc_status cdcc_submit(cdcc_server* s, const cdcc_job_desc* d,
                        uint64_t* ticket) {
  if (!s || !d || !ticket) return CDCC_EINVAL;
  if (d->nocc < 1 || d->nvir < 1 || d->nchol < 1 || d->nx < 0 ||
      !d->orb_irrep || !d->eps || !d->chol_irrep || !d->L ||
      (d->nx > 0 && !d->dL))
    return CDCC_EINVAL;
  auto j = std::make_shared<Job>();
  j->nirrep = d->nirrep;
  j->nocc = d->nocc;
  j->nvir = d->nvir;
  j->nchol = d->nchol;
  j->nx = d->nx;
  const int n = d->nocc + d->nvir;
  if (!copy_in(j->orb_irrep, d->orb_irrep, n) ||
      !copy_in(j->chol_irrep, d->chol_irrep, d->nchol) ||
      !copy_in(j->eps, d->eps, n))
    return CDCC_ECUDA;
  std::vector<int> o, v, q;
  cdcc_job_desc tmp = j->desc();
  if (!counts(tmp, o, v, q)) return CDCC_EINVAL;
  std::vector<int> nn(d->nirrep);
  for (int g = 0; g < d->nirrep; ++g) nn[g] = o[g] + v[g];
  if (d->x_irrep) {
    if (!copy_in(j->x_irrep, d->x_irrep, d->nx)) return CDCC_ECUDA;
    j->has_xirrep = true;
    for (int x = 0; x < d->nx; ++x)
      if (j->x_irrep[x] < 0 || j->x_irrep[x] >= d->nirrep)
        return CDCC_EINVAL;
  }
  size_t ndl = 0;
  for (int x = 0; x < d->nx; ++x)
    ndl += packed_size(nn, q, d->nirrep, j->has_xirrep ? j->x_irrep[x] : 0);
  if (!copy_in(j->L, d->L, packed_size(nn, q, d->nirrep, 0)) ||
      !copy_in(j->dL, d->dL, ndl))
    return CDCC_ECUDA;
  // ladder mode from the job's size only
  const Footprint fs =
      footprint(j->desc(), s->opt.precision, CDCC_LADDER_STORED, 0.0,
                s->opt.perm_cache_gb, s->opt.ladder_slices_gb,
                s->opt.ladder_pm != 0);
  j->ladder = (double)fs.ladder_bytes <= s->sopt.stored_max_gb * 1e9
                  ? CDCC_LADDER_STORED
                  : CDCC_LADDER_OTF;
  if (s->opt.ladder == CDCC_LADDER_STORED || s->opt.ladder == CDCC_LADDER_OTF)
    j->ladder = s->opt.ladder;
  const double bgb = s->opt.ladder_batch_gb > 0 ? s->opt.ladder_batch_gb : 2.0;
  j->est_bytes = footprint(j->desc(), s->opt.precision, j->ladder, bgb,
                           s->opt.perm_cache_gb, s->opt.ladder_slices_gb,
                           s->opt.ladder_pm != 0)
                     .bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return CDCC_ESTATE;
  j->ticket = s->next_ticket++;
  j->t_submit = Clock::now();
  s->jobs[j->ticket] = j;
  s->queue.push_back(j);
  *ticket = j->ticket;
  s->cv_sched.notify_all();
  return CDCC_OK;
}

static void fill_result(const Job& j, cdcc_result* r) {
  double* g = r->g;
  std::memset(r, 0, sizeof(*r));
  r->g = g;
  r->state = j.state;
  r->status = j.status;
  r->nx = j.nx;
  r->ladder = j.ladder;
  r->retries = j.retries;
  r->t_wait = j.t_wait;
  if (j.state == CDCC_JOB_DONE || j.state == CDCC_JOB_FAILED) {
    r->t_run = j.t_run;
    std::strncpy(r->message, j.message.c_str(), sizeof(r->message) - 1);
  }
  if (j.state == CDCC_JOB_DONE) {
    r->e_corr = j.e_corr;
    r->err_dE = j.err_dE;
    if (g && j.nx > 0) std::memcpy(g, j.g.data(), (size_t)j.nx * 8);
  }
}

cdcc_status cdcc_poll(cdcc_server* s, uint64_t ticket, cdcc_result* res) {
  if (!s || !res) return CDCC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return CDCC_EINVAL;
  fill_result(*it->second, res);
  return CDCC_OK;
}

cdcc_status cdcc_wait(cdcc_server* s, uint64_t ticket, double timeout_s,
                      cdcc_result* res) {
  if (!s || !res) return CDCC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return CDCC_EINVAL;
  std::shared_ptr<Job> j = it->second;
  const auto done = [&] {
    return j->state == CDCC_JOB_DONE || j->state == CDCC_JOB_FAILED;
  };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(
                 lk, std::chrono::duration<double>(timeout_s), done)) {
    fill_result(*j, res);
    return CDCC_ETIMEOUT;
  }
  fill_result(*j, res);
  return CDCC_OK;
}

int cdcc_server_max_active_seen(const cdcc_server* s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(const_cast<cdcc_server*>(s)->mu);
  return s->max_seen;
}

void cdcc_server_destroy(cdcc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (auto& j : s->queue) {
      j->state = CDCC_JOB_FAILED;
      j->status = CDCC_ESTATE;
      j->message = "server shut down before the job started";
    }
    s->queue.clear();
    s->cv_sched.notify_all();
    for (auto& c : s->cv_slot) c.notify_all();
    s->cv_done.notify_all();
  }
  s->dispatcher.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& c : s->cv_slot) c.notify_all();
  }
  for (auto& w : s->workers) w.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete s;
}

}  // extern "C"
