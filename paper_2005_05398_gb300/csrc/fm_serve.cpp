// Request loop for independent problems: admission by device-memory budget, one context and
// one CUDA stream per running request, continuous refill of the slots as requests finish.
// The paper solves one problem at a time; this part has no counterpart there.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fm_internal.h"

namespace {

constexpr int kMaxBypass = 8;  // later requests may pass a waiting one at most this often

struct Pending {
  int64_t id = 0;
  fm_request r{};
  int64_t bytes = 0;
  double t_submit = 0.0;
  int bypassed = 0;
};

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

fm_opts request_opts(const fm_request& r, int device, void* stream) {
  fm_opts o;
  fm_default_opts(&o);
  o.precision = r.precision;
  o.restart_m = 40;
  o.ncv = 20;
  o.max_restarts = 8;  // bounded work per eigen-request; an unconverged one reports FM_ERR_NOT_CONVERGED
  o.device = device;
  o.stream = stream;
  return o;
}

// device bytes of a request: its context plus the vectors the server allocates for it
int request_bytes(const fm_request& r, int64_t* bytes, int64_t* n_out) {
  const fm_opts o = request_opts(r, 0, nullptr);
  int64_t b = 0;
  int rc = fm_estimate_bytes(&r.sys, &r.grid, 1, &r.split, &o, &b);
  if (rc) return rc;
  // unknowns: n_M * sum over the solved components of n_x n_y n_z
  const int M0 = (1 - r.sys.tau) / 2, nM = r.sys.J - M0 + 1;
  const int ncomp = (r.split.mode == FM_SPLIT_SCHRODINGER) ? 1 : (r.sys.identical_pair == 12 ? 2 : 3);
  const int64_t n = (int64_t)nM * ncomp * (2 * r.grid.nint_x) * (2 * r.grid.nint_y) * (2 * r.grid.nint_z + 2);
  const int64_t vec = (r.kind == FM_REQ_SOLVE) ? 2 : 1 + (r.out_host ? r.k : 0);
  *bytes = b + vec * n * 8;
  *n_out = n;
  return FM_OK;
}

}  // namespace

struct fm_server {
  int device = 0;
  int64_t budget = 0;
  int flags = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::map<int64_t, fm_result> done;
  std::map<int64_t, bool> known;   // submitted and not yet collected
  int64_t next_id = 1, in_use = 0, peak_in_use = 0;
  int busy = 0, peak_busy = 0;
  bool stop = false;
  std::vector<std::thread> workers;

  // Under the lock: the first waiting request (in arrival order) that fits next to the running
  // ones; a request passed over kMaxBypass times stops the scan until it fits itself.
  bool pick(Pending* out) {
    for (size_t i = 0; i < queue.size(); ++i) {
      if (queue[i].bytes <= budget - in_use) {
        for (size_t q = 0; q < i; ++q) ++queue[q].bypassed;
        *out = queue[i];
        queue.erase(queue.begin() + (long)i);
        return true;
      }
      if (queue[i].bypassed >= kMaxBypass) return false;
    }
    return false;
  }

  void run(const Pending& p, cudaStream_t stream, fm_result* res) {
    const fm_request& r = p.r;
    if (flags & FM_SERVER_DRY_RUN) {
      std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(std::max(0.0, r.sim_ms)));
      res->status = FM_OK;
      return;
    }
    fm_opts o = request_opts(r, device, stream);
    fm_ctx* c = nullptr;
    double* b = nullptr;
    double* x = nullptr;
    int rc = fm_create(&r.sys, &r.grid, 1, &r.split, &o, &c);
    if (rc == FM_OK) {
      const int64_t n = c->N;
      res->n = n;
      const int nvec = (r.kind == FM_REQ_SOLVE) ? 1 : r.k;
      // stream-ordered on the slot's stream: allocating and releasing them does not synchronise the device,
      // so the other slots' kernels keep running
      if (cudaMallocAsync((void**)&b, n * 8, stream) != cudaSuccess ||
          cudaMallocAsync((void**)&x, (size_t)n * 8 * ((r.kind == FM_REQ_EIGS && !r.out_host) ? 1 : nvec), stream) !=
              cudaSuccess) {
        cudaGetLastError();
        rc = FM_ERR_OOM;
      }
      if (rc == FM_OK) rc = fmi::fill_normal(c, b, r.seed);
      fm_info info{};
      if (rc == FM_OK && r.kind == FM_REQ_SOLVE) {
        if (cudaMemsetAsync(x, 0, n * 8, stream) != cudaSuccess) rc = FM_ERR_CUDA;
        if (rc == FM_OK) rc = fm_solve(c, r.E, b, x, &info);
        if (rc == FM_OK || rc == FM_ERR_NOT_CONVERGED) {
          double h = 0.0;
          const int rc2 = fmi::dot_many(c, x, n, 1, x, &h);
          res->out_norm = std::sqrt(std::max(h, 0.0));
          if (rc2) rc = rc2;
        }
      } else if (rc == FM_OK) {
        rc = fm_eigs(c, r.E, r.k, b, res->evals, r.out_host ? x : nullptr, &info);
        res->out_norm = 1.0;
      }
      res->iters = info.iters;
      res->resid = info.resid;
      if ((rc == FM_OK || rc == FM_ERR_NOT_CONVERGED) && r.out_host) {
        if (cudaMemcpyAsync(r.out_host, x, (size_t)n * 8 * nvec, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
          rc = FM_ERR_CUDA;
      }
    }
    if (b) cudaFreeAsync(b, stream);
    if (x) cudaFreeAsync(x, stream);
    if (c) fm_destroy(c);  // synchronises the slot's stream, after which b and x are back in the pool
    res->status = rc;
  }

  void worker() {
    cudaStream_t stream = nullptr;
    if (!(flags & FM_SERVER_DRY_RUN)) {
      cudaSetDevice(device);
      cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    }
    while (true) {
      Pending p;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return (stop && queue.empty()) || pick(&p); });
        if (p.id == 0) break;  // stopping and nothing left
        in_use += p.bytes;
        ++busy;
        peak_in_use = std::max(peak_in_use, in_use);
        peak_busy = std::max(peak_busy, busy);
      }
      fm_result res{};
      res.bytes = p.bytes;
      res.t_submit_ms = p.t_submit;
      res.t_start_ms = now_ms(t0);
      run(p, stream, &res);
      res.t_end_ms = now_ms(t0);
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= p.bytes;
        --busy;
        done[p.id] = res;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (stream) cudaStreamDestroy(stream);
  }
};

extern "C" {

int fm_server_create(int device, int64_t hbm_budget, int slots, int flags, fm_server** out) {
  if (!out) return FM_ERR_ARG;
  *out = nullptr;
  if (slots < 1 || slots > 64 || (flags & ~FM_SERVER_DRY_RUN)) return FM_ERR_ARG;
  if ((flags & FM_SERVER_DRY_RUN) && hbm_budget <= 0) return FM_ERR_ARG;
  if (!(flags & FM_SERVER_DRY_RUN) && hbm_budget <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) return FM_ERR_CUDA;
    // what is free now (another allocator in the process may hold part of the device), less a margin of
    // 5 % of the device for the CUDA context, the library's module and allocator slack
    hbm_budget = (int64_t)fr - (int64_t)(0.05 * (double)tot);
    if (hbm_budget <= 0) return FM_ERR_OOM;
  }
  fm_server* s = new fm_server();
  s->device = device;
  s->budget = hbm_budget;
  s->flags = flags;
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < slots; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return FM_OK;
}

int fm_server_submit(fm_server* s, const fm_request* r, int64_t* id) {
  if (!s || !r || !id) return FM_ERR_ARG;
  if (r->kind != FM_REQ_SOLVE && r->kind != FM_REQ_EIGS) return FM_ERR_ARG;
  if (r->kind == FM_REQ_EIGS && (r->k < 1 || r->k > 8)) return FM_ERR_ARG;
  if (!std::isfinite(r->E) || r->precision < 0 || r->precision > 2) return FM_ERR_ARG;
  Pending p;
  p.r = *r;
  int64_t n = 0;
  int rc = request_bytes(*r, &p.bytes, &n);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return FM_ERR_ARG;
  if (p.bytes > s->budget) return FM_ERR_OOM;
  p.id = s->next_id++;
  p.t_submit = now_ms(s->t0);
  s->queue.push_back(p);
  s->known[p.id] = true;
  *id = p.id;
  s->cv_work.notify_all();
  return FM_OK;
}

int fm_server_wait(fm_server* s, int64_t id, double timeout_ms, fm_result* out) {
  if (!s || !out) return FM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->known.count(id)) return FM_ERR_ARG;
  auto ready = [&] { return s->done.count(id) > 0; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
    return FM_ERR_TIMEOUT;
  }
  *out = s->done[id];
  s->done.erase(id);
  s->known.erase(id);
  return FM_OK;
}

int fm_server_stats(fm_server* s, int64_t* in_use, int64_t* peak_in_use, int* busy, int* peak_busy, int* queued) {
  if (!s) return FM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (in_use) *in_use = s->in_use;
  if (peak_in_use) *peak_in_use = s->peak_in_use;
  if (busy) *busy = s->busy;
  if (peak_busy) *peak_busy = s->peak_busy;
  if (queued) *queued = (int)s->queue.size();
  return FM_OK;
}

void fm_server_destroy(fm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
