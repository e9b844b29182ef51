// stmg_server.cu -- continuous-batching request server for forward and adjoint solves.
//
// A fixed set of worker threads, each with its own CUDA stream, takes requests from one
// FIFO queue.  A request is admitted when its device footprint (stmg_footprint) fits in
// the memory budget next to the requests already running; requests that arrive while
// others run are admitted as workers and memory free up, and their kernels overlap on the
// GPU (one stream per worker).  All device memory comes from one arena allocated when the
// server starts, handed to the hierarchies through the allocator hooks of
// stmg_create_with_allocator, so admission is exact and no cudaMalloc / cudaFree (which
// can synchronise the device) runs while requests are being served.  Finished
// hierarchies stay resident in a cache and are reused (stmg_update_material) by later
// requests of the same grid and options; the cache is trimmed when memory is needed.
//
// Each result depends only on its own request: every kernel and reduction has a launch
// configuration fixed by the problem size, so a request gives the same bits alone and in
// any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "stmg.h"
#include "stmg_internal.h"

namespace {

// First-fit arena over one device allocation, 256-byte granularity, coalescing frees.
class Arena {
 public:
  cudaError_t init(size_t bytes) {
    size_ = bytes / 256 * 256;
    cudaError_t e = cudaMalloc(&base_, size_);
    if (e == cudaSuccess) free_[0] = size_;
    return e;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    std::lock_guard<std::mutex> g(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        in_use_ += bytes;
        peak_ = std::max(peak_, in_use_);
        return static_cast<char*>(base_) + off;
      }
    }
    return nullptr;
  }
  void release(void* p) {
    std::lock_guard<std::mutex> g(mu_);
    const size_t off = static_cast<char*>(p) - static_cast<char*>(base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    in_use_ -= len;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }
  size_t size() const { return size_; }
  size_t peak() {
    std::lock_guard<std::mutex> g(mu_);
    return peak_;
  }

 private:
  void* base_ = nullptr;
  size_t size_ = 0, in_use_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;            // offset -> length
  std::unordered_map<size_t, size_t> used_;  // offset -> length
  std::mutex mu_;
};

void* arena_alloc(size_t bytes, void* ctx) { return static_cast<Arena*>(ctx)->alloc(bytes); }
void arena_free(void* p, void* ctx) { static_cast<Arena*>(ctx)->release(p); }

struct Job {
  long long id = 0;
  int nel = 0, nt = 0;
  double L = 0, tT = 0;
  std::vector<double> k, c;
  const double* q = nullptr;
  double q_value = 0;
  int adjoint = 0;
  double* out = nullptr;
  stmg_opts opts{};
  std::string key;
  long long need = 0;
  stmg_result res{};
  bool done = false;
  bool alone = false;  // the arena could not place it next to others: run it on an emptied arena
};

struct Idle {
  std::string key;
  stmg_t h;
  long long bytes;
};

template <class T>
void append_field(std::string& k, const T& v) {
  k.append(reinterpret_cast<const char*>(&v), sizeof(v));
}

// Cache key of a request's hierarchy: the grid and every option field, one by one, so
// that the struct's padding bytes (whatever a caller left in them) never enter the key.
std::string job_key(const Job& j) {
  const stmg_opts& o = j.opts;
  std::string k;
  append_field(k, o.nu);
  append_field(k, o.omega);
  append_field(k, o.lambda_crit);
  append_field(k, o.interp);
  append_field(k, o.reassembly);
  append_field(k, o.min_nel);
  append_field(k, o.num_levels);
  append_field(k, o.max_levels);
  append_field(k, o.max_coarse_dofs);
  append_field(k, o.deff_fixed);
  append_field(k, o.precision);
  append_field(k, o.tol);
  append_field(k, o.div_tol);
  append_field(k, o.max_cycles);
  append_field(k, o.mixed_first_cycles);
  append_field(k, o.mixed_inner_cycles);
  append_field(k, j.nel);
  append_field(k, j.nt);
  append_field(k, j.L);
  append_field(k, j.tT);
  return k;
}

}  // namespace

struct stmg_server_s {
  stmg_server_opts o{};
  int device = 0;
  Arena arena;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<long long, std::unique_ptr<Job>> jobs;
  std::list<Idle> idle;  // least recently used first
  long long idle_bytes = 0, inflight = 0, next_id = 1;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> threads;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void destroy_idle(stmg_server_s* S, std::list<Idle>::iterator it) {
  stmg_destroy(it->h);
  S->idle_bytes -= it->bytes;
  S->idle.erase(it);
}

void worker_main(stmg_server_s* S, int w) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  const long long budget = (long long)S->arena.size();
  for (;;) {
    Job* job = nullptr;
    stmg_t h = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop && S->queue.empty()) break;
        if (!S->queue.empty()) {
          Job* head = S->queue.front();
          if (head->alone) {
            // its free bytes were split into pieces: wait until nothing runs, release the
            // cached hierarchies, and run it on the emptied arena
            if (S->running == 0) {
              while (!S->idle.empty()) destroy_idle(S, S->idle.begin());
              job = head;
              S->queue.pop_front();
              S->inflight += job->need;
              ++S->running;
              break;
            }
            S->cv_work.wait(lk);
            continue;
          }
          // reuse a resident hierarchy of the same grid and options if there is one
          for (auto it = S->idle.begin(); it != S->idle.end(); ++it)
            if (it->key == head->key) {
              h = it->h;
              S->idle_bytes -= it->bytes;
              S->idle.erase(it);
              break;
            }
          // trim the cache (least recently used first) until the request fits
          while (!h && S->inflight + S->idle_bytes + head->need > budget && !S->idle.empty())
            destroy_idle(S, S->idle.begin());
          if (h || S->inflight + S->idle_bytes + head->need <= budget) {
            job = head;
            S->queue.pop_front();
            S->inflight += job->need;
            ++S->running;
            break;
          }
          if (S->running == 0) {  // cannot fit even alone
            job = head;
            S->queue.pop_front();
            job->res.status = STMG_ENOMEM;
            job->res.t_start = job->res.t_end = S->now();
            job->done = true;
            S->cv_done.notify_all();
            job = nullptr;
            continue;
          }
        }
        S->cv_work.wait(lk);
      }
      if (!job) break;
    }
    job->res.t_start = S->now();
    job->res.worker = w;
    stmg_status st = STMG_OK;
    if (h) {
      st = stmg_set_stream(h, stream);
      if (st == STMG_OK) st = stmg_update_material(h, job->k.data(), job->c.data());
    } else {
      st = stmg_create_with_allocator(&h, job->nel, job->nt, job->L, job->tT, job->k.data(), job->c.data(), &job->opts,
                                      stream, arena_alloc, arena_free, &S->arena);
    }
    double* qdev = nullptr;
    if (st == STMG_OK && job->q) {
      // element loads staged through the arena for the duration of the solve
      const size_t nq = (size_t)(job->nt + 1) * job->nel * sizeof(double);
      qdev = static_cast<double*>(S->arena.alloc(nq));
      if (!qdev) st = STMG_ENOMEM;
      else if (cudaMemcpyAsync(qdev, job->q, nq, cudaMemcpyDefault, stream) != cudaSuccess) st = STMG_ECUDA;
    }
    const double scale = job->adjoint ? job->tT / job->nt : 1.0;
    if (st == STMG_OK)
      st = stmg_solve_resident(h, job->adjoint != 0, qdev, job->q_value, scale, job->out, &job->res.cycles,
                               &job->res.relres, &job->res.theta);
    // not converged: again with twice the smoothing sweeps, up to max_nu (a decision that
    // depends only on this request); the hierarchy is rebuilt with the new options, in the
    // memory the old one held (the footprint does not depend on nu)
    while ((st == STMG_EMAXITER || st == STMG_EDIVERGED) && S->o.max_nu > 0 && 2 * job->opts.nu <= S->o.max_nu) {
      stmg_destroy(h);
      h = nullptr;
      job->opts.nu *= 2;
      job->key = job_key(*job);
      st = stmg_create_with_allocator(&h, job->nel, job->nt, job->L, job->tT, job->k.data(), job->c.data(),
                                      &job->opts, stream, arena_alloc, arena_free, &S->arena);
      if (st == STMG_OK)
        st = stmg_solve_resident(h, job->adjoint != 0, qdev, job->q_value, scale, job->out, &job->res.cycles,
                                 &job->res.relres, &job->res.theta);
    }
    if (qdev) S->arena.release(qdev);
    if (st == STMG_ENOMEM && !job->alone) {
      // the free bytes did not hold it in one piece next to the others: back to the head of
      // the queue, to run once the running requests are done
      if (h) stmg_destroy(h);
      std::lock_guard<std::mutex> lk(S->mu);
      --S->running;
      S->inflight -= job->need;
      job->alone = true;
      S->queue.push_front(job);
      S->cv_work.notify_all();
      continue;
    }
    job->res.status = st;
    job->res.nu = job->opts.nu;
    job->res.bytes = h ? stmg_device_bytes(h) : 0;
    job->res.t_end = S->now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      --S->running;
      S->inflight -= job->need;
      if (h) {
        if (S->o.cache && (st == STMG_OK || st == STMG_EMAXITER || st == STMG_EDIVERGED)) {
          S->idle.push_back(Idle{job->key, h, stmg_device_bytes(h)});
          S->idle_bytes += S->idle.back().bytes;
        } else {
          stmg_destroy(h);
        }
      }
      job->done = true;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void stmg_server_default_opts(stmg_server_opts* o) {
  if (!o) return;
  o->workers = 4;
  o->budget_bytes = 0;
  o->cache = 1;
  o->max_nu = 0;
}

stmg_status stmg_server_create(stmg_server_t* out, const stmg_server_opts* opts) {
  if (!out) return STMG_EINVAL;
  *out = nullptr;
  stmg_server_opts o;
  if (opts) o = *opts;
  else stmg_server_default_opts(&o);
  if (o.workers < 1 || o.workers > 64 || o.budget_bytes < 0) {
    stmg::set_global_error("stmg_server_create: need 1 <= workers <= 64 and budget_bytes >= 0");
    return STMG_EINVAL;
  }
  auto* S = new (std::nothrow) stmg_server_s();
  if (!S) return STMG_ENOMEM;
  S->o = o;
  cudaGetDevice(&S->device);
  size_t freeb = 0, total = 0;
  cudaMemGetInfo(&freeb, &total);
  const size_t budget = o.budget_bytes > 0 ? (size_t)o.budget_bytes : freeb / 2;
  if (S->arena.init(budget) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    stmg::set_global_error("stmg_server_create: could not allocate the memory arena");
    return STMG_ENOMEM;
  }
  S->t0 = std::chrono::steady_clock::now();
  for (int w = 0; w < o.workers; ++w) S->threads.emplace_back(worker_main, S, w);
  *out = S;
  return STMG_OK;
}

double stmg_server_now(stmg_server_t S) { return S ? S->now() : 0.0; }

stmg_status stmg_server_submit(stmg_server_t S, const stmg_request* r, long long* ticket) {
  if (!S || !r || !ticket) return STMG_EINVAL;
  if (r->nel < 1 || r->nt < 1 || !r->k_el || !r->c_el) {
    stmg::set_global_error("stmg_server_submit: need nel, nt >= 1 and host k_el, c_el");
    return STMG_EINVAL;
  }
  auto job = std::make_unique<Job>();
  job->nel = r->nel;
  job->nt = r->nt;
  job->L = r->L;
  job->tT = r->t_end;
  job->k.assign(r->k_el, r->k_el + r->nel);
  job->c.assign(r->c_el, r->c_el + r->nel);
  job->q = r->q_el;
  job->q_value = r->q_value;
  job->adjoint = r->adjoint;
  job->out = r->out;
  job->opts = r->opts;
  job->need = stmg_footprint(r->nel, r->nt, r->L, r->t_end, r->k_el, r->c_el, &r->opts);
  if (job->need < 0) {
    stmg::set_global_error("stmg_server_submit: invalid problem definition");
    return STMG_EINVAL;
  }
  if (r->q_el) job->need += (long long)((size_t)(r->nt + 1) * r->nel * sizeof(double) + 255) / 256 * 256;
  job->key = job_key(*job);
  job->res.status = -1;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return STMG_EINVAL;
  job->id = S->next_id++;
  job->res.t_submit = S->now();
  *ticket = job->id;
  S->queue.push_back(job.get());
  S->jobs[job->id] = std::move(job);
  S->cv_work.notify_one();
  return STMG_OK;
}

stmg_status stmg_server_result(stmg_server_t S, long long ticket, int wait, stmg_result* out) {
  if (!S || !out) return STMG_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return STMG_EINVAL;
  Job* j = it->second.get();
  if (wait) S->cv_done.wait(lk, [&] { return j->done; });
  *out = j->res;
  if (!j->done) out->status = -1;
  return STMG_OK;
}

stmg_status stmg_server_drain(stmg_server_t S) {
  if (!S) return STMG_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] {
    if (!S->queue.empty() || S->running) return false;
    return true;
  });
  return STMG_OK;
}

long long stmg_server_peak_bytes(stmg_server_t S) { return S ? (long long)S->arena.peak() : 0; }

void stmg_server_destroy(stmg_server_t S) {
  if (!S) return;
  stmg_server_drain(S);
  {
    // cached hierarchies first, while the worker streams they last ran on still exist
    std::lock_guard<std::mutex> lk(S->mu);
    while (!S->idle.empty()) destroy_idle(S, S->idle.begin());
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->threads)
    if (t.joinable()) t.join();
  delete S;
}

}  // extern "C"
