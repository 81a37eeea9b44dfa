// Serving runtime: continuous batching of solve requests over a pool of CUDA streams.
//
// Requests of the same shape (d, p, n) share a cached solver handle (a "bucket") whose
// max_batch right-hand-side slots run as a session: every slot follows the refinement loop on
// its own schedule, one chunk of Krylov iterations per step.  A pool of worker threads picks the
// bucket that is due (its last step, or its oldest pending request, is oldest), admits pending
// requests of that shape into free slots (all right-hand sides of a request together,
// parameters may differ per right-hand side), runs one step on the bucket's stream and hands
// back the slots that finished.  So requests join and leave between chunks of iterations while
// the bucket's other solves keep running, and buckets of different shapes step concurrently.
// A new bucket is admitted only when its device footprint fits in the HBM budget, evicting idle
// buckets (least recently used) if needed.  Every kernel is masked per slot and every reduction
// has a fixed order per slot, so a request's result does not depend on what else runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "cd_internal.h"

namespace cd {
size_t solver_bytes(int d, int p, int n, const cd_options& opt);
}

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t id = 0;
  int d = 0, p = 0, n = 0, nrhs = 0;
  std::vector<double> alpha, beta, b, x;
  std::vector<cd_result> res;
  cd_status status = CD_OK;
  bool done = false, cancelled = false;
  int remaining = 0;  // right-hand sides still in session slots
  Clock::time_point t_submit, t_done;
};

struct Bucket {
  int d = 0, p = 0, n = 0;
  cd_solver h = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  bool running = false;
  std::deque<uint64_t> pending;
  Clock::time_point last_used;
  // session slots of the bucket's handle: owner request and right-hand side index
  std::vector<std::pair<uint64_t, int>> owner;
  int busy = 0;
  // a bucket without a solver whose admission found no room is skipped until then, so that the
  // buckets holding memory keep stepping and can finish
  Clock::time_point blocked_until{};
};

}  // namespace

// A request gets back the FP64 vector x, not the refinement's x + x_lo; the residual of x exceeds
// that of x + x_lo by the rounding of x (about eps |A| |x|), which at beta/alpha near 1e+-6 is a
// sizeable part of 1e-10.  The sessions therefore refine to kReturnMargin times the requested
// tolerance, and a request's status is judged on the returned x against the requested one.
static constexpr double kReturnMargin = 0.5;

struct cd_server_s {
  cd_server_options opt{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<std::tuple<int, int, int>, Bucket> buckets;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1;
  size_t mem_used = 0;
  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, solves = 0, slot_steps = 0;
  std::vector<double> latencies;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;

  void worker_loop();
};

namespace {

static double seconds_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

// Finishes a request (under the server lock).
static void finish(cd_server_s* S, Request& r, cd_status st) {
  r.status = st;
  r.done = true;
  r.t_done = Clock::now();
  S->t_last_done = r.t_done;
  if (st == CD_OK) {
    S->completed += 1;
    S->latencies.push_back(seconds_between(r.t_submit, r.t_done));
  } else {
    S->failed += 1;
  }
}

}  // namespace

void cd_server_s::worker_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    if (stop) return;
    // the idle bucket whose oldest pending request is oldest
    Bucket* pick = nullptr;
    Clock::time_point oldest = Clock::time_point::max();
    const auto now = Clock::now();
    for (auto& kv : buckets) {
      Bucket& bk = kv.second;
      // drop cancelled and timed-out requests from the queue
      while (!bk.pending.empty()) {
        auto it = reqs.find(bk.pending.front());
        if (it == reqs.end() || it->second->done) {
          bk.pending.pop_front();
          continue;
        }
        Request& r = *it->second;
        if (opt.timeout_s > 0 && seconds_between(r.t_submit, now) > opt.timeout_s) {
          finish(this, r, CD_TIMEOUT);
          bk.pending.pop_front();
          cv_done.notify_all();
          continue;
        }
        break;
      }
      if (bk.running || (bk.pending.empty() && bk.busy == 0)) continue;
      if (!bk.h && now < bk.blocked_until) continue;
      // a bucket with solves in flight is due by its last step, one with only pending
      // requests by its oldest request
      const Clock::time_point due = bk.busy > 0 ? bk.last_used : reqs[bk.pending.front()]->t_submit;
      if (due < oldest) {
        oldest = due;
        pick = &bk;
      }
    }
    if (!pick) {
      cv_work.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    Bucket& bk = *pick;
    // admission: make room for the bucket's solver within the HBM budget
    if (!bk.h) {
      cd_options so = opt.solve;
      so.max_batch = opt.max_batch;
      so.rtol = opt.solve.rtol * kReturnMargin;
      const size_t need = cd::solver_bytes(bk.d, bk.p, bk.n, so);
      if (need > opt.hbm_budget) {
        for (uint64_t id : bk.pending) finish(this, *reqs[id], CD_ENOMEM);
        bk.pending.clear();
        cv_done.notify_all();
        continue;
      }
      while (mem_used + need > opt.hbm_budget) {
        Bucket* lru = nullptr;
        for (auto& kv : buckets) {
          Bucket& o = kv.second;
          if (o.h && !o.running && o.pending.empty() && o.busy == 0 &&
              (!lru || o.last_used < lru->last_used))
            lru = &o;
        }
        if (!lru) break;
        cd_solver hv = lru->h;
        cudaStream_t sv = lru->stream;
        mem_used -= lru->bytes;
        lru->h = nullptr;
        lru->stream = nullptr;
        lru->bytes = 0;
        lk.unlock();
        cd_destroy(hv);
        cudaStreamDestroy(sv);
        lk.lock();
      }
      if (mem_used + need > opt.hbm_budget) {  // the solvers in use must finish first
        bk.blocked_until = Clock::now() + std::chrono::milliseconds(20);
        continue;
      }
      bk.running = true;
      mem_used += need;
      lk.unlock();
      cudaStream_t st = nullptr;
      cd_solver h = nullptr;
      cd_status cs = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess
                         ? cd_create(&h, bk.d, bk.p, bk.n, 1.0, 1.0, &so, st)
                         : CD_ECUDA;
      lk.lock();
      bk.running = false;
      if (cs != CD_OK) {
        mem_used -= need;
        if (st) cudaStreamDestroy(st);
        for (uint64_t id : bk.pending) finish(this, *reqs[id], cs);
        bk.pending.clear();
        cv_done.notify_all();
        continue;
      }
      bk.h = h;
      bk.stream = st;
      bk.bytes = need;
    }
    // admission into free session slots (every right-hand side of a request at once, in arrival
    // order), then one step of the bucket's session: slots join and leave between chunks of
    // Krylov iterations, so a request does not wait for the solves already running
    if (bk.owner.empty()) bk.owner.assign(opt.max_batch, std::make_pair(uint64_t(0), -1));
    std::vector<std::pair<Request*, int>> admit;
    int free_slots = opt.max_batch - bk.busy;
    while (!bk.pending.empty()) {
      Request* r = reqs[bk.pending.front()].get();
      if (r->nrhs > free_slots) break;
      for (int i = 0; i < r->nrhs; ++i) admit.push_back(std::make_pair(r, i));
      free_slots -= r->nrhs;
      r->remaining = r->nrhs;
      r->x.assign((size_t)r->nrhs * cd_dofs(bk.d, bk.p, bk.n), 0.0);
      r->res.assign(r->nrhs, cd_result{});
      bk.pending.pop_front();
    }
    bk.busy += (int)admit.size();
    bk.running = true;
    cd_solver h = bk.h;
    const size_t N = cd_dofs(bk.d, bk.p, bk.n);
    lk.unlock();
    std::vector<std::pair<Request*, cd_status>> failed_adm;
    for (auto& a : admit) {
      int slot = -1;
      const cd_status as = cd::sess_admit(h, a.first->b.data() + (size_t)a.second * N,
                                          a.first->alpha[a.second], a.first->beta[a.second], &slot);
      if (as != CD_OK) {
        failed_adm.push_back(std::make_pair(a.first, as));
        continue;
      }
      bk.owner[slot] = std::make_pair(a.first->id, a.second);
    }
    std::vector<int> fin;
    const cd_status ss = cd::sess_step(h, fin);
    std::vector<std::pair<int, cd_result>> outs;
    for (int slot : fin) {
      const std::pair<uint64_t, int> own = bk.owner[slot];
      Request* r = nullptr;
      {
        std::lock_guard<std::mutex> lk2(mu);
        auto it = reqs.find(own.first);
        if (it != reqs.end()) r = it->second.get();
      }
      cd_result res{};
      std::vector<double> tmp(N);
      const cd_status ts = cd::sess_take(h, slot, tmp.data(), &res);
      if (ts != CD_OK)
        res.status = ts;
      else if (res.status == CD_OK || res.status == CD_NOT_CONVERGED)  // the returned x itself
        res.status = res.relres <= opt.solve.rtol ? CD_OK : CD_NOT_CONVERGED;
      if (r) std::memcpy(r->x.data() + (size_t)own.second * N, tmp.data(), N * sizeof(double));
      outs.push_back(std::make_pair(slot, res));
    }
    lk.lock();
    for (auto& f : failed_adm) {  // not admitted: the request fails
      bk.busy -= 1;
      if (!f.first->done) finish(this, *f.first, f.second);
    }
    for (auto& o : outs) {
      const std::pair<uint64_t, int> own = bk.owner[o.first];
      bk.owner[o.first] = std::make_pair(uint64_t(0), -1);
      bk.busy -= 1;
      auto it = reqs.find(own.first);
      if (it == reqs.end()) continue;
      Request& r = *it->second;
      r.res[own.second] = o.second;
      solves += 1;
      if (--r.remaining == 0 && !r.done) {
        cd_status worst = CD_OK;
        for (const cd_result& q : r.res)
          if (q.status != CD_OK && worst == CD_OK) worst = (cd_status)q.status;
        finish(this, r, worst);
      }
    }
    if (ss != CD_OK) {  // a failed step: the bucket's solves in flight fail
      for (size_t k = 0; k < bk.owner.size(); ++k) {
        if (bk.owner[k].second < 0) continue;
        auto it = reqs.find(bk.owner[k].first);
        if (it != reqs.end() && !it->second->done) finish(this, *it->second, ss);
      }
    }
    batches += 1;
    slot_steps += (uint64_t)(bk.busy + outs.size());
    bk.running = false;
    bk.last_used = Clock::now();
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

void cd_server_default_options(cd_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget = 0;
  o->workers = 8;
  o->max_batch = 16;
  o->timeout_s = 0.0;
  cd_default_options(&o->solve);
  o->solve.precond = CD_PC_MG;
}

cd_status cd_server_create(cd_server* out, const cd_server_options* opt) {
  if (!out) return CD_EINVAL;
  *out = nullptr;
  std::unique_ptr<cd_server_s> S(new cd_server_s());
  cd_server_default_options(&S->opt);
  if (opt) S->opt = *opt;
  if (S->opt.workers < 1 || S->opt.workers > 256 || S->opt.max_batch < 1 ||
      S->opt.max_batch > 4096) {
    cd::set_error("invalid server options");
    return CD_EINVAL;
  }
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cd::set_error("no CUDA device");
    return CD_ECUDA;
  }
  if (S->opt.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cd::set_error("cudaMemGetInfo failed");
      return CD_ECUDA;
    }
    S->opt.hbm_budget = (size_t)(0.8 * (double)fr);
  }
  cd_server_s* raw = S.get();
  for (int i = 0; i < S->opt.workers; ++i) S->workers.emplace_back([raw] { raw->worker_loop(); });
  *out = S.release();
  return CD_OK;
}

cd_status cd_server_submit(cd_server S, int d, int p, int n, const double* alphas,
                           const double* betas, const double* b_host, int nrhs, uint64_t* ticket) {
  if (!S || !b_host || !ticket || !alphas || !betas) return CD_EINVAL;
  if ((d != 2 && d != 3) || p < 1 || n < 1 || n + p - 2 < 2 || nrhs < 1 || nrhs > S->opt.max_batch) {
    cd::set_error("cd_server_submit: bad shape or nrhs outside [1, max_batch]");
    return CD_EINVAL;
  }
  for (int i = 0; i < nrhs; ++i)
    if (!(alphas[i] > 0) || !(betas[i] > 0) || !std::isfinite(alphas[i]) || !std::isfinite(betas[i])) {
      cd::set_error("cd_server_submit: alpha and beta must be finite and > 0");
      return CD_EINVAL;
    }
  std::unique_ptr<Request> r(new Request());
  r->d = d;
  r->p = p;
  r->n = n;
  r->nrhs = nrhs;
  const size_t N = cd_dofs(d, p, n);
  r->alpha.assign(alphas, alphas + nrhs);
  r->beta.assign(betas, betas + nrhs);
  r->b.assign(b_host, b_host + (size_t)nrhs * N);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->any_submit) {
    S->any_submit = true;
    S->t_first_submit = r->t_submit;
  }
  r->id = S->next_id++;
  *ticket = r->id;
  Bucket& bk = S->buckets[std::make_tuple(d, p, n)];
  bk.d = d;
  bk.p = p;
  bk.n = n;
  bk.pending.push_back(r->id);
  S->reqs[r->id] = std::move(r);
  S->submitted += 1;
  S->cv_work.notify_one();
  return CD_OK;
}

static cd_status take_result(cd_server S, uint64_t ticket, double* x_host, cd_result* res) {
  auto it = S->reqs.find(ticket);
  Request& r = *it->second;
  if (x_host && !r.x.empty()) std::memcpy(x_host, r.x.data(), r.x.size() * sizeof(double));
  if (res)
    for (int i = 0; i < r.nrhs; ++i) {
      if (i < (int)r.res.size()) {
        res[i] = r.res[i];
      } else {
        std::memset(&res[i], 0, sizeof(cd_result));
        res[i].status = r.status;
      }
    }
  const cd_status st = r.status;
  S->reqs.erase(it);
  return st;
}

cd_status cd_server_poll(cd_server S, uint64_t ticket, double* x_host, cd_result* res, int* done) {
  if (!S || !done) return CD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return CD_EINVAL;
  *done = it->second->done ? 1 : 0;
  if (!*done) return CD_OK;
  return take_result(S, ticket, x_host, res);
}

cd_status cd_server_wait(cd_server S, uint64_t ticket, double* x_host, cd_result* res,
                         double timeout_s) {
  if (!S) return CD_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return CD_EINVAL;
  Request* r = it->second.get();
  auto pred = [&] { return r->done; };
  if (timeout_s > 0) {
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return CD_TIMEOUT;
  } else {
    S->cv_done.wait(lk, pred);
  }
  return take_result(S, ticket, x_host, res);
}

cd_status cd_server_cancel(cd_server S, uint64_t ticket) {
  if (!S) return CD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return CD_EINVAL;
  Request& r = *it->second;
  if (r.done) return CD_OK;
  Bucket& bk = S->buckets[std::make_tuple(r.d, r.p, r.n)];
  auto pos = std::find(bk.pending.begin(), bk.pending.end(), ticket);
  if (pos == bk.pending.end()) return CD_EINVAL;  // already on the GPU: it will finish normally
  bk.pending.erase(pos);
  finish(S, r, CD_CANCELLED);
  S->cv_done.notify_all();
  return CD_OK;
}

cd_status cd_server_stats_get(cd_server S, cd_server_stats* out) {
  if (!S || !out) return CD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->batches = S->batches;
  out->solves = S->solves;
  out->bytes_in_use = S->mem_used;
  for (auto& kv : S->buckets)
    if (kv.second.h) out->handles += 1;
  if (!S->latencies.empty()) {
    std::vector<double> v = S->latencies;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    out->p50_s = q(0.50);
    out->p99_s = q(0.99);
  }
  out->mean_batch = S->batches ? (double)S->slot_steps / (double)S->batches : 0.0;
  if (S->any_submit && S->solves > 0) {
    const double span = seconds_between(S->t_first_submit, S->t_last_done);
    out->solves_per_s = span > 0 ? (double)S->solves / span : 0.0;
  }
  return CD_OK;
}

cd_status cd_server_destroy(cd_server S) {
  if (!S) return CD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->buckets) {
    if (kv.second.h) cd_destroy(kv.second.h);
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
  delete S;
  return CD_OK;
}

}  // extern "C"
