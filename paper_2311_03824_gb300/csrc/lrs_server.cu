// Serving through the C ABI (include/lrs.h, lrs_server_*): a request loop
// with continuous batching for many reconstruction problems (Section I-A
// problems of any n, m, q, r, rho and operator kind) on one GPU.
//
// A request is admitted in submission order as soon as a slot is free and
// its device footprint fits what the requests in flight leave of the HBM
// budget; compatible Gaussian requests queued right behind it may join it as
// one batch (batch > 1).  Each slot is a worker thread with its own CUDA
// stream; it runs the request (or batch) through the public calls (lrs_create, lrs_set_measurements,
// lrs_init, lrs_iterate, lrs_get, lrs_destroy), so the work of concurrent
// requests overlaps on the GPU.  A Gaussian request's persistent sweep gets
// a share of the SMs (lrs_options.grid) sized by the requests running when
// it starts.  Finishing releases the slot and the memory, which admits the
// next requests.  The library's kernels do not depend on what else runs nor
// on the grid a sweep gets, so every result equals the one of the request
// solved alone.
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

#include "../../include/lrs.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t ticket = 0;
  lrs_request req{};
  size_t footprint = 0;
  lrs_result res{};
  bool done = false;
};

thread_local std::string g_srv_err;

lrs_status srv_fail(lrs_status st, const std::string& m) {
  g_srv_err = m;
  return st;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct lrs_server_s {
  lrs_server_options opt{};
  int sms = 148;
  int device = 0;                 // the creating thread's device: the workers use it
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_admit;   // dispatcher: a slot or memory freed, a submission
  std::condition_variable cv_done;    // waiters: a request finished
  std::condition_variable cv_work;    // workers: a job handed over
  std::deque<std::shared_ptr<Job>> pending;
  std::deque<std::vector<std::shared_ptr<Job>>> ready;   // admitted groups, not yet taken
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  int64_t next_admit = 0;
  size_t in_use = 0;
  int running = 0;
  bool stopping = false;          // no new submissions; queued requests still run
  bool dispatcher_done = false;   // every submitted request has been handed to a worker
  std::vector<std::thread> workers;
  std::thread dispatcher;
  double seconds() const {
    return std::chrono::duration<double>(Clock::now() - t0).count();
  }
};

namespace {

// The library's solver for one request on the worker's stream.
lrs_status run_request(const lrs_request& rq, int grid, cudaStream_t stream, std::string* msg) {
  lrs_options o = rq.opt;
  o.stream = stream;
  if (rq.kind == LRS_OP_GAUSSIAN && o.grid == 0) o.grid = grid;
  // steady iterations replay as a CUDA graph (bit-identical to eager launches)
  if (rq.kind == LRS_OP_GAUSSIAN && !o.reduce && !o.profile) o.use_graph = 1;
  lrs_t h = nullptr;
  lrs_status st = lrs_create(rq.n, rq.m, rq.q, rq.r, rq.rho, rq.kind, &o, &h);
  if (st == LRS_OK) st = lrs_set_measurements(h, rq.y, rq.A_or_mask, rq.mem_kind);
  if (st == LRS_OK) st = lrs_init(h);
  if (st == LRS_OK) st = lrs_iterate(h, o.T > 0 ? o.T : 200, nullptr);
  if (st == LRS_OK && (rq.U || rq.B || rq.S_idx || rq.S_val))
    st = lrs_get(h, rq.U, rq.B, rq.S_idx, rq.S_val, rq.out_mem_kind);
  if (st != LRS_OK) *msg = lrs_last_error();
  lrs_destroy(h);
  return st;
}

// Requests admitted together: each is created, given its measurements and
// initialised on the worker's stream, then their iterations run in one
// persistent launch per sweep (lrs_iterate_batch; each alone when the
// handles cannot share a launch, with the same results), then the outputs.
void run_group(const std::vector<std::shared_ptr<Job>>& g, int grid, cudaStream_t stream,
               std::vector<lrs_status>* st, std::vector<std::string>* msg) {
  const size_t n = g.size();
  std::vector<lrs_t> hs(n, nullptr);
  for (size_t i = 0; i < n; ++i) {
    const lrs_request& rq = g[i]->req;
    lrs_options o = rq.opt;
    o.stream = stream;
    if (o.grid == 0) o.grid = grid;
    if (o.engine == 0) o.engine = 2;
    lrs_status e = lrs_create(rq.n, rq.m, rq.q, rq.r, rq.rho, rq.kind, &o, &hs[i]);
    if (e == LRS_OK) e = lrs_set_measurements(hs[i], rq.y, rq.A_or_mask, rq.mem_kind);
    if (e == LRS_OK) e = lrs_init(hs[i]);
    (*st)[i] = e;
    if (e != LRS_OK) (*msg)[i] = lrs_last_error();
  }
  std::vector<lrs_t> ok;
  std::vector<size_t> at;
  for (size_t i = 0; i < n; ++i)
    if ((*st)[i] == LRS_OK) {
      ok.push_back(hs[i]);
      at.push_back(i);
    }
  const int T = g[0]->req.opt.T > 0 ? g[0]->req.opt.T : 200;
  if (!ok.empty()) {
    lrs_status e = lrs_iterate_batch(ok.data(), static_cast<int32_t>(ok.size()), T);
    if (e == LRS_ERR_UNSUPPORTED) {
      for (size_t j = 0; j < ok.size(); ++j) {
        (*st)[at[j]] = lrs_iterate(ok[j], T, nullptr);
        if ((*st)[at[j]] != LRS_OK) (*msg)[at[j]] = lrs_last_error();
      }
    } else if (e != LRS_OK) {
      const std::string m = lrs_last_error();
      for (size_t j : at) {
        (*st)[j] = e;
        (*msg)[j] = m;
      }
    }
  }
  for (size_t i = 0; i < n; ++i) {
    const lrs_request& rq = g[i]->req;
    if ((*st)[i] == LRS_OK && (rq.U || rq.B || rq.S_idx || rq.S_val)) {
      (*st)[i] = lrs_get(hs[i], rq.U, rq.B, rq.S_idx, rq.S_val, rq.out_mem_kind);
      if ((*st)[i] != LRS_OK) (*msg)[i] = lrs_last_error();
    }
    lrs_destroy(hs[i]);
  }
}

void worker_main(lrs_server_s* s, int wi) {
  cudaStream_t stream = nullptr;
  bool have_stream = false;
  for (;;) {
    std::vector<std::shared_ptr<Job>> group;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->dispatcher_done || !s->ready.empty(); });
      if (s->ready.empty()) break;   // stopping, and every request has been handed over
      group = s->ready.front();
      s->ready.pop_front();
    }
    const size_t n = group.size();
    const int grid = group[0]->res.grid;
    const double t_start = s->seconds();
    for (auto& job : group) {
      job->res.worker = wi;
      job->res.start_s = t_start;
    }
    std::vector<lrs_status> st(n, LRS_OK);
    std::vector<std::string> msg(n);
    if (s->opt.runner) {
      for (size_t i = 0; i < n; ++i) {
        st[i] = static_cast<lrs_status>(s->opt.runner(s->opt.runner_ctx, &group[i]->req, grid, wi));
        if (st[i] != LRS_OK) msg[i] = "the runner reported a failure";
      }
    } else {
      if (!have_stream) {
        cudaSetDevice(s->device);
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess) {
          have_stream = true;
        } else {
          cudaGetLastError();
        }
      }
      if (!have_stream) {
        for (size_t i = 0; i < n; ++i) {
          st[i] = LRS_ERR_CUDA;
          msg[i] = "lrs_server: no CUDA stream for the worker";
        }
      } else if (n == 1) {
        st[0] = run_request(group[0]->req, grid, stream, &msg[0]);
      } else {
        run_group(group, grid, stream, &st, &msg);
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t_end = s->seconds();
      for (size_t i = 0; i < n; ++i) {
        Job& job = *group[i];
        job.res.status = st[i];
        std::snprintf(job.res.message, sizeof(job.res.message), "%s", msg[i].c_str());
        job.res.end_s = t_end;
        job.done = true;
        s->in_use -= job.footprint;
      }
      s->running -= 1;
    }
    s->cv_done.notify_all();
    s->cv_admit.notify_all();
  }
  if (have_stream) cudaStreamDestroy(stream);
}

// Requests that may run their iterations in one launch: Gaussian, task
// engine (or automatic), no reducer, same rank, A_k form and iteration count.
bool batchable(const lrs_request& a) {
  return a.kind == LRS_OP_GAUSSIAN && (a.opt.engine == 0 || a.opt.engine == 2) && !a.opt.reduce;
}
bool same_batch(const lrs_request& a, const lrs_request& b) {
  return batchable(a) && batchable(b) && a.r == b.r && a.opt.a_dtype == b.opt.a_dtype &&
         a.opt.T == b.opt.T;
}

// Admission: first come, first served; the head request starts when a slot
// is free and its footprint fits the budget left.  After lrs_server_destroy
// the queue is drained the same way before the dispatcher leaves.
void dispatcher_main(lrs_server_s* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_admit.wait(lk, [&] {
      if (s->pending.empty()) return s->stopping;
      const auto& j = s->pending.front();
      return s->running < s->opt.slots && s->in_use + j->footprint <= s->opt.hbm_budget;
    });
    if (s->pending.empty()) break;  // stopping with nothing queued
    // a slot runs one request, or one batch of requests
    std::vector<std::shared_ptr<Job>> group;
    s->running += 1;
    for (;;) {
      auto job = s->pending.front();
      s->pending.pop_front();
      s->in_use += job->footprint;
      job->res.admitted = s->next_admit++;
      group.push_back(job);
      if (static_cast<int>(group.size()) >= std::max(1, s->opt.batch) || s->pending.empty())
        break;
      const auto& nx = s->pending.front();
      if (!same_batch(group[0]->req, nx->req) || s->in_use + nx->footprint > s->opt.hbm_budget)
        break;
    }
    const int grid = std::max(16, (2 * s->sms) / std::max(1, s->running));
    for (auto& job : group) {
      job->res.grid = grid;
      job->res.group = group[0]->res.admitted;
      job->res.group_size = static_cast<int32_t>(group.size());
    }
    s->ready.push_back(std::move(group));
    s->cv_work.notify_one();
  }
  s->dispatcher_done = true;
  s->cv_work.notify_all();
}

}  // namespace

extern "C" {

size_t lrs_request_footprint(const lrs_request* rq) {
  if (!rq) return 0;
  const int64_t n = rq->n, m = rq->m, q = rq->q, r = rq->r;
  const int64_t rho = std::max<int32_t>(rq->opt.rho_max > 0 ? rq->opt.rho_max : rq->rho, 1);
  int64_t b = 0;
  if (rq->kind == LRS_OP_DFT2D_MASK) {
    b = q * m * (8 + 4 + 8 + 4) + q * n * 8 + 8 * n * r * 8 + q * rho * 12;
  } else {
    const int64_t ns = round_up(n, 32);
    const int eb = rq->opt.a_dtype == LRS_A_FP32 ? 4 : rq->opt.a_dtype == LRS_A_FP8_HI ? 1 : 2;
    const int64_t stored = q * m * ns * eb;
    const int64_t exact = rq->opt.a_dtype != LRS_A_FP32 ? q * m * n * 4 : 0;
    const int64_t staging = rq->mem_kind == 0 ? std::min<int64_t>(q * m * n * 4, int64_t(256) << 20) : 0;
    const int64_t scratch = q * (n + ns + 2 * m + 16 * 16 * 2 + 4 * 16 * m) * 4;
    b = stored + exact + staging + scratch + q * m * 8 + q * rho * 8 + 4 * n * 16;
  }
  return static_cast<size_t>(b + b / 10) + (size_t(64) << 20);
}

lrs_status lrs_server_create(const lrs_server_options* opt, lrs_server_t* out) {
  if (!out) return srv_fail(LRS_ERR_ARG, "lrs_server_create: out is NULL");
  *out = nullptr;
  lrs_server_options o{};
  if (opt) o = *opt;
  if (o.slots < 0 || o.sms < 0 || o.batch < 0 || o.batch > 64)
    return srv_fail(LRS_ERR_ARG, "lrs_server_create: negative option or batch above 64");
  if (o.slots == 0) o.slots = 8;
  int sms = o.sms;
  if (!o.runner) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      return srv_fail(LRS_ERR_CUDA, "lrs_server_create: no CUDA device");
    }
    if (sms == 0) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (o.hbm_budget == 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return srv_fail(LRS_ERR_CUDA, "lrs_server_create: cudaMemGetInfo failed");
      }
      o.hbm_budget = fr / 100 * 85;
    }
  }
  if (o.hbm_budget == 0) return srv_fail(LRS_ERR_ARG, "lrs_server_create: hbm_budget is 0");
  auto* s = new lrs_server_s();
  s->opt = o;
  if (!o.runner) cudaGetDevice(&s->device);
  s->sms = sms > 0 ? sms : 148;
  s->t0 = Clock::now();
  for (int i = 0; i < o.slots; ++i) s->workers.emplace_back(worker_main, s, i);
  s->dispatcher = std::thread(dispatcher_main, s);
  *out = s;
  return LRS_OK;
}

lrs_status lrs_server_submit(lrs_server_t s, const lrs_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return srv_fail(LRS_ERR_ARG, "lrs_server_submit: NULL argument");
  if (!req->y || !req->A_or_mask) return srv_fail(LRS_ERR_ARG, "lrs_server_submit: no measurements");
  if (req->mem_kind != 0 && req->mem_kind != 1)
    return srv_fail(LRS_ERR_ARG, "lrs_server_submit: mem_kind must be 0 or 1");
  if (req->n < 1 || req->m < 1 || req->q < 1 || req->r < 1 || req->rho < 0 || req->rho > req->n)
    return srv_fail(LRS_ERR_ARG, "lrs_server_submit: bad sizes");
  auto job = std::make_shared<Job>();
  job->req = *req;
  job->footprint = lrs_request_footprint(req);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return srv_fail(LRS_ERR_STATE, "lrs_server_submit: server is stopping");
    if (job->footprint > s->opt.hbm_budget)
      return srv_fail(LRS_ERR_OOM, "lrs_server_submit: the request needs more than the whole budget");
    job->ticket = s->next_ticket++;
    job->res.submit_s = s->seconds();
    job->res.footprint = job->footprint;
    s->jobs[job->ticket] = job;
    s->pending.push_back(job);
    *ticket = job->ticket;
  }
  s->cv_admit.notify_all();
  return LRS_OK;
}

lrs_status lrs_server_wait(lrs_server_t s, uint64_t ticket, int32_t timeout_ms, lrs_result* res) {
  if (!s || !res) return srv_fail(LRS_ERR_ARG, "lrs_server_wait: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return srv_fail(LRS_ERR_ARG, "lrs_server_wait: unknown ticket");
  auto job = it->second;
  auto ready = [&] { return job->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return srv_fail(LRS_ERR_TIMEOUT, "lrs_server_wait: the request has not finished");
  }
  *res = job->res;
  s->jobs.erase(ticket);
  return LRS_OK;
}

lrs_status lrs_server_destroy(lrs_server_t s) {
  if (!s) return LRS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_admit.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  s->cv_work.notify_all();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  delete s;
  return LRS_OK;
}

const char* lrs_server_last_error(void) { return g_srv_err.c_str(); }

}  // extern "C"
