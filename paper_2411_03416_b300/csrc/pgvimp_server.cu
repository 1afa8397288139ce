// pgvimp_server.cu -- continuous-batching planning server (host runtime).
//
// Requests (problem + options) arrive from any host thread.  A scheduler
// thread packs queued requests of a compatible kind (state dimension,
// dynamics kind, execution form, and for SLR plans the iteration counts) into
// a batch as soon as a launch slot, device memory and pinned staging are
// free, and launches the whole plan (upload, prior, iterations, result download) on one of
// several streams, so that batches admitted while others run overlap on the
// GPU; each batch's launch sequence is captured into a CUDA graph and launched
// as one.  A stream callback hands the finished batch back to the scheduler,
// which copies each plan's result out, frees the batch's memory and admits
// the next requests.  Device memory and pinned host staging come from two
// pools allocated once at creation (first-fit with coalescing), so the
// serving loop itself makes no CUDA allocation or free call, neither of
// which could overlap with running work.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pgvimp_internal.h"
#include "pgvimp_plan.h"
#include "pgvimp_pool.h"

namespace pgv {
namespace {

// Deep copy of a problem (the caller may free its arrays after submit).
struct OwnedProblem {
  pgvimp_problem p;
  std::vector<double> A, a, B, Qc, mu0, K0, muN, KN, dh, soff, srad;
  std::vector<float> sdf;
  std::vector<int> slink;

  template <typename T>
  static const T* copy(std::vector<T>& v, const T* src, size_t cnt) {
    if (!src || !cnt) return nullptr;
    v.assign(src, src + cnt);
    return v.data();
  }
  void take(const pgvimp_problem& s) {
    p = s;
    const size_t n = s.n, m = s.m, N = s.N, nn = n * n;
    p.A = copy(A, s.A, s.A ? (s.A_per_step ? N : 1) * nn : 0);
    p.a = copy(a, s.a, s.a ? (s.a_per_step ? N : 1) * n : 0);
    p.B = copy(B, s.B, n * m);
    p.Qc = copy(Qc, s.Qc, m * m);
    p.mu0 = copy(mu0, s.mu0, n);
    p.K0 = copy(K0, s.K0, nn);
    p.muN = copy(muN, s.muN, n);
    p.KN = copy(KN, s.KN, nn);
    const bool three = (s.cost_kind == PGVIMP_COST_POINT3D || s.cost_kind == PGVIMP_COST_ARM);
    const size_t cells = (s.cost_kind == PGVIMP_COST_NONE || !s.sdf)
                             ? 0
                             : (size_t)s.sdf_nx * s.sdf_ny * (three ? std::max(s.sdf_nz, 1) : 1);
    p.sdf = copy(sdf, s.sdf, cells);
    const bool arm = (s.cost_kind == PGVIMP_COST_ARM);
    p.arm_dh = copy(dh, arm ? s.arm_dh : nullptr, arm ? 4 * (size_t)s.arm_dof : 0);
    p.sphere_link = copy(slink, arm ? s.sphere_link : nullptr, arm ? (size_t)s.n_spheres : 0);
    p.sphere_off = copy(soff, arm ? s.sphere_off : nullptr, arm ? 3 * (size_t)s.n_spheres : 0);
    p.sphere_r = copy(srad, arm ? s.sphere_r : nullptr, arm ? (size_t)s.n_spheres : 0);
  }
};

// Requests that may share a batch.
struct GroupKey {
  int n, dyn, iters, slr, tpb;
  bool operator==(const GroupKey& o) const {
    return n == o.n && dyn == o.dyn && iters == o.iters && slr == o.slr && tpb == o.tpb;
  }
};

struct Request {
  uint64_t id = 0;
  OwnedProblem prob;
  pgvimp_options opt;
  GroupKey key;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = 0;   // 0 queued, 1 on the device, 2 finished
  pgvimp_status status = PGVIMP_OK;
  std::string err;
  std::vector<double> mu, Sd;
  pgvimp_step_info last;
  int n_logs = 0, batch_size = 0;
};

struct Flight;

}  // namespace
}  // namespace pgv

using namespace pgv;

struct pgvimp_server {
  pgvimp_server_config cfg;
  int device = 0;
  char* dev_pool = nullptr;
  char* host_pool = nullptr;
  RangeAllocator dev_alloc, host_alloc;
  std::vector<cudaStream_t> streams;
  std::vector<cudaGraphExec_t> execs;   // per stream slot: the last captured launch sequence
  std::vector<char> slot_busy;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Flight*> finished;   // handed back by the stream callbacks
  int inflight = 0;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t launched_batches = 0, launched_plans = 0;
  uint64_t graph_launches = 0, graph_instantiations = 0;   // batches launched as one graph; graphs built
  double host_launch_ms = 0.0, host_collect_ms = 0.0;   // scheduler time spent preparing / collecting batches
  std::thread worker;
  std::chrono::steady_clock::time_point t0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace pgv {
namespace {

struct Flight {
  pgvimp_server* S = nullptr;
  pgvimp_batch* b = nullptr;
  std::vector<Request*> reqs;
  int slot = -1;
  size_t dev_off = 0, dev_bytes = 0, hin_off = 0, hin_bytes = 0, hout_off = 0, hout_bytes = 0;
  pgvimp_status launch_status = PGVIMP_OK;
  std::string launch_err;
};

pgvimp_status server_fail(pgvimp_status st, const std::string& m) {
  set_thread_error(m);
  return st;
}

void CUDART_CB on_flight_done(void* p) {
  Flight* f = static_cast<Flight*>(p);
  std::lock_guard<std::mutex> lk(f->S->mu);
  f->S->finished.push_back(f);
  f->S->cv_sched.notify_all();
}

// Creates the batch in the flight's pool ranges and queues the whole plan on
// its stream, ending with a host callback.  Runs on the scheduler thread
// without the server lock.
pgvimp_status launch_flight(pgvimp_server* S, Flight* f) {
  std::vector<pgvimp_problem> probs;
  std::vector<pgvimp_options> opts;
  for (Request* r : f->reqs) {
    probs.push_back(r->prob.p);
    opts.push_back(r->opt);
  }
  pgvimp_status st = batch_create_staged((int)probs.size(), probs.data(), opts.data(), S->cfg.precision,
                                         S->dev_pool + f->dev_off, f->dev_bytes, S->host_pool + f->hin_off,
                                         S->host_pool + f->hout_off, &f->b, false);
  if (st != PGVIMP_OK) return st;
  void* s = S->streams[f->slot];
  cudaStream_t cs = static_cast<cudaStream_t>(s);
  auto enqueue = [&]() -> pgvimp_status {
    pgvimp_status q;
    if ((q = pgvimp_batch_upload(f->b, s)) || (q = pgvimp_batch_reset(f->b, s)) || (q = pgvimp_batch_run(f->b, 0, s)) ||
        (q = pgvimp_batch_download_results(f->b, s)))
      return q;
    cudaError_t e = cudaLaunchHostFunc(cs, on_flight_done, f);
    if (e != cudaSuccess) return server_fail(PGVIMP_ECUDA, std::string("cudaLaunchHostFunc: ") + cudaGetErrorString(e));
    return PGVIMP_OK;
  };
  // The flight's whole launch sequence (copy in, prior, iterations, copy out,
  // completion callback) is captured into a graph and launched as one.  The
  // slot's executable graph is updated in place when the sequence has the same
  // shape as the slot's last one (same kernels, new arena and argument values)
  // and instantiated anew otherwise; the slot is idle while it is updated.
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    st = enqueue();
    cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (st != PGVIMP_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    cudaGraphExec_t& ex = S->execs[f->slot];
    if (ec == cudaSuccess && g) {
      if (ex) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
          cudaGetLastError();   // a shape change: build a new executable graph
          cudaGraphExecDestroy(ex);
          ex = nullptr;
        }
      }
      if (!ex && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) ++S->graph_instantiations;
      cudaGraphDestroy(g);
      if (ex && cudaGraphLaunch(ex, cs) == cudaSuccess) {
        ++S->graph_launches;
        return PGVIMP_OK;
      }
    } else if (g) {
      cudaGraphDestroy(g);
    }
    cudaGetLastError();
  } else {
    cudaGetLastError();
  }
  // capture, instantiation or graph launch unavailable: launch the sequence directly
  return enqueue();
}

// Copies each plan's result out of a finished flight (scheduler thread, no
// lock: the flight's requests are touched by nobody else while running).
void collect_flight(Flight* f) {
  const int cnt = (int)f->reqs.size();
  for (int i = 0; i < cnt; ++i) {
    Request* r = f->reqs[i];
    r->batch_size = cnt;
    if (f->launch_status != PGVIMP_OK) {
      r->status = f->launch_status;
      r->err = f->launch_err;
      continue;
    }
    const int code = batch_plan_status(f->b, i);
    if (code != 0) {
      r->status = PGVIMP_ENOTPD;
      r->err = code == 1   ? "prior precision not positive definite"
               : code == 2 ? "initial marginals not positive definite"
               : code == 3 ? "a factor marginal became not positive definite"
                           : "SLR linearisation failed";
    }
    const size_t n = r->prob.p.n, N = r->prob.p.N;
    r->mu.resize((N + 1) * n);
    r->Sd.resize((N + 1) * n * n);
    const int cap = std::max(1, r->opt.iters * std::max(1, r->opt.slr_iters));
    std::vector<pgvimp_step_info> logs(cap);
    int nl = 0;
    pgvimp_batch_result(f->b, i, r->mu.data(), r->Sd.data(), nullptr, nullptr, nullptr, logs.data(), cap, &nl);
    r->n_logs = nl;
    std::memset(&r->last, 0, sizeof(r->last));
    if (nl > 0) r->last = logs[std::min(nl, cap) - 1];
  }
  if (f->b) pgvimp_batch_destroy(f->b);
  f->b = nullptr;
}

void release_flight(pgvimp_server* S, Flight* f) {
  if (f->dev_bytes) S->dev_alloc.release(f->dev_off, f->dev_bytes);
  if (f->hin_bytes) S->host_alloc.release(f->hin_off, f->hin_bytes);
  if (f->hout_bytes) S->host_alloc.release(f->hout_off, f->hout_bytes);
  if (f->slot >= 0) S->slot_busy[f->slot] = 0;
}

// Picks up to max_batch queued requests of the head's group (FIFO) that fit
// the free pools together, reserving their memory; nullptr if none fits now.
Flight* form_flight(pgvimp_server* S) {
  Request* head = S->queue.front();
  std::vector<Request*> cand;
  for (Request* r : S->queue) {
    if (r->key == head->key) cand.push_back(r);
    if ((int)cand.size() >= S->cfg.max_batch) break;
  }
  int slot = -1;
  for (int k = 0; k < (int)S->slot_busy.size(); ++k)
    if (!S->slot_busy[k]) {
      slot = k;
      break;
    }
  if (slot < 0) return nullptr;
  for (size_t cnt = cand.size(); cnt >= 1; cnt = (cnt == 1) ? 0 : (cnt + 1) / 2) {
    std::vector<pgvimp_problem> probs;
    std::vector<pgvimp_options> opts;
    for (size_t i = 0; i < cnt; ++i) {
      probs.push_back(cand[i]->prob.p);
      opts.push_back(cand[i]->opt);
    }
    BatchSizes sz;
    if (batch_sizes((int)cnt, probs.data(), opts.data(), S->cfg.precision, &sz, false) != PGVIMP_OK) {
      if (cnt == 1) break;
      continue;
    }
    Flight* f = new (std::nothrow) Flight();
    if (!f) return nullptr;
    f->S = S;
    bool ok = S->dev_alloc.alloc(sz.dev, &f->dev_off);
    if (ok) f->dev_bytes = sz.dev;
    ok = ok && S->host_alloc.alloc(sz.host_in, &f->hin_off);
    if (ok) f->hin_bytes = sz.host_in;
    ok = ok && S->host_alloc.alloc(sz.host_out, &f->hout_off);
    if (ok) f->hout_bytes = sz.host_out;
    if (!ok) {
      release_flight(S, f);
      delete f;
      continue;
    }
    f->slot = slot;
    S->slot_busy[slot] = 1;
    f->reqs.assign(cand.begin(), cand.begin() + cnt);
    return f;
  }
  return nullptr;
}

void scheduler(pgvimp_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // retire finished batches
    while (!S->finished.empty()) {
      Flight* f = S->finished.back();
      S->finished.pop_back();
      lk.unlock();
      const double tc = S->now_ms();
      collect_flight(f);
      lk.lock();
      S->host_collect_ms += S->now_ms() - tc;
      const double t = S->now_ms();
      for (Request* r : f->reqs) {
        r->state = 2;
        r->t_done = t;
      }
      release_flight(S, f);
      --S->inflight;
      delete f;
      S->cv_done.notify_all();
    }
    if (S->stop) {
      if (S->inflight == 0) break;
      S->cv_sched.wait(lk);
      continue;
    }
    // admit
    bool wait_deadline = false;
    double deadline = 0.0;
    if (!S->queue.empty() && S->inflight < S->cfg.max_inflight) {
      Request* head = S->queue.front();
      int group = 0;
      for (Request* r : S->queue)
        if (r->key == head->key && ++group >= S->cfg.max_batch) break;
      const double now = S->now_ms();
      if (group >= S->cfg.max_batch || now - head->t_submit >= S->cfg.batch_window_ms) {
        Flight* f = form_flight(S);
        if (f) {
          const double t = S->now_ms();
          for (Request* r : f->reqs) {
            r->state = 1;
            r->t_start = t;
            S->queue.erase(std::find(S->queue.begin(), S->queue.end(), r));
          }
          ++S->inflight;
          S->launched_batches += 1;
          S->launched_plans += f->reqs.size();
          lk.unlock();
          const double tl = S->now_ms();
          pgvimp_status st = launch_flight(S, f);
          S->host_launch_ms += S->now_ms() - tl;
          if (st != PGVIMP_OK) {
            f->launch_status = st;
            const char* e = pgvimp_last_error(nullptr);
            f->launch_err = e ? e : "launch failed";
            // no callback was queued: hand the flight back directly once the
            // stream has drained whatever was queued before the failure
            cudaStreamSynchronize(S->streams[f->slot]);
            lk.lock();
            S->finished.push_back(f);
          } else {
            lk.lock();
          }
          continue;
        }
        // nothing fits now: wait for a batch to finish
      } else {
        wait_deadline = true;
        deadline = head->t_submit + S->cfg.batch_window_ms;
      }
    }
    if (wait_deadline) {
      const double wait = std::max(0.0, deadline - S->now_ms());
      S->cv_sched.wait_for(lk, std::chrono::duration<double, std::milli>(wait));
    } else {
      S->cv_sched.wait(lk);
    }
  }
}

}  // namespace
}  // namespace pgv

extern "C" pgvimp_status pgvimp_server_create(const pgvimp_server_config* cfg, pgvimp_server** out) {
  if (!cfg || !out) return server_fail(PGVIMP_EINVAL, "config or out is NULL");
  *out = nullptr;
  pgvimp_server_config c = *cfg;
  if (c.precision != PGVIMP_PREC_PLAIN_FP64 && c.precision != PGVIMP_PREC_MIXED && c.precision != PGVIMP_PREC_MIXED_DF)
    return server_fail(PGVIMP_EINVAL, "unknown precision");
  if (c.hbm_budget_bytes < ((size_t)1 << 20)) return server_fail(PGVIMP_EINVAL, "hbm_budget_bytes must be >= 1 MiB");
  if (c.max_inflight < 1 || c.max_inflight > 64) return server_fail(PGVIMP_EINVAL, "max_inflight must be in 1..64");
  if (c.max_batch < 1 || c.max_batch > (1 << 20)) return server_fail(PGVIMP_EINVAL, "max_batch must be >= 1");
  if (c.plan_threads < -1 || (c.plan_threads > 1 && c.plan_threads != kLaneThreads &&
                              (c.plan_threads < 32 || c.plan_threads > kCrMaxThreads || (c.plan_threads & 31))))
    return server_fail(PGVIMP_EINVAL, "plan_threads must be -1, 0, 1, 16, or a multiple of 32 in 32..256");
  if (!(c.batch_window_ms >= 0.0) || !(c.batch_window_ms < 1e7)) return server_fail(PGVIMP_EINVAL, "bad batch_window_ms");
  if (c.host_staging_bytes == 0) c.host_staging_bytes = std::min<size_t>(c.hbm_budget_bytes, (size_t)4 << 30);
  pgvimp_server* S = new (std::nothrow) pgvimp_server();
  if (!S) return server_fail(PGVIMP_ENOMEM, "host allocation failed");
  S->cfg = c;
  S->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaMalloc(&S->dev_pool, c.hbm_budget_bytes);
  if (e != cudaSuccess) {
    delete S;
    return server_fail(PGVIMP_ENOMEM, std::string("device pool: ") + cudaGetErrorString(e));
  }
  e = cudaMallocHost(&S->host_pool, c.host_staging_bytes);
  if (e != cudaSuccess) {
    cudaFree(S->dev_pool);
    delete S;
    return server_fail(PGVIMP_ENOMEM, std::string("pinned staging pool: ") + cudaGetErrorString(e));
  }
  S->dev_alloc.reset(c.hbm_budget_bytes);
  S->host_alloc.reset(c.host_staging_bytes);
  for (int k = 0; k < c.max_inflight; ++k) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
      cudaFreeHost(S->host_pool);
      cudaFree(S->dev_pool);
      delete S;
      return server_fail(PGVIMP_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    S->streams.push_back(s);
  }
  S->slot_busy.assign(c.max_inflight, 0);
  S->execs.assign(c.max_inflight, nullptr);
  S->worker = std::thread(scheduler, S);
  *out = S;
  return PGVIMP_OK;
}

extern "C" pgvimp_status pgvimp_submit(pgvimp_server* S, const pgvimp_problem* problem, const pgvimp_options* options,
                                       uint64_t* request_id) {
  if (!S || !problem || !options || !request_id) return server_fail(PGVIMP_EINVAL, "NULL argument");
  pgvimp_options o = *options;
  if (S->cfg.plan_threads >= 0) o.plan_threads = S->cfg.plan_threads;
  BatchSizes sz;
  pgvimp_status st = batch_sizes(1, problem, &o, S->cfg.precision, &sz);   // validates the request
  if (st != PGVIMP_OK) return st;
  if (round_up(sz.dev) > S->dev_alloc.total() || round_up(sz.host_in) + round_up(sz.host_out) > S->host_alloc.total())
    return server_fail(PGVIMP_ENOMEM, "request larger than the server's memory budget");
  Request* r = new (std::nothrow) Request();
  if (!r) return server_fail(PGVIMP_ENOMEM, "host allocation failed");
  r->prob.take(*problem);
  r->opt = o;
  const bool slr = problem->dyn_kind != PGVIMP_DYN_LINEAR;
  r->key = GroupKey{problem->n, problem->dyn_kind, slr ? o.iters : 0, slr ? o.slr_iters : 0, o.plan_threads};
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    delete r;
    return server_fail(PGVIMP_EINVAL, "server is shutting down");
  }
  r->id = S->next_id++;
  r->t_submit = S->now_ms();
  S->reqs[r->id] = r;
  S->queue.push_back(r);
  *request_id = r->id;
  S->cv_sched.notify_all();
  return PGVIMP_OK;
}

extern "C" pgvimp_status pgvimp_poll(pgvimp_server* S, uint64_t request_id, int timeout_ms, double* mu,
                                     double* Sigma, pgvimp_request_info* info) {
  if (!S) return server_fail(PGVIMP_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request_id);
  if (it == S->reqs.end()) return server_fail(PGVIMP_EINVAL, "unknown request id (or already collected)");
  Request* r = it->second;
  auto done = [&] { return r->state == 2; };
  if (!done()) {
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    if (!done()) return server_fail(PGVIMP_ENOTREADY, "request not finished");
  }
  if (mu && !r->mu.empty()) std::memcpy(mu, r->mu.data(), sizeof(double) * r->mu.size());
  if (Sigma && !r->Sd.empty()) std::memcpy(Sigma, r->Sd.data(), sizeof(double) * r->Sd.size());
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = r->status;
    info->n = r->prob.p.n;
    info->N = r->prob.p.N;
    info->n_logs = r->n_logs;
    info->batch_size = r->batch_size;
    info->submit_ms = r->t_submit;
    info->start_ms = r->t_start;
    info->done_ms = r->t_done;
    info->last = r->last;
  }
  const pgvimp_status st = r->status;
  const std::string err = r->err;
  S->reqs.erase(it);
  delete r;
  if (st != PGVIMP_OK) return server_fail(st, err);
  return PGVIMP_OK;
}

extern "C" pgvimp_status pgvimp_server_stats(pgvimp_server* S, pgvimp_server_stats_t* out) {
  if (!S || !out) return server_fail(PGVIMP_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->queued = (int)S->queue.size();
  out->inflight = S->inflight;
  out->batches = S->launched_batches;
  out->plans = S->launched_plans;
  out->dev_used = S->dev_alloc.used();
  out->host_used = S->host_alloc.used();
  out->now_ms = S->now_ms();
  out->host_launch_ms = S->host_launch_ms;
  out->host_collect_ms = S->host_collect_ms;
  out->graph_launches = S->graph_launches;
  out->graph_instantiations = S->graph_instantiations;
  return PGVIMP_OK;
}

extern "C" pgvimp_status pgvimp_server_destroy(pgvimp_server* S) {
  if (!S) return PGVIMP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_sched.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();   // returns once no batch is on the device
  for (auto& kv : S->reqs) delete kv.second;
  for (cudaGraphExec_t ex : S->execs)
    if (ex) cudaGraphExecDestroy(ex);
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  if (S->host_pool) cudaFreeHost(S->host_pool);
  if (S->dev_pool) cudaFree(S->dev_pool);
  delete S;
  return PGVIMP_OK;
}
