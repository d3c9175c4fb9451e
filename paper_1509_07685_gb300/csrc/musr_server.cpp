// musr_server.cpp -- continuous-batching serving of many fits, and musr_fit.
//
// The paper's offload (Section 4) runs one fit at a time: the host minimiser
// sends a parameter vector, the device returns the cost.  Serving many fits at
// once keeps every fit's histograms resident and advances all fits together:
//
//   the active fits are split into two lanes that the device evaluates in turn;
//   worker loop, one half-step for lane L:
//     every fit of lane L names its next trial point(s) (BFGS state machine);
//     its points go to the device in one copy; one persistent multi-fit launch
//       per (precision, theory shape, cost) group evaluates them all, and one copy
//       brings every value and gradient back -- queued behind the other lane's work;
//     queued fits are admitted while the arena (the HBM budget) has room -- a fit's
//       histograms, decomposition tables and evaluation buffers come from it;
//     the other lane's results are waited for, its fits' minimisers advance, and
//       finished fits release their memory.
//   So the device evaluates one lane while the host advances the other.
//
// Fits that arrive while others run join the lighter lane at the next half-step.
// A fit's result does not depend on what else is in the batch: its launches
// use its own decomposition and its own fixed-order reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "musr.h"
#include "musr_bfgs.h"
#include "musr_dev.h"
#include "musr_host.h"

namespace musr {
namespace {

constexpr double kSplitNoiseRel = 2e-8;  // rounding noise of the SPLIT cost, relative
constexpr double kSplitEdm = 1e-5;       // EDM target of SPLIT fits
constexpr double kFp64Edm = 1e-7;
// Decomposition of every served fit (SPLIT tiles of 4096 bins): many fits fill the
// GPU together, and a fixed choice keeps a fit's result independent of the mix.
constexpr int kServeVariant = 3;
constexpr int kAdmitBatch = 32;  // fits configured together by the helper threads

struct Request {
  int64_t id = 0;
  std::vector<unsigned char> counts_copy;  // empty when the caller lends the counts
  const void* counts = nullptr;            // counts_copy.data() or the caller's buffer
  int dtype = 0, H = 0, nslots = 0, P = 0, mode = 0, prec = 0, maxit = 0;
  int64_t B = 0;
  std::vector<double> t0, consts, x0;
  double bw = 0.0, fr[2] = {0.0, 0.0}, gtol = 0.0, t_submit = 0.0;
  std::vector<musr_term> terms;
  std::vector<int32_t> map;
};

struct Active {
  std::unique_ptr<Request> req;
  musr_ctx* ctx = nullptr;
  Bfgs bfgs;
  int shape = 0;
  int lane = 0;
  int64_t bins = 0;
  double load = 0.0;  // device work of one evaluation, (histogram, bin) pairs x (1 + P)
  double t_admit = 0.0;
  bool first = true;
  int nvec = 0;
  size_t poff = 0, ooff = 0;
  std::vector<double> pts, f, g;  // this step's trial points, values and gradients
};

// Helper threads that run fn(i) for i in [0, n) together with the calling thread (the
// fits' minimiser steps are independent of one another).
class TaskPool {
 public:
  // Helper threads make `device` their current CUDA device (admission uploads from them).
  TaskPool(int nthreads, int device) {
    for (int t = 0; t < nthreads; ++t)
      th_.emplace_back([this, device] {
        cudaSetDevice(device);
        loop();
      });
  }
  ~TaskPool() {
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void run(int n, const std::function<void(int)>& fn) {
    if (n <= 0) return;
    if (th_.empty() || n == 1) {
      for (int i = 0; i < n; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> l(mu_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      pending_ = static_cast<int>(th_.size());
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> l(mu_);
    done_.wait(l, [&] { return pending_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work() {
    for (int i; (i = next_.fetch_add(1)) < n_;) (*fn_)(i);
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> l(mu_);
        cv_.wait(l, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
      }
      work();
      std::lock_guard<std::mutex> l(mu_);
      if (--pending_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0;
  std::atomic<int> next_{0};
  int pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

struct Done {
  musr_fit_result res{};
  std::vector<double> x;
};

size_t dtype_size(int dtype) { return dtype == MUSR_DTYPE_FP64 ? 8 : 4; }

}  // namespace

// One of the two groups of active fits that the device evaluates in turn: its launch
// buffers (host pinned and device) and the event that marks its results on the host.
struct Lane {
  std::vector<Active*> launched;  // fits whose points are on the device
  double* h_params = nullptr;
  double* h_out = nullptr;
  Job* h_jobs = nullptr;
  size_t hp_cap = 0, ho_cap = 0, hj_cap = 0;
  void* d_params = nullptr;
  void* d_out = nullptr;
  void* d_jobs = nullptr;
  size_t dp_cap = 0, do_cap = 0, dj_cap = 0;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
  double load = 0.0;  // sum of its fits' Active::load
};

}  // namespace musr

using namespace musr;

struct musr_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  int max_active = 1;
  Arena arena;
  std::thread worker;
  std::unique_ptr<TaskPool> pool;  // helpers of the worker (minimiser steps, admission)
  bool admit_serial = false;       // the last parallel admission found the arena full
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<std::unique_ptr<Request>> queue;
  std::unordered_map<int64_t, Done> done;
  std::unordered_set<int64_t> live;    // submitted, not finished (queued, being admitted or active)
  std::unordered_set<int64_t> cancel;  // live fits asked to stop that the worker has not ended yet
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  musr_server_stats stats{};
  std::string err;
  // worker-owned
  std::vector<std::unique_ptr<Active>> active;
  musr::Lane lanes[2];
  int next_lane = 0;
  std::string worker_error;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Destroys a served fit's context.  Callers guarantee that none of its device work is
// pending (its lane's results were waited for, or it never launched and its setup was
// waited for), so the shared stream -- busy with the other lane -- is not waited on.
void release(musr_ctx* ctx) {
  if (!ctx) return;
  ctx->owner_waited = true;
  musr_ctx_destroy(ctx);
}

bool grow_host(void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return true;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  bytes = bytes * 3 / 2 + 4096;
  if (cudaMallocHost(p, bytes) != cudaSuccess) return false;
  *cap = bytes;
  return true;
}

bool grow_dev(void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  bytes = bytes * 3 / 2 + 4096;
  if (cudaMalloc(p, bytes) != cudaSuccess) return false;
  *cap = bytes;
  return true;
}

void finish(musr_server* s, Active* a, int status) {
  Done d;
  d.res.status = status;
  d.res.iters = a->bfgs.iters();
  d.res.nfev = a->bfgs.nfev();
  d.res.nparams = a->req->P;
  d.res.f = a->bfgs.f();
  d.res.edm = a->bfgs.edm();
  d.res.t_submit = a->req->t_submit;
  d.res.t_admit = a->t_admit;
  d.res.t_done = s->now();
  d.x = a->bfgs.x();
  release(a->ctx);
  a->ctx = nullptr;
  std::lock_guard<std::mutex> lock(s->mu);
  s->done[a->req->id] = std::move(d);
  s->live.erase(a->req->id);
  s->cancel.erase(a->req->id);
  s->stats.completed += 1;
  s->stats.active -= 1;
  s->cv_done.notify_all();
}

// Ends a fit that never ran (refused, or canceled before it ran); s->mu held.
void reject_locked(musr_server* s, std::unique_ptr<Request> r, int status) {
  Done d;
  d.res.status = status;
  d.res.nparams = r->P;
  d.res.f = NAN;
  d.res.t_submit = r->t_submit;
  d.res.t_done = s->now();
  d.x = r->x0;
  s->done[r->id] = std::move(d);
  s->live.erase(r->id);
  s->cancel.erase(r->id);
  if (status == MUSR_ECANCELED)
    s->stats.canceled += 1;
  else
    s->stats.rejected += 1;
  s->cv_done.notify_all();
}

void reject(musr_server* s, std::unique_ptr<Request> r, int status) {
  std::lock_guard<std::mutex> lock(s->mu);
  reject_locked(s, std::move(r), status);
}

// Configures a context for the request inside the arena; MUSR_ENOMEM when the
// arena is full now, another status when the request can never run.
int configure(musr_server* s, const Request& r, musr_ctx** out) {
  double t[5];
  t[0] = s->now();
  musr_ctx* ctx = nullptr;
  int rc = musr_ctx_create(&ctx, s->device, 0, s->stream);
  if (rc) return rc;
  ctx->arena = &s->arena;
  // Every setup copy and kernel of this fit goes on this thread's stream, waited for
  // once at the end (the serving stream keeps running the current step meanwhile).
  ctx->setup_stream = cudaStreamPerThread;
  t[1] = s->now();
  rc = musr_upload_histograms(ctx, r.counts, r.dtype, r.H, r.B, r.t0.data(), r.bw, r.fr);
  t[2] = s->now();
  if (!rc) rc = musr_set_theory(ctx, r.terms.data(), static_cast<int>(r.terms.size()));
  if (!rc)
    rc = musr_set_map(ctx, r.map.data(), r.nslots, r.P, r.consts.empty() ? nullptr : r.consts.data(),
                      static_cast<int>(r.consts.size()));
  if (!rc) rc = check_ready(ctx, r.mode, r.prec);
  if (!rc) rc = ensure_compiled(ctx, r.prec, kServeVariant);
  t[3] = s->now();
  if (!rc) rc = ensure_eval(ctx, r.prec, kServeVariant, r.P > 0 ? r.P : 1);
  // wait even after a failure: nothing may still write to memory the context gives back
  const cudaError_t e = cudaStreamSynchronize(cudaStreamPerThread);
  if (!rc) rc = e == cudaSuccess ? finish_upload_check(ctx) : cuda_fail(ctx, e, "fit setup");
  ctx->setup_stream = nullptr;
  t[4] = s->now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stats.cfg_create_s += t[1] - t[0];
    s->stats.cfg_upload_s += t[2] - t[1];
    s->stats.cfg_plan_s += t[3] - t[2];
    s->stats.cfg_buffers_s += t[4] - t[3];
  }
  if (rc) {
    release(ctx);
    return rc;
  }
  *out = ctx;
  return MUSR_OK;
}

// Moves a configured request into the active set.
void activate(musr_server* s, std::unique_ptr<Request> r, musr_ctx* ctx) {
  auto a = std::make_unique<Active>();
  a->ctx = ctx;
  a->shape = ctx->comp[r->prec][kServeVariant].hs.shape;
  musr_bins_in_fit(ctx, &a->bins);
  a->load = static_cast<double>(a->bins) * (1 + r->P);
  a->lane = s->lanes[0].load <= s->lanes[1].load ? 0 : 1;
  s->lanes[a->lane].load += a->load;
  a->t_admit = s->now();
  a->bfgs.start(r->x0.data(), r->P, r->gtol, r->maxit, 0.0, r->prec == MUSR_SPLIT ? kSplitEdm : kFp64Edm);
  // the counts are on the device now: drop the host copy (or forget the caller's buffer)
  std::vector<unsigned char>().swap(r->counts_copy);
  r->counts = nullptr;
  a->req = std::move(r);
  std::lock_guard<std::mutex> lock(s->mu);
  s->stats.active += 1;
  s->active.push_back(std::move(a));
}

// Device memory a request needs at most: its counts, and evaluation buffers for P + 1
// simultaneous points (the minimiser's widest step) with a generous bound on work items.
size_t estimate_bytes(const Request& r) {
  const size_t stride = static_cast<size_t>((r.B + 63) / 64 * 64);
  const size_t esz = r.dtype == MUSR_DTYPE_FP64 ? 8 : 4;
  size_t counts = static_cast<size_t>(r.H) * stride * esz;
  // histograms moved onto a common time grid pass through a packed scratch copy
  for (double t : r.t0)
    if (std::floor(t) != std::floor(r.t0[0])) {
      counts += static_cast<size_t>(r.H) * static_cast<size_t>(r.B) * esz + 8 * static_cast<size_t>(r.H) + 256;
      break;
    }
  const size_t items = (static_cast<size_t>(r.H) + 1) * (static_cast<size_t>(r.B) / 2048 + 2);
  const size_t rows = items * static_cast<size_t>(r.P + 1) * 100 * sizeof(double);  // <= 100 doubles a row
  return counts + rows + (size_t(4) << 20);
}

// Admits queued fits, first come first served, while there are free slots and the arena
// (the HBM budget) has room.  When the arena clearly holds a whole batch, the batch is
// configured by the helper threads in parallel (uploads and planning overlap); otherwise
// one at a time, so that a fit that waits for memory keeps its place.  With
// during_step, admission stops after the first batch once the device has finished the
// step's work, so that admitting barely lengthens a step (the rest waits for the next).
void admit(musr_server* s, bool during_step = false) {
  for (bool first = true;; first = false) {
    if (during_step && !first && cudaStreamQuery(s->stream) == cudaSuccess) return;
    const int room = s->max_active - static_cast<int>(s->active.size());
    if (room <= 0) return;
    std::vector<std::unique_ptr<Request>> batch;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->queue.empty()) return;
      size_t need = 0;
      const size_t free_bytes = s->arena.capacity() - s->arena.used();
      const int cap = s->admit_serial ? 1 : std::min(room, kAdmitBatch);
      while (!s->queue.empty() && static_cast<int>(batch.size()) < cap) {
        const size_t e = estimate_bytes(*s->queue.front());
        if (!batch.empty() && need + e > free_bytes / 2) break;
        need += e;
        batch.push_back(std::move(s->queue.front()));
        s->queue.pop_front();
        s->stats.queued -= 1;
      }
    }
    s->admit_serial = false;
    const int n = static_cast<int>(batch.size());
    std::vector<musr_ctx*> ctxs(n, nullptr);
    std::vector<int> rcs(n, MUSR_OK);
    s->pool->run(n, [&](int i) { rcs[i] = configure(s, *batch[i], &ctxs[i]); });
    for (int i = 0; i < n; ++i) {
      if (rcs[i] == MUSR_ENOMEM && (!s->active.empty() || n > 1)) {
        // The arena is full now: this fit and every later one of the batch go back to the
        // head of the queue in order (their memory released); retry one at a time.
        std::lock_guard<std::mutex> lock(s->mu);
        for (int j = n - 1; j >= i; --j) {
          release(ctxs[j]);
          s->queue.push_front(std::move(batch[j]));
          s->stats.queued += 1;
        }
        s->admit_serial = true;
        if (!s->active.empty()) return;  // wait for a running fit to release memory
        break;
      }
      if (rcs[i]) {
        reject(s, std::move(batch[i]), rcs[i]);
        continue;
      }
      bool canceled;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        canceled = s->cancel.count(batch[i]->id) > 0;
      }
      if (canceled) {  // canceled while it was configured: its setup was waited for
        release(ctxs[i]);
        reject(s, std::move(batch[i]), MUSR_ECANCELED);
        continue;
      }
      activate(s, std::move(batch[i]), ctxs[i]);
    }
  }
}

// Launches lane L: each of its fits names its next trial point(s), and all of them are
// evaluated by one multi-fit launch per group, queued on the stream behind whatever the
// other lane has in flight; the results come back to the lane's pinned buffer.
int launch_lane(musr_server* s, int L) {
  Lane& lane = s->lanes[L];
  // Fits of lane L asked to stop end here: lane L's last results were delivered in the
  // previous half-step, so none of their work is on the device.
  bool any_cancel;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    any_cancel = !s->cancel.empty();
  }
  if (any_cancel) {
    std::vector<Active*> stop;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto& a : s->active)
        if (a->lane == L && s->cancel.count(a->req->id)) stop.push_back(a.get());
    }
    if (!stop.empty()) {
      for (Active* a : stop) {
        lane.load -= a->load;
        finish(s, a, MUSR_ECANCELED);
      }
      std::lock_guard<std::mutex> lock(s->mu);
      s->stats.canceled += static_cast<int64_t>(stop.size());
      s->stats.completed -= static_cast<int64_t>(stop.size());
      std::vector<std::unique_ptr<Active>> keep;
      for (auto& a : s->active)
        if (a->ctx) keep.push_back(std::move(a));
      s->active.swap(keep);
    }
  }
  std::vector<Active*> fits;
  for (auto& a : s->active)
    if (a->lane == L) fits.push_back(a.get());
  lane.launched.clear();
  if (fits.empty()) return MUSR_OK;
  const double t_req = s->now();
  s->pool->run(static_cast<int>(fits.size()), [&](int i) { fits[i]->nvec = fits[i]->bfgs.request(&fits[i]->pts); });
  const double t_min = s->now() - t_req;
  size_t np = 0, no = 0;
  int nv = 0;
  for (Active* a : fits) {
    if (a->nvec == 0) continue;
    a->poff = np;
    a->ooff = no;
    np += static_cast<size_t>(a->nvec) * a->req->P;
    no += static_cast<size_t>(a->nvec) * (1 + a->req->P);
    nv += a->nvec;
    lane.launched.push_back(a);
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stats.minimizer_s += t_min;
  }
  if (lane.launched.empty()) return MUSR_OK;
  if (!grow_host(reinterpret_cast<void**>(&lane.h_params), &lane.hp_cap, (np + 1) * sizeof(double)) ||
      !grow_host(reinterpret_cast<void**>(&lane.h_out), &lane.ho_cap, (no + 1) * sizeof(double)) ||
      !grow_host(reinterpret_cast<void**>(&lane.h_jobs), &lane.hj_cap, (nv + 1) * sizeof(Job)) ||
      !grow_dev(&lane.d_params, &lane.dp_cap, (np + 1) * sizeof(double)) ||
      !grow_dev(&lane.d_out, &lane.do_cap, (no + 1) * sizeof(double)) ||
      !grow_dev(&lane.d_jobs, &lane.dj_cap, (nv + 1) * sizeof(Job)))
    return MUSR_ENOMEM;
  if (!lane.done && cudaEventCreateWithFlags(&lane.done, cudaEventDisableTiming) != cudaSuccess) return MUSR_ECUDA;
  for (Active* a : lane.launched)
    std::memcpy(lane.h_params + a->poff, a->pts.data(), static_cast<size_t>(a->nvec) * a->req->P * sizeof(double));
  // Group by (precision, shape, cost): one launch each, jobs contiguous per group.
  std::map<int, std::vector<Active*>> groups;
  for (Active* a : lane.launched) groups[(a->req->prec * 16 + a->shape) * 2 + a->req->mode].push_back(a);
  double* d_params = static_cast<double*>(lane.d_params);
  double* d_out = static_cast<double*>(lane.d_out);
  Job* d_jobs = static_cast<Job*>(lane.d_jobs);
  struct Launch {
    int prec, shape, mode, first, njobs, items;
  };
  std::vector<Launch> launches;
  int jpos = 0;
  for (auto& kv : groups) {
    Launch Lc{kv.second[0]->req->prec, kv.second[0]->shape, kv.second[0]->req->mode, jpos, 0, 0};
    for (Active* a : kv.second) {
      fill_jobs(a->ctx, Lc.prec, kServeVariant, Lc.mode, 1, a->nvec, d_params + a->poff, d_out + a->ooff,
                lane.h_jobs + jpos, Lc.items);
      Lc.items += a->nvec * a->ctx->comp[Lc.prec][kServeVariant].hs.nitems;
      Lc.njobs += a->nvec;
      jpos += a->nvec;
    }
    launches.push_back(Lc);
  }
  cudaError_t e = cudaMemcpyAsync(d_params, lane.h_params, np * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_jobs, lane.h_jobs, jpos * sizeof(Job), cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return MUSR_ECUDA;
  for (const Launch& Lc : launches) {
    if (Lc.items == 0) continue;
    LaunchInfo info;
    if (launch_eval(Lc.prec, Lc.shape, Lc.mode, 1, d_jobs + Lc.first, Lc.njobs, Lc.items, s->num_sms, s->stream,
                    &info))
      return MUSR_ECUDA;
  }
  e = cudaMemcpyAsync(lane.h_out, d_out, no * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(lane.done, s->stream);
  if (e != cudaSuccess) return MUSR_ECUDA;
  lane.in_flight = true;
  std::lock_guard<std::mutex> lock(s->mu);
  s->stats.steps += 1;
  s->stats.launches += static_cast<int64_t>(launches.size());
  s->stats.evals += nv;
  return MUSR_OK;
}

// Waits for lane L's results, advances its fits' minimisers (in parallel: fits are
// independent) and retires the finished ones.
int deliver_lane(musr_server* s, int L) {
  Lane& lane = s->lanes[L];
  if (!lane.in_flight) return MUSR_OK;
  const double t_wait = s->now();
  const cudaError_t e = cudaEventSynchronize(lane.done);
  lane.in_flight = false;
  if (e != cudaSuccess) return MUSR_ECUDA;
  const double t_del = s->now();
  const std::vector<Active*>& fits = lane.launched;
  s->pool->run(static_cast<int>(fits.size()), [&](int i) {
    Active* a = fits[i];
    const int P = a->req->P;
    a->f.resize(a->nvec);
    a->g.resize(static_cast<size_t>(a->nvec) * P);
    for (int v = 0; v < a->nvec; ++v) {
      const double* o = lane.h_out + a->ooff + static_cast<size_t>(v) * (1 + P);
      a->f[v] = o[0];
      std::memcpy(a->g.data() + static_cast<size_t>(v) * P, o + 1, sizeof(double) * P);
    }
    a->bfgs.deliver(a->f.data(), a->g.data());
    if (a->first && std::isfinite(a->f[0]) && a->req->prec == MUSR_SPLIT)
      a->bfgs.set_f_noise(kSplitNoiseRel * std::fabs(a->f[0]));
    a->first = false;
  });
  double bin_evals = 0.0;
  bool retired = false;
  for (Active* a : fits) {
    bin_evals += static_cast<double>(a->bins) * a->nvec;
    a->nvec = 0;
    if (a->bfgs.done()) {
      lane.load -= a->load;
      finish(s, a, a->bfgs.status());
      retired = true;
    }
  }
  lane.launched.clear();
  if (retired) {
    std::vector<std::unique_ptr<Active>> keep;
    for (auto& a : s->active)
      if (a->ctx) keep.push_back(std::move(a));
    s->active.swap(keep);
  }
  if (s->lanes[0].launched.empty() && s->lanes[1].launched.empty() && s->active.empty())
    s->lanes[0].load = s->lanes[1].load = 0.0;  // no drift from rounding
  std::lock_guard<std::mutex> lock(s->mu);
  s->stats.bin_evals += bin_evals;
  s->stats.wait_s += t_del - t_wait;
  s->stats.minimizer_s += s->now() - t_del;
  return MUSR_OK;
}

// Ends every running fit with `status` after a failed launch or wait.
void fail_all(musr_server* s, int status) {
  cudaStreamSynchronize(s->stream);
  cudaGetLastError();
  for (auto& ln : s->lanes) {
    ln.in_flight = false;
    ln.launched.clear();
    ln.load = 0.0;
  }
  std::vector<std::unique_ptr<Active>> act;
  act.swap(s->active);
  for (auto& a : act) finish(s, a.get(), status);
  s->worker_error = "serving step failed";
}

void worker_main(musr_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    const bool idle = s->active.empty() && !s->lanes[0].in_flight && !s->lanes[1].in_flight;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (idle) s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
    }
    if (idle) {
      admit(s);
      if (s->active.empty()) continue;
    }
    // Half-step: launch lane L behind the other lane's work, admit while the device
    // runs, then take the other lane's results.
    const int L = s->next_lane;
    s->next_lane = 1 - L;
    const double t = s->now();
    int rc = launch_lane(s, L);
    if (!rc) {
      const double t_adm = s->now();
      admit(s, true);
      const double t_adm_end = s->now();
      std::lock_guard<std::mutex> lock(s->mu);
      s->stats.admit_s += t_adm_end - t_adm;
    }
    if (!rc) rc = deliver_lane(s, 1 - L);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stats.busy_s += s->now() - t;
    }
    if (rc) fail_all(s, rc);  // a CUDA failure ends every running fit with that status
  }
  cudaStreamSynchronize(s->stream);
  for (auto& a : s->active) release(a->ctx);
  s->active.clear();
}

bool copy_request(const musr_fit_request* q, Request* r, std::string* why) {
  if (!q->counts || !q->t0 || !q->map || !q->x0 || (q->nterms > 0 && !q->terms) ||
      (q->nconsts > 0 && !q->consts)) {
    *why = "NULL pointer in the request";
    return false;
  }
  if (q->nhist < 1 || q->nbins < 1 || q->nslots < 2 || q->nslots > MUSR_MAX_SLOTS || q->nparams < 0 ||
      q->nparams > MUSR_MAX_PARAMS || q->nterms < 0 || q->nterms > MUSR_MAX_TERMS || q->nconsts < 0) {
    *why = "size out of range";
    return false;
  }
  if (q->dtype != MUSR_DTYPE_INT32 && q->dtype != MUSR_DTYPE_FP32 && q->dtype != MUSR_DTYPE_FP64) {
    *why = "bad dtype";
    return false;
  }
  if ((q->mode != MUSR_CHI2 && q->mode != MUSR_MLE) || (q->precision != MUSR_FP64 && q->precision != MUSR_SPLIT)) {
    *why = "bad mode or precision";
    return false;
  }
  for (int k = 0; k < q->nterms; ++k)
    for (int m = 0; m < q->terms[k].nprim && m < MUSR_MAX_PRIMS; ++m)
      if (q->terms[k].kind[m] == MUSR_PRIM_DKT) {
        *why = "the dynamic Kubo-Toyabe primitive needs tables solved per evaluation: fit it with a context";
        return false;
      }
  const size_t n = static_cast<size_t>(q->nhist) * q->nbins * dtype_size(q->dtype);
  if (q->flags & ~MUSR_REQ_BORROW_COUNTS) {
    *why = "unknown request flags";
    return false;
  }
  if (q->flags & MUSR_REQ_BORROW_COUNTS) {
    r->counts = q->counts;
  } else {
    r->counts_copy.assign(static_cast<const unsigned char*>(q->counts),
                          static_cast<const unsigned char*>(q->counts) + n);
    r->counts = r->counts_copy.data();
  }
  r->dtype = q->dtype;
  r->H = q->nhist;
  r->B = q->nbins;
  r->t0.assign(q->t0, q->t0 + q->nhist);
  r->bw = q->bin_width_ns;
  r->fr[0] = q->fit_range_us[0];
  r->fr[1] = q->fit_range_us[1];
  r->terms.assign(q->terms, q->terms + q->nterms);
  r->map.assign(q->map, q->map + static_cast<size_t>(q->nhist) * q->nslots);
  r->nslots = q->nslots;
  r->P = q->nparams;
  r->consts.assign(q->consts, q->consts + q->nconsts);
  r->x0.assign(q->x0, q->x0 + q->nparams);
  r->mode = q->mode;
  r->prec = q->precision;
  r->maxit = q->maxit > 0 ? q->maxit : 1000;
  r->gtol = q->gtol > 0 ? q->gtol : 1e-8;
  for (double v : r->x0)
    if (!std::isfinite(v)) {
      *why = "x0 must be finite";
      return false;
    }
  return true;
}

}  // namespace

extern "C" {

int musr_server_create(musr_server** out, int device, size_t hbm_budget_bytes, int max_active) {
  if (!out) return MUSR_EINVAL;
  *out = nullptr;
  if (max_active < 1 || hbm_budget_bytes < (size_t(1) << 20)) return MUSR_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return MUSR_ECUDA;
  }
  if (device < 0 || device >= ndev) return MUSR_EINVAL;
  auto s = std::make_unique<musr_server>();
  s->device = device;
  s->max_active = max_active;
  s->t0 = std::chrono::steady_clock::now();
  DeviceScope ds(device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return MUSR_ECUDA;
  if (s->arena.init(hbm_budget_bytes)) {
    cudaStreamDestroy(s->stream);
    return MUSR_ENOMEM;
  }
  s->stats.arena_bytes = s->arena.capacity();
  const unsigned hw = std::thread::hardware_concurrency();
  s->pool = std::make_unique<TaskPool>(hw > 2 ? static_cast<int>(std::min(hw - 2, 15u)) : 0, device);
  s->worker = std::thread(worker_main, s.get());
  *out = s.release();
  return MUSR_OK;
}

void musr_server_destroy(musr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  DeviceScope ds(s->device);
  cudaStreamSynchronize(s->stream);
  for (auto& ln : s->lanes) {
    if (ln.h_params) cudaFreeHost(ln.h_params);
    if (ln.h_out) cudaFreeHost(ln.h_out);
    if (ln.h_jobs) cudaFreeHost(ln.h_jobs);
    if (ln.d_params) cudaFree(ln.d_params);
    if (ln.d_out) cudaFree(ln.d_out);
    if (ln.d_jobs) cudaFree(ln.d_jobs);
    if (ln.done) cudaEventDestroy(ln.done);
  }
  cudaStreamDestroy(s->stream);
  delete s;
}

int musr_server_submit(musr_server* s, const musr_fit_request* req, int64_t* out_id) {
  if (!s || !req || !out_id) return MUSR_EINVAL;
  auto r = std::make_unique<Request>();
  std::string why;
  if (!copy_request(req, r.get(), &why)) {
    std::lock_guard<std::mutex> lock(s->mu);
    s->err = why;
    return MUSR_EINVAL;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return MUSR_ESTATE;
  r->id = s->next_id++;
  r->t_submit = s->now();
  *out_id = r->id;
  s->live.insert(r->id);
  s->queue.push_back(std::move(r));
  s->stats.submitted += 1;
  s->stats.queued += 1;
  s->cv_work.notify_one();
  return MUSR_OK;
}

static int take_result(musr_server* s, int64_t id, musr_fit_result* res, double* x_out) {
  auto it = s->done.find(id);
  if (it == s->done.end()) return MUSR_EAGAIN;
  if (res) *res = it->second.res;
  if (x_out) std::memcpy(x_out, it->second.x.data(), sizeof(double) * it->second.x.size());
  s->done.erase(it);
  return MUSR_OK;
}

int musr_server_poll(musr_server* s, int64_t id, musr_fit_result* res, double* x_out) {
  if (!s || id <= 0) return MUSR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (id >= s->next_id) return MUSR_EINVAL;
  return take_result(s, id, res, x_out);
}

int musr_server_wait(musr_server* s, int64_t id, int timeout_ms, musr_fit_result* res, double* x_out) {
  if (!s || id <= 0) return MUSR_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  if (id >= s->next_id) return MUSR_EINVAL;
  auto ready = [&] { return s->done.count(id) > 0; };
  if (timeout_ms > 0) {
    if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return MUSR_ETIMEOUT;
  } else {
    s->cv_done.wait(lock, ready);
  }
  return take_result(s, id, res, x_out);
}

int musr_server_cancel(musr_server* s, int64_t id) {
  if (!s || id <= 0) return MUSR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (id >= s->next_id) return MUSR_EINVAL;
  if (s->done.count(id)) return MUSR_ESTATE;  // finished: its result stands
  if (!s->live.count(id)) return MUSR_EINVAL;  // its result was taken already
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if ((*it)->id == id) {  // still queued: ends now, without running
      std::unique_ptr<Request> r = std::move(*it);
      s->queue.erase(it);
      s->stats.queued -= 1;
      reject_locked(s, std::move(r), MUSR_ECANCELED);
      return MUSR_OK;
    }
  // being admitted or active: the worker ends it at its next step boundary
  s->cancel.insert(id);
  s->cv_work.notify_one();
  return MUSR_OK;
}

int musr_server_stats_get(musr_server* s, musr_server_stats* out) {
  if (!s || !out) return MUSR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->arena_used = s->arena.used();
  out->clock_s = s->now();
  return MUSR_OK;
}

// One fit on a configured context, synchronous: the same minimiser as the
// serving loop, each request (one point, or P points for the curvature
// estimate) one batched launch.
int musr_fit(musr_ctx* ctx, const double* x0, int mode, int precision, int maxit, double gtol, double* x_out,
             musr_fit_result* res) {
  if (!ctx || !x0 || !x_out || !res) return MUSR_EINVAL;
  const int P = ctx->P;
  Bfgs b;
  b.start(x0, P, gtol > 0 ? gtol : 1e-8, maxit > 0 ? maxit : 1000, 0.0,
          precision == MUSR_SPLIT ? kSplitEdm : kFp64Edm);
  std::vector<double> pts, vals, grads;
  bool first = true;
  const auto t0 = std::chrono::steady_clock::now();
  while (!b.done()) {
    const int n = b.request(&pts);
    vals.resize(n);
    grads.resize(static_cast<size_t>(n) * P);
    const int rc = musr_eval_batch(ctx, pts.data(), n, P, mode, precision, vals.data(), grads.data());
    if (rc != MUSR_OK && rc != MUSR_ENONFINITE) return rc;
    b.deliver(vals.data(), grads.data());
    if (first && std::isfinite(vals[0]) && precision == MUSR_SPLIT) b.set_f_noise(kSplitNoiseRel * std::fabs(vals[0]));
    first = false;
  }
  std::memset(res, 0, sizeof(*res));
  res->status = b.status();
  res->iters = b.iters();
  res->nfev = b.nfev();
  res->nparams = P;
  res->f = b.f();
  res->edm = b.edm();
  res->t_done = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  std::memcpy(x_out, b.x().data(), sizeof(double) * P);
  return MUSR_OK;
}

}  // extern "C"
