// serve.cu -- continuous-batching request loop (hlc_serve_*).
//
// Requests (locations, data, theta, parameters) are queued with copies of
// their inputs.  A fixed set of slot workers, each with its own context
// (stream, workspaces), admit requests in arrival order as slots and device
// memory free up: a request is admitted when its estimated device footprint
// fits in what the budget has left.  An admitted request builds its tree and
// runs one likelihood evaluation on its slot's stream, so the work of all
// admitted requests overlaps on the device.  Results stay until polled.  Every evaluation follows its own fixed plan
// with fixed-order reductions, so a result does not depend on what else runs.

#include <math.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hlc.h"
#include "serve.h"

namespace hlc {

struct Request {
  uint64_t id = 0;
  std::vector<double> xy, z;
  int64_t n = 0;
  hlc_theta th{};
  hlc_params p{};
  int status = HLC_PENDING;
  hlc_result res{};
  size_t footprint = 0;
  std::chrono::steady_clock::time_point t_submit;
};

// The admission rule of the request loop, kept apart from the threads so
// that it can be replayed on the host: the request at the head of the queue
// is admitted when a slot is free and its footprint fits in what the budget
// has left, or when nothing else is running (a request larger than the
// whole budget then runs alone rather than never).  Arrival order is kept.
struct Admission {
  size_t budget = 0;
  int max_slots = 1;
  size_t in_use = 0;
  int running = 0;
  size_t peak = 0;
  bool fits(size_t fp) const {
    return running < max_slots && (in_use + fp <= budget || running == 0);
  }
  void admit(size_t fp) {
    in_use += fp;
    running += 1;
    if (in_use > peak) peak = in_use;
  }
  void release(size_t fp) {
    in_use -= fp;
    running -= 1;
  }
};

struct Serve {
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_id = 1;
  Admission adm;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<hlc_ctx*> slot_ctx;
};

// Device footprint estimate of one evaluation before its tree exists: two
// arenas (C~ and L~) of n (3 leaf + 7.5 log2(n / leaf) kmax) doubles -- the
// dense near field plus low-rank blocks of kmax columns whose summed row
// count grows like n log n on uniform points -- plus temporaries and
// vectors.  Low-rank blocks narrower than kmax reserve fewer columns, so the
// estimate errs on the high side for small trees.
size_t serve_footprint(int64_t n, const hlc_params& p) {
  const double lv = log2(fmax(2.0, (double)n / p.leaf));
  const double arena = 8.0 * n * (3.0 * p.leaf + 7.5 * lv * p.kmax);
  return (size_t)(2.6 * arena + 64.0 * n + (64 << 20));
}

}  // namespace hlc

using namespace hlc;

namespace {

// The slot workers use the public API only.
void worker(hlc::Serve* S, int slot) {
  hlc_ctx* c = S->slot_ctx[slot];
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->queue.empty()) return S->stopping;
        return S->adm.fits(S->queue.front()->footprint);
      });
      if (S->queue.empty()) return;  // stopping and drained
      r = S->queue.front();
      S->queue.pop_front();
      S->adm.admit(r->footprint);
    }
    hlc_tree* t = nullptr;
    hlc_result res{};
    int st = hlc_build_tree(c, r->xy.data(), r->n, &r->p, &t);
    if (st == HLC_OK) st = hlc_loglik(c, t, &r->th, r->z.data(), &res);
    if (t) hlc_tree_free(t);
    // A mixed-precision factorisation can meet a non-positive pivot where
    // the FP64 one does not (smooth kernels, small nugget): such a request is
    // evaluated again in FP64 rather than failed.
    if ((st == HLC_ERR_NOT_SPD || st == HLC_ERR_NUMERIC) && r->p.precision != HLC_FP64) {
      hlc_params p64 = r->p;
      p64.precision = HLC_FP64;
      t = nullptr;
      res = hlc_result{};
      st = hlc_build_tree(c, r->xy.data(), r->n, &p64, &t);
      if (st == HLC_OK) st = hlc_loglik(c, t, &r->th, r->z.data(), &res);
      if (t) hlc_tree_free(t);
    }
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->t_submit).count();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->adm.release(r->footprint);
      res.ms_total = ms;
      r->res = res;
      r->status = st;
    }
    S->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int hlc_serve_start(hlc_ctx* ctx, size_t budget, int max_slots) {
  if (!ctx || max_slots < 1 || max_slots > 64 || budget == 0) return HLC_ERR_ARG;
  hlc::Serve*& S = serve_of(ctx);
  if (S) return HLC_ERR_STATE;
  std::unique_ptr<hlc::Serve> s(new (std::nothrow) hlc::Serve());
  if (!s) return HLC_ERR_OOM;
  s->device = device_of(ctx);
  s->adm.budget = budget;
  s->adm.max_slots = max_slots;
  for (int i = 0; i < max_slots; ++i) {
    hlc_ctx* c = nullptr;
    const int st = hlc_create(&c, s->device);
    if (st != HLC_OK) {
      for (hlc_ctx* x : s->slot_ctx) hlc_destroy(x);
      return st;
    }
    // Slots share the SMs, so their solves use wave-by-wave launches: a
    // grid-barrier kernel needs all of its CTAs resident at once.
    set_persistent(c, false);
    s->slot_ctx.push_back(c);
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker, s.get(), i);
  S = s.release();
  return HLC_OK;
}

int hlc_serve_submit(hlc_ctx* ctx, const double* xy, const double* z, int64_t n, const hlc_theta* th,
                     const hlc_params* p, uint64_t* req_id) {
  if (!ctx || !xy || !z || n <= 0 || !th || !req_id) return HLC_ERR_ARG;
  hlc::Serve* S = serve_of(ctx);
  if (!S) return HLC_ERR_STATE;
  auto r = std::make_shared<Request>();
  r->xy.assign(xy, xy + 2 * n);
  r->z.assign(z, z + n);
  r->n = n;
  r->th = *th;
  if (p)
    r->p = *p;
  else
    hlc_default_params(&r->p);
  r->footprint = serve_footprint(n, r->p);
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return HLC_ERR_STATE;
    r->id = S->next_id++;
    S->all[r->id] = r;
    S->queue.push_back(r);
    *req_id = r->id;
  }
  S->cv.notify_all();
  return HLC_OK;
}

int hlc_serve_poll(hlc_ctx* ctx, uint64_t req_id, hlc_result* out) {
  if (!ctx || !out) return HLC_ERR_ARG;
  hlc::Serve* S = serve_of(ctx);
  if (!S) return HLC_ERR_STATE;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(req_id);
  if (it == S->all.end()) return HLC_ERR_ARG;
  if (it->second->status == HLC_PENDING) return HLC_PENDING;
  *out = it->second->res;
  const int st = it->second->status;
  S->all.erase(it);
  return st;
}

size_t hlc_serve_footprint(int64_t n, const hlc_params* p) {
  hlc_params q;
  if (p)
    q = *p;
  else
    hlc_default_params(&q);
  if (n <= 0 || q.leaf < 1 || q.kmax < 1) return 0;
  return serve_footprint(n, q);
}

int hlc_serve_admission_replay(size_t budget, int max_slots, int64_t nreq, const size_t* footprint,
                               const double* duration, double* start, size_t* peak) {
  if (budget == 0 || max_slots < 1 || nreq < 0 || (nreq > 0 && (!footprint || !duration || !start)) || !peak)
    return HLC_ERR_ARG;
  hlc::Admission adm;
  adm.budget = budget;
  adm.max_slots = max_slots;
  struct Run {
    double end;
    size_t fp;
  };
  std::vector<Run> run;
  double now = 0.0;
  int64_t head = 0;
  while (head < nreq || !run.empty()) {
    // admit from the head of the queue while the rule allows
    while (head < nreq && adm.fits(footprint[head])) {
      if (!(duration[head] >= 0.0)) return HLC_ERR_ARG;
      adm.admit(footprint[head]);
      start[head] = now;
      run.push_back(Run{now + duration[head], footprint[head]});
      ++head;
    }
    if (run.empty()) break;  // cannot happen: an empty loop admits the head
    // advance to the next completion
    size_t first = 0;
    for (size_t i = 1; i < run.size(); ++i)
      if (run[i].end < run[first].end) first = i;
    now = run[first].end;
    adm.release(run[first].fp);
    run.erase(run.begin() + (std::ptrdiff_t)first);
  }
  *peak = adm.peak;
  return HLC_OK;
}

int hlc_serve_stop(hlc_ctx* ctx) {
  if (!ctx) return HLC_ERR_ARG;
  hlc::Serve*& S = serve_of(ctx);
  if (!S) return HLC_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv.notify_all();
  for (std::thread& w : S->workers) w.join();
  for (hlc_ctx* c : S->slot_ctx) hlc_destroy(c);
  delete S;
  S = nullptr;
  return HLC_OK;
}

}  // extern "C"
