// Serving loop: continuous batching of amplitude requests over resident plans.
//
// Requests (plan, bitstrings, precision, output) are queued by tn_server_submit. Worker threads,
// each with its own CUDA stream and its own workspaces, take the oldest admissible request and
// merge into it the other queued requests for the same plan and precision (up to the plan's
// batch size), run them as one device batch (the tn_amplitudes path), and scatter the results.
// A request is admissible when the device memory of its batch fits the HBM budget next to the
// batches in flight, so requests that arrive while others run are started as soon as a worker
// and memory are free, and their work overlaps on the device. A worker's workspace lives only as
// long as its batch (it is released when the batch ends), so the device memory the server holds is
// the sum of the admitted batches' footprints. Latency = completion - submission.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tn_host.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  tn_plan *plan = nullptr;
  std::vector<uint64_t> bits;   // copied at submission
  int64_t n = 0;
  tn_precision prec = TN_FP64;
  tn_c128 *out = nullptr;
  double t_submit = 0, t_done = 0;
  tn_status status = TN_OK;
  std::string error;
  bool done = false;
};

}  // namespace

struct tn_server {
  tn_server_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, Request *> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_ticket = 1;
  double admitted = 0, peak_admitted = 0;
  int inflight = 0, max_inflight_seen = 0;
  double busy_since = -1, busy_total = 0;
  int64_t submitted = 0, completed = 0, failed = 0, rejected = 0, amplitudes = 0, cancelled = 0;
  std::vector<double> latencies;
};

namespace {

int words_of(const tn_plan *p) { return (p->c->n + 63) / 64; }

// device bytes of a batch of n bitstrings of plan p in precision prec
double footprint(const tn_plan *p, tn_precision prec, int64_t n) {
  const int kind = prec == TN_FP64 ? 0 : 1;
  const int64_t ch = std::min<int64_t>(n, p->chunk[kind]);
  return (double)plan_ws_bytes(p, kind, std::max<int64_t>(ch, 1), p->slice_chunk[kind]);
}

void worker_main(tn_server *s, int wid) {
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // oldest request whose batch fits the budget next to the batches in flight
    Request *head = nullptr;
    double need = 0;
    for (;;) {
      head = nullptr;
      for (Request *r : s->queue) {
        need = footprint(r->plan, r->prec, r->n);
        if (s->inflight == 0 || s->admitted + need <= s->cfg.hbm_budget_bytes) { head = r; break; }
      }
      if (head || (s->stop && s->queue.empty())) break;
      s->cv_work.wait(lk);
    }
    if (!head) break;
    // merge the queued requests of the same plan and precision into one batch
    std::vector<Request *> batch{head};
    int64_t total = head->n;
    const int kind = head->prec == TN_FP64 ? 0 : 1;
    const int64_t cap = std::max<int64_t>(head->plan->chunk[kind], head->n);
    for (Request *r : s->queue)
      if (r != head && r->plan == head->plan && r->prec == head->prec && total + r->n <= cap &&
          (s->inflight == 0 || s->admitted + footprint(head->plan, head->prec, total + r->n) <= s->cfg.hbm_budget_bytes)) {
        batch.push_back(r);
        total += r->n;
      }
    for (Request *r : batch) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    need = footprint(head->plan, head->prec, total);
    s->admitted += need;
    s->peak_admitted = std::max(s->peak_admitted, s->admitted);
    if (s->inflight++ == 0) s->busy_since = now_s();
    s->max_inflight_seen = std::max(s->max_inflight_seen, s->inflight);
    lk.unlock();

    // run: one device batch for the merged requests
    tn_plan *p = head->plan;
    const int words = words_of(p);
    std::vector<uint64_t> bits((size_t)total * words);
    std::vector<tn_c128> res((size_t)total);
    int64_t off = 0;
    for (Request *r : batch) {
      std::memcpy(bits.data() + off * words, r->bits.data(), (size_t)r->n * words * 8);
      off += r->n;
    }
    Workspace ws;   // this batch's buffers, released before its footprint leaves the admitted sum
    tn_status status = run_amplitudes(p, ws, bits.data(), total, head->prec, res.data(), st);
    std::string err = status == TN_OK ? std::string() : std::string(tn_last_error());
    if (st) cudaStreamSynchronize(st);
    ws_release(p->c->mem, ws);
    const double t = now_s();

    lk.lock();
    off = 0;
    for (Request *r : batch) {
      if (status == TN_OK) std::memcpy(r->out, res.data() + off, (size_t)r->n * sizeof(tn_c128));
      off += r->n;
      r->status = status;
      r->error = err;
      r->t_done = t;
      r->done = true;
      if (status == TN_OK) {
        s->completed++;
        s->amplitudes += r->n;
        s->latencies.push_back(t - r->t_submit);
      } else {
        s->failed++;
      }
    }
    s->admitted -= need;
    if (--s->inflight == 0) s->busy_total += t - s->busy_since;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  lk.unlock();
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  (void)wid;
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" tn_status tn_server_create(const tn_server_cfg *cfg, tn_server **out) {
  if (!out) return tn_fail(TN_ERR_ARG, "tn_server_create: out is NULL");
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return tn_fail(TN_ERR_CUDA, "no CUDA device available: the server has no CPU fallback");
  }
  tn_server *s = new tn_server();
  if (cfg) s->cfg = *cfg;
  if (!(s->cfg.hbm_budget_bytes > 0)) s->cfg.hbm_budget_bytes = 16.0 * (1ull << 30);
  if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 4;
  if (s->cfg.n_streams <= 0) s->cfg.n_streams = s->cfg.max_inflight;
  const int nw = std::min(s->cfg.max_inflight, s->cfg.n_streams);
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < nw; ++i)
    s->workers.emplace_back([s, i, dev] {
      cudaSetDevice(dev);
      worker_main(s, i);
    });
  *out = s;
  return TN_OK;
}

extern "C" tn_status tn_server_submit(tn_server *s, tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                                      tn_c128 *out, uint64_t *ticket) {
  if (!s || !p || !ticket || n < 0 || (n > 0 && (!bits || !out)))
    return tn_fail(TN_ERR_ARG, "tn_server_submit: bad arguments");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  if (p->generation != p->c->generation) return tn_fail(TN_ERR_STATE, "plan is stale: the circuit was re-evolved");
  const double need = footprint(p, prec, std::max<int64_t>(n, 1));
  std::lock_guard<std::mutex> lk(s->mu);
  if (need > s->cfg.hbm_budget_bytes) {
    s->rejected++;
    return tn_fail(TN_ERR_OOM, "request needs %.0f bytes of device memory, more than the server budget %.0f", need,
                   s->cfg.hbm_budget_bytes);
  }
  Request *r = new Request();
  r->ticket = s->next_ticket++;
  r->plan = p;
  r->n = n;
  r->prec = prec;
  r->out = out;
  r->bits.assign(bits, bits + (size_t)n * words_of(p));
  r->t_submit = now_s();
  s->reqs[r->ticket] = r;
  s->submitted++;
  *ticket = r->ticket;
  if (n == 0) {
    r->done = true;
    r->t_done = r->t_submit;
    s->completed++;
    s->latencies.push_back(0);
    return TN_OK;
  }
  s->queue.push_back(r);
  s->cv_work.notify_one();
  return TN_OK;
}

extern "C" tn_status tn_server_wait(tn_server *s, uint64_t ticket, int64_t timeout_ms) {
  if (!s) return tn_fail(TN_ERR_ARG, "tn_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return tn_fail(TN_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  Request *r = it->second;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, [&] { return r->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) {
    return tn_fail(TN_ERR_TIMEOUT, "ticket %llu not complete after %lld ms", (unsigned long long)ticket,
                   (long long)timeout_ms);
  }
  const tn_status st = r->status;
  if (st != TN_OK) tn_fail(st, "%s", r->error.c_str());
  s->reqs.erase(it);
  delete r;
  return st;
}

extern "C" tn_status tn_server_cancel(tn_server *s, uint64_t ticket) {
  if (!s) return tn_fail(TN_ERR_ARG, "tn_server_cancel: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return tn_fail(TN_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  Request *r = it->second;
  auto q = std::find(s->queue.begin(), s->queue.end(), r);
  if (q == s->queue.end())
    return tn_fail(TN_ERR_STATE, "ticket %llu is %s: only queued requests can be cancelled",
                   (unsigned long long)ticket, r->done ? "complete" : "running");
  s->queue.erase(q);
  s->reqs.erase(it);
  delete r;
  s->cancelled++;
  s->cv_work.notify_all();   // the budget a worker was waiting on may have been this request's
  return TN_OK;
}

extern "C" tn_status tn_server_stats_get(tn_server *s, tn_server_stats *o) {
  if (!s || !o) return tn_fail(TN_ERR_ARG, "tn_server_stats_get: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(o, 0, sizeof *o);
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->rejected = s->rejected;
  o->amplitudes = s->amplitudes;
  o->busy_seconds = s->busy_total + (s->inflight > 0 ? now_s() - s->busy_since : 0);
  o->p50_latency_s = percentile(s->latencies, 0.50);
  o->p99_latency_s = percentile(s->latencies, 0.99);
  o->max_inflight_seen = s->max_inflight_seen;
  o->peak_admitted_bytes = s->peak_admitted;
  o->cancelled = s->cancelled;
  return TN_OK;
}

extern "C" void tn_server_free(tn_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
}
