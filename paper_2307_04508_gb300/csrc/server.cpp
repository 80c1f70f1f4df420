// Request server for G0W0 solves: continuous admission of requests of mixed
// sizes onto a fixed set of worker slots.
//
// Each slot owns an ltgw context and a non-blocking CUDA stream, and runs one
// solve at a time on a host thread of its own, so the kernels of different
// requests overlap on the device.  A request is admitted as soon as a slot is
// free and its estimated device footprint fits in what the budget leaves
// after the requests already running.  Admission goes in arrival order, but a
// request that does not fit may be passed by later ones that do, at most
// kMaxBypass times: after that nothing is admitted ahead of it, so a large
// request waits for memory to drain instead of starving behind small ones.
// Completions record the queueing, service and total latency of every request.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ltgw.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  uint64_t ticket = 0;
  ltgw_request req{};
  size_t footprint = 0;
  Clock::time_point t_submit;
  int bypassed = 0;   // later requests admitted ahead of this one
  int retries = 0;    // solves that ran out of device memory
  bool alone = false;        // admitted with nothing else running
  bool after_trim = false;   // re-run alone after the idle slots released their workspace
};

constexpr int kMaxBypass = 8;
// A request that runs out of device memory beside others goes back with its
// footprint doubled until it runs alone; one that fails alone is re-run once
// after the idle slots released their workspace.  Doubling from the smallest
// footprint (64 MiB) reaches any budget within 40 retries.
constexpr int kMaxRetries = 40;

struct Slot {
  std::thread th;
  bool has_job = false;
  Pending job;
  size_t retained = 0;       // workspace its context keeps between requests
  ltgw_ctx *ctx = nullptr;   // used by its own thread only, except that an idle slot's
                             // workspace may be released under the server's lock
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct ltgw_server {
  int device = 0;
  size_t budget = 0, in_flight = 0;
  size_t retained = 0;   // workspace kept by the slots between requests
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::list<Pending> queue;   // erasing one request keeps pointers to the others valid
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<ltgw_completion> done;
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  ltgw_status init_status = LTGW_OK;
  int init_pending = 0;
  Clock::time_point t_created = Clock::now();

  // Admit queued requests while a slot is free: the oldest that fits in the
  // remaining budget first; a request that does not fit is passed (and
  // counted) until it has been passed kMaxBypass times, after which the scan
  // stops at it.  With nothing running, the oldest request is admitted
  // whatever its footprint.  Caller holds mu.
  void dispatch_locked() {
    std::vector<Pending *> passed;
    auto it = queue.begin();
    while (it != queue.end()) {
      Slot *free_slot = nullptr;
      for (auto &s : slots)
        if (!s->has_job && !busy_slot(s.get())) { free_slot = s.get(); break; }
      if (!free_slot) return;
      const bool fits = in_flight + retained + it->footprint <= budget || running == 0;
      if (!fits) {
        if (it->bypassed >= kMaxBypass) return;
        passed.push_back(&*it);
        ++it;
        continue;
      }
      for (Pending *q : passed) ++q->bypassed;
      free_slot->job = *it;
      free_slot->job.alone = running == 0;
      free_slot->has_job = true;
      in_flight += it->footprint;
      ++running;
      it = queue.erase(it);
      cv_work.notify_all();
    }
  }
  std::vector<Slot *> busy;
  bool busy_slot(Slot *s) const { return std::find(busy.begin(), busy.end(), s) != busy.end(); }

  void worker(Slot *slot) {
    cudaSetDevice(device);
    ltgw_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    ltgw_status st = ltgw_create(&ctx, device);
    if (st == LTGW_OK && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = LTGW_ERR_DEVICE;
    }
    {
      std::lock_guard<std::mutex> lock(mu);
      slot->ctx = ctx;
      if (st != LTGW_OK && init_status == LTGW_OK) init_status = st;
      --init_pending;
      cv_done.notify_all();
    }
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
      cv_work.wait(lock, [&] { return stop || slot->has_job; });
      if (!slot->has_job) break;
      Pending job = slot->job;
      slot->has_job = false;
      busy.push_back(slot);
      lock.unlock();
      const Clock::time_point t_start = Clock::now();
      ltgw_status rs = LTGW_ERR_DEVICE;
      if (ctx) {
        const ltgw_request &r = job.req;
        rs = ltgw_solve(ctx, &r.p, r.eps, r.B_ov, r.B_tgt, r.targets, r.n_tgt, r.shift, r.tau_x, r.tau_w,
                        r.sigma_iw, r.e_qp, r.qp_status, stream);
      }
      const Clock::time_point t_end = Clock::now();
      // a slot keeps at most its share of a quarter of the budget between requests;
      // what it keeps counts against admission (see dispatch_locked)
      size_t keep = 0;
      if (ctx) {
        if (rs == LTGW_ERR_NOMEM || ltgw_workspace_bytes(ctx) > budget / (4 * slots.size())) ltgw_trim(ctx);
        keep = ltgw_workspace_bytes(ctx);
      }
      lock.lock();
      busy.erase(std::find(busy.begin(), busy.end(), slot));
      in_flight -= job.footprint;
      retained += keep - slot->retained;
      slot->retained = keep;
      --running;
      // Out of device memory.  Beside other requests the estimate was short: the
      // request goes back to the head of the queue with its footprint doubled (at
      // most the budget: then it runs alone).  Alone, the idle slots' retained
      // workspace may be what was missing: they release it (their threads are
      // waiting for work, their contexts unused), and the request runs alone
      // once more.  Failing after that, it fails.
      if (rs == LTGW_ERR_NOMEM && job.retries < kMaxRetries && !(job.alone && job.after_trim)) {
        job.retries++;
        if (job.alone) {
          for (auto &o : slots)
            if (o.get() != slot && !o->has_job && !busy_slot(o.get()) && o->ctx && o->retained) {
              ltgw_trim(o->ctx);
              retained -= o->retained;
              o->retained = 0;
            }
          job.after_trim = true;
          job.footprint = budget;
        } else {
          job.footprint = std::min(budget, 2 * job.footprint);
        }
        job.bypassed = kMaxBypass;   // nothing passes it again
        queue.push_front(job);
        dispatch_locked();
        cv_done.notify_all();
        continue;
      }
      ltgw_completion c{};
      c.ticket = job.ticket;
      c.status = rs;
      c.queue_ms = ms_between(job.t_submit, t_start);
      c.service_ms = ms_between(t_start, t_end);
      c.latency_ms = ms_between(job.t_submit, t_end);
      c.start_ms = ms_between(t_created, t_start);
      c.end_ms = ms_between(t_created, t_end);
      if (rs != LTGW_OK && ctx) {
        const char *m = ltgw_last_error(ctx);
        size_t k = 0;
        for (; m && m[k] && k + 1 < sizeof(c.message); ++k) c.message[k] = m[k];
        c.message[k] = 0;
      }
      done.push_back(c);
      dispatch_locked();
      cv_done.notify_all();
    }
    slot->ctx = nullptr;   // no other thread reaches the context from here on
    lock.unlock();
    if (stream) cudaStreamDestroy(stream);
    if (ctx) ltgw_destroy(ctx);
  }
};

extern "C" {

size_t ltgw_request_footprint(const ltgw_params *p, int n_tgt) {
  if (!p || n_tgt < 1) return 0;
  const size_t n_aux = (size_t)p->n_aux, n_occ = (size_t)p->n_occ, n_virt = (size_t)p->n_virt;
  const size_t n_orb = n_occ + n_virt, n_act = n_occ - (size_t)p->n_frozen;
  // N: auxiliary functions after the NAF step, not known before the solve;
  // estimated as half of n_aux with NAF on (a request whose solve then runs
  // out of memory beside others is retried by the server with more room)
  const size_t n_ov = n_act * n_virt, T = (size_t)n_tgt, n_om = (size_t)p->n_omega;
  const size_t N = p->naf_thresh >= 0.0 ? (n_aux + 1) / 2 : n_aux;
  const size_t n_tau = p->use_laplace ? (size_t)p->n_tau : 0;
  size_t d = 0;  // doubles
  d += n_aux * n_occ * n_virt + T * n_aux * n_orb;            // inputs staged on the device
  if (p->naf_thresh >= 0.0) d += 10 * n_aux * n_aux;           // NAF metric, reflectors, vectors, scratch
  d += n_tau * N * N + 2 * n_om * N * N;                       // Laplace moments, Pi, C
  d += n_om * (N * N + 128 * N + 4096);                        // screening sweep scratch
  d += T * N * n_orb + n_om * T * n_orb;                       // projected targets, W
  // the tensor-core partial tiles (FP32, one 128 x 128 tile per split), the
  // largest of the contractions: the metric (lower tiles, up to 64 splits of
  // the pairs), the projection (every tile, n_aux / 2048 splits) and the Pi
  // build (lower tiles x scales, 64 splits per block of pairs)
  auto cdiv = [](size_t a, size_t b) { return (a + b - 1) / b; };
  const size_t nI = cdiv(n_aux, 128), nN = cdiv(N, 128), t = n_tau ? n_tau : n_om;
  const size_t tile = 128 * 128 / 2;   // doubles per FP32 tile
  const size_t k_part = nI * (nI + 1) / 2 * std::min<size_t>(64, cdiv(n_ov, 2048)) * tile;
  const size_t p_part = nN * cdiv(n_ov, 128) * cdiv(n_aux, 2048) * tile;
  const size_t pi_part = nN * (nN + 1) / 2 * t * std::min<size_t>(64, cdiv(n_ov, 2048)) * tile;
  const size_t partials = std::max(k_part, std::max(p_part, pi_part));
  if (p->precision == LTGW_FP64_EMU) {
    // projected ov block; the largest slice set (6 slices: 4 bytes per A digit,
    // 2 per B digit, of the metric's n_aux x n_ov operands) and the partials
    d += N * n_ov + 9 * n_aux * n_ov / 2 + partials;
  } else if (p->precision != LTGW_FP64) {
    d += (2 * n_aux * n_ov + N * n_ov) / 2 + n_om * N * N / 2;  // FP32 copies, BF16 hi / lo of the ov block
    if (p->precision == LTGW_FP8 || p->precision == LTGW_FP8_PI)
      d += 3 * ((n_tau ? n_tau : n_om) + 1) * N * n_ov / 8;     // FP8 codes (two-term: 3 per value)
    d += partials;
  } else {
    d += N * n_ov;                                              // projected ov block
  }
  return d * sizeof(double) + (64u << 20);                     // + fixed slack
}

ltgw_status ltgw_server_create(ltgw_server **out, int device, int n_slots, size_t hbm_budget_bytes) {
  if (!out || n_slots < 1 || n_slots > 64 || hbm_budget_bytes == 0) return LTGW_ERR_BAD_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  ltgw_server *s = new ltgw_server();
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->init_pending = n_slots;
  for (int i = 0; i < n_slots; ++i) s->slots.emplace_back(new Slot());
  for (auto &slot : s->slots) {
    Slot *sp = slot.get();
    sp->th = std::thread([s, sp] { s->worker(sp); });
  }
  {
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv_done.wait(lock, [&] { return s->init_pending == 0; });
  }
  if (s->init_status != LTGW_OK) {
    ltgw_status st = s->init_status;
    ltgw_server_destroy(s);
    return st;
  }
  *out = s;
  return LTGW_OK;
}

ltgw_status ltgw_server_submit(ltgw_server *s, const ltgw_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return LTGW_ERR_BAD_ARG;
  if (!req->eps || !req->B_ov || !req->B_tgt || !req->targets || !req->shift || !req->sigma_iw || !req->e_qp ||
      !req->qp_status || req->n_tgt < 1)
    return LTGW_ERR_BAD_ARG;
  const size_t fp = ltgw_request_footprint(&req->p, req->n_tgt);
  if (fp > s->budget) return LTGW_ERR_NOMEM;
  std::lock_guard<std::mutex> lock(s->mu);
  Pending p;
  p.ticket = s->next_ticket++;
  p.req = *req;
  p.footprint = fp;
  p.t_submit = Clock::now();
  s->queue.push_back(p);
  *ticket = p.ticket;
  s->dispatch_locked();
  return LTGW_OK;
}

int ltgw_server_poll(ltgw_server *s, ltgw_completion *out, int max_out) {
  if (!s || !out || max_out < 1) return 0;
  std::lock_guard<std::mutex> lock(s->mu);
  int n = 0;
  while (n < max_out && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

ltgw_status ltgw_server_wait_all(ltgw_server *s, double timeout_s) {
  if (!s) return LTGW_ERR_BAD_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                      [&] { return s->queue.empty() && s->running == 0; });
  return ok ? LTGW_OK : LTGW_ERR_TIMEOUT;
}

void ltgw_server_destroy(ltgw_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto &slot : s->slots)
    if (slot->th.joinable()) slot->th.join();
  delete s;
}

}  // extern "C"
