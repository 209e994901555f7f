// Serving loop (an addition; the paper solves one sweep at a time): continuous batching of parameter
// sweeps from different seeds, admission by device-memory footprint,
// per-request latency.
//
// Each registered seed owns a CUDA stream and a worker thread. Requests
// enter a FIFO; a request is admitted when the registered seeds' resident
// bytes plus the workspace of all admitted, unfinished requests stay within
// the budget. Workers of different seeds run concurrently, so their kernels
// overlap on the device; the seed's factors and recycled Krylov space stay
// resident.
//
// Mixed-precision traces (the default path) run through a continuous-
// batching engine per seed: a fixed set of slots, each holding one
// parameter vector's solve. Every engine step is one refinement step of all
// occupied slots (FP64-accurate residual, then one recycled FP32 inner
// solve, which ends within one or two GMRES cycles); a system whose residual
// meets the tolerance retires at the step boundary and its slot is refilled
// at once from the admitted requests, one vector per request in turn, so a
// request that arrives while the seed is busy starts at the next step
// instead of waiting for the running requests to finish. A request is
// published when its last vector retires. Gradients and FP64 requests run as
// whole lockstep batches between engine steps.
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

#include "lyap_internal.h"
#include "mixed.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int seed = 0;
  int nv = 0;
  bool grad = false;
  std::vector<double> v;
  size_t bytes = 0;
  Clock::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 admitted, 2 running, 3 done, 4 cancelled
  int rc = LYAP_OK;
  int placed = 0, finished = 0;  // engine: vectors given a slot, vectors retired
  std::vector<double> f, g;
  std::vector<lyap_result_info> info;
  std::string error;  // the worker's error detail when rc != LYAP_OK
};

struct SeedSlot;

}  // namespace

struct lyap_server {
  lyap_ctx* ctx = nullptr;
  lyap_opts opts{};
  size_t budget = 0;
  size_t resident = 0;
  size_t admitted_bytes = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  std::vector<std::unique_ptr<SeedSlot>> seeds;
  uint64_t next_id = 1;
  bool shutdown = false;
  int inflight = 0;  // admitted or running, not yet published
};

namespace {

struct SeedSlot {
  lyap_server* srv = nullptr;
  lyap_seed* sd = nullptr;
  int id = 0;
  cudaStream_t stream = nullptr;
  std::deque<uint64_t> ready;
  std::condition_variable cv;
  std::thread worker;
  // continuous-batching engine (mixed-precision traces)
  MixedEngine* eng = nullptr;
  std::vector<std::pair<uint64_t, int>> owner;  // slot -> (request, vector index); request 0: free
  std::deque<uint64_t> filling;                 // engine requests with vectors not yet placed
  int occupied = 0;
};

// Device bytes a request of nv vectors may hold while it runs: the Krylov
// workspace (basis, preconditioned basis, recycled pairs, iterate, residual),
// the small dense matrices, the FP64 solution/residual vectors, and for the
// mixed path the float-float residual panel (k^2 n pairs of float2) and the
// Woodbury capacitance inverses and partial sums. Gradients double the solve
// part.
size_t request_bytes(const lyap_seed* sd, const lyap_opts& o, int nv, bool grad) {
  const size_t n = (size_t)sd->n, k = (size_t)sd->k, N = n * k;
  const size_t vec = o.precision == LYAP_FP64 ? 16 : 8;
  const size_t LD = (size_t)(o.m + o.s + 1);
  size_t per = (size_t)(2 * o.m + 2 * o.s + 6) * N * vec + LD * LD * 8 * 16 + (size_t)4 * N * 16;
  if (grad) per *= 2;
  if (o.precision != LYAP_FP64) per += k * k * n * 16;
  if (o.pbar > 0) per += (size_t)2 * o.pbar * o.pbar * 8 + (n / 32 + 2) * (size_t)o.pbar * 8;  // Cap^{-1}, partials
  return per * (size_t)nv;
}

// Admit queued requests in arrival order while the budget allows (caller holds mu).
void admit_locked(lyap_server* s) {
  while (!s->queue.empty()) {
    const uint64_t id = s->queue.front();
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second.state != 0) {
      s->queue.pop_front();
      continue;
    }
    Request& r = it->second;
    if (s->resident + s->admitted_bytes + r.bytes > s->budget && s->inflight > 0) break;
    s->queue.pop_front();
    r.state = 1;
    s->admitted_bytes += r.bytes;
    ++s->inflight;
    SeedSlot& slot = *s->seeds[r.seed];
    slot.ready.push_back(id);
    slot.cv.notify_one();
  }
}

constexpr int kEngineSlots = 512;  // slots per seed unless opts.batch sets another count

bool engine_path(const lyap_server* s, const SeedSlot* slot, const Request& r) {
  return s->opts.precision == LYAP_BF16_IR && !r.grad && slot->sd->mixed != nullptr;
}

// Publish a finished request (caller holds mu).
void finish_locked(lyap_server* s, Request& r, int rc) {
  r.rc = rc;
  if (rc != LYAP_OK) r.error = lyap_last_error();  // the worker thread's detail
  r.t_done = Clock::now();
  r.state = 3;
  s->admitted_bytes -= r.bytes;
  --s->inflight;
}

// Solve batch-path requests (gradients, FP64) as lockstep batches.
void run_batches(lyap_server* s, SeedSlot* slot, const std::vector<uint64_t>& batch) {
  for (int want_grad = 0; want_grad < 2; ++want_grad) {
    std::vector<uint64_t> ids;
    std::vector<double> v;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint64_t id : batch) {
        Request& r = s->reqs[id];
        if (r.grad == (want_grad != 0)) {
          ids.push_back(id);
          v.insert(v.end(), r.v.begin(), r.v.end());
        }
      }
    }
    if (ids.empty()) continue;
    const int k = slot->sd->k;
    const int nv = (int)(v.size() / k);
    std::vector<double> f(nv), g(want_grad ? (size_t)nv * k : 0);
    std::vector<lyap_result_info> info(nv);
    lyap_opts o = s->opts;
    o.stream = slot->stream;
    o.batch = 0;
    int rc = want_grad ? lyap_grad(slot->sd, nv, v.data(), LYAP_MEM_HOST, &o, f.data(), g.data(), info.data())
                       : lyap_trace_EX(slot->sd, nv, v.data(), LYAP_MEM_HOST, &o, f.data(), info.data());
    std::lock_guard<std::mutex> lk(s->mu);
    int off = 0;
    for (uint64_t id : ids) {
      Request& r = s->reqs[id];
      r.f.assign(f.begin() + off, f.begin() + off + r.nv);
      if (want_grad) r.g.assign(g.begin() + (size_t)off * k, g.begin() + (size_t)(off + r.nv) * k);
      r.info.assign(info.begin() + off, info.begin() + off + r.nv);
      off += r.nv;
      finish_locked(s, r, rc);
    }
    admit_locked(s);
    s->cv_done.notify_all();
  }
}

// Give free engine slots to the filling requests, one vector per request in
// turn (caller holds mu).
void fill_slots_locked(lyap_server* s, SeedSlot* slot, std::vector<EngineJoin>& joins) {
  const int k = slot->sd->k;
  int next_free = 0;
  const int cap = (int)slot->owner.size();
  while (!slot->filling.empty()) {
    bool placed_any = false;
    for (size_t q = 0; q < slot->filling.size(); ++q) {
      while (next_free < cap && slot->owner[next_free].first != 0) ++next_free;
      if (next_free >= cap) return;
      Request& r = s->reqs[slot->filling[q]];
      if (r.placed >= r.nv) continue;
      slot->owner[next_free] = {r.id, r.placed};
      joins.push_back(EngineJoin{next_free, r.v.data() + (size_t)r.placed * k});
      ++r.placed;
      ++slot->occupied;
      placed_any = true;
    }
    while (!slot->filling.empty() && s->reqs[slot->filling.front()].placed >= s->reqs[slot->filling.front()].nv)
      slot->filling.pop_front();
    if (!placed_any) return;
  }
}

void worker_loop(SeedSlot* slot) {
  lyap_server* s = slot->srv;
  cudaSetDevice(slot->sd->device);
  for (;;) {
    std::vector<uint64_t> batch;
    std::vector<EngineJoin> joins;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      slot->cv.wait(lk, [&] {
        return s->shutdown || !slot->ready.empty() || slot->occupied > 0 || !slot->filling.empty();
      });
      if (s->shutdown && slot->ready.empty() && slot->occupied == 0 && slot->filling.empty()) break;
      while (!slot->ready.empty()) {
        const uint64_t id = slot->ready.front();
        slot->ready.pop_front();
        auto it = s->reqs.find(id);
        if (it == s->reqs.end() || it->second.state != 1) continue;
        Request& r = it->second;
        r.state = 2;
        if (engine_path(s, slot, r)) {
          r.f.assign(r.nv, 0.0);
          r.info.assign(r.nv, lyap_result_info{});
          slot->filling.push_back(id);
        } else {
          batch.push_back(id);
        }
      }
      if (!slot->filling.empty() && !slot->eng) {
        const int cap = s->opts.batch > 0 ? s->opts.batch : kEngineSlots;
        lk.unlock();
        MixedEngine* e = nullptr;
        const int rc = lyap_engine_create(slot->sd, cap, s->opts, &e);
        lk.lock();
        if (rc != LYAP_OK) {  // fail the waiting engine requests
          for (uint64_t id : slot->filling) finish_locked(s, s->reqs[id], rc);
          slot->filling.clear();
          admit_locked(s);
          s->cv_done.notify_all();
        } else {
          slot->eng = e;
          slot->owner.assign(cap, {0, 0});
        }
      }
      if (slot->eng) fill_slots_locked(s, slot, joins);
    }
    if (!batch.empty()) run_batches(s, slot, batch);
    if (!slot->eng || (joins.empty() && slot->occupied == 0)) continue;
    lyap_opts o = s->opts;
    o.stream = slot->stream;
    std::vector<EngineDone> done;
    const int rc = lyap_engine_step(slot->sd, *slot->eng, o, slot->stream, joins, done);
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc != LYAP_OK) {
      // every request with a vector in the engine fails; the engine restarts empty
      for (auto& ow : slot->owner)
        if (ow.first != 0) {
          Request& r = s->reqs[ow.first];
          if (r.state == 2) finish_locked(s, r, rc);
          ow = {0, 0};
        }
      for (uint64_t id : slot->filling)
        if (s->reqs[id].state == 2) finish_locked(s, s->reqs[id], rc);
      slot->filling.clear();
      slot->occupied = 0;
      lyap_engine_free(slot->sd, slot->eng);
      slot->eng = nullptr;
    } else {
      for (const EngineDone& d : done) {
        const auto ow = slot->owner[d.slot];
        slot->owner[d.slot] = {0, 0};
        --slot->occupied;
        Request& r = s->reqs[ow.first];
        r.f[ow.second] = d.f;
        r.info[ow.second] = d.info;
        if (++r.finished == r.nv) finish_locked(s, r, LYAP_OK);
      }
    }
    admit_locked(s);
    s->cv_done.notify_all();
  }
  if (slot->eng) {
    lyap_engine_free(slot->sd, slot->eng);
    slot->eng = nullptr;
  }
}

}  // namespace

extern "C" int lyap_serve_create(lyap_ctx* ctx, const lyap_opts* opts, lyap_server** out) {
  if (!ctx || !out) return LYAP_EINVAL;
  *out = nullptr;
  std::unique_ptr<lyap_server> s(new lyap_server());
  s->ctx = ctx;
  lyap_opts_default(&s->opts);
  if (opts) s->opts = *opts;
  LY_CUDA(cudaSetDevice(ctx->device));
  size_t freeb = 0, totalb = 0;
  LY_CUDA(cudaMemGetInfo(&freeb, &totalb));
  s->budget = s->opts.hbm_budget ? s->opts.hbm_budget : (size_t)(0.8 * (double)freeb);
  *out = s.release();
  return LYAP_OK;
}

extern "C" int lyap_serve_register_seed(lyap_server* s, lyap_seed* sd, int* seed_id) {
  if (!s || !sd || !seed_id) return LYAP_EINVAL;
  std::unique_ptr<SeedSlot> slot(new SeedSlot());
  slot->srv = s;
  slot->sd = sd;
  LY_CUDA(cudaSetDevice(s->ctx->device));
  LY_CUDA(cudaStreamCreateWithFlags(&slot->stream, cudaStreamNonBlocking));
  std::lock_guard<std::mutex> lk(s->mu);
  slot->id = (int)s->seeds.size();
  *seed_id = slot->id;
  s->resident += sd->resident_bytes;
  SeedSlot* raw = slot.get();
  s->seeds.push_back(std::move(slot));
  raw->worker = std::thread(worker_loop, raw);
  return LYAP_OK;
}

extern "C" int lyap_serve_estimate(lyap_server* s, int seed_id, int nv, int want_grad, size_t* bytes) {
  if (!s || !bytes || nv <= 0) return LYAP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (seed_id < 0 || seed_id >= (int)s->seeds.size()) return LYAP_ENOTFOUND;
  *bytes = request_bytes(s->seeds[seed_id]->sd, s->opts, nv, want_grad != 0);
  return LYAP_OK;
}

extern "C" int lyap_serve_submit(lyap_server* s, int seed_id, int nv, const double* v, int want_grad,
                                 uint64_t* ticket) {
  if (!s || !ticket || nv <= 0 || !v) return LYAP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (seed_id < 0 || seed_id >= (int)s->seeds.size()) return LYAP_ENOTFOUND;
  const lyap_seed* sd = s->seeds[seed_id]->sd;
  LY_TRY(lyap_check_v(nv, sd->k, v));
  Request r;
  r.id = s->next_id++;
  r.seed = seed_id;
  r.nv = nv;
  r.grad = want_grad != 0;
  r.v.assign(v, v + (size_t)nv * sd->k);
  r.bytes = request_bytes(sd, s->opts, nv, r.grad);
  if (s->resident + r.bytes > s->budget) {
    lyap_set_last_error("request needs more device memory than the server budget");
    return LYAP_ENOMEM;
  }
  r.t_submit = Clock::now();
  *ticket = r.id;
  s->reqs.emplace(r.id, std::move(r));
  s->queue.push_back(*ticket);
  admit_locked(s);
  return LYAP_OK;
}

extern "C" int lyap_serve_run(lyap_server* s, int max_ms, int* busy) {
  if (!s) return LYAP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->inflight == 0 && s->queue.empty(); };
  if (max_ms <= 0) s->cv_done.wait(lk, idle);
  else s->cv_done.wait_for(lk, std::chrono::milliseconds(max_ms), idle);
  if (busy) *busy = idle() ? 0 : 1;
  return LYAP_OK;
}

extern "C" int lyap_serve_poll(lyap_server* s, uint64_t ticket, double* trace_out, double* grad_out,
                               lyap_result_info* info, double* latency_s) {
  if (!s) return LYAP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LYAP_ENOTFOUND;
  Request& r = it->second;
  if (r.state == 4) {
    s->reqs.erase(it);
    return LYAP_ECANCELLED;
  }
  if (r.state != 3) return LYAP_PENDING;
  const int rc = r.rc;
  const int k = s->seeds[r.seed]->sd->k;
  if (rc == LYAP_OK) {
    if (trace_out) std::memcpy(trace_out, r.f.data(), sizeof(double) * r.nv);
    if (grad_out && r.grad) std::memcpy(grad_out, r.g.data(), sizeof(double) * (size_t)r.nv * k);
    if (info) std::memcpy(info, r.info.data(), sizeof(lyap_result_info) * r.nv);
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
  if (rc != LYAP_OK) lyap_set_last_error(r.error);
  s->reqs.erase(it);
  return rc;
}

extern "C" int lyap_serve_cancel(lyap_server* s, uint64_t ticket) {
  if (!s) return LYAP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LYAP_ENOTFOUND;
  if (it->second.state == 0) {
    it->second.state = 4;  // still queued: never admitted
    return LYAP_OK;
  }
  return LYAP_EINVAL;  // admitted or running requests complete normally
}

extern "C" void lyap_serve_destroy(lyap_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->shutdown = true;
    for (auto& slot : s->seeds) slot->cv.notify_all();
  }
  for (auto& slot : s->seeds) {
    if (slot->worker.joinable()) slot->worker.join();
    if (slot->stream) cudaStreamDestroy(slot->stream);
  }
  delete s;
}
