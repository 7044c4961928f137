// serve.cu -- continuous-batching serving loop (crnt_submit / crnt_poll).
//
// Requests (transport blocks with their LLRs) arrive from many cells at any
// time.  A worker thread batches whatever is pending into the next free
// slot -- a CUDA stream with its own reusable plan -- and launches the fused
// decode there, while earlier batches are still running on other slots, so
// work admitted later overlaps on the device with work admitted earlier.
// Finished batches are harvested by polling their events; results wait in a
// done queue for crnt_poll.
//
// The submitting threads do the per-TB work: crnt_submit validates and
// prepares each TB (segmentation, soft-buffer binding, CB descriptors) and
// copies its LLRs (a CPU memcpy) into a ring of page-locked host memory that
// the decode kernel reads in place over the CPU-GPU link; it also reserves
// the TB's output bytes in a second page-locked ring, which the kernel
// writes and crnt_poll hands out in place.  Neither side issues a copy of
// payload data: the worker only assembles batches, launches and collects.
//
// Admission: by in-flight TB count, by space in the two rings (the memory a
// request holds while queued, running or unpolled) and, unless the context
// is configured otherwise, by predicted completion (see Admission below);
// a refused crnt_submit returns CRNT_EAGAIN and queues nothing.  Waits are
// bounded: the worker sleeps on a condition variable with a timeout and
// crnt_poll honours its timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"
#include "serve_model.h"

namespace crnt {

namespace {
constexpr int kSlots = 12;             // concurrent batches on the device
constexpr uint32_t kMaxBatchTbs = 1024;
}  // namespace

struct Req {
  uint64_t ticket;
  crnt_tb_params tb;
  std::unique_ptr<TbPrep> prep;  // prepared by the submitting thread
  int64_t llr_off;   // byte offset of its LLRs in the LLR ring
  uint64_t alloc;    // allocation sequence number (ring release order)
  int64_t out_off;   // byte offset of its decoded bits in the output ring
  uint64_t out_alloc;
  int64_t t_submit;
  double work;       // expected decode work: trellis steps x iteration limit
  double ahead;      // outstanding work when its subframe was admitted (itself included)
};

struct Done {
  crnt_tb_result res;
  const uint8_t* bits;  // in the output ring, or null
  uint64_t out_alloc;   // released at the crnt_poll after the one handing it out
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  crnt_plan plan;
  std::vector<Req> reqs;
  std::vector<crnt_tb_params> tbs;
  std::vector<const TbPrep*> preps;
  std::vector<int64_t> llr_base, out_base;
  std::vector<crnt_tb_result> tmp;
  bool busy = false;
  int64_t t_start = 0;
};

struct Serving {
  crnt_ctx* ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Req> pending;
  std::deque<Done> done;
  std::vector<Done> polled;  // results handed out by the last crnt_poll
  std::vector<std::unique_ptr<Slot>> slots;
  uint64_t next_ticket = 1;
  uint64_t inflight_tbs = 0;  // queued + running
  double work_out = 0;        // expected work of the TBs queued and running
  Admission adm;
  int device_error = 0;
  int8_t* arena = nullptr;    // page-locked LLR ring (host address)
  int8_t* arena_dev = nullptr;  // the same ring as kernels address it
  Ring ring;
  uint8_t* out_arena = nullptr;  // page-locked output ring the kernels write
  uint8_t* out_arena_dev = nullptr;
  Ring out_ring;
  // counters of crnt_serve_stats: those under mu, and the time counters
  // the worker and the submitting threads add without it
  crnt_serve_stats st{};
  std::atomic<uint64_t> t_plan{0}, t_launch{0}, t_harvest{0}, t_copy{0};
  int64_t t_loop0 = 0;

  void run();
  bool launch(Slot* s, std::vector<Req>&& batch);
  void harvest(Slot* s, bool failed);
};

bool Serving::launch(Slot* s, std::vector<Req>&& batch) {
  s->reqs = std::move(batch);
  const int64_t t0 = now_ns();
  const uint32_t n = (uint32_t)s->reqs.size();
  s->tbs.resize(n);
  s->preps.resize(n);
  s->llr_base.resize(n);
  s->out_base.resize(n);
  for (uint32_t i = 0; i < n; i++) {
    const Req& r = s->reqs[i];
    s->tbs[i] = r.tb;
    s->preps[i] = r.prep.get();
    s->llr_base[i] = r.llr_off;
    s->out_base[i] = r.out_off;
  }
  if (plan_assemble(ctx, s->tbs.data(), s->preps.data(), n, &s->plan, s->stream,
                    s->llr_base.data(), s->out_base.data()) != CRNT_OK)
    return false;
  s->t_start = now_ns();
  t_plan += (uint64_t)(s->t_start - t0);
  if (plan_launch(&s->plan, arena_dev, out_arena_dev, s->stream, nullptr, nullptr, nullptr, true) !=
          CRNT_OK ||
      plan_fetch_results(&s->plan, s->stream) != CRNT_OK ||
      cudaEventRecord(s->ev, s->stream) != cudaSuccess)
    return false;
  t_launch += (uint64_t)(now_ns() - s->t_start);
  s->busy = true;
  return true;
}

void Serving::harvest(Slot* s, bool failed) {
  const uint32_t n = (uint32_t)s->reqs.size();
  const int64_t t_done = now_ns();
  std::vector<Done> out(n);
  if (!failed) {
    s->tmp.resize(n);
    plan_fill_results(&s->plan, s->tmp.data());
    s->plan.upload_pending = false;  // the slot's event passed the upload
  }
  uint64_t late = 0;
  const int64_t deadline = (int64_t)ctx->cfg.deadline_us * 1000;
  Admission::Batch bt;
  double work = 0;
  for (uint32_t i = 0; i < n; i++) {
    Done& d = out[i];
    const Req& r = s->reqs[i];
    if (failed) {
      memset(&d.res, 0, sizeof d.res);
      d.res.status = CRNT_EDEVICE;
      d.bits = nullptr;
    } else {
      d.res = s->tmp[i];
      d.bits = out_arena + r.out_off;
    }
    d.out_alloc = r.out_alloc;
    d.res.ticket = r.ticket;
    d.res.t_submit_ns = (uint64_t)r.t_submit;
    d.res.t_start_ns = (uint64_t)s->t_start;
    d.res.t_done_ns = (uint64_t)t_done;
    late += t_done - r.t_submit > deadline;
    // (the worker is the model's only writer, so it reads it without the lock)
    work += r.work;
    adm.observe(bt, r.ahead, (double)(t_done - r.t_submit) * 1e-3, (double)ctx->cfg.deadline_us);
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : out) done.push_back(std::move(d));
    for (auto& r : s->reqs) ring.release(r.alloc);
    inflight_tbs -= n;
    work_out = inflight_tbs ? std::max(0.0, work_out - work) : 0.0;
    if (!failed) adm.update(bt, (double)ctx->cfg.deadline_us);
    st.done_tbs += n;
    st.late_tbs += late;
  }
  s->reqs.clear();
  s->busy = false;
  cv_done.notify_all();
  t_harvest += (uint64_t)(now_ns() - t_done);
}

void Serving::run() {
  cudaSetDevice(ctx->device);
  int64_t last_progress = now_ns();
  for (;;) {
    bool progress = false, any_busy = false;
    for (auto& sp : slots) {
      Slot* s = sp.get();
      if (!s->busy) continue;
      const cudaError_t q = cudaEventQuery(s->ev);
      if (q == cudaSuccess) {
        harvest(s, false);
        progress = true;
      } else if (q != cudaErrorNotReady) {
        device_error = CRNT_EDEVICE;
        harvest(s, true);
        progress = true;
      } else {
        any_busy = true;
      }
    }
    Slot* free_slot = nullptr;
    for (auto& sp : slots)
      if (!sp->busy) {
        free_slot = sp.get();
        break;
      }
    std::vector<Req> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (stop && pending.empty() && !any_busy) break;
      if (free_slot && !pending.empty()) {
        while (!pending.empty() && batch.size() < kMaxBatchTbs) {
          batch.push_back(std::move(pending.front()));
          pending.pop_front();
        }
      } else if (!progress && !any_busy) {
        cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    if (!batch.empty()) {
      {
        std::lock_guard<std::mutex> lk(mu);
        st.batches++;
      }
      if (!launch(free_slot, std::move(batch))) harvest(free_slot, true);
      progress = true;
    }
    // While batches run the worker polls their events: it yields (keeping
    // the core) for up to 300 us after the last progress, so a finished
    // batch is harvested within microseconds, then backs off to short sleeps
    // (a sleep lasts some 50 us on Linux).
    if (progress) {
      last_progress = now_ns();
    } else if (now_ns() - last_progress < 300000) {
      std::this_thread::yield();
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
  }
}

static Serving* serving_get(crnt_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->serving_mu);
  if (ctx->serving) return ctx->serving;
  std::unique_ptr<Serving> sv(new (std::nothrow) Serving);
  if (!sv) return nullptr;
  sv->ctx = ctx;
  cudaSetDevice(ctx->device);
  sv->ring.cap = (size_t)std::min<uint64_t>(ctx->cfg.mem_budget / 8, 256ull << 20);
  sv->out_ring.cap = (size_t)std::min<uint64_t>(ctx->cfg.mem_budget / 32, 64ull << 20);
  if (cudaHostAlloc((void**)&sv->arena, sv->ring.cap, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&sv->arena_dev, sv->arena, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&sv->out_arena, sv->out_ring.cap, cudaHostAllocMapped) !=
          cudaSuccess ||
      cudaHostGetDevicePointer((void**)&sv->out_arena_dev, sv->out_arena, 0) != cudaSuccess) {
    cudaGetLastError();
    if (sv->arena) cudaFreeHost(sv->arena);
    if (sv->out_arena) cudaFreeHost(sv->out_arena);
    return nullptr;
  }
  for (int i = 0; i < kSlots; i++) {
    // buffers for the largest batch up front: no allocation (and none of the
    // device-wide synchronisation a cudaFree implies) while serving
    std::unique_ptr<Slot> s(new (std::nothrow) Slot);
    if (!s || cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
        !plan_reserve(&s->plan, kMaxBatchTbs, kMaxBatchTbs * CRNT_MAX_CB))
      return nullptr;
    sv->slots.push_back(std::move(s));
  }
  sv->t_loop0 = now_ns();
  sv->th = std::thread([p = sv.get()] { p->run(); });
  ctx->serving = sv.release();
  return ctx->serving;
}

void serving_stop(crnt_ctx* ctx) {
  Serving* sv;
  {
    std::lock_guard<std::mutex> lk(ctx->serving_mu);
    sv = ctx->serving;
    ctx->serving = nullptr;
  }
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  for (auto& s : sv->slots) {
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->stream) cudaStreamDestroy(s->stream);
  }
  if (sv->arena) cudaFreeHost(sv->arena);
  if (sv->out_arena) cudaFreeHost(sv->out_arena);
  delete sv;
}

}  // namespace crnt

using namespace crnt;

extern "C" {

int crnt_submit(crnt_ctx* ctx, const crnt_tb_params* tbs, const int8_t* const* llrs, uint32_t n,
                uint64_t* tickets_out) {
  if (!ctx || !tbs || !llrs || !tickets_out || n == 0) return CRNT_EINVAL;
  std::vector<Req> reqs(n);
  double work = 0;
  for (uint32_t i = 0; i < n; i++) {
    lte::Seg s;
    int rc = validate(tbs[i], &s);
    if (rc) return rc;
    reqs[i].work = (double)(s.Cm * s.Km + (s.C - s.Cm) * s.Kp) * tbs[i].max_iter;
    work += reqs[i].work;
    if (!llrs[i]) return CRNT_EINVAL;
    if ((tbs[i].flags & CRNT_F_HARQ) && !tbs[i].new_data) {
      std::lock_guard<std::mutex> lk(ctx->harq_mu);
      if (!ctx->harq.keys.count(std::make_tuple(tbs[i].cell, tbs[i].ue, tbs[i].harq_pid)))
        return CRNT_ENOTFOUND;
    }
  }
  Serving* sv = serving_get(ctx);
  if (!sv) return CRNT_EDEVICE;
  const int64_t t = now_ns();
  // gives back what admission took (with the lock held), for refusals and
  // for a TB that fails its preparation
  auto give_back = [&](uint32_t n_llr, uint32_t n_out) {
    for (uint32_t j = 0; j < n_llr; j++) sv->ring.release(reqs[j].alloc);
    for (uint32_t j = 0; j < n_out; j++) sv->out_ring.release(reqs[j].out_alloc);
  };
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->device_error) return sv->device_error;
    sv->st.submit_calls++;
    sv->st.offered_tbs += n;
    if (sv->inflight_tbs + n > ctx->cfg.max_inflight) {
      sv->st.refused_calls++;
      return CRNT_EAGAIN;
    }
    const double ahead = sv->work_out + work;
    if (ctx->cfg.admission == 0 && sv->inflight_tbs > 0 &&
        sv->adm.predict(ahead) > (double)ctx->cfg.deadline_us) {
      sv->st.refused_calls++;
      sv->st.refused_deadline++;
      return CRNT_EAGAIN;
    }
    for (uint32_t i = 0; i < n; i++) {
      size_t off, oo;
      if (!sv->ring.alloc(tbs[i].G, &off, &reqs[i].alloc)) {
        give_back(i, i);
        sv->st.refused_calls++;
        return CRNT_EAGAIN;
      }
      if (!sv->out_ring.alloc(tbs[i].A / 8, &oo, &reqs[i].out_alloc)) {
        give_back(i + 1, i);
        sv->st.refused_calls++;
        return CRNT_EAGAIN;
      }
      reqs[i].llr_off = (int64_t)off;
      reqs[i].out_off = (int64_t)oo;
    }
    sv->inflight_tbs += n;
    sv->work_out = ahead;
    for (uint32_t i = 0; i < n; i++) reqs[i].ahead = ahead;
    sv->st.admitted_tbs += n;
  }
  // This thread prepares its TBs (descriptors, soft-buffer binding), so the
  // serving worker only assembles batches.
  for (uint32_t i = 0; i < n; i++) {
    reqs[i].prep.reset(new (std::nothrow) TbPrep);
    const int rc = reqs[i].prep ? tb_prepare(ctx, tbs[i], reqs[i].prep.get()) : CRNT_ENOMEM;
    if (rc) {
      std::lock_guard<std::mutex> lk(sv->mu);
      give_back(n, n);
      sv->inflight_tbs -= n;
      sv->work_out = sv->inflight_tbs ? std::max(0.0, sv->work_out - work) : 0.0;
      sv->st.admitted_tbs -= n;
      return rc;
    }
  }
  // the LLRs are in the ring before the requests become visible (the
  // worker's launch, which reads them, follows the publication below)
  const int64_t tc = now_ns();
  for (uint32_t i = 0; i < n; i++) memcpy(sv->arena + reqs[i].llr_off, llrs[i], tbs[i].G);
  sv->t_copy += (uint64_t)(now_ns() - tc);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (uint32_t i = 0; i < n; i++) {
      reqs[i].ticket = sv->next_ticket++;
      reqs[i].tb = tbs[i];
      reqs[i].t_submit = t;
      tickets_out[i] = reqs[i].ticket;
      sv->pending.push_back(std::move(reqs[i]));
    }
  }
  sv->cv_work.notify_one();
  return CRNT_OK;
}

int crnt_poll(crnt_ctx* ctx, crnt_tb_result* done, const uint8_t** bits, uint32_t max,
              uint32_t timeout_us) {
  if (!ctx || !done || max == 0) return CRNT_EINVAL;
  Serving* sv = serving_get(ctx);
  if (!sv) return CRNT_EDEVICE;
  std::unique_lock<std::mutex> lk(sv->mu);
  // the bytes handed out by the previous call are no longer needed
  for (const Done& d : sv->polled) sv->out_ring.release(d.out_alloc);
  sv->polled.clear();
  if (sv->done.empty() && timeout_us)
    sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                         [sv] { return !sv->done.empty(); });
  uint32_t k = 0;
  while (k < max && !sv->done.empty()) {
    sv->polled.push_back(sv->done.front());
    sv->done.pop_front();
    k++;
  }
  for (uint32_t i = 0; i < k; i++) {
    done[i] = sv->polled[i].res;
    if (bits) bits[i] = sv->polled[i].bits;
  }
  return (int)k;
}

int crnt_serve_stats_get(crnt_ctx* ctx, crnt_serve_stats* out) {
  if (!ctx || !out) return CRNT_EINVAL;
  memset(out, 0, sizeof *out);
  std::lock_guard<std::mutex> lk(ctx->serving_mu);
  Serving* sv = ctx->serving;
  if (!sv) return CRNT_OK;
  {
    std::lock_guard<std::mutex> lk2(sv->mu);
    *out = sv->st;
    out->model_a_us = sv->adm.a;
    out->model_rate = 1.0 / sv->adm.b;
    out->model_sigma_us = sv->adm.sigma;
  }
  out->worker_plan_ns = sv->t_plan.load();
  out->worker_launch_ns = sv->t_launch.load();
  out->worker_harvest_ns = sv->t_harvest.load();
  out->submit_copy_ns = sv->t_copy.load();
  out->worker_ns = (uint64_t)(now_ns() - sv->t_loop0);
  return CRNT_OK;
}

}  // extern "C"
