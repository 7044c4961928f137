// serve.cu -- continuous-batching serving loop (crnt_submit / crnt_poll).
//
// Requests (transport blocks with their LLRs) arrive from many cells at any
// time.  A worker thread batches whatever is pending into the next free
// slot -- a CUDA stream with its own reusable plan and pinned/device
// buffers -- and launches the fused decode there, while earlier batches are
// still running on other slots, so work admitted later overlaps on the
// device with work admitted earlier.  Finished batches are harvested by
// polling their events; results wait in a done queue for crnt_poll.
// Admission is by in-flight TB count and by LLR bytes (the device memory a
// request pins while queued or running); beyond either, crnt_submit returns
// CRNT_EAGAIN.  Waits are bounded: the worker sleeps on a condition variable
// with a timeout and crnt_poll honours its timeout.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

namespace crnt {

namespace {
constexpr int kSlots = 6;              // concurrent batches on the device
constexpr uint32_t kMaxBatchTbs = 1024;
}  // namespace

struct Req {
  uint64_t ticket;
  crnt_tb_params tb;
  std::vector<int8_t> llr;
  int64_t t_submit;
};

struct Done {
  crnt_tb_result res;
  std::vector<uint8_t> bits;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  crnt_plan plan;
  Buf d_llr, d_out;
  Buf h_llr{true}, h_out{true};
  std::vector<Req> reqs;
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
  uint64_t inflight_tbs = 0, inflight_bytes = 0;  // queued + running
  int device_error = 0;

  void run();
  bool launch(Slot* s, std::vector<Req>&& batch);
  void harvest(Slot* s, bool failed);
};

bool Serving::launch(Slot* s, std::vector<Req>&& batch) {
  s->reqs = std::move(batch);
  const uint32_t n = (uint32_t)s->reqs.size();
  std::vector<crnt_tb_params> tbs(n);
  size_t bytes = 0;
  for (uint32_t i = 0; i < n; i++) {
    tbs[i] = s->reqs[i].tb;
    bytes += s->reqs[i].llr.size();
  }
  if (!s->h_llr.ensure(bytes) || !s->d_llr.ensure(bytes)) return false;
  size_t off = 0;
  for (auto& r : s->reqs) {
    memcpy((uint8_t*)s->h_llr.p + off, r.llr.data(), r.llr.size());
    off += r.llr.size();
  }
  if (plan_build(ctx, tbs.data(), n, &s->plan, s->stream) != CRNT_OK) return false;
  const size_t out_bytes = s->plan.info.out_bytes;
  if (!s->d_out.ensure(out_bytes) || !s->h_out.ensure(out_bytes)) return false;
  s->t_start = now_ns();
  if (cudaMemcpyAsync(s->d_llr.p, s->h_llr.p, bytes, cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess ||
      plan_launch(&s->plan, (const int8_t*)s->d_llr.p, (uint8_t*)s->d_out.p, s->stream, nullptr,
                  nullptr, nullptr) != CRNT_OK ||
      cudaMemcpyAsync(s->h_out.p, s->d_out.p, out_bytes, cudaMemcpyDeviceToHost, s->stream) !=
          cudaSuccess ||
      plan_fetch_results(&s->plan, s->stream) != CRNT_OK ||
      cudaEventRecord(s->ev, s->stream) != cudaSuccess)
    return false;
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
  }
  size_t off = 0, bytes = 0;
  for (uint32_t i = 0; i < n; i++) {
    Done& d = out[i];
    const Req& r = s->reqs[i];
    if (failed) {
      memset(&d.res, 0, sizeof d.res);
      d.res.status = CRNT_EDEVICE;
    } else {
      d.res = s->tmp[i];
      const uint8_t* src = (const uint8_t*)s->h_out.p + off;
      d.bits.assign(src, src + r.tb.A / 8);
    }
    off += r.tb.A / 8;
    bytes += r.llr.size();
    d.res.ticket = r.ticket;
    d.res.t_submit_ns = (uint64_t)r.t_submit;
    d.res.t_start_ns = (uint64_t)s->t_start;
    d.res.t_done_ns = (uint64_t)t_done;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : out) done.push_back(std::move(d));
    inflight_tbs -= n;
    inflight_bytes -= bytes;
  }
  s->reqs.clear();
  s->busy = false;
  cv_done.notify_all();
}

void Serving::run() {
  cudaSetDevice(ctx->device);
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
      if (!launch(free_slot, std::move(batch))) harvest(free_slot, true);
      progress = true;
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(5));
  }
}

static Serving* serving_get(crnt_ctx* ctx) {
  std::lock_guard<std::mutex> lk(ctx->serving_mu);
  if (ctx->serving) return ctx->serving;
  std::unique_ptr<Serving> sv(new (std::nothrow) Serving);
  if (!sv) return nullptr;
  sv->ctx = ctx;
  cudaSetDevice(ctx->device);
  for (int i = 0; i < kSlots; i++) {
    std::unique_ptr<Slot> s(new (std::nothrow) Slot);
    if (!s || cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
    sv->slots.push_back(std::move(s));
  }
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
  delete sv;
}

}  // namespace crnt

using namespace crnt;

extern "C" {

int crnt_submit(crnt_ctx* ctx, const crnt_tb_params* tbs, const int8_t* const* llrs, uint32_t n,
                uint64_t* tickets_out) {
  if (!ctx || !tbs || !llrs || !tickets_out || n == 0) return CRNT_EINVAL;
  uint64_t bytes = 0;
  for (uint32_t i = 0; i < n; i++) {
    lte::Seg s;
    int rc = validate(tbs[i], &s);
    if (rc) return rc;
    if (!llrs[i]) return CRNT_EINVAL;
    if ((tbs[i].flags & CRNT_F_HARQ) && !tbs[i].new_data) {
      std::lock_guard<std::mutex> lk(ctx->harq_mu);
      if (!ctx->harq.keys.count(std::make_tuple(tbs[i].cell, tbs[i].ue, tbs[i].harq_pid)))
        return CRNT_ENOTFOUND;
    }
    bytes += tbs[i].G;
  }
  Serving* sv = serving_get(ctx);
  if (!sv) return CRNT_EDEVICE;
  const int64_t t = now_ns();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->device_error) return sv->device_error;
    if (sv->inflight_tbs + n > ctx->cfg.max_inflight ||
        sv->inflight_bytes + bytes > ctx->cfg.mem_budget / 4)
      return CRNT_EAGAIN;
    for (uint32_t i = 0; i < n; i++) {
      Req r;
      r.ticket = sv->next_ticket++;
      r.tb = tbs[i];
      r.llr.assign(llrs[i], llrs[i] + tbs[i].G);
      r.t_submit = t;
      tickets_out[i] = r.ticket;
      sv->pending.push_back(std::move(r));
    }
    sv->inflight_tbs += n;
    sv->inflight_bytes += bytes;
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
  sv->polled.clear();
  if (sv->done.empty() && timeout_us)
    sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                         [sv] { return !sv->done.empty(); });
  uint32_t k = 0;
  while (k < max && !sv->done.empty()) {
    sv->polled.push_back(std::move(sv->done.front()));
    sv->done.pop_front();
    k++;
  }
  for (uint32_t i = 0; i < k; i++) {
    done[i] = sv->polled[i].res;
    if (bits) bits[i] = sv->polled[i].bits.empty() ? nullptr : sv->polled[i].bits.data();
  }
  return (int)k;
}

}  // extern "C"
