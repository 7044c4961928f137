// serve.cu -- continuous-batching serving loop (crnt_submit / crnt_poll).
//
// Requests (transport blocks with their LLRs) arrive from many cells at any
// time.  A worker thread batches whatever is pending into the next free
// slot -- a CUDA stream with its own reusable plan and pinned/device
// buffers -- and launches the fused decode there, while earlier batches are
// still running on other slots, so work admitted later overlaps on the
// device with work admitted earlier.  Finished batches are harvested by
// polling their events; results wait in a done queue for crnt_poll.
// crnt_submit copies each TB's LLRs (a CPU memcpy) into a ring of
// page-locked host memory that the decode kernel reads in place over the
// CPU-GPU link, and the kernel writes the decoded bits straight into
// page-locked output buffers, so neither side issues a copy: the worker only
// plans and launches.  Admission is by in-flight TB count and by space in
// that ring (the memory a request holds while queued or running); beyond
// either, crnt_submit returns CRNT_EAGAIN.  Waits are bounded: the worker sleeps on a condition variable
// with a timeout and crnt_poll honours its timeout.
#include <cuda_runtime.h>

#include <algorithm>
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
constexpr int kSlots = 12;             // concurrent batches on the device
constexpr uint32_t kMaxBatchTbs = 1024;
}  // namespace

struct Req {
  uint64_t ticket;
  crnt_tb_params tb;
  int64_t llr_off;   // byte offset of its LLRs in the LLR ring
  uint64_t alloc;    // allocation sequence number (ring release order)
  int64_t t_submit;
};

// Ring holding the LLRs of queued and running requests, released in
// allocation order.  Each allocation is contiguous.
struct Ring {
  size_t cap = 0, head = 0, tail = 0;
  struct A {
    size_t end;
    bool done;
  };
  std::deque<A> q;
  uint64_t first_seq = 0;  // sequence number of q.front()
  bool alloc(size_t n, size_t* off, uint64_t* seq) {
    if (q.empty()) head = tail = 0;
    if (head >= tail) {  // free space: [head, cap) and [0, tail)
      if (cap - head >= n) {
        *off = head;
      } else if (tail > n) {
        *off = 0;
      } else {
        return false;
      }
    } else if (tail - head > n) {  // free space: [head, tail)
      *off = head;
    } else {
      return false;
    }
    head = *off + n;
    *seq = first_seq + q.size();
    q.push_back(A{head, false});
    return true;
  }
  void release(uint64_t seq) {
    q[seq - first_seq].done = true;
    while (!q.empty() && q.front().done) {
      tail = q.front().end;
      q.pop_front();
      first_seq++;
    }
  }
};

struct Done {
  crnt_tb_result res;
  std::vector<uint8_t> bits;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  crnt_plan plan;
  Buf h_out{true};  // page-locked; the kernel writes the decoded bits here
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
  uint64_t inflight_tbs = 0;  // queued + running
  int device_error = 0;
  int8_t* arena = nullptr;    // page-locked LLR ring (host address)
  int8_t* arena_dev = nullptr;  // the same ring as kernels address it
  Ring ring;

  void run();
  bool launch(Slot* s, std::vector<Req>&& batch);
  void harvest(Slot* s, bool failed);
};

bool Serving::launch(Slot* s, std::vector<Req>&& batch) {
  s->reqs = std::move(batch);
  const uint32_t n = (uint32_t)s->reqs.size();
  std::vector<crnt_tb_params> tbs(n);
  std::vector<int64_t> base(n);
  for (uint32_t i = 0; i < n; i++) {
    tbs[i] = s->reqs[i].tb;
    base[i] = s->reqs[i].llr_off;
  }
  if (plan_build(ctx, tbs.data(), n, &s->plan, s->stream, base.data()) != CRNT_OK) return false;
  const size_t out_bytes = s->plan.info.out_bytes;
  if (!s->h_out.ensure(out_bytes)) return false;
  uint8_t* out_dev = nullptr;
  if (cudaHostGetDevicePointer((void**)&out_dev, s->h_out.p, 0) != cudaSuccess) return false;
  s->t_start = now_ns();
  if (plan_launch(&s->plan, arena_dev, out_dev, s->stream, nullptr, nullptr, nullptr, true) !=
          CRNT_OK ||
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
    s->plan.upload_pending = false;  // the slot's event passed the upload
  }
  size_t off = 0;
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
    d.res.ticket = r.ticket;
    d.res.t_submit_ns = (uint64_t)r.t_submit;
    d.res.t_start_ns = (uint64_t)s->t_start;
    d.res.t_done_ns = (uint64_t)t_done;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : out) done.push_back(std::move(d));
    for (auto& r : s->reqs) ring.release(r.alloc);
    inflight_tbs -= n;
  }
  s->reqs.clear();
  s->busy = false;
  cv_done.notify_all();
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
  if (cudaHostAlloc((void**)&sv->arena, sv->ring.cap, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&sv->arena_dev, sv->arena, 0) != cudaSuccess) {
    cudaGetLastError();
    if (sv->arena) cudaFreeHost(sv->arena);
    return nullptr;
  }
  for (int i = 0; i < kSlots; i++) {
    // buffers for the largest batch up front: no allocation (and none of the
    // device-wide synchronisation a cudaFree implies) while serving
    std::unique_ptr<Slot> s(new (std::nothrow) Slot);
    if (!s || cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
        !plan_reserve(&s->plan, kMaxBatchTbs, kMaxBatchTbs * CRNT_MAX_CB) ||
        !s->h_out.ensure((size_t)kMaxBatchTbs * 4096))
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
  if (sv->arena) cudaFreeHost(sv->arena);
  delete sv;
}

}  // namespace crnt

using namespace crnt;

extern "C" {

int crnt_submit(crnt_ctx* ctx, const crnt_tb_params* tbs, const int8_t* const* llrs, uint32_t n,
                uint64_t* tickets_out) {
  if (!ctx || !tbs || !llrs || !tickets_out || n == 0) return CRNT_EINVAL;
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
  }
  Serving* sv = serving_get(ctx);
  if (!sv) return CRNT_EDEVICE;
  const int64_t t = now_ns();
  std::vector<Req> reqs(n);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->device_error) return sv->device_error;
    if (sv->inflight_tbs + n > ctx->cfg.max_inflight) return CRNT_EAGAIN;
    for (uint32_t i = 0; i < n; i++) {
      size_t off;
      if (!sv->ring.alloc(tbs[i].G, &off, &reqs[i].alloc)) {
        for (uint32_t j = 0; j < i; j++) sv->ring.release(reqs[j].alloc);
        return CRNT_EAGAIN;
      }
      reqs[i].llr_off = (int64_t)off;
    }
    sv->inflight_tbs += n;
  }
  // the LLRs are in the ring before the requests become visible (the
  // worker's launch, which reads them, follows the publication below)
  for (uint32_t i = 0; i < n; i++) memcpy(sv->arena + reqs[i].llr_off, llrs[i], tbs[i].G);
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
