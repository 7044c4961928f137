// crnt_api.cu -- host runtime and C ABI of the decoding library.
//
// The planner turns a batch of transport blocks into code-block descriptors
// and work items (the device counterpart of the paper's Algorithm 1 queuing
// step), binds HARQ processes to device soft buffers, and launches the fused
// decode kernel whose CTAs drain the work queue (Algorithm 2).  The serving
// loop (crnt_submit / crnt_poll) batches requests continuously on a pool of
// CUDA streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/crnt.h"
#include "crnt_internal.h"
#include "lte_params.h"

using namespace crnt;

namespace {

constexpr uint32_t kGA = 0x1864CFBu;
constexpr uint32_t kGB = 0x1800063u;
constexpr int kXpowA = 2400;  // words of the longest TB (75400 bits) + margin
constexpr int kXpowB = 200;   // words of the longest CB (6144 bits) + margin
constexpr int kSoftSlot = 13 * 18528 + 32;  // soft bytes of the largest TB

uint32_t gf_mul(uint32_t a, uint32_t b, uint32_t g) {
  uint32_t r = 0;
  for (int i = 23; i >= 0; i--) {
    r <<= 1;
    if (r & 0x1000000u) r ^= g;
    if ((a >> i) & 1u) r ^= b;
  }
  return r;
}

// x^(32 s) mod g for s = 0..n-1
std::vector<uint32_t> xpow_table(uint32_t g, int n) {
  std::vector<uint32_t> t(n);
  uint32_t x32 = 1;  // x^32 mod g by 32 shifts of 1
  for (int i = 0; i < 32; i++) {
    x32 <<= 1;
    if (x32 & 0x1000000u) x32 ^= g;
  }
  uint32_t cur = 1;
  for (int s = 0; s < n; s++) {
    t[s] = cur;
    cur = gf_mul(cur, x32, g);
  }
  return t;
}

// Exact division q / W as (q * M) >> s for 0 <= q < qmax.
bool find_divider(int W, int qmax, int* M, int* s) {
  for (int sh = 0; sh < 32; sh++) {
    const uint64_t m = ((1ull << sh) + W - 1) / W;
    if (m * (uint64_t)qmax >= (1ull << 32)) break;
    bool ok = true;
    for (int q = 0; q < qmax && ok; q++) ok = (int)((q * m) >> sh) == q / W;
    if (ok) {
      *M = (int)m;
      *s = sh;
      return true;
    }
  }
  return false;
}

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int validate(const crnt_tb_params& t, lte::Seg* seg) {
  if (t.A < 16 || t.A > 75376 || (t.A & 7)) return CRNT_EINVAL;
  if (t.Qm != 2 && t.Qm != 4 && t.Qm != 6) return CRNT_EINVAL;
  if (t.NL != 1 && t.NL != 2) return CRNT_EINVAL;
  if (t.rv > 3 || t.max_iter < 1 || t.max_iter > 16) return CRNT_EINVAL;
  if (t.G == 0 || t.G % (t.Qm * t.NL)) return CRNT_EINVAL;
  if (!lte::segment((int)t.A + 24, seg) || seg->C > CRNT_MAX_CB) return CRNT_EINVAL;
  // every CB must receive at least one LLR
  if (lte::e_r((int)t.G, t.Qm, t.NL, seg->C, 0) < 1) return CRNT_EINVAL;
  return CRNT_OK;
}

// Window count for a CB of size K: the caller's P clamped to [1, K/8] and
// [1, CRNT_MAX_P]; P = 0 picks windows of about 48 trellis steps.
int clamp_p(int K, int P) {
  if (P <= 0) P = (K + 47) / 48;
  P = std::min(P, K / 8);
  P = std::min(P, (int)CRNT_MAX_P);
  return std::max(P, 1);
}

}  // namespace

struct HarqPool {
  int8_t* arena = nullptr;
  uint32_t slots = 0;
  std::map<std::tuple<uint32_t, uint32_t, uint32_t>, uint32_t> keys;
  std::vector<uint32_t> free_list;
};

struct crnt_ctx {
  int device = 0;
  crnt_config cfg{};
  int num_sms = 0;
  uint32_t* xpowA = nullptr;
  uint32_t* xpowB = nullptr;
  HarqPool harq;
  std::mutex mu;  // guards harq and the staging buffers
  DevBuf stage_in, stage_out;
  cudaStream_t stream = nullptr;
  // serving
  struct Serving* serving = nullptr;
};

struct crnt_plan {
  crnt_ctx* ctx = nullptr;
  std::vector<crnt_tb_params> tbs;
  std::vector<CbDesc> cbs;        // sorted (work-item order)
  std::vector<int> cb_tb, cb_r;   // sorted index -> (tb, r)
  std::vector<TbDesc> tdesc;
  std::vector<WorkItem> items;
  std::vector<lte::Seg> segs;
  std::vector<uint16_t> p_used;
  crnt_plan_info info{};
  int smem = 0;
  // device
  void* d_desc = nullptr;   // cbs | tbs | items
  void* d_scratch = nullptr;
  size_t scratch_zero = 0;  // bytes to clear before each launch
  DecParams prm{};
  // host staging for results
  uint8_t* h_res = nullptr;  // pinned: cb_iters | cb_ok | tb_ok
  size_t res_bytes = 0;
  ~crnt_plan() {
    if (d_desc) cudaFree(d_desc);
    if (d_scratch) cudaFree(d_scratch);
    if (h_res) cudaFreeHost(h_res);
  }
};

// ------------------------------------------------------------------ API
extern "C" {

int crnt_version(void) { return CRNT_VERSION; }

const char* crnt_strerror(int code) {
  switch (code) {
    case CRNT_OK: return "ok";
    case CRNT_EINVAL: return "invalid argument";
    case CRNT_ENOMEM: return "out of memory or memory budget";
    case CRNT_EAGAIN: return "admission refused, retry later";
    case CRNT_ETIMEDOUT: return "bounded wait expired";
    case CRNT_EDEVICE: return "CUDA error";
    case CRNT_ENOTFOUND: return "not found";
    default: return "unknown error";
  }
}

int crnt_qpp_params(uint32_t K, uint32_t* f1, uint32_t* f2) {
  const int i = lte::index_of((int)K);
  if (i < 0 || !f1 || !f2) return CRNT_EINVAL;
  *f1 = lte::kF1[i];
  *f2 = lte::kF2[i];
  return CRNT_OK;
}

int crnt_tb_layout(const crnt_tb_params* tb, crnt_cb_layout* cbs, uint32_t* C) {
  if (!tb || !cbs || !C) return CRNT_EINVAL;
  lte::Seg s;
  int rc = validate(*tb, &s);
  if (rc) return rc;
  uint32_t eoff = 0, soff = 0;
  for (int r = 0; r < s.C; r++) {
    const int K = lte::cb_k(s, r);
    crnt_cb_layout& c = cbs[r];
    c.K = K;
    c.F = r == 0 ? s.F : 0;
    c.E = lte::e_r((int)tb->G, tb->Qm, tb->NL, s.C, r);
    c.k0 = lte::k0(K, tb->rv);
    c.Ncb = lte::ncb(K);
    c.llr_offset = eoff;
    c.soft_offset = soff;
    c.crc_b = s.C > 1;
    c.P = (uint32_t)clamp_p(K, tb->P);
    c.W = (K + c.P - 1) / c.P;
    eoff += c.E;
    soff += c.Ncb;
  }
  *C = s.C;
  return CRNT_OK;
}

int crnt_create(crnt_ctx** out, const crnt_config* cfg) {
  if (!out) return CRNT_EINVAL;
  *out = nullptr;
  crnt_ctx* c = new (std::nothrow) crnt_ctx;
  if (!c) return CRNT_ENOMEM;
  if (cfg) c->cfg = *cfg;
  if (!c->cfg.harq_slots) c->cfg.harq_slots = 4096;
  if (!c->cfg.mem_budget) c->cfg.mem_budget = 8ull << 30;
  if (!c->cfg.max_inflight) c->cfg.max_inflight = 4096;
  if (!c->cfg.deadline_us) c->cfg.deadline_us = 1000;
  c->device = c->cfg.device;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->device < 0 || c->device >= ndev) {
    cudaGetLastError();
    delete c;
    return CRNT_EDEVICE;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    delete c;
    return CRNT_EDEVICE;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  std::vector<uint32_t> xa = xpow_table(kGA, kXpowA), xb = xpow_table(kGB, kXpowB);
  if (cudaMalloc(&c->xpowA, 4 * kXpowA) != cudaSuccess ||
      cudaMalloc(&c->xpowB, 4 * kXpowB) != cudaSuccess ||
      cudaMemcpy(c->xpowA, xa.data(), 4 * kXpowA, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->xpowB, xb.data(), 4 * kXpowB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    crnt_destroy(c);
    return CRNT_EDEVICE;
  }
  *out = c;
  return CRNT_OK;
}

static void serving_stop(crnt_ctx*) {}

int crnt_destroy(crnt_ctx* ctx) {
  if (!ctx) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  serving_stop(ctx);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->xpowA) cudaFree(ctx->xpowA);
  if (ctx->xpowB) cudaFree(ctx->xpowB);
  if (ctx->harq.arena) cudaFree(ctx->harq.arena);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return CRNT_OK;
}

static int harq_bind(crnt_ctx* ctx, const crnt_tb_params& t, int64_t* off) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  HarqPool& h = ctx->harq;
  if (!h.arena) {
    const uint64_t bytes = (uint64_t)ctx->cfg.harq_slots * kSoftSlot;
    if (bytes > ctx->cfg.mem_budget) return CRNT_ENOMEM;
    if (cudaMalloc(&h.arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      h.arena = nullptr;
      return CRNT_ENOMEM;
    }
    h.slots = ctx->cfg.harq_slots;
    for (uint32_t i = 0; i < h.slots; i++) h.free_list.push_back(h.slots - 1 - i);
  }
  auto key = std::make_tuple(t.cell, t.ue, t.harq_pid);
  auto it = h.keys.find(key);
  uint32_t slot;
  if (it != h.keys.end()) {
    slot = it->second;
  } else {
    if (!t.new_data) return CRNT_ENOTFOUND;
    if (h.free_list.empty()) return CRNT_EAGAIN;
    slot = h.free_list.back();
    h.free_list.pop_back();
    h.keys[key] = slot;
  }
  *off = (int64_t)slot * kSoftSlot;
  return CRNT_OK;
}

int crnt_harq_release(crnt_ctx* ctx, uint32_t cell, uint32_t ue, uint32_t harq_pid) {
  if (!ctx) return CRNT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->harq.keys.find(std::make_tuple(cell, ue, harq_pid));
  if (it == ctx->harq.keys.end()) return CRNT_ENOTFOUND;
  ctx->harq.free_list.push_back(it->second);
  ctx->harq.keys.erase(it);
  return CRNT_OK;
}

int crnt_plan_create(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, crnt_plan** out) {
  if (!ctx || !tbs || !out || n == 0) return CRNT_EINVAL;
  *out = nullptr;
  std::unique_ptr<crnt_plan> pl(new (std::nothrow) crnt_plan);
  if (!pl) return CRNT_ENOMEM;
  pl->ctx = ctx;
  pl->tbs.assign(tbs, tbs + n);
  pl->segs.resize(n);
  pl->p_used.resize(n);
  pl->tdesc.resize(n);
  std::vector<CbDesc> all;  // TB order
  std::vector<int> all_tb, all_r;
  int64_t llr_off = 0, out_off = 0, dbg_off = 0;
  uint64_t steps = 0, info_bits = 0;
  std::map<std::pair<int, int>, std::pair<int, int>> divcache;
  for (uint32_t t = 0; t < n; t++) {
    const crnt_tb_params& tp = tbs[t];
    lte::Seg& s = pl->segs[t];
    int rc = validate(tp, &s);
    if (rc) return rc;
    int64_t soft_base = -1;
    if (tp.flags & CRNT_F_HARQ) {
      rc = harq_bind(ctx, tp, &soft_base);
      if (rc) return rc;
    }
    TbDesc& td = pl->tdesc[t];
    td.out_off = out_off;
    td.A = (int)tp.A;
    td.C = s.C;
    td.cb0 = (int)all.size();
    pl->p_used[t] = (uint16_t)clamp_p(s.Kp, tp.P);
    const int B = (int)tp.A + 24;
    int pay_off = 0, eoff = 0, soff = 0;
    for (int r = 0; r < s.C; r++) {
      CbDesc d;
      memset(&d, 0, sizeof d);
      const int K = lte::cb_k(s, r);
      const int F = r == 0 ? s.F : 0;
      const int Pr = clamp_p(K, tp.P);
      const int W = (K + Pr - 1) / Pr;
      d.K = K;
      d.F = F;
      d.E = lte::e_r((int)tp.G, tp.Qm, tp.NL, s.C, r);
      d.k0 = lte::k0(K, tp.rv);
      d.W = W;
      d.P = (K + W - 1) / W;
      auto key = std::make_pair(K, W);
      auto dc = divcache.find(key);
      if (dc == divcache.end()) {
        int M, sh;
        if (!find_divider(W, K + 4, &M, &sh)) return CRNT_EINVAL;
        dc = divcache.emplace(key, std::make_pair(M, sh)).first;
      }
      d.divM = dc->second.first;
      d.divS = dc->second.second;
      const int ki = lte::index_of(K);
      d.f1 = lte::kF1[ki];
      d.f2 = lte::kF2[ki];
      d.f2x2 = (int)((2ll * d.f2) % K);
      d.f2sub = (int)((2ll * kSub * d.f2) % K);
      d.f2jump = (int)((2ll * kSub * kSub * d.f2) % K);
      d.R = lte::rows(K);
      d.ND = 32 * d.R - (K + 4);
      d.Nv = 3 * (K + 4) - 2 * F;
      const int X = d.ND + F;
      if ((X >> 5) + 1 > d.R) return CRNT_EINVAL;
      uint32_t mb = 0, m2 = 0;
      for (int c = 0; c < 32; c++) {
        const int pc = lte::bitrev5(c);
        if (pc < (X & 31)) mb |= 1u << c;
        if (pc < d.ND - 1) m2 |= 1u << c;
      }
      d.maskB = mb;
      d.mask2 = m2;
      int rank0 = 0;
      for (int w = 0; w < d.k0; w++) rank0 += lte::w_non_null(K, F, w) ? 1 : 0;
      d.rank0 = rank0;
      d.tb = (int)t;
      d.r = r;
      d.llr_off = llr_off + eoff;
      d.soft_off = soft_base >= 0 ? soft_base + soff : -1;
      d.pay_bits = K - F - s.L;
      d.pay_off = pay_off;
      d.n_after = B - pay_off - d.pay_bits;
      d.dbg_off = (int32_t)dbg_off;
      d.crc_b = s.C > 1;
      d.max_iter = tp.max_iter;
      d.early_stop = tp.early_stop ? 1 : 0;
      d.new_data = tp.new_data ? 1 : 0;
      pay_off += d.pay_bits;
      eoff += d.E;
      soff += lte::ncb(K);
      dbg_off += K + 4;
      steps += K;
      all.push_back(d);
      all_tb.push_back((int)t);
      all_r.push_back(r);
    }
    if (eoff != (int)tp.G || pay_off != B) return CRNT_EINVAL;
    llr_off += tp.G;
    out_off += tp.A / 8;
    info_bits += tp.A;
  }
  // ---- work items: group CBs of equal (K, P), longest work first
  std::vector<int> order(all.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const CbDesc &a = all[x], &b = all[y];
    const int ca = a.W * a.max_iter, cb = b.W * b.max_iter;
    if (ca != cb) return ca > cb;
    if (a.K != b.K) return a.K > b.K;
    return a.P > b.P;
  });
  pl->cbs.reserve(all.size());
  std::vector<std::pair<int, WorkItem>> items;  // (cost, item)
  size_t i = 0;
  int max_slot_bytes = 0;
  while (i < order.size()) {
    const CbDesc& h = all[order[i]];
    const int slot = align16(dec_cb_smem(h.K, h.P, h.W));
    if (slot > kSmemBudget) return CRNT_EINVAL;
    const int gmax = std::max(1, std::min(kThreads / h.P, kSmemBudget / slot));
    WorkItem wi;
    wi.cb0 = (int)pl->cbs.size();
    wi.n = 0;
    wi.smem_per_cb = slot;
    wi.pad0 = 0;
    while (i < order.size() && wi.n < gmax) {
      const CbDesc& c = all[order[i]];
      if (c.K != h.K || c.P != h.P) break;
      pl->cbs.push_back(c);
      pl->cb_tb.push_back(all_tb[order[i]]);
      pl->cb_r.push_back(all_r[order[i]]);
      wi.n++;
      i++;
    }
    max_slot_bytes = std::max(max_slot_bytes, wi.n * slot);
    items.push_back(std::make_pair(h.W * h.max_iter, wi));
  }
  for (auto& it : items) pl->items.push_back(it.second);
  pl->smem = 2048 + max_slot_bytes;

  cudaSetDevice(ctx->device);
  const int per_sm = decode_occupancy(pl->smem);
  if (per_sm < 1) return CRNT_EDEVICE;
  const int grid = std::min<int>((int)pl->items.size(), per_sm * ctx->num_sms);

  crnt_plan_info& inf = pl->info;
  inf.n_tb = n;
  inf.n_cb = (uint32_t)pl->cbs.size();
  inf.llr_bytes = (uint64_t)llr_off;
  inf.out_bytes = (uint64_t)out_off;
  inf.info_bits = info_bits;
  inf.trellis_steps = steps;
  inf.dbg_elems = (uint64_t)dbg_off;
  inf.n_items = (uint32_t)pl->items.size();
  inf.grid = (uint32_t)grid;

  // ---- device buffers
  const size_t ncb = pl->cbs.size();
  const size_t b_cbs = sizeof(CbDesc) * ncb, b_tbs = sizeof(TbDesc) * n,
               b_items = sizeof(WorkItem) * pl->items.size();
  const size_t off_tbs = (b_cbs + 255) & ~size_t(255);
  const size_t off_items = off_tbs + ((b_tbs + 255) & ~size_t(255));
  const size_t desc_bytes = off_items + b_items;
  if (cudaMalloc(&pl->d_desc, desc_bytes) != cudaSuccess) {
    cudaGetLastError();
    return CRNT_ENOMEM;
  }
  std::vector<uint8_t> host(desc_bytes, 0);
  memcpy(host.data(), pl->cbs.data(), b_cbs);
  memcpy(host.data() + off_tbs, pl->tdesc.data(), b_tbs);
  memcpy(host.data() + off_items, pl->items.data(), b_items);
  if (cudaMemcpy(pl->d_desc, host.data(), desc_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return CRNT_EDEVICE;
  // scratch: state | tb_done | tb_crc (zeroed each launch) | cb_iters | cb_ok | tb_ok
  const size_t s_state = 256, s_done = ((4 * n + 255) & ~size_t(255)),
               s_crc = ((8 * n + 255) & ~size_t(255));
  pl->scratch_zero = s_state + s_done + s_crc;
  pl->res_bytes = 2 * ncb + n;
  if (cudaMalloc(&pl->d_scratch, pl->scratch_zero + pl->res_bytes) != cudaSuccess) {
    cudaGetLastError();
    return CRNT_ENOMEM;
  }
  if (cudaMallocHost((void**)&pl->h_res, pl->res_bytes) != cudaSuccess) {
    cudaGetLastError();
    return CRNT_ENOMEM;
  }
  uint8_t* sc = (uint8_t*)pl->d_scratch;
  DecParams& p = pl->prm;
  p.cbs = (const CbDesc*)pl->d_desc;
  p.tbs = (const TbDesc*)((uint8_t*)pl->d_desc + off_tbs);
  p.items = (const WorkItem*)((uint8_t*)pl->d_desc + off_items);
  p.n_items = (int)pl->items.size();
  p.n_cbs = (int)ncb;
  p.n_tbs = (int)n;
  p.soft = ctx->harq.arena;
  p.state = (DecState*)sc;
  p.tb_done = (int32_t*)(sc + s_state);
  p.tb_crc = (uint32_t*)(sc + s_state + s_done);
  p.cb_iters = sc + pl->scratch_zero;
  p.cb_ok = p.cb_iters + ncb;
  p.tb_ok = p.cb_ok + ncb;
  p.xpowA = ctx->xpowA;
  p.xpowB = ctx->xpowB;
  *out = pl.release();
  return CRNT_OK;
}

int crnt_plan_get_info(const crnt_plan* plan, crnt_plan_info* info) {
  if (!plan || !info) return CRNT_EINVAL;
  *info = plan->info;
  return CRNT_OK;
}

int crnt_plan_launch_debug(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream,
                           int8_t* dbg_d, int16_t* dbg_ext, uint8_t* dbg_hard) {
  if (!plan || !llr || !out) return CRNT_EINVAL;
  if ((dbg_ext == nullptr) != (dbg_hard == nullptr)) return CRNT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DecParams p = plan->prm;
  p.llr = llr;
  p.out = out;
  p.soft = plan->ctx->harq.arena;
  p.dbg_d = dbg_d;
  p.dbg_ext = dbg_ext;
  p.dbg_hard = dbg_hard;
  if (cudaMemsetAsync(plan->d_scratch, 0, plan->scratch_zero, s) != cudaSuccess) return CRNT_EDEVICE;
  if (launch_decode(p, (int)plan->info.grid, plan->smem, s) != cudaSuccess) return CRNT_EDEVICE;
  return CRNT_OK;
}

int crnt_plan_launch(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream) {
  return crnt_plan_launch_debug(plan, llr, out, stream, nullptr, nullptr, nullptr);
}

int crnt_plan_results(crnt_plan* plan, crnt_tb_result* res, void* stream) {
  if (!plan || !res) return CRNT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(plan->h_res, plan->prm.cb_iters, plan->res_bytes, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CRNT_EDEVICE;
  const size_t ncb = plan->cbs.size();
  const uint32_t n = plan->info.n_tb;
  for (uint32_t t = 0; t < n; t++) {
    crnt_tb_result& r = res[t];
    memset(&r, 0, sizeof r);
    const lte::Seg& sg = plan->segs[t];
    r.status = CRNT_OK;
    r.C = (uint8_t)sg.C;
    r.K_plus = (uint16_t)sg.Kp;
    r.K_minus = (uint16_t)sg.Km;
    r.F = (uint16_t)sg.F;
    r.P_used = plan->p_used[t];
    r.tb_crc_ok = plan->h_res[2 * ncb + t];
  }
  for (size_t i = 0; i < ncb; i++) {
    crnt_tb_result& r = res[plan->cb_tb[i]];
    r.cb_iters[plan->cb_r[i]] = plan->h_res[i];
    r.cb_crc_ok[plan->cb_r[i]] = plan->h_res[ncb + i];
  }
  return CRNT_OK;
}

int crnt_plan_destroy(crnt_plan* plan) {
  if (!plan) return CRNT_EINVAL;
  cudaSetDevice(plan->ctx->device);
  delete plan;
  return CRNT_OK;
}

int crnt_decode_batch(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, const int8_t* llr,
                      uint8_t* out, crnt_tb_result* res) {
  if (!ctx || !tbs || !llr || !out || !res || n == 0) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  crnt_plan* plan = nullptr;
  int rc = crnt_plan_create(ctx, tbs, n, &plan);
  if (rc) return rc;
  const bool llr_dev = is_device_ptr(llr), out_dev = is_device_ptr(out);
  std::unique_lock<std::mutex> lk(ctx->mu);
  const int8_t* d_llr = llr;
  uint8_t* d_out = out;
  cudaStream_t s = ctx->stream;
  rc = CRNT_OK;
  if (!llr_dev) {
    if (ctx->stage_in.ensure(plan->info.llr_bytes) != cudaSuccess ||
        cudaMemcpyAsync(ctx->stage_in.p, llr, plan->info.llr_bytes, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      rc = CRNT_EDEVICE;
    d_llr = (const int8_t*)ctx->stage_in.p;
  }
  if (!rc && !out_dev) {
    if (ctx->stage_out.ensure(plan->info.out_bytes) != cudaSuccess) rc = CRNT_EDEVICE;
    d_out = (uint8_t*)ctx->stage_out.p;
  }
  if (!rc) rc = crnt_plan_launch(plan, d_llr, d_out, s);
  if (!rc && !out_dev &&
      cudaMemcpyAsync(out, d_out, plan->info.out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = CRNT_EDEVICE;
  if (!rc) rc = crnt_plan_results(plan, res, s);
  lk.unlock();
  crnt_plan_destroy(plan);
  return rc;
}

int crnt_decode_tb(crnt_ctx* ctx, const int8_t* llr, const crnt_tb_params* tb, uint8_t* out,
                   crnt_tb_result* res) {
  return crnt_decode_batch(ctx, tb, 1, llr, out, res);
}

int crnt_encode_batch(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, const uint8_t* bits,
                      uint8_t* e_out) {
  if (!ctx || !tbs || !bits || !e_out || n == 0) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  std::vector<EncCb> cbs;
  std::vector<int64_t> in_off(n);
  std::vector<int32_t> As(n);
  int64_t ioff = 0, eoff = 0;
  for (uint32_t t = 0; t < n; t++) {
    lte::Seg s;
    int rc = validate(tbs[t], &s);
    if (rc) return rc;
    in_off[t] = ioff;
    As[t] = (int32_t)tbs[t].A;
    int pay_off = 0;
    for (int r = 0; r < s.C; r++) {
      EncCb c;
      memset(&c, 0, sizeof c);
      const int K = lte::cb_k(s, r);
      c.K = K;
      c.F = r == 0 ? s.F : 0;
      c.E = lte::e_r((int)tbs[t].G, tbs[t].Qm, tbs[t].NL, s.C, r);
      c.R = lte::rows(K);
      c.ND = 32 * c.R - (K + 4);
      const int k0 = lte::k0(K, tbs[t].rv);
      int rank0 = 0;
      for (int w = 0; w < k0; w++) rank0 += lte::w_non_null(K, c.F, w) ? 1 : 0;
      c.rank0 = rank0;
      const int ki = lte::index_of(K);
      c.f1 = lte::kF1[ki];
      c.f2 = lte::kF2[ki];
      c.tb = (int)t;
      c.pay_bits = K - c.F - s.L;
      c.pay_off = pay_off;
      c.crc_b = s.C > 1;
      c.e_off = eoff;
      pay_off += c.pay_bits;
      eoff += c.E;
      cbs.push_back(c);
    }
    ioff += tbs[t].A / 8;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = ctx->stream;
  const size_t b_cbs = sizeof(EncCb) * cbs.size(), b_off = 8 * n, b_A = 4 * n;
  const size_t o_off = (b_cbs + 255) & ~size_t(255), o_A = o_off + ((b_off + 255) & ~size_t(255));
  const size_t o_bits = o_A + ((b_A + 255) & ~size_t(255));
  const bool bits_dev = is_device_ptr(bits), out_dev = is_device_ptr(e_out);
  const size_t total = o_bits + (bits_dev ? 0 : (size_t)ioff);
  if (ctx->stage_in.ensure(total) != cudaSuccess) return CRNT_ENOMEM;
  if (!out_dev && ctx->stage_out.ensure((size_t)eoff) != cudaSuccess) return CRNT_ENOMEM;
  std::vector<uint8_t> host(o_bits, 0);
  memcpy(host.data(), cbs.data(), b_cbs);
  memcpy(host.data() + o_off, in_off.data(), b_off);
  memcpy(host.data() + o_A, As.data(), b_A);
  uint8_t* base = (uint8_t*)ctx->stage_in.p;
  if (cudaMemcpyAsync(base, host.data(), o_bits, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CRNT_EDEVICE;
  if (!bits_dev &&
      cudaMemcpyAsync(base + o_bits, bits, (size_t)ioff, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CRNT_EDEVICE;
  EncParams p;
  p.cbs = (const EncCb*)base;
  p.tb_in_off = (const int64_t*)(base + o_off);
  p.tb_A = (const int32_t*)(base + o_A);
  p.tb_bits = bits_dev ? bits : base + o_bits;
  p.e_out = out_dev ? e_out : (uint8_t*)ctx->stage_out.p;
  p.xpowA = ctx->xpowA;
  p.xpowB = ctx->xpowB;
  if (launch_encode(p, (int)cbs.size(), st) != cudaSuccess) return CRNT_EDEVICE;
  if (!out_dev &&
      cudaMemcpyAsync(e_out, p.e_out, (size_t)eoff, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CRNT_EDEVICE;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRNT_EDEVICE;
  return CRNT_OK;
}

int crnt_encode_tb(crnt_ctx* ctx, const uint8_t* bits, const crnt_tb_params* tb, uint8_t* e_out) {
  return crnt_encode_batch(ctx, tb, 1, bits, e_out);
}

int crnt_submit(crnt_ctx*, const crnt_tb_params*, const int8_t* const*, uint32_t, uint64_t*) {
  return CRNT_EINVAL;
}
int crnt_poll(crnt_ctx*, crnt_tb_result*, const uint8_t**, uint32_t, uint32_t) { return CRNT_EINVAL; }

}  // extern "C"
