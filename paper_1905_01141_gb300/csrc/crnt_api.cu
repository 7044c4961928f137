// crnt_api.cu -- host runtime and C ABI of the decoding library.
//
// The planner turns a batch of transport blocks into code-block descriptors
// and work items (the device counterpart of the paper's Algorithm 1 queuing
// step), binds HARQ processes to device soft buffers, and launches the fused
// decode kernel whose CTAs drain the work queue (Algorithm 2).  Plans keep
// grow-only buffers, so re-planning a batch no larger than a previous one
// allocates nothing.  The serving loop lives in serve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "runtime.h"

using namespace crnt;

namespace crnt {

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
  uint32_t x32 = 1;
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

// Exact division q / W as (q * M) >> s for 0 <= q < qmax, verified
// exhaustively over q < 8192 (every K + 4 <= 6148 is below that bound), so one
// divider per W serves every CB; kept in a lock-free table filled on first use
// (racing threads compute and store the same value).
bool find_divider(int W, int qmax, int* M, int* s) {
  constexpr int kQ = 8192;
  static std::atomic<uint64_t> table[lte::kZ + 1];
  if (W < 1 || W > lte::kZ || qmax > kQ) return false;
  uint64_t v = table[W].load(std::memory_order_relaxed);
  if (!v) {
    for (int sh = 0; sh < 32 && !v; sh++) {
      const uint64_t m = ((1ull << sh) + W - 1) / W;
      if (m * (uint64_t)kQ >= (1ull << 32)) break;
      bool ok = true;
      for (int q = 0; q < kQ && ok; q++) ok = (int)((q * m) >> sh) == q / W;
      if (ok) v = (m << 8) | (uint64_t)sh | (1ull << 63);
    }
    if (!v) return false;
    table[W].store(v, std::memory_order_relaxed);
  }
  *M = (int)((v & ~(1ull << 63)) >> 8);
  *s = (int)(v & 0xFF);
  return true;
}


// Address under which kernels can use p: device and managed memory as is,
// page-locked host memory (cudaHostAlloc / cudaHostRegister) through its
// mapped device address -- kernels then read and write it in place over the
// CPU-GPU link; nullptr for pageable host memory, which must be staged.
// host_memory: p is page-locked or pageable host memory.
bool host_memory(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown to CUDA: pageable
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}
void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return (void*)p;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  return nullptr;
}

// Column masks of the circular-buffer rank formula (see rm_geom.cuh): bit c
// of maskB is [P(c) < (ND + F) mod 32], bit c of mask2 is [P(c) < ND - 1],
// with P the bit-reversal column permutation.  kColsBelow[x] holds the
// columns c with P(c) < x.
struct ColsBelow {
  uint32_t m[33];
  constexpr ColsBelow() : m() {
    for (int x = 0; x <= 32; x++) {
      uint32_t v = 0;
      for (int c = 0; c < 32; c++) {
        int pc = 0;
        for (int i = 0; i < 5; i++) pc |= ((c >> i) & 1) << (4 - i);
        if (pc < x) v |= 1u << c;
      }
      m[x] = v;
    }
  }
};
constexpr ColsBelow kColsBelow{};

void rm_masks(int ND, int F, uint32_t* maskB, uint32_t* mask2) {
  const int X = ND + F;
  *maskB = kColsBelow.m[X & 31];
  *mask2 = ND >= 1 ? kColsBelow.m[ND - 1 < 32 ? ND - 1 : 32] : 0u;
}

// Non-NULL positions before k0.  k0 = R (24 rv + 2) always starts a column:
// column 2 or 26 of v0 (rv 0, 1) or column 9 or 21 of the v1/v2 part.
int rank_of_k0(int K, int F, int rv, uint32_t maskB, uint32_t mask2) {
  const int R = lte::rows(K), ND = 32 * R - (K + 4), X = ND + F, xa = X >> 5;
  const int k0 = lte::k0(K, rv);
  auto pre0 = [&](int c) { return xa * c + __builtin_popcount(maskB & ((1u << c) - 1u)); };
  if (k0 < 32 * R) {
    const int c = k0 / R;
    return c * R - pre0(c);
  }
  const int c = (k0 - 32 * R) / (2 * R);
  return (32 * R - X) + 2 * R * c - pre0(c) - __builtin_popcount(mask2 & ((1u << c) - 1u));
}

int harq_bind(crnt_ctx* ctx, const crnt_tb_params& t, int64_t* off) {
  std::lock_guard<std::mutex> lk(ctx->harq_mu);
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

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Process-wide window-count table (crnt_tune_set / crnt_autotune).
std::atomic<uint8_t> g_tuned[lte::kNumK];
// Process-wide forward-recursion radix per CB size (2 or 4; 0 reads as 2).
std::atomic<uint8_t> g_radix[lte::kNumK];
// Process-wide CTA shape per CB size: 1 = one CB per thread (windows across
// the threads), 2 = CB pairs in 16-bit lanes; 0 reads as 1.
std::atomic<uint8_t> g_shape[lte::kNumK];

int tuned_p(int K) {
  const int ki = lte::index_of(K);
  return ki < 0 ? 0 : (int)g_tuned[ki].load(std::memory_order_relaxed);
}

thread_local int t_radix_override = -1;
thread_local int t_shape_override = -1;

uint8_t shape_of(int K) {
  if (t_shape_override > 0) return (uint8_t)t_shape_override;
  const int ki = lte::index_of(K);
  return ki >= 0 && g_shape[ki].load(std::memory_order_relaxed) == 2 ? 2 : 1;
}

// De-rate-matching map of CB size K with P windows and F filler bits: the
// circular buffer w = [v0, interlace(v1, v2)] of TS 36.212 5.1.4.1 walked in
// order; the r-th non-NULL position p gets (p << 16) | destination, the
// destination being stream s, bit y - ND of its sub-block interleaver input
// (y the padded index; NULL when y < ND, a dummy, or, in streams 0 and 1,
// when y < ND + F, a filler bit), stored at s tp + transposed index, or, for
// the four tail bits of each stream, 3 tp + 3 (y - ND - K) + s.  Returns the
// number of non-NULL positions (entries written: at most n).  fkey (may be
// null, n entries): per entry, the bit index y - ND where a filler count
// above it would make the position NULL (streams 0 and 1, bits below 64),
// else 64 -- the map of F > 0 is the F = 0 map without the entries whose key
// is below F.
static int build_dm(uint32_t* hd, uint8_t* fkey, int n, int K, int P, int F) {
  const int W = (K + P - 1) / P, tp = W * P;
  const int R = lte::rows(K), KPI = 32 * R, ND = KPI - (K + 4);
  std::vector<uint32_t> tr((size_t)K);  // transposed index of bit d, by walking
  for (int d = 0, r = 0, c = 0; d < K; d++) {
    tr[(size_t)d] = (uint32_t)(r * P + c);
    if (++r == W) {
      r = 0;
      c++;
    }
  }
  int nv = 0;
  auto put = [&](int p, int s, int y) {
    if (y < ND || (s < 2 && y < ND + F)) return;  // NULL
    const int di = y - ND;
    const int dst = di < K ? s * tp + (int)tr[(size_t)di] : 3 * tp + 3 * (di - K) + s;
    if (nv < n) {
      hd[nv] = ((uint32_t)p << 16) | (uint32_t)dst;
      if (fkey) fkey[nv] = (uint8_t)(s < 2 && di < 64 ? di : 64);
    }
    nv++;
  };
  for (int c = 0; c < 32; c++) {
    int pc = 0;
    for (int b = 0; b < 5; b++) pc |= ((c >> b) & 1) << (4 - b);
    for (int i = 0; i < R; i++) put(c * R + i, 0, pc + 32 * i);
  }
  for (int c = 0; c < 32; c++) {
    int pc = 0;
    for (int b = 0; b < 5; b++) pc |= ((c >> b) & 1) << (4 - b);
    for (int i = 0; i < R; i++) {
      const int p = KPI + 2 * (c * R + i);
      put(p, 1, pc + 32 * i);
      put(p + 1, 2, (pc + 32 * i + 1) % KPI);
    }
  }
  return nv;
}

// Byte offset of the (K, P, F) de-rate-matching map inside the (K, P) entry
// (after the address tables, from a 16-byte boundary; maps for F = 0, 8,
// ..., 56 in turn).  A map holds 3 (K + 4) - 2 F entries of 4 bytes, a
// multiple of 16 bytes (K + 4 is a multiple of 4, F of 8), so every map
// starts on a 16-byte boundary and the decoder may bulk-copy it in 16-byte
// units.
static size_t dm_offset(int K, int P, int F) {
  const int W = (K + P - 1) / P, ng = (W + kSub - 1) / kSub + 2;
  size_t off = ((size_t)ng * P * 24 + 15) & ~size_t(15);
  for (int f = 0; f < F; f += 8) off += (size_t)(3 * (K + 4) - 2 * f) * 4;
  return off;
}

// Interleaved-pass address table of CB size K with P windows (layout of
// CbDesc::qt / qq): entry (g, p, k), step j = kSub g + k of window p, holds
// the transposed index of q = PI(p W + j) in ht and q in hq.  ki: K's index.
static void build_qt(uint32_t* ht, uint16_t* hq, int ki, int K, int P) {
  const int W = (K + P - 1) / P;
  const int64_t f1 = lte::kF1[ki], f2 = lte::kF2[ki];
  for (int p = 0; p < P; p++) {
    const int lo = p * W, len = std::min(W, K - lo);
    for (int j = 0; j < len; j++) {
      const int64_t i = lo + j;
      const int q = (int)((f1 * i + (f2 * i % K) * i) % K);
      const size_t e = ((size_t)(j / kSub) * P + p) * kSub + j % kSub;
      ht[e] = (uint32_t)((q % W) * P + q / W);
      hq[e] = (uint16_t)q;
    }
  }
}

// Copies h (bytes) into the tables' device memory (caller holds qs->mu).
static const uint8_t* qt_upload(QTabs* qs, const void* h, size_t bytes) {
  const size_t need = al256(bytes);
  if (qs->left < need) {
    const size_t sz = std::max(need, (size_t)8 << 20);
    void* p = nullptr;
    if (cudaMalloc(&p, sz) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    qs->chunks.push_back(p);
    qs->cur = (uint8_t*)p;
    qs->left = sz;
  }
  uint8_t* dev = qs->cur;
  if (cudaMemcpyAsync(dev, h, bytes, cudaMemcpyHostToDevice, qs->stream) != cudaSuccess ||
      cudaStreamSynchronize(qs->stream) != cudaSuccess)
    return nullptr;
  qs->cur += need;
  qs->left -= need;
  return dev;
}

// Tables of CB size K with P windows.  Entry (g, p, k) of the first is step
// j = kSub g + k of window p of the interleaved pass: natural position q =
// PI(p W + j) (QPP, Sec. IV-B Fig. 4's interleaver) and its transposed
// shared-memory index (q mod W) P + q / W, laid out as the decoder reads
// them (one 16-byte group of kSub addresses per window, windows adjacent);
// steps past a window's end and the two extra last groups are zero.  The
// de-rate-matching map without filler bits follows.
const uint4* qtab_get(crnt_ctx* ctx, int K, int P) {
  QTabs* qs = ctx->qtabs;
  const int ki = lte::index_of(K);
  if (!qs || ki < 0 || P < 1 || P > (int)CRNT_MAX_P) return nullptr;
  const uint4* r = qs->t[ki][P].load(std::memory_order_acquire);
  if (r) return r;
  std::lock_guard<std::mutex> lk(qs->mu);
  r = qs->t[ki][P].load(std::memory_order_relaxed);
  if (r) return r;
  const int W = (K + P - 1) / P;
  if ((K + W - 1) / W != P) return nullptr;
  const int ng = (W + kSub - 1) / kSub + 2, Nv = 3 * (K + 4);
  const size_t tb = (size_t)ng * P * 16;
  const size_t bytes = dm_offset(K, P, 64);
  std::vector<uint8_t> h(bytes, 0);
  build_qt((uint32_t*)h.data(), (uint16_t*)(h.data() + tb), ki, K, P);
  std::vector<uint8_t> fkey((size_t)Nv);
  uint32_t* m0 = (uint32_t*)(h.data() + dm_offset(K, P, 0));
  if (build_dm(m0, fkey.data(), Nv, K, P, 0) != Nv) return nullptr;
  // filler counts F < K: the F = 0 map without the filler bits (the maps of
  // F >= K, which no segmentation produces, stay zero and are never used)
  for (int F = 8; F < 64 && F < K; F += 8) {
    uint32_t* mf = (uint32_t*)(h.data() + dm_offset(K, P, F));
    const int nmax = Nv - 2 * F;
    int nf = 0;
    for (int r = 0; r < Nv; r++)
      if (fkey[(size_t)r] >= F) {
        if (nf < nmax) mf[nf] = m0[r];
        nf++;
      }
    if (nf != nmax) return nullptr;
  }
  r = (const uint4*)qt_upload(qs, h.data(), bytes);
  if (r) qs->t[ki][P].store(r, std::memory_order_release);
  return r;
}

// The de-rate-matching map of (K, P, F) (F, a multiple of 8 below 64 by the
// segmentation of TS 36.212 5.1.2, only on a TB's first CB), stored in the
// (K, P) entry.
const uint32_t* dmap_get(crnt_ctx* ctx, int K, int P, int F) {
  if ((F & 7) || F < 0 || F >= 64 || F >= K) return nullptr;
  const uint4* t = qtab_get(ctx, K, P);
  return t ? (const uint32_t*)((const uint8_t*)t + dm_offset(K, P, F)) : nullptr;
}

uint8_t radix4_of(int K) {
  if (t_radix_override >= 0) return (uint8_t)t_radix_override;
  const int ki = lte::index_of(K);
  return ki >= 0 && g_radix[ki].load(std::memory_order_relaxed) == 4 ? 1 : 0;
}

// Window count for a CB of size K: the caller's P clamped to [1, K/8] and
// [1, CRNT_MAX_P]; P = 0 takes the table's entry, else windows of about 48
// trellis steps.
int clamp_p(int K, int P) {
  if (P <= 0) {
    P = tuned_p(K);
    if (P <= 0) P = (K + 47) / 48;
  }
  P = std::min(P, K / 8);
  P = std::min(P, (int)CRNT_MAX_P);
  return std::max(P, 1);
}

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int validate(const crnt_tb_params& t, lte::Seg* seg) {
  if (t.A < 16 || t.A > 75376 || (t.A & 7)) return CRNT_EINVAL;
  if (t.Qm != 2 && t.Qm != 4 && t.Qm != 6) return CRNT_EINVAL;
  if (t.NL != 1 && t.NL != 2) return CRNT_EINVAL;
  if (t.rv > 3 || t.max_iter < 1 || t.max_iter > 16 || t.early_stop > 2) return CRNT_EINVAL;
  if (t.G == 0 || t.G % (t.Qm * t.NL)) return CRNT_EINVAL;
  if (!lte::segment((int)t.A + 24, seg) || seg->C > CRNT_MAX_CB) return CRNT_EINVAL;
  if (lte::e_r((int)t.G, t.Qm, t.NL, seg->C, 0) < 1) return CRNT_EINVAL;
  if (t.flags & CRNT_F_PUSCH) {
    const int ncol = pusch_cols(t);
    if (ncol > kPuschMaxCols || t.c_init >> 31 || t.G > (uint32_t)(kPuschChunk * kPuschMaxChunks) ||
        t.G % (uint32_t)(t.Qm * t.NL * ncol))
      return CRNT_EINVAL;
  }
  return CRNT_OK;
}

namespace {

bool make_tmpl(int K, int Preq, KTmpl* t) {
  const int ki = lte::index_of(K);
  if (ki < 0) return false;
  const int Pr = clamp_p(K, Preq);
  t->K = K;
  t->W = (K + Pr - 1) / Pr;
  t->P = (K + t->W - 1) / t->W;
  if (!find_divider(t->W, K + 4, &t->divM, &t->divS)) return false;
  t->f1 = lte::kF1[ki];
  t->f2 = lte::kF2[ki];
  t->f2x2 = (int)((2ll * t->f2) % K);
  t->f2sub = (int)((2ll * kSub * t->f2) % K);
  t->f2jump = (int)((2ll * kSub * kSub * t->f2) % K);
  t->R = lte::rows(K);
  t->ND = 32 * t->R - (K + 4);
  t->ncb = lte::ncb(K);
  t->slot = align16(dec_cb_smem(K, t->P, t->W));
  rm_masks(t->ND, 0, &t->maskB0, &t->mask2);
  for (int rv = 0; rv < 4; rv++) t->rank0[rv] = rank_of_k0(K, 0, rv, t->maskB0, t->mask2);
  return true;
}

// Templates of the P = 0 window count (table entry or built-in), filled on
// first use and rebuilt when the table entry changes (ready holds the window
// count the template was built for).
const KTmpl* auto_tmpl(int K) {
  static std::mutex mu;
  static KTmpl table[lte::kNumK];
  static std::atomic<int> ready[lte::kNumK];
  const int ki = lte::index_of(K);
  if (ki < 0) return nullptr;
  const int want = clamp_p(K, 0);
  if (ready[ki].load(std::memory_order_acquire) != want) {
    std::lock_guard<std::mutex> lk(mu);
    if (ready[ki].load(std::memory_order_relaxed) != want) {
      if (!make_tmpl(K, want, &table[ki])) return nullptr;
      ready[ki].store(want, std::memory_order_release);
    }
  }
  return &table[ki];
}

}  // namespace

// Everything about one TB that does not depend on the batch it joins
// (tb_prepare), then the batch (plan_assemble).  Pass 1 of the batch fixes
// each TB's offsets and the sort key of each CB; pass 2 copies the CB
// descriptors in sorted (work-item) order straight into the pinned staging
// buffer and adds the TB's offsets.
int tb_prepare(crnt_ctx* ctx, const crnt_tb_params& tp, TbPrep* out) {
  lte::Seg& s = out->s;
  int rc = validate(tp, &s);
  if (rc) return rc;
  TbPre& pr = out->pr;
  pr.llr = pr.dbg = 0;
  pr.cb0 = 0;
  pr.soft = -1;
  for (int h = 0; h < 2; h++) {
    const int K = h ? s.Kp : s.Km;
    KTmpl& tm = h ? pr.tp : pr.tm;
    if (h == 0 && s.Cm == 0) continue;
    if (tp.P == 0) {
      const KTmpl* a = auto_tmpl(K);
      if (!a) return CRNT_EINVAL;
      tm = *a;
    } else if (!make_tmpl(K, tp.P, &tm)) {
      return CRNT_EINVAL;
    }
    if (tm.slot > kSmemBudget) return CRNT_EINVAL;
  }
  if (((pr.tp.ND + s.F) >> 5) + 1 > pr.tp.R ||
      (s.Cm && ((pr.tm.ND + s.F) >> 5) + 1 > pr.tm.R))
    return CRNT_EINVAL;
  // the soft buffer is bound last: a TB refused above binds none
  if (tp.flags & CRNT_F_HARQ) {
    rc = harq_bind(ctx, tp, &pr.soft);
    if (rc) return rc;
  }
  const int Gp = (int)tp.G / (tp.NL * tp.Qm);
  pr.n_lo = s.C - Gp % s.C;
  pr.E_lo = tp.NL * tp.Qm * (Gp / s.C);
  pr.E_hi = tp.NL * tp.Qm * ((Gp + s.C - 1) / s.C);
  out->p_used = (uint16_t)pr.tp.P;
  // CB descriptors in r order: LLR and debug offsets from the TB's own
  // first LLR byte and debug element, TB index 0
  for (int r = 0; r < s.C; r++) {
    const KTmpl& tm = r < s.Cm ? pr.tm : pr.tp;
    const int F = r == 0 ? s.F : 0;
    const int nm = std::min(r, s.Cm), np = r - nm;  // earlier CBs of size K-, K+
    const int sumK = nm * s.Km + np * s.Kp;
    const int sumNcb = nm * (s.Cm ? pr.tm.ncb : 0) + np * pr.tp.ncb;
    const int eoff = r <= pr.n_lo ? r * pr.E_lo : pr.n_lo * pr.E_lo + (r - pr.n_lo) * pr.E_hi;
    const int pay_off = sumK - (r > 0 ? s.F : 0) - r * s.L;
    CbDesc& d = out->cb[r];
    d.K = tm.K;
    d.F = F;
    d.E = r < pr.n_lo ? pr.E_lo : pr.E_hi;
    d.k0 = lte::k0(tm.K, tp.rv);
    d.P = tm.P;
    d.W = tm.W;
    d.divM = tm.divM;
    d.divS = tm.divS;
    d.f1 = tm.f1;
    d.f2 = tm.f2;
    d.f2x2 = tm.f2x2;
    d.f2sub = tm.f2sub;
    d.f2jump = tm.f2jump;
    d.R = tm.R;
    d.ND = tm.ND;
    d.Nv = 3 * (tm.K + 4) - 2 * F;
    if (F == 0) {
      d.maskB = tm.maskB0;
      d.mask2 = tm.mask2;
      d.rank0 = tm.rank0[tp.rv];
    } else {
      rm_masks(tm.ND, F, &d.maskB, &d.mask2);
      d.rank0 = rank_of_k0(tm.K, F, tp.rv, d.maskB, d.mask2);
    }
    d.tb = 0;
    d.r = r;
    d.llr_off = eoff;
    d.soft_off = pr.soft >= 0 ? pr.soft + sumNcb : -1;
    d.pay_bits = tm.K - F - s.L;
    d.pay_off = pay_off;
    d.n_after = ((int)tp.A + 24) - pay_off - d.pay_bits;
    d.dbg_off = sumK + 4 * r;
    d.crc_b = s.C > 1;
    d.max_iter = tp.max_iter;
    d.early_stop = tp.early_stop;  // 0 none, 1 CRC, 2 mutual information
    d.new_data = tp.new_data ? 1 : 0;
    d.purge = (tp.flags & CRNT_F_PURGE) && s.C > 1 ? 1 : 0;
    d.radix4 = radix4_of(tm.K);
    d.qt = qtab_get(ctx, tm.K, tm.P);
    d.qq = qtab_q(d.qt, tm.K, tm.P);
    d.dm = dmap_get(ctx, tm.K, tm.P, F);
    memset(d.pad0, 0, sizeof d.pad0);
  }
  return CRNT_OK;
}

int plan_build(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, crnt_plan* pl,
               cudaStream_t stream, const int64_t* llr_base, uint32_t batch_cbs) {
  if (pl->prep.size() < n) pl->prep.resize(n);
  pl->prep_ptr.resize(n);
  for (uint32_t t = 0; t < n; t++) {
    const int rc = tb_prepare(ctx, tbs[t], &pl->prep[t]);
    if (rc) return rc;
    pl->prep_ptr[t] = &pl->prep[t];
  }
  return plan_assemble(ctx, tbs, pl->prep_ptr.data(), n, pl, stream, llr_base, nullptr,
                       batch_cbs);
}

int plan_assemble(crnt_ctx* ctx, const crnt_tb_params* tbs, const TbPrep* const* preps,
                  uint32_t n, crnt_plan* pl, cudaStream_t stream, const int64_t* llr_base,
                  const int64_t* out_base, uint32_t batch_cbs) {
  pl->ctx = ctx;
  pl->tbs.assign(tbs, tbs + n);
  pl->segs.resize(n);
  pl->p_used.resize(n);
  pl->tdesc.resize(n);
  pl->base.resize(n);
  pl->keyed.clear();
  pl->owner.clear();
  pl->items.clear();
  int64_t llr_off = 0, out_off = 0, dbg_off = 0;
  uint64_t steps = 0, info_bits = 0;
  uint32_t ncb = 0;
  bool pusch_any = false;
  for (uint32_t t = 0; t < n; t++) {
    const crnt_tb_params& tp = tbs[t];
    const TbPrep& pp = *preps[t];
    const lte::Seg& s = pp.s;
    pl->segs[t] = s;
    pl->p_used[t] = pp.p_used;
    TbBase& b = pl->base[t];
    b.llr = llr_base ? llr_base[t] : llr_off;
    b.dbg = dbg_off;
    b.cb0 = ncb;
    pusch_any |= (tp.flags & CRNT_F_PUSCH) != 0;
    TbDesc& td = pl->tdesc[t];
    td.out_off = out_base ? out_base[t] : out_off;
    td.A = (int)tp.A;
    td.C = s.C;
    td.cb0 = (int)ncb;
    td.pad0 = 0;
    for (int r = 0; r < s.C; r++) {
      const CbDesc& c = pp.cb[r];
      const uint64_t cost = (uint64_t)(c.W * c.max_iter);  // < 2^17
      // descending W max_iter, then K, then P; ascending filler count F
      // (CBs of one (K, P, F) are adjacent, so CB pairs share their
      // de-rate-matching map), then (t, r) -- one integer sorted ascending:
      // cost 17 bits, K 13, P 8, F / 8 3, CB index 22
      pl->keyed.push_back(((0x1FFFFull - cost) << 46) | ((uint64_t)(0x1FFF - c.K) << 33) |
                          ((uint64_t)(0xFF - c.P) << 25) | ((uint64_t)(c.F >> 3) << 22) |
                          (uint64_t)(ncb + r));
      pl->owner.push_back(t);
      dbg_off += c.K + 4;
      steps += c.K;
    }
    ncb += s.C;
    if (ncb >= (1u << 22)) return CRNT_EINVAL;
    llr_off += tp.G;
    out_off += tp.A / 8;
    info_bits += tp.A;
  }
  std::sort(pl->keyed.begin(), pl->keyed.end());
  // With TBs in received PUSCH order the front stage writes every TB's
  // e-sequence into the plan's scratch, concatenated in TB order, and the
  // decoder reads it there.
  pl->pusch = pusch_any;
  pl->n_pch = 0;
  if (pusch_any) {
    pl->ptb.resize(n);
    pl->pch.clear();
    int64_t e = 0;
    for (uint32_t t = 0; t < n; t++) {
      pusch_tb(tbs[t], pl->base[t].llr, e, &pl->ptb[t]);
      pusch_tiles(pl->ptb[t], (int)t, pl->pch);
      pl->base[t].llr = e;
      e += tbs[t].G;
    }
    pl->n_pch = (int)pl->pch.size();
    if (!pl->d_rx.ensure((size_t)e + 16)) return CRNT_ENOMEM;
  }

  // ---- one device buffer: descriptors | zeroed per-launch state | results
  // | work items.  The state (queue head, error word, TB accumulators) and
  // the results are contiguous, so one copy brings both back.
  const size_t b_cbs = sizeof(CbDesc) * ncb, b_tbs = sizeof(TbDesc) * n;
  const size_t off_tbs = al256(b_cbs), off_zero = off_tbs + al256(b_tbs);
  const size_t s_state = 256, s_crc = al256(8 * n), s_sat = al256(4 * n);
  pl->zero_off = off_zero;
  pl->scratch_zero = s_state + s_crc + s_sat;
  const size_t off_res = off_zero + pl->scratch_zero;
  pl->res_bytes = (3 * (size_t)ncb + n + 15) & ~size_t(15);
  const size_t off_items = off_res + pl->res_bytes;
  const size_t off_ptb = al256(off_items + sizeof(WorkItem) * ncb);
  const size_t off_pch = off_ptb + (pusch_any ? al256(sizeof(PuschTb) * n) : 0);
  const size_t max_desc = off_pch + (pusch_any ? sizeof(PuschChunk) * pl->pch.size() : 0);
  // The previous upload from h_desc must have completed before the staging
  // buffer is rewritten, and no launch may still read the device buffers if
  // they are about to grow.  Waiting on the upload's event (not the whole
  // stream) lets LLR copies already queued on the stream keep running.
  if (!pl->desc_ev &&
      cudaEventCreateWithFlags(&pl->desc_ev, cudaEventDisableTiming) != cudaSuccess)
    return CRNT_EDEVICE;
  if (pl->upload_pending && cudaEventSynchronize(pl->desc_ev) != cudaSuccess)
    return CRNT_EDEVICE;
  pl->upload_pending = false;
  if (max_desc > pl->d_desc.n && cudaStreamSynchronize(stream) != cudaSuccess)
    return CRNT_EDEVICE;
  if (!pl->d_desc.ensure(max_desc) || !pl->h_desc.ensure(max_desc) ||
      !pl->h_res.ensure(pl->scratch_zero + pl->res_bytes))
    return CRNT_ENOMEM;
  uint8_t* h = (uint8_t*)pl->h_desc.p;
  CbDesc* hc = (CbDesc*)h;
  WorkItem* hi = (WorkItem*)(h + off_items);
  pl->cb_tb.resize(ncb);
  pl->cb_r.resize(ncb);

  // ---- pass 2: descriptors in sorted order
  bool radix4_any = false, qtab_all = true;
  for (uint32_t i = 0; i < ncb; i++) {
    const uint32_t g = (uint32_t)(pl->keyed[i] & 0x3FFFFF);
    const uint32_t t = pl->owner[g];
    const TbBase& b = pl->base[t];
    const int r = (int)(g - b.cb0);
    CbDesc& d = hc[i];
    d = preps[t]->cb[r];
    d.tb = (int)t;
    d.llr_off += b.llr;
    d.dbg_off = (int32_t)(d.dbg_off + b.dbg);
    radix4_any |= d.radix4 != 0;
    qtab_all &= d.qt != nullptr;
    pl->cb_tb[i] = (int)t;
    pl->cb_r[i] = r;
  }

  // ---- pass 3: work items of equal (K, P).  A CB size whose shape-table
  // entry is 2 forms CB pairs (two CBs on the same threads in 16-bit lanes,
  // one pair slot) when every CB of the batch has its address tables (the
  // pair kernel reads them) and the CB uses the radix-2 recursion; an odd
  // CB left over runs alone.  Otherwise as many CBs as the CTA's threads
  // and shared memory allow.
  // Pairs shorten a batch that fills at least two waves of CTAs in either
  // shape; a smaller batch (one subframe, a few TBs) finishes sooner with
  // one CB per thread (more CTAs in flight, one CB each), so it runs that
  // way -- the shape never changes a decoded value.  A chunk of a larger
  // call counts that call's CBs (batch_cbs): its kernels overlap the other
  // chunks', so throughput, not the chunk's own latency, decides.
  const int pair_min_cbs =
      ctx->cfg.pair_min_cbs ? (int)ctx->cfg.pair_min_cbs : 2 * kCtasPerSm * ctx->num_sms;
  const bool allow_pairs =
      qtab_all && (int64_t)std::max<uint32_t>(ncb, batch_cbs) >= (int64_t)pair_min_cbs;
  int max_item_bytes = 0;
  bool pair_any = false;
  WorkItem wi{0, 0, 0, 0};
  int gmax = 0, iK = -1, iP = -1, islot = 0;
  auto close_item = [&]() {
    if (wi.mode == 1 && wi.n == 1) {
      wi.mode = 0;
      wi.smem_per_cb = islot;
    }
    pair_any |= wi.mode == 1;
    max_item_bytes = std::max(max_item_bytes, wi.mode == 1 ? wi.smem_per_cb : wi.n * wi.smem_per_cb);
    hi[pl->items.size()] = wi;
    pl->items.push_back(wi);
  };
  for (uint32_t i = 0; i < ncb; i++) {
    const CbDesc& d = hc[i];
    if (wi.n == 0 || wi.n >= gmax || d.K != iK || d.P != iP) {
      if (wi.n) close_item();
      iK = d.K;
      iP = d.P;
      islot = align16(dec_cb_smem(d.K, d.P, d.W));
      const int pslot = dec_pair_smem(d.K, d.P, d.W);
      wi.cb0 = (int)i;
      wi.n = 0;
      if (allow_pairs && shape_of(d.K) == 2 && !d.radix4 && d.qt && pslot <= kSmemBudgetPair) {
        wi.mode = 1;
        wi.smem_per_cb = pslot;
        gmax = 2;
      } else {
        wi.mode = 0;
        wi.smem_per_cb = islot;
        gmax = std::max(1, std::min(kThreads / d.P, kSmemBudget / islot));
      }
    }
    wi.n++;
  }
  if (wi.n) close_item();
  pl->n_cb = ncb;
  pl->smem = kSmemFixed + max_item_bytes;
  if (pl->timing && (!pl->d_time.ensure(32 * (size_t)ncb) || !pl->h_time.ensure(32 * (size_t)ncb)))
    return CRNT_ENOMEM;
  static std::mutex occ_mu;
  static std::map<int, int> occ_cache;  // (dynamic smem, kernel flags) -> resident CTAs per SM
  int per_sm;
  {
    const int key = pl->smem * 8 + (radix4_any ? 1 : 0) + (qtab_all ? 2 : 0) + (pair_any ? 4 : 0);
    std::lock_guard<std::mutex> lk(occ_mu);
    auto it = occ_cache.find(key);
    if (it == occ_cache.end())
      it = occ_cache.emplace(key, decode_occupancy(pl->smem, radix4_any, qtab_all, pair_any)).first;
    per_sm = it->second;
  }
  if (per_sm < 1) return CRNT_EDEVICE;
  const int grid = std::min<int>((int)pl->items.size(), per_sm * ctx->num_sms);

  crnt_plan_info& inf = pl->info;
  inf.n_tb = n;
  inf.n_cb = ncb;
  inf.llr_bytes = (uint64_t)llr_off;
  inf.out_bytes = (uint64_t)out_off;
  inf.info_bits = info_bits;
  inf.trellis_steps = steps;
  inf.dbg_elems = (uint64_t)dbg_off;
  inf.n_items = (uint32_t)pl->items.size();
  inf.grid = (uint32_t)grid;
  inf.pair_items = 0;
  for (const WorkItem& w : pl->items) inf.pair_items += w.mode == 1 ? 1u : 0u;
  inf.smem_bytes = (uint32_t)pl->smem;

  // ---- upload: descriptors, TB table, zeroed state and work items in one
  // copy (asynchronous on `stream`)
  memcpy(h + off_tbs, pl->tdesc.data(), b_tbs);
  memset(h + off_zero, 0, pl->scratch_zero);
  pl->desc_bytes = off_items + sizeof(WorkItem) * pl->items.size();
  if (pusch_any) {
    memcpy(h + off_ptb, pl->ptb.data(), sizeof(PuschTb) * n);
    memcpy(h + off_pch, pl->pch.data(), sizeof(PuschChunk) * pl->pch.size());
    pl->desc_bytes = max_desc;
  }
  pl->off_ptb = off_ptb;
  pl->off_pch = off_pch;
  if (cudaMemcpyAsync(pl->d_desc.p, h, pl->desc_bytes, cudaMemcpyHostToDevice, stream) !=
          cudaSuccess ||
      cudaEventRecord(pl->desc_ev, stream) != cudaSuccess)
    return CRNT_EDEVICE;
  pl->upload_pending = true;
  pl->state_fresh = true;
  uint8_t* dd = (uint8_t*)pl->d_desc.p;
  DecParams& p = pl->prm;
  memset(&p, 0, sizeof p);
  p.cbs = (const CbDesc*)dd;
  p.tbs = (const TbDesc*)(dd + off_tbs);
  p.items = (const WorkItem*)(dd + off_items);
  p.n_items = (int)pl->items.size();
  p.n_cbs = (int)ncb;
  p.n_tbs = (int)n;
  p.state = (DecState*)(dd + off_zero);
  p.tb_crc = (uint32_t*)(dd + off_zero + s_state);
  p.tb_sat = (uint32_t*)(dd + off_zero + s_state + s_crc);
  p.cb_iters = dd + off_res;
  p.cb_runs = p.cb_iters + 2 * (size_t)ncb;
  p.cb_ok = p.cb_iters + ncb;
  p.tb_ok = p.cb_iters + 3 * (size_t)ncb;  // cb_iters | cb_ok | cb_runs | tb_ok
  p.xpowA = ctx->xpowA;
  p.xpowB = ctx->xpowB;
  p.mi_tab = ctx->mi_tab;
  p.radix4_any = radix4_any ? 1 : 0;
  p.qtab_all = qtab_all && ncb > 0 ? 1 : 0;
  p.pair_any = pair_any ? 1 : 0;
  return CRNT_OK;
}

bool plan_reserve(crnt_plan* pl, uint32_t max_tbs, uint32_t max_cbs) {
  const size_t zero = 256 + al256(8 * (size_t)max_tbs) + al256(4 * (size_t)max_tbs);
  const size_t res = (3 * (size_t)max_cbs + max_tbs + 15) & ~size_t(15);
  const size_t desc = al256(sizeof(CbDesc) * max_cbs) + al256(sizeof(TbDesc) * max_tbs) + zero +
                      res + sizeof(WorkItem) * max_cbs;
  return pl->d_desc.ensure(desc) && pl->h_desc.ensure(desc) && pl->h_res.ensure(zero + res);
}

int plan_launch(crnt_plan* pl, const int8_t* llr, uint8_t* out, cudaStream_t s, int8_t* dbg_d,
                int16_t* dbg_ext, uint8_t* dbg_hard, bool state_uploaded, const uint32_t* gate,
                uint32_t gate_us) {
  if (gate && pl->pusch) return CRNT_EINVAL;
  DecParams p = pl->prm;
  p.gate = gate;
  p.gate_us = gate_us;
  p.llr = llr;
  p.out = out;
  p.soft = pl->ctx->harq.arena;
  p.dbg_d = dbg_d;
  p.dbg_ext = dbg_ext;
  p.dbg_hard = dbg_hard;
  p.cb_time = pl->timing ? (uint64_t*)pl->d_time.p : nullptr;
  // the queue head and the TB accumulators start at zero: the upload of
  // plan_build wrote zeros, a later launch of the same plan clears them
  if (!(state_uploaded && pl->state_fresh) &&
      cudaMemsetAsync((uint8_t*)pl->d_desc.p + pl->zero_off, 0, pl->scratch_zero, s) !=
          cudaSuccess)
    return CRNT_EDEVICE;
  pl->state_fresh = false;
  if (pl->pusch) {
    // front stage: received order -> e-sequence in the plan's scratch
    const uint8_t* dd = (const uint8_t*)pl->d_desc.p;
    if (!pl->ctx->gold ||
        launch_pusch(false, (const PuschTb*)(dd + pl->off_ptb), (const PuschChunk*)(dd + pl->off_pch),
                     pl->n_pch, gold_tables_view(pl->ctx->gold), llr, (int8_t*)pl->d_rx.p,
                     s) != cudaSuccess)
      return CRNT_EDEVICE;
    p.llr = (const int8_t*)pl->d_rx.p;
  }
  if (launch_decode(p, (int)pl->info.grid, pl->smem, s) != cudaSuccess) return CRNT_EDEVICE;
  return CRNT_OK;
}

int plan_fetch_results(crnt_plan* pl, cudaStream_t s) {
  if (cudaMemcpyAsync(pl->h_res.p, (uint8_t*)pl->d_desc.p + pl->zero_off,
                      pl->scratch_zero + pl->res_bytes, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return CRNT_EDEVICE;
  return CRNT_OK;
}

void plan_fill_results(const crnt_plan* pl, crnt_tb_result* res) {
  const size_t ncb = pl->n_cb;
  const uint32_t n = pl->info.n_tb;
  const int32_t err = ((const DecState*)pl->h_res.p)->err;  // a bounded device wait expired
  const uint8_t* h = (const uint8_t*)pl->h_res.p + pl->scratch_zero;
  // per-TB saturating-pass counts: the last part of the zeroed scratch; the
  // TB CRC words (TB CRC24A accumulated over its CBs, failed-CB flag) before
  const uint32_t* sat = (const uint32_t*)(h - ((4 * (size_t)n + 255) & ~size_t(255)));
  const uint32_t* crc = (const uint32_t*)((const uint8_t*)pl->h_res.p + 256);
  for (uint32_t t = 0; t < n; t++) {
    crnt_tb_result& r = res[t];
    memset(&r, 0, sizeof r);
    const lte::Seg& sg = pl->segs[t];
    r.status = err ? CRNT_ETIMEDOUT : CRNT_OK;
    r.C = (uint8_t)sg.C;
    r.K_plus = (uint16_t)sg.Kp;
    r.K_minus = (uint16_t)sg.Km;
    r.F = (uint16_t)sg.F;
    r.P_used = pl->p_used[t];
    r.sat_passes = (uint16_t)std::min<uint32_t>(sat[t], 65535u);
    r.tb_crc_ok = sg.C == 1 ? h[3 * ncb + t] : (crc[2 * t] == 0u && crc[2 * t + 1] == 0u);
  }
  for (size_t i = 0; i < ncb; i++) {
    crnt_tb_result& r = res[pl->cb_tb[i]];
    r.cb_iters[pl->cb_r[i]] = h[i];
    r.cb_crc_ok[pl->cb_r[i]] = h[ncb + i];
    r.cb_iters_run[pl->cb_r[i]] = h[2 * ncb + i];
  }
}

}  // namespace crnt

// ------------------------------------------------------------------ C ABI
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

int crnt_interleaver_map(uint32_t K, uint32_t P, uint32_t* map, uint32_t n) {
  const int ki = lte::index_of((int)K);
  if (!map || ki < 0) return CRNT_EINVAL;
  const int Pr = clamp_p((int)K, (int)P), W = ((int)K + Pr - 1) / Pr;
  const int Pe = ((int)K + W - 1) / W, ng = (W + kSub - 1) / kSub;
  if (n < (uint32_t)(W * Pe)) return CRNT_EINVAL;
  std::vector<uint32_t> ht((size_t)ng * Pe * kSub, 0u);
  std::vector<uint16_t> hq(ht.size(), 0);
  build_qt(ht.data(), hq.data(), ki, (int)K, Pe);
  for (int p = 0; p < Pe; p++)
    for (int j = 0; j < W; j++) {
      const size_t e = ((size_t)(j / kSub) * Pe + p) * kSub + j % kSub;
      map[(size_t)p * W + j] = ((uint32_t)hq[e] << 16) | ht[e];
    }
  return CRNT_OK;
}

int crnt_derm_map(uint32_t K, uint32_t P, uint32_t F, uint32_t rv, uint32_t* map, uint32_t n) {
  if (!map || lte::index_of((int)K) < 0 || rv > 3 || (F & 7) || F >= 64 || F >= K)
    return CRNT_EINVAL;
  const int Pr = clamp_p((int)K, (int)P), W = ((int)K + Pr - 1) / Pr;
  const int Pe = ((int)K + W - 1) / W;
  const int Nv = 3 * ((int)K + 4) - 2 * (int)F;
  if (n < (uint32_t)Nv) return CRNT_EINVAL;
  std::vector<uint32_t> h((size_t)Nv);
  if (build_dm(h.data(), nullptr, Nv, (int)K, Pe, (int)F) != Nv) return CRNT_EINVAL;
  uint32_t mb = 0, m2 = 0;
  rm_masks(32 * lte::rows((int)K) - ((int)K + 4), (int)F, &mb, &m2);
  const int rank0 = rank_of_k0((int)K, (int)F, (int)rv, mb, m2);
  for (int k = 0; k < Nv; k++) map[k] = h[(size_t)((k + rank0) % Nv)];
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
  // mutual-information stop rule: T(x) = round(2^16 log2(1 + exp(-x/8)))
  int32_t mi[kMiTable];
  for (int x = 0; x < kMiTable; x++)
    mi[x] = (int32_t)std::floor(65536.0 * std::log2(1.0 + std::exp(-(double)x / 8.0)) + 0.5);
  if (cudaMalloc(&c->xpowA, 4 * kXpowA) != cudaSuccess ||
      cudaMalloc(&c->xpowB, 4 * kXpowB) != cudaSuccess ||
      cudaMalloc(&c->mi_tab, sizeof mi) != cudaSuccess ||
      cudaMemcpy(c->xpowA, xa.data(), 4 * kXpowA, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->xpowB, xb.data(), 4 * kXpowB, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->mi_tab, mi, sizeof mi, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    crnt_destroy(c);
    return CRNT_EDEVICE;
  }
  // jump-ahead tables of the PUSCH scrambling sequence (37 KB)
  {
    const std::vector<uint32_t> g = gold_tables_host();
    if (cudaMalloc(&c->gold, 4 * g.size()) != cudaSuccess ||
        cudaMemcpy(c->gold, g.data(), 4 * g.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      crnt_destroy(c);
      return CRNT_EDEVICE;
    }
  }
  // the per-(K, P) tables (interleaved-pass addresses, de-rate-matching
  // maps) of the window counts P = 0 requests get, now (others on first
  // use); without them the decoder computes addresses and walks the buffer
  c->qtabs = new (std::nothrow) QTabs;
  if (c->qtabs &&
      cudaStreamCreateWithFlags(&c->qtabs->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c->qtabs;
    c->qtabs = nullptr;
  }
  if (c->qtabs) {
    for (int i = 0; i < lte::kNumK; i++) {
      const int K = lte::k_of(i), Pr = clamp_p(K, 0), W = (K + Pr - 1) / Pr;
      qtab_get(c, K, (K + W - 1) / W);
    }
  }
  *out = c;
  return CRNT_OK;
}

int crnt_destroy(crnt_ctx* ctx) {
  if (!ctx) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  serving_stop(ctx);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (int c = 0; c < crnt_ctx::kBatchChunks; c++) {
    if (ctx->chunk_stream[c]) {
      cudaStreamSynchronize(ctx->chunk_stream[c]);
      cudaStreamDestroy(ctx->chunk_stream[c]);
    }
    if (ctx->chunk_ev[c]) cudaEventDestroy(ctx->chunk_ev[c]);
    delete ctx->cached[c];
    ctx->cached[c] = nullptr;
  }
  ctx->stage_in.release();
  ctx->stage_out.release();
  if (ctx->xpowA) cudaFree(ctx->xpowA);
  if (ctx->xpowB) cudaFree(ctx->xpowB);
  if (ctx->mi_tab) cudaFree(ctx->mi_tab);
  if (ctx->gold) cudaFree(ctx->gold);
  if (ctx->qtabs) {
    for (void* p : ctx->qtabs->chunks) cudaFree(p);
    if (ctx->qtabs->stream) cudaStreamDestroy(ctx->qtabs->stream);
    delete ctx->qtabs;
    ctx->qtabs = nullptr;
  }
  if (ctx->harq.arena) cudaFree(ctx->harq.arena);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return CRNT_OK;
}

int crnt_harq_release(crnt_ctx* ctx, uint32_t cell, uint32_t ue, uint32_t harq_pid) {
  if (!ctx) return CRNT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->harq_mu);
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
  cudaSetDevice(ctx->device);
  int rc = plan_build(ctx, tbs, n, pl.get(), ctx->stream);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = CRNT_EDEVICE;
  if (rc) return rc;
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
  return plan_launch(plan, llr, out, (cudaStream_t)stream, dbg_d, dbg_ext, dbg_hard);
}

int crnt_plan_launch(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream) {
  return crnt_plan_launch_debug(plan, llr, out, stream, nullptr, nullptr, nullptr);
}

int crnt_plan_launch_gated(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream,
                           const uint32_t* ready, uint32_t timeout_us) {
  if (!plan || !llr || !out || !ready || timeout_us < 1 || timeout_us > 10000000u)
    return CRNT_EINVAL;
  return plan_launch(plan, llr, out, (cudaStream_t)stream, nullptr, nullptr, nullptr, false,
                     ready, timeout_us);
}

int crnt_plan_results(crnt_plan* plan, crnt_tb_result* res, void* stream) {
  if (!plan || !res) return CRNT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (plan_fetch_results(plan, s) != CRNT_OK || cudaStreamSynchronize(s) != cudaSuccess)
    return CRNT_EDEVICE;
  plan_fill_results(plan, res);
  return CRNT_OK;
}

int crnt_plan_set_timing(crnt_plan* plan, int enable) {
  if (!plan) return CRNT_EINVAL;
  cudaSetDevice(plan->ctx->device);
  if (enable && (!plan->d_time.ensure(32 * (size_t)plan->n_cb + 32) ||
                 !plan->h_time.ensure(32 * (size_t)plan->n_cb + 32)))
    return CRNT_ENOMEM;
  plan->timing = enable != 0;
  return CRNT_OK;
}

int crnt_plan_timing(crnt_plan* plan, crnt_cb_timing* out, uint32_t n, void* stream) {
  if (!plan || !out || !plan->timing || n < plan->n_cb) return CRNT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ncb = plan->n_cb;
  if (plan_fetch_results(plan, s) != CRNT_OK ||
      cudaMemcpyAsync(plan->h_time.p, plan->d_time.p, 32 * ncb, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CRNT_EDEVICE;
  const uint64_t* t = (const uint64_t*)plan->h_time.p;
  const uint8_t* runs = (const uint8_t*)plan->h_res.p + plan->scratch_zero + 2 * ncb;
  for (size_t i = 0; i < ncb; i++) {
    const int tb = plan->cb_tb[i], r = plan->cb_r[i];
    crnt_cb_timing& o = out[plan->tdesc[tb].cb0 + r];
    memset(&o, 0, sizeof o);
    o.tb = (uint32_t)tb;
    o.r = (uint32_t)r;
    o.t_start_ns = t[4 * i];
    o.t_derm_ns = t[4 * i + 1];
    o.t_iter_ns = t[4 * i + 2];
    o.t_done_ns = t[4 * i + 3];
    o.iterations = runs[i];
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
  // device buffers are used in place; host LLRs are copied into the arena
  // (page-locked ones by DMA at the link's rate, which beat the kernels
  // reading them in place over the link); page-locked output is written in
  // place, pageable output staged
  const bool llr_host = host_memory(llr);
  const int8_t* llr_view = llr_host ? nullptr : (const int8_t*)device_view(llr);
  uint8_t* out_view = (uint8_t*)device_view(out);
  const bool llr_dev = llr_view != nullptr, out_dev = out_view != nullptr;
  std::lock_guard<std::mutex> lk(ctx->stage_mu);
  constexpr int NC = crnt_ctx::kBatchChunks;
  // Chunks of about 5 %, 30 % and 65 % of the TBs (one chunk for small
  // batches): the device starts on the small first chunk while the host
  // plans the next ones and their LLRs are still in flight.  Chunk c runs on
  // its own stream, so a later chunk's CTAs fill the SMs as an earlier
  // chunk's drain.  (Measured on a 320-TB TTI from page-locked buffers:
  // 0.620 ms per call, against 0.632 for 3/22/75 %, 0.648 for 15/40/45 %,
  // 0.654 for 5/45/50 %.)
  uint32_t bnd[NC + 1] = {0, n, n, n};
  // the call's CBs: C = 1 for B = A + 24 <= 6144, else ceil(B / 6120) (TS
  // 36.212 5.1.2); invalid TBs are refused by the planner
  uint32_t total_cbs = 0;
  for (uint32_t t = 0; t < n; t++) {
    const uint32_t B = tbs[t].A + 24u;
    total_cbs += B <= 6144u ? 1u : (B + 6119u) / 6120u;
  }
  int nch = 1;
  if (n >= 24) {
    nch = 3;
    bnd[1] = (5 * n) / 100;
    bnd[2] = (35 * n) / 100;
  }
  for (int c = 0; c < nch; c++) {
    if (!ctx->cached[c]) {
      ctx->cached[c] = new (std::nothrow) crnt_plan;
      if (!ctx->cached[c]) return CRNT_ENOMEM;
    }
    if (!ctx->chunk_stream[c] &&
        cudaStreamCreateWithFlags(&ctx->chunk_stream[c], cudaStreamNonBlocking) != cudaSuccess)
      return CRNT_EDEVICE;
    if (!ctx->chunk_ev[c] &&
        cudaEventCreateWithFlags(&ctx->chunk_ev[c], cudaEventDisableTiming) != cudaSuccess)
      return CRNT_EDEVICE;
  }
  // byte offsets of each chunk's LLRs and decoded bits
  int64_t llr_at[NC + 1] = {0, 0, 0, 0}, out_at[NC + 1] = {0, 0, 0, 0};
  {
    int64_t lb = 0, ob = 0;
    int c = 0;
    for (uint32_t t = 0; t <= n; t++) {
      while (c <= nch && bnd[c] == t) {
        llr_at[c] = lb;
        out_at[c] = ob;
        c++;
      }
      if (t < n) {
        lb += tbs[t].G;
        ob += tbs[t].A / 8;
      }
    }
  }
  // every previous call has completed (this call is synchronous), so the
  // staging buffers can grow without waiting
  const int8_t* d_llr = llr_view;
  if (!llr_dev) {
    if (!ctx->stage_in.ensure((size_t)llr_at[nch])) return CRNT_ENOMEM;
    d_llr = (const int8_t*)ctx->stage_in.p;
  }
  uint8_t* d_out = out_view;
  if (!out_dev) {
    if (!ctx->stage_out.ensure((size_t)out_at[nch] + 16)) return CRNT_ENOMEM;
    d_out = (uint8_t*)ctx->stage_out.p;
  }
  // Host-to-device copies share one copy engine in issue order, so chunk c's
  // LLRs are issued just before its planning (which they overlap) and ahead
  // of its descriptor upload, not all at once ahead of every upload.
  auto copy_llrs = [&](int c) {
    const size_t bytes = (size_t)(llr_at[c + 1] - llr_at[c]);
    if (llr_dev || bytes == 0) return true;
    return cudaMemcpyAsync((int8_t*)ctx->stage_in.p + llr_at[c], llr + llr_at[c], bytes,
                           cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess &&
           cudaEventRecord(ctx->chunk_ev[c], ctx->stream) == cudaSuccess;
  };
  int rc = CRNT_OK;
  int launched = 0;
  for (int c = 0; c < nch && rc == CRNT_OK; c++) {
    const uint32_t t0 = bnd[c], m = bnd[c + 1] - bnd[c];
    if (m == 0) continue;
    cudaStream_t s = ctx->chunk_stream[c];
    crnt_plan* plan = ctx->cached[c];
    if (!copy_llrs(c)) {
      rc = CRNT_EDEVICE;
      break;
    }
    rc = plan_build(ctx, tbs + t0, m, plan, s, nullptr, total_cbs);
    if (rc) break;
    if (!llr_dev && llr_at[c + 1] > llr_at[c] &&
        cudaStreamWaitEvent(s, ctx->chunk_ev[c], 0) != cudaSuccess) {
      rc = CRNT_EDEVICE;
      break;
    }
    rc = plan_launch(plan, d_llr + llr_at[c], d_out + out_at[c], s, nullptr, nullptr, nullptr,
                     true);
    if (rc) break;
    launched = c + 1;
    const size_t ob = (size_t)(out_at[c + 1] - out_at[c]);
    if ((!out_dev && ob &&
         cudaMemcpyAsync(out + out_at[c], d_out + out_at[c], ob, cudaMemcpyDeviceToHost, s) !=
             cudaSuccess) ||
        plan_fetch_results(plan, s) != CRNT_OK)
      rc = CRNT_EDEVICE;
  }
  // wait for everything issued, also on failure, before returning
  bool dev_ok = cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  for (int c = 0; c < nch; c++)
    dev_ok = (cudaStreamSynchronize(ctx->chunk_stream[c]) == cudaSuccess) && dev_ok;
  if (rc) return rc;
  if (!dev_ok) return CRNT_EDEVICE;
  for (int c = 0; c < nch; c++) ctx->cached[c]->upload_pending = false;  // streams drained
  for (int c = 0; c < launched; c++)
    if (bnd[c + 1] > bnd[c]) plan_fill_results(ctx->cached[c], res + bnd[c]);
  return CRNT_OK;
}

int crnt_decode_tb(crnt_ctx* ctx, const int8_t* llr, const crnt_tb_params* tb, uint8_t* out,
                   crnt_tb_result* res) {
  return crnt_decode_batch(ctx, tb, 1, llr, out, res);
}

int crnt_encode_batch(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, const uint8_t* bits,
                      uint8_t* e_out) {
  if (!ctx || !tbs || !bits || !e_out || n == 0) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->stage_mu);
  // pass 1: validate, count CBs and bytes
  std::vector<lte::Seg>& segs = ctx->enc_segs;
  segs.resize(n);
  size_t ncb = 0;
  int64_t ioff = 0, eoff = 0;
  bool pusch_any = false;
  for (uint32_t t = 0; t < n; t++) {
    int rc = validate(tbs[t], &segs[t]);
    if (rc) return rc;
    ncb += (size_t)segs[t].C;
    ioff += tbs[t].A / 8;
    eoff += tbs[t].G;
    pusch_any |= (tbs[t].flags & CRNT_F_PUSCH) != 0;
  }
  // the transmit stage's descriptors and tiles
  std::vector<PuschTb>& eq = ctx->enc_ptb;
  std::vector<PuschChunk>& ech = ctx->enc_pch;
  eq.resize(pusch_any ? n : 0);
  ech.clear();
  if (pusch_any) {
    int64_t e = 0;
    for (uint32_t t = 0; t < n; t++) {
      pusch_tb(tbs[t], e, e, &eq[t]);
      pusch_tiles(eq[t], (int)t, ech);
      e += tbs[t].G;
    }
  }
  const size_t nch = ech.size();
  // device or page-locked buffers are used in place; pageable ones staged
  const uint8_t* bits_view = (const uint8_t*)device_view(bits);
  uint8_t* out_view = (uint8_t*)device_view(e_out);
  const size_t b_cbs = sizeof(EncCb) * ncb, b_off = 8 * (size_t)n, b_A = 4 * (size_t)n;
  const size_t o_off = al256(b_cbs), o_A = o_off + al256(b_off);
  // with TBs in PUSCH order: the transmit stage's descriptors, and the coded
  // bits first go to the e-sequence scratch enc_e
  const size_t o_ptb = o_A + al256(b_A);
  const size_t o_pch = o_ptb + (pusch_any ? al256(sizeof(PuschTb) * n) : 0);
  const size_t o_bits = o_pch + (pusch_any ? al256(sizeof(PuschChunk) * nch) : 0);
  const size_t total = o_bits + (bits_view ? 0 : (size_t)ioff);
  if (!ctx->stage_in.ensure(total) || !ctx->enc_host.ensure(o_bits)) return CRNT_ENOMEM;
  if (!out_view && !ctx->stage_out.ensure((size_t)eoff)) return CRNT_ENOMEM;
  if (pusch_any && (!ctx->gold || !ctx->enc_e.ensure((size_t)eoff + 16))) return CRNT_ENOMEM;
  // pass 2: descriptors straight into page-locked staging
  uint8_t* h = (uint8_t*)ctx->enc_host.p;
  EncCb* hc = (EncCb*)h;
  int64_t* h_off = (int64_t*)(h + o_off);
  int32_t* h_A = (int32_t*)(h + o_A);
  size_t k = 0;
  ioff = 0;
  eoff = 0;
  for (uint32_t t = 0; t < n; t++) {
    const lte::Seg& s = segs[t];
    h_off[t] = ioff;
    h_A[t] = (int32_t)tbs[t].A;
    int pay_off = 0;
    for (int r = 0; r < s.C; r++) {
      EncCb& c = hc[k++];
      memset(&c, 0, sizeof c);
      const int K = lte::cb_k(s, r);
      c.K = K;
      c.F = r == 0 ? s.F : 0;
      c.E = lte::e_r((int)tbs[t].G, tbs[t].Qm, tbs[t].NL, s.C, r);
      c.R = lte::rows(K);
      c.ND = 32 * c.R - (K + 4);
      uint32_t mb, m2;
      rm_masks(c.ND, c.F, &mb, &m2);
      c.rank0 = rank_of_k0(K, c.F, tbs[t].rv, mb, m2);
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
    }
    ioff += tbs[t].A / 8;
  }
  if (pusch_any) {
    memcpy(h + o_ptb, eq.data(), sizeof(PuschTb) * n);
    memcpy(h + o_pch, ech.data(), sizeof(PuschChunk) * nch);
  }
  cudaStream_t st = ctx->stream;
  uint8_t* base = (uint8_t*)ctx->stage_in.p;
  if (cudaMemcpyAsync(base, h, o_bits, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CRNT_EDEVICE;
  if (!bits_view &&
      cudaMemcpyAsync(base + o_bits, bits, (size_t)ioff, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CRNT_EDEVICE;
  EncParams p;
  p.cbs = (const EncCb*)base;
  p.tb_in_off = (const int64_t*)(base + o_off);
  p.tb_A = (const int32_t*)(base + o_A);
  p.tb_bits = bits_view ? bits_view : base + o_bits;
  uint8_t* final_out = out_view ? out_view : (uint8_t*)ctx->stage_out.p;
  p.e_out = pusch_any ? (uint8_t*)ctx->enc_e.p : final_out;
  p.xpowA = ctx->xpowA;
  p.xpowB = ctx->xpowB;
  if (launch_encode(p, (int)ncb, st) != cudaSuccess) return CRNT_EDEVICE;
  if (pusch_any &&
      launch_pusch(true, (const PuschTb*)(base + o_ptb), (const PuschChunk*)(base + o_pch),
                   (int)nch, gold_tables_view(ctx->gold), (const int8_t*)ctx->enc_e.p,
                   (int8_t*)final_out, st) != cudaSuccess)
    return CRNT_EDEVICE;
  if (!out_view &&
      cudaMemcpyAsync(e_out, final_out, (size_t)eoff, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CRNT_EDEVICE;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRNT_EDEVICE;
  return CRNT_OK;
}

int crnt_encode_tb(crnt_ctx* ctx, const uint8_t* bits, const crnt_tb_params* tb, uint8_t* e_out) {
  return crnt_encode_batch(ctx, tb, 1, bits, e_out);
}

}  // extern "C"
