// tune.cu -- the window-count autotuner and the process-wide table it fills.
//
// For each of the 188 CB sizes K the tuner decodes full batches of
// single-CB TBs (A = K - 24, rate 1/3, 6 iterations, no early stop) with a
// few candidate window counts P and keeps the fastest whose windows are at
// least w_min trellis steps long.  The decode work does not depend on the
// LLR values on the clamp-free path, so the inputs are zeros.  Candidates:
// minimum window lengths w in {w_lo, 32, 40, 48, 56, 64, 80, 96} (w_lo: the
// shortest allowed, which also uses the most threads), each giving
// P = floor(K / w) windows of ceil(K / P) >= w steps, timed in both CTA
// shapes -- one CB per thread, and CB pairs in 16-bit lanes -- and, for CB
// pairs only, P = ceil(K / w) windows of at most w steps, which for these w
// (multiples of 8) fill the pair path's 8-step sub-windows.  Each candidate
// counts with its faster shape; the kept window count takes its faster
// shape.  At that count the tuner also times the radix-4 forward recursion
// (one CB per thread), selecting it when it is more than 1 % faster than
// both.  Shape and radix never change a decoded value, only the speed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace crnt {
extern std::atomic<uint8_t> g_tuned[lte::kNumK];
extern std::atomic<uint8_t> g_radix[lte::kNumK];
extern std::atomic<uint8_t> g_shape[lte::kNumK];

namespace {

// Decode time (ms, mean of 3 launches after one warm-up) of n single-CB TBs
// of size K with window request P.
int time_batch(crnt_ctx* ctx, crnt_plan* plan, int K, int P, int n, int8_t* d_llr,
               uint8_t* d_out, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  crnt_tb_params t;
  memset(&t, 0, sizeof t);
  t.A = (uint32_t)(K - 24);
  t.G = (uint32_t)(3 * K + 12);
  t.Qm = 2;
  t.NL = 1;
  t.P = (uint16_t)P;
  t.max_iter = 6;
  t.early_stop = 0;
  t.new_data = 1;
  std::vector<crnt_tb_params> tbs((size_t)n, t);
  int rc = plan_build(ctx, tbs.data(), (uint32_t)n, plan, ctx->stream);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  if (plan_launch(plan, d_llr, d_out, s, nullptr, nullptr, nullptr, true) != CRNT_OK)
    return CRNT_EDEVICE;
  if (cudaEventRecord(e0, s) != cudaSuccess) return CRNT_EDEVICE;
  for (int r = 0; r < 3; r++)
    if (plan_launch(plan, d_llr, d_out, s, nullptr, nullptr, nullptr) != CRNT_OK)
      return CRNT_EDEVICE;
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
    return CRNT_EDEVICE;
  *ms /= 3.0f;
  return cudaStreamSynchronize(s) == cudaSuccess ? CRNT_OK : CRNT_EDEVICE;
}

}  // namespace
}  // namespace crnt

using namespace crnt;

extern "C" {

int crnt_tune_get(uint8_t* P_by_k, uint32_t n) {
  if (!P_by_k) return CRNT_EINVAL;
  for (uint32_t i = 0; i < n && i < (uint32_t)lte::kNumK; i++)
    P_by_k[i] = g_tuned[i].load(std::memory_order_relaxed);
  return CRNT_OK;
}

int crnt_tune_set(const uint8_t* P_by_k, uint32_t n) {
  if (!P_by_k || n != (uint32_t)lte::kNumK) return CRNT_EINVAL;
  for (int i = 0; i < lte::kNumK; i++) {
    if (P_by_k[i] > CRNT_MAX_P) return CRNT_EINVAL;
  }
  for (int i = 0; i < lte::kNumK; i++) g_tuned[i].store(P_by_k[i], std::memory_order_relaxed);
  return CRNT_OK;
}

int crnt_tune_radix_get(uint8_t* radix_by_k, uint32_t n) {
  if (!radix_by_k) return CRNT_EINVAL;
  for (uint32_t i = 0; i < n && i < (uint32_t)lte::kNumK; i++) {
    const uint8_t r = g_radix[i].load(std::memory_order_relaxed);
    radix_by_k[i] = r == 4 ? 4 : 2;
  }
  return CRNT_OK;
}

int crnt_tune_radix_set(const uint8_t* radix_by_k, uint32_t n) {
  if (!radix_by_k || n != (uint32_t)lte::kNumK) return CRNT_EINVAL;
  for (int i = 0; i < lte::kNumK; i++) {
    const uint8_t r = radix_by_k[i];
    if (r != 0 && r != 2 && r != 4) return CRNT_EINVAL;
  }
  for (int i = 0; i < lte::kNumK; i++)
    g_radix[i].store(radix_by_k[i] == 4 ? 4 : 2, std::memory_order_relaxed);
  return CRNT_OK;
}

int crnt_tune_shape_get(uint8_t* shape_by_k, uint32_t n) {
  if (!shape_by_k) return CRNT_EINVAL;
  for (uint32_t i = 0; i < n && i < (uint32_t)lte::kNumK; i++)
    shape_by_k[i] = g_shape[i].load(std::memory_order_relaxed) == 2 ? 2 : 1;
  return CRNT_OK;
}

int crnt_tune_shape_set(const uint8_t* shape_by_k, uint32_t n) {
  if (!shape_by_k || n != (uint32_t)lte::kNumK) return CRNT_EINVAL;
  for (int i = 0; i < lte::kNumK; i++) {
    const uint8_t v = shape_by_k[i];
    if (v > 2) return CRNT_EINVAL;
  }
  for (int i = 0; i < lte::kNumK; i++)
    g_shape[i].store(shape_by_k[i] == 2 ? 2 : 1, std::memory_order_relaxed);
  return CRNT_OK;
}

int crnt_autotune(crnt_ctx* ctx, uint32_t w_min, uint8_t* P_by_k) {
  if (!ctx) return CRNT_EINVAL;
  if (w_min == 0) w_min = 32;
  if (w_min > (uint32_t)lte::kZ) return CRNT_EINVAL;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> lk(ctx->stage_mu);
  // candidates per K, and per candidate a batch of two CBs per resident
  // thread slot (two waves of CTAs), at most 64 MiB of LLRs
  struct Cand {
    int K, P, n;
    bool one;                  // timed with one CB per thread as well as in pairs
    float rate, rate1, rate2;  // best, one CB per thread, CB pairs (0: not timed)
  };
  std::vector<std::vector<Cand>> cands(lte::kNumK);
  const size_t slots = (size_t)kCtasPerSm * ctx->num_sms;
  size_t max_llr = 0, max_out = 0;
  for (int i = 0; i < lte::kNumK; i++) {
    const int K = lte::k_of(i);
    const int pmax = std::max(1, std::min(K / 8, (int)CRNT_MAX_P));
    const int w_lo = std::max((int)w_min, (K + pmax - 1) / pmax);
    // one CB per thread: P = floor(K / w), windows of >= w steps; CB pairs
    // also P = ceil(K / w) for w a multiple of the pair path's checkpoint
    // interval, windows of <= w steps that fill whole sub-windows (ragged
    // sub-windows cost the pair path more than it saves)
    const int ws[] = {w_lo, 32, 40, 48, 56, 64, 80, 96};
    for (int k = 0; k < 2 * 8; k++) {
      const int w = ws[k % 8];
      const bool one = k < 8;
      if (w < w_lo) continue;
      const int P = one ? clamp_p(K, std::max(1, K / w)) : clamp_p(K, (K + w - 1) / w);
      const int W = (K + P - 1) / P;
      if (!one && W < (int)w_min) continue;
      bool dup = false;
      for (Cand& c : cands[i])
        if (c.P == P) {
          dup = true;
          c.one |= one;
        }
      if (dup) continue;
      const int slot = align16(dec_cb_smem(K, (K + W - 1) / W, W));
      const int g = std::max(1, std::min(kThreads / P, kSmemBudget / slot));
      // two waves in either shape (a pair CTA holds two CBs)
      size_t n = 2 * std::max(slots * (size_t)g, (size_t)(kCtasPerSmPair * 2 * ctx->num_sms));
      n = std::min(n, (size_t)(64u << 20) / (size_t)(3 * K + 12));
      cands[i].push_back(Cand{K, P, (int)n, one, 0.0f, 0.0f, 0.0f});
      max_llr = std::max(max_llr, n * (size_t)(3 * K + 12));
      max_out = std::max(max_out, n * (size_t)((K - 24) / 8) + 16);
    }
  }
  int8_t* d_llr = nullptr;
  uint8_t* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CRNT_OK;
  if (cudaMalloc(&d_llr, max_llr) != cudaSuccess || cudaMalloc(&d_out, max_out) != cudaSuccess ||
      cudaMemset(d_llr, 0, max_llr) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = CRNT_ENOMEM;
  uint8_t table[lte::kNumK], radix[lte::kNumK], shape[lte::kNumK];
  memset(table, 0, sizeof table);
  memset(radix, 2, sizeof radix);
  memset(shape, 1, sizeof shape);
  {
    crnt_plan plan;  // re-planned per candidate; its buffers only grow
    for (int i = 0; i < lte::kNumK && rc == CRNT_OK; i++) {
      float best = 0.0f;
      t_radix_override = 0;
      for (Cand& c : cands[i]) {
        for (int sh = 1; sh <= 2 && rc == CRNT_OK; sh++) {
          const int W = (c.K + c.P - 1) / c.P;
          if (sh == 1 && !c.one) continue;
          if (sh == 2 && dec_pair_smem(c.K, (c.K + W - 1) / W, W) > kSmemBudgetPair) continue;
          t_shape_override = sh;
          float ms = 0.0f;
          rc = time_batch(ctx, &plan, c.K, c.P, c.n, d_llr, d_out, e0, e1, &ms);
          (sh == 1 ? c.rate1 : c.rate2) = (float)c.n * (float)c.K / ms;
        }
        if (rc) break;
        c.rate = std::max(c.rate1, c.rate2);
        best = std::max(best, c.rate);
      }
      t_shape_override = -1;
      if (rc) break;
      // the longest windows among the candidates within 1 % of the fastest
      const Cand* pick = nullptr;
      for (const Cand& c : cands[i])
        if (c.rate >= 0.99f * best && (!pick || c.P < pick->P)) pick = &c;
      table[i] = (uint8_t)pick->P;
      if (pick->rate2 > pick->rate1) shape[i] = 2;
      // the radix-4 forward recursion (one CB per thread) at that window count
      float ms4 = 0.0f;
      t_radix_override = 1;
      t_shape_override = 1;
      rc = time_batch(ctx, &plan, pick->K, pick->P, pick->n, d_llr, d_out, e0, e1, &ms4);
      t_shape_override = -1;
      if (rc) break;
      if ((float)pick->n * (float)pick->K / ms4 > 1.01f * pick->rate) {
        radix[i] = 4;
        shape[i] = 1;
      }
    }
    t_radix_override = -1;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_llr) cudaFree(d_llr);
  if (d_out) cudaFree(d_out);
  if (rc) return rc;
  for (int i = 0; i < lte::kNumK; i++) {
    g_tuned[i].store(table[i], std::memory_order_relaxed);
    g_radix[i].store(radix[i], std::memory_order_relaxed);
    g_shape[i].store(shape[i], std::memory_order_relaxed);
  }
  if (P_by_k) memcpy(P_by_k, table, sizeof table);
  return CRNT_OK;
}

}  // extern "C"
