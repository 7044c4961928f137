// runtime.h -- host runtime objects shared by the C ABI (crnt_api.cu) and
// the serving loop (serve.cu): the context, reusable batch plans, and the
// HARQ soft-buffer pool.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/crnt.h"
#include "crnt_internal.h"
#include "lte_params.h"

namespace crnt {

// Grow-only device or pinned host buffer.
struct Buf {
  void* p = nullptr;
  size_t n = 0;
  bool host = false;
  Buf() = default;
  explicit Buf(bool pinned_host) : host(pinned_host) {}
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) host ? cudaFreeHost(p) : cudaFree(p);
    p = nullptr;
    n = 0;
  }
  bool ensure(size_t bytes) {
    if (bytes <= n) return true;
    release();
    const size_t want = bytes + bytes / 4 + 4096;
    cudaError_t e = host ? cudaMallocHost(&p, want) : cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    n = want;
    return true;
  }
};

struct HarqPool {
  int8_t* arena = nullptr;
  uint32_t slots = 0;
  std::map<std::tuple<uint32_t, uint32_t, uint32_t>, uint32_t> keys;
  std::vector<uint32_t> free_list;
};

struct Serving;

// Tables of one (K, P) on the context's device: the interleaved SISO pass's
// addresses (CbDesc::qt, qq) and the de-rate-matching maps of the eight
// filler counts (CbDesc::dm); built on the host and uploaded on first use,
// kept until the context is destroyed.
struct QTabs {
  std::mutex mu;  // guards building (readers use the atomics)
  std::atomic<const uint4*> t[lte::kNumK][CRNT_MAX_P + 1];
  std::vector<void*> chunks;  // device allocations
  uint8_t* cur = nullptr;     // free space in the last chunk
  size_t left = 0;
  cudaStream_t stream = nullptr;
  QTabs() {
    for (auto& row : t)
      for (auto& x : row) x.store(nullptr, std::memory_order_relaxed);
  }
};

// Fields of a CB descriptor fixed by (K, requested P) alone.
struct KTmpl {
  int32_t K, W, P, divM, divS, f1, f2, f2x2, f2sub, f2jump, R, ND, ncb, slot;
  uint32_t maskB0, mask2;  // column masks with no filler bits
  int32_t rank0[4];        // rank of k0 per rv with no filler bits
};

}  // namespace crnt

struct crnt_ctx {
  int device = 0;
  crnt_config cfg{};
  int num_sms = 0;
  uint32_t* xpowA = nullptr;
  uint32_t* xpowB = nullptr;
  int32_t* mi_tab = nullptr;  // [kMiTable] table of the mutual-information stop rule
  uint32_t* gold = nullptr;   // [kGoldWords] jump-ahead tables of the PUSCH scrambling sequence
  crnt::QTabs* qtabs = nullptr;  // interleaved-pass address tables
  crnt::HarqPool harq;
  std::mutex harq_mu;     // guards harq
  std::mutex stage_mu;    // guards the staging buffers and the cached plan
  crnt::Buf stage_in, stage_out;
  crnt::Buf enc_host{true};             // page-locked encoder descriptor staging
  crnt::Buf enc_e;                       // encoder's e-sequence ahead of the PUSCH transmit stage
  std::vector<crnt::PuschTb> enc_ptb;    // its per-TB descriptors
  std::vector<crnt::PuschChunk> enc_pch; // and tiles
  std::vector<crnt::lte::Seg> enc_segs;  // encoder planning scratch
  // crnt_decode_batch splits a batch into up to kBatchChunks chunks, each
  // with a reused plan and its own stream, so that planning and copying a
  // chunk overlap the decoding of the chunks before it
  static constexpr int kBatchChunks = 3;
  crnt_plan* cached[kBatchChunks] = {};
  cudaStream_t chunk_stream[kBatchChunks] = {};
  cudaEvent_t chunk_ev[kBatchChunks] = {};  // LLR copy of chunk c done
  cudaStream_t stream = nullptr;
  crnt::Serving* serving = nullptr;
  std::mutex serving_mu;
};

// Per-TB planning record (pass 1 of plan_build).
struct TbPre {
  int64_t llr, soft, dbg;   // TB's first LLR byte, soft-buffer base (-1), debug base
  uint32_t cb0;             // global index of its first CB (TB order)
  int n_lo, E_lo, E_hi;     // the first n_lo CBs get E_lo rate-matched bits, the rest E_hi
  crnt::KTmpl tm, tp;       // descriptor templates of K- and K+
};

// One TB prepared for any batch (tb_prepare): its segmentation, soft-buffer
// binding and templates, and its CB descriptors in r order with the LLR and
// debug offsets counted from the TB's own first LLR byte and debug element.
struct TbPrep {
  crnt::lte::Seg s;
  TbPre pr;
  uint16_t p_used;
  crnt::CbDesc cb[CRNT_MAX_CB];
};

// Where a batch put one TB.
struct TbBase {
  int64_t llr, dbg;  // its first LLR byte (from the launch's LLR pointer), debug base
  uint32_t cb0;      // index of its first CB in TB order
};

// A planned batch.  Its buffers are grow-only, so re-planning a plan object
// (plan_build) allocates nothing once it has seen a batch as large.
struct crnt_plan {
  crnt_ctx* ctx = nullptr;
  std::vector<crnt_tb_params> tbs;
  std::vector<TbBase> base;
  std::vector<TbPrep> prep;             // plan_build's prepared TBs
  std::vector<const TbPrep*> prep_ptr;
  std::vector<uint64_t> keyed;       // sort keys (low bits: CB index in TB order)
  std::vector<uint32_t> owner;       // CB index in TB order -> TB
  std::vector<int> cb_tb, cb_r;      // sorted index -> (tb, r)
  std::vector<crnt::TbDesc> tdesc;
  std::vector<crnt::WorkItem> items;
  std::vector<crnt::lte::Seg> segs;
  std::vector<uint16_t> p_used;
  uint32_t n_cb = 0;
  crnt_plan_info info{};
  int smem = 0;
  crnt::Buf d_desc;                  // device: descriptors, zeroed state, results, items
  crnt::Buf h_desc{true}, h_res{true};  // pinned: descriptor staging | state + results
  cudaEvent_t desc_ev = nullptr;     // recorded after the last descriptor upload
  bool upload_pending = false;       // desc_ev may not have completed yet
  bool state_fresh = false;          // the zeroed state was just uploaded
  ~crnt_plan() {
    if (desc_ev) cudaEventDestroy(desc_ev);
  }
  size_t desc_bytes = 0, zero_off = 0, scratch_zero = 0, res_bytes = 0;
  crnt::DecParams prm{};
  // PUSCH front stage (TBs with CRNT_F_PUSCH): per-TB and per-chunk
  // descriptors (also in d_desc at off_ptb / off_pch) and the e-sequence
  // scratch the decoder then reads
  bool pusch = false;
  std::vector<crnt::PuschTb> ptb;
  std::vector<crnt::PuschChunk> pch;
  int n_pch = 0;
  size_t off_ptb = 0, off_pch = 0;
  crnt::Buf d_rx;
  // performance captor (crnt_plan_set_timing): 4 timestamps per sorted CB
  bool timing = false;
  crnt::Buf d_time, h_time{true};
};

namespace crnt {
// Host planning + descriptor upload on `stream` (asynchronous when the plan's
// buffers are already large enough; allocates otherwise).  llr_base (may be
// null): byte offset of each TB's LLRs from the LLR pointer given at launch;
// null means the TBs' LLRs are concatenated in order.
// batch_cbs: CBs of the whole call this batch belongs to, when larger than
// the batch itself (it decides whether CB pairs are formed); 0 = the batch's.
int plan_build(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, crnt_plan* pl,
               cudaStream_t stream, const int64_t* llr_base = nullptr, uint32_t batch_cbs = 0);
// The two halves of plan_build: tb_prepare validates one TB, binds its soft
// buffer (CRNT_F_HARQ; last, so a TB refused binds none) and writes its CB
// descriptors; plan_assemble plans a batch of prepared TBs.  out_base (may
// be null): byte offset of each TB's output from the output pointer given at
// launch; null means concatenated in order.
int tb_prepare(crnt_ctx* ctx, const crnt_tb_params& tp, TbPrep* out);
int plan_assemble(crnt_ctx* ctx, const crnt_tb_params* tbs, const TbPrep* const* preps,
                  uint32_t n, crnt_plan* pl, cudaStream_t stream, const int64_t* llr_base,
                  const int64_t* out_base, uint32_t batch_cbs = 0);
// Size a plan's buffers for batches of up to max_tbs TBs and max_cbs CBs, so
// that planning such batches later allocates nothing.
bool plan_reserve(crnt_plan* pl, uint32_t max_tbs, uint32_t max_cbs);
// state_uploaded: the caller launches right after plan_build, whose upload
// already zeroed the per-launch state (skips one memset).
// gate, gate_us: see crnt_plan_launch_gated (null: no wait).
int plan_launch(crnt_plan* pl, const int8_t* llr, uint8_t* out, cudaStream_t s, int8_t* dbg_d,
                int16_t* dbg_ext, uint8_t* dbg_hard, bool state_uploaded = false,
                const uint32_t* gate = nullptr, uint32_t gate_us = 0);
// Enqueue the D2H copy of the per-CB / per-TB results into h_res.
int plan_fetch_results(crnt_plan* pl, cudaStream_t s);
// Fill res[n] from h_res (after the stream has passed plan_fetch_results).
void plan_fill_results(const crnt_plan* pl, crnt_tb_result* res);
int validate(const crnt_tb_params& t, lte::Seg* seg);
// Window count of the process-wide table for CB size K (0 = built-in).
int tuned_p(int K);
// The interleaved-pass address table of CB size K split into P windows of
// W = ceil(K / P) steps (P as used: ceil(K / W) == P); its natural-position
// part follows at qtab_q.  Null when it cannot be built (no device memory):
// the decoder then computes the addresses.
const uint4* qtab_get(crnt_ctx* ctx, int K, int P);
inline const uint2* qtab_q(const uint4* t, int K, int P) {
  const int W = (K + P - 1) / P;
  return t ? (const uint2*)(t + (size_t)((W + kSub - 1) / kSub + 2) * P) : nullptr;
}
// The de-rate-matching map of (K, P, F) (CbDesc::dm), null if it cannot be built.
const uint32_t* dmap_get(crnt_ctx* ctx, int K, int P, int F);
// 1 if the radix table selects the radix-4 forward recursion for CB size K.
// t_radix_override >= 0 replaces the table for plans built on this thread
// (the autotuner's candidates).
uint8_t radix4_of(int K);
extern thread_local int t_radix_override;
// CTA shape for CB size K from the shape table (1 one CB per thread, 2 CB
// pairs); t_shape_override > 0 replaces it for plans built on this thread.
uint8_t shape_of(int K);
extern thread_local int t_shape_override;
// Window count used for CB size K when a TB requests P (0 = table / built-in).
int clamp_p(int K, int P);
void serving_stop(crnt_ctx* ctx);
// The jump-ahead tables of the PUSCH scrambling sequence (kGoldWords words,
// layout of GoldTables), built on the host.
std::vector<uint32_t> gold_tables_host();
// Interleaver columns of a TB with CRNT_F_PUSCH (n_symb, 0 = 12).
inline int pusch_cols(const crnt_tb_params& t) { return t.n_symb ? t.n_symb : 12; }
// Front-stage descriptor of a TB (mode 0, a plain copy, without CRNT_F_PUSCH)
// and its tiles appended to out.
void pusch_tb(const crnt_tb_params& tp, int64_t in_off, int64_t out_off, PuschTb* q);
void pusch_tiles(const PuschTb& q, int tb, std::vector<PuschChunk>& out);
int64_t now_ns();
}  // namespace crnt
