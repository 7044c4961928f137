// noalloc.cu -- crnt_decode_batch_static: the batched decode for callers that
// cannot allocate device memory (for example code running under a memory
// pool they do not own, or an allocator that is forbidden at that point).
//
// Everything the decode kernel needs besides the caller's inputs and outputs
// -- the code-block descriptors, the work queue, the CRC shift tables, the
// mutual-information table of stop rule 2 and the per-launch scratch (queue
// head, per-TB counters and CRC accumulators, per-CB results) -- lives in one
// file-scope __device__ array of fixed size.
// The host side plans into fixed static arrays of the same capacity.  Nothing
// is allocated on the device or in pinned host memory; the kernel is the same
// fused decode kernel the other entry points launch.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the parts that must start at zero are cleared by each call.
// Calls that overlap on the GPU (on different streams, or from several host
// threads) race on the array; the host side serialises concurrent calls with
// a mutex, but the caller must not let two calls' GPU work overlap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "runtime.h"

namespace crnt {
namespace {

constexpr int kStaticTbs = 64;
constexpr int kStaticCbs = kStaticTbs * 13;
constexpr int kXA = 2400, kXB = 200;
constexpr int kMaxDevices = 64;

// Layout of the device workspace (byte offsets, each 256-aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCbs = 0;
constexpr size_t kOffTbs = kOffCbs + al(sizeof(CbDesc) * kStaticCbs);
constexpr size_t kOffItems = kOffTbs + al(sizeof(TbDesc) * kStaticTbs);
constexpr size_t kOffXA = kOffItems + al(sizeof(WorkItem) * kStaticCbs);
constexpr size_t kOffXB = kOffXA + al(4 * kXA);
constexpr size_t kOffState = kOffXB + al(4 * kXB);
constexpr size_t kOffCrc = kOffState + 256;
constexpr size_t kOffSat = kOffCrc + al(8 * kStaticTbs);  // per-TB saturating-pass counts
constexpr size_t kZeroBytes = kOffSat + al(4 * kStaticTbs) - kOffState;
constexpr size_t kOffRes = kOffSat + al(4 * kStaticTbs);  // cb_iters | cb_ok | cb_runs | tb_ok
constexpr size_t kResBytes = 3 * kStaticCbs + kStaticTbs;
constexpr size_t kOffMi = al(kOffRes + kResBytes);        // mutual-information table
constexpr size_t kStaticBytes = kOffMi + al(4 * kMiTable);
static_assert(kStaticBytes <= 512 * 1024, "static decode workspace stays within 512 KiB");

// The workspace.  Host code must not take its address directly: the name is
// a host-side stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_workspace[kStaticBytes];

std::mutex g_mu;                       // serialises host-side use
void* g_dev_ptr[kMaxDevices] = {};     // workspace address per device
int g_num_sms[kMaxDevices] = {};

// host-side planning storage (static: nothing is allocated per call)
CbDesc h_all[kStaticCbs];
int h_all_tb[kStaticCbs], h_all_r[kStaticCbs], h_order[kStaticCbs];
CbDesc h_cbs[kStaticCbs];
int h_cb_tb[kStaticCbs], h_cb_r[kStaticCbs];
TbDesc h_tbs[kStaticTbs];
WorkItem h_items[kStaticCbs];
lte::Seg h_segs[kStaticTbs];
uint16_t h_pused[kStaticTbs];
uint8_t h_back[kOffRes - kOffCrc + kResBytes];  // TB CRC words | counts | results

int clamp_windows(int K, int P) {
  if (P <= 0) P = tuned_p(K);  // the process-wide table (a read, no allocation)
  if (P <= 0) P = (K + 47) / 48;
  P = std::min(P, K / 8);
  P = std::min(P, (int)CRNT_MAX_P);
  return std::max(P, 1);
}

uint32_t gf_mul24(uint32_t a, uint32_t b, uint32_t g) {
  uint32_t r = 0;
  for (int i = 23; i >= 0; i--) {
    r <<= 1;
    if (r & 0x1000000u) r ^= g;
    if ((a >> i) & 1u) r ^= b;
  }
  return r;
}

void xpow_fill(uint32_t g, int n, uint32_t* t) {
  uint32_t x32 = 1;
  for (int i = 0; i < 32; i++) {
    x32 <<= 1;
    if (x32 & 0x1000000u) x32 ^= g;
  }
  uint32_t cur = 1;
  for (int s = 0; s < n; s++) {
    t[s] = cur;
    cur = gf_mul24(cur, x32, g);
  }
}

// q / W == (q * M) >> s for 0 <= q < qmax, searched and verified; small
// direct-mapped cache in static storage.
bool divider(int W, int qmax, int* M, int* s) {
  struct E {
    int W, qmax, M, s;
  };
  static E cache[256];
  E& e = cache[(unsigned)(W * 131 + qmax) & 255u];
  if (e.W == W && e.qmax == qmax) {
    *M = e.M;
    *s = e.s;
    return true;
  }
  for (int sh = 0; sh < 32; sh++) {
    const uint64_t m = ((1ull << sh) + W - 1) / W;
    if (m * (uint64_t)qmax >= (1ull << 32)) break;
    bool ok = true;
    for (int q = 0; q < qmax && ok; q++) ok = (int)((q * m) >> sh) == q / W;
    if (ok) {
      e = E{W, qmax, (int)m, sh};
      *M = (int)m;
      *s = sh;
      return true;
    }
  }
  return false;
}

void masks(int ND, int F, uint32_t* mb, uint32_t* m2) {
  const int X = ND + F;
  *mb = 0;
  *m2 = 0;
  for (int c = 0; c < 32; c++) {
    const int pc = lte::bitrev5(c);
    if (pc < (X & 31)) *mb |= 1u << c;
    if (pc < ND - 1) *m2 |= 1u << c;
  }
}

int k0_rank(int K, int F, int rv, uint32_t mb, uint32_t m2) {
  const int R = lte::rows(K), ND = 32 * R - (K + 4), X = ND + F, xa = X >> 5;
  const int k0 = lte::k0(K, rv);
  auto pre0 = [&](int c) { return xa * c + __builtin_popcount(mb & ((1u << c) - 1u)); };
  if (k0 < 32 * R) {
    const int c = k0 / R;
    return c * R - pre0(c);
  }
  const int c = (k0 - 32 * R) / (2 * R);
  return (32 * R - X) + 2 * R * c - pre0(c) - __builtin_popcount(m2 & ((1u << c) - 1u));
}

// One-time set-up on the current device: workspace address, CRC and
// mutual-information tables.
int setup(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return CRNT_EDEVICE;
  if (g_dev_ptr[dev]) return CRNT_OK;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_workspace) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return CRNT_EDEVICE;
  }
  static uint32_t xa[kXA], xb[kXB];
  static int32_t mi[kMiTable];
  xpow_fill(0x1864CFBu, kXA, xa);
  xpow_fill(0x1800063u, kXB, xb);
  // stop rule 2: T(x) = round(2^16 log2(1 + exp(-x/8))), as crnt_create builds it
  for (int x = 0; x < kMiTable; x++)
    mi[x] = (int32_t)std::floor(65536.0 * std::log2(1.0 + std::exp(-(double)x / 8.0)) + 0.5);
  if (cudaMemcpy((uint8_t*)ptr + kOffXA, xa, sizeof xa, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((uint8_t*)ptr + kOffXB, xb, sizeof xb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy((uint8_t*)ptr + kOffMi, mi, sizeof mi, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CRNT_EDEVICE;
  g_dev_ptr[dev] = ptr;
  return CRNT_OK;
}

// The address under which the kernel can use a caller buffer: device and
// managed memory as is, page-locked host memory through its mapped device
// address; nullptr for anything else (pageable host memory cannot be read by
// the kernel, and this entry point has no staging buffer to copy it into).
// cudaPointerGetAttributes allocates nothing.
void* kernel_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return (void*)p;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  return nullptr;
}

}  // namespace
}  // namespace crnt

using namespace crnt;

extern "C" int crnt_decode_batch_static(const crnt_tb_params* tbs, uint32_t n, const int8_t* llr,
                                        uint8_t* out, crnt_tb_result* res, void* stream) {
  if (!tbs || !llr || !out || !res || n == 0) return CRNT_EINVAL;
  if (n > (uint32_t)kStaticTbs) return CRNT_ENOMEM;
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CRNT_EDEVICE;
  int rc = setup(dev);
  if (rc) return rc;
  uint8_t* ws = (uint8_t*)g_dev_ptr[dev];
  cudaStream_t s = (cudaStream_t)stream;
  const int8_t* llr_k = (const int8_t*)kernel_view(llr);
  uint8_t* out_k = (uint8_t*)kernel_view(out);
  if (!llr_k || !out_k) return CRNT_EINVAL;  // pageable or unknown memory

  // ---- host planning into static storage
  int ncb = 0;
  int64_t llr_off = 0, out_off = 0;
  for (uint32_t t = 0; t < n; t++) {
    const crnt_tb_params& tp = tbs[t];
    lte::Seg& sg = h_segs[t];
    rc = validate(tp, &sg);
    if (rc) return rc;
    if (tp.flags & CRNT_F_HARQ) return CRNT_EINVAL;   // no soft-buffer arena here
    if (tp.flags & CRNT_F_PUSCH) return CRNT_EINVAL;  // no front-stage scratch here
    if (ncb + sg.C > kStaticCbs) return CRNT_ENOMEM;
    TbDesc& td = h_tbs[t];
    memset(&td, 0, sizeof td);
    td.out_off = out_off;
    td.A = (int)tp.A;
    td.C = sg.C;
    td.cb0 = ncb;
    const int B = (int)tp.A + 24;
    int pay_off = 0, eoff = 0;
    for (int r = 0; r < sg.C; r++) {
      CbDesc& d = h_all[ncb];
      memset(&d, 0, sizeof d);
      const int K = lte::cb_k(sg, r);
      const int F = r == 0 ? sg.F : 0;
      const int Pr = clamp_windows(K, tp.P);
      const int W = (K + Pr - 1) / Pr;
      d.K = K;
      d.F = F;
      d.E = lte::e_r((int)tp.G, tp.Qm, tp.NL, sg.C, r);
      d.k0 = lte::k0(K, tp.rv);
      d.W = W;
      d.P = (K + W - 1) / W;  // the windows actually run (ceil(K / W) <= Pr)
      if (K == sg.Kp) h_pused[t] = (uint16_t)d.P;
      if (!divider(W, K + 4, &d.divM, &d.divS)) return CRNT_EINVAL;
      const int ki = lte::index_of(K);
      d.f1 = lte::kF1[ki];
      d.f2 = lte::kF2[ki];
      d.f2x2 = (int)((2ll * d.f2) % K);
      d.f2sub = (int)((2ll * kSub * d.f2) % K);
      d.f2jump = (int)((2ll * kSub * kSub * d.f2) % K);
      d.R = lte::rows(K);
      d.ND = 32 * d.R - (K + 4);
      d.Nv = 3 * (K + 4) - 2 * F;
      if (((d.ND + F) >> 5) + 1 > d.R) return CRNT_EINVAL;
      masks(d.ND, F, &d.maskB, &d.mask2);
      d.rank0 = k0_rank(K, F, tp.rv, d.maskB, d.mask2);
      d.tb = (int)t;
      d.r = r;
      d.llr_off = llr_off + eoff;
      d.soft_off = -1;
      d.pay_bits = K - F - sg.L;
      d.pay_off = pay_off;
      d.n_after = B - pay_off - d.pay_bits;
      d.crc_b = sg.C > 1;
      d.max_iter = tp.max_iter;
      d.early_stop = tp.early_stop;  // 0 none, 1 CRC, 2 mutual information
      d.new_data = 1;
      d.purge = (tp.flags & CRNT_F_PURGE) && sg.C > 1 ? 1 : 0;
      d.radix4 = radix4_of(K);  // the process-wide radix table (a read)
      h_all_tb[ncb] = (int)t;
      h_all_r[ncb] = r;
      pay_off += d.pay_bits;
      eoff += d.E;
      ncb++;
    }
    if (eoff != (int)tp.G || pay_off != B) return CRNT_EINVAL;
    llr_off += tp.G;
    out_off += tp.A / 8;
  }
  // work items: CBs of equal (K, P) share a CTA, longest work first; ties
  // keep TB order (index as the last key: std::sort allocates nothing)
  for (int i = 0; i < ncb; i++) h_order[i] = i;
  std::sort(h_order, h_order + ncb, [](int x, int y) {
    const CbDesc &a = h_all[x], &b = h_all[y];
    const int ca = a.W * a.max_iter, cb = b.W * b.max_iter;
    if (ca != cb) return ca > cb;
    if (a.K != b.K) return a.K > b.K;
    if (a.P != b.P) return a.P > b.P;
    return x < y;
  });
  int nitems = 0, max_slot = 0, k = 0;
  for (int i = 0; i < ncb;) {
    const CbDesc& h = h_all[h_order[i]];
    const int slot = align16(dec_cb_smem(h.K, h.P, h.W));
    if (slot > kSmemBudget) return CRNT_EINVAL;
    const int gmax = std::max(1, std::min(kThreads / h.P, kSmemBudget / slot));
    WorkItem& wi = h_items[nitems++];
    wi.cb0 = k;
    wi.n = 0;
    wi.smem_per_cb = slot;
    wi.mode = 0;
    while (i < ncb && wi.n < gmax) {
      const CbDesc& c = h_all[h_order[i]];
      if (c.K != h.K || c.P != h.P) break;
      h_cbs[k] = c;
      h_cb_tb[k] = h_all_tb[h_order[i]];
      h_cb_r[k] = h_all_r[h_order[i]];
      k++;
      wi.n++;
      i++;
    }
    max_slot = std::max(max_slot, wi.n * slot);
  }
  const int smem = kSmemFixed + max_slot;
  bool radix4_any = false;
  for (int i = 0; i < ncb; i++) radix4_any |= h_cbs[i].radix4 != 0;
  const int per_sm = decode_occupancy(smem, radix4_any, false, false);
  if (per_sm < 1) return CRNT_EDEVICE;
  const int grid = std::min(nitems, per_sm * g_num_sms[dev]);

  // ---- descriptors in, scratch cleared, launch, results out
  DecParams p;
  memset(&p, 0, sizeof p);
  p.cbs = (const CbDesc*)(ws + kOffCbs);
  p.tbs = (const TbDesc*)(ws + kOffTbs);
  p.items = (const WorkItem*)(ws + kOffItems);
  p.n_items = nitems;
  p.n_cbs = ncb;
  p.n_tbs = (int)n;
  p.llr = llr_k;
  p.out = out_k;
  p.soft = nullptr;
  p.state = (DecState*)(ws + kOffState);
  p.tb_crc = (uint32_t*)(ws + kOffCrc);
  p.tb_sat = (uint32_t*)(ws + kOffSat);
  p.cb_iters = ws + kOffRes;  // cb_iters | cb_ok | cb_runs | tb_ok, as the plan path
  p.cb_ok = p.cb_iters + ncb;
  p.cb_runs = p.cb_iters + 2 * (size_t)ncb;
  p.tb_ok = p.cb_iters + 3 * (size_t)ncb;
  p.xpowA = (const uint32_t*)(ws + kOffXA);
  p.xpowB = (const uint32_t*)(ws + kOffXB);
  p.mi_tab = (const int32_t*)(ws + kOffMi);
  for (int i = 0; i < ncb; i++) p.radix4_any |= h_cbs[i].radix4;
  const size_t back_bytes = (kOffRes - kOffCrc) + 3 * (size_t)ncb + n;
  bool ok =
      cudaMemcpyAsync(ws + kOffCbs, h_cbs, sizeof(CbDesc) * ncb, cudaMemcpyHostToDevice, s) ==
          cudaSuccess &&
      cudaMemcpyAsync(ws + kOffTbs, h_tbs, sizeof(TbDesc) * n, cudaMemcpyHostToDevice, s) ==
          cudaSuccess &&
      cudaMemcpyAsync(ws + kOffItems, h_items, sizeof(WorkItem) * nitems, cudaMemcpyHostToDevice,
                      s) == cudaSuccess &&
      cudaMemsetAsync(ws + kOffState, 0, kZeroBytes, s) == cudaSuccess &&
      launch_decode(p, grid, smem, s) == cudaSuccess &&
      cudaMemcpyAsync(h_back, ws + kOffCrc, back_bytes, cudaMemcpyDeviceToHost, s) ==
          cudaSuccess;
  // wait for whatever was enqueued, also on failure, so that no kernel of
  // this call still uses the shared workspace when the next call clears it
  ok = (cudaStreamSynchronize(s) == cudaSuccess) && ok;
  if (!ok) {
    cudaGetLastError();
    return CRNT_EDEVICE;
  }
  const uint32_t* crc = (const uint32_t*)h_back;  // per TB: CRC24A word, failed-CB flag
  const uint32_t* sat = (const uint32_t*)(h_back + (kOffSat - kOffCrc));
  const uint8_t* h_res = h_back + (kOffRes - kOffCrc);
  for (uint32_t t = 0; t < n; t++) {
    crnt_tb_result& r = res[t];
    memset(&r, 0, sizeof r);
    r.status = CRNT_OK;
    r.C = (uint8_t)h_segs[t].C;
    r.K_plus = (uint16_t)h_segs[t].Kp;
    r.K_minus = (uint16_t)h_segs[t].Km;
    r.F = (uint16_t)h_segs[t].F;
    r.P_used = h_pused[t];
    r.sat_passes = (uint16_t)std::min<uint32_t>(sat[t], 65535u);
    r.tb_crc_ok =
        h_segs[t].C == 1 ? h_res[3 * ncb + t] : (crc[2 * t] == 0u && crc[2 * t + 1] == 0u);
  }
  for (int i = 0; i < ncb; i++) {
    crnt_tb_result& r = res[h_cb_tb[i]];
    r.cb_iters[h_cb_r[i]] = h_res[i];
    r.cb_crc_ok[h_cb_r[i]] = h_res[ncb + i];
    r.cb_iters_run[h_cb_r[i]] = h_res[2 * ncb + i];
  }
  return CRNT_OK;
}
