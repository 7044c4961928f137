// decode.cu -- fused uplink decode of a batch of LTE code blocks on sm_103a.
//
// One persistent launch decodes every CB of a batch of transport blocks:
//   de-rate-matching + HARQ combining (the "decoder-bits conditioning" the
//   paper counts in its pre-processing, Sec. V), the iterative turbo decoder
//   (Sec. IV-B "Decoding function", Fig. 4: SISO1 -> interleave -> SISO2 ->
//   de-interleave), the hard decision with a CRC stop after each iteration,
//   and TB reassembly with the TB CRC24A check (a TB is good only when all of
//   its CBs are, Sec. IV-B "Scheduler").  CTAs pull work items from a device
//   queue, the GPU counterpart of the paper's FIFO thread pool (Algorithm 2).
//
// Arithmetic (identical to the CPU oracle, written independently):
//   S = Ls + La, gamma(u,p) = [u=0] S + [p=0] Lp,
//   alpha'[s] = sat16(m[s] - m[0]) with m[s] the exact best incoming sum,
//   beta likewise, Lambda = sat16(best_u0 - best_u1), Le = sat16(Lambda - S),
//   exchanged a-priori = floor(3 Le / 4).
// Windows: W = ceil(K/P), window p = [pW, min(pW+W, K)), one thread each;
// interior boundaries start from zeros, then from the neighbour's boundary
// metrics of the previous iteration (next-iteration initialisation).
//
// Layout in shared memory (per CB slot): channel LLRs and the extrinsic are
// stored transposed, element k at (k mod W) * P + k / W, so that the P
// window threads of a warp touch consecutive addresses at every step.
// Forward metrics are checkpointed every kSub steps and recomputed, kSub
// steps at a time, into registers during the backward pass.
#include <cstdint>
#include <type_traits>

#include "crnt_internal.h"
#include "rm_geom.cuh"

namespace crnt {
namespace {

constexpr int MINF = -16384;
constexpr uint32_t GA = 0x1864CFBu;  // gCRC24A with the D^24 term
constexpr uint32_t GB = 0x1800063u;  // gCRC24B with the D^24 term

// ---------------------------------------------------------------- trellis
// State s = 4 r1 + 2 r2 + r3 of the 8-state RSC (g0 = 1+D^2+D^3 feedback,
// g1 = 1+D+D^3).  Input u: register input a = u ^ r2 ^ r3, next state
// (a, r1, r2), parity a ^ r1 ^ r3 = u ^ r1 ^ r2.
__host__ __device__ constexpr int nxt(int s, int u) {
  return (((u ^ (s >> 1) ^ s) & 1) << 2) | ((s >> 1) & 3);
}
__host__ __device__ constexpr int par(int s, int u) { return (u ^ (s >> 2) ^ (s >> 1)) & 1; }
// branch-metric code: bit1 = [u == 0] (carries S), bit0 = [p == 0] (carries Lp)
__host__ __device__ constexpr int gcode(int s, int u) {
  return ((u == 0) ? 2 : 0) | ((par(s, u) == 0) ? 1 : 0);
}

// Predecessor k (k = r3 of the old state) of state n and its branch code.
__host__ __device__ constexpr int pred(int n, int k) { return 2 * (n & 3) + k; }
__host__ __device__ constexpr int pred_u(int n, int k) { return ((n >> 2) ^ n ^ k) & 1; }
__host__ __device__ constexpr int pcode(int n, int k) { return gcode(pred(n, k), pred_u(n, k)); }

constexpr bool check_pred() {
  for (int n = 0; n < 8; n++)
    for (int k = 0; k < 2; k++)
      if (nxt(pred(n, k), pred_u(n, k)) != n) return false;
  return true;
}
static_assert(check_pred(), "trellis predecessor formula");

__device__ __forceinline__ int gval(int code, int S, int T, int Lp) {
  return code == 3 ? T : code == 2 ? S : code == 1 ? Lp : 0;
}

// State metrics are held with an offset: stored value = metric + OFF, so a
// saturated int16 metric occupies exactly [0, 65535].  Offsets cancel in
// every comparison and in Lambda.
constexpr int OFF = 32768;
constexpr int MINF_OFF = MINF + OFF;

// max(x0 + g0, x1 + g1) with the add folded into a DPX add-max when one of
// the branch metrics is zero.
__device__ __forceinline__ int acs2(int x0, int c0, int x1, int c1, int S, int T, int Lp) {
  if (c1 == 0) return __viaddmax_s32(x0, gval(c0, S, T, Lp), x1);
  if (c0 == 0) return __viaddmax_s32(x1, gval(c1, S, T, Lp), x0);
  return __viaddmax_s32(x0, gval(c0, S, T, Lp), x1 + gval(c1, S, T, Lp));
}

// Normalisation by state 0 with int16 saturation, in offset form:
// o[s] = sat16(m[s] - m[0]) + OFF.  CHK: the exact path -- one OR over the
// results detects a value outside [0, 65535] and only then are the clamps
// applied.  !CHK: the caller has proved (window_fast) that no value can
// saturate, so sat16 is the identity and normalisation only subtracts a
// per-step constant from all eight metrics.  Such a constant cancels in
// every max-plus comparison and in Lambda (a difference of two maxima over
// the same alpha and beta), so the clamp-free path skips it and carries
// unnormalised int32 metrics; they are normalised only where they are
// stored as 16-bit values (checkpoints, window seeds: pack_norm).  The
// window_fast bound implies 8 g <= 32767, the largest metric moves by at
// most g per step, so over at most 6144 steps the metrics stay within 2^25
// of their start values, far inside int32.
template <bool CHK>
__device__ __forceinline__ void normalise(const int m[8], int o[8]) {
  if (!CHK) {
#pragma unroll
    for (int s = 0; s < 8; s++) o[s] = m[s];
    return;
  }
  const int base = OFF - m[0];
  o[0] = OFF;
#pragma unroll
  for (int s = 1; s < 8; s++) o[s] = m[s] + base;
  if (CHK) {
    const unsigned any = (unsigned)(o[1] | o[2] | o[3] | o[4] | o[5] | o[6] | o[7]);
    if (any > 0xFFFFu) {
#pragma unroll
      for (int s = 1; s < 8; s++) o[s] = min(max(o[s], 0), 65535);
    }
  }
}

template <bool CHK>
__device__ __forceinline__ void alpha_step(const int a[8], int o[8], int S, int T, int Lp) {
  int m[8];
#pragma unroll
  for (int n = 0; n < 8; n++)
    m[n] = acs2(a[pred(n, 0)], pcode(n, 0), a[pred(n, 1)], pcode(n, 1), S, T, Lp);
  normalise<CHK>(m, o);
}

// Two trellis steps at once (radix-4 forward recursion): every state n at
// step k + 2 takes the best of its four two-step paths n0 -> n1 -> n, each
// weighing gamma_k(n0 -> n1) + gamma_{k+1}(n1 -> n).  Clamp-free path only:
// there the radix-2 recursion is the exact max-plus product and, since a
// maximum distributes over an added constant, max over n1 of (max over n0 of
// (a[n0] + g0) + g1) equals this maximum over the four paths as integers, so
// both radices give the same metrics (and the same checkpoints after
// pack_norm).  The sixteen two-step branch sums are the pairs of the two
// steps' four branch values {0, Lp, S, S + Lp}; the unrolled loops use them
// with compile-time indices, so only the nonzero pairs cost an add.
__device__ __forceinline__ void alpha_step_r4(const int a[8], int o[8], int S0, int L0, int S1,
                                              int L1) {
  const int g0[4] = {0, L0, S0, S0 + L0};
  const int g1[4] = {0, L1, S1, S1 + L1};
#pragma unroll
  for (int n = 0; n < 8; n++) {
    int src[4], code0[4], code1[4];
#pragma unroll
    for (int k1 = 0; k1 < 2; k1++)
#pragma unroll
      for (int k0 = 0; k0 < 2; k0++) {
        const int n1 = pred(n, k1);
        src[2 * k1 + k0] = pred(n1, k0);
        code0[2 * k1 + k0] = pcode(n1, k0);
        code1[2 * k1 + k0] = pcode(n, k1);
      }
    // start the chain from a path with a zero branch sum when there is one
    int z = -1;
#pragma unroll
    for (int i = 0; i < 4; i++)
      if (z < 0 && code0[i] == 0 && code1[i] == 0) z = i;
    const int first = z < 0 ? 0 : z;
    int acc = a[src[first]];
    if (z < 0) acc += g0[code0[first]] + g1[code1[first]];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (i == first) continue;
      const int c0 = code0[i], c1 = code1[i];
      if (c0 == 0 && c1 == 0) acc = max(acc, a[src[i]]);
      else if (c0 == 0) acc = __viaddmax_s32(a[src[i]], g1[c1], acc);
      else if (c1 == 0) acc = __viaddmax_s32(a[src[i]], g0[c0], acc);
      else acc = __viaddmax_s32(a[src[i]], g0[c0] + g1[c1], acc);
    }
    o[n] = acc;
  }
}

template <bool CHK>
__device__ __forceinline__ void beta_step(int b[8], int S, int T, int Lp) {
  int m[8];
#pragma unroll
  for (int s = 0; s < 8; s++)
    m[s] = acs2(b[nxt(s, 0)], gcode(s, 0), b[nxt(s, 1)], gcode(s, 1), S, T, Lp);
  normalise<CHK>(m, b);
}

// Terminating tail step: each state leaves on the branch that feeds a = 0.
__device__ __forceinline__ void beta_tail_step(int b[8], int Ls, int Lp) {
  int m[8];
#pragma unroll
  for (int s = 0; s < 8; s++) {
    const int u = ((s >> 1) ^ s) & 1;  // r2 ^ r3
    m[s] = b[nxt(s, u)] + gval(gcode(s, u), Ls, Ls + Lp, Lp);
  }
  normalise<true>(m, b);
}

__device__ __forceinline__ int max8(const int v[8]) {
  return max(__vimax3_s32(__vimax3_s32(v[0], v[1], v[2]), __vimax3_s32(v[3], v[4], v[5]), v[6]),
             v[7]);
}
__device__ __forceinline__ int min8(const int v[8]) {
  return min(__vimin3_s32(__vimin3_s32(v[0], v[1], v[2]), __vimin3_s32(v[3], v[4], v[5]), v[6]),
             v[7]);
}

// Lambda and the extrinsic of one step: returns Le, writes Lambda.  Four
// add-max chains over the transitions grouped by (u, parity); Lp joins the
// parity-0 groups and S (common to u = 0) is added back at the end.
template <bool CHK>
__device__ __forceinline__ int app_step(const int a[8], const int b[8], int S, int Lp, int* lam_out) {
  int acc[4];
  bool first[4] = {true, true, true, true};
#pragma unroll
  for (int s = 0; s < 8; s++)
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int c = gcode(s, u);
      const int n = nxt(s, u);
      if (first[c]) {
        acc[c] = a[s] + b[n];
        first[c] = false;
      } else {
        acc[c] = __viaddmax_s32(a[s], b[n], acc[c]);
      }
    }
  const int d = __viaddmax_s32(acc[3], Lp, acc[2]) - __viaddmax_s32(acc[1], Lp, acc[0]);
  int lam = S + d;
  int le = d;
  if (CHK && (((unsigned)(lam + 32768) | (unsigned)(le + 32768)) > 0xFFFFu)) {
    lam = min(max(lam, -32768), 32767);
    le = min(max(lam - S, -32768), 32767);
  }
  *lam_out = lam;
  return le;
}

// Largest |metric difference| a window pass can reach, from the spreads of
// its start metrics and the branch-metric range g >= |S| + |Lp| of every
// step.  Between two states the metrics of the exact (unsaturated) max-plus
// recursion differ by at most spread_start + k g after k steps and by at most
// 3 g after 3 or more steps (every state pair is joined by exactly one
// 3-step path of the 8-state trellis).  Lambda and Le are bounded by
// spread_alpha + spread_beta + 2 g.  If that stays within int16, no
// saturation can occur in the pass and the clamp-free path is exact.
__device__ __forceinline__ bool window_fast(const int a[8], const int b[8], int g) {
  const int sa = max8(a) - min8(a), sb = max8(b) - min8(b);
  const int Sa = max(sa + 2 * g, 3 * g), Sb = max(sb + 2 * g, 3 * g);
  return Sa + Sb + 2 * g <= 32767;
}

__device__ __forceinline__ int scale_ext(int le) { return (le * 3) >> 2; }

__device__ __forceinline__ uint4 pack8(const int v[8]) {
  uint4 r;
  r.x = __byte_perm(v[0], v[1], 0x5410);
  r.y = __byte_perm(v[2], v[3], 0x5410);
  r.z = __byte_perm(v[4], v[5], 0x5410);
  r.w = __byte_perm(v[6], v[7], 0x5410);
  return r;
}
// pack8 of normalised metrics: the exact path keeps them normalised at
// every step; the clamp-free path normalises here, where the stored value
// must equal the exact path's sat16(m[s] - m[0]) + OFF (no saturation by
// the window_fast bound).
template <bool CHK>
__device__ __forceinline__ uint4 pack_norm(const int v[8]) {
  if (CHK) return pack8(v);
  int o[8];
  const int base = OFF - v[0];
#pragma unroll
  for (int s = 0; s < 8; s++) o[s] = v[s] + base;
  return pack8(o);
}
__device__ __forceinline__ void unpack8(uint4 r, int v[8]) {
  v[0] = r.x & 0xFFFF; v[1] = r.x >> 16;
  v[2] = r.y & 0xFFFF; v[3] = r.y >> 16;
  v[4] = r.z & 0xFFFF; v[5] = r.z >> 16;
  v[6] = r.w & 0xFFFF; v[7] = r.w >> 16;
}

// ---------------------------------------------------------------- helpers
// (x + y) mod K for x in [0, K), y in [0, K]: the unsigned minimum of x + y
// (no overflow: below 2K) and x + y - K (wraps to a large unsigned value when
// negative), as one add and one DPX add-min.  (x - y) mod K is x + (K - y).
__device__ __forceinline__ int modadd(int x, int y, int K) {
  return (int)__viaddmin_u32((unsigned)x, (unsigned)y, (unsigned)(x + y - K));
}
__device__ __forceinline__ int modsub(int x, int y, int K) { return modadd(x, K - y, K); }
__device__ __forceinline__ int qpp_at(int x, int f1, int f2, int K) {
  int t = (f2 * x) % K;
  t = (t * x) % K;
  return (t + f1 * x) % K;
}
// Dynamic shared memory of the decode kernel: CRC tables (2 KiB), the
// mutual-information table, then the CB slots.
extern __shared__ __align__(16) uint8_t smem[];

// A CB's view of its shared-memory slot.  In a one-CB slot element t of a
// stream or of the extrinsic sits at index t (str = 1); in a pair slot lane
// L's element t sits at index 2 t (str = 2) of pointers offset by L.
struct CbSlot {
  int8_t* sys;
  int8_t* par1;
  int8_t* par2;
  int16_t* ext;
  int8_t* tail;
  uint32_t* hard;
  uint4* seed;   // [4][P]: alpha dec0, alpha dec1, beta dec0, beta dec1
  uint4* ck;     // one-CB slot: [P][ceil(W / kSub)]; pair slot: per thread 2 ceil(W / kSubP)
  int* flags;    // [0] done, [1] iterations, [2] CB CRC, [3] TB CRC part, [4..5] max |Le|,
                 // [6] stopped by a purge, [7] window passes on the saturating path,
                 // [8] / [9] mutual information of this / the previous iteration
                 // (2^16 units per bit, summed over the CB), [10] iterations run
  int str;       // index stride of sys / par1 / par2 / ext
  int ck_stride; // uint4 of checkpoints per thread
  int8_t* stage; // where the CB's received LLRs are staged before de-rate-matching
  int stage_cap; // bytes available there (free until the first SISO pass)
};
__device__ __forceinline__ CbSlot make_slot(uint8_t* base, int K, int P, int W) {
  CbSlot s;
  const int tp = W * P;
  const int nck = (W + kSub - 1) / kSub;
  const int nwords = (K + 31) / 32 + 1;
  s.sys = (int8_t*)base;
  s.par1 = s.sys + tp;
  s.par2 = s.sys + 2 * tp;
  uint8_t* q = base + align16(3 * tp);
  s.ext = (int16_t*)q;
  q += align16(2 * tp);
  s.tail = (int8_t*)q;
  q += 16;
  s.hard = (uint32_t*)q;
  q += align16(4 * nwords);
  s.seed = (uint4*)q;
  q += 4 * P * 16;
  s.ck = (uint4*)q;
  q += P * nck * 16;
  s.flags = (int*)q;
  s.str = 1;
  s.ck_stride = nck;
  s.stage = (int8_t*)s.seed;
  s.stage_cap = 16 * P * (4 + nck);
  return s;
}
// Lane L (0 or 1) of a pair slot (layout: pair_layout).  Both lanes share
// the checkpoint area and the staging area (the seeds and checkpoints of both
// CBs), which the pair's two CBs use one after the other.
__device__ __forceinline__ CbSlot make_pair_slot(uint8_t* base, int K, int P, int W, int L) {
  const PairLayout l = pair_layout(K, P, W);
  const int tp = W * P;
  CbSlot s;
  s.sys = (int8_t*)base + L;
  s.par1 = (int8_t*)base + 2 * tp + L;
  s.par2 = (int8_t*)base + 4 * tp + L;
  s.ext = (int16_t*)(base + l.o_ext) + L;
  s.tail = (int8_t*)(base + l.o_tail + 16 * L);
  s.hard = (uint32_t*)(base + l.o_hard + l.hard_bytes * L);
  s.seed = (uint4*)(base + l.o_seed + l.seed_bytes * L);
  s.ck = (uint4*)(base + l.o_ck);
  s.flags = (int*)(base + l.o_flags + 64 * L);
  s.str = 2;
  s.ck_stride = l.ck_per_thread / 16;
  s.stage = (int8_t*)(base + l.o_seed);
  s.stage_cap = l.o_flags - l.o_seed;
  return s;
}
// transposed shared-memory index of natural position q < K
__device__ __forceinline__ int tr_idx(int q, const CbDesc& d) {
  const int w = (int)(((unsigned)q * (unsigned)d.divM) >> d.divS);
  return (q - w * d.W) * d.P + w;
}

__device__ __forceinline__ uint32_t gf_mulmod(uint32_t a, uint32_t b, uint32_t g) {
  uint32_t r = 0;
#pragma unroll
  for (int i = 23; i >= 0; i--) {
    r <<= 1;
    if (r & 0x1000000u) r ^= g;
    if ((a >> i) & 1u) r ^= b;
  }
  return r;
}

// CRC register update over one 32-bit word (MSB first), byte table tab.
__device__ __forceinline__ uint32_t crc_word(uint32_t r, uint32_t w, const uint32_t* tab) {
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t byte = (w >> (24 - 8 * k)) & 0xFFu;
    r = ((r << 8) & 0xFFFFFFu) ^ tab[((r >> 16) ^ byte) & 0xFFu];
  }
  return r;
}

// ---------------------------------------------------------------- de-RM
// De-rate-matching + HARQ combining of one CB into its shared-memory slot:
// every non-NULL circular-buffer position gathers, in order, the received
// LLRs e_k with k = rank - rank(k0) (mod Nv), k < E, adding them with
// saturation to [-127, 127] onto the stored soft value (or 0 for new data),
// and writes the result to its d-stream (and back to the soft buffer).
// The received LLRs e are read from `e`: the CB's LLRs in global memory, or
// their copy staged in shared memory by stage_llrs.
// STR: the slot's index stride (1 one-CB slot, 2 lane of a pair slot; the
// caller zeroes a pair slot's extrinsics).
// ---- bulk copies: cp.async.bulk global -> shared, completed on an
// mbarrier (transaction count in bytes).  A CTA owns two barriers (Bulk);
// every thread tracks the parity each waits for next (the same sequence of
// waits runs on all threads).  Waits are bounded: after 2^22 polls the
// wait records an error in the launch state (reported as CRNT_ETIMEDOUT),
// waits once more with the same bound for the copy still in flight, and
// returns.
struct Bulk {
  uint32_t bar;    // shared address of barrier 0; barrier 1 at bar + 8
  uint32_t phase;  // bit b: parity barrier b completes next
  int32_t* err;
};
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bulk_fence() {
  // orders this thread's (and, after a barrier, the CTA's) earlier
  // shared-memory accesses before the asynchronous proxy's writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one copy of `bytes` (a multiple of 16, both addresses 16-byte aligned),
// announced on the barrier by this thread's arrival
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_poll(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 22); i++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_wait(Bulk& bk, int b) {
  const uint32_t bar = bk.bar + 8u * (uint32_t)b, par = (bk.phase >> b) & 1u;
  if (!mbar_poll(bar, par)) {
    atomicCAS(bk.err, 0, 2);
    mbar_poll(bar, par);
  }
  bk.phase ^= 1u << b;
}

// Where one CB's de-rate-matched LLRs come from and go (the map path).
struct DermTarget {
  const int8_t* e;  // its E received LLRs (staged copy or global)
  int8_t* base;     // the slot's streams (sys, then par1, par2)
  int8_t* tail;     // its tail LLRs
  int8_t* soft;     // its soft buffer, or null
  bool combine;     // add the soft buffer's contents
  int rank0, E;
};
__device__ __forceinline__ DermTarget derm_target(const CbDesc& d, const CbSlot& sl,
                                                  const int8_t* e, int8_t* soft_arena) {
  DermTarget t;
  t.e = e;
  t.base = sl.sys;
  t.tail = sl.tail;
  t.soft = d.soft_off >= 0 ? soft_arena + d.soft_off : nullptr;
  t.combine = t.soft != nullptr && !d.new_data;
  t.rank0 = d.rank0;
  t.E = d.E;
  return t;
}

// De-rate-matching of a CB into its slot.  d2 / s2 / e2 (optional, only
// with a map): a second CB with the same (K, P, F) -- the other CB of a
// pair -- de-rate-matched in the same pass over the map, which is then
// streamed into shared memory once for both.
template <int STR>
__device__ void derm_cb(const CbDesc& d, const CbSlot& sl, const int8_t* e,
                        int8_t* __restrict__ soft_arena, int tid, int nthr, uint8_t* mbuf,
                        int mbuf_bytes, Bulk& bk, const CbDesc* d2 = nullptr,
                        const CbSlot* s2 = nullptr, const int8_t* e2 = nullptr) {
  // descriptor fields in registers: the shared-memory stores below go
  // through generic pointers and would otherwise force reloads
  const int K = d.K, F = d.F, R = d.R, E = d.E, Nv = d.Nv, rank0 = d.rank0;
  const int P = d.P, W = d.W, divS = d.divS;
  const unsigned divM = d.divM;
  const RmGeom g{K, F, R, d.ND, d.maskB, d.mask2};
  int8_t* soft = d.soft_off >= 0 ? soft_arena + d.soft_off : nullptr;
  const bool combine = soft != nullptr && !d.new_data;
  auto tr = [&](int q) {
    const int w = (int)(((unsigned)q * divM) >> divS);
    return (q - w * W) * P + w;
  };
  int8_t* const streams[3] = {sl.sys, sl.par1, sl.par2};
  const uint32_t* __restrict__ dm = d.dm;
  if (dm != nullptr) {
    // with the (K, P, F) map: one circular-buffer rank r per thread and
    // step; the map gives its buffer position (soft buffer) and its place in
    // the slot (streams at s W P, tail bits after 3 W P).  NULL positions
    // (dummies, filler bits) are not visited: no step reads their soft
    // entries, and the filler loop below fills the filler places.
    const int tp3 = 3 * W * P;
    const DermTarget tA = derm_target(d, sl, e, soft_arena);
    DermTarget tB = tA;
    if (d2) tB = derm_target(*d2, *s2, e2, soft_arena);
    // rank r's received LLRs are e[k], e[k + Nv], ... for k = r - rank0
    // (mod Nv) below E, summed (with the soft buffer's entry when combining)
    // and saturated to int8
    auto visit = [&](const DermTarget& t, uint32_t m, int r) {
      int k = r - t.rank0;
      if (k < 0) k += Nv;
      const int pos = (int)(m >> 16), dst = (int)(m & 0xFFFFu);
      int acc = t.combine ? t.soft[pos] : 0;
      for (; k < t.E; k += Nv) acc = max(min(acc + (int)t.e[k], 127), -127);
      const int8_t v = (int8_t)acc;
      if (dst < tp3) t.base[STR * dst] = v;  // streams are contiguous: s tp + t -> STR (s tp + t)
      else t.tail[dst - tp3] = v;
      if (t.soft) t.soft[pos] = v;
    };
    // the common case -- no soft buffer and E <= Nv, so at most one LLR per
    // rank -- with the same result: max(e[k], -127), or 0 when k >= E
    auto visit_one = [&](const DermTarget& t, uint32_t m, int r) {
      int k = r - t.rank0;
      if (k < 0) k += Nv;
      const int dst = (int)(m & 0xFFFFu);
      const int8_t v = k < t.E ? (int8_t)max((int)t.e[k], -127) : (int8_t)0;
      if (dst < tp3) t.base[STR * dst] = v;
      else t.tail[dst - tp3] = v;
    };
    // both CBs of a pair in the common case: their streams are interleaved
    // byte by byte (STR 2, B's at A's + 1), so one 16-bit store places both
    auto visit_two = [&](uint32_t m, int r) {
      int kA = r - tA.rank0, kB = r - tB.rank0;
      if (kA < 0) kA += Nv;
      if (kB < 0) kB += Nv;
      const int dst = (int)(m & 0xFFFFu);
      const int vA = kA < tA.E ? max((int)tA.e[kA], -127) : 0;
      const int vB = kB < tB.E ? max((int)tB.e[kB], -127) : 0;
      if (dst < tp3) {
        *(uint16_t*)(tA.base + 2 * dst) = (uint16_t)((vA & 0xFF) | ((vB & 0xFF) << 8));
      } else {
        tA.tail[dst - tp3] = (int8_t)vA;
        tB.tail[dst - tp3] = (int8_t)vB;
      }
    };
    // two consecutive ranks r, r + 1 of both CBs (r even; Nv is even, so
    // r + 1 < Nv): one 8-byte map read, the second offsets from the first
    auto visit_two2 = [&](uint2 mm, int r) {
      int kA = r - tA.rank0, kB = r - tB.rank0;
      if (kA < 0) kA += Nv;
      if (kB < 0) kB += Nv;
      const int kA1 = kA + 1 == Nv ? 0 : kA + 1, kB1 = kB + 1 == Nv ? 0 : kB + 1;
      const int d0 = (int)(mm.x & 0xFFFFu), d1 = (int)(mm.y & 0xFFFFu);
      const int vA0 = kA < tA.E ? max((int)tA.e[kA], -127) : 0;
      const int vB0 = kB < tB.E ? max((int)tB.e[kB], -127) : 0;
      const int vA1 = kA1 < tA.E ? max((int)tA.e[kA1], -127) : 0;
      const int vB1 = kB1 < tB.E ? max((int)tB.e[kB1], -127) : 0;
      if (d0 < tp3) {
        *(uint16_t*)(tA.base + 2 * d0) = (uint16_t)((vA0 & 0xFF) | ((vB0 & 0xFF) << 8));
      } else {
        tA.tail[d0 - tp3] = (int8_t)vA0;
        tB.tail[d0 - tp3] = (int8_t)vB0;
      }
      if (d1 < tp3) {
        *(uint16_t*)(tA.base + 2 * d1) = (uint16_t)((vA1 & 0xFF) | ((vB1 & 0xFF) << 8));
      } else {
        tA.tail[d1 - tp3] = (int8_t)vA1;
        tB.tail[d1 - tp3] = (int8_t)vB1;
      }
    };
    auto run = [&](auto vis, auto wide) {
      constexpr bool WIDE = decltype(wide)::value;
      if (mbuf_bytes >= 2048) {
        // the map streamed through mbuf (free until the first SISO pass) in
        // two alternating chunks of ce entries, each one bulk copy; chunk c +
        // 2 is issued once every thread is done with chunk c.  The map starts
        // 16-byte aligned and holds a multiple of 4 entries, so every copy is
        // whole 16-byte units inside the map.
        const int ce = min(2048, ((mbuf_bytes >> 1) >> 4) << 2);
        const int nch = (Nv + ce - 1) / ce;
        const uint32_t b0 = smem_u32(mbuf);
        auto issue = [&](int c) {
          const int r0 = c * ce;
          const uint32_t bytes = 4u * (uint32_t)(min(Nv, r0 + ce) - r0);
          bulk_load(b0 + 4u * (uint32_t)((c & 1) * ce), dm + r0, bytes, bk.bar + 8u * (c & 1));
        };
        if (tid == 0) {
          bulk_fence();
          issue(0);
          if (nch > 1) issue(1);
        }
        for (int c = 0; c < nch; c++) {
          bulk_wait(bk, c & 1);
          const uint32_t* m = (const uint32_t*)mbuf + (c & 1) * ce;
          const int r0 = c * ce, r1 = min(Nv, r0 + ce);
          if constexpr (WIDE) {
            // ranks in pairs (r1 - r0 is even: Nv and ce are)
#pragma unroll 2
            for (int r = r0 + 2 * tid; r < r1; r += 2 * nthr)
              vis(*(const uint2*)(m + (r - r0)), r);
          } else {
#pragma unroll 4
            for (int r = r0 + tid; r < r1; r += nthr) vis(m[r - r0], r);
          }
          __syncthreads();  // chunk c read by all: its buffer can be refilled
          if (tid == 0 && c + 2 < nch) {
            bulk_fence();
            issue(c + 2);
          }
        }
      } else if constexpr (WIDE) {
        for (int r = 2 * tid; r < Nv; r += 2 * nthr) vis(__ldg((const uint2*)(dm + r)), r);
      } else {
#pragma unroll 8
        for (int r = tid; r < Nv; r += nthr) vis(__ldg(dm + r), r);
      }
    };
    const std::false_type narrow{};
    const bool one = tA.soft == nullptr && E <= Nv && (!d2 || (tB.soft == nullptr && tB.E <= Nv));
    if (d2) {
      if (one && STR == 2 && tB.base == tA.base + 1)
        run(visit_two2, std::true_type{});
      else if (one)
        run([&](uint32_t m, int r) { visit_one(tA, m, r); visit_one(tB, m, r); }, narrow);
      else
        run([&](uint32_t m, int r) { visit(tA, m, r); visit(tB, m, r); }, narrow);
    } else if (one) {
      run([&](uint32_t m, int r) { visit_one(tA, m, r); }, narrow);
    } else {
      run([&](uint32_t m, int r) { visit(tA, m, r); }, narrow);
    }
  }
  // otherwise rows x = unit * R + i, walked with (unit, i) updated incrementally
  const int nrows = dm != nullptr ? 0 : 64 * R;
  int unit = tid / R, i = tid - (tid / R) * R;
  const int du = nthr / R, di_ = nthr - du * R;
  for (int x = tid; x < nrows; x += nthr) {
    rm_visit(
        g, unit, i,
        [&](int p, int st, int di, int rank) {
          int k = rank - rank0;
          if (k < 0) k += Nv;
          int acc = combine ? soft[p] : 0;
          for (; k < E; k += Nv) acc = max(min(acc + (int)e[k], 127), -127);
          const int8_t v = (int8_t)acc;
          if (di < K) streams[st][STR * tr(di)] = v;
          else sl.tail[3 * (di - K) + st] = v;
          if (soft) soft[p] = v;
        },
        [&](int p) {
          if (soft && !combine) soft[p] = 0;
        });
    unit += du;
    i += di_;
    if (i >= R) {
      i -= R;
      unit++;
    }
  }
  // filler: known zero bits in the systematic stream, unknown parity 1
  for (int k = tid; k < F; k += nthr) {
    const int t = tr(k);
    sl.sys[STR * t] = 127;
    sl.par1[STR * t] = 0;
    if (d2) {
      s2->sys[STR * t] = 127;
      s2->par1[STR * t] = 0;
    }
  }
  if (STR == 1) {
    const int tp = W * P;
    uint4* ext16 = (uint4*)sl.ext;  // the ext area is 16-byte aligned and padded
    for (int k = tid; k < (2 * tp + 15) / 16; k += nthr) ext16[k] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int k = 0; k < 10; k++) sl.flags[k] = 0;
    if (d2)
      for (int k = 0; k < 10; k++) s2->flags[k] = 0;
  }
}

// Copy of the CB's E received LLRs into the slot's seed + checkpoint area,
// which the first SISO pass writes before reading.  Bulk 16-byte loads, all
// issued before any is consumed, replace the de-rate-matcher's scattered
// dependent byte loads from global memory.  The copy keeps the global
// address modulo 16 (byte k at stage + (e & 15) + k) so that the 16-byte
// body is aligned on both sides; the head and tail bytes are copied singly
// and no byte outside [e, e + E) is read.  llr_src gives the pointer the
// de-rate-matcher reads: the staged copy, or the global LLRs when E does not
// fit (heavy repetition; stage_llrs then copies nothing).
__device__ __forceinline__ const int8_t* llr_src(const CbDesc& d, const CbSlot& sl,
                                                 const int8_t* llr) {
  const int8_t* e = llr + d.llr_off;
  if (d.E + 15 > sl.stage_cap) return e;
  return (const int8_t*)sl.stage + ((uintptr_t)e & 15u);
}
__device__ void stage_llrs(const CbDesc& d, const CbSlot& sl, const int8_t* __restrict__ llr,
                           int tid, int nthr) {
  const int8_t* e = llr + d.llr_off;
  const int E = d.E;
  const int8_t* src = llr_src(d, sl, llr);
  if (src == e) return;
  const int s0 = (int)((uintptr_t)e & 15u);
  int8_t* st = sl.stage + s0;
  const int head = min(E, (16 - s0) & 15);
  const int n16 = (E - head) >> 4;
  const int tail0 = head + 16 * n16;
  for (int k = tid; k < head; k += nthr) st[k] = e[k];
  for (int k = tail0 + tid; k < E; k += nthr) st[k] = e[k];
  const int4* gsrc = (const int4*)(e + head);
  int4* sdst = (int4*)(st + head);
  constexpr int kBatch = 1;
  for (int i0 = tid; i0 < n16; i0 += kBatch * nthr) {
    int4 v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const int i = i0 + u * nthr;
      if (i < n16) v[u] = __ldg(gsrc + i);
    }
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const int i = i0 + u * nthr;
      if (i < n16) sdst[i] = v[u];
    }
  }
}

// ---------------------------------------------------------------- SISO
// Per-window state of one SISO pass.
struct Win {
  const int8_t* __restrict__ sys;
  const int8_t* __restrict__ par;
  int16_t* ext;
  uint32_t* hard;
  int K, P, W, divM, divS;  // geometry (tr_idx)
  int f2x2;                 // QPP first-difference step
  int p, lo, len, pad;
  bool hard_on;             // DEC 1: form the hard decisions
  bool r4;                  // radix-4 forward recursion on the clamp-free path
  const uint4* __restrict__ qt;  // interleaved-pass address table (QT kernels)
  const uint2* __restrict__ qq;  // its natural positions, 16 bits each
};

__device__ __forceinline__ int tr_w(const Win& w, int q) {
  const int t = (int)(((unsigned)q * (unsigned)w.divM) >> w.divS);
  return (q - t * w.W) * w.P + t;
}

// Load the branch-metric inputs of step j (window-relative) of pass DEC.
// DEC 1 walks the QPP addresses (q, dq) and returns the natural position;
// with QT the caller passes the step's transposed address tq, read from the
// CB's address table, and q, dq are not used.
// STR: index stride of the slot (2 when the window is one lane of a pair slot).
template <int DEC, bool QT, int STR = 1>
__device__ __forceinline__ void load_step(const Win& w, int j, int& q, int& dq, int tq, int& S,
                                          int& Lp, int& t) {
  const int idx = j * w.P + w.p;
  if (DEC == 0) {
    t = idx;
  } else if (QT) {
    t = tq;
  } else {
    t = tr_w(w, q);
  }
  S = (int)w.sys[STR * t] + (int)w.ext[STR * t];
  Lp = w.par[STR * idx];
  if (DEC == 1 && !QT) {
    q = modadd(q, dq, w.K);
    dq = modadd(dq, w.f2x2, w.K);
  }
}

// Component k (compile-time after unrolling) of a table entry.
__device__ __forceinline__ int comp4(const uint4& e, int k) {
  return k == 0 ? (int)e.x : k == 1 ? (int)e.y : k == 2 ? (int)e.z : (int)e.w;
}
__device__ __forceinline__ int comp2(const uint2& e, int k) {
  const unsigned v = k < 2 ? e.x : e.y;
  return (k & 1) ? (int)(v >> 16) : (int)(v & 0xFFFFu);
}

// Backward processing of one sub-window [j0, j0 + slen) of a window:
// recompute forward metrics from the checkpoint into registers, then walk
// back computing Lambda / Le and the backward metrics.  FULL: slen == kSub
// (no per-step guards).  mx / mn track the largest / smallest extrinsic
// written.  With
// w.hard_on (DEC 1 only) the hard decisions sign(Lambda) are also recorded
// at the natural positions; HM selects that test at compile time (0: no
// hard decisions, 1: hard decisions, 2: read w.hard_on).  QT (DEC 1): te
// holds the sub-window's four transposed addresses and qe (with hard
// decisions) their natural positions.
template <int DEC, bool FULL, bool CHK, bool QT, int HM, int STR = 1>
__device__ __forceinline__ void sub_window_back(const Win& w, uint4 ck, int j0, int slen, int q,
                                                int dq, uint4 te, uint2 qe, int b[8], int& mx,
                                                int& mn) {
  int A[kSub][8];
  int Sv[kSub], Lv[kSub], Qv[kSub];
  int vprev = 0;  // extrinsics enter the max / min tracking in pairs
  unpack8(ck, A[0]);
#pragma unroll
  for (int jj = 0; jj < kSub; jj++) {
    if (FULL || jj < slen) {
      if (!QT) Qv[jj] = q;
      int t;
      load_step<DEC, QT, STR>(w, j0 + jj, q, dq, QT ? comp4(te, jj) : 0, Sv[jj], Lv[jj], t);
      if (QT) Qv[jj] = t;
      if (jj + 1 < kSub && (FULL || jj + 1 < slen))
        alpha_step<CHK>(A[jj], A[jj + 1], Sv[jj], Sv[jj] + Lv[jj], Lv[jj]);
    }
  }
#pragma unroll
  for (int jj = kSub - 1; jj >= 0; jj--) {
    if (FULL || jj < slen) {
      const int S = Sv[jj], Lp = Lv[jj];
      int lam;
      const int le = app_step<CHK>(A[jj], b, S, Lp, &lam);
      const int v = scale_ext(le);
      if (jj & 1) {
        vprev = v;
      } else {
        mx = __vimax3_s32(mx, vprev, v);
        mn = __vimin3_s32(mn, vprev, v);
      }
      w.ext[STR * (DEC == 0 ? (j0 + jj) * w.P + w.p : QT ? Qv[jj] : tr_w(w, Qv[jj]))] =
          (int16_t)v;
      if (DEC == 1 && (HM == 1 || (HM == 2 && w.hard_on))) {  // ORs a zero when lam >= 0
        const int qq = (QT ? comp2(qe, jj) : Qv[jj]) + w.pad;
        atomicOr(&w.hard[qq >> 5], ((unsigned)lam >> 31) << (31 - (qq & 31)));
      }
      beta_step<CHK>(b, S, S + Lp, Lp);
    }
  }
}

// Forward and backward recursions of one window (after the seeds are read).
// R4: the kernel instantiation that carries the radix-4 forward recursion
// (used by CBs with radix4 set, on clamp-free passes).  QT: the interleaved
// pass reads its addresses from the CB's table (w.qt, one uint4 of four
// transposed addresses per kSub-step group and window, plus two zero groups
// at the end so that groups can always be fetched two ahead).  The table
// lives in global memory (L2), so its loads are issued ahead of use: groups
// 0 and 1 (pf0, pf1) before the pass's barrier, then two groups ahead in the
// forward pass and one sub-window ahead in the backward pass, whose first
// group is fetched before the forward pass.
template <int DEC, bool CHK, bool R4, bool QT, int STR = 1>
__device__ __forceinline__ void window_pass(const Win& w, const CbDesc* __restrict__ dp,
                                            uint4* ck, uint4* seedA, uint4* seedB, int a[8],
                                            int b[8], int& mx, int& mn, uint4 pf0, uint4 pf1) {
  constexpr bool TQ = QT && DEC == 1;  // table addresses in this pass
  const int K = w.K, P = w.P, p = w.p, lo = w.lo, len = w.len;
  const int f1 = dp->f1, f2 = dp->f2;
  const int f2sub = DEC ? dp->f2sub : 0, f2jump = DEC ? dp->f2jump : 0;
  const uint4* __restrict__ tq = TQ ? w.qt + p : nullptr;  // group g at tq[g * P]

  // ---- forward pass with a checkpoint every kSub steps
  int q = 0, dq = 0;
  if (DEC == 1 && !TQ) {
    q = qpp_at(lo, f1, f2, K);
    dq = (f1 + (f2 * ((2 * lo + 1) % K)) % K) % K;
  }
  const int nsub = (len + kSub - 1) / kSub;
  uint4 te = pf0, te1 = pf1, tb = make_uint4(0u, 0u, 0u, 0u);
  uint2 qn = make_uint2(0u, 0u);
  if (TQ) {
    tb = __ldg(tq + (nsub - 1) * P);
    if (w.hard_on) qn = __ldg(w.qq + (nsub - 1) * P + p);
  }
  int j0 = 0;
  if (R4 && !CHK && w.r4) {  // radix-4 forward recursion (same metrics, see alpha_step_r4)
    for (; j0 + kSub <= len; j0 += kSub) {
      ck[j0 / kSub] = pack_norm<CHK>(a);
      const uint4 cur = te;
      if (TQ) {
        te = te1;
        te1 = __ldg(tq + (j0 / kSub + 2) * P);
      }
#pragma unroll
      for (int jj = 0; jj < kSub; jj += 4) {
        int S0, L0, S1, L1, t, o[8];
        load_step<DEC, TQ, STR>(w, j0 + jj, q, dq, comp4(cur, jj), S0, L0, t);
        load_step<DEC, TQ, STR>(w, j0 + jj + 1, q, dq, comp4(cur, jj + 1), S1, L1, t);
        alpha_step_r4(a, o, S0, L0, S1, L1);
        load_step<DEC, TQ, STR>(w, j0 + jj + 2, q, dq, comp4(cur, jj + 2), S0, L0, t);
        load_step<DEC, TQ, STR>(w, j0 + jj + 3, q, dq, comp4(cur, jj + 3), S1, L1, t);
        alpha_step_r4(o, a, S0, L0, S1, L1);
      }
    }
  } else {
    for (; j0 + kSub <= len; j0 += kSub) {
      ck[j0 / kSub] = pack_norm<CHK>(a);
      const uint4 cur = te;
      if (TQ) {
        te = te1;
        te1 = __ldg(tq + (j0 / kSub + 2) * P);
      }
#pragma unroll
      for (int jj = 0; jj < kSub; jj += 2) {
        int S, Lp, t, o[8];
        load_step<DEC, TQ, STR>(w, j0 + jj, q, dq, comp4(cur, jj), S, Lp, t);
        alpha_step<CHK>(a, o, S, S + Lp, Lp);
        load_step<DEC, TQ, STR>(w, j0 + jj + 1, q, dq, comp4(cur, jj + 1), S, Lp, t);
        alpha_step<CHK>(o, a, S, S + Lp, Lp);
      }
    }
  }
  if (j0 < len) {
    ck[j0 / kSub] = pack_norm<CHK>(a);
    for (int j = j0; j < len; j++) {
      int S, Lp, t, o[8];
      load_step<DEC, TQ, STR>(w, j, q, dq, TQ ? comp4(te, j - j0) : 0, S, Lp, t);
      alpha_step<CHK>(a, o, S, S + Lp, Lp);
#pragma unroll
      for (int s = 0; s < 8; s++) a[s] = o[s];
    }
  }
  if (p + 1 < P) seedA[p + 1] = pack_norm<CHK>(a);

  // ---- backward pass, one sub-window at a time from the end.  QPP state
  // at the start of the last sub-window, walked backwards by kSub steps:
  // PI(x - kSub) = PI(x) - J(x - kSub) with J(x) = kSub f1 + f2 (2 kSub x +
  // kSub^2), J(x - kSub) = J(x) - 2 kSub^2 f2, delta(x - kSub) = delta(x) -
  // 2 kSub f2.  With the table, sub-window sw reads group sw instead.
  int pis = 0, dls = 0, jmp = 0;
  if (DEC == 1 && !TQ) {
    const int is = lo + kSub * (nsub - 1);
    pis = qpp_at(is, f1, f2, K);
    dls = (f1 + (f2 * ((2 * is + 1) % K)) % K) % K;
    int t = (2 * kSub * is - kSub * kSub) % K;
    if (t < 0) t += K;
    jmp = ((kSub * f1) % K + (f2 * t) % K) % K;
  }
  int sw = nsub - 1;
  te = tb;
  const int last_len = len - kSub * sw;
  if (last_len < kSub) {
    const uint4 cur = te;
    const uint2 qcur = qn;
    if (TQ) {
      te = __ldg(tq + max(sw - 1, 0) * P);
      if (w.hard_on) qn = __ldg(w.qq + max(sw - 1, 0) * P + p);
    }
    sub_window_back<DEC, false, CHK, TQ, 2, STR>(w, ck[sw], kSub * sw, last_len, pis, dls, cur, qcur,
                                            b, mx, mn);
    if (DEC == 1 && !TQ) {
      pis = modsub(pis, jmp, K);
      dls = modsub(dls, f2sub, K);
      jmp = modsub(jmp, f2jump, K);
    }
    sw--;
  }
  // the full sub-windows, in two copies so that passes without hard
  // decisions carry no per-step test for them
  auto full_back = [&](auto hm) {
    constexpr int HM = decltype(hm)::value;
    for (; sw >= 0; sw--) {
      const uint4 cur = te;
      const uint2 qcur = qn;
      if (TQ) {
        te = __ldg(tq + max(sw - 1, 0) * P);
        if (HM == 1) qn = __ldg(w.qq + max(sw - 1, 0) * P + p);
      }
      sub_window_back<DEC, true, CHK, TQ, HM, STR>(w, ck[sw], kSub * sw, kSub, pis, dls, cur, qcur, b,
                                              mx, mn);
      if (DEC == 1 && !TQ) {
        pis = modsub(pis, jmp, K);
        dls = modsub(dls, f2sub, K);
        jmp = modsub(jmp, f2jump, K);
      }
    }
  };
  if (DEC == 1 && w.hard_on)
    full_back(std::integral_constant<int, 1>());
  else
    full_back(std::integral_constant<int, 0>());
  if (p > 0) seedB[p - 1] = pack_norm<CHK>(b);
}

// One SISO pass of window p of one CB.  DEC = 0: natural order (encoder 1),
// DEC = 1: QPP order (encoder 2).  All threads of the CTA call it (run =
// false for idle threads) because it contains barriers.  flags[4 + d] holds
// the largest |extrinsic| written by the last pass of decoder d, which
// bounds |La| for the pass that reads it.  hard (DEC 1): the hard decisions
// of this iteration are used (a CRC check follows); otherwise they are not
// formed, since the next iteration overwrites them unread.
template <int DEC, bool R4, bool QT>
__device__ __forceinline__ void siso_pass(const CbDesc* __restrict__ dp, uint8_t* base, int p,
                                          bool run, bool first, bool hard) {
  const int K = dp->K, P = dp->P, W = dp->W;
  const CbSlot sl = make_slot(base, K, P, W);
  uint4* seedA = sl.seed + DEC * P;
  uint4* seedB = sl.seed + (2 + DEC) * P;
  uint4* ck = sl.ck + p * ((W + kSub - 1) / kSub);

  int a[8], b[8];
  int m_in = 0;
  uint4 pf0 = make_uint4(0u, 0u, 0u, 0u), pf1 = pf0;
  if (QT && DEC == 1 && run) {  // the first two address groups, fetched across the barrier
    const uint4* __restrict__ qt = dp->qt;
    pf0 = __ldg(qt + p);
    pf1 = __ldg(qt + P + p);
  }
  if (run) {
    if (p == 0) {
      a[0] = OFF;
#pragma unroll
      for (int s = 1; s < 8; s++) a[s] = MINF_OFF;
    } else if (first) {
#pragma unroll
      for (int s = 0; s < 8; s++) a[s] = OFF;
    } else {
      unpack8(seedA[p], a);
    }
    if (p == P - 1) {
      b[0] = OFF;
#pragma unroll
      for (int s = 1; s < 8; s++) b[s] = MINF_OFF;
    } else if (first) {
#pragma unroll
      for (int s = 0; s < 8; s++) b[s] = OFF;
    } else {
      unpack8(seedB[p], b);
    }
    m_in = sl.flags[5 - DEC];
    if (p == 0) sl.flags[4 + DEC] = 0;  // written by this pass after the barrier
    if (DEC == 1 && hard) {
      const int nwords = (K + 31) / 32;
      for (int w = p; w < nwords; w += P) sl.hard[w] = 0u;
    }
  }
  __syncthreads();
  if (run) {
    Win w;
    w.sys = sl.sys;
    w.par = DEC ? sl.par2 : sl.par1;
    w.ext = sl.ext;
    w.hard = sl.hard;
    w.hard_on = hard;
    w.r4 = R4 && dp->radix4 != 0;
    w.qt = QT ? dp->qt : nullptr;
    w.qq = QT ? dp->qq : nullptr;
    w.K = K;
    w.P = P;
    w.W = W;
    w.divM = dp->divM;
    w.divS = dp->divS;
    w.f2x2 = dp->f2x2;
    w.p = p;
    w.lo = p * W;
    w.len = min(W, K - w.lo);
    w.pad = ((K + 31) / 32) * 32 - K;
    if (p == P - 1) {
      const int8_t* t = sl.tail + (DEC ? 6 : 0);
#pragma unroll
      for (int j = 2; j >= 0; j--) beta_tail_step(b, t[2 * j], t[2 * j + 1]);
    }
    int mx = 0, mn = 0;
    if (window_fast(a, b, 254 + m_in)) {
      window_pass<DEC, false, R4, QT>(w, dp, ck, seedA, seedB, a, b, mx, mn, pf0, pf1);
    } else {
      window_pass<DEC, true, R4, QT>(w, dp, ck, seedA, seedB, a, b, mx, mn, pf0, pf1);
      atomicAdd(&sl.flags[7], 1);  // counted per CB, reported per TB
    }
    atomicMax(&sl.flags[4 + DEC], max(mx, -mn));
  }
  __syncthreads();
}

// CRC of the CB's hard bits held by this thread's share of words.  mode 0:
// the CB's own CRC over bits [F, K); mode 1: CRC24A over [F, K - 24) followed
// by 24 zeros (the TB CRC contribution).
__device__ uint32_t crc_share(const CbDesc& d, const CbSlot& sl, int p, const uint32_t* tab,
                              uint32_t g, const uint32_t* xpow, int mode) {
  const int K = d.K, P = d.P;
  const int nw = (K + 31) / 32;
  const int pad = nw * 32 - K;
  const int per = (nw + P - 1) / P;
  const int w0 = p * per;
  const int w1 = min(nw, w0 + per);
  if (w0 >= w1) return 0u;
  const int fq = pad + d.F;  // first message bit position in padded order
  uint32_t r = 0;
  for (int w = w0; w < w1; w++) {
    uint32_t word = sl.hard[w];
    const int wq = 32 * w;
    if (fq > wq) word = (fq >= wq + 32) ? 0u : (word & (0xFFFFFFFFu >> (fq - wq)));
    if (mode == 1 && w == nw - 1) word &= 0xFF000000u;  // drop the CB CRC (last 24 bits)
    r = crc_word(r, word, tab);
  }
  const int after = nw - w1;
  return after ? gf_mulmod(r, __ldg(&xpow[after]), g) : r;
}

// ---------------------------------------------------------------- CB pairs
// A thread of a pair item runs window p of two CBs of equal (K, P) at once:
// CB A in the low and CB B in the high 16-bit lane of each register, every
// add-max a DPX s16x2 instruction.  Both CBs' streams and extrinsics are
// interleaved in the pair slot, so one load serves both lanes, and the
// interleaved pass's addresses (equal for both) come from one table read.
// The lanes hold metrics relative to state 0 of the last normalisation,
// which happens every kSubP steps (checkpoints in the forward pass, sub-
// window ends in the backward pass).  pair_fast proves, per lane, that the
// pass is clamp-free (window_fast) and that no lane value leaves int16, so
// the results equal the one-CB path's exactly; otherwise (and for a CB whose
// partner has stopped) each lane runs the one-CB code on its stride-2 view.

__device__ __forceinline__ unsigned prmt(unsigned a, unsigned b, unsigned sel) {
  unsigned d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}
// the two bytes of x's low half, sign-extended into the two 16-bit lanes
__device__ __forceinline__ unsigned sext8x2(unsigned x) { return prmt(x, 0u, 0x9180u); }
__device__ __forceinline__ int lane_lo(unsigned x) { return (int)(short)(x & 0xFFFFu); }
__device__ __forceinline__ int lane_hi(unsigned x) { return (int)x >> 16; }
__device__ __forceinline__ unsigned pack_lanes(int lo, int hi) {
  return prmt((unsigned)lo, (unsigned)hi, 0x5410u);
}

__device__ __forceinline__ unsigned gval_p(int code, unsigned S, unsigned T, unsigned L) {
  return code == 3 ? T : code == 2 ? S : code == 1 ? L : 0u;
}
__device__ __forceinline__ unsigned acs_p(unsigned x0, int c0, unsigned x1, int c1, unsigned S,
                                          unsigned T, unsigned L) {
  if (c1 == 0) return __viaddmax_s16x2(x0, gval_p(c0, S, T, L), x1);
  if (c0 == 0) return __viaddmax_s16x2(x1, gval_p(c1, S, T, L), x0);
  return __viaddmax_s16x2(x0, gval_p(c0, S, T, L), __vadd2(x1, gval_p(c1, S, T, L)));
}
__device__ __forceinline__ void alpha_step_p(const unsigned a[8], unsigned o[8], unsigned S,
                                             unsigned L) {
  const unsigned T = __vadd2(S, L);
#pragma unroll
  for (int n = 0; n < 8; n++)
    o[n] = acs_p(a[pred(n, 0)], pcode(n, 0), a[pred(n, 1)], pcode(n, 1), S, T, L);
}
__device__ __forceinline__ void beta_step_p(unsigned b[8], unsigned S, unsigned L) {
  const unsigned T = __vadd2(S, L);
  unsigned m[8];
#pragma unroll
  for (int s = 0; s < 8; s++)
    m[s] = acs_p(b[nxt(s, 0)], gcode(s, 0), b[nxt(s, 1)], gcode(s, 1), S, T, L);
#pragma unroll
  for (int s = 0; s < 8; s++) b[s] = m[s];
}
// subtract each lane's state-0 metric (a constant per lane: exact here)
__device__ __forceinline__ void norm_p(unsigned v[8]) {
#pragma unroll
  for (int s = 1; s < 8; s++) v[s] = __vsub2(v[s], v[0]);
  v[0] = 0u;
}
// Le of both lanes (Lambda - S, exact); Lambda = S + Le.
__device__ __forceinline__ unsigned app_step_p(const unsigned a[8], const unsigned b[8], unsigned L) {
  unsigned acc[4];
  bool first[4] = {true, true, true, true};
#pragma unroll
  for (int s = 0; s < 8; s++)
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int c = gcode(s, u);
      const int n = nxt(s, u);
      if (first[c]) {
        acc[c] = __vadd2(a[s], b[n]);
        first[c] = false;
      } else {
        acc[c] = __viaddmax_s16x2(a[s], b[n], acc[c]);
      }
    }
  return __vsub2(__viaddmax_s16x2(acc[3], L, acc[2]), __viaddmax_s16x2(acc[1], L, acc[0]));
}

// Largest |metric - metric of state 0 at the last normalisation| a lane can
// reach within kSubP steps of a normalisation, from start metrics v (offset
// form), |branch metric| <= g.  Within the sub-window that starts at the
// window's start: upward at most the start maximum + 8 g; downward the start
// minimum - 2 g for the first two steps, after which every state lies within
// 3 g of the best one (each state pair is joined by one 3-step path), so at
// least -11 g.  Sub-windows that start 3 or more steps into the window: 11 g.
// short_first: the recursion normalises after only 1 or 2 steps (the
// backward pass when the window's last sub-window is that short); the next
// sub-window then starts with a spread of at most spread + 2 g, so it reaches
// spread + 10 g.
__device__ __forceinline__ int lane_reach(const int v[8], int g, bool short_first) {
  const int hi = max8(v) - v[0], lo = v[0] - min8(v);
  int r = max(max(hi + kSubP * g, lo + 2 * g), (kSubP + 3) * g);
  if (short_first) r = max(r, hi + lo + (kSubP + 2) * g);
  return r;
}
// The pass of one lane may run on 16-bit lanes: clamp-free (window_fast) and
// every alpha + beta + Lp sum of Lambda within int16.  len: the window's steps.
__device__ __forceinline__ bool pair_fast(const int a[8], const int b[8], int g, int len) {
  const int last = len - kSubP * ((len - 1) / kSubP);
  const bool short_first = len > kSubP && last < 3;
  return window_fast(a, b, g) &&
         lane_reach(a, g, false) + lane_reach(b, g, short_first) + g <= 32767;
}

// offset-form metrics of lanes A and B -> signed 16-bit lane pairs
__device__ __forceinline__ void to_lanes(const int vA[8], const int vB[8], unsigned o[8]) {
#pragma unroll
  for (int s = 0; s < 8; s++) o[s] = pack_lanes(vA[s], vB[s]) ^ 0x80008000u;
}
// normalised lane pairs -> the two CBs' stored boundary metrics (offset form,
// as pack_norm writes them)
__device__ __forceinline__ void store_lanes(unsigned v[8], uint4* dA, uint4* dB) {
  norm_p(v);
  unsigned x[8];
#pragma unroll
  for (int s = 0; s < 8; s++) x[s] = v[s] ^ 0x80008000u;
  *dA = make_uint4(prmt(x[0], x[1], 0x5410u), prmt(x[2], x[3], 0x5410u), prmt(x[4], x[5], 0x5410u),
                   prmt(x[6], x[7], 0x5410u));
  *dB = make_uint4(prmt(x[0], x[1], 0x7632u), prmt(x[2], x[3], 0x7632u), prmt(x[4], x[5], 0x7632u),
                   prmt(x[6], x[7], 0x7632u));
}

struct WinP {
  const uint16_t* __restrict__ sys;  // [transposed index]: sys of A | sys of B << 8
  const uint16_t* __restrict__ par;  // [window index]: the pass's parity LLRs, A | B << 8
  uint32_t* ext;                     // [transposed index]: a-priori of A | of B << 16
  uint32_t* hardA;
  uint32_t* hardB;
  const uint4* __restrict__ qt;      // interleaved-pass address groups (DEC 1)
  const uint2* __restrict__ qq;      // their natural positions
  int P, p, len, pad, ng;            // ng: groups of 4 steps in the table (incl. 2 zero groups)
};

template <int DEC>
__device__ __forceinline__ void load_step_p(const WinP& w, int j, int tq, unsigned& S,
                                            unsigned& L, int& t) {
  const int idx = j * w.P + w.p;
  t = DEC == 0 ? idx : tq;
  S = __vadd2(sext8x2(w.sys[t]), w.ext[t]);
  L = sext8x2(w.par[idx]);
}

__device__ __forceinline__ int comp8(const uint4& g0, const uint4& g1, int jj) {
  return comp4(jj < 4 ? g0 : g1, jj & 3);
}
__device__ __forceinline__ int comp8q(const uint2& q0, const uint2& q1, int jj) {
  return comp2(jj < 4 ? q0 : q1, jj & 3);
}

// Backward processing of sub-window [j0, j0 + slen) of the pair: forward
// metrics recomputed from the checkpoint, then Lambda / Le / beta walking
// back.  HM: hard decisions of both lanes (DEC 1).
template <int DEC, bool FULL, int HM>
__device__ __forceinline__ void sub_window_back_p(const WinP& w, const uint4* ck, int j0, int slen,
                                                  uint4 g0, uint4 g1, uint2 q0, uint2 q1,
                                                  unsigned b[8], unsigned& mx, unsigned& mn) {
  unsigned A[kSubP][8];
  unsigned Sv[kSubP], Lv[kSubP];
  int Tv[kSubP];
  unsigned vprev = 0u;
  {
    const uint4 c0 = ck[0], c1 = ck[1];
    A[0][0] = c0.x; A[0][1] = c0.y; A[0][2] = c0.z; A[0][3] = c0.w;
    A[0][4] = c1.x; A[0][5] = c1.y; A[0][6] = c1.z; A[0][7] = c1.w;
  }
#pragma unroll
  for (int jj = 0; jj < kSubP; jj++) {
    if (FULL || jj < slen) {
      load_step_p<DEC>(w, j0 + jj, DEC ? comp8(g0, g1, jj) : 0, Sv[jj], Lv[jj], Tv[jj]);
      if (jj + 1 < kSubP && (FULL || jj + 1 < slen)) alpha_step_p(A[jj], A[jj + 1], Sv[jj], Lv[jj]);
    }
  }
#pragma unroll
  for (int jj = kSubP - 1; jj >= 0; jj--) {
    if (FULL || jj < slen) {
      const unsigned d = app_step_p(A[jj], b, Lv[jj]);
      const int lo = lane_lo(d), hi = lane_hi(d);
      const unsigned v = pack_lanes(scale_ext(lo), scale_ext(hi));
      if (jj & 1) {
        vprev = v;
      } else {
        mx = __vimax3_s16x2(mx, vprev, v);
        mn = __vimin3_s16x2(mn, vprev, v);
      }
      w.ext[Tv[jj]] = v;
      if (DEC == 1 && HM) {  // ORs a zero where Lambda >= 0
        const unsigned lam = __vadd2(Sv[jj], d);
        const int q = comp8q(q0, q1, jj) + w.pad;
        const unsigned bit = 31u - (unsigned)(q & 31);
        atomicOr(&w.hardA[q >> 5], ((lam >> 15) & 1u) << bit);
        atomicOr(&w.hardB[q >> 5], (lam >> 31) << bit);
      }
      beta_step_p(b, Sv[jj], Lv[jj]);
    }
  }
  norm_p(b);
}

// Both recursions of window p for the pair (start metrics a, b as lane
// pairs, normalised).  Writes the checkpoints (thread-private ck), the
// extrinsics, the hard decisions (HM), the boundary metrics of both CBs and
// the packed max / min of the extrinsics written.
template <int DEC, int HM>
__device__ __forceinline__ void window_pass_p(const WinP& w, uint4* ck, unsigned a[8], unsigned b[8],
                                              uint4* seedA_A, uint4* seedA_B, uint4* seedB_A,
                                              uint4* seedB_B, unsigned& mx, unsigned& mn,
                                              uint4 pf0, uint4 pf1) {
  const int P = w.P, p = w.p, len = w.len;
  const uint4* __restrict__ tq = DEC ? w.qt + p : nullptr;  // group g at tq[g * P]
  const int nsub = (len + kSubP - 1) / kSubP;
  const int glast = w.ng - 1;
  // ---- forward, normalised and checkpointed every kSubP steps
  uint4 g0 = pf0, g1 = pf1;
#pragma unroll 1
  for (int sw = 0; sw < nsub; sw++) {
    norm_p(a);
    ck[2 * sw] = make_uint4(a[0], a[1], a[2], a[3]);
    ck[2 * sw + 1] = make_uint4(a[4], a[5], a[6], a[7]);
    const uint4 c0 = g0, c1 = g1;
    if (DEC) {  // the next sub-window's two groups, fetched one sub-window ahead
      g0 = __ldg(tq + min(2 * sw + 2, glast) * P);
      g1 = __ldg(tq + min(2 * sw + 3, glast) * P);
    }
    const int j0 = kSubP * sw;
    if (j0 + kSubP <= len) {
#pragma unroll
      for (int jj = 0; jj < kSubP; jj += 2) {
        unsigned S, L, o[8];
        int t;
        load_step_p<DEC>(w, j0 + jj, DEC ? comp8(c0, c1, jj) : 0, S, L, t);
        alpha_step_p(a, o, S, L);
        load_step_p<DEC>(w, j0 + jj + 1, DEC ? comp8(c0, c1, jj + 1) : 0, S, L, t);
        alpha_step_p(o, a, S, L);
      }
    } else {
      for (int j = j0; j < len; j++) {
        unsigned S, L, o[8];
        int t;
        load_step_p<DEC>(w, j, DEC ? comp8(c0, c1, j - j0) : 0, S, L, t);
        alpha_step_p(a, o, S, L);
#pragma unroll
        for (int s = 0; s < 8; s++) a[s] = o[s];
      }
    }
  }
  if (p + 1 < P) store_lanes(a, seedA_A + p + 1, seedA_B + p + 1);
  // ---- backward, one sub-window at a time from the end
  int sw = nsub - 1;
  uint4 t0 = make_uint4(0u, 0u, 0u, 0u), t1 = t0;
  uint2 n0 = make_uint2(0u, 0u), n1 = n0;
  if (DEC) {
    t0 = __ldg(tq + (2 * sw) * P);
    t1 = __ldg(tq + (2 * sw + 1) * P);
    if (HM) {
      n0 = __ldg(w.qq + (2 * sw) * P + p);
      n1 = __ldg(w.qq + (2 * sw + 1) * P + p);
    }
  }
  const int last_len = len - kSubP * sw;
  if (last_len < kSubP) {
    const uint4 c0 = t0, c1 = t1;
    const uint2 m0 = n0, m1 = n1;
    if (DEC) {
      const int gs = 2 * max(sw - 1, 0);
      t0 = __ldg(tq + gs * P);
      t1 = __ldg(tq + (gs + 1) * P);
      if (HM) {
        n0 = __ldg(w.qq + gs * P + p);
        n1 = __ldg(w.qq + (gs + 1) * P + p);
      }
    }
    sub_window_back_p<DEC, false, HM>(w, ck + 2 * sw, kSubP * sw, last_len, c0, c1, m0, m1, b, mx,
                                      mn);
    sw--;
  }
#pragma unroll 1
  for (; sw >= 0; sw--) {
    const uint4 c0 = t0, c1 = t1;
    const uint2 m0 = n0, m1 = n1;
    if (DEC) {
      const int gs = 2 * max(sw - 1, 0);
      t0 = __ldg(tq + gs * P);
      t1 = __ldg(tq + (gs + 1) * P);
      if (HM) {
        n0 = __ldg(w.qq + gs * P + p);
        n1 = __ldg(w.qq + (gs + 1) * P + p);
      }
    }
    sub_window_back_p<DEC, true, HM>(w, ck + 2 * sw, kSubP * sw, kSubP, c0, c1, m0, m1, b, mx, mn);
  }
  if (p > 0) store_lanes(b, seedB_A + p - 1, seedB_B + p - 1);
}

// Start metrics of window p of one CB for a pass, as siso_pass reads them
// but kept packed (offset form, pack8 layout): alpha from the known start,
// zeros or the stored seed; beta likewise (the tail steps follow after the
// barrier).  Clears the flag this pass writes and, for a checked pass, the
// hard decisions.  Runs before the pass's barrier: other threads overwrite
// the seeds during the pass.
__device__ __forceinline__ uint4 start_init(int p, int first_p, bool first, const uint4* seed) {
  const unsigned z = (unsigned)OFF | ((unsigned)OFF << 16);
  if (p == first_p) {
    const unsigned m = (unsigned)MINF_OFF | ((unsigned)MINF_OFF << 16);
    return make_uint4((unsigned)OFF | ((unsigned)MINF_OFF << 16), m, m, m);
  }
  if (first) return make_uint4(z, z, z, z);
  return seed[p];
}
template <int DEC>
__device__ __forceinline__ void pass_start_p(const CbSlot& sl, int K, int P, int p, bool first,
                                             bool hard, uint4& a, uint4& b, int& m_in) {
  a = start_init(p, 0, first, sl.seed + DEC * P);
  b = start_init(p, P - 1, first, sl.seed + (2 + DEC) * P);
  m_in = sl.flags[5 - DEC];
  if (p == 0) sl.flags[4 + DEC] = 0;  // written by this pass after the barrier
  if (DEC == 1 && hard) {
    const int nwords = (K + 31) / 32;
    for (int w = p; w < nwords; w += P) sl.hard[w] = 0u;
  }
}

// packed start metrics (offset form) -> int[8] with the tail steps of the
// last window applied
template <int DEC>
__device__ __forceinline__ void lane_start(uint4 pa, uint4 pb, const int8_t* tail, bool last,
                                           int a[8], int b[8]) {
  unpack8(pa, a);
  unpack8(pb, b);
  if (last) {
    const int8_t* t = tail + (DEC ? 6 : 0);
#pragma unroll
    for (int j = 2; j >= 0; j--) beta_tail_step(b, t[2 * j], t[2 * j + 1]);
  }
}

// One lane of a pair slot through the one-CB code (stride-2 view): the
// fallback when pair_fast fails, and the path of a CB whose partner stopped.
// pa, pb: the lane's packed start metrics.  Not inlined: the pass gets its
// own register allocation, apart from the item loop around it.
template <int DEC>
__device__ __noinline__ void lane_pass(const CbDesc* __restrict__ dp, uint8_t* base, int L, int p,
                                       bool hard, uint4 pa, uint4 pb, int m_in, uint4 pf0,
                                       uint4 pf1) {
  const int K = dp->K, P = dp->P, W = dp->W;
  const CbSlot sl = make_pair_slot(base, K, P, W, L);
  int a[8], b[8];
  lane_start<DEC>(pa, pb, sl.tail, p == P - 1, a, b);
  Win w;
  w.sys = sl.sys;
  w.par = DEC ? sl.par2 : sl.par1;
  w.ext = sl.ext;
  w.hard = sl.hard;
  w.hard_on = hard;
  w.r4 = false;
  w.qt = dp->qt;
  w.qq = dp->qq;
  w.K = K;
  w.P = P;
  w.W = W;
  w.divM = dp->divM;
  w.divS = dp->divS;
  w.f2x2 = dp->f2x2;
  w.p = p;
  w.lo = p * W;
  w.len = min(W, K - w.lo);
  w.pad = ((K + 31) / 32) * 32 - K;
  uint4* ck = sl.ck + p * sl.ck_stride;
  uint4* seedA = sl.seed + DEC * P;
  uint4* seedB = sl.seed + (2 + DEC) * P;
  int mx = 0, mn = 0;
  if (window_fast(a, b, 254 + m_in)) {
    window_pass<DEC, false, false, true, 2>(w, dp, ck, seedA, seedB, a, b, mx, mn, pf0, pf1);
  } else {
    window_pass<DEC, true, false, true, 2>(w, dp, ck, seedA, seedB, a, b, mx, mn, pf0, pf1);
    atomicAdd(&sl.flags[7], 1);
  }
  atomicMax(&sl.flags[4 + DEC], max(mx, -mn));
}

// The pass of window p of both lanes on 16-bit lanes (pair_fast holds for
// both).  paX / pbX: packed start metrics of lane X (tail steps done).  Not
// inlined: inside the item loop the inlined pass spills (measured slower).
template <int DEC, int HM>
__device__ __noinline__ void pair_pass(const CbDesc* __restrict__ dA, uint8_t* base, int p,
                                       uint4 paA, uint4 pbA, uint4 paB, uint4 pbB, uint4 pf0,
                                       uint4 pf1) {
  const int K = dA->K, P = dA->P, W = dA->W;
  const PairLayout l = pair_layout(K, P, W);
  WinP w;
  w.sys = (const uint16_t*)base;
  w.par = (const uint16_t*)(base + (DEC ? 4 : 2) * W * P);
  w.ext = (uint32_t*)(base + l.o_ext);
  w.hardA = (uint32_t*)(base + l.o_hard);
  w.hardB = (uint32_t*)(base + l.o_hard + l.hard_bytes);
  w.qt = dA->qt;
  w.qq = dA->qq;
  w.P = P;
  w.p = p;
  w.len = min(W, K - p * W);
  w.pad = ((K + 31) / 32) * 32 - K;
  w.ng = (W + kSub - 1) / kSub + 2;
  unsigned a[8], b[8];
  a[0] = prmt(paA.x, paB.x, 0x5410u); a[1] = prmt(paA.x, paB.x, 0x7632u);
  a[2] = prmt(paA.y, paB.y, 0x5410u); a[3] = prmt(paA.y, paB.y, 0x7632u);
  a[4] = prmt(paA.z, paB.z, 0x5410u); a[5] = prmt(paA.z, paB.z, 0x7632u);
  a[6] = prmt(paA.w, paB.w, 0x5410u); a[7] = prmt(paA.w, paB.w, 0x7632u);
  b[0] = prmt(pbA.x, pbB.x, 0x5410u); b[1] = prmt(pbA.x, pbB.x, 0x7632u);
  b[2] = prmt(pbA.y, pbB.y, 0x5410u); b[3] = prmt(pbA.y, pbB.y, 0x7632u);
  b[4] = prmt(pbA.z, pbB.z, 0x5410u); b[5] = prmt(pbA.z, pbB.z, 0x7632u);
  b[6] = prmt(pbA.w, pbB.w, 0x5410u); b[7] = prmt(pbA.w, pbB.w, 0x7632u);
#pragma unroll
  for (int s = 0; s < 8; s++) {
    a[s] ^= 0x80008000u;  // offset form -> signed lanes
    b[s] ^= 0x80008000u;
  }
  uint4* ck = (uint4*)(base + l.o_ck + p * l.ck_per_thread);
  uint4* sAa = (uint4*)(base + l.o_seed) + DEC * P;
  uint4* sBa = (uint4*)(base + l.o_seed + l.seed_bytes) + DEC * P;
  unsigned mx = 0u, mn = 0u;
  window_pass_p<DEC, HM>(w, ck, a, b, sAa, sBa, sAa + 2 * P, sBa + 2 * P, mx, mn, pf0, pf1);
  int* flA = (int*)(base + l.o_flags);
  atomicMax(&flA[4 + DEC], max(lane_lo(mx), -lane_lo(mn)));
  atomicMax(&flA[16 + 4 + DEC], max(lane_hi(mx), -lane_hi(mn)));  // lane B: 64 bytes on
}

// One SISO pass of window p of both CBs of a pair item.  runA / runB: the
// CB still iterates; hardA / hardB: its hard decisions are used (a CRC check
// follows).  All threads of the CTA call it (it contains barriers).
template <int DEC>
__device__ __forceinline__ void siso_pass_pair(const CbDesc* __restrict__ dA,
                                               const CbDesc* __restrict__ dB, uint8_t* base, int p,
                                               bool runA, bool runB, bool first, bool hardA,
                                               bool hardB) {
  const int K = dA->K, P = dA->P, W = dA->W;
  uint4 paA, pbA, paB, pbB;
  int mA = 0, mB = 0;
  uint4 pf0 = make_uint4(0u, 0u, 0u, 0u), pf1 = pf0;
  if (DEC == 1 && (runA || runB)) {  // the first two address groups, fetched across the barrier
    pf0 = __ldg(dA->qt + p);
    pf1 = __ldg(dA->qt + P + p);
  }
  if (runA) pass_start_p<DEC>(make_pair_slot(base, K, P, W, 0), K, P, p, first, hardA, paA, pbA, mA);
  if (runB) pass_start_p<DEC>(make_pair_slot(base, K, P, W, 1), K, P, p, first, hardB, paB, pbB, mB);
  __syncthreads();
  if (runA && runB) {
    const bool last = p == P - 1;
    const int len = min(W, K - p * W);
    const int8_t* tailA = (const int8_t*)(base + pair_layout(K, P, W).o_tail);
    int a[8], b[8];
    lane_start<DEC>(paA, pbA, tailA, last, a, b);
    bool ok = pair_fast(a, b, 254 + mA, len);
    const uint4 tA = pack8(b);
    lane_start<DEC>(paB, pbB, tailA + 16, last, a, b);
    ok = ok && pair_fast(a, b, 254 + mB, len);
    if (ok) {
      if (DEC == 1 && (hardA || hardB))
        pair_pass<DEC, 1>(dA, base, p, paA, tA, paB, pack8(b), pf0, pf1);
      else
        pair_pass<DEC, 0>(dA, base, p, paA, tA, paB, pack8(b), pf0, pf1);
    } else {
      lane_pass<DEC>(dA, base, 0, p, hardA, paA, pbA, mA, pf0, pf1);
      lane_pass<DEC>(dB, base, 1, p, hardB, paB, pbB, mB, pf0, pf1);
    }
  } else if (runA) {
    lane_pass<DEC>(dA, base, 0, p, hardA, paA, pbA, mA, pf0, pf1);
  } else if (runB) {
    lane_pass<DEC>(dB, base, 1, p, hardB, paB, pbB, mB, pf0, pf1);
  }
  __syncthreads();
}

// The GPU's global nanosecond timer (the performance captor's clock).
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Timestamp k of the CBs cb0 .. cb0 + n - 1 (thread 0 of the item).
__device__ __forceinline__ void stamp(const DecParams& prm, int cb0, int n, int k, uint64_t t) {
  if (prm.cb_time)
    for (int g = 0; g < n; g++) prm.cb_time[4 * (cb0 + g) + k] = t;
}

// Stop rule of one CB after iteration it (thread p = 0 of the CB, after the
// CRC shares of a checked iteration were combined in fl[2]): CRC pass, the
// mutual-information rule, the iteration limit, or a purge of its TB.
__device__ __forceinline__ void stop_rule(const DecParams& prm, const CbDesc* __restrict__ dp,
                                          int* fl, int it, int my_max, bool check,
                                          int* s_remaining) {
  const bool ok = check && fl[2] == 0;
  fl[2] = 0;
  const int tb = dp->tb;
  bool stop = ok || it == my_max;
  if (dp->early_stop == 2) {
    // mutual-information rule: stop once the mean changed by at most
    // 2^-10 bit (from iteration 2); the CRC decides success
    const int S = fl[8], dS = abs(S - fl[9]);
    stop = (it >= 2 && (long long)dS * 1024 <= (long long)dp->K * 65536) || it == my_max;
    fl[9] = S;
    fl[8] = 0;
  }
  if (stop) {
    fl[0] = 1;
    fl[1] = ok ? it : my_max + 1;
    fl[10] = it;
    atomicSub(s_remaining, 1);
    // a failed CB fails its TB: flag it now (the TB CRC step flags it
    // again) so that purging CBs of the TB can stop
    if (!ok && dp->crc_b) atomicOr(&prm.tb_crc[2 * tb + 1], 1u);
  } else if (dp->purge && *(volatile uint32_t*)&prm.tb_crc[2 * tb + 1] != 0u) {
    fl[0] = 1;
    fl[1] = 0;
    fl[6] = 1;
    fl[10] = it;
    atomicSub(s_remaining, 1);
  }
}

// The hard-decision CRC share (and, for stop rule 2, the mutual-information
// share) of thread p after a checked iteration.
__device__ __forceinline__ void check_share(const DecParams& prm, const CbDesc& d,
                                            const CbSlot& sl, int p, const uint32_t* tabA,
                                            const uint32_t* tabB, const int* mi_tab) {
  const uint32_t r = crc_share(d, sl, p, d.crc_b ? tabB : tabA, d.crc_b ? GB : GA,
                               d.crc_b ? prm.xpowB : prm.xpowA, 0);
  if (r) atomicXor((unsigned*)&sl.flags[2], r);
  if (d.early_stop == 2) {
    // stop rule 2: mutual information of the a-priori LLRs the next
    // iteration would use (the scaled extrinsics of decoder 2, held in the
    // ext array; its padding entries are 0 and add nothing)
    int mi = 0;
    for (int t = p; t < d.W * d.P; t += d.P)
      mi += 65536 - mi_tab[min(abs((int)sl.ext[sl.str * t]), kMiTable - 1)];
    atomicAdd(&sl.flags[8], mi);
  }
}

// Debug copy of a CB's de-rate-matched streams (all threads of the CTA).
__device__ void debug_streams(const DecParams& prm, const CbDesc& dg, const CbSlot& sg, int tid,
                              int nthr) {
  const int D = dg.K + 4;
  int8_t* out = prm.dbg_d + 3 * (int64_t)dg.dbg_off;
  for (int k = tid; k < D; k += nthr) {
    if (k < dg.K) {
      const int t = sg.str * tr_idx(k, dg);
      out[k] = sg.sys[t];
      out[D + k] = sg.par1[t];
      out[2 * D + k] = sg.par2[t];
    } else {
      out[k] = sg.tail[3 * (k - dg.K)];
      out[D + k] = sg.tail[3 * (k - dg.K) + 1];
      out[2 * D + k] = sg.tail[3 * (k - dg.K) + 2];
    }
  }
}

// Phase 2, part 1 (thread p of the CB): payload bytes, the CB's CRC24A
// contribution to its TB, debug copies of the final extrinsic and hard bits.
__device__ void finish_share(const DecParams& prm, const CbDesc& d, const CbSlot& sl, int p,
                             const uint32_t* tabA) {
  const bool purged = sl.flags[6] != 0;
  if (purged) return;
  const TbDesc tb = prm.tbs[d.tb];
  const int nw = (d.K + 31) / 32;
  const int pad = nw * 32 - d.K;
  const int nbytes = d.pay_bits / 8;
  uint8_t* out = prm.out + tb.out_off;
  for (int m = p; m < nbytes; m += d.P) {
    const int tbbit = d.pay_off + 8 * m;
    if (tbbit >= tb.A) break;
    const int q = pad + d.F + 8 * m;
    out[tbbit >> 3] = (uint8_t)(sl.hard[q >> 5] >> (24 - (q & 31)));
  }
  if (d.crc_b) {
    const uint32_t r = crc_share(d, sl, p, tabA, GA, prm.xpowA, 1);
    if (r) atomicXor((unsigned*)&sl.flags[3], r);
  }
  if (prm.dbg_ext) {
    for (int k = p; k < d.K; k += d.P) {
      prm.dbg_ext[d.dbg_off + k] = sl.ext[sl.str * tr_idx(k, d)];
      const int q = pad + k;
      prm.dbg_hard[d.dbg_off + k] = (uint8_t)((sl.hard[q >> 5] >> (31 - (q & 31))) & 1u);
    }
  }
}

// Phase 2, part 2 (thread p = 0 of the CB, after a barrier): per-CB results;
// a single-CB TB's result; otherwise the CB's contribution to its TB's
// CRC24A (by linearity) and failure word, which the host reads after the
// launch.
__device__ void finish_cb(const DecParams& prm, const CbDesc& d, const CbSlot& sl,
                          int sorted_idx, const uint32_t* tabA) {
  const bool purged = sl.flags[6] != 0;
  const bool cb_ok = !purged && sl.flags[1] <= d.max_iter;
  prm.cb_iters[sorted_idx] = (uint8_t)sl.flags[1];
  if (prm.cb_runs) prm.cb_runs[sorted_idx] = (uint8_t)sl.flags[10];
  prm.cb_ok[sorted_idx] = cb_ok ? 1 : 0;
  if (prm.tb_sat && sl.flags[7]) atomicAdd(&prm.tb_sat[d.tb], (unsigned)sl.flags[7]);
  const TbDesc tb = prm.tbs[d.tb];
  if (tb.C == 1) {
    prm.tb_ok[d.tb] = cb_ok ? 1 : 0;
  } else {
    uint32_t contrib = (uint32_t)sl.flags[3];
    // shift past the TB bits that follow this CB's payload: 32 a + 8 b
    const int na = d.n_after >> 5, nb = (d.n_after >> 3) & 3;
    if (na) contrib = gf_mulmod(contrib, __ldg(&prm.xpowA[na]), GA);
    for (int k = 0; k < nb; k++)
      contrib = ((contrib << 8) & 0xFFFFFFu) ^ tabA[(contrib >> 16) & 0xFFu];
    // fire-and-forget: the host decides the TB from the two words once the
    // launch is complete (TB CRC24A zero and no failed CB)
    atomicXor(&prm.tb_crc[2 * d.tb], contrib);
    if (!cb_ok) atomicOr(&prm.tb_crc[2 * d.tb + 1], 1u);
  }
}

// A pair item: two CBs of equal (K, P) on threads 0..P-1, one pair slot.
__device__ __forceinline__ void run_pair_item(const DecParams& prm, const WorkItem& wi, uint8_t* slots, int tid,
                              const uint32_t* tabA, const uint32_t* tabB, const int* mi_tab,
                              int* s_remaining, int* s_maxit, Bulk& bk) {
  const CbDesc* cbs = prm.cbs + wi.cb0;
  const CbDesc* dA = cbs;
  const CbDesc* dB = cbs + 1;
  const int K = dA->K, P = dA->P, W = dA->W;
  const bool mine = tid < P;
  const int p = tid;
  const CbSlot sA = make_pair_slot(slots, K, P, W, 0);
  const CbSlot sB = make_pair_slot(slots, K, P, W, 1);
  if (tid == 0) stamp(prm, wi.cb0, 2, 0, gtime());
  // ---- phase 0: de-rate-matching of both CBs, one after the other (they
  // share the staging area, and the extrinsic area holds the streamed map),
  // then the pair's extrinsics cleared
  const PairLayout l = pair_layout(K, P, W);
  uint8_t* const ext_area = slots + l.o_ext;
  const int ext_bytes = align16(4 * W * P);
  // When both CBs use the same map (same K, P, F) and their LLRs fit the
  // staging area together -- B's from the first 16-byte boundary after A's
  // -- one pass over the map de-rate-matches both.
  const int offB = (dA->E + 30) & ~15;
  if (dA->dm != nullptr && dA->dm == dB->dm && ext_bytes >= 2048 &&
      offB + dB->E + 15 <= sA.stage_cap) {
    CbSlot sB2 = sB;
    sB2.stage = sA.stage + offB;
    sB2.stage_cap = sA.stage_cap - offB;
    stage_llrs(*dA, sA, prm.llr, tid, kThreads);
    stage_llrs(*dB, sB2, prm.llr, tid, kThreads);
    __syncthreads();
    derm_cb<2>(*dA, sA, llr_src(*dA, sA, prm.llr), prm.soft, tid, kThreads, ext_area, ext_bytes,
               bk, dB, &sB, llr_src(*dB, sB2, prm.llr));
  } else {
    stage_llrs(*dA, sA, prm.llr, tid, kThreads);
    __syncthreads();
    derm_cb<2>(*dA, sA, llr_src(*dA, sA, prm.llr), prm.soft, tid, kThreads, ext_area, ext_bytes,
               bk);
    __syncthreads();
    stage_llrs(*dB, sB, prm.llr, tid, kThreads);
    __syncthreads();
    derm_cb<2>(*dB, sB, llr_src(*dB, sB, prm.llr), prm.soft, tid, kThreads, ext_area, ext_bytes,
               bk);
  }
  __syncthreads();
  {
    uint4* e16 = (uint4*)ext_area;
    for (int k = tid; k < ext_bytes / 16; k += kThreads) e16[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    *s_remaining = 2;
    *s_maxit = max((int)dA->max_iter, (int)dB->max_iter);
  }
  __syncthreads();
  if (tid == 0) stamp(prm, wi.cb0, 2, 1, gtime());
  if (prm.dbg_d) {
    debug_streams(prm, *dA, sA, tid, kThreads);
    debug_streams(prm, *dB, sB, tid, kThreads);
  }
  // ---- phase 1: turbo iterations of both CBs
  const int maxit = *s_maxit;
  for (int it = 1; it <= maxit; it++) {
    const int maxA = dA->max_iter, maxB = dB->max_iter;
    const bool runA = mine && sA.flags[0] == 0 && it <= maxA;
    const bool runB = mine && sB.flags[0] == 0 && it <= maxB;
    const bool first = (it == 1);
    siso_pass_pair<0>(dA, dB, slots, p, runA, runB, first, false, false);
    const bool checkA = runA && (dA->early_stop || it == maxA);
    const bool checkB = runB && (dB->early_stop || it == maxB);
    siso_pass_pair<1>(dA, dB, slots, p, runA, runB, first, checkA, checkB);
    if (checkA) check_share(prm, *dA, sA, p, tabA, tabB, mi_tab);
    if (checkB) check_share(prm, *dB, sB, p, tabA, tabB, mi_tab);
    __syncthreads();
    if (p == 0) {
      if (runA) stop_rule(prm, dA, sA.flags, it, maxA, checkA, s_remaining);
      if (runB) stop_rule(prm, dB, sB.flags, it, maxB, checkB, s_remaining);
    }
    __syncthreads();
    if (*s_remaining == 0) break;
  }
  // ---- phase 2: results of both CBs
  if (tid == 0) stamp(prm, wi.cb0, 2, 2, gtime());
  if (mine) {
    finish_share(prm, *dA, sA, p, tabA);
    finish_share(prm, *dB, sB, p, tabA);
  }
  __syncthreads();
  // the two CBs' results on threads of different warps, concurrently
  if (tid == 0) finish_cb(prm, *dA, sA, wi.cb0, tabA);
  if (tid == 32) finish_cb(prm, *dB, sB, wi.cb0 + 1, tabA);
  if (prm.cb_time) {
    __syncthreads();
    if (tid == 0) stamp(prm, wi.cb0, 2, 3, gtime());
  }
}

// A work item of one or more CBs, P threads each (windows across threads).
template <bool R4, bool QT>
__device__ __forceinline__ void run_single_item(const DecParams& prm, const WorkItem& wi,
                                                uint8_t* slots, int tid, const uint32_t* tabA,
                                                const uint32_t* tabB, const int* mi_tab,
                                                int* s_remaining, int* s_maxit, Bulk& bk) {
  const CbDesc* cbs = prm.cbs + wi.cb0;
  const int P = cbs[0].P;
  const int G = wi.n;
  const int mycb = tid / P;
  const int p = tid - mycb * P;
  const bool mine = mycb < G;
  const CbDesc* dp = cbs + (mine ? mycb : 0);
  if (tid == 0) stamp(prm, wi.cb0, G, 0, gtime());

  // ---- phase 0: de-rate-matching of every CB of the item (LLRs staged
  // in shared memory first)
  for (int g = 0; g < G; g++) {
    const CbDesc& dg = cbs[g];
    const CbSlot sg = make_slot(slots + g * wi.smem_per_cb, dg.K, dg.P, dg.W);
    stage_llrs(dg, sg, prm.llr, tid, kThreads);
  }
  __syncthreads();
  for (int g = 0; g < G; g++) {
    const CbDesc& dg = cbs[g];
    const CbSlot sg = make_slot(slots + g * wi.smem_per_cb, dg.K, dg.P, dg.W);
    derm_cb<1>(dg, sg, llr_src(dg, sg, prm.llr), prm.soft, tid, kThreads, (uint8_t*)sg.ext,
               align16(2 * dg.W * dg.P), bk);
  }
  if (tid == 0) {
    *s_remaining = G;
    int mx = 0;
    for (int g = 0; g < G; g++) mx = max(mx, (int)cbs[g].max_iter);
    *s_maxit = mx;
  }
  __syncthreads();
  if (tid == 0) stamp(prm, wi.cb0, G, 1, gtime());
  uint8_t* mybase = slots + (mine ? mycb : 0) * wi.smem_per_cb;
  int* const fl = make_slot(mybase, dp->K, dp->P, dp->W).flags;
  if (prm.dbg_d) {
    for (int g = 0; g < G; g++) {
      const CbDesc& dg = cbs[g];
      debug_streams(prm, dg, make_slot(slots + g * wi.smem_per_cb, dg.K, dg.P, dg.W), tid,
                    kThreads);
    }
  }

  // ---- phase 1: turbo iterations (only the flags pointer stays live
  // across the SISO passes; descriptor fields are re-read when needed)
  const int maxit = *s_maxit;
  for (int it = 1; it <= maxit; it++) {
    const int my_max = mine ? (int)dp->max_iter : 0;
    const bool run = mine && fl[0] == 0 && it <= my_max;
    const bool first = (it == 1);
    siso_pass<0, R4, QT>(dp, mybase, p, run, first, false);
    const bool check = run && (dp->early_stop || it == my_max);
    siso_pass<1, R4, QT>(dp, mybase, p, run, first, check);
    if (check) {
      const CbDesc& d = *dp;
      check_share(prm, d, make_slot(mybase, d.K, d.P, d.W), p, tabA, tabB, mi_tab);
    }
    __syncthreads();
    if (run && p == 0) stop_rule(prm, dp, fl, it, my_max, check, s_remaining);
    __syncthreads();
    if (*s_remaining == 0) break;
  }

  // ---- phase 2: results, payload bytes, TB CRC, debug copies
  if (tid == 0) stamp(prm, wi.cb0, G, 2, gtime());
  const CbDesc d = *dp;
  const CbSlot sl = make_slot(mybase, d.K, d.P, d.W);
  if (mine) finish_share(prm, d, sl, p, tabA);
  __syncthreads();
  if (mine && p == 0) finish_cb(prm, d, sl, wi.cb0 + mycb, tabA);
  if (prm.cb_time) {
    __syncthreads();
    if (tid == 0) stamp(prm, wi.cb0, G, 3, gtime());
  }
}
// The same, not inlined: the pair kernel runs one-CB items rarely, and the
// pair path keeps the kernel's registers to itself.
template <bool R4, bool QT>
__device__ __noinline__ void run_single_item_call(const DecParams& prm, const WorkItem& wi,
                                                  uint8_t* slots, int tid, const uint32_t* tabA,
                                                  const uint32_t* tabB, const int* mi_tab,
                                                  int* s_remaining, int* s_maxit, Bulk& bk) {
  run_single_item<R4, QT>(prm, wi, slots, tid, tabA, tabB, mi_tab, s_remaining, s_maxit, bk);
}

// The launch gate (crnt_plan_launch_gated): thread 0 of a CTA polls the
// ready word with system-scope acquire loads until it is non-zero -- the
// LLRs written before it are then visible to this CTA, whose other threads
// pass the barrier after it -- or until gate_us microseconds of %globaltimer
// (and at most 2^24 polls of at least a microsecond each) have passed.
// Expiry is recorded once in state->err, where later CTAs see it and stop
// without waiting again.  Returns 0 when open, 1 when expired.
__device__ __noinline__ int gate_wait(const DecParams& prm) {
  volatile int32_t* err = &prm.state->err;
  if (*err) return 1;
  const uint64_t t0 = gtime(), limit = (uint64_t)prm.gate_us * 1000ull;
  for (uint32_t it = 0; it < (1u << 24); it++) {
    uint32_t v;
    asm volatile("ld.acquire.sys.u32 %0, [%1];" : "=r"(v) : "l"(prm.gate) : "memory");
    if (v) return 0;
    if (*err) return 1;
    if (gtime() - t0 > limit) break;
    __nanosleep(1000);
  }
  atomicCAS(&prm.state->err, 0, 1);
  return 1;
}

// R4 = false: the radix-2 kernel; R4 = true adds the radix-4 forward
// recursion for CBs that select it (a separate instantiation, so the radix-2
// kernel's code is not affected by the option).  QT: every CB carries an
// address table for its interleaved pass (else the addresses are computed).
// PAIR: the batch has CB-pair items (needs QT); the kernel is then built for
// two CTAs per SM (more registers per thread for the packed path).
template <bool R4, bool QT, bool PAIR>
__global__ void __launch_bounds__(kThreads, PAIR ? kCtasPerSmPair : kCtasPerSm)
    decode_kernel(DecParams prm) {
  __shared__ int s_item;
  __shared__ int s_remaining;
  __shared__ int s_maxit;
  __shared__ __align__(8) uint64_t s_bar[2];
  uint32_t* tabA = (uint32_t*)smem;
  uint32_t* tabB = tabA + 256;
  int* mi_tab = (int*)(smem + 2048);
  uint8_t* slots = smem + kSmemFixed;
  const int tid = threadIdx.x;

  if (prm.mi_tab)
    for (int i = tid; i < kMiTable; i += kThreads) mi_tab[i] = __ldg(&prm.mi_tab[i]);
  for (int i = tid; i < 512; i += kThreads) {
    const uint32_t g = (i < 256) ? GA : GB;
    uint32_t r = (uint32_t)(i & 255) << 16;
    for (int k = 0; k < 8; k++) r = (r & 0x800000u) ? ((r << 1) ^ g) : (r << 1);
    (i < 256 ? tabA : tabB)[i & 255] = r & 0xFFFFFFu;
  }

  Bulk bk{smem_u32(s_bar), 0u, &prm.state->err};
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bk.bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bk.bar + 8u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (prm.gate) {
    if (tid == 0) s_item = gate_wait(prm);
    __syncthreads();
    if (s_item) return;  // expired: nothing of the batch is decoded
  }
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(&prm.state->head, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= prm.n_items) break;
    const WorkItem wi = prm.items[item];
    if (PAIR && wi.mode == 1) {
      run_pair_item(prm, wi, slots, tid, tabA, tabB, mi_tab, &s_remaining, &s_maxit, bk);
      continue;
    }
    if (PAIR)
      run_single_item_call<R4, QT>(prm, wi, slots, tid, tabA, tabB, mi_tab, &s_remaining,
                                   &s_maxit, bk);
    else
      run_single_item<R4, QT>(prm, wi, slots, tid, tabA, tabB, mi_tab, &s_remaining, &s_maxit,
                              bk);
  }
}

}  // namespace

int decode_max_smem() {
  return (kSmemBudgetPair > kSmemBudget ? kSmemBudgetPair : kSmemBudget) + kSmemFixed;
}

template <bool R4, bool QT, bool PAIR>
cudaError_t set_attr_one() {
  return cudaFuncSetAttribute(decode_kernel<R4, QT, PAIR>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, decode_max_smem());
}
static cudaError_t set_attr() {
  static cudaError_t e = [] {
    cudaError_t r = set_attr_one<false, false, false>();
    if (r == cudaSuccess) r = set_attr_one<false, true, false>();
    if (r == cudaSuccess) r = set_attr_one<true, false, false>();
    if (r == cudaSuccess) r = set_attr_one<true, true, false>();
    if (r == cudaSuccess) r = set_attr_one<false, true, true>();
    if (r == cudaSuccess) r = set_attr_one<true, true, true>();
    return r;
  }();
  return e;
}

template <bool R4, bool QT, bool PAIR>
int occupancy_one(int smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decode_kernel<R4, QT, PAIR>, kThreads,
                                                    smem) != cudaSuccess)
    return 0;
  return n;
}

// Resident CTAs per SM at this dynamic shared memory for the instantiation a
// launch with these flags uses (see launch_decode).
int decode_occupancy(int smem, bool radix4_any, bool qtab_all, bool pair_any) {
  if (set_attr() != cudaSuccess) return 0;
  if (pair_any && qtab_all)
    return radix4_any ? occupancy_one<true, true, true>(smem) : occupancy_one<false, true, true>(smem);
  if (radix4_any)
    return qtab_all ? occupancy_one<true, true, false>(smem) : occupancy_one<true, false, false>(smem);
  return qtab_all ? occupancy_one<false, true, false>(smem) : occupancy_one<false, false, false>(smem);
}

cudaError_t launch_decode(const DecParams& p, int grid, int smem, cudaStream_t s) {
  if (smem > decode_max_smem()) return cudaErrorInvalidValue;
  if (p.pair_any && !p.qtab_all) return cudaErrorInvalidValue;
  if (set_attr() != cudaSuccess) return cudaErrorInvalidValue;
  if (p.pair_any) {
    if (p.radix4_any)
      decode_kernel<true, true, true><<<grid, kThreads, smem, s>>>(p);
    else
      decode_kernel<false, true, true><<<grid, kThreads, smem, s>>>(p);
  } else if (p.radix4_any) {
    if (p.qtab_all)
      decode_kernel<true, true, false><<<grid, kThreads, smem, s>>>(p);
    else
      decode_kernel<true, false, false><<<grid, kThreads, smem, s>>>(p);
  } else {
    if (p.qtab_all)
      decode_kernel<false, true, false><<<grid, kThreads, smem, s>>>(p);
    else
      decode_kernel<false, false, false><<<grid, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace crnt
