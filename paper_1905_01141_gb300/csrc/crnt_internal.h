// crnt_internal.h -- descriptors shared by the host planner and the kernels.
//
// The host planner (crnt_api.cu) turns transport blocks into code-block (CB)
// descriptors and work items; the decode kernel (decode.cu) and the encode
// kernel (encode.cu) consume them.  Nothing here is part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace crnt {

constexpr int kThreads = 128;          // threads per decode CTA
constexpr int kCtasPerSm = 3;          // resident decode CTAs per SM (register-bound)
constexpr int kSmemBudget = 72 * 1024; // dynamic smem per decode CTA (one CB per thread)
constexpr int kMaxP = kThreads;        // windows per SISO pass (one thread each)
constexpr int kSub = 4;                // sub-window length of the alpha recompute
// CB pairs: one thread runs window p of two CBs of equal (K, P) in the two
// 16-bit lanes of its registers.  Kernels that carry pair items hold two
// CTAs per SM (up to 255 registers a thread) of at most kSmemBudgetPair
// bytes each; the pair path checkpoints its forward metrics every kSubP steps.
constexpr int kCtasPerSmPair = 2;
constexpr int kSmemBudgetPair = 110 * 1024;
constexpr int kSubP = 8;
constexpr int kMaxK = 6144;
// Fixed shared memory of a decode CTA ahead of the CB slots: the CRC24A /
// CRC24B byte tables (2 x 256 words) and the mutual-information table (128
// words).
constexpr int kSmemFixed = 2048 + 512;
constexpr int kMiTable = 128;
constexpr int kMaxCb = 16;

// One code block of a batch, fixed at plan time.
struct CbDesc {
  int32_t K, F, E, k0;     // CB size, filler bits, rate-matched length, start
  int32_t P, W;            // windows and window length (W = ceil(K/P))
  int32_t divM, divS;      // q / W == (q * divM) >> divS for 0 <= q < K + 4
  int32_t f1, f2;          // QPP parameters
  int32_t f2x2;            // 2 f2 mod K: step of the QPP first difference
  int32_t f2sub, f2jump;   // 2 kSub f2 and 2 kSub^2 f2 mod K: steps of the
                           // kSub-step QPP differences (sub-window jumps)
  int32_t R, ND, Nv, rank0;     // sub-block rows, dummies, non-NULL count, rank of k0
  uint32_t maskB, mask2;   // column masks of the rank formula (see derm)
  int32_t tb;              // transport block index in the batch
  int32_t r;               // CB index inside the TB
  int64_t llr_off;         // byte offset of the CB's E LLRs in the LLR buffer
  int64_t soft_off;        // byte offset of the CB's Ncb soft buffer, -1 = none
  int32_t pay_bits;        // payload bits in the TB (K - F - L)
  int32_t pay_off;         // TB bit offset of the payload (multiple of 8)
  int32_t n_after;         // TB bits after the payload (for the TB CRC)
  int32_t dbg_off;         // element offset of the CB in debug arrays
  uint8_t crc_b;           // 1: CRC24B per CB (C > 1); 0: CRC24A (C == 1)
  uint8_t max_iter, early_stop, new_data;
  uint8_t purge;           // 1: stop when another CB of the TB has failed
  uint8_t radix4;          // 1: radix-4 forward recursion where the pass is clamp-free
  uint8_t pad0[2];
  const uint4* qt;         // interleaved-pass address table of (K, P), or null:
                           // [ceil(W/kSub) + 2 groups][P windows] x kSub
                           // transposed addresses (the last two groups zero)
  const uint2* qq;         // the same steps' natural positions (uint16, same order)
  const uint32_t* dm;      // de-rate-matching map of (K, P, F), or null:
                           // per circular-buffer rank r < Nv, (position << 16) |
                           // destination (stream s: s W P + transposed index;
                           // tail bit: 3 W P + 3 (d - K) + s)
};

struct TbDesc {
  int64_t out_off;  // byte offset of the TB's A/8 output bytes
  int32_t A, C;
  int32_t cb0;      // index of its first CB in the CB array (TB order)
  int32_t pad0;
};

// A work item: n consecutive CBs (sorted order) of equal K and P, decoded
// together by one CTA.  mode 0: one CB per P threads (n <= kThreads / P);
// mode 1: a CB pair (n = 2) in one pair slot, both CBs on the same P threads.
struct WorkItem {
  int32_t cb0, n;
  int32_t smem_per_cb;  // mode 0: bytes per CB slot; mode 1: bytes of the pair slot
  int32_t mode;
};

// Per-batch device state written by the kernel.
struct DecState {
  int32_t head;       // work-queue head
  int32_t err;        // a bounded wait expired (0 = none): 1 the launch's gate,
                      // 2 a bulk copy into shared memory
};

struct DecParams {
  const CbDesc* cbs;      // sorted by work item
  const TbDesc* tbs;
  const WorkItem* items;
  int32_t n_items, n_cbs, n_tbs;
  const int8_t* llr;
  uint8_t* out;
  int8_t* soft;           // soft-buffer arena base
  DecState* state;
  uint32_t* tb_crc;       // [2 n_tbs] per TB: xor of its CBs' CRC24A contributions, and
                          // nonzero once a CB failed (read by purge, and by the host)
  uint8_t* cb_iters;      // [n_cbs] by sorted CB index
  uint8_t* cb_ok;         // [n_cbs]
  uint8_t* cb_runs;       // [n_cbs] iterations run (may be null)
  uint8_t* tb_ok;         // [n_tbs]
  uint32_t* tb_sat;       // [n_tbs] window passes on the saturating path (may be null)
  uint64_t* cb_time;      // optional: [4 n_cbs] by sorted CB index, %globaltimer ns at
                          // dequeue, de-rate-matched, iterations done, results written
  const uint32_t* xpowA;  // x^(32 s) mod gCRC24A, s < 2400
  const uint32_t* xpowB;  // x^(32 s) mod gCRC24B, s < 200
  const int32_t* mi_tab;  // [kMiTable] mutual-information table (stop rule 2)
  int8_t* dbg_d;          // optional: [sum (K+4)] x 3 d-streams per CB
  int16_t* dbg_ext;       // optional: [sum K] final extrinsic, natural order
  uint8_t* dbg_hard;      // optional: [sum K] hard decisions
  int32_t radix4_any;     // some CB selects the radix-4 forward recursion
  int32_t qtab_all;       // every CB has an interleaved-pass address table
  int32_t pair_any;       // some work item is a CB pair (needs qtab_all)
  const uint32_t* gate;   // optional: no LLR is read before *gate != 0
  uint32_t gate_us;       // bound of that wait (us); on expiry state->err is set
};

// Encoder launch description: one CB per CTA.
struct EncCb {
  int32_t K, F, E;
  int32_t R, ND, rank0;       // circular-buffer geometry and rank of k0
  int32_t f1, f2;             // QPP parameters
  int32_t tb;                 // transport block index
  int32_t pay_bits, pay_off;  // payload bits of the CB and their TB bit offset
  uint8_t crc_b;              // 1: CRC24B attached (C > 1)
  uint8_t pad0[3];
  int64_t e_off;              // first output byte (one coded bit per byte)
};

struct EncParams {
  const EncCb* cbs;
  const uint8_t* tb_bits;     // packed TB payloads (MSB first)
  const int64_t* tb_in_off;   // [n_tbs] byte offset of each payload
  const int32_t* tb_A;        // [n_tbs] payload bits
  uint8_t* e_out;
  const uint32_t* xpowA;      // x^(32 s) mod gCRC24A
  const uint32_t* xpowB;      // x^(32 s) mod gCRC24B
};

// PUSCH front stage (pusch.cu): one CTA of kPuschThreads handles one tile of
// whole interleaver rows of a TB; the scrambling sequence's jump-ahead
// tables have a coarse step of kPuschChunk positions, so TBs of G up to
// kPuschChunk x kPuschMaxChunks bits.
constexpr int kPuschThreads = 128;
constexpr int kPuschChunk = 32 * kPuschThreads;
constexpr int kPuschMaxChunks = 48;
constexpr int kGoldWords = kPuschMaxChunks * 32 + 2 * 31 * kPuschThreads;

struct PuschTb {
  int64_t in_off;   // byte offset of the TB's input (transmitted order, or e-sequence for TX)
  int64_t out_off;  // byte offset of its output
  int32_t G, qmnl, ncol, rows;  // bits, bits per symbol vector, interleaver columns, rows
  uint32_t c_init;  // scrambling initialisation (31 bits)
  int32_t mode;     // 1: descramble + de-interleave (TX: interleave + scramble); 0: copy
};
struct PuschChunk {
  int32_t tb, n0;   // TB index and first interleaver row of the tile
};
// One front-stage tile: whole interleaver rows, at most kPuschTile bytes.
constexpr int kPuschTile = 8192;
constexpr int kPuschMaxCols = 14;  // interleaver columns (SC-FDMA data symbols) at most
__host__ __device__ inline int pusch_tile_rows(int qmnl, int ncol) {
  const int r = kPuschTile / (qmnl * ncol);
  return r > 0 ? r : 1;
}
struct GoldTables {
  const uint32_t* x1c;  // [kPuschMaxChunks] x1 state at step 1600 + kPuschChunk c
  const uint32_t* a2c;  // [kPuschMaxChunks][31] columns of the x2 jump to that step
  const uint32_t* t1;   // [kPuschThreads][31] columns of the x1 jump by 32 t
  const uint32_t* t2;   // [kPuschThreads][31] columns of the x2 jump by 32 t
};
cudaError_t launch_pusch(bool tx, const PuschTb* tbs, const PuschChunk* chunks, int n_chunks,
                         GoldTables g, const int8_t* in, int8_t* out, cudaStream_t s);
GoldTables gold_tables_view(const uint32_t* d);

// Kernel launchers (decode.cu / encode.cu).  The decode kernel instantiation
// is chosen from p.radix4_any, p.qtab_all and p.pair_any.
cudaError_t launch_decode(const DecParams& p, int grid, int smem, cudaStream_t s);
int decode_max_smem();
// resident decode CTAs per SM at this dynamic smem, for the instantiation a
// launch with these flags uses
int decode_occupancy(int smem, bool radix4_any, bool qtab_all, bool pair_any);
cudaError_t launch_encode(const EncParams& p, int n_cbs, cudaStream_t s);

// Shared-memory bytes of one CB slot in the decode kernel.
__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int dec_cb_smem(int K, int P, int W) {
  int tp = W * P;                       // transposed array length (>= K)
  int nck = (W + kSub - 1) / kSub;      // checkpoints per window
  int nwords = (K + 31) / 32 + 1;       // hard-decision words
  return align16(3 * tp)                // sys, par1, par2 (int8)
         + align16(2 * tp)              // ext (int16)
         + 16                           // 12 tail LLRs
         + align16(4 * nwords)          // hard bits
         + 4 * P * 16                   // alpha/beta seeds of both decoders
         + P * nck * 16                 // alpha checkpoints
         + 64;                          // per-CB flags
}

// Pair slot of two CBs of size K with P windows of W steps: the three
// streams of both CBs interleaved byte by byte ([sys | par1 | par2], 2 W P
// bytes each: byte 2 t + L holds CB L's element at transposed index t), the
// extrinsics as 16-bit pairs (4 W P bytes), then per CB its tail LLRs, hard
// decisions and boundary seeds, the checkpoints of the P threads (ceil(W /
// kSubP) pairs of 8 packed registers each, 32 bytes) and per CB its flags.
struct PairLayout {
  int o_ext, o_tail, o_hard, hard_bytes, o_seed, seed_bytes, o_ck, ck_per_thread, o_flags, total;
};
__host__ __device__ inline PairLayout pair_layout(int K, int P, int W) {
  PairLayout l;
  const int tp = W * P;
  const int nwords = (K + 31) / 32 + 1;
  l.o_ext = align16(6 * tp);
  l.o_tail = l.o_ext + align16(4 * tp);
  l.o_hard = l.o_tail + 32;
  l.hard_bytes = align16(4 * nwords);
  l.o_seed = l.o_hard + 2 * l.hard_bytes;
  l.seed_bytes = 4 * P * 16;
  l.o_ck = l.o_seed + 2 * l.seed_bytes;
  l.ck_per_thread = 32 * ((W + kSubP - 1) / kSubP);
  l.o_flags = l.o_ck + P * l.ck_per_thread;
  l.total = l.o_flags + 2 * 64;
  return l;
}
__host__ __device__ inline int dec_pair_smem(int K, int P, int W) {
  return align16(pair_layout(K, P, W).total);
}

}  // namespace crnt
