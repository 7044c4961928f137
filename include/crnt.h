/*
 * crnt.h -- C ABI of the GB300 (sm_103a) LTE uplink channel-decoding library.
 *
 * The library decodes the uplink shared-channel transport blocks (TBs) of
 * many UEs and cells on one GPU: code-block segmentation, de-rate-matching
 * with HARQ soft combining, fixed-point max-log-MAP turbo decoding with a
 * CRC stop, and TB reassembly -- the channel-decoding function whose
 * parallelisation by UE and by code block (CB) is the subject of
 * "Higher aggregation of gNodeBs in Cloud-RAN architectures via parallel
 * computing" (Sec. IV-B "Decoding function", Fig. 4; Algorithms 1-2).  The
 * downlink turbo encoder and rate matcher (Sec. IV-B "Encoding function",
 * Fig. 3) are provided too.  Numeric definitions follow TS 36.212 (CRC
 * Sec. 5.1.1, segmentation Sec. 5.1.2, turbo code Sec. 5.1.3.2, rate
 * matching Sec. 5.1.4.1).
 *
 * Conventions for every entry point:
 *  - LLRs are int8, L = log P(bit=0)/P(bit=1) scaled by the caller (BPSK
 *    0 -> +1); -128 is treated as -127.  Hard decision: bit = (L < 0).
 *  - TB bits are packed MSB first, A/8 bytes per TB; A must be a multiple
 *    of 8 in [16, 75376] (all LTE TB sizes are).
 *  - Coded bits produced by the encoder are one bit per byte (0/1).
 *  - Buffers are owned by the caller unless stated otherwise.  Pointers may
 *    be host or device memory where a function says so; the library finds
 *    out which with cudaPointerGetAttributes.
 *  - Every function returns CRNT_OK (0) or a negative CRNT_E* code and
 *    never throws across the ABI.  A TB that fails its CRC is not an error:
 *    it is reported in crnt_tb_result.tb_crc_ok.
 */
#ifndef CRNT_H
#define CRNT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRNT_VERSION 2

#define CRNT_OK 0
#define CRNT_EINVAL (-1)    /* malformed argument */
#define CRNT_ENOMEM (-2)    /* device or host allocation failed / budget exceeded */
#define CRNT_EAGAIN (-3)    /* admission refused for now: retry later */
#define CRNT_ETIMEDOUT (-4) /* a bounded wait expired */
#define CRNT_EDEVICE (-5)   /* CUDA error: the context should be destroyed */
#define CRNT_ENOTFOUND (-6) /* no such ticket / HARQ process */

#define CRNT_MAX_CB 16     /* code blocks per TB supported (A <= 75376 needs 13) */
#define CRNT_MAX_P 128     /* windows per SISO pass */

typedef struct crnt_ctx crnt_ctx;
typedef struct crnt_plan crnt_plan;

/* Context configuration.  Zero fields take the default in brackets. */
typedef struct crnt_config {
    int32_t device;          /* CUDA device ordinal [0] */
    uint32_t harq_slots;     /* HARQ soft-buffer slots kept on the device [4096] */
    uint64_t mem_budget;     /* device bytes for soft buffers + in-flight work [8 GiB] */
    uint32_t max_inflight;   /* serving: TBs on the device at once [4096] */
    uint32_t deadline_us;    /* serving: latency target from crnt_submit to the
                                result [1000] */
    uint32_t pair_min_cbs;   /* CB pairs (shape table) only in batches of at least
                                this many CBs [two waves of one-CB CTAs: 6 x SMs];
                                1 = in every batch */
    uint32_t admission;      /* serving: 0 = refuse a subframe whose predicted
                                completion passes deadline_us (and beyond the
                                in-flight and memory limits) [0]; 1 = only the
                                in-flight and memory limits */
} crnt_config;

/* Per-TB parameters (40 bytes). */
typedef struct crnt_tb_params {
    uint32_t A;          /* TB size in bits without CRC24A, multiple of 8, 16..75376 */
    uint32_t G;          /* rate-matched bits (= LLRs) of the TB, multiple of Qm*NL */
    uint16_t P;          /* windows per SISO pass, 0 = autotuned per K; clamped to
                            [1, min(K/8, CRNT_MAX_P)] */
    uint8_t Qm;          /* 2, 4 or 6 bits per modulation symbol (used for E_r) */
    uint8_t NL;          /* 1 or 2 layers */
    uint8_t rv;          /* redundancy version 0..3 */
    uint8_t max_iter;    /* 1..16 turbo iterations */
    uint8_t early_stop;  /* stop rule per CB: 0 none (max_iter iterations),
                            1 at its first CRC pass, 2 when the mean mutual
                            information of the exchanged extrinsic LLRs changes
                            by at most 2^-10 bit between iterations (the
                            paper's rule, Sec. IV-B; the CRC then only decides
                            success) */
    uint8_t new_data;    /* 1: clear the HARQ soft buffer before combining */
    uint32_t cell, ue, harq_pid; /* HARQ process key (flags bit 0 set) */
    uint32_t flags;      /* bit 0 (CRNT_F_HARQ): combine into the library-owned
                            soft buffer of (cell, ue, harq_pid); bit 1
                            (CRNT_F_PURGE): purge on failure, see below; bit 2
                            (CRNT_F_PUSCH): received PUSCH order, see below */
    uint32_t c_init;     /* CRNT_F_PUSCH: scrambling initialisation, 31 bits
                            (TS 36.211 5.3.1: n_RNTI 2^14 + q 2^13 +
                            floor(n_s / 2) 2^9 + N_ID^cell) */
    uint16_t n_symb;     /* CRNT_F_PUSCH: channel-interleaver columns C_mux, the
                            SC-FDMA data symbols of the subframe [0 = 12] */
    uint16_t pad0;
} crnt_tb_params;

#define CRNT_F_HARQ 1u
/* Purge on failure (Algorithm 2's purge of a failed TB's remaining CBs): as
 * soon as one CB of the TB fails (max_iter iterations without a CRC pass),
 * its other CBs stop at their next iteration boundary.  The TB result is the
 * same (tb_crc_ok = 0); a stopped CB reports cb_iters = 0, cb_crc_ok = 0 and
 * writes no payload bytes (they are left as they were).  Which CBs stop
 * depends on timing; TBs that decode are never affected. */
#define CRNT_F_PURGE 2u
/* Received PUSCH order (the demultiplexing ahead of the decoder, Sec. IV-B
 * Fig. 4): the TB's G LLRs (or, for the encoder, its G output bits) are the
 * code word as sent on the channel -- channel-interleaved for data without
 * control information (TS 36.212 5.2.2.8: G / (Qm NL) symbols written row by
 * row into n_symb columns, read column by column) and scrambled with the
 * length-31 Gold sequence of c_init (TS 36.211 5.3.1 / 7.2; a set sequence
 * bit flips an LLR's sign).  The decoder descrambles and de-interleaves
 * before de-rate-matching; the encoder interleaves and scrambles after rate
 * matching.  G must be a multiple of Qm NL n_symb and at most 196608. */
#define CRNT_F_PUSCH 4u

/* Per-TB result (96 bytes). */
typedef struct crnt_tb_result {
    int32_t status;                 /* CRNT_OK or a negative code for this TB */
    uint8_t tb_crc_ok;              /* 1: every CB CRC and the TB CRC24A passed */
    uint8_t C;                      /* code blocks */
    uint16_t K_plus, K_minus, F;    /* segmentation (TS 36.212 5.1.2) */
    uint8_t cb_iters[CRNT_MAX_CB];  /* iterations run per CB; max_iter+1 = failure
                                       (the paper's loss convention, Sec. IV-B) */
    uint8_t cb_crc_ok[CRNT_MAX_CB];
    uint8_t cb_iters_run[CRNT_MAX_CB]; /* iterations actually run per CB (a failure
                                       under a stop rule may stop before max_iter;
                                       a purged CB reports the ones it ran) */
    uint16_t P_used;                /* window count used for K+ (after clamping: the
                                       windows the decoder actually runs) */
    uint16_t sat_passes;            /* window passes of this TB's CBs that ran the
                                       saturating int16 arithmetic (the decoder's exact
                                       path; every other pass was proved unable to
                                       saturate and ran clamp-free), capped at 65535 */
    uint64_t ticket;                /* serving ticket (0 elsewhere) */
    uint64_t t_submit_ns, t_start_ns, t_done_ns; /* serving timestamps (CLOCK_MONOTONIC) */
} crnt_tb_result;

/* One code block of a TB as laid out by the library (host-side query). */
typedef struct crnt_cb_layout {
    uint32_t K, F, E, k0, Ncb;  /* size, filler, rate-matched length, start, buffer */
    uint32_t llr_offset;        /* first LLR of the CB inside the TB's G LLRs */
    uint32_t soft_offset;       /* first byte of its soft buffer inside the TB's */
    uint32_t crc_b;             /* 1: CRC24B attached (C > 1) */
    uint32_t P;                 /* window count after clamping (tb->P, or autotuned) */
    uint32_t W;                 /* window length ceil(K/P); ceil(K/W) windows are used */
} crnt_cb_layout;

/* Aggregate sizes of a plan (host-side query). */
typedef struct crnt_plan_info {
    uint32_t n_tb, n_cb;
    uint64_t llr_bytes;   /* sum of G: input LLRs, concatenated in TB order */
    uint64_t out_bytes;   /* sum of A/8: output bytes, concatenated in TB order */
    uint64_t info_bits;   /* sum of A */
    uint64_t trellis_steps; /* sum of K over CBs (one SISO pass visits each once) */
    uint64_t dbg_elems;   /* sum of (K+4) over CBs: length of the debug arrays */
    uint32_t n_items, grid;
    uint32_t pair_items;  /* work items that decode a CB pair (shape table entry 2) */
    uint32_t smem_bytes;  /* dynamic shared memory of one decode CTA */
} crnt_plan_info;

/* ---- library ---------------------------------------------------------- */
int crnt_version(void);
const char* crnt_strerror(int code);

/* ---- host-side parameter queries (no GPU needed) ---------------------- */

/* QPP interleaver parameters (f1, f2) of CB size K (TS 36.212 Table
 * 5.1.3-3; turbo interleaver of Sec. IV-B Figs. 3-4).  CRNT_EINVAL if K is
 * not one of the 188 CB sizes. */
int crnt_qpp_params(uint32_t K, uint32_t* f1, uint32_t* f2);

/* Segmentation and rate-matching layout of one TB (TS 36.212 5.1.2 and
 * 5.1.4.1; replaces the split loop of Algorithm 1).  cbs must hold
 * CRNT_MAX_CB entries; *C receives the CB count.  Validates A, G, Qm, NL, rv
 * as described at crnt_tb_params; CRNT_EINVAL otherwise. */
int crnt_tb_layout(const crnt_tb_params* tb, crnt_cb_layout* cbs, uint32_t* C);

/* Interleaved-pass addresses of a CB of size K split into P windows (P
 * clamped like crnt_tb_params::P; 0 = the window table's), as the decoder
 * reads them: entry p W + j (window p, step j, W = ceil(K / P)) holds, for
 * j < the window's length, q = PI(p W + j) (the QPP interleaver, TS 36.212
 * 5.1.3.2.3) in bits 16..31 and its transposed shared-memory index
 * (q mod W) P + q / W in bits 0..15; 0 past a window's end.  Host-side query
 * (no GPU).  CRNT_EINVAL for an unknown K, a null map or n < W P. */
int crnt_interleaver_map(uint32_t K, uint32_t P, uint32_t* map, uint32_t n);

/* De-rate-matching map of a CB of size K with F filler bits split into P
 * windows (P clamped like crnt_tb_params::P; 0 = the window table's), the
 * map the decoder reads (TS 36.212 5.1.4.1 circular buffer): entry k, for
 * k < Nv = 3 (K + 4) - 2 F, describes where the k-th received LLR of
 * redundancy version rv lands (the k-th non-NULL buffer position from k0;
 * with E > Nv LLR k + Nv lands there too).  Bits 0..15: its place in the
 * CB's shared-memory slot -- for bit d < K of stream s, s W P + (d mod W) P
 * + d / W with W = ceil(K / P); for tail bit d >= K, 3 W P + 3 (d - K) + s;
 * bits 16..31: its circular-buffer position.  Host-side query (no GPU).
 * CRNT_EINVAL for an unknown K, rv > 3, F not a multiple of 8 below 64, a
 * null map or n < Nv. */
int crnt_derm_map(uint32_t K, uint32_t P, uint32_t F, uint32_t rv, uint32_t* map, uint32_t n);

/* ---- window-count table (autotuner) ----------------------------------- */
/* A TB that asks for P = 0 gets, for each CB size K, the window count of a
 * process-wide table shared by every context: entry i holds P for the i-th
 * of the CRNT_NUM_K CB sizes in increasing order (40, 48, ..., 6144); 0
 * selects the built-in choice (windows of about 48 trellis steps).  Entries
 * are clamped like a requested P.  The window count changes the decoded
 * values (window seeds, Sec. IV-B parallelisation over P), so a table fixes
 * the results of P = 0 requests; crnt_tb_layout reports it.  The paper has no
 * tuner: its thread counts are configured by hand. */
#define CRNT_NUM_K 188
int crnt_tune_get(uint8_t* P_by_k, uint32_t n);       /* copies min(n, 188) entries */
int crnt_tune_set(const uint8_t* P_by_k, uint32_t n); /* n must be 188 */
/* Forward-recursion radix per CB size, a second process-wide table: entry i
 * is 2 (one trellis step per forward update, the default) or 4 (two steps
 * per update: each state takes the best of its four two-step paths).  The
 * radix-4 recursion runs only in window passes that the decoder has proved
 * free of int16 saturation; there the maximum over two-step paths equals two
 * radix-2 steps exactly, so the radix never changes a decoded value, only
 * the speed.  Passes that may saturate always use radix 2.  get writes 2 or
 * 4; set accepts 0 (= 2), 2 or 4 and needs n = 188. */
int crnt_tune_radix_get(uint8_t* radix_by_k, uint32_t n);
int crnt_tune_radix_set(const uint8_t* radix_by_k, uint32_t n);
/* CTA shape per CB size, a third process-wide table (the paper's
 * parallelism granularity per worker, Sec. IV-B "Scheduler", chosen by
 * measurement).  Entry i is 1 (the default: the P windows of a CB run on P
 * threads, one window each) or 2 (CB pairs: two CBs of that size and window
 * count run on the same P threads, window p of both in the two 16-bit halves
 * of each register, so every add-max instruction advances two CBs; such
 * batches run two CTAs per SM).  A pass that cannot be proved to stay within
 * 16 bits runs one CB at a time, so the shape never changes a decoded value,
 * only the speed.  Pairs need the context's per-(K, P) tables and the
 * radix-2 recursion; the allocation-free entry point runs shape 1.  get
 * writes 1 or 2; set accepts 0 (= 1), 1 or 2 and needs n = 188. */
int crnt_tune_shape_get(uint8_t* shape_by_k, uint32_t n);
int crnt_tune_shape_set(const uint8_t* shape_by_k, uint32_t n);
/* Measure on ctx's GPU the batched decode throughput (6 iterations, full
 * batches of single-CB TBs per K) of candidate window counts for every CB
 * size -- P = floor(K / w) in both CTA shapes and, for CB pairs, P = ceil(K /
 * w) (windows filling the pair path's 8-step sub-windows), w in {32, 40,
 * 48, 56, 64, 80, 96} -- keep for each K the longest windows (at least w_min
 * trellis steps, 0 = 32; smaller windows cost BLER) within 1 % of the
 * fastest candidate, install the table and copy it to P_by_k (188 entries,
 * may be NULL).  At the kept window count it installs the faster shape in
 * the shape table and times the radix-4 forward recursion, installing the
 * radix table (4 where it is more than 1 % faster than both shapes, else 2).  Blocking; takes a few seconds; allocates device
 * memory for its inputs and frees it. */
int crnt_autotune(crnt_ctx* ctx, uint32_t w_min, uint8_t* P_by_k);

/* ---- context ---------------------------------------------------------- */
/* Create a context on cfg->device (NULL cfg = defaults).  Allocates the
 * HARQ soft-buffer arena lazily.  CRNT_EDEVICE if CUDA is unusable. */
int crnt_create(crnt_ctx** out, const crnt_config* cfg);
/* Destroy a context and every plan and buffer it owns. */
int crnt_destroy(crnt_ctx* ctx);

/* ---- batched decode: one persistent launch per batch ------------------- */
/* Plan a batch of n TBs: segmentation, per-CB parameters, the window count
 * per K and the work queue (the device counterpart of Algorithms 1-2).
 * Copies tbs; allocates the plan's device descriptors and result buffers.
 * HARQ keys (CRNT_F_HARQ) are bound to soft-buffer slots here. */
int crnt_plan_create(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, crnt_plan** out);
int crnt_plan_get_info(const crnt_plan* plan, crnt_plan_info* info);
/* Enqueue the decode of the planned batch on a CUDA stream (NULL = default):
 * llr (device, llr_bytes) in, out (device, out_bytes) out.  Asynchronous,
 * allocates nothing and may be captured in a CUDA graph.  A batch with
 * CRNT_F_PUSCH TBs first runs the front stage (descramble, de-interleave)
 * into the plan's scratch, allocated by crnt_plan_create.  The optional debug
 * arrays (device, may be NULL) receive per CB at offset o = sum of (K+4) of
 * the CBs before it in TB order: dbg_d[3o ..] the de-rate-matched streams
 * d0|d1|d2 (K+4 int8 each), dbg_ext[o ..] the final exchanged extrinsic
 * (K int16, natural order), dbg_hard[o ..] the final hard decisions (K). */
int crnt_plan_launch(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream);
int crnt_plan_launch_debug(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream,
                           int8_t* dbg_d, int16_t* dbg_ext, uint8_t* dbg_hard);
/* As crnt_plan_launch, but no CTA reads an LLR before the 32-bit word at
 * `ready` (device memory, or page-locked host memory) is non-zero, so a
 * decode can be enqueued before its LLRs have arrived (ahead of a fronthaul
 * transfer into llr): the writer stores the LLRs, then the non-zero word
 * with release semantics.  Each CTA's first thread polls the word (acquire
 * load, system scope) for at most timeout_us microseconds (1 ..
 * 10 000 000) measured on %globaltimer.  When a CTA's wait expires, the
 * CTAs stop (those that saw the word non-zero first may have decoded some
 * CBs) and crnt_plan_results reports CRNT_ETIMEDOUT for every TB of the
 * batch; the plan and the context stay usable.  CRNT_EINVAL for plans with
 * CRNT_F_PUSCH TBs. */
int crnt_plan_launch_gated(crnt_plan* plan, const int8_t* llr, uint8_t* out, void* stream,
                           const uint32_t* ready, uint32_t timeout_us);
/* Wait for the stream and fill res[n] (host).  CRNT_EDEVICE on a CUDA error. */
int crnt_plan_results(crnt_plan* plan, crnt_tb_result* res, void* stream);

/* Per-CB timestamps of a launch (the paper's performance captor, Sec. IV-B:
 * the delay of each CB split into pre-processing -- de-rate-matching --,
 * channel coding -- the turbo iterations -- and post-processing -- hard
 * decisions into the TB, the TB CRC), taken on the GPU's %globaltimer
 * (nanoseconds).  The stamps belong to the CB's work item, so CBs decoded
 * together by one CTA share them. */
typedef struct crnt_cb_timing {
    uint32_t tb, r;        /* TB index in the plan, CB index in the TB */
    uint64_t t_start_ns;   /* a CTA took the CB's work item from the queue */
    uint64_t t_derm_ns;    /* its LLRs were de-rate-matched */
    uint64_t t_iter_ns;    /* its turbo iterations ended */
    uint64_t t_done_ns;    /* its payload bits and results were written */
    uint8_t iterations;    /* iterations run */
    uint8_t pad[7];
} crnt_cb_timing;
/* Record the timestamps in every later launch of the plan (enable = 1; the
 * first call allocates their device and page-locked buffers, 32 + 32 bytes
 * per CB) or stop recording (0). */
int crnt_plan_set_timing(crnt_plan* plan, int enable);
/* After a launch with timing on: wait for the stream and fill out[n_cb]
 * (host), CBs in TB order.  CRNT_EINVAL if timing is off or n < n_cb. */
int crnt_plan_timing(crnt_plan* plan, crnt_cb_timing* out, uint32_t n, void* stream);
int crnt_plan_destroy(crnt_plan* plan);

/* Blocking decode of n TBs.  llr: concatenated G LLRs of every TB (host or
 * device); out: concatenated A/8 bytes (host or device); res: n results
 * (host).  Device buffers are used in place; host LLRs are copied into the
 * context's device arena (page-locked ones by DMA); a page-locked host out
 * (cudaHostAlloc, cudaHostRegister) is written in place by the kernels over
 * the CPU-GPU link, a pageable one staged.  Batches of 24 or more TBs are
 * decoded as three chunks whose planning and copies overlap the decoding of
 * earlier chunks. */
int crnt_decode_batch(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, const int8_t* llr,
                      uint8_t* out, crnt_tb_result* res);
/* Blocking decode of one TB (n = 1 of the above). */
int crnt_decode_tb(crnt_ctx* ctx, const int8_t* llr, const crnt_tb_params* tb, uint8_t* out,
                   crnt_tb_result* res);

/* ---- allocation-free batched decode ------------------------------------ */
/* No counterpart in the paper.  The same fused decode for callers that must
 * not allocate device memory -- for example code that runs inside another
 * framework's memory pool or between phases where allocation is forbidden --
 * and so cannot create a context (crnt_create allocates).  Descriptors, the
 * work queue, the CRC and mutual-information tables and per-launch scratch
 * live in one fixed file-scope device array of about 153 KiB held by every
 * GPU that loads the library; no cudaMalloc, cudaFree, pinned or library
 * allocation happens in this call.  llr (concatenated G LLRs) in, out
 * (concatenated A/8 bytes) out, both device, managed or page-locked host
 * memory (pageable host memory gives CRNT_EINVAL: there is nowhere to stage
 * it), res[n] (host) results, the same fields as crnt_decode_batch; runs on
 * `stream` (NULL = default) on the current device and returns after that
 * stream has finished the decode, also when it fails.  Limits: n <= 64 TBs
 * and at most 832 code blocks in total, else CRNT_ENOMEM ("exceeds the
 * static workspace"); no HARQ combining and no PUSCH front stage
 * (CRNT_F_HARQ or CRNT_F_PUSCH gives CRNT_EINVAL);
 * purge on failure and all stop rules work as elsewhere.  Without a context
 * there are no per-(K, P) tables, so the kernel computes its interleaver
 * addresses and circular-buffer walk (same results).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * uploads the tables with synchronous copies, so make that first call before
 * any stream capture.  Every call shares the array: calls whose GPU work overlaps (two
 * streams, or two host threads) race on it, so do not overlap them. */
int crnt_decode_batch_static(const crnt_tb_params* tbs, uint32_t n, const int8_t* llr,
                             uint8_t* out, crnt_tb_result* res, void* stream);

/* ---- downlink encode (Sec. IV-B "Encoding function", Fig. 3) ------------ */
/* Encode n TBs: CRC24A, segmentation with CRC24B and filler, turbo encode
 * (2 RSC + QPP, trellis termination), sub-block interleave and bit
 * selection from k0(rv), and for CRNT_F_PUSCH TBs the channel interleaver
 * and scrambling.  bits: concatenated A/8 bytes per TB (host or device);
 * e_out: concatenated G bytes (one coded bit per byte, host or device).  Device and page-locked host buffers are used in place by the
 * kernel; pageable host buffers are staged.  Blocking. */
int crnt_encode_batch(crnt_ctx* ctx, const crnt_tb_params* tbs, uint32_t n, const uint8_t* bits,
                      uint8_t* e_out);
int crnt_encode_tb(crnt_ctx* ctx, const uint8_t* bits, const crnt_tb_params* tb, uint8_t* e_out);

/* ---- serving: continuous batching ------------------------------------- */
/* Submit n TBs whose LLRs are host buffers llrs[i] (G_i bytes each) -- one
 * subframe, say.  The TBs are prepared (segmentation, soft-buffer binding,
 * descriptors) and their LLRs copied on the calling thread before return;
 * the serving worker batches and launches them; tickets_out[i] receives a
 * ticket.  CRNT_EAGAIN when admission is refused, and nothing of the call is
 * queued: beyond max_inflight TBs, when the library's page-locked LLR or
 * output ring is full (results not yet polled hold output space), or --
 * with crnt_config.admission 0 -- when the call's predicted completion
 * passes deadline_us while other work is outstanding (the prediction is
 * fitted to the completions seen: latency against the decode work ahead).
 * If a TB fails its preparation (another code) nothing is queued either, but
 * soft buffers already bound for earlier CRNT_F_HARQ TBs of the call stay
 * bound.
 * TBs that share a HARQ key (cell, ue, harq_pid) must not be in flight at
 * the same time (a retransmission is submitted after the previous
 * transmission's result was polled, as the HARQ round trip implies).
 * Several threads may submit at once; each call copies its own LLRs. */
int crnt_submit(crnt_ctx* ctx, const crnt_tb_params* tbs, const int8_t* const* llrs, uint32_t n,
                uint64_t* tickets_out);
/* Collect up to max finished TBs, waiting at most timeout_us for the first.
 * done[i] gets the result (ticket set); bits[i] a pointer to its A/8 output
 * bytes, owned by the library and valid until the next crnt_poll.  Returns
 * the number collected (>= 0) or a negative code. */
int crnt_poll(crnt_ctx* ctx, crnt_tb_result* done, const uint8_t** bits, uint32_t max,
              uint32_t timeout_us);
/* Forget the soft buffer of a HARQ process.  CRNT_ENOTFOUND if unknown. */
int crnt_harq_release(crnt_ctx* ctx, uint32_t cell, uint32_t ue, uint32_t harq_pid);

/* Serving counters since the context's serving loop started (all zero
 * before the first crnt_submit) -- the serving side of the paper's
 * performance captor (Sec. IV-B): where time goes between submission and
 * result, and what admission turned away.  Cumulative: take differences to
 * measure an interval.  A subframe is one crnt_submit call.  Safe to call
 * from any thread while serving runs (a consistent snapshot of the counts;
 * the time counters are read separately).  Returns CRNT_OK, or CRNT_EINVAL
 * for a null argument. */
typedef struct crnt_serve_stats {
    uint64_t submit_calls;     /* crnt_submit calls that reached admission */
    uint64_t refused_calls;    /* of which refused with CRNT_EAGAIN */
    uint64_t refused_deadline; /* of the refused: predicted completion past deadline_us */
    uint64_t offered_tbs;      /* TBs in those calls */
    uint64_t admitted_tbs;
    uint64_t done_tbs;         /* results handed to the done queue */
    uint64_t late_tbs;         /* of which finished later than submit + deadline_us */
    uint64_t batches;          /* decode launches of the serving worker */
    uint64_t worker_plan_ns;   /* worker time assembling batches (plans of prepared TBs) */
    uint64_t worker_launch_ns; /* worker time in launch calls */
    uint64_t worker_harvest_ns;/* worker time collecting finished batches */
    uint64_t worker_ns;        /* wall time since the loop started */
    uint64_t submit_copy_ns;   /* submitting threads' time copying LLRs */
    double model_a_us;         /* admission model: latency with nothing ahead */
    double model_rate;         /* admission model: trellis step-iterations per us */
    double model_sigma_us;     /* admission model: spread of its residuals */
} crnt_serve_stats;
int crnt_serve_stats_get(crnt_ctx* ctx, crnt_serve_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* CRNT_H */
