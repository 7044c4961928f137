// pusch.cu -- the PUSCH front stage of the decoder's input: descrambling
// (TS 36.211 Sec. 5.3.1, the length-31 Gold sequence of Sec. 7.2) and the
// uplink channel de-interleaver for data without control information (TS
// 36.212 Sec. 5.2.2.8) -- the demultiplexing that hands the decoder each
// code word's LLRs in the paper's Fig. 4 (Sec. IV-B "Decoding function") --
// and, for the encoder, the transmit direction (interleave, scramble).
//
// One CTA handles a tile of whole rows of a TB's interleaver matrix (up to
// kPuschTile bytes): in transmitted order that is one segment per column, in
// e-sequence order one contiguous range, so both sides are read and written
// contiguously and the transposition happens in shared memory.  The tile's
// scrambling words -- 32 sequence bits each -- come first: the 31-bit
// register state of each component at step n holds x(n .. n + 30), so a word
// is the xor of the two states at its position plus one recurrence step for
// bit 31.  The states come from jump-ahead tables built once per context
// (GF(2) matrix powers of the two register updates): per 4096 steps the x1
// state and the columns of the x2 jump, per 32 t steps within them the
// columns of both jumps.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace crnt {

namespace {

constexpr int kNc = 1600;  // the Gold sequence's initial offset (TS 36.211 Sec. 7.2)

// ---------------------------------------------------------------- host tables
// A 31x31 GF(2) matrix as its 31 columns (bit i of column j = entry (i, j)).
struct Mat31 {
  uint32_t col[31];
};
uint32_t apply(const Mat31& m, uint32_t v) {
  uint32_t r = 0;
  for (int j = 0; j < 31; j++)
    if ((v >> j) & 1u) r ^= m.col[j];
  return r;
}
Mat31 mul(const Mat31& a, const Mat31& b) {  // a * b
  Mat31 r;
  for (int j = 0; j < 31; j++) r.col[j] = apply(a, b.col[j]);
  return r;
}
Mat31 identity() {
  Mat31 r;
  for (int j = 0; j < 31; j++) r.col[j] = 1u << j;
  return r;
}
// One step of a register whose state holds x(n .. n + 30) in bits 0 .. 30:
// shift down, the new bit x(n + 31) = xor of the tap bits enters at bit 30.
Mat31 step_matrix(uint32_t taps) {
  Mat31 m;
  for (int j = 0; j < 31; j++) {
    const uint32_t e = 1u << j;
    const uint32_t nb = (uint32_t)__builtin_popcount(e & taps) & 1u;
    m.col[j] = (e >> 1) | (nb << 30);
  }
  return m;
}
Mat31 power(Mat31 m, uint64_t n) {
  Mat31 r = identity();
  while (n) {
    if (n & 1u) r = mul(r, m);
    m = mul(m, m);
    n >>= 1;
  }
  return r;
}
// taps of x1(n+31) = x1(n+3) + x1(n) and x2(n+31) = x2(n+3) + x2(n+2) + x2(n+1) + x2(n)
constexpr uint32_t kTaps1 = (1u << 3) | 1u;
constexpr uint32_t kTaps2 = (1u << 3) | (1u << 2) | (1u << 1) | 1u;

// ---------------------------------------------------------------- device
__device__ __forceinline__ uint32_t jump(const uint32_t* __restrict__ cols, uint32_t v) {
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < 31; j++)
    if ((v >> j) & 1u) r ^= __ldg(cols + j);
  return r;
}

// Register states at sequence position n (a multiple of 32): the 31-bit
// state of each component holds x(m .. m + 30) for m = n + 1600, reached by
// the table jumps.
__device__ __forceinline__ void gold_state(const GoldTables& g, uint32_t c_init, int n,
                                           uint32_t& s1, uint32_t& s2) {
  const int c = n / kPuschChunk, t = (n - c * kPuschChunk) >> 5;
  s1 = jump(g.t1 + 31 * t, __ldg(g.x1c + c));
  s2 = jump(g.t2 + 31 * t, jump(g.a2c + 31 * c, c_init));
}
// new bits of the two recurrences from a state, bit j = x(m + 31 + j) (j < 28)
__device__ __forceinline__ uint32_t next1(uint32_t s) { return (s >> 3) ^ s; }
__device__ __forceinline__ uint32_t next2(uint32_t s) { return (s >> 3) ^ (s >> 2) ^ (s >> 1) ^ s; }
// The scrambling word at the states' position (bit j = c(n + j), bit 31 one
// recurrence step on), then both states advanced by 32 positions (28 + 4).
__device__ __forceinline__ uint32_t gold_word_step(uint32_t& s1, uint32_t& s2) {
  const uint32_t w = (s1 ^ s2) | (((next1(s1) ^ next2(s2)) & 1u) << 31);
  s1 = (s1 >> 28) | ((next1(s1) & 0x0FFFFFFFu) << 3);
  s2 = (s2 >> 28) | ((next2(s2) & 0x0FFFFFFFu) << 3);
  s1 = (s1 >> 4) | ((next1(s1) & 0xFu) << 27);
  s2 = (s2 >> 4) | ((next2(s2) & 0xFu) << 27);
  return w;
}
constexpr int kGoldParts = 4;  // threads per column segment building its words

// One tile: rows [r0, r0 + nr) of a TB's interleaver matrix, all ncol
// columns.  In transmitted order the tile is ncol segments (column c: symbols
// c R + r0 ..), in e-sequence order one contiguous range (symbols r0 ncol ..).
// TX = false: in holds received LLRs (transmitted order); the segments are
// read, descrambled (-128 reads as -127, the sign flips where c = 1) and
// transposed in shared memory, the range written out.  TX = true: in holds
// coded bits in e-sequence order; the range is read and the segments written
// interleaved and scrambled.  Mode-0 TBs (one column of one-byte symbols) are
// copied unchanged.
template <bool TX>
__global__ void __launch_bounds__(kPuschThreads) pusch_kernel(const PuschTb* __restrict__ tbs,
                                                              const PuschChunk* __restrict__ chunks,
                                                              GoldTables g, const int8_t* in,
                                                              int8_t* out) {
  __shared__ int8_t tile[kPuschTile];
  __shared__ uint32_t gw[kPuschTile / 32 + 2 * 16];
  const PuschChunk ch = chunks[blockIdx.x];
  const PuschTb t = tbs[ch.tb];
  const int qmnl = t.qmnl, ncol = t.ncol, R = t.rows;
  const int r0 = ch.n0;
  const int nr = min(pusch_tile_rows(qmnl, ncol), R - r0);
  const int seg = nr * qmnl;           // bytes of one column segment
  const int wpc = (seg + 31) / 32 + 1;  // scrambling words kept per column
  const int tid = threadIdx.x;
  if (t.mode) {  // the segments' scrambling words: one jump per thread, then steps
    for (int k = tid; k < ncol * kGoldParts; k += kPuschThreads) {
      const int c = k / kGoldParts, part = k - c * kGoldParts;
      const int w0 = part * wpc / kGoldParts, w1 = (part + 1) * wpc / kGoldParts;
      int n = ((((c * R + r0) * qmnl) >> 5) + w0) << 5;
      uint32_t s1 = 0u, s2 = 0u;
      if (w0 < w1 && n < t.G) gold_state(g, t.c_init, n, s1, s2);
      for (int w = w0; w < w1; w++, n += 32) {
        const uint32_t word = gold_word_step(s1, s2);
        gw[c * wpc + w] = n < t.G ? word : 0u;
      }
    }
  }
  __syncthreads();
  const int e0 = r0 * ncol * qmnl;  // the tile's first e-sequence position
  const int tb = nr * ncol * qmnl;   // its bytes
  const int8_t* src = in + t.in_off;
  int8_t* dst = out + t.out_off;
  if (TX) {
    for (int k = tid; k < tb; k += kPuschThreads) tile[k] = src[e0 + k];
    __syncthreads();
  }
  // offset k of a segment -> row k / qmnl by a multiply-shift (exact for k <
  // 2^20 / (qmnl - 1), far above a segment's at most kPuschTile bytes)
  const uint32_t rcp = qmnl > 1 ? ((1u << 20) + (uint32_t)qmnl - 1u) / (uint32_t)qmnl : 0u;
  for (int c = 0; c < ncol; c++) {
    const int p0 = (c * R + r0) * qmnl;  // the segment's first transmitted position
    const uint32_t* gc = gw + c * wpc - (p0 >> 5);
    for (int k = tid; k < seg; k += kPuschThreads) {
      const int sr = qmnl > 1 ? (int)(((uint32_t)k * rcp) >> 20) : k;
      const int b = k - sr * qmnl;
      const int i = p0 + k;
      const int e = (sr * ncol + c) * qmnl + b;
      const uint32_t flip = t.mode ? (gc[i >> 5] >> (i & 31)) & 1u : 0u;
      if (TX) {
        dst[i] = (int8_t)(tile[e] ^ (int8_t)flip);
      } else {
        const int v = max((int)src[i], -127);
        tile[e] = (int8_t)(flip ? -v : v);
      }
    }
  }
  if (!TX) {
    __syncthreads();
    for (int k = tid; k < tb; k += kPuschThreads) dst[e0 + k] = tile[k];
  }
}

}  // namespace

// Jump-ahead tables on the host: per chunk c the x1 state at step kNc +
// kPuschChunk c and the columns of the x2 jump to that step from the
// initial state; per thread t the columns of both jumps by 32 t.
std::vector<uint32_t> gold_tables_host() {
  std::vector<uint32_t> h((size_t)kGoldWords, 0u);
  uint32_t* x1c = h.data();
  uint32_t* a2c = x1c + kPuschMaxChunks;
  uint32_t* t1 = a2c + 31 * kPuschMaxChunks;
  uint32_t* t2 = t1 + 31 * kPuschThreads;
  const Mat31 A1 = step_matrix(kTaps1), A2 = step_matrix(kTaps2);
  const Mat31 C1 = power(A1, kPuschChunk), C2 = power(A2, kPuschChunk);
  Mat31 J1 = power(A1, kNc), J2 = power(A2, kNc);
  for (int c = 0; c < kPuschMaxChunks; c++) {
    x1c[c] = apply(J1, 1u);  // x1(0) = 1, x1(1 .. 30) = 0
    memcpy(a2c + 31 * c, J2.col, sizeof J2.col);
    J1 = mul(C1, J1);
    J2 = mul(C2, J2);
  }
  const Mat31 S1 = power(A1, 32), S2 = power(A2, 32);
  Mat31 T1 = identity(), T2 = identity();
  for (int t = 0; t < kPuschThreads; t++) {
    memcpy(t1 + 31 * t, T1.col, sizeof T1.col);
    memcpy(t2 + 31 * t, T2.col, sizeof T2.col);
    T1 = mul(S1, T1);
    T2 = mul(S2, T2);
  }
  return h;
}

GoldTables gold_tables_view(const uint32_t* d) {
  GoldTables g;
  g.x1c = d;
  g.a2c = d + kPuschMaxChunks;
  g.t1 = g.a2c + 31 * kPuschMaxChunks;
  g.t2 = g.t1 + 31 * kPuschThreads;
  return g;
}

void pusch_tiles(const PuschTb& q, int tb, std::vector<PuschChunk>& out) {
  const int rt = pusch_tile_rows(q.qmnl, q.ncol);
  for (int r0 = 0; r0 < q.rows; r0 += rt) out.push_back(PuschChunk{(int32_t)tb, r0});
}

void pusch_tb(const crnt_tb_params& tp, int64_t in_off, int64_t out_off, PuschTb* q) {
  q->in_off = in_off;
  q->out_off = out_off;
  q->G = (int32_t)tp.G;
  q->mode = (tp.flags & CRNT_F_PUSCH) ? 1 : 0;
  q->qmnl = q->mode ? tp.Qm * tp.NL : 1;  // mode 0: a copy, one column of bytes
  q->ncol = q->mode ? pusch_cols(tp) : 1;
  q->rows = q->G / (q->qmnl * q->ncol);
  q->c_init = tp.c_init;
}

cudaError_t launch_pusch(bool tx, const PuschTb* tbs, const PuschChunk* chunks, int n_chunks,
                         GoldTables g, const int8_t* in, int8_t* out, cudaStream_t s) {
  if (n_chunks <= 0) return cudaSuccess;
  if (tx)
    pusch_kernel<true><<<n_chunks, kPuschThreads, 0, s>>>(tbs, chunks, g, in, out);
  else
    pusch_kernel<false><<<n_chunks, kPuschThreads, 0, s>>>(tbs, chunks, g, in, out);
  return cudaGetLastError();
}

}  // namespace crnt
