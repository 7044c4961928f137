// pusch.cu -- the PUSCH front stage of the decoder's input: descrambling
// (TS 36.211 Sec. 5.3.1, the length-31 Gold sequence of Sec. 7.2) and the
// uplink channel de-interleaver for data without control information (TS
// 36.212 Sec. 5.2.2.8) -- the demultiplexing that hands the decoder each
// code word's LLRs in the paper's Fig. 4 (Sec. IV-B "Decoding function") --
// and, for the encoder, the transmit direction (interleave, scramble).
//
// One CTA handles 4096 positions of one TB's transmitted sequence.  Its 128
// threads first produce the 4096 scrambling bits c(n0 .. n0 + 4095), 32 per
// thread: the 31-bit register state of each component at step n holds
// x(n .. n + 30), so a thread's word is the xor of the two states at its
// start plus one recurrence step for bit 31.  The states come from jump-ahead
// tables built once per context (GF(2) matrix powers of the two register
// updates): per chunk of 4096 steps the x1 state and the columns of the x2
// jump, per thread offset 32 t the columns of both jumps.  Then the threads
// move the chunk's LLRs (bits) between transmitted order and the e-sequence
// order, flipping signs (bits) where c = 1.
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

// TX = false: in holds a TB's received LLRs in transmitted order, out gets
// the e-sequence (descrambled: -128 reads as -127, the sign flips where c =
// 1; de-interleaved).  TX = true: in holds coded bits (0/1 per byte) in
// e-sequence order, out gets them interleaved and scrambled.  Mode-0 TBs are
// copied unchanged.
template <bool TX>
__global__ void __launch_bounds__(kPuschThreads) pusch_kernel(const PuschTb* __restrict__ tbs,
                                                              const PuschChunk* __restrict__ chunks,
                                                              GoldTables g, const int8_t* in,
                                                              int8_t* out) {
  __shared__ uint32_t cbits[kPuschChunk / 32];
  const PuschChunk ch = chunks[blockIdx.x];
  const PuschTb t = tbs[ch.tb];
  const int n0 = ch.n0;
  const int len = min(kPuschChunk, t.G - n0);
  const int tid = threadIdx.x;
  if (t.mode) {
    const int c = n0 / kPuschChunk;
    const uint32_t s1 = jump(g.t1 + 31 * tid, __ldg(g.x1c + c));
    const uint32_t s2 = jump(g.t2 + 31 * tid, jump(g.a2c + 31 * c, t.c_init));
    const uint32_t b1 = ((s1 >> 3) ^ s1) & 1u;
    const uint32_t b2 = ((s2 >> 3) ^ (s2 >> 2) ^ (s2 >> 1) ^ s2) & 1u;
    cbits[tid] = (s1 ^ s2) | ((b1 ^ b2) << 31);  // bit j: c(n0 + 32 tid + j)
  }
  __syncthreads();
  const int8_t* src = in + t.in_off;
  int8_t* dst = out + t.out_off;
  for (int k = tid; k < len; k += kPuschThreads) {
    const int i = n0 + k;  // transmitted position
    int j = i;             // e-sequence position
    bool flip = false;
    if (t.mode) {
      const int s = i / t.qmnl, b = i - s * t.qmnl;
      const int col = s / t.rows, row = s - col * t.rows;
      j = (row * t.ncol + col) * t.qmnl + b;
      flip = (cbits[k >> 5] >> (k & 31)) & 1u;
    }
    if (TX) {
      dst[i] = (int8_t)(src[j] ^ (flip ? 1 : 0));
    } else {
      const int v = max((int)src[i], -127);
      dst[j] = (int8_t)(flip ? -v : v);
    }
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
