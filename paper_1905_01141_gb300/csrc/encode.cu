// encode.cu -- downlink turbo encoder and rate matcher (Sec. IV-B "Encoding
// function", Fig. 3: CB segmentation, two 8-state RSC encoders around the
// QPP interleaver, rate 1/3 output, puncturing / bit selection, multiplexing).
//
// One CTA encodes one code block:
//   1. the CB bits: filler zeros, the TB payload slice, the TB CRC24A (for
//      the CB that carries it; computed by that CTA), the CB CRC24B (C > 1);
//   2. both constituent encoders in parallel over chunks: each thread runs
//      its chunk from state 0 with a byte-wise transition table, a serial
//      scan over the chunk end states (the RSC is linear over GF(2)) gives
//      every chunk its true start state, then each chunk is re-encoded;
//   3. trellis termination (3 tail steps per encoder, TS 36.212 5.1.3.2.2);
//   4. rate matching: every non-NULL circular-buffer position writes its bit
//      to the output indices k = rank - rank(k0) + t Nv < E.
#include <cstdint>

#include "crnt_internal.h"
#include "rm_geom.cuh"

namespace crnt {
namespace {

constexpr int kEncThreads = 128;
constexpr uint32_t GA = 0x1864CFBu;
constexpr uint32_t GB = 0x1800063u;

// One RSC step from state s = 4 r1 + 2 r2 + r3 with input u: a = u^r2^r3,
// parity u^r1^r2, next state (a, r1, r2).
__device__ __forceinline__ int rsc_step(int s, int u, int* par) {
  const int r1 = (s >> 2) & 1, r2 = (s >> 1) & 1, r3 = s & 1;
  const int a = u ^ r2 ^ r3;
  *par = u ^ r1 ^ r2;
  return (a << 2) | (r1 << 1) | r2;
}

__device__ __forceinline__ uint32_t gf_mulmod(uint32_t a, uint32_t b, uint32_t g) {
  uint32_t r = 0;
  for (int i = 23; i >= 0; i--) {
    r <<= 1;
    if (r & 0x1000000u) r ^= g;
    if ((a >> i) & 1u) r ^= b;
  }
  return r;
}

__device__ __forceinline__ uint32_t crc_byte(uint32_t r, uint32_t byte, const uint32_t* tab) {
  return ((r << 8) & 0xFFFFFFu) ^ tab[((r >> 16) ^ byte) & 0xFFu];
}

// CRC of n bytes produced by get(j), computed in parallel by the CTA: each
// thread runs the byte table over a contiguous chunk, shifts its remainder
// past the bytes that follow, and the partials are xor-reduced.
template <class Get>
__device__ uint32_t crc_bytes(int n, Get&& get, const uint32_t* tab, uint32_t g,
                              const uint32_t* xpow, uint32_t* red) {
  const int tid = threadIdx.x;
  const int per = ((n + kEncThreads - 1) / kEncThreads + 3) & ~3;  // multiple of 4
  const int b0 = tid * per, b1 = min(n, b0 + per);
  uint32_t r = 0;
  for (int j = b0; j < b1; j++) r = crc_byte(r, get(j), tab);
  if (b0 < b1) {
    const int after = n - b1;
    if (after >> 2) r = gf_mulmod(r, __ldg(&xpow[after >> 2]), g);
    for (int k = 0; k < (after & 3); k++) r = crc_byte(r, 0u, tab);
  }
  if (tid == 0) *red = 0u;
  __syncthreads();
  if (r) atomicXor(red, r);
  __syncthreads();
  const uint32_t out = *red;
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(kEncThreads) encode_kernel(EncParams prm) {
  __shared__ uint32_t tabA[256], tabB[256];
  __shared__ uint16_t rtab[8][256];  // (end state << 8) | parity byte
  __shared__ uint8_t cbits[kMaxK];   // CB bits (0/1)
  __shared__ uint8_t cbits2[kMaxK];  // the same bits in QPP order (input of encoder 2)
  __shared__ uint8_t zpar[2][kMaxK]; // parity of encoder 1 / 2
  __shared__ uint8_t tail[12];
  __shared__ uint8_t zs[2][kEncThreads], st0[2][kEncThreads + 1];
  __shared__ uint32_t red, tbcrc;
  const int tid = threadIdx.x;
  const EncCb d = prm.cbs[blockIdx.x];
  const int K = d.K, F = d.F;
  const int L = d.crc_b ? 24 : 0;

  for (int i = tid; i < 512; i += kEncThreads) {
    const uint32_t g = (i < 256) ? GA : GB;
    uint32_t r = (uint32_t)(i & 255) << 16;
    for (int k = 0; k < 8; k++) r = (r & 0x800000u) ? ((r << 1) ^ g) : (r << 1);
    (i < 256 ? tabA : tabB)[i & 255] = r & 0xFFFFFFu;
  }
  for (int i = tid; i < 8 * 256; i += kEncThreads) {
    int s = i >> 8, pb = 0;
    const int byte = i & 255;
    for (int k = 7; k >= 0; k--) {
      int par;
      s = rsc_step(s, (byte >> k) & 1, &par);
      pb = (pb << 1) | par;
    }
    rtab[i >> 8][byte] = (uint16_t)((s << 8) | pb);
  }
  __syncthreads();

  // ---- 1. CB bits
  const uint8_t* tb = prm.tb_bits + prm.tb_in_off[d.tb];
  const int A = prm.tb_A[d.tb];
  if (d.pay_off + d.pay_bits > A) {  // this CB carries the TB CRC24A
    const uint32_t c = crc_bytes(A / 8, [&](int j) { return (uint32_t)tb[j]; }, tabA, GA,
                                 prm.xpowA, &red);
    if (tid == 0) tbcrc = c;
    __syncthreads();
  }
  for (int k = tid; k < K - L; k += kEncThreads) {
    uint8_t b = 0;
    if (k >= F) {
      const int t = d.pay_off + (k - F);
      b = t < A ? (tb[t >> 3] >> (7 - (t & 7))) & 1 : (tbcrc >> (23 - (t - A))) & 1;
    }
    cbits[k] = b;
  }
  __syncthreads();
  if (L) {
    const uint32_t c = crc_bytes(
        (K - L) / 8,
        [&](int j) {
          uint32_t v = 0;
          for (int q = 0; q < 8; q++) v = (v << 1) | cbits[8 * j + q];
          return v;
        },
        tabB, GB, prm.xpowB, &red);
    for (int k = tid; k < 24; k += kEncThreads) cbits[K - 24 + k] = (c >> (23 - k)) & 1;
    __syncthreads();
  }

  // ---- 2. constituent encoders over chunks of whole bytes
  const int nbytes = K / 8;
  const int cpb = (nbytes + kEncThreads - 1) / kEncThreads;  // bytes per chunk
  const int j0 = tid * cpb, j1 = min(nbytes, j0 + cpb);
  const int f1 = d.f1, f2 = d.f2;
  // encoder 2 input c'[i] = c[PI(i)], PI(i) = (f1 i + f2 i^2) mod K: each
  // thread walks its own bit range with the first differences
  // PI(i+1) = PI(i) + D(i), D(i+1) = D(i) + 2 f2 (mod K)
  {
    const int i0 = 8 * j0, i1 = 8 * j1;
    if (i0 < i1) {
      int pi = (int)(((long long)f1 * i0 + (long long)f2 * i0 % K * i0) % K);
      int dl = (int)(((long long)f1 + (long long)f2 * (2 * i0 + 1)) % K);
      const int f2x2 = (int)((2ll * f2) % K);
      for (int i = i0; i < i1; i++) {
        cbits2[i] = cbits[pi];
        pi += dl;
        if (pi >= K) pi -= K;
        dl += f2x2;
        if (dl >= K) dl -= K;
      }
    }
  }
  __syncthreads();
  auto in_byte = [&](int enc, int j) -> int {
    const uint8_t* c = enc == 0 ? cbits : cbits2;
    int v = 0;
    for (int q = 0; q < 8; q++) v = (v << 1) | c[8 * j + q];
    return v;
  };
  for (int enc = 0; enc < 2; enc++) {
    int s = 0;
    for (int j = j0; j < j1; j++) s = rtab[s][in_byte(enc, j)] >> 8;
    zs[enc][tid] = (uint8_t)s;
  }
  __syncthreads();
  if (tid < 2) {
    // zero-input transition of a full chunk, then a serial scan of starts
    const int enc = tid;
    uint8_t zmap[8];
    for (int s = 0; s < 8; s++) {
      int x = s;
      for (int j = 0; j < cpb; j++) x = rtab[x][0] >> 8;
      zmap[s] = (uint8_t)x;
    }
    int cur = 0;
    for (int t = 0; t < kEncThreads; t++) {
      st0[enc][t] = (uint8_t)cur;
      cur = zmap[cur] ^ zs[enc][t];  // linearity: M^len(start) xor zero-state response
    }
  }
  __syncthreads();
  for (int enc = 0; enc < 2; enc++) {
    int s = st0[enc][tid];
    for (int j = j0; j < j1; j++) {
      const int e = rtab[s][in_byte(enc, j)];
      const int pb = e & 0xFF;
      for (int q = 0; q < 8; q++) zpar[enc][8 * j + q] = (pb >> (7 - q)) & 1;
      s = e >> 8;
    }
    if (j1 == nbytes && j0 < j1) {
      // ---- 3. termination: three steps with a = 0 (u = r2 ^ r3)
      for (int k = 0; k < 3; k++) {
        const int u = ((s >> 1) ^ s) & 1;
        int par;
        s = rsc_step(s, u, &par);
        tail[6 * enc + 2 * k] = (uint8_t)u;
        tail[6 * enc + 2 * k + 1] = (uint8_t)par;
      }
    }
  }
  __syncthreads();

  // ---- 4. rate matching into e_out
  RmGeom gg{K, F, d.R, d.ND, 0u, 0u};
  {
    const int X = d.ND + F;
    for (int c = 0; c < 32; c++) {
      const int pc = (int)(__brev((unsigned)c) >> 27);
      if (pc < (X & 31)) gg.maskB |= 1u << c;
      if (pc < d.ND - 1) gg.mask2 |= 1u << c;
    }
  }
  const int R = d.R, E = d.E;
  const int Nv = 3 * (K + 4) - 2 * F;
  uint8_t* out = prm.e_out + d.e_off;
  // rows x = unit * R + i, walked with (unit, i) updated incrementally
  int unit = tid / R, i = tid - (tid / R) * R;
  const int du = kEncThreads / R, di_ = kEncThreads - du * R;
  for (int x = tid; x < 64 * R; x += kEncThreads) {
    rm_visit(
        gg, unit, i,
        [&](int p, int st, int di, int rank) {
          (void)p;
          uint8_t v;
          if (di >= K) v = tail[3 * (di - K) + st];
          else v = st == 0 ? cbits[di] : zpar[st - 1][di];
          int k = rank - d.rank0;
          if (k < 0) k += Nv;
          for (; k < E; k += Nv) out[k] = v;
        },
        [&](int) {});
    unit += du;
    i += di_;
    if (i >= R) {
      i -= R;
      unit++;
    }
  }
}

}  // namespace

cudaError_t launch_encode(const EncParams& p, int n_cbs, cudaStream_t s) {
  if (n_cbs <= 0) return cudaSuccess;
  encode_kernel<<<n_cbs, kEncThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace crnt
