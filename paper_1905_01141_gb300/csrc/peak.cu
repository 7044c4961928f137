// peak.cu -- issue-rate probe of the integer instructions the decoder is
// built from, to ground the ALU-issue roofline used for the decode kernel.
//
// Each thread runs 8 independent dependency chains of one instruction kind
// (enough independent work per warp to keep a pipe busy), fully resident:
// blocks = SMs x 4 (the probe kernel uses few registers and no shared
// memory).  Every block times itself with clock64; warp-instructions per SM
// clock = (resident warps of an SM x chains x steps) / (elapsed cycles).
// Kinds: 0 = DPX add-max s32 (VIADDMNMX, the ACS / Lambda instruction),
// 1 = DPX add-max s16x2 (the packed form), 2 = 32-bit integer multiply-add
// (IMAD, FMA pipe), 3 = add-max and multiply-add interleaved 1:1.
//
// A measurement tool, not part of the decoding library: it is built into its
// own shared object (libcrnt_probe.so) with the one entry point
//   int crnt_int_issue_probe(int device, int kind, double* warp_instr_per_clk_per_sm);
// returning CRNT_OK, CRNT_EINVAL for an unknown kind or a null result, or
// CRNT_EDEVICE on a CUDA error.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/crnt.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(int iters, int seed, int* sink,
                                                              long long* cycles) {
  int a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = (int)threadIdx.x * (c + 3) + seed;
  const int x = seed ^ (int)blockIdx.x, y = seed + 7;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        if (KIND == 0) {
          a[c] = __viaddmax_s32(a[c], x, y + c);
        } else if (KIND == 1) {
          a[c] = (int)__viaddmax_s16x2((unsigned)a[c], (unsigned)x, (unsigned)(y + c));
        } else if (KIND == 2) {
          a[c] = a[c] * x + y;
        } else {
          a[c] = (c & 1) ? a[c] * x + y : __viaddmax_s32(a[c], x, y + c);
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  int s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s ^= a[c];
  if (s == 0x7F3A1C2B) sink[0] = s;  // keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
cudaError_t run(int blocks, int iters, int* sink, long long* cyc) {
  probe_kernel<KIND><<<blocks, kProbeThreads>>>(iters, 12345, sink, cyc);
  return cudaGetLastError();
}

}  // namespace

extern "C" int crnt_int_issue_probe(int device, int kind, double* warp_instr_per_clk_per_sm) {
  if (!warp_instr_per_clk_per_sm || kind < 0 || kind > 3) return CRNT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return CRNT_EDEVICE;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * kProbeBlocksPerSm;
  const int iters = 4096;
  int* sink = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&sink, 4) != cudaSuccess || cudaMalloc(&cyc, 8 * (size_t)blocks) != cudaSuccess) {
    if (sink) cudaFree(sink);
    return CRNT_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // first pass warms up
    switch (kind) {
      case 0: e = run<0>(blocks, iters, sink, cyc); break;
      case 1: e = run<1>(blocks, iters, sink, cyc); break;
      case 2: e = run<2>(blocks, iters, sink, cyc); break;
      default: e = run<3>(blocks, iters, sink, cyc); break;
    }
  }
  std::vector<long long> h((size_t)blocks);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(h.data(), cyc, 8 * (size_t)blocks, cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) return CRNT_EDEVICE;
  long long worst = 0;
  for (long long c : h) worst = c > worst ? c : worst;
  const double warps_per_sm = (double)kProbeBlocksPerSm * kProbeThreads / 32.0;
  const double instr = warps_per_sm * (double)iters * kUnroll * kChains;
  *warp_instr_per_clk_per_sm = instr / (double)worst;
  return CRNT_OK;
}
