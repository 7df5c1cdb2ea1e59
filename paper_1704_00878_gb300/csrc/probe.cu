// probe.cu -- issue-rate probe of the integer instructions of the DP cell
// update (a measurement aid, see include/msa_probe.h).
#include "common.cuh"
#include "msa_probe.h"

namespace {

template <int OP>
__device__ __forceinline__ unsigned probe_op(unsigned a, unsigned b, unsigned c) {
  if constexpr (OP == MSA_PROBE_VIADDMAX_S16X2) return __viaddmax_s16x2(a, b, c);
  else if constexpr (OP == MSA_PROBE_VIMAX3_S16X2) return __vimax3_s16x2(a, b, c);
  else if constexpr (OP == MSA_PROBE_VIADDMAX_S32) return (unsigned)__viaddmax_s32((int)a, (int)b, (int)c);
  else {
    unsigned d;
    asm("prmt.b32 %0, %1, %2, 0x9180;" : "=r"(d) : "r"(a), "r"(c));
    return d ^ b;
  }
}

// 8 independent chains per thread, 16 unrolled steps per iteration.
template <int OP>
__global__ void k_probe(int iters, unsigned *out, unsigned seed) {
  unsigned a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = seed * (threadIdx.x + u + 1);
  const unsigned b = seed * 7 + 3, c = seed * 13 + 5;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = probe_op<OP>(a[u], b + r, c ^ (unsigned)u);
    }
  }
  unsigned x = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) x ^= a[u];
  if (x == 0x9e3779b9u) out[0] = x;  // keeps the chains alive
}

template <int OP>
cudaError_t run_probe(int sms, double *ops_s) {
  unsigned *out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  const int threads = 256, blocks = sms * 8, iters = 2048;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe<OP><<<blocks, threads>>>(8, out, 1u);
  cudaEventRecord(e0);
  k_probe<OP><<<blocks, threads>>>(iters, out, 1u);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess) *ops_s = (double)blocks * threads * iters * 16.0 * 8.0 / (ms * 1e-3);
  return e;
}

}  // namespace

extern "C" int msa_probe_int_rate(int op, double *ops_per_sec_out, double *ops_per_clk_sm_out) {
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MSA_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  double rate = 0.0;
  cudaError_t e;
  switch (op) {
    case MSA_PROBE_VIADDMAX_S16X2: e = run_probe<MSA_PROBE_VIADDMAX_S16X2>(sms, &rate); break;
    case MSA_PROBE_VIMAX3_S16X2: e = run_probe<MSA_PROBE_VIMAX3_S16X2>(sms, &rate); break;
    case MSA_PROBE_VIADDMAX_S32: e = run_probe<MSA_PROBE_VIADDMAX_S32>(sms, &rate); break;
    case MSA_PROBE_PRMT: e = run_probe<MSA_PROBE_PRMT>(sms, &rate); break;
    default: return MSA_EINVAL;
  }
  if (e != cudaSuccess) return MSA_ECUDA;
  if (ops_per_sec_out) *ops_per_sec_out = rate;
  if (ops_per_clk_sm_out) *ops_per_clk_sm_out = rate / (double)sms / ((double)khz * 1e3);
  return MSA_OK;
}
