// FP64 issue-rate probe: the denominator of the roofline of the FP64 kernels.
//
// On this GPU every FP64 stage of the path is bound by FP64 instruction issue
// rather than by HBM, so each kernel's fraction of its bound needs the FP64
// rate the device actually delivers. The probe runs independent chains of
// dependent fused multiply-adds, eight per thread (enough to cover the FP64
// latency with sixteen warps per SM), two 256-thread blocks per SM, and times
// them with CUDA events on the context's stream. An FMA counts as one FP64
// operation, as in the operation counts of the kernels.
#include "afid_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma_chains(int iters, double b, double c,
                                                              double* __restrict__ sink) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3 * (threadIdx.x + 1) + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  // every warp stores its sum, so no chain can be dropped as dead code
  if ((threadIdx.x & 31) == 0) sink[blockIdx.x * (kThreads / 32) + threadIdx.x / 32] = s;
}

}  // namespace

extern "C" afid_status afid_probe_fp64_rate(afid_ctx* c, int iters, double* ops_per_s, double* ms_out) {
  if (!c || !ops_per_s || iters < 1) return AFID_ERR_INVALID_ARG;
  const int blocks = 2 * c->num_sms;
  if ((size_t)blocks * (kThreads / 32) > (size_t)3 * c->part_len) return AFID_ERR_INVALID_ARG;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AFID_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AFID_ERR_CUDA;
  }
  // b, c keep the chains bounded: a -> a b + c converges to c / (1 - b)
  const double b = 0.999999, cc = 1e-7;
  bool ok = true;
  k_fp64_fma_chains<<<blocks, kThreads, 0, c->stream>>>(iters / 8 + 1, b, cc, c->part);  // warm-up
  ok = ok && cudaEventRecord(e0, c->stream) == cudaSuccess;
  k_fp64_fma_chains<<<blocks, kThreads, 0, c->stream>>>(iters, b, cc, c->part);
  ok = ok && cudaEventRecord(e1, c->stream) == cudaSuccess;
  ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
  float ms = 0.f;
  ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->launches += 2;
  if (!ok || cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return AFID_ERR_CUDA;
  const double ops = (double)blocks * kThreads * kChains * (double)iters;
  *ops_per_s = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return AFID_OK;
}
