// hpcg_probe.cu -- measurement aid: the issue rate of FP64 fused multiply-adds
// on this GPU, the denominator of the FP64 term of the binding roofline that
// the benchmark reports beside the HBM term (the FP64 pipe is narrow on this
// GPU, so FP64 instruction counts can bind before bytes do).
#include <cuda_runtime.h>

#include "hpcg.h"
#include "hpcg_ctx.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent FMA chains per thread (hides the FMA latency)

// Every thread runs kProbeChains chains of `iters` dependent FMAs each; the
// values stay finite (a contraction towards 1e-6 / (1 - 0.999999)) and their
// sum is stored, so no FMA can be dropped by the compiler.
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(int iters, double *sink) {
  double a[kProbeChains];
  const double m = 0.999999, c = 1e-6;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  sink[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int hpcg_probe_fp64_rate(int blocks, int iters, double *sink_dev, double *ms_host, double *fma_host, void *stream) {
  if (blocks < 1 || iters < 1 || !sink_dev || !ms_host || !fma_host) return HPCG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  int rc = HPCG_OK;
  k_fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, sink_dev);  // warm-up (clocks, instruction cache)
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEventRecord(e0, s);
  k_fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, sink_dev);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) rc = cuda_fail(e, "k_fp64_fma_probe");
  *ms_host = ms;
  *fma_host = (double)blocks * kProbeThreads * kProbeChains * (double)iters;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// ---------------------------------------------------------------------------
// Diagnostic: the integer-pipe int64 -> FP64 conversion of the fixed-point and
// block-floating-point kernels, beside CUDA's own conversion.
#include "hpcg_fixed.cuh"

namespace {
__global__ void k_fx_to_double_check(long n, const long long *__restrict__ q, const int *__restrict__ e, double *__restrict__ out,
                                     double *__restrict__ ref) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = hpcg::fx_to_double(q[i], e[i]);
  ref[i] = ldexp(__ll2double_rn(q[i]), e[i] - 1080);  // rounded once, then scaled exactly by a power of two
}
}  // namespace

extern "C" int hpcg_fx_to_double_check(long n, const long long *q_dev, const int *e_dev, double *out_dev, double *ref_dev,
                                       void *stream) {
  if (n < 0 || (n > 0 && (!q_dev || !e_dev || !out_dev || !ref_dev))) return HPCG_ERR_INVALID_ARG;
  if (n == 0) return HPCG_OK;
  k_fx_to_double_check<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, q_dev, e_dev, out_dev, ref_dev);
  CKL("k_fx_to_double_check");
  return HPCG_OK;
}
