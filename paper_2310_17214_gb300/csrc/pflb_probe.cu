// pflb_probe.cu -- device diagnostic: the FP64 FMA rate of the GPU.
//
// The FP64 step and the Newton chemistry are bound by the FP64 pipe, whose
// rate differs widely between GPUs of one generation; the roofline of those
// paths needs it measured.  Each thread runs eight independent FMA chains
// (enough to cover the pipe latency), the grid fills every SM, and the
// kernel is timed with CUDA events.
#include <cuda_runtime.h>

#include "../../include/pflb.h"

namespace {

__global__ void __launch_bounds__(256) fma64_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int pflb_probe_fp64_fma(int device, double* tflops) {
  if (!tflops) return PFLB_ERR_ARG;
  *tflops = 0;
  if (cudaSetDevice(device) != cudaSuccess) return PFLB_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return PFLB_ERR_CUDA;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return PFLB_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, iters = 4096;
  int rc = PFLB_OK;
  float best = -1.f;
  for (int rep = 0; rep < 4 && rc == PFLB_OK; ++rep) {  // first run warms up
    cudaEventRecord(e0);
    fma64_kernel<<<blocks, 256>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    float ms = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = PFLB_ERR_CUDA;
    else if (rep > 0 && (best < 0 || ms < best))
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == PFLB_OK && best > 0)
    *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (best * 1e-3) / 1e12;
  return rc;
}
