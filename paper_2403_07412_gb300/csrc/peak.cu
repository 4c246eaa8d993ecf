// FP64 FMA throughput of this GPU: the roofline denominator for the likelihood
// kernels, which are bound by the FP64 pipe.  Each thread runs eight independent
// register-resident DFMA chains; four warps per SM are launched per block so every
// SM sub-partition has a warp issuing DFMAs, and enough blocks to cover each SM twice.
#include <algorithm>

#include "common.cuh"

namespace vecchia {

__global__ void __launch_bounds__(256) dfma_chain_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-9 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace vecchia

extern "C" int vecchia_fp64_peak(double* gflops_out, void* stream) {
  using namespace vecchia;
  if (!gflops_out) return VECCHIA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 2, iters = 8192;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * threads * blocks) != cudaSuccess) return VECCHIA_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = VECCHIA_OK;
  for (int rep = 0; rep < 4 && !rc; ++rep) {
    cudaEventRecord(e0, s);
    dfma_chain_kernel<<<blocks, threads, 0, s>>>(buf, iters, 1.0000000001, 1e-9);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = VECCHIA_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  if (!rc && cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  const double flops = 2.0 * 8.0 * iters * (double)threads * blocks;
  *gflops_out = flops / (best * 1e-3) / 1e9;
  return VECCHIA_OK;
}
