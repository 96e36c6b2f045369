// peaks.cu -- nb_measure_peaks: arithmetic throughput of the current GPU
// measured with dependent FMA chains (FP32 and FP64) and the hardware rsqrt,
// the denominators of the force kernels' rooflines (the FP64 force path is
// bound by the FP64 pipe, which on GB300 runs at 1/64 of the FP32 rate).
#include "nb_internal.cuh"

namespace {

constexpr int kBlocksPerSM = 8, kThreads = 256;

__global__ void ffma_loop(float* out, int iters, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
        x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
      x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dfma_loop(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

__global__ void rsqrt_loop(float* out, int iters) {
  float x0 = 1.0f + threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = nb_rsqrt_approx(x0); x1 = nb_rsqrt_approx(x1); x2 = nb_rsqrt_approx(x2); x3 = nb_rsqrt_approx(x3);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

}  // namespace

extern "C" int nb_measure_peaks(nb_ctx* c, double* fp32_tflops, double* fp64_tflops, double* rsqrt_tops) {
  if (!c) return NB_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return NB_ECUDA;
  const int blocks = c->sm_count * kBlocksPerSM;
  // scratch for the loop results: the split-j partial buffer (at least 2^21 doubles)
  float* fo = (float*)c->part;
  double* dout = c->part;
  cudaEvent_t e0 = c->ev[6], e1 = c->ev[7];
  float ms = 0.0f;
  const double threads = (double)blocks * kThreads;
  // FP32: 8 chains x 16 FMA x iters per thread
  const int it32 = 4000, it64 = 200, itr = 2000;
  ffma_loop<<<blocks, kThreads, 0, c->stream>>>(fo, 10, 0.999f, 0.001f);
  cudaEventRecord(e0, c->stream);
  ffma_loop<<<blocks, kThreads, 0, c->stream>>>(fo, it32, 0.999f, 0.001f);
  cudaEventRecord(e1, c->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return NB_ECUDA;
  if (fp32_tflops) *fp32_tflops = 2.0 * 8 * 16 * it32 * threads / (ms * 1e-3) / 1e12;
  dfma_loop<<<blocks, kThreads, 0, c->stream>>>(dout, 2, 0.999, 0.001);
  cudaEventRecord(e0, c->stream);
  dfma_loop<<<blocks, kThreads, 0, c->stream>>>(dout, it64, 0.999, 0.001);
  cudaEventRecord(e1, c->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return NB_ECUDA;
  if (fp64_tflops) *fp64_tflops = 2.0 * 4 * 16 * it64 * threads / (ms * 1e-3) / 1e12;
  rsqrt_loop<<<blocks, kThreads, 0, c->stream>>>(fo, 2);
  cudaEventRecord(e0, c->stream);
  rsqrt_loop<<<blocks, kThreads, 0, c->stream>>>(fo, itr);
  cudaEventRecord(e1, c->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return NB_ECUDA;
  if (rsqrt_tops) *rsqrt_tops = 4.0 * 16 * itr * threads / (ms * 1e-3) / 1e12;
  c->launches += 6;
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ECUDA;
}
