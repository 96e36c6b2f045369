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

// one CTA: each warp runs `iters` FP64 FMAs on lanes < active, in `ilp`
// independent chains (1 or 4), timed by the SM clock; per-warp cycles to cyc
__global__ void dfma_issue(long long* cyc, double* out, int iters, int active, int ilp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  const double a = 0.999999, b = 1e-7;
  __syncthreads();
  const long long t0 = clock64();
  if (lane < active) {
    if (ilp == 1) {
      for (int i = 0; i < iters; ++i) x0 = fma(x0, a, b);
    } else {
      for (int i = 0; i < iters; i += 4) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      }
    }
  }
  __syncwarp();
  const long long t1 = clock64();
  out[threadIdx.x] = x0 + x1 + x2 + x3;
  if (lane == 0) cyc[w] = t1 - t0;
}

}  // namespace

// cycles per FP64 FMA of the probe dfma_issue in a warp layout (the largest
// warp's count over the instructions each warp issued)
static int fp64_issue_case(nb_ctx* c, int warps, int active, int ilp, double* cycles) {
  const int iters = 4096;
  long long* cyc = reinterpret_cast<long long*>(c->part);
  double* out = c->part + 64;
  for (int rep = 0; rep < 2; ++rep) dfma_issue<<<1, 32 * warps, 0, c->stream>>>(cyc, out, iters, active, ilp);
  long long h[32] = {0};
  if (cudaMemcpyAsync(h, cyc, sizeof(long long) * warps, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NB_ECUDA;
  long long mx = 0;
  for (int k = 0; k < warps; ++k) mx = h[k] > mx ? h[k] : mx;
  *cycles = (double)mx / iters;
  c->launches += 2;
  return NB_OK;
}

extern "C" int nb_measure_fp64_issue(nb_ctx* c, double* dep32, double* dep1, double* indep4, double* sm16) {
  if (!c) return NB_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return NB_ECUDA;
  double v[4] = {0, 0, 0, 0};
  int r = fp64_issue_case(c, 1, 32, 1, &v[0]);  // one warp, all lanes, dependent chain
  if (!r) r = fp64_issue_case(c, 1, 1, 1, &v[1]);  // one warp, one lane
  if (!r) r = fp64_issue_case(c, 1, 32, 4, &v[2]);  // one warp, four independent chains
  if (!r) r = fp64_issue_case(c, 16, 32, 1, &v[3]);  // 16 warps on one SM
  if (r) {
    cudaGetLastError();
    return r;
  }
  if (dep32) *dep32 = v[0];
  if (dep1) *dep1 = v[1];
  if (indep4) *indep4 = v[2];
  if (sm16) *sm16 = v[3] / 16.0;  // SM cycles per warp instruction with 16 warps issuing
  return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ECUDA;
}

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
