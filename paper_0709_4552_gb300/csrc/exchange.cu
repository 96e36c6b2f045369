// exchange.cu -- device side of the calls the parallel algorithms of Sec. 4.2
// (copy) and Sec. 4.3 (ring) make on each rank's context (entry points in
// capi.cu, driver in the package's distributed module):
//   - particles gathered from / scattered into the state by particle index
//     (the copy algorithm's all-gather of the corrected block);
//   - the visiting block of the ring algorithm -- predicted positions and
//     velocities of particles held by another rank -- put into i-arrays the
//     force items read (force_common.cuh ISrc), with the j-store slot of each
//     particle this rank holds, so that the self pair stays excluded;
//   - force rows copied out, or added onto the block's running sums.
#include "force_common.cuh"

namespace {

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

__global__ void gather_slots_kernel(const int32_t* __restrict__ slots, int64_t n, int64_t n_pad,
                                    const double* __restrict__ src, int rows, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = slots[k];
    s = s < 0 ? 0 : (s >= n_pad ? n_pad - 1 : s);
    for (int r = 0; r < rows; ++r) dst[k * rows + r] = src[r * n_pad + s];
  }
}

__global__ void scatter_slots_kernel(const int32_t* __restrict__ slots, int64_t n, int64_t n_pad,
                                     const double* __restrict__ src, int rows, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = slots[k];
    s = s < 0 ? 0 : (s >= n_pad ? n_pad - 1 : s);
    for (int r = 0; r < rows; ++r) dst[r * n_pad + s] = src[k * rows + r];
  }
}

// the visiting block: SoA FP64 rows, the double-single split of the mixed
// path (hi = fl32(x), lo = fl32(x - hi), as the predictor writes), the list
// of positions and each particle's slot here (or -1)
__global__ void ext_prepare_kernel(int64_t n, int64_t cap, const double* __restrict__ xi,
                                   const double* __restrict__ vi, const int64_t* __restrict__ gid, int64_t base,
                                   int64_t N, const int32_t* __restrict__ iperm, double* __restrict__ ex,
                                   double* __restrict__ ev, float4* __restrict__ eA, float4* __restrict__ eB,
                                   float2* __restrict__ eC, int32_t* __restrict__ eself,
                                   int32_t* __restrict__ eident) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float hi[3], lo[3], vf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = xi[3 * k + c], v = vi[3 * k + c];
      ex[c * cap + k] = x;
      ev[c * cap + k] = v;
      hi[c] = __double2float_rn(x);
      lo[c] = __double2float_rn(x - (double)hi[c]);
      vf[c] = __double2float_rn(v);
    }
    eA[k] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    eB[k] = make_float4(lo[0], lo[1], lo[2], vf[0]);
    eC[k] = make_float2(vf[1], vf[2]);
    const int64_t local = gid ? gid[k] - base : -1;
    eself[k] = (local >= 0 && local < N) ? (iperm ? iperm[local] : (int32_t)local) : -1;
    eident[k] = (int32_t)k;
  }
}

// acc, jerk [n][3] and pot [n] from the force rows F[7][fstride]; added to
// what the outputs hold when accumulate != 0
__global__ void forces_out_kernel(int64_t n, const double* __restrict__ F, int64_t fstride, double* __restrict__ acc,
                                  double* __restrict__ jerk, double* __restrict__ pot, int accumulate) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (acc) acc[3 * k + c] = accumulate ? acc[3 * k + c] + F[c * fstride + k] : F[c * fstride + k];
      if (jerk) jerk[3 * k + c] = accumulate ? jerk[3 * k + c] + F[(3 + c) * fstride + k] : F[(3 + c) * fstride + k];
    }
    if (pot) pot[k] = accumulate ? pot[k] + F[6 * fstride + k] : F[6 * fstride + k];
  }
}

}  // namespace

cudaError_t nb_launch_gather_slots(nb_ctx* c, const int32_t* slots, int64_t n, const double* src, int rows,
                                   double* dst) {
  if (n <= 0) return cudaSuccess;
  c->launches += 1;
  gather_slots_kernel<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(slots, n, c->n_pad, src, rows, dst);
  return cudaGetLastError();
}

cudaError_t nb_launch_scatter_slots(nb_ctx* c, const int32_t* slots, int64_t n, const double* src, int rows,
                                    double* dst) {
  if (n <= 0) return cudaSuccess;
  c->launches += 1;
  scatter_slots_kernel<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(slots, n, c->n_pad, src, rows,
                                                                                   dst);
  return cudaGetLastError();
}

cudaError_t nb_ext_reserve(nb_ctx* c, int64_t n) {
  if (n <= c->ext_cap) return cudaSuccess;
  void* ps[] = {c->ext_x, c->ext_v, c->ext_A, c->ext_B, c->ext_C, c->ext_self, c->ext_ident, c->ext_gid};
  for (void* p : ps)
    if (p) cudaFree(p);
  c->ext_x = c->ext_v = nullptr;
  c->ext_A = c->ext_B = nullptr;
  c->ext_C = nullptr;
  c->ext_self = c->ext_ident = nullptr;
  c->ext_gid = nullptr;
  c->ext_cap = 0;
  const int64_t cap = ((n + 1023) / 1024) * 1024;
  cudaError_t e = cudaMalloc((void**)&c->ext_x, 3 * cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_v, 3 * cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_A, cap * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_B, cap * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_C, cap * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_self, cap * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_ident, cap * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->ext_gid, cap * sizeof(int64_t));
  if (e == cudaSuccess) c->ext_cap = cap;
  return e;
}

cudaError_t nb_launch_ext_prepare(nb_ctx* c, int64_t n, const double* xi, const double* vi, const int64_t* gid,
                                  int64_t base) {
  if (n <= 0) return cudaSuccess;
  c->launches += 1;
  ext_prepare_kernel<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
      n, c->ext_cap, xi, vi, gid, base, c->n, c->perm_valid ? c->iperm : nullptr, c->ext_x, c->ext_v, c->ext_A,
      c->ext_B, c->ext_C, c->ext_self, c->ext_ident);
  return cudaGetLastError();
}

cudaError_t nb_forces_ext(nb_ctx* c, int64_t n, const nb_tuning& cfg) {
  nbk::ISrc is;
  is.A = c->ext_A;
  is.B = c->ext_B;
  is.C = c->ext_C;
  is.x = c->ext_x;
  is.v = c->ext_v;
  is.stride = c->ext_cap;
  is.self = c->ext_self;
  return c->precision == NB_FP64 ? nb_forces_fp64(c, c->ext_ident, n, cfg, &is)
                                 : nb_forces_mixed(c, c->ext_ident, n, cfg, nullptr, &is);
}

cudaError_t nb_launch_forces_out(nb_ctx* c, int64_t n, double* acc, double* jerk, double* pot, int accumulate) {
  if (n <= 0) return cudaSuccess;
  c->launches += 1;
  forces_out_kernel<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(n, c->F, c->n_pad, acc, jerk, pot,
                                                                                accumulate);
  return cudaGetLastError();
}
