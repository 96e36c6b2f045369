// noalloc.cu -- nb_forces_fp64_noalloc: FP64 direct-sum forces for callers
// that cannot allocate device memory.
//
// Who needs it: applications that own every byte of device memory themselves
// (a host framework with its own memory pool that does not allow a library to
// call cudaMalloc behind its back) and latency-critical loops in which a
// cudaMalloc/cudaFree could stall the device or fail part-way through a run.
// Such a caller cannot use nb_create, which allocates the context's arrays.
//
// This entry point takes the caller's device buffers directly and allocates
// nothing.  The split-j partial sums it needs live in one file-scope
// __device__ array (NB_NOALLOC_SCRATCH_DOUBLES doubles, 32 MiB, held by every
// GPU that loads the library until the process exits).  Host code may not use
// that array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress while that device is current
// and keeps it (a one-time set-up; make that first call before any stream
// capture).  The address is kept together with the unique id of the CUDA
// context it was looked up in: after a device reset (a new primary context,
// where the module and its array may be loaded elsewhere) the next call sees
// a different id and looks the address up again instead of writing to a
// freed one.  Every call shares the array and it keeps the previous call's
// contents; the kernels write every partial they later read, so nothing has to
// start at zero.  Calls whose work overlaps on the GPU (different streams, no
// ordering between them) race on the array and must not be issued.
#include <mutex>

#include "nb_internal.cuh"

namespace {

constexpr int kNT = 128;  // i-particles per CTA (one per thread)
constexpr int kJT = 64;   // j-particles per shared-memory tile
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_scratch[NB_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices];               // device address of g_scratch, per device
unsigned long long g_scratch_ctx[kMaxDevices];    // id of the context it belongs to

// the current CUDA context's unique id (driver API, reached through the
// runtime's entry-point query so the library needs no link to libcuda);
// 0 when it cannot be read, which forces a fresh look-up on every call
unsigned long long current_context_id() {
  typedef int (*get_current_fn)(void**);
  typedef int (*get_id_fn)(void*, unsigned long long*);
  static get_current_fn get_current = nullptr;
  static get_id_fn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (get_current_fn)f1;
      get_id = (get_id_fn)f2;
    }
    cudaGetLastError();
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Same pairwise sums as the library's FP64 path (Sec. 4.1 step 4, Eq. 3),
// reading row-major [N][3] caller arrays: CTA (x, y) = (i-tile, j-split);
// partial sums of split y go to part[y][7][pstride], in FP64 with per-tile
// partials folded by TwoSum.  The self pair (j == i) is excluded by index.
__global__ void __launch_bounds__(kNT) noalloc_force_kernel(int64_t N, const double* __restrict__ m,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ v, double eps2,
                                                            const int32_t* __restrict__ list, int64_t n,
                                                            int64_t j_per_split, double* __restrict__ part,
                                                            int64_t pstride) {
  __shared__ double sx[3][kJT], sv[3][kJT], sm[kJT];
  const int tid = threadIdx.x;
  const int64_t pos0 = (int64_t)blockIdx.x * kNT + tid;
  const int64_t pos = pos0 < n ? pos0 : n - 1;
  int64_t self = list[pos];
  self = self < 0 ? 0 : (self >= N ? N - 1 : self);
  double xi[3], vi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xi[c] = x[3 * self + c];
    vi[c] = v[3 * self + c];
  }
  double hi[7], lo[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) hi[c] = lo[c] = 0.0;
  const int64_t jlo = (int64_t)blockIdx.y * j_per_split;
  const int64_t jhi = min(jlo + j_per_split, N);
  for (int64_t jt = jlo; jt < jhi; jt += kJT) {
    __syncthreads();
    for (int q = tid; q < kJT; q += kNT) {
      const int64_t j = jt + q;
      const bool in = j < jhi;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sx[c][q] = in ? x[3 * j + c] : 1.0e15;
        sv[c][q] = in ? v[3 * j + c] : 0.0;
      }
      sm[q] = in ? m[j] : 0.0;
    }
    __syncthreads();
    double p[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) p[c] = 0.0;
    for (int q = 0; q < kJT; ++q) {
      const double dx = sx[0][q] - xi[0], dy = sx[1][q] - xi[1], dz = sx[2][q] - xi[2];
      const double wx = sv[0][q] - vi[0], wy = sv[1][q] - vi[1], wz = sv[2][q] - vi[2];
      const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
      const double rw = fma(dz, wz, fma(dy, wy, dx * wx));
      const double rinv = (jt + q == self) ? 0.0 : nb_rsqrt_fp64(r2);
      const double rinv2 = rinv * rinv;
      const double mr = sm[q] * rinv;
      const double mr3 = mr * rinv2;
      const double a3 = (rw * -3.0) * rinv2;
      p[6] += mr;
      p[0] = fma(mr3, dx, p[0]);
      p[1] = fma(mr3, dy, p[1]);
      p[2] = fma(mr3, dz, p[2]);
      p[3] = fma(mr3, fma(a3, dx, wx), p[3]);
      p[4] = fma(mr3, fma(a3, dy, wy), p[4]);
      p[5] = fma(mr3, fma(a3, dz, wz), p[5]);
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      const double s = hi[c] + p[c];
      const double bp = s - hi[c];
      lo[c] += (hi[c] - (s - bp)) + (p[c] - bp);
      hi[c] = s;
    }
  }
  if (pos0 >= n) return;
  double* o = part + (int64_t)blockIdx.y * 7 * pstride;
#pragma unroll
  for (int c = 0; c < 7; ++c) o[c * pstride + pos0] = hi[c] + lo[c];
}

// sum the splits in a fixed order and write the caller's [n][3] outputs
__global__ void noalloc_reduce_kernel(const double* __restrict__ part, int64_t pstride, int nsplit, int64_t n,
                                      double* __restrict__ acc, double* __restrict__ jerk,
                                      double* __restrict__ pot) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double s[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double t = 0.0;
      for (int q = 0; q < nsplit; ++q) t += part[((int64_t)q * 7 + c) * pstride + k];
      s[c] = t;
    }
    if (acc)
      for (int c = 0; c < 3; ++c) acc[3 * k + c] = s[c];
    if (jerk)
      for (int c = 0; c < 3; ++c) jerk[3 * k + c] = s[3 + c];
    if (pot) pot[k] = -s[6];
  }
}

// device address of the scratch array for the current device (set up once)
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NB_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx_id = current_context_id();
  if (!g_scratch_ptr[dev] || ctx_id == 0 || ctx_id != g_scratch_ctx[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return NB_ECUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
    g_scratch_ctx[dev] = ctx_id;
  }
  *out = g_scratch_ptr[dev];
  return NB_OK;
}

}  // namespace

extern "C" int nb_forces_fp64_noalloc(int64_t N, const double* m, const double* x, const double* v, double eps,
                                      const int32_t* i_idx, int64_t n, double* acc, double* jerk, double* pot,
                                      void* cuda_stream) {
  if (N < 1 || n < 0 || n > N || !m || !x || !v || (n > 0 && !i_idx) || !(eps >= 0.0)) return NB_EINVAL;
  if (n > NB_NOALLOC_MAX_ACTIVE) return NB_EINVAL;  // the partial sums would not fit the fixed scratch
  if (n == 0) return NB_OK;
  double* scratch = nullptr;
  int r = scratch_for_current_device(&scratch);
  if (r != NB_OK) return r;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return NB_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int64_t itiles = (n + kNT - 1) / kNT;
  const int64_t pstride = ((n + 31) / 32) * 32;
  const int64_t tiles = (N + kJT - 1) / kJT;
  // enough CTAs for about four waves, at least one j-tile per split, within the scratch
  int64_t nsplit = (16 * (int64_t)sms + itiles - 1) / itiles;
  const int64_t cap = NB_NOALLOC_SCRATCH_DOUBLES / (7 * pstride);
  if (nsplit > cap) nsplit = cap;
  if (nsplit > tiles) nsplit = tiles;
  if (nsplit > 4096) nsplit = 4096;
  if (nsplit < 1) nsplit = 1;
  const int64_t tps = (tiles + nsplit - 1) / nsplit;
  nsplit = (tiles + tps - 1) / tps;
  noalloc_force_kernel<<<dim3((unsigned)itiles, (unsigned)nsplit), kNT, 0, s>>>(N, m, x, v, eps * eps, i_idx, n,
                                                                                tps * kJT, scratch, pstride);
  if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
  int g = (int)((n + 255) / 256);
  if (g > 8 * sms) g = 8 * sms;
  noalloc_reduce_kernel<<<g, 256, 0, s>>>(scratch, pstride, (int)nsplit, n, acc, jerk, pot);
  if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
  return NB_OK;
}
