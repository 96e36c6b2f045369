// spatial.cu -- spatial (Morton) order of the mixed path's j-store.
//
// The mixed force kernel forms position differences from double-single pairs
// (9 FP32 adds per pair).  When a warp's i-particles and a j-tile are far apart
// compared with their distance from the origin, the FP32 "hi" parts alone give
// the difference to FP32 accuracy (1 add per coordinate).  That needs warps
// and tiles that are spatially compact, so the predictor writes the j-store
// in Morton order of the particles' positions (perm[slot] = particle) and the
// block selection lists active particles in the same order.  The order is a
// pure layout choice: every sum is over the same pairs.
//
// nb_spatial_sort: bounding box -> 30-bit Morton keys on a 1024^3 grid ->
// stable least-significant-digit radix sort (4 passes of 8 bits; per-block
// digit histograms, one scan, stable scatter ranked with warp match) ->
// perm and its inverse.  Deterministic.
// nb_launch_tile_boxes: per j-tile of 128 slots, the box of the FP32 hi
// positions of its real particles and their largest |coordinate|.
#include <float.h>

#include "nb_internal.cuh"

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                          // elements per thread per block
constexpr int kSortChunk = kSortThreads * kSortItems;  // 2048 elements per block
constexpr int kRadix = 256;

__global__ void bbox_partial(int64_t N, int64_t n_pad, const double* __restrict__ x, double* __restrict__ red) {
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) {
      const double v = x[c * n_pad + i];
      lo[c] = fmin(lo[c], v);
      hi[c] = fmax(hi[c], v);
    }
  __shared__ double s[6][kSortThreads];
  for (int c = 0; c < 3; ++c) {
    s[c][threadIdx.x] = lo[c];
    s[3 + c][threadIdx.x] = hi[c];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) {
        s[c][threadIdx.x] = fmin(s[c][threadIdx.x], s[c][threadIdx.x + w]);
        s[3 + c][threadIdx.x] = fmax(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) red[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void bbox_final(int nb, double* __restrict__ red, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double b[6] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int k = 0; k < nb; ++k)
      for (int c = 0; c < 3; ++c) {
        b[c] = fmin(b[c], red[k * 6 + c]);
        b[3 + c] = fmax(b[3 + c], red[k * 6 + 3 + c]);
      }
    for (int c = 0; c < 6; ++c) out[c] = b[c];
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t a) {  // 10 bits -> every third bit
  a &= 0x3FFu;
  a = (a | (a << 16)) & 0x030000FFu;
  a = (a | (a << 8)) & 0x0300F00Fu;
  a = (a | (a << 4)) & 0x030C30C3u;
  a = (a | (a << 2)) & 0x09249249u;
  return a;
}

__global__ void morton_keys(int64_t N, int64_t n_pad, const double* __restrict__ x, const double* __restrict__ box,
                            uint32_t* __restrict__ key, int32_t* __restrict__ val) {
  double scale = fmax(box[3] - box[0], fmax(box[4] - box[1], box[5] - box[2]));
  scale = scale > 0.0 ? 1023.0 / scale : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t q[3];
    for (int c = 0; c < 3; ++c) {
      double f = (x[c * n_pad + i] - box[c]) * scale;
      f = f < 0.0 ? 0.0 : (f > 1023.0 ? 1023.0 : f);
      q[c] = (uint32_t)f;
    }
    key[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    val[i] = (int32_t)i;
  }
}

__global__ void radix_count(const uint32_t* __restrict__ key, int64_t N, int shift, int32_t* __restrict__ hist,
                            int nblocks) {
  __shared__ int cnt[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortChunk;
  for (int it = 0; it < kSortItems; ++it) {
    const int64_t e = base + it * kSortThreads + threadIdx.x;
    if (e < N) atomicAdd(&cnt[(key[e] >> shift) & 0xFFu], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// exclusive scan of n ints in one CTA of 1024 threads
__global__ void scan_exclusive(int32_t* __restrict__ a, int64_t n) {
  __shared__ int32_t s[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < n; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const int32_t v = i < n ? a[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int32_t add = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) a[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
}

// stable scatter: elements of a block keep their order among equal digits
__global__ void radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                              uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t N, int shift,
                              const int32_t* __restrict__ hist, int nblocks) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ int32_t base[kRadix];
  __shared__ int32_t wcnt[kWarps][kRadix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) base[d] = hist[(int64_t)d * nblocks + blockIdx.x];
  const int64_t chunk = (int64_t)blockIdx.x * kSortChunk;
  for (int it = 0; it < kSortItems; ++it) {
    for (int q = threadIdx.x; q < kWarps * kRadix; q += blockDim.x) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t e = chunk + it * kSortThreads + threadIdx.x;
    const bool valid = e < N;
    const uint32_t k = valid ? kin[e] : 0u;
    const int digit = valid ? (int)((k >> shift) & 0xFFu) : kRadix;  // kRadix: no element
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[wid][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      int off = 0;
      for (int w = 0; w < wid; ++w) off += wcnt[w][digit];
      const int64_t pos = (int64_t)base[digit] + off + rank;
      kout[pos] = k;
      vout[pos] = vin[e];
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
      int t = 0;
      for (int w = 0; w < kWarps; ++w) t += wcnt[w][d];
      base[d] += t;
    }
    __syncthreads();
  }
}

__global__ void invert_perm(int64_t N, const int32_t* __restrict__ perm, int32_t* __restrict__ iperm) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    iperm[perm[k]] = (int32_t)k;
}

// box of tile t (slots [t*JT, t*JT+JT) intersected with [0, N)): (lo, rmax), (hi, 0)
template <int JT>
__global__ void tile_boxes(int64_t N, int64_t ntiles, const float4* __restrict__ jA, float4* __restrict__ box) {
  const int64_t t = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX}, r = 0.0f;
  for (int q = lane; q < JT; q += 32) {
    const int64_t s = t * JT + q;
    if (s >= N) break;
    const float4 a = jA[s];
    const float p[3] = {a.x, a.y, a.z};
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], p[c]);
      hi[c] = fmaxf(hi[c], p[c]);
      r = fmaxf(r, fabsf(p[c]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
    r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
  }
  if (lane == 0) {
    box[2 * t] = make_float4(lo[0], lo[1], lo[2], r);
    box[2 * t + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
  }
}

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// keys: slot of each listed particle (clamped); values: list positions
__global__ void list_keys(const int32_t* __restrict__ list, int64_t n, const int32_t* __restrict__ iperm,
                          int64_t N, uint32_t* __restrict__ key, int32_t* __restrict__ val) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = list[k];
    p = p < 0 ? 0 : (p >= N ? N - 1 : p);
    key[k] = (uint32_t)iperm[p];
    val[k] = (int32_t)k;
  }
}

// stable LSD radix sort of (skey[0], sval[0])[0..n) on the low `bits` bits;
// *cur = the buffer holding the result
cudaError_t sort_pairs(nb_ctx* c, int64_t n, int bits, int* cur) {
  const int nblocks = (int)((n + kSortChunk - 1) / kSortChunk);
  int b = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_count<<<nblocks, kSortThreads, 0, c->stream>>>(c->skey[b], n, shift, c->shist, nblocks);
    scan_exclusive<<<1, 1024, 0, c->stream>>>(c->shist, (int64_t)nblocks * kRadix);
    radix_scatter<<<nblocks, kSortThreads, 0, c->stream>>>(c->skey[b], c->sval[b], c->skey[b ^ 1], c->sval[b ^ 1],
                                                           n, shift, c->shist, nblocks);
    b ^= 1;
    c->launches += 3;
  }
  *cur = b;
  return cudaGetLastError();
}

}  // namespace

cudaError_t nb_spatial_sort(nb_ctx* c) {
  const int64_t N = c->n;
  if (N <= 0) return cudaSuccess;
  const int nbb = grid_for(N, kSortThreads, 1024);
  double* box = c->red + NB_BBOX_OFFSET;
  bbox_partial<<<nbb, kSortThreads, 0, c->stream>>>(N, c->n_pad, c->x, c->red);
  bbox_final<<<1, 32, 0, c->stream>>>(nbb, c->red, box);
  morton_keys<<<grid_for(N, 256, c->sm_count * 16), 256, 0, c->stream>>>(N, c->n_pad, c->x, box, c->skey[0],
                                                                         c->sval[0]);
  int cur = 0;
  cudaError_t e = sort_pairs(c, N, 30, &cur);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(c->perm, c->sval[cur], N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  invert_perm<<<grid_for(N, 256, c->sm_count * 16), 256, 0, c->stream>>>(N, c->perm, c->iperm);
  c->launches += 4;
  return cudaGetLastError();
}

// Processing order of a caller's active list in the spatial order: list
// positions sorted by the j-store slot of their particle (stable).  The
// mixed kernel then forms warps of nearby particles; results still go to the
// caller's positions.  Returns a device array of n positions.
cudaError_t nb_list_order(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** ord) {
  list_keys<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(d_list, n, c->iperm, c->n, c->skey[0],
                                                                       c->sval[0]);
  int bits = 1;
  while (bits < 31 && ((int64_t)1 << bits) < c->n) ++bits;
  int cur = 0;
  cudaError_t e = sort_pairs(c, n, bits, &cur);
  if (e != cudaSuccess) return e;
  c->launches += 1;
  *ord = c->sval[cur];
  return cudaGetLastError();
}

cudaError_t nb_launch_tile_boxes(nb_ctx* c) {
  const int64_t ntiles = (c->n + NB_BOX_TILE - 1) / NB_BOX_TILE;
  if (ntiles <= 0) return cudaSuccess;
  const int warps = 8;
  tile_boxes<NB_BOX_TILE><<<(unsigned)((ntiles + warps - 1) / warps), warps * 32, 0, c->stream>>>(c->n, ntiles, c->jA,
                                                                                                    c->tbox);
  c->launches += 1;
  return cudaGetLastError();
}
