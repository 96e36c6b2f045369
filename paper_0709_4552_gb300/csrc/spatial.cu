// spatial.cu -- resident spatial (Morton) order of the mixed path.
//
// The mixed force kernel forms position differences from double-single pairs
// (9 FP32 adds per pair).  When a warp's i-particles and a j-tile are far apart
// compared with their distance from the origin, the FP32 "hi" parts alone give
// the difference to FP32 accuracy (1 add per coordinate).  That needs warps
// and tiles that are spatially compact, so the particle arrays are kept in
// Morton order of the positions (row s holds particle perm[s]): the predictor,
// block selection, force and corrector kernels then walk rows and every
// access is coalesced, while the j-store and the active lists come out
// spatially ordered.  The order is a pure layout choice: every sum is over
// the same pairs.
//
// nb_spatial_sort: bounding box -> 30-bit Morton keys on a 1024^3 grid ->
// stable least-significant-digit radix sort (4 passes of 8 bits; per-block
// digit histograms, one scan, stable scatter ranked with warp match) -> the
// rows gathered into a scratch block and copied back, perm composed and
// inverted.  Deterministic.
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

// one CTA of kSortThreads: strided partial minima/maxima, then a tree (min
// and max are exact, so the order does not matter)
__global__ void bbox_final(int nb, const double* __restrict__ red, double* __restrict__ out) {
  double b[6] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int k = threadIdx.x; k < nb; k += blockDim.x)
    for (int c = 0; c < 3; ++c) {
      b[c] = fmin(b[c], red[k * 6 + c]);
      b[3 + c] = fmax(b[3 + c], red[k * 6 + 3 + c]);
    }
  __shared__ double s[6][kSortThreads];
  for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = b[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) {
        s[c][threadIdx.x] = fmin(s[c][threadIdx.x], s[c][threadIdx.x + w]);
        s[3 + c][threadIdx.x] = fmax(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = s[threadIdx.x][0];
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
    key[i] = nb_spread10(q[0]) | (nb_spread10(q[1]) << 1) | (nb_spread10(q[2]) << 2);
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

// box of tile t (slots [t*JT, t*JT+JT) intersected with [0, N)): (lo, rmax), (hi, 0);
// an empty intersection gives lo = +FLT_MAX, hi = -FLT_MAX, rmax = 0
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

// keys: the listed slots (clamped); values: list positions
__global__ void list_keys(const int32_t* __restrict__ list, int64_t n, int64_t N, uint32_t* __restrict__ key,
                          int32_t* __restrict__ val) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = list[k];
    p = p < 0 ? 0 : (p >= N ? N - 1 : p);
    key[k] = (uint32_t)p;
    val[k] = (int32_t)k;
  }
}

// the 16 FP64 rows of the master state: m, x[3], v[3], a[3], jerk[3], pot, t, dt
constexpr int kStateRows = 16;
struct StateRows {
  double* row[kStateRows];
};

StateRows state_rows(nb_ctx* c) {
  StateRows r;
  double* arr[8] = {c->m, c->x, c->v, c->a, c->jk, c->pot, c->t, c->dt};
  const int cnt[8] = {1, 3, 3, 3, 3, 1, 1, 1};
  int q = 0;
  for (int i = 0; i < 8; ++i)
    for (int k = 0; k < cnt[i]; ++k) r.row[q++] = arr[i] + (int64_t)k * c->n_pad;
  return r;
}

// scratch[q][s] = row_q[src[s]] for s < N (a gather of every state row)
__global__ void gather_state(int64_t N, int64_t n_pad, StateRows rows, const int32_t* __restrict__ src,
                             double* __restrict__ scratch) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t from = src[s];
#pragma unroll
    for (int q = 0; q < kStateRows; ++q) scratch[q * n_pad + s] = rows.row[q][from];
  }
}

__global__ void copy_state_back(int64_t N, int64_t n_pad, StateRows rows, const double* __restrict__ scratch) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < kStateRows; ++q) rows.row[q][s] = scratch[q * n_pad + s];
}

// out[s] = a[b[s]] (composition of two orders), or b[s] when a is null
__global__ void compose(int64_t N, const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                        int32_t* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
    out[s] = a ? a[b[s]] : b[s];
}

// out[k] = map[in[k]] with in[k] clamped to [0, N) (in == out allowed)
__global__ void map_list(const int32_t* in, int64_t n, const int32_t* __restrict__ map, int64_t N, int32_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = in[k];
    p = p < 0 ? 0 : (p >= N ? N - 1 : p);
    out[k] = map[p];
  }
}

// a caller's list: NB_ST_BADLIST unless ascending within [0, N); with map,
// out[k] = map[in[k]] (in[k] clamped to [0, N))
__global__ void check_map_list(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ map, int64_t N,
                               int32_t* __restrict__ out, unsigned int* __restrict__ flag) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = in[k];
    if (v < 0 || v >= N || (k > 0 && in[k - 1] >= v)) atomicOr(flag, NB_ST_BADLIST);
    if (map) {
      const int64_t p = v < 0 ? 0 : (v >= N ? N - 1 : v);
      out[k] = map[p];
    }
  }
}

// dst[k * rows + r] = src[r * n_pad + iperm[first + k]]
__global__ void gather_rows(const double* __restrict__ src, int rows, int64_t n_pad, const int32_t* __restrict__ iperm,
                            int64_t first, int64_t count, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = iperm[first + k];
    for (int r = 0; r < rows; ++r) dst[k * rows + r] = src[r * n_pad + s];
  }
}

// reorder every state row by src (new row s = old row src[s]) in place
cudaError_t reorder_state(nb_ctx* c, const int32_t* src) {
  c->state_ver++;  // rows move: any row-keyed copy of the state (the j-memory) is stale
  if (!c->pscratch) {
    cudaError_t e = cudaMalloc(&c->pscratch, (size_t)kStateRows * c->n_pad * sizeof(double));
    if (e != cudaSuccess) {
      c->pscratch = nullptr;
      return e;
    }
  }
  const StateRows rows = state_rows(c);
  const int g = grid_for(c->n, 256, c->sm_count * 16);
  gather_state<<<g, 256, 0, c->stream>>>(c->n, c->n_pad, rows, src, c->pscratch);
  copy_state_back<<<g, 256, 0, c->stream>>>(c->n, c->n_pad, rows, c->pscratch);
  c->launches += 2;
  return cudaGetLastError();
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

// stable sort of the rows by the keys in skey[0] (values = row numbers in
// sval[0]) on the low `bits` bits, then the state reordered to that order
cudaError_t nb_order_rows_by_keys(nb_ctx* c, int bits) {
  const int64_t N = c->n;
  int cur = 0;
  cudaError_t e = sort_pairs(c, N, bits, &cur);
  if (e != cudaSuccess) return e;
  // sval[cur][s] = the current row that becomes row s
  const int32_t* sigma = c->sval[cur];
  e = reorder_state(c, sigma);
  if (e != cudaSuccess) return e;
  const int g = grid_for(N, 256, c->sm_count * 16);
  int32_t* np = c->sval[cur ^ 1];
  compose<<<g, 256, 0, c->stream>>>(N, c->perm_valid ? c->perm : nullptr, sigma, np);
  e = cudaMemcpyAsync(c->perm, np, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  invert_perm<<<g, 256, 0, c->stream>>>(N, c->perm, c->iperm);
  c->launches += 2;
  return cudaGetLastError();
}

cudaError_t nb_spatial_sort(nb_ctx* c) {
  const int64_t N = c->n;
  if (N <= 0) return cudaSuccess;
  const int nbb = grid_for(N, kSortThreads, 1024);
  double* box = c->red + NB_BBOX_OFFSET;
  bbox_partial<<<nbb, kSortThreads, 0, c->stream>>>(N, c->n_pad, c->x, c->red);
  bbox_final<<<1, kSortThreads, 0, c->stream>>>(nbb, c->red, box);
  morton_keys<<<grid_for(N, 256, c->sm_count * 16), 256, 0, c->stream>>>(N, c->n_pad, c->x, box, c->skey[0],
                                                                         c->sval[0]);
  c->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return nb_order_rows_by_keys(c, 30);
}

cudaError_t nb_unsort(nb_ctx* c) {
  if (!c->perm_valid) return cudaSuccess;
  // particle p = old row iperm[p]
  cudaError_t e = reorder_state(c, c->iperm);
  if (e != cudaSuccess) return e;
  c->perm_valid = false;
  c->pred_valid = false;
  c->f_valid = false;
  return cudaSuccess;
}

cudaError_t nb_map_to_slots(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** out) {
  if (!c->perm_valid || n <= 0) {
    *out = d_list;
    return cudaSuccess;
  }
  map_list<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(d_list, n, c->iperm, c->n, c->mlist);
  c->launches += 1;
  *out = c->mlist;
  return cudaGetLastError();
}

cudaError_t nb_check_map_to_slots(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** out) {
  if (n <= 0) {
    *out = d_list;
    return cudaSuccess;
  }
  c->launches += 1;
  check_map_list<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(
      d_list, n, c->perm_valid ? c->iperm : nullptr, c->n, c->perm_valid ? c->mlist : nullptr, &c->status->flags);
  *out = c->perm_valid ? c->mlist : d_list;
  return cudaGetLastError();
}

cudaError_t nb_map_to_particles(nb_ctx* c, const int32_t* in, int64_t n, int32_t* out) {
  if (n <= 0) return cudaSuccess;
  if (!c->perm_valid) {
    if (in == out) return cudaSuccess;
    return cudaMemcpyAsync(out, in, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
  }
  map_list<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(in, n, c->perm, c->n, out);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t nb_gather_rows(nb_ctx* c, const double* src, int rows, int64_t first, int64_t count, double* dst) {
  if (count <= 0) return cudaSuccess;
  gather_rows<<<grid_for(count, 256, c->sm_count * 16), 256, 0, c->stream>>>(src, rows, c->n_pad, c->iperm, first,
                                                                             count, dst);
  c->launches += 1;
  return cudaGetLastError();
}

// Processing order of a caller's active list (mapped to slots) in the
// spatial order: list positions sorted by slot (stable).  The mixed kernel
// then forms warps of nearby particles; results still go to the caller's
// positions.  Returns a device array of n positions.
cudaError_t nb_list_order(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** ord) {
  list_keys<<<grid_for(n, 256, c->sm_count * 16), 256, 0, c->stream>>>(d_list, n, c->n, c->skey[0], c->sval[0]);
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
  // every tile up to n_pad (tiles of padding alone get an empty box: always far)
  const int64_t ntiles = c->n > 0 ? c->n_pad / NB_BOX_TILE : 0;
  if (ntiles <= 0) return cudaSuccess;
  const int warps = 8;
  tile_boxes<NB_BOX_TILE><<<(unsigned)((ntiles + warps - 1) / warps), warps * 32, 0, c->stream>>>(c->n, ntiles, c->jA,
                                                                                                    c->tbox);
  c->launches += 1;
  return cudaGetLastError();
}
