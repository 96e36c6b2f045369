// integrator.cu -- the HBM-bound / FP64-bookkeeping kernels around the force
// kernel: predictor (Sec. 4.1 step 3), block selection (step 2), Hermite
// corrector with the power-of-two block-step rule (step 5, block steps of
// Sec. 2), initial steps (step 1), energy reduction, and layout helpers.
#include <math.h>

#include "hermite.cuh"
#include "nb_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int threads, int cap = 1 << 20) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Predictor (Sec. 4.1 step 3) to time t (own_time: h = 0, i.e. t = t_i), for
// i < N; padding particles [N, n_pad) get m = 0 far away.  Arithmetic in
// hermite.cuh.
// ---------------------------------------------------------------------------
__global__ void predict_kernel(int64_t N, int64_t n_pad, const double* __restrict__ m,
                               const double* __restrict__ x, const double* __restrict__ v,
                               const double* __restrict__ a, const double* __restrict__ jk,
                               const double* __restrict__ ti, double t, int own_time,
                               double* __restrict__ xp, double* __restrict__ vp,
                               float4* __restrict__ jA, float4* __restrict__ jB,
                               float2* __restrict__ jC, int write_fp64, int write_mixed) {
  // rows in the resident order: row i of every array is one particle
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
       i += (int64_t)gridDim.x * blockDim.x) {
    double px[3], pv[3], mi;
    if (i < N) {
      mi = m[i];
      nbh::taylor(i, n_pad, own_time ? 0.0 : t - ti[i], x, v, a, jk, px, pv);
    } else {
      mi = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) { px[d] = NB_PAD_POS; pv[d] = 0.0; }
    }
    nbh::store_predicted(i, n_pad, px, pv, mi, xp, vp, jA, jB, jC, write_fp64 != 0, write_mixed != 0);
  }
}

// Corrector and new block step (Sec. 4.1 step 5) for list position k,
// particle i = list[k], forces F[.][k]; arithmetic in hermite.cuh.
__global__ void correct_kernel(int64_t n, int64_t n_pad, const int32_t* __restrict__ list,
                               const double* __restrict__ F, int64_t fstride, double t, double eta,
                               double dt_min, double dt_max, double* __restrict__ x,
                               double* __restrict__ v, double* __restrict__ a, double* __restrict__ jk,
                               double* __restrict__ pot, double* __restrict__ ti, double* __restrict__ dt,
                               const double* __restrict__ xp, const double* __restrict__ vp,
                               nb_dev_status* __restrict__ st, float4* __restrict__ jm, int64_t N,
                               const double* __restrict__ m) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = list[k];
    i = i < 0 ? 0 : (i >= n_pad ? n_pad - 1 : i);  // never out of bounds on a bad list
    double f[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) f[c] = F[c * fstride + k];
    nbh::correct_row(i, n_pad, t, f, eta, dt_min, dt_max, x, v, a, jk, pot, ti, dt, xp, vp, st);
    // the corrected particle's j-memory record (on-the-fly j prediction)
    if (jm) nbh::write_jm_record(i, N, n_pad, m, x, v, a, jk, dt, jm);
  }
}

// initial steps: dt = pow2floor(eta |a| / |j|) clamped; t_i = 0 (Sec. 4.1 step 1)
__global__ void initial_dt_kernel(int64_t N, int64_t n_pad, const double* __restrict__ F,
                                  int64_t fstride, double eta, double dt_min, double dt_max,
                                  double* __restrict__ a, double* __restrict__ jk,
                                  double* __restrict__ pot, double* __restrict__ ti,
                                  double* __restrict__ dt, nb_dev_status* __restrict__ st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double na2 = 0, nj2 = 0;
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double av = F[c * fstride + i], jv = F[(3 + c) * fstride + i];
      a[c * n_pad + i] = av;
      jk[c * n_pad + i] = jv;
      na2 += av * av;
      nj2 += jv * jv;
      finite = finite && isfinite(av) && isfinite(jv);
    }
    pot[i] = F[6 * fstride + i];
    const double nj = sqrt(nj2);
    const double d = (nj > 0.0) ? eta * sqrt(na2) / nj : (double)INFINITY;
    dt[i] = nbh::clamp_dt(nbh::pow2_floor(d), dt_min, dt_max);
    ti[i] = 0.0;
    if (!finite) atomicOr(&st->flags, NB_ST_NUMERIC);
  }
}

// ---------------------------------------------------------------------------
// Block selection (Sec. 4.1 step 2): t_next = min_i (t_i + dt_i); active
// list = ascending {i : t_i + dt_i == t_next}.  Positive doubles order like
// their bit patterns, so the minimum is taken on the 64-bit pattern.  Each
// CTA owns a contiguous chunk; counts are scanned in one CTA; indices are
// written in order (ballot + popc within warps, warp prefix within the CTA).
// ---------------------------------------------------------------------------
__global__ void sel_min_kernel(int64_t N, int64_t chunk, const double* __restrict__ ti,
                               const double* __restrict__ dt, unsigned long long* __restrict__ out) {
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(lo + chunk, N);
  unsigned long long best = 0x7FF0000000000000ULL;  // +inf
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(ti[i] + dt[i]);
    best = b < best ? b : best;
  }
  __shared__ unsigned long long sm[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    best = threadIdx.x < nw ? sm[threadIdx.x] : 0x7FF0000000000000ULL;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
      best = w < best ? w : best;
    }
    if (threadIdx.x == 0) out[blockIdx.x] = best;
  }
}

__global__ void sel_min_final_kernel(int nb, unsigned long long* __restrict__ mins) {
  unsigned long long best = 0x7FF0000000000000ULL;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) best = mins[i] < best ? mins[i] : best;
  __shared__ unsigned long long sm[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    best = threadIdx.x < nw ? sm[threadIdx.x] : 0x7FF0000000000000ULL;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
      best = w < best ? w : best;
    }
    if (threadIdx.x == 0) mins[nb] = best;
  }
}

__global__ void sel_count_kernel(int64_t N, int64_t chunk, const double* __restrict__ ti,
                                 const double* __restrict__ dt,
                                 const unsigned long long* __restrict__ tmin, int nb,
                                 int32_t* __restrict__ cnt) {
  const double tn = __longlong_as_double((long long)tmin[nb]);
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(lo + chunk, N);
  int c = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += (ti[i] + dt[i] == tn) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    cnt[blockIdx.x] = s;
  }
}

// exclusive scan of nb counts in one CTA (nb <= 1024); total to cnt[nb]
__global__ void sel_scan_kernel(int nb, int32_t* __restrict__ cnt) {
  __shared__ int32_t s[1025];
  const int t = threadIdx.x;
  s[t] = (t < nb) ? cnt[t] : 0;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int i = 0; i < nb; ++i) {
      const int32_t c = s[i];
      s[i] = run;
      run += c;
    }
    s[nb] = run;
  }
  __syncthreads();
  if (t < nb) cnt[t] = s[t];
  if (t == 0) cnt[nb] = s[nb];
}

__global__ void sel_write_kernel(int64_t N, int64_t chunk, const double* __restrict__ ti,
                                 const double* __restrict__ dt,
                                 const unsigned long long* __restrict__ tmin, int nb,
                                 const int32_t* __restrict__ off, int32_t* __restrict__ act) {
  const double tn = __longlong_as_double((long long)tmin[nb]);
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(lo + chunk, N);
  __shared__ int wsum[32];
  int base = off[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t seg = lo; seg < hi; seg += blockDim.x) {
    const int64_t i = seg + threadIdx.x;
    const bool f = (i < hi) && (ti[i] + dt[i] == tn);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int wpre = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = wsum[w];
      if (w < wid) wpre += c;
      tot += c;
    }
    if (f) act[base + wpre + pre] = (int32_t)i;
    base += tot;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Energy: K = sum m v^2 / 2, W = sum m pot / 2; fixed-order two-pass FP64.
// ---------------------------------------------------------------------------
__global__ void energy_partial_kernel(int64_t N, int64_t n_pad, const double* __restrict__ m,
                                      const double* __restrict__ v, const double* __restrict__ pot,
                                      double* __restrict__ red) {
  double k = 0.0, w = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v0 = v[i], v1 = v[n_pad + i], v2 = v[2 * n_pad + i];
    k += 0.5 * m[i] * (v0 * v0 + v1 * v1 + v2 * v2);
    w += 0.5 * m[i] * pot[i];
  }
  __shared__ double sk[kThreads], sw[kThreads];
  sk[threadIdx.x] = k;
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sk[threadIdx.x] += sk[threadIdx.x + s];
      sw[threadIdx.x] += sw[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    red[2 * blockIdx.x] = sk[0];
    red[2 * blockIdx.x + 1] = sw[0];
  }
}

__global__ void energy_final_kernel(int nb, const double* __restrict__ red, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double k = 0.0, w = 0.0;
    for (int b = 0; b < nb; ++b) {
      k += red[2 * b];
      w += red[2 * b + 1];
    }
    out[0] = k;
    out[1] = w;
  }
}

// ---------------------------------------------------------------------------
// layout helpers and list validation
// ---------------------------------------------------------------------------
__global__ void fill_ident_kernel(int64_t n, int32_t* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

__global__ void aos_to_soa_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                  int64_t count, int64_t stride) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    dst[i] = src[3 * i];
    dst[stride + i] = src[3 * i + 1];
    dst[2 * stride + i] = src[3 * i + 2];
  }
}

__global__ void soa_to_aos_kernel(const double* __restrict__ src, int64_t stride,
                                  double* __restrict__ dst, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    dst[3 * i] = src[i];
    dst[3 * i + 1] = src[stride + i];
    dst[3 * i + 2] = src[2 * stride + i];
  }
}

__global__ void check_list_kernel(const int32_t* __restrict__ l, int64_t n, int64_t N,
                                  unsigned int* __restrict__ flag) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = l[k];
    const bool bad = v < 0 || v >= N || (k > 0 && l[k - 1] >= v);
    if (bad) atomicOr(flag, NB_ST_BADLIST);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t nb_launch_predict(nb_ctx* c, double t, bool own_time) {
  const bool mixed = c->precision == NB_MIXED;
  c->launches += 1;
  predict_kernel<<<grid_for(c->n_pad, kThreads, c->sm_count * 16), kThreads, 0, c->stream>>>(
      c->n, c->n_pad, c->m, c->x, c->v, c->a, c->jk, c->t, t, own_time ? 1 : 0, c->xp, c->vp, c->jA,
      c->jB, c->jC, 1, mixed ? 1 : 0);
  if (mixed && c->perm_valid) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return nb_launch_tile_boxes(c);
  }
  return cudaGetLastError();
}

cudaError_t nb_launch_select(nb_ctx* c) {
  const int nb = c->sel_ctas;
  int64_t chunk = (c->n + nb - 1) / nb;
  chunk = ((chunk + 255) / 256) * 256;
  const int used = (int)((c->n + chunk - 1) / chunk);
  c->launches += 5;
  sel_min_kernel<<<used, 256, 0, c->stream>>>(c->n, chunk, c->t, c->dt, c->sel_min);
  sel_min_final_kernel<<<1, 1024, 0, c->stream>>>(used, c->sel_min);
  // the result sits at sel_min[used]; copy it to the fixed slot sel_min[sel_ctas]
  cudaError_t e = cudaSuccess;
  if (used != nb) {
    e = cudaMemcpyAsync(c->sel_min + nb, c->sel_min + used, sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  sel_count_kernel<<<used, 256, 0, c->stream>>>(c->n, chunk, c->t, c->dt, c->sel_min, nb, c->sel_cnt);
  sel_scan_kernel<<<1, 1024, 0, c->stream>>>(used, c->sel_cnt);
  if (used != nb) {
    e = cudaMemcpyAsync(c->sel_cnt + nb, c->sel_cnt + used, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        c->stream);
    if (e != cudaSuccess) return e;
  }
  sel_write_kernel<<<used, 256, 0, c->stream>>>(c->n, chunk, c->t, c->dt, c->sel_min, nb, c->sel_cnt,
                                               c->act);
  return cudaGetLastError();
}

cudaError_t nb_launch_correct(nb_ctx* c, const int32_t* d_list, int64_t n, double t, bool write_jm) {
  if (n <= 0) return cudaSuccess;
  c->launches += 1;
  correct_kernel<<<grid_for(n, 128, c->sm_count * 32), 128, 0, c->stream>>>(
      n, c->n_pad, d_list, c->F, c->n_pad, t, c->eta, c->dt_min, c->dt_max, c->x, c->v, c->a, c->jk,
      c->pot, c->t, c->dt, c->xp, c->vp, c->status, write_jm ? c->jm : nullptr, c->n, c->m);
  return cudaGetLastError();
}

cudaError_t nb_launch_initial_dt(nb_ctx* c) {
  c->launches += 1;
  initial_dt_kernel<<<grid_for(c->n, kThreads, c->sm_count * 16), kThreads, 0, c->stream>>>(
      c->n, c->n_pad, c->F, c->n_pad, c->eta, c->dt_min, c->dt_max, c->a, c->jk, c->pot, c->t, c->dt,
      c->status);
  return cudaGetLastError();
}

cudaError_t nb_launch_energy(nb_ctx* c, const double* d_pot, double* d_out2) {
  const int nb = grid_for(c->n, kThreads, 1024);
  c->launches += 2;
  energy_partial_kernel<<<nb, kThreads, 0, c->stream>>>(c->n, c->n_pad, c->m, c->v, d_pot, c->red);
  energy_final_kernel<<<1, 32, 0, c->stream>>>(nb, c->red, d_out2);
  return cudaGetLastError();
}

cudaError_t nb_launch_fill_ident(nb_ctx* c) {
  c->launches += 1;
  fill_ident_kernel<<<grid_for(c->n_pad, kThreads, c->sm_count * 16), kThreads, 0, c->stream>>>(
      c->n_pad, c->ident);
  return cudaGetLastError();
}

cudaError_t nb_launch_aos_to_soa(const double* src, double* dst, int64_t count, int64_t stride_dst,
                                 cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  aos_to_soa_kernel<<<grid_for(count, kThreads, 4096), kThreads, 0, s>>>(src, dst, count, stride_dst);
  return cudaGetLastError();
}

cudaError_t nb_launch_soa_to_aos(const double* src, int64_t stride_src, double* dst, int64_t count,
                                 cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  soa_to_aos_kernel<<<grid_for(count, kThreads, 4096), kThreads, 0, s>>>(src, stride_src, dst, count);
  return cudaGetLastError();
}

cudaError_t nb_launch_check_list(const int32_t* d_list, int64_t n, int64_t N, unsigned int* d_flag,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  check_list_kernel<<<grid_for(n, kThreads, 4096), kThreads, 0, s>>>(d_list, n, N, d_flag);
  return cudaGetLastError();
}
