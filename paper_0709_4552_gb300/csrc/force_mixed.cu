// force_mixed.cu -- host-driven launch of the mixed-precision force item
// (force_common.cuh; Sec. 4.1 step 4, Eq. 3) for sm_103a.
//
// Grid: (i-tiles of NT*IPT active particles) x (j-range splits).  With one
// split the item writes final results into F; otherwise double-single
// partials [split][7][n] (an FP32 pair per 8-byte slot) that the split-j
// reduction sums in FP32, in a fixed order (deterministic for a given launch
// configuration), and converts to FP64 once per result.
#include "force_common.cuh"

namespace {

// minimum resident CTAs per SM asked of the register allocator for the
// 128-thread, one-i-per-thread shape (0 = no request)
#ifndef NB_MIXED_MINB
#define NB_MIXED_MINB 0
#endif
#if NB_MIXED_MINB > 0
#define NB_MIXED_BOUNDS(NT, IPT) __launch_bounds__(NT, ((IPT) == 1 && (NT) == 128) ? NB_MIXED_MINB : 1)
#else
#define NB_MIXED_BOUNDS(NT, IPT) __launch_bounds__(NT)
#endif

template <int NT, int IPT, int JT>
__global__ void NB_MIXED_BOUNDS(NT, IPT) force_mixed_kernel(
    const float4* __restrict__ jA, const float4* __restrict__ jB, const float2* __restrict__ jC,
    int64_t n_j, const int32_t* __restrict__ list, int64_t n, int64_t tiles, float eps2,
    double* __restrict__ out, int64_t ostride, int finalize, const float4* __restrict__ tbox,
    const int32_t* __restrict__ ord, const nbk::ISrc is) {
  __shared__ __align__(16) nbk::MixedSmem<JT> sm;
  const int split = blockIdx.y;
  const int64_t jlo = nbk::split_begin(split, gridDim.y, tiles) * JT;
  const int64_t jhi = min(nbk::split_begin(split + 1, gridDim.y, tiles) * JT, n_j);
  double* o = finalize ? out : out + (int64_t)split * 7 * ostride;
  nbk::mixed_item<NT, IPT, JT>(sm, jA, jB, jC, jlo, jhi, n_j, list, n, (int64_t)blockIdx.x * (NT * IPT),
                               eps2, o, ostride, finalize != 0, tbox, ord, 0, nbk::FusedArgs(), is, true);
}

// the same item with on-the-fly prediction of the j-tiles from the j-memory
// (Sec. 4.4 step 4); the i-particles' predicted rows are in jA/jB/jC
template <int NT, int JT>
__global__ void __launch_bounds__(NT) force_mixed_fused_kernel(
    const float4* __restrict__ jA, const float4* __restrict__ jB, const float2* __restrict__ jC,
    int64_t n_j, const int32_t* __restrict__ list, int64_t n, int64_t tiles, float eps2,
    double* __restrict__ out, int64_t ostride, int finalize, const float4* __restrict__ tbox,
    const int32_t* __restrict__ ord, const float4* __restrict__ jm, int64_t jm_stride,
    const double* __restrict__ tj, double T) {
  __shared__ __align__(16) nbk::FusedSmem<JT> sm;
  const int split = blockIdx.y;
  const int64_t jlo = nbk::split_begin(split, gridDim.y, tiles) * JT;
  const int64_t jhi = min(nbk::split_begin(split + 1, gridDim.y, tiles) * JT, n_j);
  double* o = finalize ? out : out + (int64_t)split * 7 * ostride;
  nbk::FusedArgs fa;
  fa.jm = jm;
  fa.stride = jm_stride;
  fa.tj = tj;
  fa.T = T;
  nbk::mixed_item<NT, 1, JT>(sm, jA, jB, jC, jlo, jhi, n_j, list, n, (int64_t)blockIdx.x * NT, eps2, o, ostride,
                             finalize != 0, tbox, ord, 0, fa, nbk::ISrc(), true);
}

// Split-j reduction of double-single partials: CTA (32 x kQL threads) =
// 32 consecutive list positions (coalesced rows) x kQL lanes over the
// splits; lane ty sums splits ty, ty + kQL, ... in order (loads in batches of
// kB, so that a thread waits for one round trip per batch), then a fixed
// pairwise tree over ty; one FP64 conversion per result.  Also writes the
// caller's AoS outputs when given.
constexpr int kQL = 32, kB = 8;
__global__ void __launch_bounds__(32 * kQL) split_reduce_ds_kernel(const float2* __restrict__ part, int64_t stride,
                                                                  int nsplit, int64_t n, double* __restrict__ F,
                                                                  int64_t fstride, double* __restrict__ acc,
                                                                  double* __restrict__ jerk,
                                                                  double* __restrict__ pot) {
  __shared__ float2 sm[kQL][33];
  const int tx = threadIdx.x, ty = threadIdx.y, c = blockIdx.y;
  for (int64_t k0 = (int64_t)blockIdx.x * 32; k0 < n; k0 += (int64_t)gridDim.x * 32) {
    const int64_t k = k0 + tx;
    float hi = 0.0f, lo = 0.0f;
    if (k < n) {
      const float2* src = part + (int64_t)c * stride + k;
      const int64_t step = (int64_t)kQL * 7 * stride;  // kQL splits further on
      int q = ty;
      for (; q + (kB - 1) * kQL < nsplit; q += kB * kQL) {
        float2 v[kB];
#pragma unroll
        for (int b = 0; b < kB; ++b) v[b] = src[(int64_t)q * 7 * stride + b * step];
#pragma unroll
        for (int b = 0; b < kB; ++b) nbk::ds_add(hi, lo, v[b].x, v[b].y);
      }
      for (; q < nsplit; q += kQL) {
        const float2 v = src[(int64_t)q * 7 * stride];
        nbk::ds_add(hi, lo, v.x, v.y);
      }
    }
    sm[ty][tx] = make_float2(hi, lo);
    __syncthreads();
#pragma unroll
    for (int h = kQL / 2; h > 0; h >>= 1) {
      if (ty < h) {
        float2 a = sm[ty][tx];
        const float2 b = sm[ty + h][tx];
        nbk::ds_add(a.x, a.y, b.x, b.y);
        sm[ty][tx] = a;
      }
      __syncthreads();
    }
    if (ty == 0 && k < n) {
      const double s = (double)sm[0][tx].x + (double)sm[0][tx].y;
      const double val = c == 6 ? -s : s;
      F[c * fstride + k] = val;
      if (c < 3) {
        if (acc) acc[3 * k + c] = val;
      } else if (c < 6) {
        if (jerk) jerk[3 * k + (c - 3)] = val;
      } else if (pot) {
        pot[k] = val;
      }
    }
    __syncthreads();
  }
}

// resident CTAs per SM of an instantiation (0 when the query fails)
template <int NT, int IPT, int JT>
int per_sm_of() {
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_mixed_kernel<NT, IPT, JT>, NT, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  return per_sm;
}

template <int NT, int IPT, int JT>
cudaError_t launch(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg, float eps2,
                   const int32_t* ord, const nbk::ISrc& is) {
  const int per_sm = per_sm_of<NT, IPT, JT>();
  if (per_sm == 0) return cudaErrorInvalidValue;
  int nsplit = cfg.nsplit > 0 ? cfg.nsplit : nb_auto_split(c, n, cfg, per_sm);
  const int64_t per_cta = (int64_t)NT * IPT;
  const int64_t itiles = (n + per_cta - 1) / per_cta;
  const int64_t n_j = ((c->n + JT - 1) / JT) * JT;  // padding particles (m = 0) fill the last tile
  const int64_t tiles = n_j / JT;
  if (nsplit > tiles) nsplit = (int)tiles;
  if (nsplit < 1) nsplit = 1;
  dim3 grid((unsigned)itiles, (unsigned)nsplit);
  const bool fin = nsplit == 1;
  const int64_t ostride = fin ? c->n_pad : ((n + 31) / 32) * 32;
  double* out = fin ? c->F : c->part;
  if (!fin && (int64_t)nsplit * 7 * ostride > c->part_elems) return cudaErrorInvalidValue;
  c->launches += fin ? 1 : 2;
  // resident spatial order: far-tile boxes when the tiles match (unless the
  // context asks for double-single differences on every tile)
  const float4* tbox = (c->perm_valid && c->far_tiles) ? c->tbox : nullptr;
  force_mixed_kernel<NT, IPT, JT><<<grid, NT, 0, c->stream>>>(c->jA, c->jB, c->jC, n_j, d_list, n, tiles,
                                                              eps2, out, ostride, fin ? 1 : 0, tbox, ord, is);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || fin) return e;
  return nb_launch_split_reduce_ds(c, n, nsplit, ostride);
}

}  // namespace

// forces on d_list with the j-tiles predicted to T on the fly (default launch
// shape: 128 threads, one i per thread, 128-particle j-tiles); boxes, when
// given, are the j-memory tile boxes grown by each particle's reach
cudaError_t nb_forces_mixed_fused(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                                  const int32_t* ord, double T, const float4* boxes) {
  constexpr int NT = 128, JT = 128;
  if (n <= 0) return cudaSuccess;
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_mixed_fused_kernel<NT, JT>, NT, 0) != cudaSuccess)
    return cudaGetLastError();
  const nb_tuning shape{1, NT, JT, cfg.nsplit};
  int nsplit = cfg.nsplit > 0 ? cfg.nsplit : nb_auto_split(c, n, shape, per_sm);
  const int64_t itiles = (n + NT - 1) / NT;
  const int64_t n_j = ((c->n + JT - 1) / JT) * JT;
  const int64_t tiles = n_j / JT;
  if (nsplit > tiles) nsplit = (int)tiles;
  if (nsplit < 1) nsplit = 1;
  const bool fin = nsplit == 1;
  const int64_t ostride = fin ? c->n_pad : ((n + 31) / 32) * 32;
  double* out = fin ? c->F : c->part;
  if (!fin && (int64_t)nsplit * 7 * ostride > c->part_elems) return cudaErrorInvalidValue;
  c->launches += fin ? 1 : 2;
  const float eps2 = (float)(c->eps * c->eps);
  force_mixed_fused_kernel<NT, JT><<<dim3((unsigned)itiles, (unsigned)nsplit), NT, 0, c->stream>>>(
      c->jA, c->jB, c->jC, n_j, d_list, n, tiles, eps2, out, ostride, fin ? 1 : 0, boxes, ord, c->jm, c->n_pad,
      c->t, T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || fin) return e;
  return nb_launch_split_reduce_ds(c, n, nsplit, ostride);
}

cudaError_t nb_launch_split_reduce_ds(nb_ctx* c, int64_t n, int nsplit, int64_t stride) {
  int64_t g = (n + 31) / 32;
  if (g > (int64_t)c->sm_count * 4) g = (int64_t)c->sm_count * 4;
  if (g < 1) g = 1;
  split_reduce_ds_kernel<<<dim3((unsigned)g, 7), dim3(32, kQL), 0, c->stream>>>(
      reinterpret_cast<const float2*>(c->part), stride, nsplit, n, c->F, c->n_pad, c->fo_acc, c->fo_jerk, c->fo_pot);
  if (c->fo_acc || c->fo_jerk || c->fo_pot) c->fo_done = true;
  return cudaGetLastError();
}

int nb_mixed_ctas_per_sm(const nb_tuning& cfg) {
#define NB_PER_SM_CASE(NT_, IPT_, JT_) \
  if (cfg.threads == NT_ && cfg.ipt == IPT_ && cfg.jtile == JT_) return per_sm_of<NT_, IPT_, JT_>();
#define NB_PER_SM_JT(NT_, IPT_) NB_PER_SM_CASE(NT_, IPT_, 64) NB_PER_SM_CASE(NT_, IPT_, 128) NB_PER_SM_CASE(NT_, IPT_, 256)
#define NB_PER_SM_IPT(NT_) NB_PER_SM_JT(NT_, 1) NB_PER_SM_JT(NT_, 2) NB_PER_SM_JT(NT_, 4)
  NB_PER_SM_IPT(64)
  NB_PER_SM_IPT(128)
  NB_PER_SM_IPT(256)
#undef NB_PER_SM_IPT
#undef NB_PER_SM_JT
#undef NB_PER_SM_CASE
  return 0;
}

bool nb_mixed_supported(const nb_tuning& t) {
  const bool thr = t.threads == 64 || t.threads == 128 || t.threads == 256;
  const bool ipt = t.ipt == 1 || t.ipt == 2 || t.ipt == 4;
  const bool jt = t.jtile == 64 || t.jtile == 128 || t.jtile == 256;
  return thr && ipt && jt;
}

#define NB_MIXED_CASE(NT_, IPT_, JT_)                            \
  if (cfg.threads == NT_ && cfg.ipt == IPT_ && cfg.jtile == JT_) \
    return launch<NT_, IPT_, JT_>(c, d_list, n, cfg, eps2, ord, is);

cudaError_t nb_forces_mixed(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                            const int32_t* ord, const nbk::ISrc* isrc) {
  if (n <= 0) return cudaSuccess;
  const nbk::ISrc is = isrc ? *isrc : nbk::ISrc();
  const float eps2 = (float)(c->eps * c->eps);
#define NB_MIXED_JT(NT_, IPT_) NB_MIXED_CASE(NT_, IPT_, 64) NB_MIXED_CASE(NT_, IPT_, 128) NB_MIXED_CASE(NT_, IPT_, 256)
#define NB_MIXED_IPT(NT_) NB_MIXED_JT(NT_, 1) NB_MIXED_JT(NT_, 2) NB_MIXED_JT(NT_, 4)
  NB_MIXED_IPT(64)
  NB_MIXED_IPT(128)
  NB_MIXED_IPT(256)
#undef NB_MIXED_IPT
#undef NB_MIXED_JT
  return cudaErrorInvalidValue;
}
