// force_fp64.cu -- host-driven launch of the FP64 force item
// (force_common.cuh; Sec. 4.1 step 4, Eq. 3), the accuracy reference path,
// plus the split-j reduction shared with the mixed path and the automatic
// split choice.
#include "force_common.cuh"

namespace {

template <int NT, int JT>
__global__ void __launch_bounds__(NT) force_fp64_kernel(
    const double* __restrict__ xp, const double* __restrict__ vp, const double* __restrict__ m,
    int64_t n_pad, int64_t n_j, const int32_t* __restrict__ list, int64_t n, int64_t j_per_split,
    double eps2, double* __restrict__ out, int64_t ostride, int finalize) {
  __shared__ nbk::Fp64Smem<JT> sm;
  const int split = blockIdx.y;
  const int64_t jlo = (int64_t)split * j_per_split;
  const int64_t jhi = min(jlo + j_per_split, n_j);
  double* o = finalize ? out : out + (int64_t)split * 7 * ostride;
  nbk::fp64_item<NT, JT>(sm, xp, vp, m, n_pad, jlo, jhi, list, n, (int64_t)blockIdx.x * NT, eps2, o, ostride,
                         finalize != 0);
}

// split-j reduction: F[c][k] = sum over s = 0..S-1 (in this order) of
// part[s][c][k]; the potential is negated (kernels sum +m/s).
__global__ void split_reduce_kernel(const double* __restrict__ part, int64_t stride, int nsplit,
                                    int64_t n, double* __restrict__ F, int64_t fstride) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double s = 0.0;
      for (int q = 0; q < nsplit; ++q) s += part[((int64_t)q * 7 + c) * stride + k];
      F[c * fstride + k] = c == 6 ? -s : s;
    }
  }
}

template <int NT, int JT>
cudaError_t launch(nb_ctx* c, const int32_t* d_list, int64_t n, int nsplit) {
  const int64_t itiles = (n + NT - 1) / NT;
  const int64_t n_j = ((c->n + JT - 1) / JT) * JT;
  const int64_t tiles = n_j / JT;
  if (nsplit > tiles) nsplit = (int)tiles;
  if (nsplit < 1) nsplit = 1;
  const int64_t tiles_per_split = (tiles + nsplit - 1) / nsplit;
  nsplit = (int)((tiles + tiles_per_split - 1) / tiles_per_split);
  const int64_t j_per_split = tiles_per_split * JT;
  const bool fin = nsplit == 1;
  const int64_t ostride = fin ? c->n_pad : ((n + 31) / 32) * 32;
  double* out = fin ? c->F : c->part;
  if (!fin && (int64_t)nsplit * 7 * ostride > c->part_elems) return cudaErrorInvalidValue;
  dim3 grid((unsigned)itiles, (unsigned)nsplit);
  c->launches += fin ? 1 : 2;
  force_fp64_kernel<NT, JT><<<grid, NT, 0, c->stream>>>(c->xp, c->vp, c->m, c->n_pad, n_j, d_list, n,
                                                        j_per_split, c->eps * c->eps, out, ostride,
                                                        fin ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || fin) return e;
  return nb_launch_split_reduce(c, d_list, n, nsplit, ostride);
}

}  // namespace

cudaError_t nb_launch_split_reduce(nb_ctx* c, const int32_t* d_list, int64_t n, int nsplit,
                                   int64_t stride) {
  (void)d_list;
  int g = (int)((n + 255) / 256);
  if (g > c->sm_count * 8) g = c->sm_count * 8;
  if (g < 1) g = 1;
  split_reduce_kernel<<<g, 256, 0, c->stream>>>(c->part, stride, nsplit, n, c->F, c->n_pad);
  return cudaGetLastError();
}

bool nb_fp64_supported(const nb_tuning& t) {
  return t.ipt == 1 && (t.threads == 64 || t.threads == 128 || t.threads == 256) &&
         (t.jtile == 32 || t.jtile == 64 || t.jtile == 128);
}

bool nb_mixed_supported(const nb_tuning& t);

bool nb_tuning_supported(int precision, const nb_tuning& cfg) {
  if (cfg.nsplit < 0 || cfg.nsplit > 4096) return false;
  return precision == NB_FP64 ? nb_fp64_supported(cfg) : nb_mixed_supported(cfg);
}

nb_tuning nb_default_tuning(int precision) {
  if (precision == NB_FP64) return nb_tuning{1, 128, 64, 0};
  // one i per thread, two j per packed FP32x2 instruction: measured fastest at
  // N = 2^20 (more i per thread saves shared loads but costs occupancy)
  return nb_tuning{1, 128, 128, 0};
}

// Split-j factor: enough CTAs for about four waves of resident CTAs on all
// SMs, at least one j-tile per split, within the partial-sum scratch.
int nb_auto_split(const nb_ctx* c, int64_t n, const nb_tuning& cfg) {
  const int64_t per_cta = (int64_t)cfg.threads * cfg.ipt;
  const int64_t itiles = (n + per_cta - 1) / per_cta;
  const int64_t resident = (int64_t)c->sm_count * (cfg.threads <= 128 ? 4 : 2);
  const int64_t want = 4 * resident;
  if (itiles >= want) return 1;
  int64_t s = (want + itiles - 1) / itiles;
  const int64_t tiles = (c->n + cfg.jtile - 1) / cfg.jtile;
  if (s > tiles) s = tiles;
  const int64_t ostride = ((n + 31) / 32) * 32;
  const int64_t cap = c->part_elems / (7 * ostride);
  if (s > cap) s = cap;
  if (s > 4096) s = 4096;
  return (int)(s < 1 ? 1 : s);
}

#define NB_FP64_CASE(NT_, JT_) \
  if (cfg.threads == NT_ && cfg.jtile == JT_) return launch<NT_, JT_>(c, d_list, n, nsplit);

cudaError_t nb_forces_fp64(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg) {
  if (n <= 0) return cudaSuccess;
  const int nsplit = cfg.nsplit > 0 ? cfg.nsplit : nb_auto_split(c, n, cfg);
  NB_FP64_CASE(64, 32) NB_FP64_CASE(64, 64) NB_FP64_CASE(64, 128)
  NB_FP64_CASE(128, 32) NB_FP64_CASE(128, 64) NB_FP64_CASE(128, 128)
  NB_FP64_CASE(256, 32) NB_FP64_CASE(256, 64) NB_FP64_CASE(256, 128)
  return cudaErrorInvalidValue;
}
