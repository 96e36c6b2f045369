// force_fp64.cu -- host-driven launch of the FP64 force item
// (force_common.cuh; Sec. 4.1 step 4, Eq. 3), the accuracy reference path,
// plus the split-j reduction shared with the mixed path and the automatic
// split choice.
#include <algorithm>

#include "force_common.cuh"

namespace {

template <int NT, int JT>
__global__ void __launch_bounds__(NT) force_fp64_kernel(
    const double* __restrict__ xp, const double* __restrict__ vp, const double* __restrict__ m,
    int64_t n_pad, int64_t N, const int32_t* __restrict__ list, int64_t n, int64_t tiles,
    double eps2, double* __restrict__ out, int64_t ostride, int finalize, const nbk::ISrc is) {
  __shared__ nbk::Fp64Smem<JT> sm;
  const int split = blockIdx.y;
  // j-range of this split, cut at N: the item fills the rest of the last
  // tile with massless far-away particles, so rows >= N are never read
  const int64_t jlo = nbk::split_begin(split, gridDim.y, tiles) * JT;
  const int64_t jhi = min(nbk::split_begin(split + 1, gridDim.y, tiles) * JT, N);
  double* o = finalize ? out : out + (int64_t)split * 7 * ostride;
  nbk::fp64_item<NT, JT>(sm, xp, vp, m, n_pad, jlo, jhi, list, n, (int64_t)blockIdx.x * NT, eps2, o, ostride,
                         finalize != 0, is);
}

// split-j reduction: F[c][k] = sum over s = 0..S-1 (in this order) of
// part[s][c][k]; the potential is negated (kernels sum +m/s).
// Split-j reduction of part[S][7][stride] into F (the sign of the potential
// applied here).  Block = 32 list positions x QL split lanes for one row c:
// lane y sums splits y, y + QL, y + 2 QL, ... in order, then a fixed binary
// tree combines the lanes, so the result depends only on S and QL (one
// launch configuration = one summation order), and a long split list is
// read by QL warps at once instead of one dependent chain per position.
template <int QL>
__global__ void split_reduce_kernel(const double* __restrict__ part, int64_t stride, int nsplit,
                                    int64_t n, double* __restrict__ F, int64_t fstride) {
  __shared__ double sm[QL][33];
  const int tx = threadIdx.x, ty = threadIdx.y, c = blockIdx.y;
  for (int64_t k0 = (int64_t)blockIdx.x * 32; k0 < n; k0 += (int64_t)gridDim.x * 32) {
    const int64_t k = k0 + tx;
    double s = 0.0;
    if (k < n) {
      // splits ty, ty + QL, ... added in order, loaded 8 at a time (one
      // round trip per batch instead of per split)
      int q = ty;
      for (; q + 7 * QL < nsplit; q += 8 * QL) {
        double v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) v[b] = part[((int64_t)(q + b * QL) * 7 + c) * stride + k];
#pragma unroll
        for (int b = 0; b < 8; ++b) s += v[b];
      }
      for (; q < nsplit; q += QL) s += part[((int64_t)q * 7 + c) * stride + k];
    }
    sm[ty][tx] = s;
    __syncthreads();
#pragma unroll
    for (int h = QL / 2; h > 0; h >>= 1) {
      if (ty < h) sm[ty][tx] += sm[ty + h][tx];
      __syncthreads();
    }
    if (ty == 0 && k < n) F[c * fstride + k] = c == 6 ? -sm[0][tx] : sm[0][tx];
    __syncthreads();
  }
}

template <int NT, int JT>
cudaError_t launch(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg, const nbk::ISrc& is) {
  static int per_sm = 0;  // resident CTAs per SM of this instantiation
  if (per_sm == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, force_fp64_kernel<NT, JT>, NT, 0) !=
                         cudaSuccess)
    return cudaGetLastError();
  int nsplit = cfg.nsplit > 0 ? cfg.nsplit : nb_auto_split(c, n, cfg, per_sm);
  const int64_t itiles = (n + NT - 1) / NT;
  const int64_t n_j = ((c->n + JT - 1) / JT) * JT;
  const int64_t tiles = n_j / JT;
  if (nsplit > tiles) nsplit = (int)tiles;
  if (nsplit < 1) nsplit = 1;
  const bool fin = nsplit == 1;
  const int64_t ostride = fin ? c->n_pad : ((n + 31) / 32) * 32;
  double* out = fin ? c->F : c->part;
  if (!fin && (int64_t)nsplit * 7 * ostride > c->part_elems) return cudaErrorInvalidValue;
  dim3 grid((unsigned)itiles, (unsigned)nsplit);
  c->launches += fin ? 1 : 2;
  force_fp64_kernel<NT, JT><<<grid, NT, 0, c->stream>>>(c->xp, c->vp, c->m, c->n_pad, c->n, d_list, n,
                                                        tiles, c->eps * c->eps, out, ostride, fin ? 1 : 0, is);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || fin) return e;
  return nb_launch_split_reduce(c, d_list, n, nsplit, ostride);
}

}  // namespace

cudaError_t nb_launch_split_reduce(nb_ctx* c, const int32_t* d_list, int64_t n, int nsplit,
                                   int64_t stride) {
  (void)d_list;
  int64_t g = (n + 31) / 32;
  if (g > (int64_t)c->sm_count * 16) g = (int64_t)c->sm_count * 16;
  if (g < 1) g = 1;
  const dim3 grid((unsigned)g, 7);
  if (nsplit >= 32)
    split_reduce_kernel<32><<<grid, dim3(32, 32), 0, c->stream>>>(c->part, stride, nsplit, n, c->F, c->n_pad);
  else
    split_reduce_kernel<4><<<grid, dim3(32, 4), 0, c->stream>>>(c->part, stride, nsplit, n, c->F, c->n_pad);
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

// Split-j factor: at least four waves of resident CTAs (per_sm per SM), the
// count of CTAs chosen so that the last wave is nearly full and the splits'
// tile counts nearly equal; at least one j-tile per split, within the
// partial-sum scratch.
int nb_auto_split(const nb_ctx* c, int64_t n, const nb_tuning& cfg, int per_sm) {
  const int64_t per_cta = (int64_t)cfg.threads * cfg.ipt;
  const int64_t itiles = (n + per_cta - 1) / per_cta;
  const int64_t R = (int64_t)c->sm_count * (per_sm > 0 ? per_sm : 1);
  if (itiles >= 4 * R) return 1;
  const int64_t tiles = (c->n + cfg.jtile - 1) / cfg.jtile;
  const int64_t ostride = ((n + 31) / 32) * 32;
  int64_t cap = std::min<int64_t>(tiles, c->part_elems / (7 * ostride));
  cap = std::min<int64_t>(cap, 4096);
  if (cap < 1) return 1;
  const int64_t s0 = std::min<int64_t>((4 * R + itiles - 1) / itiles, cap);
  int64_t best = s0;
  double best_e = -1.0;
  for (int64_t s = s0; s <= std::min<int64_t>(cap, 2 * s0); ++s) {
    const int64_t total = itiles * s;
    const int64_t waves = (total + R - 1) / R;
    const int64_t tmax = (tiles + s - 1) / s;  // tiles of the longest split
    const double e = ((double)total / (double)(waves * R)) * ((double)tiles / (double)(s * tmax));
    if (e > best_e + 1e-9) {
      best = s;
      best_e = e;
    }
    if (e >= 0.95) break;
  }
  return (int)best;
}

#define NB_FP64_CASE(NT_, JT_) \
  if (cfg.threads == NT_ && cfg.jtile == JT_) return launch<NT_, JT_>(c, d_list, n, cfg, is);

cudaError_t nb_forces_fp64(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                           const nbk::ISrc* isrc) {
  if (n <= 0) return cudaSuccess;
  const nbk::ISrc is = isrc ? *isrc : nbk::ISrc();
  NB_FP64_CASE(64, 32) NB_FP64_CASE(64, 64) NB_FP64_CASE(64, 128)
  NB_FP64_CASE(128, 32) NB_FP64_CASE(128, 64) NB_FP64_CASE(128, 128)
  NB_FP64_CASE(256, 32) NB_FP64_CASE(256, 64) NB_FP64_CASE(256, 128)
  return cudaErrorInvalidValue;
}
