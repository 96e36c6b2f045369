// onboard.cu -- support kernels of the on-the-fly j prediction, GRAPE's split
// of a block step (Sec. 4.4 steps 3-7): the host predicts only the n active
// i-particles (step 3), the board predicts every j-particle as it streams
// through its pipelines (step 4) and computes the forces (step 5), the host
// corrects the block (step 7) and sends the corrected particles back to the
// board's j-memory (the 72 bytes per particle of t_comm).
//
// Here the "board" is the mixed force kernel (force_common.cuh, FusedSmem) and
// the j-memory an array of double-single records kept beside the FP64 state:
//   - nb_launch_jm_write: the records of a list of rows (after a correction)
//     or of every row (after any other change of the state), from the FP64
//     state; the reach Rd bounds how far a particle can move within its
//     current step, |delta_c| <= |v_c| h + |a_c| h^2/2 + |j_c| h^3/6 with
//     h <= dt_i, summed over components;
//     (the host loop's corrector writes the records of the rows it corrects
//     itself, hermite.cuh write_jm_record);
//   - nb_launch_jm_host_side, one launch: the active rows predicted in FP64
//     (hermite.cuh, the same arithmetic as the full predictor) into xp, vp
//     and jA/jB/jC, which the corrector and the force item's i-loads read;
//     and the boxes of the 128-row tiles for the far test, from the
//     unpredicted hi parts grown by each particle's reach (and a margin for
//     the FP32 roundings of the prediction), so that they contain the
//     predicted hi parts at any block time within every member's step.
#include <float.h>
#include <stdlib.h>

#include "hermite.cuh"
#include "nb_internal.cuh"

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

__global__ void jm_write_kernel(int64_t count, const int32_t* __restrict__ list, int64_t N, int64_t n_pad,
                                const double* __restrict__ m, const double* __restrict__ x,
                                const double* __restrict__ v, const double* __restrict__ a,
                                const double* __restrict__ jk, const double* __restrict__ dt,
                                float4* __restrict__ jm) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = list ? (int64_t)list[k] : k;
    i = i < 0 ? 0 : (i >= n_pad ? n_pad - 1 : i);  // a bad list never writes out of bounds
    nbh::write_jm_record(i, N, n_pad, m, x, v, a, jk, dt, jm);
  }
}

// One launch for the host side of the split: blocks [0, box_blocks) compute
// the boxes of the 128-row tiles (one warp per tile: (lo, rmax), (hi, 0) of
// the predicted hi parts, bounded from the records), the other blocks
// predict the listed (active) rows to t (Sec. 4.4 step 3) with the FP64
// predictor of every driver (hermite.cuh) into xp, vp and jA/jB/jC.
__global__ void jm_host_side_kernel(int64_t box_blocks, int64_t N, int64_t ntiles, int64_t n_pad,
                                    const float4* __restrict__ jm, float4* __restrict__ box, int64_t n,
                                    const int32_t* __restrict__ list, const double* __restrict__ m,
                                    const double* __restrict__ x, const double* __restrict__ v,
                                    const double* __restrict__ a, const double* __restrict__ jk,
                                    const double* __restrict__ ti, double t, double* __restrict__ xp,
                                    double* __restrict__ vp, float4* __restrict__ jA, float4* __restrict__ jB,
                                    float2* __restrict__ jC) {
  if ((int64_t)blockIdx.x >= box_blocks) {
    const int64_t nthreads = (int64_t)(gridDim.x - box_blocks) * blockDim.x;
    for (int64_t k = (blockIdx.x - box_blocks) * (int64_t)blockDim.x + threadIdx.x; k < n; k += nthreads) {
      int64_t i = list[k];
      i = i < 0 ? 0 : (i >= n_pad ? n_pad - 1 : i);
      double px[3], pv[3];
      nbh::taylor(i, n_pad, t - ti[i], x, v, a, jk, px, pv);
      nbh::store_predicted(i, n_pad, px, pv, m[i], xp, vp, jA, jB, jC, true, true);
    }
    return;
  }
  const int64_t tl = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tl >= ntiles) return;
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int q = lane; q < NB_BOX_TILE; q += 32) {
    const int64_t s = tl * NB_BOX_TILE + q;
    if (s >= N) break;
    const float4 r0 = jm[s];
    const float reach = jm[n_pad + s].w;
    const float p[3] = {r0.x, r0.y, r0.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // the reach plus the roundings of the hi parts (before and after the
      // prediction) and of this arithmetic: 2^-22 of |x| + reach covers them
      const float g = reach + 0x1p-22f * (fabsf(p[c]) + reach);
      lo[c] = fminf(lo[c], p[c] - g);
      hi[c] = fmaxf(hi[c], p[c] + g);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
  }
  if (lane == 0) {
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) r = fmaxf(r, fmaxf(fabsf(lo[c]), fabsf(hi[c])));
    if (!(lo[0] <= hi[0])) r = 0.0f;  // no real particle in the tile
    box[2 * tl] = make_float4(lo[0], lo[1], lo[2], r);
    box[2 * tl + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
  }
}

}  // namespace

cudaError_t nb_launch_jm_write(nb_ctx* c, const int32_t* d_list, int64_t count) {
  if (count <= 0) return cudaSuccess;
  c->launches += 1;
  jm_write_kernel<<<grid_for(count, kThreads, c->sm_count * 16), kThreads, 0, c->stream>>>(
      count, d_list, c->n, c->n_pad, c->m, c->x, c->v, c->a, c->jk, c->dt, c->jm);
  return cudaGetLastError();
}

cudaError_t nb_launch_jm_host_side(nb_ctx* c, const int32_t* d_list, int64_t n, double t, bool boxes) {
  const int64_t ntiles = boxes ? (c->n + NB_BOX_TILE - 1) / NB_BOX_TILE : 0;
  const int64_t box_blocks = (ntiles + 7) / 8;  // 8 warps, 8 tiles per block
  const int64_t list_blocks = n > 0 ? grid_for(n, kThreads, c->sm_count * 16) : 0;
  if (box_blocks + list_blocks == 0) return cudaSuccess;
  c->launches += 1;
  jm_host_side_kernel<<<(unsigned)(box_blocks + list_blocks), kThreads, 0, c->stream>>>(
      box_blocks, c->n, ntiles, c->n_pad, c->jm, c->tbox, n, d_list, c->m, c->x, c->v, c->a, c->jk, c->t, t,
      c->xp, c->vp, c->jA, c->jB, c->jC);
  return cudaGetLastError();
}

int nb_jm_ensure(nb_ctx* c) {
  if (!c->jm) {
    if (cudaMalloc((void**)&c->jm, (size_t)5 * c->n_pad * sizeof(float4)) != cudaSuccess) {
      cudaGetLastError();
      c->jm = nullptr;
      return NB_ENOMEM;
    }
    c->jm_ver = c->state_ver - 1;
  }
  if (c->jm_ver != c->state_ver) {
    if (nb_launch_jm_write(c, nullptr, c->n_pad) != cudaSuccess) return NB_ECUDA;
    c->jm_ver = c->state_ver;
  }
  return NB_OK;
}
