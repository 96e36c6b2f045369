// ensemble.cu -- device-driven block steps for one or many independent
// systems ("clusters"): the CUDA-graph integration loop of a single system
// (nb_integrate with use_graph) and the batched ensemble (nb_ensemble_*).
//
// Every kernel reads the block state from device memory, so a whole block
// step -- selection (Sec. 4.1 step 2), prediction (3), forces (4), correction
// (5) -- needs no host round trip, and the loop of steps 2-6 runs as one CUDA
// graph whose body sits in a device-side while node.  All clusters advance
// together: each body iteration takes the next block step of every cluster
// that has not reached t_end (each at its own block time), and the force work
// of all clusters is flattened into one list of (cluster, i-tile, j-split)
// items that a persistent kernel spreads over all SMs.  Clusters of very
// different size and block size therefore share the GPU without a per-cluster
// critical path.
//
// Cluster c owns particles [off[c], off[c+1]) of the j-store and the same
// slots of the active list and of the force results.
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "force_common.cuh"
#include "hermite.cuh"

namespace {

#ifndef NB_ENS_ITEM_WAVES
#define NB_ENS_ITEM_WAVES 4
#endif
constexpr int kItemWaves = NB_ENS_ITEM_WAVES;  // force items planned per resident CTA
constexpr int kCorrItem = 128;    // active particles per corrector item (= its threads per CTA)
constexpr int kSelChunk = 512;    // particles per selection chunk (chunks never straddle clusters)
// batched item shapes: i-tile = threads per CTA, one i per thread.  An
// ensemble of small clusters has small active blocks (n = 0.20 N^0.81 is 18
// at N = 256 and 169 at N = 4096), so it takes 32-particle i-tiles that
// leave few lanes idle; the single-system graph loop takes 128.
constexpr int kMixIPT = 1, kMixJT = 128;  // batched mixed item: j-tile
constexpr int kF64JT = 64;                // batched FP64 item: j-tile
constexpr int64_t kMaxIters = 50000000;                  // hard cap on loop iterations

struct BParams {
  double t_end, eta, dt_min, dt_max;
  int64_t max_iters;
  int64_t seg_iters;  // > 0: stop after this many block steps of this launch (ctrl[3] = 1)
};

struct Batch {
  int32_t C = 0;
  int64_t N = 0;
  int32_t nchunks = 0;
  // device
  int64_t* off = nullptr;          // [C+1]
  float* eps2f = nullptr;          // [C]
  double* eps2d = nullptr;         // [C]
  int32_t* cid = nullptr;          // [n_pad] cluster of a particle / slot
  int32_t* ch_cluster = nullptr;   // [nchunks]
  int64_t* ch_lo = nullptr;        // [nchunks]
  int64_t* ch_hi = nullptr;        // [nchunks]
  int32_t* cl_ch0 = nullptr;       // [C+1] first chunk of each cluster
  unsigned long long* ch_min = nullptr;  // [nchunks]
  int32_t* ch_cnt = nullptr;       // [nchunks]
  double* tnext = nullptr;         // [C]
  int32_t* nact = nullptr;         // [C]
  int32_t* itiles = nullptr;       // [C]
  int32_t* nsplit = nullptr;       // [C]
  int64_t* jps = nullptr;          // [C] j per split
  int64_t* item_off = nullptr;     // [C+1]
  int64_t* ritem_off = nullptr;    // [C+1] split-reduction items (32 positions) per cluster
  int64_t* citem_off = nullptr;    // [C+1] corrector items (kCorrItem active particles) per cluster
  unsigned long long* wq = nullptr;  // force-item counter of the current step
  int64_t* part_off = nullptr;     // [C]
  int64_t* pstride = nullptr;      // [C]
  int64_t* ctrl = nullptr;         // [4]: any active, iterations, interactions (as int64), spare
  BParams* prm = nullptr;
  double* esum = nullptr;          // [2C] per-cluster energies
  // spatial order within each cluster (mixed ensembles of at most 2^11 clusters)
  int64_t* tile_off = nullptr;     // [C+1] first 128-row box tile of each cluster
  int32_t* tile_cl = nullptr;      // [ntiles] cluster of each box tile
  float4* tbox = nullptr;          // [2 ntiles] boxes of the predicted tiles
  double* cbox = nullptr;          // [6C] bounding box of each cluster
  int64_t ntiles = 0;
  int cl_bits = 0;                 // bits of a cluster number in the sort keys
  // host
  std::vector<int64_t> h_off;
  int nt = 128;                    // i-tile (threads per CTA) of the force items: 32, 64 or 128
  int waves = kItemWaves;          // force items planned per resident CTA (sets the split-j length)
  int64_t nc_median = 0;           // median cluster size (the autotuner's bin)
  int grid_mixed = 0, grid_fp64 = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t exec_key = -1;           // precision, far-tile pass and item shape the graph was built for
  nb_ctx* child = nullptr;         // per-cluster reference path
};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

// ---------------------------------------------------------------------------
// selection (Sec. 4.1 step 2) per cluster: t_next[c] = min (t_i + dt_i) over
// the cluster; active slots off[c] + k, k < n_c, ascending index.
// ---------------------------------------------------------------------------
__global__ void b_sel_min(const int64_t* __restrict__ lo, const int64_t* __restrict__ hi,
                          const double* __restrict__ ti, const double* __restrict__ dt,
                          unsigned long long* __restrict__ ch_min) {
  const int j = blockIdx.x;
  unsigned long long best = 0x7FF0000000000000ULL;
  for (int64_t i = lo[j] + threadIdx.x; i < hi[j]; i += blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(ti[i] + dt[i]);
    best = b < best ? b : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
  }
  __shared__ unsigned long long sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = sm[w] < best ? sm[w] : best;
    best = sm[0] < best ? sm[0] : best;
    ch_min[j] = best;
  }
}

// the cluster's block time: minimum over its chunks, by the calling warp
// (every lane returns it)
__device__ __forceinline__ double cluster_tmin(const unsigned long long* ch_min, int a, int b) {
  const int lane = threadIdx.x & 31;
  unsigned long long best = 0x7FF0000000000000ULL;
  for (int q = a + lane; q < b; q += 32) best = ch_min[q] < best ? ch_min[q] : best;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
  }
  return __longlong_as_double((long long)best);
}

// (also: an active cluster's block time must exceed the one it had at the
// previous iteration of this launch, else the state has no valid steps, e.g.
// dt = 0: NB_ST_STALLED, and the plan ends the loop)
__global__ void b_sel_count(const int32_t* __restrict__ ch_cluster, const int64_t* __restrict__ lo,
                            const int64_t* __restrict__ hi, const int32_t* __restrict__ cl_ch0,
                            const unsigned long long* __restrict__ ch_min, const double* __restrict__ ti,
                            const double* __restrict__ dt, double* __restrict__ tnext,
                            int32_t* __restrict__ ch_cnt, const int64_t* __restrict__ ctrl,
                            const BParams* __restrict__ prm, nb_dev_status* __restrict__ st) {
  const int j = blockIdx.x;
  const int c = ch_cluster[j];
  __shared__ double tn;
  if (threadIdx.x < 32) {
    const double t = cluster_tmin(ch_min, cl_ch0[c], cl_ch0[c + 1]);
    if (threadIdx.x == 0) {
      tn = t;
      if (j == cl_ch0[c]) {
        if (ctrl[1] > 0 && t <= prm->t_end && !(t > tnext[c])) atomicOr(&st->flags, NB_ST_STALLED);
        tnext[c] = t;
      }
    }
  }
  __syncthreads();
  int cnt = 0;
  for (int64_t i = lo[j] + threadIdx.x; i < hi[j]; i += blockDim.x) cnt += (ti[i] + dt[i] == tn) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ int sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    ch_cnt[j] = s;
  }
}

__global__ void b_sel_write(const int32_t* __restrict__ ch_cluster, const int64_t* __restrict__ lo,
                            const int64_t* __restrict__ hi, const int32_t* __restrict__ cl_ch0,
                            const int32_t* __restrict__ ch_cnt, const int64_t* __restrict__ off,
                            const double* __restrict__ ti, const double* __restrict__ dt,
                            const double* __restrict__ tnext, const BParams* __restrict__ prm,
                            int32_t* __restrict__ act, int32_t* __restrict__ nact) {
  const int j = blockIdx.x;
  const int c = ch_cluster[j];
  const double tn = tnext[c];
  __shared__ int base_s;
  if (threadIdx.x < 32) {  // counts of the cluster's chunks before this one, and in all
    int b = 0, tot = 0;
    for (int q = cl_ch0[c] + (int)threadIdx.x; q < cl_ch0[c + 1]; q += 32) {
      if (q < j) b += ch_cnt[q];
      tot += ch_cnt[q];
    }
    for (int o = 16; o > 0; o >>= 1) {
      b += __shfl_xor_sync(0xffffffffu, b, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (threadIdx.x == 0) {
      base_s = b;
      if (j == cl_ch0[c]) nact[c] = (tn <= prm->t_end) ? tot : 0;
    }
  }
  __syncthreads();
  int base = (int)off[c] + base_s;
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t seg = lo[j]; seg < hi[j]; seg += blockDim.x) {
    const int64_t i = seg + threadIdx.x;
    const bool f = (i < hi[j]) && (ti[i] + dt[i] == tn);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int wpre = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int cc = wsum[w];
      if (w < wid) wpre += cc;
      tot += cc;
    }
    if (f) act[base + wpre + pre] = (int32_t)i;
    base += tot;
    __syncthreads();
  }
}

// all particles active at their own time (initial forces / energies)
__global__ void b_all_active(int32_t C, const int64_t* __restrict__ off, int64_t N, int32_t* __restrict__ act,
                             int32_t* __restrict__ nact, double* __restrict__ tnext) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    act[i] = (int32_t)i;
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      nact[c] = (int32_t)(off[c + 1] - off[c]);
      tnext[c] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// plan: per cluster i-tiles and j-splits, flattened item offsets, partial-sum
// offsets; loop control (any cluster active, iteration cap).  One CTA.
// The j-split length L is common to all clusters and chosen so that the whole
// batch yields about 4 items per resident CTA.
// ---------------------------------------------------------------------------
__device__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  // Hillis-Steele over blockDim.x <= 1024 entries
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int64_t add = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  const int64_t incl = sh[t];
  *total = sh[blockDim.x - 1];
  __syncthreads();
  return incl - v;
}

__global__ void b_plan(int32_t C, const int64_t* __restrict__ off, const int32_t* __restrict__ nact,
                       int per_cta, int jtile, int64_t target_items, int64_t part_cap,
                       int32_t* __restrict__ itiles, int32_t* __restrict__ nsplit, int64_t* __restrict__ jps,
                       int64_t* __restrict__ item_off, int64_t* __restrict__ part_off,
                       int64_t* __restrict__ pstride, int64_t* __restrict__ ritem_off,
                       int64_t* __restrict__ citem_off, unsigned long long* __restrict__ wq,
                       int64_t* __restrict__ ctrl,
                       const BParams* __restrict__ prm, nb_dev_status* __restrict__ st,
                       cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ int64_t sh[1024];
  __shared__ int64_t s_L;
  __shared__ int s_retry;
  const int t = threadIdx.x;
  // pass 1: total slot-pair work and activity
  int64_t w = 0, anyact = 0, inter = 0;
  for (int c = t; c < C; c += blockDim.x) {
    const int64_t n = nact[c];
    const int64_t Nc = off[c + 1] - off[c];
    const int64_t it = (n + per_cta - 1) / per_cta;
    w += it * per_cta * Nc;
    anyact += n > 0;
    inter += n * Nc;
  }
  int64_t tot_w, tot_a, tot_i;
  block_excl_scan(w, sh, &tot_w);
  block_excl_scan(anyact, sh, &tot_a);
  block_excl_scan(inter, sh, &tot_i);
  if (t == 0) {
    int64_t L = tot_w / ((int64_t)per_cta * (target_items > 0 ? target_items : 1));
    L = ((L + jtile - 1) / jtile) * jtile;
    s_L = L < jtile ? jtile : L;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 40; ++attempt) {
    const int64_t L = s_L;
    int64_t item_carry = 0, part_carry = 0, ritem_carry = 0, citem_carry = 0;
    for (int c0 = 0; c0 < C; c0 += blockDim.x) {
      const int c = c0 + t;
      int64_t items = 0, psz = 0, ritems = 0, citems = 0;
      int32_t it = 0, ns = 1;
      int64_t jp = 0, ps = 0;
      if (c < C) {
        const int64_t n = nact[c];
        const int64_t Nc = off[c + 1] - off[c];
        it = (int32_t)((n + per_cta - 1) / per_cta);
        const int64_t tiles = (Nc + jtile - 1) / jtile;
        int64_t s = (Nc + L - 1) / L;
        if (s > tiles) s = tiles;
        if (s < 1) s = 1;
        const int64_t tps = (tiles + s - 1) / s;
        s = (tiles + tps - 1) / tps;
        ns = (int32_t)s;
        jp = tps * jtile;
        ps = ((n + 31) / 32) * 32;
        items = (int64_t)it * s;
        psz = s > 1 ? 7 * s * ps : 0;
        ritems = s > 1 ? 7 * ((n + 31) / 32) : 0;
        citems = (n + kCorrItem - 1) / kCorrItem;
      }
      int64_t tot_items, tot_part, tot_ritems, tot_citems;
      const int64_t ex_items = block_excl_scan(items, sh, &tot_items);
      const int64_t ex_part = block_excl_scan(psz, sh, &tot_part);
      const int64_t ex_ritems = block_excl_scan(ritems, sh, &tot_ritems);
      const int64_t ex_citems = block_excl_scan(citems, sh, &tot_citems);
      if (c < C) {
        itiles[c] = it;
        nsplit[c] = ns;
        jps[c] = jp;
        pstride[c] = ps;
        item_off[c] = item_carry + ex_items;
        part_off[c] = part_carry + ex_part;
        ritem_off[c] = ritem_carry + ex_ritems;
        citem_off[c] = citem_carry + ex_citems;
      }
      item_carry += tot_items;
      part_carry += tot_part;
      ritem_carry += tot_ritems;
      citem_carry += tot_citems;
    }
    if (t == 0) {
      item_off[C] = item_carry;
      ritem_off[C] = ritem_carry;
      citem_off[C] = citem_carry;
      s_retry = part_carry > part_cap;
      if (s_retry) s_L = s_L * 2;
    }
    __syncthreads();
    if (!s_retry) break;
  }
  if (t == 0) {
    *wq = 0;  // the force kernel of this step starts at item 0
    int64_t iters = ctrl[1] + 1;
    ctrl[1] = iters;
    ctrl[2] += tot_i;
    int go = tot_a > 0;
    if (go && (st->flags & NB_ST_STALLED)) go = 0;  // a block time did not advance (b_sel_count)
    if (go && iters > prm->max_iters) {
      atomicOr(&st->flags, NB_ST_TIMEOUT);
      go = 0;
    }
    if (go && prm->seg_iters > 0 && iters >= prm->seg_iters) {
      ctrl[3] = 1;  // this step runs; the launch ends after it with work left
      go = 0;
    }
    if (s_retry) {  // partial sums do not fit: stop with an error instead of overflowing
      atomicOr(&st->flags, NB_ST_TIMEOUT);
      go = 0;
      item_off[C] = 0;
      ritem_off[C] = 0;
      citem_off[C] = 0;
    }
    ctrl[0] = go;
    if (use_handle) cudaGraphSetConditional(handle, go ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// predictor per cluster (Sec. 4.1 step 3): particles of active clusters to
// their cluster's block time (own_time: h = 0).
// ---------------------------------------------------------------------------
__global__ void b_predict(int64_t N, int64_t n_pad, const int32_t* __restrict__ cid,
                          const int32_t* __restrict__ nact, const double* __restrict__ tnext, int own_time,
                          const double* __restrict__ m, const double* __restrict__ x,
                          const double* __restrict__ v, const double* __restrict__ a,
                          const double* __restrict__ jk, const double* __restrict__ ti,
                          double* __restrict__ xp, double* __restrict__ vp, float4* __restrict__ jA,
                          float4* __restrict__ jB, float2* __restrict__ jC, int write_fp64, int write_mixed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cid[i];
    if (nact[c] == 0) continue;
    double px[3], pv[3];
    nbh::taylor(i, n_pad, own_time ? 0.0 : tnext[c] - ti[i], x, v, a, jk, px, pv);
    nbh::store_predicted(i, n_pad, px, pv, m[i], xp, vp, jA, jB, jC, write_fp64 != 0, write_mixed != 0);
  }
}

// ---------------------------------------------------------------------------
// forces (Sec. 4.1 step 4): persistent CTAs over the flattened item list
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_cluster(const int64_t* __restrict__ item_off, int C, int64_t item) {
  int lo = 0, hi = C;  // item_off[lo] <= item < item_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (item_off[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// the next force item for this CTA from the step's work counter (reset by
// b_plan): items go to whichever CTA is free first, so uneven items (near or
// far tiles, big or small clusters) do not leave SMs idle at the end of a
// step.  One atomic per item; no waiting.
__device__ __forceinline__ int64_t next_item(unsigned long long* wq, int64_t* s_item) {
  __syncthreads();  // every thread has read the previous item
  if (threadIdx.x == 0) *s_item = (int64_t)atomicAdd(wq, 1ULL);
  __syncthreads();
  return *s_item;
}

// resident CTAs per SM asked of the register allocator: the host-launched
// mixed kernel fits 94 registers (5 CTAs of 128); the item loop must not
// cost a CTA per SM (117 registers unbounded = 4 CTAs of 128).  The FP64
// item keeps the default (bounding it to 96 registers spills).
constexpr int mixed_min_ctas(int nt) { return nt >= 128 ? 5 : 640 / nt; }

template <int NT, int IPT, int JT>
__global__ void __launch_bounds__(NT, mixed_min_ctas(NT)) b_force_mixed(
    int32_t C, const int64_t* __restrict__ off, const float* __restrict__ eps2f, int64_t n_pad,
    const float4* __restrict__ jA, const float4* __restrict__ jB, const float2* __restrict__ jC,
    const int32_t* __restrict__ act, const int32_t* __restrict__ nact, const int32_t* __restrict__ itiles,
    const int32_t* __restrict__ nsplit, const int64_t* __restrict__ jps, const int64_t* __restrict__ item_off,
    const int64_t* __restrict__ part_off, const int64_t* __restrict__ pstride, double* __restrict__ F,
    int64_t fstride, double* __restrict__ part, const float4* __restrict__ tbox,
    const int64_t* __restrict__ tile_off, unsigned long long* __restrict__ wq) {
  __shared__ __align__(16) nbk::MixedSmem<JT> sm;
  __shared__ int64_t s_item;
  const int64_t total = item_off[C];
  for (;;) {
    const int64_t item = next_item(wq, &s_item);
    if (item >= total) break;
    const int c = find_cluster(item_off, C, item);
    const int64_t local = item - item_off[c];
    const int it = itiles[c];
    const int64_t itile = local % it, split = local / it;
    const int64_t jlo = off[c] + split * jps[c];
    const int64_t jhi = min(jlo + jps[c], off[c + 1]);
    const bool fin = nsplit[c] == 1;
    double* out = fin ? F + off[c] : part + part_off[c] + split * 7 * pstride[c];
    // boxes: of the whole j-store (one system) or of the cluster's own tiles
    const float4* tb = tbox ? (tile_off ? tbox + 2 * tile_off[c] : tbox) : nullptr;
    nbk::mixed_item<NT, IPT, JT>(sm, jA, jB, jC, jlo, jhi, n_pad, act + off[c], nact[c], itile * (NT * IPT),
                                 eps2f[c], out, fin ? fstride : pstride[c], fin, tb, nullptr,
                                 tile_off ? off[c] : 0);
  }
}

template <int NT, int JT>
__global__ void __launch_bounds__(NT) b_force_fp64(
    int32_t C, const int64_t* __restrict__ off, const double* __restrict__ eps2d, int64_t n_pad,
    const double* __restrict__ xp, const double* __restrict__ vp, const double* __restrict__ m,
    const int32_t* __restrict__ act, const int32_t* __restrict__ nact, const int32_t* __restrict__ itiles,
    const int32_t* __restrict__ nsplit, const int64_t* __restrict__ jps, const int64_t* __restrict__ item_off,
    const int64_t* __restrict__ part_off, const int64_t* __restrict__ pstride, double* __restrict__ F,
    int64_t fstride, double* __restrict__ part, unsigned long long* __restrict__ wq) {
  __shared__ nbk::Fp64Smem<JT> sm;
  __shared__ int64_t s_item;
  const int64_t total = item_off[C];
  for (;;) {
    const int64_t item = next_item(wq, &s_item);
    if (item >= total) break;
    const int c = find_cluster(item_off, C, item);
    const int64_t local = item - item_off[c];
    const int it = itiles[c];
    const int64_t itile = local % it, split = local / it;
    const int64_t jlo = off[c] + split * jps[c];
    const int64_t jhi = min(jlo + jps[c], off[c + 1]);
    const bool fin = nsplit[c] == 1;
    double* out = fin ? F + off[c] : part + part_off[c] + split * 7 * pstride[c];
    nbk::fp64_item<NT, JT>(sm, xp, vp, m, n_pad, jlo, jhi, act + off[c], nact[c], itile * NT, eps2d[c], out,
                           fin ? fstride : pstride[c], fin);
  }
}

// split-j reduction of the active clusters: one item = one of the 7 result
// rows of 32 consecutive positions of one cluster with splits (item list from
// b_plan); block = 32 positions x kRedLanes split lanes; lane y sums splits
// y, y + kRedLanes, ... in order and a fixed binary tree combines the lanes
// (one summation order per split count).  Clusters with one split wrote their
// results directly and have no items.
#ifndef NB_ENS_RED_LANES
#define NB_ENS_RED_LANES 8
#endif
constexpr int kRedLanes = NB_ENS_RED_LANES;
__global__ void b_reduce(int32_t C, const int64_t* __restrict__ off, const int32_t* __restrict__ nact,
                         const int32_t* __restrict__ nsplit, const int64_t* __restrict__ part_off,
                         const int64_t* __restrict__ pstride, const int64_t* __restrict__ ritem_off,
                         const double* __restrict__ part, double* __restrict__ F, int64_t fstride) {
  __shared__ double sm[kRedLanes][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t total = ritem_off[C];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_cluster(ritem_off, C, item);
    const int S = nsplit[c];
    const int64_t n = nact[c], o = off[c], ps = pstride[c];
    const double* p = part + part_off[c];
    const int64_t local = item - ritem_off[c];
    const int r = (int)(local % 7);
    const int64_t k = (local / 7) * 32 + tx;
    double acc = 0.0;
    if (k < n)
      for (int q = ty; q < S; q += kRedLanes) acc += p[((int64_t)q * 7 + r) * ps + k];
    sm[ty][tx] = acc;
    __syncthreads();
#pragma unroll
    for (int h = kRedLanes / 2; h > 0; h >>= 1) {
      if (ty < h) sm[ty][tx] += sm[ty + h][tx];
      __syncthreads();
    }
    if (ty == 0 && k < n) F[r * fstride + o + k] = r == 6 ? -sm[0][tx] : sm[0][tx];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// spatial order within each cluster: cluster boxes, keys = cluster number
// above a 21-bit Morton code of the position in the cluster's box (a stable
// sort keeps every cluster on its own rows), boxes of 128-row tiles counted
// from each cluster's first row
// ---------------------------------------------------------------------------
__global__ void b_cluster_bbox(const int64_t* __restrict__ off, int64_t n_pad, const double* __restrict__ x,
                               double* __restrict__ cbox) {
  const int c = blockIdx.x;
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t s = off[c] + threadIdx.x; s < off[c + 1]; s += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      const double v = x[d * n_pad + s];
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  __shared__ double sm[6][256];
  for (int d = 0; d < 3; ++d) {
    sm[d][threadIdx.x] = lo[d];
    sm[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int d = 0; d < 3; ++d) {
        sm[d][threadIdx.x] = fmin(sm[d][threadIdx.x], sm[d][threadIdx.x + w]);
        sm[3 + d][threadIdx.x] = fmax(sm[3 + d][threadIdx.x], sm[3 + d][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) cbox[6 * c + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void b_cluster_keys(int64_t N, int64_t n_pad, const int32_t* __restrict__ cid,
                               const double* __restrict__ x, const double* __restrict__ cbox,
                               uint32_t* __restrict__ key, int32_t* __restrict__ val) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
    const int c = cid[s];
    const double* bx = cbox + 6 * c;
    double scale = fmax(bx[3] - bx[0], fmax(bx[4] - bx[1], bx[5] - bx[2]));
    scale = scale > 0.0 ? 127.0 / scale : 0.0;
    uint32_t q[3];
    for (int d = 0; d < 3; ++d) {
      double f = (x[d * n_pad + s] - bx[d]) * scale;
      f = f < 0.0 ? 0.0 : (f > 127.0 ? 127.0 : f);
      q[d] = (uint32_t)f;
    }
    key[s] = ((uint32_t)c << 21) | nb_spread10(q[0]) | (nb_spread10(q[1]) << 1) | (nb_spread10(q[2]) << 2);
    val[s] = (int32_t)s;
  }
}

// one warp per box tile: box of the predicted FP32 hi positions, (lo, rmax), (hi, 0)
__global__ void b_tile_boxes(int64_t ntiles, const int32_t* __restrict__ tile_cl,
                             const int64_t* __restrict__ tile_off, const int64_t* __restrict__ off,
                             const float4* __restrict__ jA, float4* __restrict__ box) {
  const int64_t g = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= ntiles) return;
  const int c = tile_cl[g];
  const int64_t s0 = off[c] + (g - tile_off[c]) * NB_BOX_TILE;
  const int64_t s1 = min(s0 + NB_BOX_TILE, off[c + 1]);
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX}, r = 0.0f;
  for (int64_t s = s0 + lane; s < s1; s += 32) {
    const float4 a = jA[s];
    const float p[3] = {a.x, a.y, a.z};
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], p[d]);
      hi[d] = fmaxf(hi[d], p[d]);
      r = fmaxf(r, fabsf(p[d]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
    r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
  }
  if (lane == 0) {
    box[2 * g] = make_float4(lo[0], lo[1], lo[2], r);
    box[2 * g + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
  }
}

// corrector + block-step rule (Sec. 4.1 step 5), per slot of active clusters
__global__ void b_correct(int32_t C, int64_t n_pad, const int64_t* __restrict__ citem_off,
                          const int64_t* __restrict__ off, const int32_t* __restrict__ nact,
                          const double* __restrict__ tnext, const int32_t* __restrict__ act,
                          const double* __restrict__ F, int64_t fstride, const BParams* __restrict__ prm,
                          double* __restrict__ x, double* __restrict__ v, double* __restrict__ a,
                          double* __restrict__ jk, double* __restrict__ pot, double* __restrict__ ti,
                          double* __restrict__ dt, const double* __restrict__ xp,
                          const double* __restrict__ vp, nb_dev_status* __restrict__ st) {
  const double eta = prm->eta, dt_min = prm->dt_min, dt_max = prm->dt_max;
  // items of kCorrItem active particles of one cluster (planned by b_plan)
  const int64_t total = citem_off[C];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_cluster(citem_off, C, item);
    const int64_t k = (item - citem_off[c]) * kCorrItem + threadIdx.x;
    if (k >= nact[c]) continue;
    const int64_t s = off[c] + k;
    int64_t i = act[s];
    i = i < 0 ? 0 : (i >= n_pad ? n_pad - 1 : i);
    double f[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) f[r] = F[r * fstride + s];
    nbh::correct_row(i, n_pad, tnext[c], f, eta, dt_min, dt_max, x, v, a, jk, pot, ti, dt, xp, vp, st);
  }
}

// initial steps for every particle of every cluster (Sec. 4.1 step 1)
__global__ void b_initial_dt(int64_t N, int64_t n_pad, const double* __restrict__ F, int64_t fstride,
                             const BParams* __restrict__ prm, double* __restrict__ a, double* __restrict__ jk,
                             double* __restrict__ pot, double* __restrict__ ti, double* __restrict__ dt,
                             nb_dev_status* __restrict__ st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double na2 = 0, nj2 = 0;
    bool finite = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double av = F[r * fstride + i], jv = F[(3 + r) * fstride + i];
      a[r * n_pad + i] = av;
      jk[r * n_pad + i] = jv;
      na2 += av * av;
      nj2 += jv * jv;
      finite = finite && isfinite(av) && isfinite(jv);
    }
    pot[i] = F[6 * fstride + i];
    const double nj = sqrt(nj2);
    const double d = (nj > 0.0) ? prm->eta * sqrt(na2) / nj : (double)INFINITY;
    dt[i] = nbh::clamp_dt(nbh::pow2_floor(d), prm->dt_min, prm->dt_max);
    ti[i] = 0.0;
    if (!finite) atomicOr(&st->flags, NB_ST_NUMERIC);
  }
}

// per-cluster energies: K = sum m v^2/2, W = sum m pot/2 (fixed order per CTA)
__global__ void b_energy(const int64_t* __restrict__ off, int64_t n_pad, const double* __restrict__ m,
                         const double* __restrict__ v, const double* __restrict__ F, int64_t fstride,
                         double* __restrict__ out) {
  const int c = blockIdx.x;
  double k = 0.0, w = 0.0;
  for (int64_t i = off[c] + threadIdx.x; i < off[c + 1]; i += blockDim.x) {
    const double v0 = v[i], v1 = v[n_pad + i], v2 = v[2 * n_pad + i];
    k += 0.5 * m[i] * (v0 * v0 + v1 * v1 + v2 * v2);
    w += 0.5 * m[i] * F[6 * fstride + i];
  }
  __shared__ double sk[256], sw[256];
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
    out[2 * c] = sk[0];
    out[2 * c + 1] = sw[0];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
Batch* batch_of(nb_ctx* c) { return (Batch*)c->ens; }

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

void batch_free(Batch* b) {
  if (!b) return;
  void* p[] = {b->off, b->eps2f, b->eps2d, b->cid, b->ch_cluster, b->ch_lo, b->ch_hi, b->cl_ch0, b->ch_min,
               b->ch_cnt, b->tnext, b->nact, b->itiles, b->nsplit, b->jps, b->item_off, b->ritem_off, b->citem_off, b->part_off,
               b->pstride, b->ctrl, b->prm, b->esum, b->wq, b->tile_off, b->tile_cl, b->tbox, b->cbox};
  for (void* q : p)
    if (q) cudaFree(q);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->child) nb_destroy(b->child);
  delete b;
}

__global__ void fill_cid(int64_t N, const int64_t* __restrict__ off, int32_t C, int32_t* __restrict__ cid) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = C;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= i) lo = mid;
      else hi = mid;
    }
    cid[i] = lo;
  }
}

// build the batch description for clusters h_off[0..C] with softenings eps
// i-tile and planned items per CTA of the force items; the persistent grids
// hold as many CTAs as fit on the SMs at that i-tile
cudaError_t set_shape(nb_ctx* c, Batch* b, int nt, int waves) {
  int pm = 0, pf = 0;
  cudaError_t e;
  if (nt == 32) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, b_force_mixed<32, kMixIPT, kMixJT>, 32, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, b_force_fp64<32, kF64JT>, 32, 0);
  } else if (nt == 64) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, b_force_mixed<64, kMixIPT, kMixJT>, 64, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, b_force_fp64<64, kF64JT>, 64, 0);
  } else if (nt == 128) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, b_force_mixed<128, kMixIPT, kMixJT>, 128, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, b_force_fp64<128, kF64JT>, 128, 0);
  } else {
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  b->nt = nt;
  b->waves = waves;
  b->grid_mixed = std::max(1, pm) * c->sm_count;
  b->grid_fp64 = std::max(1, pf) * c->sm_count;
  return cudaSuccess;
}

// the item shape for this batch: the autotuner's entry for its median cluster
// size and cluster count (and the context's precision), else the defaults
// (32-particle i-tiles for ensembles, 128 for one system; kItemWaves)
cudaError_t pick_shape(nb_ctx* c, Batch* b) {
  int nt = b->C > 1 ? 32 : 128, waves = kItemWaves;
  if (const nb_tune_entry* t = nb_tune_find(c, NB_TUNE_BATCHED, b->nc_median, b->C)) {
    nt = t->cfg.threads;
    waves = t->cfg.waves;
  }
  if (nt == b->nt && waves == b->waves) return cudaSuccess;
  return set_shape(c, b, nt, waves);
}

cudaError_t batch_build(nb_ctx* c, int32_t C, const int64_t* h_off, const double* eps, Batch** out) {
  Batch* b = new (std::nothrow) Batch();
  if (!b) return cudaErrorMemoryAllocation;
  b->C = C;
  b->N = h_off[C];
  b->h_off.assign(h_off, h_off + C + 1);
  std::vector<int32_t> chc, clch0(C + 1);
  std::vector<int64_t> chlo, chhi;
  for (int32_t q = 0; q < C; ++q) {
    clch0[q] = (int32_t)chc.size();
    for (int64_t s = h_off[q]; s < h_off[q + 1]; s += kSelChunk) {
      chc.push_back(q);
      chlo.push_back(s);
      chhi.push_back(std::min<int64_t>(s + kSelChunk, h_off[q + 1]));
    }
  }
  clch0[C] = (int32_t)chc.size();
  b->nchunks = (int32_t)chc.size();
  std::vector<float> e2f(C);
  std::vector<double> e2d(C);
  for (int32_t q = 0; q < C; ++q) {
    e2d[q] = eps[q] * eps[q];
    e2f[q] = (float)e2d[q];
  }
  cudaError_t e = cudaSuccess;
#define BA(p, n) \
  if (e == cudaSuccess) e = dalloc(&(p), (n));
  BA(b->off, C + 1) BA(b->eps2f, C) BA(b->eps2d, C) BA(b->cid, c->n_pad) BA(b->ch_cluster, b->nchunks)
  BA(b->ch_lo, b->nchunks) BA(b->ch_hi, b->nchunks) BA(b->cl_ch0, C + 1) BA(b->ch_min, b->nchunks)
  BA(b->ch_cnt, b->nchunks) BA(b->tnext, C) BA(b->nact, C) BA(b->itiles, C) BA(b->nsplit, C) BA(b->jps, C)
  BA(b->item_off, C + 1) BA(b->ritem_off, C + 1) BA(b->citem_off, C + 1) BA(b->wq, 1) BA(b->part_off, C) BA(b->pstride, C) BA(b->ctrl, 4) BA(b->prm, 1) BA(b->esum, 2 * C)
  // box tiles of 128 rows counted from each cluster's first row
  std::vector<int64_t> toff(C + 1);
  std::vector<int32_t> tcl;
  for (int32_t q = 0; q < C; ++q) {
    toff[q] = (int64_t)tcl.size();
    for (int64_t s = h_off[q]; s < h_off[q + 1]; s += NB_BOX_TILE) tcl.push_back(q);
  }
  toff[C] = (int64_t)tcl.size();
  b->ntiles = toff[C];
  while (b->cl_bits < 31 && ((int64_t)1 << b->cl_bits) < C) ++b->cl_bits;
  if (C > 1 && b->cl_bits <= 11) {
    BA(b->tile_off, C + 1) BA(b->tile_cl, b->ntiles) BA(b->tbox, 2 * b->ntiles) BA(b->cbox, 6 * C)
  }
#undef BA
  auto H2D = [&](void* d, const void* h, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c->stream);
  };
  H2D(b->off, h_off, (C + 1) * sizeof(int64_t));
  H2D(b->eps2f, e2f.data(), C * sizeof(float));
  H2D(b->eps2d, e2d.data(), C * sizeof(double));
  H2D(b->ch_cluster, chc.data(), chc.size() * sizeof(int32_t));
  H2D(b->ch_lo, chlo.data(), chlo.size() * sizeof(int64_t));
  H2D(b->ch_hi, chhi.data(), chhi.size() * sizeof(int64_t));
  H2D(b->cl_ch0, clch0.data(), clch0.size() * sizeof(int32_t));
  if (b->tile_off) {
    H2D(b->tile_off, toff.data(), toff.size() * sizeof(int64_t));
    H2D(b->tile_cl, tcl.data(), tcl.size() * sizeof(int32_t));
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ctrl, 0, 4 * sizeof(int64_t), c->stream);
  if (e == cudaSuccess && b->N > 0) {
    fill_cid<<<grid_for(b->N, 256, 4096), 256, 0, c->stream>>>(b->N, b->off, C, b->cid);
    e = cudaGetLastError();
  }
  {
    std::vector<int64_t> sz(C);
    for (int32_t q = 0; q < C; ++q) sz[q] = h_off[q + 1] - h_off[q];
    std::nth_element(sz.begin(), sz.begin() + C / 2, sz.end());
    b->nc_median = sz[C / 2];
  }
  if (e == cudaSuccess) e = set_shape(c, b, C > 1 ? 32 : 128, kItemWaves);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // host vectors go out of scope
  if (e != cudaSuccess) {
    batch_free(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

// every block step moves the earliest particle forward by at least dt_min,
// so no run can need more than t_end / dt_min + 2 loop iterations
int64_t iteration_cap(const nb_ctx* c, double t_end) {
  int64_t cap = (int64_t)ceil(t_end / c->dt_min) + 2;
  return cap > kMaxIters ? kMaxIters : cap;
}

cudaError_t set_params(nb_ctx* c, Batch* b, double t_end, int64_t seg_iters = 0) {
  BParams p{t_end, c->eta, c->dt_min, c->dt_max, iteration_cap(c, t_end), seg_iters};
  // pinned staging keeps the copy asynchronous-safe
  memcpy(c->hpin, &p, sizeof(p));
  cudaError_t e = cudaMemcpyAsync(b->prm, c->hpin, sizeof(p), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

// plan for the current active lists (b->nact, act), without loop control
cudaError_t plan_only(nb_ctx* c, Batch* b) {
  const bool mixed = c->precision == NB_MIXED;
  const int per_cta = b->nt * (mixed ? kMixIPT : 1);
  const int jt = mixed ? kMixJT : kF64JT;
  const int grid = mixed ? b->grid_mixed : b->grid_fp64;
  b_plan<<<1, 1024, 0, c->stream>>>(b->C, b->off, b->nact, per_cta, jt, b->waves * (int64_t)grid, c->part_elems,
                                    b->itiles, b->nsplit, b->jps, b->item_off, b->part_off, b->pstride,
                                    b->ritem_off, b->citem_off, b->wq, b->ctrl,
                                    b->prm, c->status, 0, 0);
  return cudaGetLastError();
}

// a single system's j-ranges start at row 0 in multiples of the j-tile, so
// the 128-row tile boxes of the spatial order line up with its tiles
bool single_boxes(const nb_ctx* c, const Batch* b) {
  return c->precision == NB_MIXED && c->n_clusters == 0 && b->C == 1;
}

// an ensemble of mixed clusters kept in spatial order within each cluster
bool cluster_boxes(const nb_ctx* c, const Batch* b) {
  return c->precision == NB_MIXED && c->n_clusters > 0 && b->tile_off != nullptr;
}

template <int NT>
void launch_force(nb_ctx* c, Batch* b, bool mixed) {
  if (mixed)
    b_force_mixed<NT, kMixIPT, kMixJT><<<b->grid_mixed, NT, 0, c->stream>>>(
        b->C, b->off, b->eps2f, c->n_pad, c->jA, c->jB, c->jC, c->act, b->nact, b->itiles, b->nsplit, b->jps,
        b->item_off, b->part_off, b->pstride, c->F, c->n_pad, c->part,
        !c->far_tiles ? nullptr : single_boxes(c, b) ? c->tbox : (cluster_boxes(c, b) ? b->tbox : nullptr),
        cluster_boxes(c, b) ? b->tile_off : nullptr, b->wq);
  else
    b_force_fp64<NT, kF64JT><<<b->grid_fp64, NT, 0, c->stream>>>(
        b->C, b->off, b->eps2d, c->n_pad, c->xp, c->vp, c->m, c->act, b->nact, b->itiles, b->nsplit, b->jps,
        b->item_off, b->part_off, b->pstride, c->F, c->n_pad, c->part, b->wq);
}

cudaError_t body_after_plan(nb_ctx* c, Batch* b, bool own_time) {
  const bool mixed = c->precision == NB_MIXED;
  const int g = grid_for(b->N, 256, c->sm_count * 16);
  b_predict<<<g, 256, 0, c->stream>>>(b->N, c->n_pad, b->cid, b->nact, b->tnext, own_time ? 1 : 0, c->m, c->x,
                                      c->v, c->a, c->jk, c->t, c->xp, c->vp, c->jA, c->jB, c->jC, 1, mixed ? 1 : 0);
  if (single_boxes(c, b)) {
    cudaError_t e = nb_launch_tile_boxes(c);  // boxes of the predicted tiles for the far test
    if (e != cudaSuccess) return e;
  } else if (cluster_boxes(c, b)) {
    b_tile_boxes<<<(unsigned)((b->ntiles + 7) / 8), 256, 0, c->stream>>>(b->ntiles, b->tile_cl, b->tile_off, b->off,
                                                                        c->jA, b->tbox);
    c->launches += 1;
  }
  if (b->nt == 32)
    launch_force<32>(c, b, mixed);
  else if (b->nt == 64)
    launch_force<64>(c, b, mixed);
  else
    launch_force<128>(c, b, mixed);
  b_reduce<<<c->sm_count * 8, dim3(32, kRedLanes), 0, c->stream>>>(
      b->C, b->off, b->nact, b->nsplit, b->part_off, b->pstride, b->ritem_off, c->part, c->F, c->n_pad);
  c->launches += 3;
  return cudaGetLastError();
}

// one block step of every active cluster, all on the device
cudaError_t capture_step(nb_ctx* c, Batch* b, cudaGraphConditionalHandle handle, int use_handle) {
  const bool mixed = c->precision == NB_MIXED;
  const int per_cta = b->nt * (mixed ? kMixIPT : 1);
  const int jt = mixed ? kMixJT : kF64JT;
  const int grid = mixed ? b->grid_mixed : b->grid_fp64;
  b_sel_min<<<b->nchunks, 256, 0, c->stream>>>(b->ch_lo, b->ch_hi, c->t, c->dt, b->ch_min);
  b_sel_count<<<b->nchunks, 256, 0, c->stream>>>(b->ch_cluster, b->ch_lo, b->ch_hi, b->cl_ch0, b->ch_min, c->t,
                                                 c->dt, b->tnext, b->ch_cnt, b->ctrl, b->prm, c->status);
  b_sel_write<<<b->nchunks, 256, 0, c->stream>>>(b->ch_cluster, b->ch_lo, b->ch_hi, b->cl_ch0, b->ch_cnt, b->off,
                                                 c->t, c->dt, b->tnext, b->prm, c->act, b->nact);
  b_plan<<<1, 1024, 0, c->stream>>>(b->C, b->off, b->nact, per_cta, jt, b->waves * (int64_t)grid, c->part_elems,
                                    b->itiles, b->nsplit, b->jps, b->item_off, b->part_off, b->pstride,
                                    b->ritem_off, b->citem_off, b->wq, b->ctrl,
                                    b->prm, c->status, handle, use_handle);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = body_after_plan(c, b, false)) != cudaSuccess) return e;
  b_correct<<<c->sm_count * 16, kCorrItem, 0, c->stream>>>(b->C, c->n_pad, b->citem_off, b->off, b->nact, b->tnext,
                                                           c->act, c->F, c->n_pad, b->prm, c->x, c->v, c->a, c->jk,
                                                           c->pot, c->t, c->dt, c->xp, c->vp, c->status);
  c->launches += 5;
  return cudaGetLastError();
}

// pick: take the item shape from the autotuner's table (else keep b's shape)
cudaError_t build_graph(nb_ctx* c, Batch* b, bool pick = true) {
  cudaError_t e0 = pick ? pick_shape(c, b) : cudaSuccess;
  if (e0 != cudaSuccess) return e0;
  const int64_t key = ((int64_t)c->precision << 32) | ((int64_t)c->far_tiles << 31) | ((int64_t)b->nt << 8) | b->waves;
  if (b->exec && b->exec_key == key) return cudaSuccess;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  // zero-initialised parameter block (the struct has no usable default constructor)
  alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
  memset(np_buf, 0, sizeof(np_buf));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  // capture on a private stream (the context's stream may be the legacy
  // default stream, which cannot be captured); the graph runs on c->stream
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int64_t launches = c->launches;
      cudaStream_t own = c->stream;
      c->stream = cap;
      cudaError_t ec = capture_step(c, b, h, 1);
      c->stream = own;
      c->launches = launches;
      cudaGraph_t got = nullptr;
      e = cudaStreamEndCapture(cap, &got);
      if (ec != cudaSuccess) e = ec;
    }
  }
  if (cap) cudaStreamDestroy(cap);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) b->exec_key = key;
  return e;
}

int finish_status(nb_ctx* c) {
  nb_dev_status st;
  if (cudaMemcpyAsync(c->hpin, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NB_ECUDA;
  memcpy(&st, c->hpin, sizeof(st));
  if (st.flags & NB_ST_TIMEOUT) return NB_ETIMEOUT;
  if (st.flags & NB_ST_STALLED) return NB_ESTATE;  // (before NaNs: the stalled state's corrections make some)
  if (st.flags & NB_ST_NUMERIC) return NB_ENUMERIC;
  return NB_OK;
}

int64_t read_ctrl(nb_ctx* c, Batch* b, int idx) {
  int64_t v = 0;
  if (cudaMemcpyAsync(c->hpin, b->ctrl + idx, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream) == cudaSuccess &&
      cudaStreamSynchronize(c->stream) == cudaSuccess)
    memcpy(&v, c->hpin, sizeof(v));
  return v;
}

// graph-driven integration of every cluster of b to t_end.  A single mixed
// system keeps its resident spatial order: the graph runs in segments of at
// most sort_interval block steps, and the order is renewed between them.
int run_graph(nb_ctx* c, Batch* b, double t_end) {
  if (build_graph(c, b) != cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  const bool seg = single_boxes(c, b);
  const int64_t cap = iteration_cap(c, t_end);
  int64_t total = 0;
  for (;;) {
    int64_t seg_iters = 0;
    if (seg) {
      const int rs = nb_ensure_sorted(c);
      if (rs != NB_OK) return rs;
      seg_iters = std::max(1, c->sort_interval - c->perm_age);
    }
    if (set_params(c, b, t_end, seg_iters) != cudaSuccess) return NB_ECUDA;
    if (cudaMemsetAsync(b->ctrl, 0, 4 * sizeof(int64_t), c->stream) != cudaSuccess) return NB_ECUDA;
    if (cudaGraphLaunch(b->exec, c->stream) != cudaSuccess) return NB_ECUDA;
    const int64_t iters = read_ctrl(c, b, 1);
    const int64_t inter = read_ctrl(c, b, 2);
    const bool more = read_ctrl(c, b, 3) != 0;
    // a finished run ends with one iteration that selects nothing
    const int64_t steps = more ? iters : (iters > 0 ? iters - 1 : 0);
    c->steps += steps;
    c->perm_age += (int)steps;
    c->interactions += (double)inter;
    c->launches += iters * (seg ? 9 : 8);
    total += iters;
    if (!more) break;
    if (total > cap) return NB_ETIMEOUT;  // cannot happen for valid block steps
  }
  c->pred_valid = false;
  c->f_valid = false;
  return finish_status(c);
}

// all particles of every cluster at their own time (Sec. 4.1 step 1): F = forces
cudaError_t all_forces(nb_ctx* c, Batch* b) {
  cudaError_t e0 = cudaMemsetAsync(b->ctrl, 0, 4 * sizeof(int64_t), c->stream);
  if (e0 != cudaSuccess) return e0;
  b_all_active<<<grid_for(b->N, 256, 4096), 256, 0, c->stream>>>(b->C, b->off, b->N, c->act, b->nact, b->tnext);
  cudaError_t e = plan_only(c, b);
  if (e != cudaSuccess) return e;
  c->launches += 2;
  return body_after_plan(c, b, true);
}

// copy rows [src + o, src + o + n) of every SoA array between contexts
cudaError_t copy_state(nb_ctx* dst, int64_t dofs, const nb_ctx* src, int64_t sofs, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  struct R {
    double* d;
    const double* s;
    int rows;
  } rs[] = {{dst->m, src->m, 1},   {dst->x, src->x, 3},     {dst->v, src->v, 3}, {dst->a, src->a, 3},
            {dst->jk, src->jk, 3}, {dst->pot, src->pot, 1}, {dst->t, src->t, 1}, {dst->dt, src->dt, 1}};
  for (const R& r : rs)
    for (int k = 0; k < r.rows; ++k) {
      cudaError_t e = cudaMemcpyAsync(r.d + k * dst->n_pad + dofs, r.s + k * src->n_pad + sofs, n * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace

void nb_ensemble_free(nb_ctx* c) {
  if (!c) return;
  batch_free(batch_of(c));
  c->ens = nullptr;
}

int nb_integrate_graph(nb_ctx* c, double t_end) {
  Batch* b = batch_of(c);
  if (c->n_clusters == 0 && (!b || b->N != c->n)) {
    batch_free(b);
    c->ens = nullptr;
    const int64_t off[2] = {0, c->n};
    const double eps = c->eps;
    if (batch_build(c, 1, off, &eps, &b) != cudaSuccess) return NB_ECUDA;
    c->ens = b;
  }
  if (c->n_clusters == 0) {  // the softening may have changed since the batch was built
    const double e2 = c->eps * c->eps;
    const float e2f = (float)e2;
    if (cudaMemcpyAsync(b->eps2d, &e2, sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->eps2f, &e2f, sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return NB_ECUDA;
  }
  return run_graph(c, b, t_end);
}

int nb_ensemble_ensure_sorted(nb_ctx* c) {
  Batch* b = batch_of(c);
  if (!b || !cluster_boxes(c, b) || b->N <= 0) return NB_OK;
  // once per set of particles: a cluster moves little against its own size in
  // the time units an ensemble run covers, and a renewal would cost the graph
  // loop a host round trip per segment
  if (c->perm_valid) return NB_OK;
  b_cluster_bbox<<<b->C, 256, 0, c->stream>>>(b->off, c->n_pad, c->x, b->cbox);
  b_cluster_keys<<<grid_for(b->N, 256, c->sm_count * 16), 256, 0, c->stream>>>(b->N, c->n_pad, b->cid, c->x, b->cbox,
                                                                              c->skey[0], c->sval[0]);
  c->launches += 2;
  if (cudaGetLastError() != cudaSuccess || nb_order_rows_by_keys(c, 21 + b->cl_bits) != cudaSuccess) return NB_ECUDA;
  c->perm_valid = true;
  c->perm_age = 0;
  c->pred_valid = false;
  c->f_valid = false;
  return NB_OK;
}

extern "C" {

int nb_ensemble_create(nb_ctx** out, int32_t n_clusters, const int64_t* offsets, const double* eps, int precision,
                       int device, void* cuda_stream) {
  if (!out) return NB_EINVAL;
  *out = nullptr;
  if (n_clusters < 1 || !offsets || !eps || offsets[0] != 0) return NB_EINVAL;
  for (int32_t q = 0; q < n_clusters; ++q)
    if (offsets[q + 1] <= offsets[q] || !(eps[q] > 0.0) || !isfinite(eps[q])) return NB_EINVAL;
  nb_ctx* c = nullptr;
  int r = nb_create(&c, offsets[n_clusters], precision, device, cuda_stream);
  if (r != NB_OK) return r;
  Batch* b = nullptr;
  if (batch_build(c, n_clusters, offsets, eps, &b) != cudaSuccess) {
    nb_destroy(c);
    return NB_ENOMEM;
  }
  c->ens = b;
  c->n_clusters = n_clusters;
  c->h_offsets = (int64_t*)malloc((n_clusters + 1) * sizeof(int64_t));
  c->h_ceps = (double*)malloc(n_clusters * sizeof(double));
  if (!c->h_offsets || !c->h_ceps) {
    nb_destroy(c);
    return NB_ENOMEM;
  }
  memcpy(c->h_offsets, offsets, (n_clusters + 1) * sizeof(int64_t));
  memcpy(c->h_ceps, eps, n_clusters * sizeof(double));
  *out = c;
  return NB_OK;
}

int nb_ensemble_initial_forces_and_dt(nb_ctx* c) {
  if (!c || !c->ens) return NB_EINVAL;
  Batch* b = batch_of(c);
  if (c->n < b->N) return NB_ESTATE;
  const int rs = nb_ensemble_ensure_sorted(c);
  if (rs != NB_OK) return rs;
  if (set_params(c, b, 0.0) != cudaSuccess) return NB_ECUDA;
  if (all_forces(c, b) != cudaSuccess) return NB_ECUDA;
  b_initial_dt<<<grid_for(b->N, 256, c->sm_count * 16), 256, 0, c->stream>>>(b->N, c->n_pad, c->F, c->n_pad, b->prm,
                                                                             c->a, c->jk, c->pot, c->t, c->dt,
                                                                             c->status);
  c->launches += 1;
  if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
  c->interactions += (double)read_ctrl(c, b, 2);
  return finish_status(c);
}

int nb_ensemble_energy(nb_ctx* c, double* ekin, double* epot) {
  if (!c || !c->ens || !ekin || !epot) return NB_EINVAL;
  Batch* b = batch_of(c);
  if (c->n < b->N) return NB_ESTATE;
  if (set_params(c, b, 0.0) != cudaSuccess) return NB_ECUDA;
  if (all_forces(c, b) != cudaSuccess) return NB_ECUDA;
  b_energy<<<b->C, 256, 0, c->stream>>>(b->off, c->n_pad, c->m, c->v, c->F, c->n_pad, b->esum);
  c->launches += 1;
  std::vector<double> h(2 * (size_t)b->C);
  if (cudaMemcpyAsync(h.data(), b->esum, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NB_ECUDA;
  for (int32_t q = 0; q < b->C; ++q) {
    ekin[q] = h[2 * q];
    epot[q] = h[2 * q + 1];
  }
  c->pred_valid = false;
  c->f_valid = false;
  return finish_status(c);
}

// nb_ensemble_autotune: the item shape (i-tile 32/64/128, items per resident
// CTA 2/4/8/16) timed on `steps` block steps of the context's own state, the
// state restored after every trial; the fastest goes into the table under the
// batch's (median cluster size, cluster count) bin
int nb_ensemble_autotune(nb_ctx* c, int64_t steps, int* i_tile, int* item_waves, double* ms_best,
                         double* ms_default) {
  if (!c) return NB_EINVAL;
  if (steps < 1 || steps > 4096) return NB_EINVAL;
  if (c->n <= 0) return NB_ESTATE;
  Batch* b = batch_of(c);
  if (c->n_clusters == 0 && (!b || b->N != c->n)) {  // a single system's graph loop
    batch_free(b);
    c->ens = nullptr;
    const int64_t off[2] = {0, c->n};
    const double eps = c->eps;
    if (batch_build(c, 1, off, &eps, &b) != cudaSuccess) return NB_ECUDA;
    c->ens = b;
  }
  if (c->n_clusters == 0) {
    const int rs = nb_ensure_sorted(c);
    if (rs != NB_OK) return rs;
    const double e2 = c->eps * c->eps;
    const float e2f = (float)e2;
    if (cudaMemcpyAsync(b->eps2d, &e2, sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->eps2f, &e2f, sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return NB_ECUDA;
  }
  if (c->n < b->N) return NB_ESTATE;
  const int64_t N = b->N, np = c->n_pad;
  // the state the trials start from (16 FP64 rows), and a run end past every step
  double* saved = nullptr;
  if (cudaMalloc((void**)&saved, (size_t)16 * np * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return NB_ENOMEM;
  }
  struct Row {
    double* p;
    int k;
  } rows[] = {{c->m, 1}, {c->x, 3}, {c->v, 3}, {c->a, 3}, {c->jk, 3}, {c->pot, 1}, {c->t, 1}, {c->dt, 1}};
  auto copy_rows = [&](bool save) -> cudaError_t {
    int64_t r = 0;
    for (const Row& q : rows)
      for (int k = 0; k < q.k; ++k, ++r) {
        double* live = q.p + k * np;
        double* keep = saved + r * np;
        cudaError_t e = cudaMemcpyAsync(save ? keep : live, save ? live : keep, N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
      }
    return cudaSuccess;
  };
  std::vector<double> ht(N);
  int r = NB_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int nt0 = b->nt, w0 = b->waves;
  const int64_t steps0 = c->steps;
  const double inter0 = c->interactions;
  int best_nt = 0, best_w = 0;
  float best = 3.4e38f, dflt = -1.0f;
  if (copy_rows(true) != cudaSuccess ||
      cudaMemcpyAsync(ht.data(), c->t, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    r = NB_ECUDA;
  } else {
    double tmax = 0.0;
    for (double v : ht) tmax = std::max(tmax, v);
    const double t_end = (floor(tmax / c->dt_max) + 1.0) * c->dt_max;
    static const int nts[] = {32, 64, 128};
    static const int ws[] = {2, 4, 8, 16};
    for (int a = 0; a < 3 && r == NB_OK; ++a)
      for (int q = 0; q < 4 && r == NB_OK; ++q) {
        if (set_shape(c, b, nts[a], ws[q]) != cudaSuccess) { r = NB_ECUDA; break; }
        // the shape is forced for the trial: the graph is built for it directly
        if (build_graph(c, b, false) != cudaSuccess) { r = NB_ECUDA; break; }
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && r == NB_OK; ++rep) {  // the first launch uploads the graph
          if (copy_rows(false) != cudaSuccess || set_params(c, b, t_end, steps) != cudaSuccess ||
              cudaMemsetAsync(b->ctrl, 0, 4 * sizeof(int64_t), c->stream) != cudaSuccess ||
              cudaEventRecord(e0, c->stream) != cudaSuccess || cudaGraphLaunch(b->exec, c->stream) != cudaSuccess ||
              cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            r = NB_ECUDA;
        }
        if (r != NB_OK) break;
        if (finish_status(c) != NB_OK) { r = NB_ENUMERIC; break; }
        if (nts[a] == (b->C > 1 ? 32 : 128) && ws[q] == kItemWaves) dflt = ms;
        if (ms < best) {
          best = ms;
          best_nt = nts[a];
          best_w = ws[q];
        }
      }
  }
  // the caller's state, counters and shape back; the winner into the table
  if (copy_rows(false) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) r = NB_ECUDA;
  cudaFree(saved);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  c->steps = steps0;
  c->interactions = inter0;
  c->pred_valid = c->f_valid = false;
  c->state_ver++;
  if (set_shape(c, b, nt0, w0) != cudaSuccess && r == NB_OK) r = NB_ECUDA;
  if (r != NB_OK) return r;
  nb_tuning cfg{1, best_nt, c->precision == NB_MIXED ? kMixJT : kF64JT, 0, best_w};
  nb_tune_store(c, NB_TUNE_BATCHED, b->nc_median, b->C, cfg, best);
  if (i_tile) *i_tile = best_nt;
  if (item_waves) *item_waves = best_w;
  if (ms_best) *ms_best = best;
  if (ms_default) *ms_default = dflt;
  return NB_OK;
}

int nb_ensemble_integrate(nb_ctx* c, double t_end, int mode) {
  if (!c || !c->ens || c->n_clusters == 0) return NB_EINVAL;
  Batch* b = batch_of(c);
  if (!(t_end > 0.0) || !isfinite(t_end) || fmod(t_end, c->dt_max) != 0.0) return NB_EINVAL;
  if (c->n < b->N) return NB_ESTATE;
  if (mode == NB_ENSEMBLE_PERSISTENT) return run_graph(c, b, t_end);
  if (mode != NB_ENSEMBLE_PER_CLUSTER) return NB_EINVAL;
  // reference: each cluster integrated on its own with host-driven per-step launches
  if (!b->child) {
    int64_t nmax = 0;
    for (int32_t q = 0; q < b->C; ++q) nmax = std::max(nmax, b->h_off[q + 1] - b->h_off[q]);
    int r = nb_create(&b->child, nmax, c->precision, c->device, (void*)c->stream);
    if (r != NB_OK) return r;
  }
  nb_ctx* ch = b->child;
  nb_set_precision(ch, c->precision);
  for (int32_t q = 0; q < b->C; ++q) {
    const int64_t o = b->h_off[q], n = b->h_off[q + 1] - o;
    if (copy_state(ch, 0, c, o, n, c->stream) != cudaSuccess) return NB_ECUDA;
    ch->n = n;
    ch->pred_valid = ch->f_valid = false;
    ch->perm_valid = false;
    ch->state_ver++;  // written behind the API: the child's j-memory is stale
    int r = nb_set_params(ch, c->h_ceps[q], c->eta, c->dt_min, c->dt_max);
    if (r == NB_OK) r = nb_integrate(ch, t_end, 0);
    if (r != NB_OK) return r;
    if (nb_unsort(ch) != cudaSuccess) return NB_ECUDA;  // back to particle order
    if (copy_state(c, o, ch, 0, n, c->stream) != cudaSuccess) return NB_ECUDA;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NB_ECUDA;
  c->interactions += ch->interactions;
  c->launches += ch->launches;
  c->steps += ch->steps;
  ch->interactions = 0;
  ch->launches = 0;
  ch->steps = 0;
  return finish_status(c);
}

}  // extern "C"
