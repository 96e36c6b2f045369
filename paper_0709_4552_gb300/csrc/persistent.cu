// persistent.cu -- the block-step loop of one system (Sec. 4.1 steps 2-5) as
// one cooperative launch: every CTA stays resident for the whole run and the
// steps are separated by grid barriers instead of kernel boundaries.  Below
// N ~ 10^4 a block step does a few microseconds of arithmetic, and a
// launch per kernel (host loop) or a graph node per kernel (graph loop) costs
// more than the work; here a step costs three barriers.
//
// Rows are cut into 128-row tiles; CTA b of G owns the contiguous tiles
// [b T / G, (b + 1) T / G).  Per block step:
//   phase 1 (after barrier A): every CTA reads the G published slice minima
//     of t_i + dt_i with their counts and takes the block time t (step 2) and
//     its own offset in the active list; it writes its own active rows there
//     (ascending), predicts its own rows to t (step 3) and, on the mixed path
//     in spatial order, computes the boxes of its own tiles.    -> barrier B
//   phase 2: force items (i-tile of 128 list positions x j-split) taken from
//     a work counter, or by block index when every CTA has an SM of its own
//     and the items fit (step 4, Eq. 3), the same items as the host-driven
//     kernels, split partials as double-single pairs.            -> barrier C
//   phase 3: every CTA sums the j-splits of its own list positions in a fixed
//     order (double-single FP32), corrects them and picks their new steps
//     (step 5; own rows' due times kept in shared memory), then publishes the
//     minimum of t_i + dt_i over its rows and how many rows reach it; a block
//     time that does not increase stops the loop (no valid steps).
//                                                                 -> barrier A
// The active block is exactly the rows at the global minimum, so a CTA whose
// own minimum is larger has none, and the counts published with the minima
// give every CTA its list offset without a further barrier.
//
// Barriers count arrivals over the whole launch; each wait is bounded in
// time and polls, after which the CTA raises the timeout bit and an abort
// flag that makes every other CTA leave at its next wait.
#include <float.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "force_common.cuh"
#include "hermite.cuh"

namespace {

constexpr int kLT = 128;                     // threads per CTA = i-tile = row tile
constexpr int kLWarps = kLT / 32;
constexpr int kLMaxPerSm = 4;                // resident CTAs per SM asked for (128 registers)
constexpr int kLMixJT = 128, kLF64JT = 64;   // j-tiles (the mixed one = the box tile)
constexpr long long kWaitNs = 4000000000LL;  // a barrier wait of the loop gives up after 4 s
constexpr unsigned int kPollCap = 1u << 26;  // ... or after this many polls
constexpr unsigned long long kInfBits = 0x7FF0000000000000ULL;  // +inf
constexpr int kLItemWaves = 2;               // force items per step: about 2 per CTA ...
constexpr int64_t kLMaxSplits = 256;         // ... with at most this many j-splits
constexpr int kMaxSmid = 1024;               // SM ids counted by the CTA placement

struct LoopCtl {
  unsigned long long bar;   // barrier arrivals in this launch
  unsigned long long wq;    // force-item counter of the current step
  unsigned int nsm;         // SMs holding CTAs of this launch
  unsigned int smrank[kMaxSmid];  // CTAs placed on each SM so far
  unsigned int abort;       // a CTA gave up waiting: every CTA leaves
  unsigned int more;        // the launch stopped after seg_steps steps
  long long steps;          // block steps taken
  long long interactions;   // sum of n N over the steps
};

struct LoopArgs {
  int64_t N, n_pad;
  double eps2;
  float eps2f;
  double eta, dt_min, dt_max, t_end;
  long long max_steps, seg_steps;
  const double* m;
  double *x, *v, *a, *jk, *pot, *t, *dt;
  double *xp, *vp;
  float4 *jA, *jB;
  float2* jC;
  float4* tbox;  // boxes of the 128-row tiles (mixed path in spatial order) or null
  int32_t* act;
  double *F, *part;
  int64_t part_elems;
  unsigned long long* smin;  // [G] slice minimum of t_i + dt_i (bit pattern)
  int32_t* scnt;             // [G] rows of the slice at that minimum
  LoopCtl* ctl;
  nb_dev_status* st;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of G co-resident CTAs.  The k-th barrier of a launch is
// complete when the arrival count reaches k G.  Ordering: the CTA barrier
// orders every thread's writes before thread 0's gpu-scope release add
// (cumulative), and thread 0's acquire load before every thread's later
// reads.  Returns false when this CTA must leave (another CTA gave up, or
// this one waited longer than wait_ns).
__device__ bool grid_barrier(LoopCtl* ctl, unsigned long long& epoch, unsigned int G, nb_dev_status* st,
                             int* s_ok, long long wait_ns = kWaitNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned long long target = epoch * (unsigned long long)G;
    red_release_add_u64(&ctl->bar, 1ULL);
    int ok = 1;
    const long long t0 = globaltimer_ns();
    unsigned int polls = 0;
    // the counter alone in the common path; the abort flag and the clock
    // every 16th poll (one L2 round trip per poll instead of two)
    while (ld_acquire_u64(&ctl->bar) < target) {
      if ((++polls & 15u) != 0u) continue;
      if (*(volatile unsigned int*)&ctl->abort) {
        ok = 0;
        break;
      }
      if (polls >= kPollCap || globaltimer_ns() - t0 > wait_ns) {
        atomicOr(&ctl->abort, 1u);
        atomicOr(&st->flags, NB_ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// (minimum, count at the minimum) combine
__device__ __forceinline__ void min_count(unsigned long long& v, int& c, unsigned long long ov, int oc) {
  if (ov < v) {
    v = ov;
    c = oc;
  } else if (ov == v) {
    c += oc;
  }
}

constexpr int kLDue = 512;  // own rows whose due times a CTA keeps in shared memory

struct LoopSmem {
  // own rows' next due time t_i + dt_i (bit pattern), kept by the corrector
  // when the CTA owns at most kLDue rows (else read from the state)
  unsigned long long due[kLDue];
  int rank;                // this CTA's rank among the CTAs on its SM
  long long item;
  unsigned long long wv[kLWarps];
  int wc[kLWarps];
  long long ws[2][kLWarps];
  float wbox[kLWarps][7];
  unsigned long long tnb;  // block time (bit pattern)
  long long before, total;
  int mine;                // this CTA has active rows this step
  int mycnt;
  int ok;
};

// due time of own row i (bit pattern)
__device__ __forceinline__ unsigned long long due_of(const LoopArgs& p, const LoopSmem& s, int64_t i, int64_t r0,
                                                     bool cached) {
  return cached ? s.due[i - r0] : (unsigned long long)__double_as_longlong(p.t[i] + p.dt[i]);
}

// minimum of t_i + dt_i over rows [r0, r1) and the number of rows at it,
// published for the other CTAs (positive doubles order like their bits)
__device__ void publish_slice(const LoopArgs& p, int64_t r0, int64_t r1, LoopSmem& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool cached = r1 - r0 <= kLDue;
  unsigned long long best = kInfBits;
  int cnt = 0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kLT) min_count(best, cnt, due_of(p, s, i, r0, cached), 1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oc = __shfl_xor_sync(0xffffffffu, cnt, o);
    min_count(best, cnt, ov, oc);
  }
  if (lane == 0) {
    s.wv[warp] = best;
    s.wc[warp] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kLWarps; ++w) min_count(best, cnt, s.wv[w], s.wc[w]);
    p.smin[blockIdx.x] = best;
    p.scnt[blockIdx.x] = cnt;
  }
}

// block time, total active count and this CTA's offset from the published
// slices (every CTA reads the same values, so every CTA decides alike)
constexpr int kLMaxG = 1024;  // CTAs a launch may have (slices read per thread below)
__device__ void read_slices(const LoopArgs& p, unsigned int G, LoopSmem& s) {
  constexpr int kPer = kLMaxG / kLT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long* smin = reinterpret_cast<const long long*>(p.smin);
  unsigned long long v[kPer];
  int c[kPer];
  unsigned long long best = kInfBits;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {  // one round of loads: minima and counts together
    const unsigned int q = threadIdx.x + u * kLT;
    v[u] = q < G ? (unsigned long long)__ldcg(smin + q) : kInfBits;
    c[u] = q < G ? __ldcg(p.scnt + q) : 0;
    best = v[u] < best ? v[u] : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
    best = ov < best ? ov : best;
  }
  if (lane == 0) s.wv[warp] = best;
  __syncthreads();
  best = s.wv[0];
#pragma unroll
  for (int w = 1; w < kLWarps; ++w) best = s.wv[w] < best ? s.wv[w] : best;
  long long tot = 0, before = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const unsigned int q = threadIdx.x + u * kLT;
    if (v[u] == best) {
      tot += c[u];
      if (q < blockIdx.x) before += c[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    before += __shfl_xor_sync(0xffffffffu, before, o);
  }
  if (lane == 0) {
    s.ws[0][warp] = tot;
    s.ws[1][warp] = before;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kLWarps; ++w) {
      tot += s.ws[0][w];
      before += s.ws[1][w];
    }
    s.tnb = best;
    s.total = tot;
    s.before = before;
    const unsigned long long mv = (unsigned long long)__ldcg(smin + blockIdx.x);
    s.mine = mv == best;
    s.mycnt = s.mine ? __ldcg(p.scnt + blockIdx.x) : 0;
  }
  __syncthreads();
}

// this CTA's active rows, ascending, to act[before ...]
__device__ void write_active(const LoopArgs& p, int64_t r0, int64_t r1, unsigned long long tnb, long long base,
                             LoopSmem& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool cached = r1 - r0 <= kLDue;
  for (int64_t r = r0; r < r1; r += kLT) {
    const int64_t i = r + threadIdx.x;
    const bool on = i < r1 && due_of(p, s, i, r0, cached) == tnb;
    const unsigned int ball = __ballot_sync(0xffffffffu, on);
    if (lane == 0) s.wc[warp] = __popc(ball);
    __syncthreads();
    int pre = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kLWarps; ++w) {
      pre += w < warp ? s.wc[w] : 0;
      all += s.wc[w];
    }
    if (on) p.act[base + pre + __popc(ball & ((1u << lane) - 1u))] = (int32_t)i;
    base += all;
    __syncthreads();
  }
}

// predictor of this CTA's rows to tn; on the mixed path in spatial order the
// box of each 128-row tile (thread q holds row q of every tile it visits):
// (min corner, max |coordinate|), (max corner, 0) of the FP32 high words
template <bool MIXED>
__device__ void predict_rows(const LoopArgs& p, int64_t r0, int64_t r1, double tn, LoopSmem& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t r = r0; r < r1; r += kLT) {
    const int64_t i = r + threadIdx.x;
    float bx[7] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX, 0.0f};
    if (i < r1) {
      double px[3], pv[3];
      nbh::taylor(i, p.n_pad, tn - p.t[i], p.x, p.v, p.a, p.jk, px, pv);
      nbh::store_predicted(i, p.n_pad, px, pv, p.m[i], p.xp, p.vp, p.jA, p.jB, p.jC, true, MIXED);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float h = __double2float_rn(px[d]);
        bx[d] = h;
        bx[3 + d] = h;
        bx[6] = fmaxf(bx[6], fabsf(h));
      }
    }
    if (MIXED && p.tbox) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          bx[d] = fminf(bx[d], __shfl_xor_sync(0xffffffffu, bx[d], o));
          bx[3 + d] = fmaxf(bx[3 + d], __shfl_xor_sync(0xffffffffu, bx[3 + d], o));
        }
        bx[6] = fmaxf(bx[6], __shfl_xor_sync(0xffffffffu, bx[6], o));
      }
      if (lane == 0)
#pragma unroll
        for (int d = 0; d < 7; ++d) s.wbox[warp][d] = bx[d];
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < kLWarps; ++w) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            bx[d] = fminf(bx[d], s.wbox[w][d]);
            bx[3 + d] = fmaxf(bx[3 + d], s.wbox[w][3 + d]);
          }
          bx[6] = fmaxf(bx[6], s.wbox[w][6]);
        }
        const int64_t tile = r / kLT;
        p.tbox[2 * tile] = make_float4(bx[0], bx[1], bx[2], bx[6]);
        p.tbox[2 * tile + 1] = make_float4(bx[3], bx[4], bx[5], 0.0f);
      }
      __syncthreads();
    }
  }
}

// split-j factor of a step: about kLItemWaves force items per CTA (taken
// from a counter, so uneven items even out), at least one j-tile per split,
// at most kLMaxSplits splits (their sums are the corrector phase's loads),
// within the partial-sum scratch
__device__ __forceinline__ int64_t loop_splits(int64_t n, int64_t jtiles, unsigned int G, int64_t part_elems) {
  const int64_t nI = (n + kLT - 1) / kLT;
  int64_t S = ((int64_t)kLItemWaves * G + nI - 1) / nI;
  if (S > jtiles) S = jtiles;
  if (S > kLMaxSplits) S = kLMaxSplits;
  const int64_t cap = part_elems / (7 * (((n + 31) / 32) * 32));
  if (S > cap) S = cap;
  return S < 1 ? 1 : S;
}

// phase 3 of a step: the j-split sums and the corrector (Sec. 4.1 step 5)
// of this CTA's own list positions [before, before + mycnt).  The step's
// values are read from shared memory here rather than kept in registers
// across the force items.
template <bool MIXED>
__device__ void correct_own(const LoopArgs& p, LoopSmem& s, int64_t jtiles, unsigned int G, int64_t r0,
                            int64_t r1) {
  const long long before = s.before;
  const int mycnt = s.mycnt;
  const double tn = __longlong_as_double((long long)s.tnb);
  const int64_t n = s.total;
  const int64_t S = loop_splits(n, jtiles, G, p.part_elems);
  const int64_t pstride = ((n + 31) / 32) * 32;
  const bool fin = S == 1;
  // own list positions, up to 128 per round: L = 128 / P' threads per
  // position (P' = the round's positions rounded up to a power of two, at
  // least 4) sum its j-splits (lane l takes splits l, l + L, ... in order;
  // a butterfly over the L lanes), and the group corrects it (step 5): lanes
  // 0-3 together when it has at least four (the correction's FP64 chain is
  // the critical path of a small block's step), else lane 0 alone: one
  // position per thread when the block is large, 32 lanes per position when
  // it is small and the splits many
  for (int k0 = 0; k0 < mycnt; k0 += kLT) {
    const int P = min(mycnt - k0, kLT);
    int Pp = 4;
    while (Pp < P) Pp <<= 1;
    const int L = kLT / Pp;
    const int q = threadIdx.x / L, l = threadIdx.x % L;
    const bool have = q < P;
    const int64_t k = before + k0 + (have ? q : 0);
    double f[7];
    if (fin) {
      if (have && l < 4)
#pragma unroll
        for (int r = 0; r < 7; ++r) f[r] = p.F[r * p.n_pad + k];
    } else if (MIXED) {
      // double-single partials (the mixed item's split output): summed and
      // exchanged in FP32 (a warp's FP64 instruction costs it 64 cycles
      // here), converted to FP64 once
      float hi[7], lo[7];
#pragma unroll
      for (int r = 0; r < 7; ++r) hi[r] = lo[r] = 0.0f;
      const float2* part2 = reinterpret_cast<const float2*>(p.part);
      if (have)
        for (int64_t sp = l; sp < S; sp += L)
#pragma unroll
          for (int r = 0; r < 7; ++r) {
            const float2 v = part2[(sp * 7 + r) * pstride + k];
            nbk::ds_add(hi[r], lo[r], v.x, v.y);
          }
      for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < 7; ++r) {
          const float oh = __shfl_xor_sync(0xffffffffu, hi[r], o);
          const float ol = __shfl_xor_sync(0xffffffffu, lo[r], o);
          nbk::ds_add(hi[r], lo[r], oh, ol);
        }
#pragma unroll
      for (int r = 0; r < 7; ++r) f[r] = (double)hi[r] + (double)lo[r];
      f[6] = -f[6];
    } else {
#pragma unroll
      for (int r = 0; r < 7; ++r) f[r] = 0.0;
      if (have)
        for (int64_t sp = l; sp < S; sp += L)
#pragma unroll
          for (int r = 0; r < 7; ++r) f[r] += p.part[(sp * 7 + r) * pstride + k];
      for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < 7; ++r) f[r] += __shfl_xor_sync(0xffffffffu, f[r], o);
      f[6] = -f[6];
    }
    const bool cached = r1 - r0 <= kLDue;
    if (L >= 4) {
      // every lane of the CTA takes this branch (L is uniform) and every
      // shuffle inside; lanes without a row read a valid own row, write nothing
      int64_t i = p.act[k];
      i = i < r0 ? r0 : (i >= r1 ? r1 - 1 : i);  // own rows only
      if (!(have && l < 4))
#pragma unroll
        for (int r = 0; r < 7; ++r) f[r] = 0.0;
      const double nd = nbh::correct_row_lanes4(i, p.n_pad, tn, f, p.eta, p.dt_min, p.dt_max, p.x, p.v, p.a, p.jk,
                                                p.pot, p.t, p.dt, p.xp, p.vp, p.st, l, (int)(threadIdx.x & 31) - l, have);
      if (have && l == 0 && cached) s.due[i - r0] = (unsigned long long)__double_as_longlong(nd);
    } else if (have && l == 0) {
      int64_t i = p.act[k];
      i = i < r0 ? r0 : (i >= r1 ? r1 - 1 : i);  // own rows only
      const double nd = nbh::correct_row(i, p.n_pad, tn, f, p.eta, p.dt_min, p.dt_max, p.x, p.v, p.a, p.jk, p.pot,
                                         p.t, p.dt, p.xp, p.vp, p.st);
      if (cached) s.due[i - r0] = (unsigned long long)__double_as_longlong(nd);
    }
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(kLT, kLMaxPerSm) loop_kernel(LoopArgs p) {
  constexpr int JT = MIXED ? kLMixJT : kLF64JT;
  using ForceSmem = typename std::conditional<MIXED, nbk::MixedSmem<kLMixJT>, nbk::Fp64Smem<kLF64JT>>::type;
  __shared__ __align__(16) ForceSmem fsm;
  __shared__ LoopSmem s;
  const unsigned int G = gridDim.x;
  const int64_t N = p.N;
  const int64_t T = (N + kLT - 1) / kLT;
  const int64_t r0 = ((int64_t)blockIdx.x * T / G) * kLT;
  const int64_t r1 = min((((int64_t)blockIdx.x + 1) * T / G) * kLT, N);
  const int64_t jtiles = (N + JT - 1) / JT;
  const int64_t n_j = jtiles * JT;
  unsigned long long epoch = 0;
  long long steps = 0;
  double tn_prev = -INFINITY;  // the previous block time (they strictly increase)

  // placement: this CTA's rank among the CTAs on its SM.  A step with few
  // force items hands them to rank-0 CTAs first (one per SM), so that they
  // do not share an SM's pipes while other SMs idle.
  if (threadIdx.x == 0) {
    unsigned int smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const unsigned int r = atomicAdd(&p.ctl->smrank[smid % kMaxSmid], 1u);
    if (r == 0) atomicAdd(&p.ctl->nsm, 1u);
    s.rank = (int)r;
  }
  // rows between N and the end of the last tile are massless far-away
  // padding in the predicted j-store (they fill the last j-tile)
  if (blockIdx.x == G - 1)
    for (int64_t i = N + threadIdx.x; i < min(T * kLT, p.n_pad); i += kLT) {
      const double px[3] = {NB_PAD_POS, NB_PAD_POS, NB_PAD_POS}, pv[3] = {0.0, 0.0, 0.0};
      nbh::store_predicted(i, p.n_pad, px, pv, 0.0, p.xp, p.vp, p.jA, p.jB, p.jC, true, MIXED);
    }
  if (r1 - r0 <= kLDue)
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kLT)
      s.due[i - r0] = (unsigned long long)__double_as_longlong(p.t[i] + p.dt[i]);
  __syncthreads();
  publish_slice(p, r0, r1, s);

  for (;;) {
    if (!grid_barrier(p.ctl, epoch, G, p.st, &s.ok)) return;  // A: slice minima published
    read_slices(p, G, s);
    const unsigned long long tnb = s.tnb;
    const double tn = __longlong_as_double((long long)tnb);
    const int64_t n = s.total;
    if (!isfinite(tn) || n <= 0) {  // no particle has a finite next time
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&p.st->flags, NB_ST_NUMERIC);
      break;
    }
    if (tn > p.t_end) break;  // every particle has reached t_end
    if (!(tn > tn_prev)) {  // no progress: a state without valid steps (dt = 0)
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&p.st->flags, NB_ST_STALLED);
      break;
    }
    tn_prev = tn;
    if (steps >= p.max_steps) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&p.st->flags, NB_ST_TIMEOUT);
      break;
    }
    if (s.mine) write_active(p, r0, r1, tnb, s.before, s);
    predict_rows<MIXED>(p, r0, r1, tn, s);
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->wq = 0;  // nobody takes items before barrier B
    if (!grid_barrier(p.ctl, epoch, G, p.st, &s.ok)) return;  // B: list and j-store complete

    // forces (Sec. 4.1 step 4): items i-tile x j-split from the step's
    // counter, taken by the CTAs of rank < ceil(items / SMs).  When every CTA
    // has an SM of its own and there are no more items than CTAs (every small
    // block), CTA b takes item b: no counter round trips at all.
    const int64_t nI = (n + kLT - 1) / kLT;
    const int64_t S = loop_splits(n, jtiles, G, p.part_elems);
    const int64_t pstride = ((n + 31) / 32) * 32;
    const bool fin = S == 1;
    const int items = (int)(nI * S);
    const unsigned int nsm = __ldcg(&p.ctl->nsm);
    const bool fixed = nsm == G && items <= (int)G;
    const bool takes = fixed ? (int)blockIdx.x < items : (int64_t)s.rank * nsm < items;
    for (int round = 0;; ++round) {
      if (!takes || (fixed && round > 0)) break;
      if (!fixed) {
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s.item = (long long)atomicAdd(&p.ctl->wq, 1ULL);
        __syncthreads();
      }
      const int item = fixed ? (int)blockIdx.x : (int)min(s.item, (long long)items);
      if (item >= items) break;
      const int itile = item % (int)nI, split = item / (int)nI;
      const int64_t jlo = nbk::split_begin(split, S, jtiles) * JT;
      // mixed: the padding rows of the last j-tile are massless far-away
      // particles in the j-store; FP64: cut at N (the item fills the tile)
      const int64_t jhi = min(nbk::split_begin(split + 1, S, jtiles) * JT, MIXED ? n_j : N);
      double* out = fin ? p.F : p.part + split * 7 * pstride;
      const int64_t ostride = fin ? p.n_pad : pstride;
      if constexpr (MIXED)
        nbk::mixed_item<kLT, 1, kLMixJT>(fsm, p.jA, p.jB, p.jC, jlo, jhi, n_j, p.act, n, itile * kLT, p.eps2f,
                                         out, ostride, fin, p.tbox, nullptr, 0, nbk::FusedArgs(), nbk::ISrc(), true);
      else
        nbk::fp64_item<kLT, kLF64JT>(fsm, p.xp, p.vp, p.m, p.n_pad, jlo, jhi, p.act, n, itile * kLT, p.eps2, out,
                                     ostride, fin);
    }
    if (!grid_barrier(p.ctl, epoch, G, p.st, &s.ok)) return;  // C: forces complete
    correct_own<MIXED>(p, s, jtiles, G, r0, r1);
    ++steps;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      p.ctl->steps = steps;
      p.ctl->interactions += (long long)s.total * (long long)N;
    }
    if (p.seg_steps > 0 && steps >= p.seg_steps) {
      if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->more = 1u;
      break;
    }
    __syncthreads();  // the corrected rows are visible to the whole CTA
    publish_slice(p, r0, r1, s);
  }
}

// the barrier alone, three times; expect = CTAs it waits for (one more than
// launched makes every wait run out)
__global__ void barrier_check_kernel(LoopCtl* ctl, unsigned int expect, long long wait_ns, nb_dev_status* st) {
  __shared__ int ok;
  unsigned long long epoch = 0;
  for (int k = 0; k < 3; ++k)
    if (!grid_barrier(ctl, epoch, expect, st, &ok, wait_ns)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->steps = 3;
}

struct PLoop {
  LoopCtl* ctl = nullptr;
  unsigned long long* smin = nullptr;
  int32_t* scnt = nullptr;
  int gmax = 0;
  int per_sm[2] = {0, 0};  // resident CTAs per SM of each instantiation (0 = not yet asked)
};

PLoop* ploop_of(nb_ctx* c) { return static_cast<PLoop*>(c->loop); }

int ctas_per_sm(nb_ctx* c, PLoop* L, bool mixed) {
  int& ps = L->per_sm[mixed ? 1 : 0];
  if (ps == 0) {
    int occ = 0;
    cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, loop_kernel<true>, kLT, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, loop_kernel<false>, kLT, 0);
    if (e != cudaSuccess) return -1;
    ps = std::min(occ, kLMaxPerSm);
  }
  return ps;
}

}  // namespace

void nb_persistent_free(nb_ctx* c) {
  PLoop* L = c ? ploop_of(c) : nullptr;
  if (!L) return;
  if (L->ctl) cudaFree(L->ctl);
  if (L->smin) cudaFree(L->smin);
  if (L->scnt) cudaFree(L->scnt);
  delete L;
  c->loop = nullptr;
}

int nb_integrate_persistent(nb_ctx* c, double t_end) {
  if (c->n > nb_persistent_max_n(c)) return NB_EINVAL;
  const bool mixed = c->precision == NB_MIXED;
  PLoop* L = ploop_of(c);
  if (!L) {
    L = new PLoop();
    c->loop = L;
  }
  const int per_sm = ctas_per_sm(c, L, mixed);
  if (per_sm < 1) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  // as many CTAs as fit, but for a small system no more than twice its row
  // tiles (at least 32): the other CTAs would own no rows and take no force
  // items of its small blocks, and each barrier waits for every CTA's arrival
  const int64_t row_tiles = (c->n + kLT - 1) / kLT;
  const int G = (int)std::min<int64_t>(std::min(c->sm_count * per_sm, kLMaxG), std::max<int64_t>(32, 2 * row_tiles));
  if (G > L->gmax) {
    if (L->smin) cudaFree(L->smin);
    if (L->scnt) cudaFree(L->scnt);
    L->smin = nullptr;
    L->scnt = nullptr;
    if (!L->ctl && cudaMalloc((void**)&L->ctl, sizeof(LoopCtl)) != cudaSuccess) return NB_ENOMEM;
    if (cudaMalloc((void**)&L->smin, G * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&L->scnt, G * sizeof(int32_t)) != cudaSuccess) {
      L->gmax = 0;
      return NB_ENOMEM;
    }
    L->gmax = G;
  }
  // no valid run needs more than t_end / dt_min + 2 block steps
  const int64_t cap = std::min<int64_t>((int64_t)ceil(t_end / c->dt_min) + 2, 50000000);
  int64_t total = 0;
  for (;;) {
    long long seg = 0;
    if (mixed) {  // resident spatial order, renewed between launches
      const int rs = nb_ensure_sorted(c);
      if (rs != NB_OK) return rs;
      seg = std::max(1, c->sort_interval - c->perm_age);
    }
    LoopArgs p;
    memset(&p, 0, sizeof(p));
    p.N = c->n;
    p.n_pad = c->n_pad;
    p.eps2 = c->eps * c->eps;
    p.eps2f = (float)p.eps2;
    p.eta = c->eta;
    p.dt_min = c->dt_min;
    p.dt_max = c->dt_max;
    p.t_end = t_end;
    p.max_steps = cap;
    p.seg_steps = seg;
    p.m = c->m;
    p.x = c->x;
    p.v = c->v;
    p.a = c->a;
    p.jk = c->jk;
    p.pot = c->pot;
    p.t = c->t;
    p.dt = c->dt;
    p.xp = c->xp;
    p.vp = c->vp;
    p.jA = c->jA;
    p.jB = c->jB;
    p.jC = c->jC;
    p.tbox = mixed && c->perm_valid && c->far_tiles ? c->tbox : nullptr;
    p.act = c->act;
    p.F = c->F;
    p.part = c->part;
    p.part_elems = c->part_elems;
    p.smin = L->smin;
    p.scnt = L->scnt;
    p.ctl = L->ctl;
    p.st = c->status;
    if (cudaMemsetAsync(L->ctl, 0, sizeof(LoopCtl), c->stream) != cudaSuccess) return NB_ECUDA;
    void* args[] = {&p};
    cudaError_t e = cudaLaunchCooperativeKernel(mixed ? (const void*)loop_kernel<true> : (const void*)loop_kernel<false>,
                                                dim3((unsigned)G), dim3(kLT), args, 0, c->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return NB_ECUDA;
    }
    LoopCtl h;
    if (cudaMemcpyAsync(c->hpin, L->ctl, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return NB_ECUDA;
    memcpy(&h, c->hpin, sizeof(h));
    c->launches += 1;
    c->steps += h.steps;
    c->perm_age += (int)h.steps;
    c->interactions += (double)h.interactions;
    total += h.steps;
    if (h.abort) return NB_ETIMEOUT;
    if (!h.more) break;
    if (total > cap) return NB_ETIMEOUT;
  }
  c->pred_valid = false;
  c->f_valid = false;
  return NB_OK;
}

// the grid barrier's bounded wait on the device: G CTAs wait for G (phantom
// = 0) or G + 1 (phantom != 0, so the first wait runs out after wait_ms)
int nb_persistent_barrier_check(nb_ctx* c, int phantom, double wait_ms) {
  PLoop* L = ploop_of(c);
  if (!L) {
    L = new PLoop();
    c->loop = L;
  }
  if (!L->ctl && cudaMalloc((void**)&L->ctl, sizeof(LoopCtl)) != cudaSuccess) return NB_ENOMEM;
  const unsigned int G = (unsigned int)c->sm_count;  // one CTA per SM is always co-resident
  const unsigned int expect = G + (phantom ? 1u : 0u);
  const long long wait_ns = (long long)(wait_ms * 1e6);
  LoopCtl* ctl = L->ctl;
  nb_dev_status* st = c->status;
  if (cudaMemsetAsync(L->ctl, 0, sizeof(LoopCtl), c->stream) != cudaSuccess) return NB_ECUDA;
  void* args[] = {&ctl, (void*)&expect, (void*)&wait_ns, &st};
  if (cudaLaunchCooperativeKernel((const void*)barrier_check_kernel, dim3(G), dim3(kLT), args, 0, c->stream) !=
      cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  LoopCtl h;
  if (cudaMemcpyAsync(c->hpin, L->ctl, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NB_ECUDA;
  memcpy(&h, c->hpin, sizeof(h));
  c->launches += 1;
  if (h.abort) return NB_ETIMEOUT;
  return h.steps == 3 ? NB_OK : NB_ECUDA;
}
