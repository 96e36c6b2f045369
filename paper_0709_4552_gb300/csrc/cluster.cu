// cluster.cu -- the block-step loop of one small system (mixed path) on one
// thread-block cluster: the paper's ring algorithm (Sec. 4.3) on one chip.
//
// The C CTAs of a cluster (16 where the GPU can co-schedule them, else 8; one
// per SM) each own at most 1024 rows -- their "N/p particles", dealt out in
// blocks of 32 rows round-robin so that the active particles, which crowd in
// a few regions of the spatial order, spread over every CTA's corrector --
// and keep them in shared memory, predicted to each block time on
// the fly from the j-memory (the GRAPE-style double-single records of
// onboard.cu, Sec. 4.4 step 4).  Per block step (Sec. 4.1 steps 2-5):
//   A  every CTA has pushed the minimum of t_i + dt_i over its rows and how
//      many rows reach it into every CTA's shared memory (distributed shared
//      memory); each takes the block time and its offset in the active list,
//      lists its active rows, predicts them in FP64 (step 3; the corrector's
//      inputs stay in shared memory) and as double-single i data, while other
//      warps predict its j rows on the fly, and pushes its particles of the
//      first force group into every CTA;
//   B  the active block, in groups of 256 (later groups gathered from the
//      owners): each CTA sums the forces of its own j rows on the group (step
//      4, Eq. 3: FP32 pairwise arithmetic on double-single differences in
//      packed FP32x2 pairs, per-chunk FP32 sums folded into double-single, the
//      self pair excluded by row), partials reduced in double-single FP32;
//   C  each owner adds the C double-single partial sums of its particles in
//      CTA order and corrects them (step 5; the four-lane corrector of
//      hermite.cuh, which also rewrites their j-memory records), then pushes
//      its next minimum.
// The barriers are the cluster's hardware barrier (no spin loop anywhere);
// every CTA reads the same published values, so every CTA takes the same
// decisions and leaves the loop at the same step (and a last barrier keeps
// every CTA's shared memory alive while others may read it).  Nothing
// leaves the chip but the state each owner writes back.
#include <cooperative_groups.h>
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "force_common.cuh"
#include "hermite.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kCT = 256;       // threads per CTA
constexpr int kCRows = 1024;   // rows per CTA at most
constexpr int kGI = 256;       // active particles per force group
constexpr int kChunk = 128;    // j per FP32 partial sum before the double-single fold
constexpr int kMaxC = 16;      // CTAs per cluster at most
constexpr int kCC = 256;       // own active particles whose corrector inputs stay in shared memory
constexpr unsigned long long kInfBits = 0x7FF0000000000000ULL;
constexpr int kRB = 32;        // rows per ownership block (dealt round-robin to the CTAs)

// row of own row index q of CTA me (blocks of kRB rows, block b owned by b % C)
__device__ __forceinline__ int64_t own_row(int q, int me, int C) {
  return ((int64_t)(q / kRB) * C + me) * kRB + (q % kRB);
}
// own row index of a row, or -1 when another CTA owns it
__device__ __forceinline__ int own_index(int64_t row, int me, int C) {
  const int64_t b = row / kRB;
  return (int)(b % C) == me ? (int)((b / C) * kRB + row % kRB) : -1;
}
// rows CTA me owns
__device__ __forceinline__ int own_count(int64_t N, int me, int C) {
  const int64_t nb = (N + kRB - 1) / kRB;  // blocks
  if (me >= nb) return 0;
  const int64_t mine = (nb - 1 - me) / C + 1;  // blocks me, me + C, ...
  const int64_t last = me + (mine - 1) * C;    // its last block (maybe partial)
  return (int)((mine - 1) * kRB + min((int64_t)kRB, N - last * kRB));
}

struct ClusterCtl {
  long long steps;
  long long interactions;
};

struct ClusterArgs {
  int64_t N, n_pad;
  float eps2f;
  double eta, dt_min, dt_max, t_end;
  long long max_steps;
  const double* m;
  double *x, *v, *a, *jk, *pot, *t, *dt;
  double *xp, *vp;
  float4* jm;
  ClusterCtl* ctl;
  nb_dev_status* st;
};

struct CSmem {
  // own active particles in list order, predicted (double-single positions,
  // FP32 velocities): A = (xh, yh, zh, vx), B = (xl, yl, zl, vy), C = (vz, row bits)
  float4 iA[kCRows], iB[kCRows];
  float2 iC[kCRows];
  // the force group's i data, the same layout (group 0 pushed by the owners,
  // later groups gathered from them)
  float4 gA[kGI], gB[kGI];
  float2 gC[kGI];
  // every CTA's (minimum of t_i + dt_i over its rows, rows at it), pushed by each
  ulonglong2 pairs[kMaxC];
  // own rows predicted to the block time (double-single positions, FP32 v, m)
  float jxh[kCRows], jyh[kCRows], jzh[kCRows], jxl[kCRows], jyl[kCRows], jzl[kCRows];
  float jvx[kCRows], jvy[kCRows], jvz[kCRows], jms[kCRows];
  int32_t irow[kCRows];
  // own rows' next due time t_i + dt_i (bit pattern), kept by the corrector
  unsigned long long due[kCRows];
  // this CTA's double-single partial sums on the group (read by the owners)
  float2 part[7][kGI];
  // the owner's sums of its particles of the group (all CTAs' partials)
  double fsum[7][kGI];
  // corrector inputs of own active particles k < kCC, kept from their
  // prediction: old t, dt, acceleration, jerk and the predicted x, v
  double cT[kCC], cDT[kCC], cA0[3][kCC], cJ0[3][kCC], cXP[3][kCC], cVP[3][kCC];
  // every CTA's offset and count in the active list (read at barrier A)
  int cbefore[kMaxC], cmine[kMaxC];
  double tn;
  long long total;
  unsigned long long wmin[kCT / 32];
  int wcnt[kCT / 32];
};

// minimum of t_i + dt_i over own rows and the rows at it, pushed into every
// CTA's pairs[me] (read there after the next cluster barrier)
__device__ void publish(CSmem& s, cg::cluster_group& cl, int me, int C, int nr) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned long long best = kInfBits;
  for (int q = tid; q < nr; q += kCT) best = s.due[q] < best ? s.due[q] : best;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, best, o);
    best = u < best ? u : best;
  }
  if (lane == 0) s.wmin[w] = best;
  __syncthreads();
  best = kInfBits;
  for (int k = 0; k < kCT / 32; ++k) best = s.wmin[k] < best ? s.wmin[k] : best;
  int cnt = 0;
  for (int q = tid; q < nr; q += kCT) cnt += s.due[q] == best;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) s.wcnt[w] = cnt;
  __syncthreads();
  if (tid < C) {
    int c = 0;
    for (int k = 0; k < kCT / 32; ++k) c += s.wcnt[k];
    *cl.map_shared_rank(&s.pairs[me], tid) = make_ulonglong2(best, (unsigned long long)c);
  }
}

// own rows at the block time, ascending, into s.irow (each thread scans a
// contiguous run of rows; a block scan places the runs in order)
__device__ void list_rows(CSmem& s, int me, int C, int nr, unsigned long long tnb) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int W = (nr + kCT - 1) / kCT;
  const int q0 = min(tid * W, nr), q1 = min(q0 + W, nr);
  int cnt = 0;
  for (int q = q0; q < q1; ++q) cnt += s.due[q] == tnb;
  int inc = cnt;  // inclusive warp scan
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) s.wcnt[w] = inc;
  __syncthreads();
  int base = 0;
  for (int k = 0; k < w; ++k) base += s.wcnt[k];
  int at = base + inc - cnt;
  for (int q = q0; q < q1; ++q)
    if (s.due[q] == tnb) s.irow[at++] = (int32_t)own_row(q, me, C);
  __syncthreads();
}

__device__ __forceinline__ void split_ds(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

__global__ void __launch_bounds__(kCT, 1) cluster_loop_kernel(ClusterArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CSmem& s = *reinterpret_cast<CSmem*>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int64_t N = p.N;
  const int nr = own_count(N, me, C);  // <= kCRows (checked by the host)
  long long steps = 0;
  double tn_prev = -INFINITY;  // the previous block time (they strictly increase)

  for (int q = tid; q < nr; q += kCT) {
    const int64_t r = own_row(q, me, C);
    s.due[q] = (unsigned long long)__double_as_longlong(p.t[r] + p.dt[r]);
  }
  __syncthreads();
  cl.sync();  // every CTA of the cluster runs before any writes another's shared memory
  publish(s, cl, me, C, nr);
  for (;;) {
    cl.sync();  // A: every CTA's minimum and count are in every CTA's pairs
    if (tid < 32) {  // lane c holds CTA c's pair; the minimum and the offsets by shuffles
      const ulonglong2 pr = tid < C ? s.pairs[tid] : make_ulonglong2(kInfBits, 0ULL);
      const unsigned long long pm = pr.x;
      const int pc = (int)pr.y;
      unsigned long long tb = pm;
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, tb, o);
        tb = u < tb ? u : tb;
      }
      const int k = (tid < C && pm == tb) ? pc : 0;
      int inc = k;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (tid >= o) inc += u;
      }
      if (tid < C) {
        s.cbefore[tid] = inc - k;
        s.cmine[tid] = k;
      }
      if (tid == 31) {
        s.tn = __longlong_as_double((long long)tb);
        s.total = inc;
      }
    }
    __syncthreads();
    const double tn = s.tn;
    const long long n = s.total;
    if (!isfinite(tn) || n <= 0) {  // no particle has a finite next time
      if (me == 0 && tid == 0) atomicOr(&p.st->flags, NB_ST_NUMERIC);
      break;
    }
    if (tn > p.t_end) break;  // every particle has reached t_end
    if (!(tn > tn_prev)) {  // no progress: a state without valid steps (dt = 0)
      if (me == 0 && tid == 0) atomicOr(&p.st->flags, NB_ST_STALLED);
      break;
    }
    tn_prev = tn;
    if (steps >= p.max_steps) {
      if (me == 0 && tid == 0) atomicOr(&p.st->flags, NB_ST_TIMEOUT);
      break;
    }
    const int mine = s.cmine[me], before = s.cbefore[me];
    const unsigned long long tnb = (unsigned long long)__double_as_longlong(tn);
    list_rows(s, me, C, nr, tnb);
    // the first iw threads (whole warps) predict the own active particles,
    // the others the own j rows: the two global round trips overlap
    const int iw = min(kCT, (mine + 31) & ~31);
    // own active particles: FP64 prediction (step 3), double-single i data
    // for the forces, and the corrector's inputs
    for (int k = tid; k < mine; k += kCT) {
      const int64_t row = s.irow[k];
      const double t0 = p.t[row], dt0 = p.dt[row];
      double a0[3], j0[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        a0[d] = p.a[d * p.n_pad + row];
        j0[d] = p.jk[d * p.n_pad + row];
      }
      double px[3], pv[3];
      nbh::taylor(row, p.n_pad, tn - t0, p.x, p.v, p.a, p.jk, px, pv);
      if (k < kCC) {
        s.cT[k] = t0;
        s.cDT[k] = dt0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          s.cA0[d][k] = a0[d];
          s.cJ0[d][k] = j0[d];
          s.cXP[d][k] = px[d];
          s.cVP[d][k] = pv[d];
        }
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          p.xp[d * p.n_pad + row] = px[d];
          p.vp[d * p.n_pad + row] = pv[d];
        }
      }
      float xh[3], xl[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) split_ds(px[d], xh[d], xl[d]);
      s.iA[k] = make_float4(xh[0], xh[1], xh[2], __double2float_rn(pv[0]));
      s.iB[k] = make_float4(xl[0], xl[1], xl[2], __double2float_rn(pv[1]));
      s.iC[k] = make_float2(__double2float_rn(pv[2]), __int_as_float((int)row));
    }
    // own j rows predicted on the fly from the j-memory (Sec. 4.4 step 4)
    for (int q = (tid - iw + kCT) % kCT; q < nr; q += kCT) {
      const int64_t row = own_row(q, me, C);
      const float4 R0 = p.jm[row], R1 = p.jm[p.n_pad + row], R2 = p.jm[2 * p.n_pad + row],
                   R3 = p.jm[3 * p.n_pad + row], R4 = p.jm[4 * p.n_pad + row];
      const float h = __double2float_rn(tn - p.t[row]);
      const float h2 = 2.0f * h, h15 = 1.5f * h;
      float hi, lo, vv;
      nbk::ds_predict(R0.x, R1.x, R2.x, R3.x, R4.x, R2.w, h, h2, h15, hi, lo, vv);
      s.jxh[q] = hi; s.jxl[q] = lo; s.jvx[q] = vv;
      nbk::ds_predict(R0.y, R1.y, R2.y, R3.y, R4.y, R3.w, h, h2, h15, hi, lo, vv);
      s.jyh[q] = hi; s.jyl[q] = lo; s.jvy[q] = vv;
      nbk::ds_predict(R0.z, R1.z, R2.z, R3.z, R4.z, R4.w, h, h2, h15, hi, lo, vv);
      s.jzh[q] = hi; s.jzl[q] = lo; s.jvz[q] = vv;
      s.jms[q] = R0.w;
    }
    if ((nr & 1) && tid == kCT - 1) {  // the pair loop's padding row: massless, far away
      s.jxh[nr] = s.jyh[nr] = s.jzh[nr] = nbk::kFarF;
      s.jxl[nr] = s.jyl[nr] = s.jzl[nr] = 0.0f;
      s.jvx[nr] = s.jvy[nr] = s.jvz[nr] = 0.0f;
      s.jms[nr] = 0.0f;
    }
    __syncthreads();
    // push this CTA's particles of the first group into every CTA's group
    // buffer (every CTA finished reading its buffer before barrier A)
    {
      const int npush = max(0, min(mine, kGI - before));
      for (int e = tid; e < npush * C; e += kCT) {
        const int k = e / C, c = e - (e / C) * C;
        *cl.map_shared_rank(&s.gA[before + k], c) = s.iA[k];
        *cl.map_shared_rank(&s.gB[before + k], c) = s.iB[k];
        *cl.map_shared_rank(&s.gC[before + k], c) = s.iC[k];
      }
    }
    cl.sync();  // B: the first group's i data is in every CTA, every CTA's i data is ready

    for (long long g0 = 0; g0 < n; g0 += kGI) {
      const int gn = (int)min((long long)kGI, n - g0);
      if (g0 > 0) {
        // a later group's i data from its owners' shared memory (the loads
        // first, then the stores: one round trip)
        for (int k = tid; k < gn; k += kCT) {
          const int pos = (int)(g0 + k);
          int c = 0;
#pragma unroll
          for (int cc = 1; cc < kMaxC; ++cc) c += (cc < C && s.cbefore[cc] <= pos) ? 1 : 0;
          const int a = pos - s.cbefore[c];
          const float4 A = *cl.map_shared_rank(&s.iA[a], c);
          const float4 B = *cl.map_shared_rank(&s.iB[a], c);
          const float2 Ci = *cl.map_shared_rank(&s.iC[a], c);
          s.gA[k] = A;
          s.gB[k] = B;
          s.gC[k] = Ci;
        }
        __syncthreads();
      }
      // own j rows on the group: P threads per particle (a power of two, at
      // most 32, lanes of one warp), each over a contiguous part of the rows
      int P = 32;
      while (P > 1 && P * gn > kCT) P >>= 1;
      const int i = tid / P, part = tid % P;
      float hi7[7], lo7[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) hi7[c] = lo7[c] = 0.0f;
      if (i < gn) {
        const float4 A = s.gA[i], B = s.gB[i];
        const float2 Ci = s.gC[i];
        const float xh = A.x, yh = A.y, zh = A.z, xl = B.x, yl = B.y, zl = B.z;
        const float vx = A.w, vy = B.w, vz = Ci.x;
        const int self = own_index(__float_as_int(Ci.y), me, C);  // -1: held by another CTA
        // pairs of own rows (2u, 2u + 1) in packed FP32x2 instructions (two j per
        // instruction, as the force item's pair loop); an odd row count ends in
        // the massless far-away padding row nr
        const int np = (nr + 1) / 2;
        const int u0 = (int)((int64_t)part * np / P), u1 = (int)((int64_t)(part + 1) * np / P);
        const float2 nxh = make_float2(-xh, -xh), nyh = make_float2(-yh, -yh), nzh = make_float2(-zh, -zh);
        const float2 nxl = make_float2(-xl, -xl), nyl = make_float2(-yl, -yl), nzl = make_float2(-zl, -zl);
        const float2 nvx = make_float2(-vx, -vx), nvy = make_float2(-vy, -vy), nvz = make_float2(-vz, -vz);
        const float2 e2 = make_float2(p.eps2f, p.eps2f), m3 = make_float2(-3.0f, -3.0f);
        const float2* JXH = reinterpret_cast<const float2*>(s.jxh);
        const float2* JYH = reinterpret_cast<const float2*>(s.jyh);
        const float2* JZH = reinterpret_cast<const float2*>(s.jzh);
        const float2* JXL = reinterpret_cast<const float2*>(s.jxl);
        const float2* JYL = reinterpret_cast<const float2*>(s.jyl);
        const float2* JZL = reinterpret_cast<const float2*>(s.jzl);
        const float2* JVX = reinterpret_cast<const float2*>(s.jvx);
        const float2* JVY = reinterpret_cast<const float2*>(s.jvy);
        const float2* JVZ = reinterpret_cast<const float2*>(s.jvz);
        const float2* JMS = reinterpret_cast<const float2*>(s.jms);
        for (int c0 = u0; c0 < u1; c0 += kChunk / 2) {
          const int c1 = min(c0 + kChunk / 2, u1);
          float2 pp[7];
#pragma unroll
          for (int c = 0; c < 7; ++c) pp[c] = make_float2(0.0f, 0.0f);
          for (int u = c0; u < c1; ++u) {
            const float2 dx = __fadd2_rn(__fadd2_rn(JXH[u], nxh), __fadd2_rn(JXL[u], nxl));
            const float2 dy = __fadd2_rn(__fadd2_rn(JYH[u], nyh), __fadd2_rn(JYL[u], nyl));
            const float2 dz = __fadd2_rn(__fadd2_rn(JZH[u], nzh), __fadd2_rn(JZL[u], nzl));
            const float2 wx = __fadd2_rn(JVX[u], nvx), wy = __fadd2_rn(JVY[u], nvy), wz = __fadd2_rn(JVZ[u], nvz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e2)));
            const float2 rw = __ffma2_rn(dz, wz, __ffma2_rn(dy, wy, __fmul2_rn(dx, wx)));
            float2 rinv = make_float2(nb_rsqrt_approx(r2.x), nb_rsqrt_approx(r2.y));
            rinv.x = (2 * u == self) ? 0.0f : rinv.x;  // the self pair, by row
            rinv.y = (2 * u + 1 == self) ? 0.0f : rinv.y;
            const float2 rinv2 = __fmul2_rn(rinv, rinv);
            const float2 mr = __fmul2_rn(JMS[u], rinv);
            const float2 mr3 = __fmul2_rn(mr, rinv2);
            const float2 a3 = __fmul2_rn(__fmul2_rn(rw, m3), rinv2);  // the jerk term formed before it is added
            pp[6] = __fadd2_rn(pp[6], mr);
            pp[0] = __ffma2_rn(mr3, dx, pp[0]);
            pp[1] = __ffma2_rn(mr3, dy, pp[1]);
            pp[2] = __ffma2_rn(mr3, dz, pp[2]);
            pp[3] = __ffma2_rn(mr3, __ffma2_rn(a3, dx, wx), pp[3]);
            pp[4] = __ffma2_rn(mr3, __ffma2_rn(a3, dy, wy), pp[4]);
            pp[5] = __ffma2_rn(mr3, __ffma2_rn(a3, dz, wz), pp[5]);
          }
#pragma unroll
          for (int c = 0; c < 7; ++c) nbk::ds_add(hi7[c], lo7[c], pp[c].x + pp[c].y, 0.0f);  // double-single fold
        }
      }
      // the P parts of a particle, lanes of one warp: a double-single
      // butterfly in FP32 (every lane; the FP64 pipe is 1/64 of FP32 here)
      for (int o = P / 2; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
          const float oh = __shfl_xor_sync(0xffffffffu, hi7[c], o);
          const float ol = __shfl_xor_sync(0xffffffffu, lo7[c], o);
          nbk::ds_add(hi7[c], lo7[c], oh, ol);
        }
      if (i < gn && part == 0)
#pragma unroll
        for (int c = 0; c < 7; ++c) s.part[c][i] = make_float2(hi7[c], lo7[c]);
      __syncthreads();
      cl.sync();  // C: every CTA's partial sums on the group are ready

      // the owner's particles of this group: the C partials in CTA order, then
      // the corrector on four lanes per particle (step 5)
      const int lo_pos = max((int)g0, before), hi_pos = min((int)g0 + gn, before + mine);
      const int own = hi_pos - lo_pos;  // CTA-uniform
      // one thread per (particle, component): the C double-single partials
      // (independent loads, one round trip) summed in CTA order
      for (int e = tid; e < own * 7; e += kCT) {
        const int k = lo_pos - (int)g0 + e / 7, c = e % 7;
        float2 pv[kMaxC];
#pragma unroll
        for (int cc = 0; cc < kMaxC; ++cc)
          pv[cc] = cc < C ? *cl.map_shared_rank(&s.part[c][k], cc) : make_float2(0.0f, 0.0f);
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int cc = 0; cc < kMaxC; ++cc)
          if (cc < C) nbk::ds_add(h, l, pv[cc].x, pv[cc].y);
        const double acc = (double)h + (double)l;
        s.fsum[c][k] = c == 6 ? -acc : acc;
      }
      __syncthreads();
      for (int k0 = 0; k0 < own; k0 += kCT / 4) {
        const int sub = tid & 3, cs = sub < 3 ? sub : 0;
        const int pos = lo_pos + k0 + (tid >> 2);
        const bool have = pos < hi_pos;
        double fo[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) fo[c] = have ? s.fsum[c][pos - (int)g0] : 0.0;
        const int kk = have ? pos - before : lo_pos - before;  // own active index
        const int64_t row = s.irow[kk];
        nbh::CorrIn in;
        if (kk < kCC) {
          in = nbh::CorrIn{s.cT[kk], s.cDT[kk], s.cA0[cs][kk], s.cJ0[cs][kk], s.cXP[cs][kk], s.cVP[cs][kk]};
        } else {
          const int64_t q = cs * p.n_pad + row;
          in = nbh::CorrIn{p.t[row], p.dt[row], p.a[q], p.jk[q], p.xp[q], p.vp[q]};
        }
        const double nd = nbh::correct_lanes4(row, p.n_pad, tn, fo, in, p.eta, p.dt_min, p.dt_max, p.x, p.v, p.a,
                                              p.jk, p.pot, p.t, p.dt, p.st, sub, (tid & 31) - sub, have, p.jm);
        if (have && sub == 0) s.due[own_index(row, me, C)] = (unsigned long long)__double_as_longlong(nd);
      }
      __syncthreads();
      if (g0 + kGI < n) cl.sync();  // D: the partials are read before the next group's are written
    }
    ++steps;
    if (me == 0 && tid == 0) {
      p.ctl->steps = steps;
      p.ctl->interactions += n * (long long)N;
    }
    __syncthreads();
    publish(s, cl, me, C, nr);
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

struct CLoop {
  ClusterCtl* ctl = nullptr;
  int csize = 0;  // CTAs per cluster (0 = not yet chosen)
};

}  // namespace

void nb_cluster_free(nb_ctx* c) {
  CLoop* L = c ? static_cast<CLoop*>(c->cloop) : nullptr;
  if (!L) return;
  if (L->ctl) cudaFree(L->ctl);
  delete L;
  c->cloop = nullptr;
}

// CTAs per cluster this GPU co-schedules with the loop's shared memory: 16, else 8 (0 = none)
int nb_cluster_size(nb_ctx* c) {
  CLoop* L = static_cast<CLoop*>(c->cloop);
  if (!L) {
    L = new CLoop();
    c->cloop = L;
  }
  if (L->csize) return L->csize;
  const size_t smem = sizeof(CSmem);
  if (cudaFuncSetAttribute(cluster_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(cluster_loop_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_loop_kernel, &cfg) == cudaSuccess && nclusters >= 1) {
      L->csize = cs;
      return cs;
    }
    cudaGetLastError();
  }
  return 0;
}

int nb_integrate_cluster(nb_ctx* c, double t_end) {
  if (c->precision != NB_MIXED || c->n_clusters > 0) return NB_EINVAL;
  const int C = nb_cluster_size(c);
  if (C < 1) return NB_ECUDA;
  if (c->n > (int64_t)C * kCRows) return NB_EINVAL;  // (whole blocks of kRB rows per CTA: kCRows / kRB of them)
  CLoop* L = static_cast<CLoop*>(c->cloop);
  if (!L->ctl && cudaMalloc((void**)&L->ctl, sizeof(ClusterCtl)) != cudaSuccess) {
    cudaGetLastError();
    return NB_ENOMEM;
  }
  const int rj = nb_jm_ensure(c);
  if (rj != NB_OK) return rj;
  ClusterArgs p;
  memset(&p, 0, sizeof(p));
  p.N = c->n;
  p.n_pad = c->n_pad;
  p.eps2f = (float)(c->eps * c->eps);
  p.eta = c->eta;
  p.dt_min = c->dt_min;
  p.dt_max = c->dt_max;
  p.t_end = t_end;
  p.max_steps = std::min<long long>((long long)ceil(t_end / c->dt_min) + 2, 50000000LL);
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
  p.jm = c->jm;
  p.ctl = L->ctl;
  p.st = c->status;
  if (cudaMemsetAsync(L->ctl, 0, sizeof(ClusterCtl), c->stream) != cudaSuccess) return NB_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = sizeof(CSmem);
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, cluster_loop_kernel, p) != cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  ClusterCtl h;
  if (cudaMemcpyAsync(c->hpin, L->ctl, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return NB_ECUDA;
  memcpy(&h, c->hpin, sizeof(h));
  c->launches += 1;
  c->steps += h.steps;
  c->interactions += (double)h.interactions;
  // the rows stayed in place and every corrected row's record was rewritten:
  // the j-memory is current for the new state
  c->state_ver++;
  c->jm_ver = c->state_ver;
  c->pred_valid = false;
  c->f_valid = false;
  return NB_OK;
}
