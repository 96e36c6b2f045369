// force_common.cuh -- the direct-sum force "work item" (Sec. 4.1 step 4,
// Eq. 3) shared by every launch shape: the grid kernels of the host-driven
// path, the persistent kernels of the graph-driven loop and of the batched
// ensemble.  One item = one i-tile (NT*IPT active particles of one list)
// against one contiguous j-range [jlo, jhi) of the j-store.
//
// For each active i and every j != i (Plummer softening eps, G = 1):
//   r = x_j - x_i, w = v_j - v_i, s^2 = r.r + eps^2,
//   acc += m_j r / s^3,  jerk += m_j (w / s^3 - 3 (r.w) r / s^5),  pot -= m_j / s.
// Items sum +m/s; the sign of the potential is applied when the item is
// final (one split) or by the split reduction.
//
// Mixed path: positions are double-single pairs (hi, lo) written by the
// predictor; r = (x_j.hi - x_i.hi) + (x_j.lo - x_i.lo) is the FP64 difference
// rounded to FP32 within about an ulp (hi difference exact for close pairs,
// Sterbenz).  Pairwise arithmetic is FP32 with one hardware rsqrt (MUFU),
// optionally refined by one Newton step (NB_MIXED_NEWTON).  The jerk term of
// a pair is formed completely before it is accumulated: its two parts
// (w / s^3 and -3 (r.w) r / s^5) cancel for close pairs, and adding them to
// the running sum one after the other costs up to 4x in the worst particle's
// error.  FP32 partial sums over one j-tile (JT pairs) are folded into
// double-single accumulators (an FP32 pair hi + lo, Knuth's TwoSum: no FP64
// instruction in the loop; NB_MIXED_DS_FOLD = 0 folds into FP64 instead).
// j-tiles (40 B per particle: float4
// hi+m, float4 lo+vx, float2 vy vz) are staged in shared memory with cp.async
// double buffering and read as warp-wide broadcasts.
//
// FP64 path: every operation in IEEE FP64, 1/s from an FP32 seed refined in
// FP64; per-tile FP64 partials folded into (hi, lo) accumulators with Knuth's
// TwoSum.  On GB300 the FP64 pipe issues 2 FMA/clk/SM (1/64 of FP32), which
// bounds this path.
//
// Self pair: excluded by index, as in the definition.  Mixed path: only the
// j-tile holding one of a warp's own i needs the test, so a warp vote picks a
// masked copy of the inner loop for that tile (no per-pair cost elsewhere).
//
// Ragged j-ranges: a tile reaching past jhi loads clamped (in-bounds)
// addresses and the slots past jhi are overwritten with a massless particle
// far away, which contributes exactly zero.
#pragma once

#include "nb_internal.cuh"

// one Newton step on the hardware rsqrt in the mixed path (1 = on)
#ifndef NB_MIXED_NEWTON
#define NB_MIXED_NEWTON 0
#endif
// FP64 accumulators of the mixed path in shared memory instead of registers
#ifndef NB_MIXED_SMEM_ACC
#define NB_MIXED_SMEM_ACC 0
#endif
// double-single (FP32 TwoSum) accumulators of the mixed path (0 = FP64)
#ifndef NB_MIXED_DS_FOLD
#define NB_MIXED_DS_FOLD 1
#endif
// unroll depth of the mixed inner loop over a j-tile
#ifndef NB_MIXED_UNROLL
#define NB_MIXED_UNROLL 4
#endif
// one i per thread: two j per instruction with the packed FP32x2 operations
// of sm_100+ (1 = on; 0 = the scalar loop)
#ifndef NB_MIXED_PACKED
#define NB_MIXED_PACKED 1
#endif
#define NB_STR_(x) #x
#define NB_PRAGMA_UNROLL(n) _Pragma(NB_STR_(unroll n))

namespace nbk {

constexpr float kFarF = 1.0e15f;

// first j-tile of split s when `tiles` tiles are shared by S splits as evenly
// as possible (split sizes differ by at most one tile)
__device__ __forceinline__ int64_t split_begin(int64_t s, int64_t S, int64_t tiles) { return s * tiles / S; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int JT>
struct MixedSmem {
  static constexpr bool kFused = false;
  float4 A[2][JT];
  float4 B[2][JT];
  float2 C[2][JT];
};

// ---- on-the-fly prediction of the j-particles (Sec. 4.4 step 4) -------------
// GRAPE predicts the j-particles on the board, in its pipelines, as they
// stream past; the host predicts only the n active i (step 3).  Here the
// force item can do the same: instead of a predicted j-store it loads the
// "j-memory" record of each particle, written from its FP64 state after every
// correction (rows in the resident order, 5 float4 rows of stride n_pad):
//   R0 = (xh, m)   R1 = (xl, Rd)   R2 = (vh, j6.x)   R3 = (vl, j6.y)   R4 = (a2, j6.z)
// with x = xh + xl and v = vh + vl the double-single splits of the FP64
// position and velocity, a2 = fl32(a/2), j6 = fl32(jerk/6), and Rd a bound
// on the distance the particle can move within its current step (the tile
// boxes of the far test are grown by it), plus its FP64 time t_j.  The item
// predicts the tile it has staged, to the block time T, into the same
// pair-interleaved shared tile the plain loader fills:
//   h = fl32(T - t_j)  (exact: a multiple of dt_min below dt_max),
//   xp = x + h (v + h (a/2 + h j/6))  in double-single FP32 (TwoSum and an
//        FMA-exact product carry the x + v h part to ~2^-48; the a and jerk
//        terms are FP32, so their rounding is 2^-24 |a h^2 / 2| at most),
//   vp = v + h (a + h j/2)  in FP32 (the mixed path's velocities are FP32).
template <int JT>
struct FusedSmem {
  static constexpr bool kFused = true;
  float4 R[2][5][JT];  // staged j-memory records (double-buffered)
  double T[2][JT];     // their times t_j
  float4 A[JT];        // the predicted tile, pair-interleaved (PairTile)
  float4 B[JT];
  float2 C[JT];
};

// Where an item's i-particles come from.  By default they are the j-store
// rows its list names (every particle's own predicted row).  For forces on
// particles held elsewhere -- the visiting block of the ring algorithm
// (Sec. 4.3), whose positions and velocities arrive from another rank -- the
// list indexes separate arrays instead, and self[k] gives the j-store slot of
// list position k's particle when this store holds it (else -1), which keeps
// the self pair excluded by index.
struct ISrc {
  const float4* __restrict__ A = nullptr;  // mixed: (x_hi, m), (x_lo, vx), (vy, vz) like jA/jB/jC
  const float4* __restrict__ B = nullptr;
  const float2* __restrict__ C = nullptr;
  const double* __restrict__ x = nullptr;  // FP64: SoA rows x[3][stride], v[3][stride]
  const double* __restrict__ v = nullptr;
  int64_t stride = 0;
  const int32_t* __restrict__ self = nullptr;
};

struct FusedArgs {
  const float4* __restrict__ jm = nullptr;  // R0..R4 rows, stride n_pad
  int64_t stride = 0;
  const double* __restrict__ tj = nullptr;  // FP64 times of the rows
  double T = 0.0;                           // block time
};

template <int NT, int JT>
__device__ __forceinline__ void mixed_load_tile(float4* sA, float4* sB, float2* sC, const float4* __restrict__ jA,
                                                const float4* __restrict__ jB, const float2* __restrict__ jC,
                                                int64_t j0, int64_t jhi) {
#pragma unroll
  for (int q = threadIdx.x; q < JT; q += NT) {
    const int64_t j = min(j0 + q, jhi - 1);
    cp_async16(&sA[q], &jA[j]);
    cp_async16(&sB[q], &jB[j]);
    cp_async8(&sC[q], &jC[j]);
  }
}

// Pair layout of one tile buffer for the packed loop: j-particles 2u and
// 2u+1 side by side, so that one 16-byte broadcast yields two (j, j+1) pairs:
//   P0[u] = (xh, xh', yh, yh')   P1[u] = (zh, zh', m, m')   (in sA)
//   P2[u] = (vx, vx', vy, vy')   P3[u] = (vz, vz', xl, xl') (in sB)
//   P4[u] = (yl, yl', zl, zl')                              (in sC)
// (u < JT/2; same 40 B per particle as the plain layout).  The float of
// particle q, pair slot (q & 1), sits at 4 (q >> 1) + (q & 1) (+2 for the
// second pair of a vector); 4-byte asynchronous copies scatter it there.
template <int JT>
struct PairTile {
  float *p0, *p1, *p2, *p3, *p4;
  __device__ __forceinline__ PairTile(float4* sA, float4* sB, float2* sC)
      : p0((float*)sA), p1((float*)(sA + JT / 2)), p2((float*)sB), p3((float*)(sB + JT / 2)), p4((float*)sC) {}
};

template <int NT, int JT>
__device__ __forceinline__ void mixed_load_tile_pairs(float4* sA, float4* sB, float2* sC,
                                                      const float4* __restrict__ jA,
                                                      const float4* __restrict__ jB,
                                                      const float2* __restrict__ jC, int64_t j0, int64_t jhi) {
  const PairTile<JT> t(sA, sB, sC);
#pragma unroll
  for (int q = threadIdx.x; q < JT; q += NT) {
    const int64_t j = min(j0 + q, jhi - 1);
    const float* a = (const float*)&jA[j];
    const float* b = (const float*)&jB[j];
    const float* c = (const float*)&jC[j];
    const int o = 4 * (q >> 1) + (q & 1);
    cp_async4(t.p0 + o, a + 0);
    cp_async4(t.p0 + o + 2, a + 1);
    cp_async4(t.p1 + o, a + 2);
    cp_async4(t.p1 + o + 2, a + 3);
    cp_async4(t.p2 + o, b + 3);
    cp_async4(t.p2 + o + 2, c + 0);
    cp_async4(t.p3 + o, c + 1);
    cp_async4(t.p3 + o + 2, b + 0);
    cp_async4(t.p4 + o, b + 1);
    cp_async4(t.p4 + o + 2, b + 2);
  }
}

template <int NT, int JT>
__device__ __forceinline__ void jm_load_tile(FusedSmem<JT>& sm, int buf, const FusedArgs& fa, int64_t j0,
                                             int64_t jhi) {
#pragma unroll
  for (int q = threadIdx.x; q < JT; q += NT) {
    const int64_t j = min(j0 + q, jhi - 1);
#pragma unroll
    for (int k = 0; k < 5; ++k) cp_async16(&sm.R[buf][k][q], &fa.jm[k * fa.stride + j]);
    cp_async8(&sm.T[buf][q], &fa.tj[j]);
  }
}

// x + delta in double-single: (xh, xl) + (p + q) with p + q = h (s + e) exact
// up to the rounding of e; TwoSum keeps the rounding error of xh + p.  The
// velocity: v + h (a + h j/2) = vh + 2h (a/2 + (3h/2) j/6) in FP32.  F2 is
// float (one coordinate) or float2 (two coordinates in the packed FP32x2
// operations, each lane rounded exactly as the scalar form).
__device__ __forceinline__ float p_add(float a, float b) { return a + b; }
__device__ __forceinline__ float p_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float p_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float p_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float p_neg(float a) { return -a; }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

template <typename F2>
__device__ __forceinline__ void ds_predict(F2 xh, F2 xl, F2 vh, F2 vl, F2 a2, F2 j6, F2 h, F2 h2, F2 h15,
                                           F2& hi, F2& lo, F2& vp) {
  const F2 u = p_fma(h, j6, a2);  // a/2 + h j/6
  const F2 hu = p_mul(h, u);
  F2 s = p_add(vh, hu);  // TwoSum(vh, hu)
  F2 bb = p_sub(s, vh);
  F2 e = p_add(p_sub(vh, p_sub(s, bb)), p_sub(hu, bb));
  e = p_add(e, vl);
  const F2 p = p_mul(h, s);  // h (s + e) = p + q, the product h s exact (FMA)
  F2 q = p_fma(h, s, p_neg(p));
  q = p_fma(h, e, q);
  const F2 S = p_add(xh, p);  // TwoSum(xh, p)
  bb = p_sub(S, xh);
  F2 E = p_add(p_sub(xh, p_sub(S, bb)), p_sub(p, bb));
  E = p_add(E, p_add(xl, q));
  hi = p_add(S, E);  // renormalise: |lo| <= ulp(hi) / 2
  lo = p_sub(E, p_sub(hi, S));
  vp = p_fma(h2, p_fma(h15, j6, a2), vh);
}

// predict the staged tile `buf` into the pair tile; slots past jhi become
// massless particles far away (every float written, so no stale shared
// memory is ever read)
template <int NT, int JT>
__device__ __forceinline__ void jm_predict_tile(FusedSmem<JT>& sm, int buf, double T, int64_t jt, int64_t jhi) {
  const PairTile<JT> pt(sm.A, sm.B, sm.C);
#pragma unroll
  for (int q = threadIdx.x; q < JT; q += NT) {
    const int o = 4 * (q >> 1) + (q & 1);
    float xh[3], xl[3], vv[3], m;
    if (jt + q < jhi) {
      const float4 r0 = sm.R[buf][0][q], r1 = sm.R[buf][1][q], r2 = sm.R[buf][2][q], r3 = sm.R[buf][3][q],
                   r4 = sm.R[buf][4][q];
      const float h = __double2float_rn(T - sm.T[buf][q]);
      const float h2 = 2.0f * h, h15 = 1.5f * h;  // exact scalings of an exact h
      float2 hi2, lo2, vp2;
      ds_predict(make_float2(r0.x, r0.y), make_float2(r1.x, r1.y), make_float2(r2.x, r2.y),
                 make_float2(r3.x, r3.y), make_float2(r4.x, r4.y), make_float2(r2.w, r3.w), make_float2(h, h),
                 make_float2(h2, h2), make_float2(h15, h15), hi2, lo2, vp2);
      ds_predict(r0.z, r1.z, r2.z, r3.z, r4.z, r4.w, h, h2, h15, xh[2], xl[2], vv[2]);
      xh[0] = hi2.x; xh[1] = hi2.y;
      xl[0] = lo2.x; xl[1] = lo2.y;
      vv[0] = vp2.x; vv[1] = vp2.y;
      m = r0.w;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xh[c] = kFarF;
        xl[c] = 0.0f;
        vv[c] = 0.0f;
      }
      m = 0.0f;
    }
    pt.p0[o] = xh[0];
    pt.p0[o + 2] = xh[1];
    pt.p1[o] = xh[2];
    pt.p1[o + 2] = m;
    pt.p2[o] = vv[0];
    pt.p2[o + 2] = vv[1];
    pt.p3[o] = vv[2];
    pt.p3[o + 2] = xl[0];
    pt.p4[o] = xl[1];
    pt.p4[o + 2] = xl[2];
  }
}

template <int JT>
__device__ __forceinline__ PairTile<JT> pair_tile(MixedSmem<JT>& sm, int buf) {
  return PairTile<JT>(sm.A[buf], sm.B[buf], sm.C[buf]);
}
template <int JT>
__device__ __forceinline__ PairTile<JT> pair_tile(FusedSmem<JT>& sm, int) {
  return PairTile<JT>(sm.A, sm.B, sm.C);
}

// One j-tile against the thread's IPT i-particles; FP32 partials in p.
// MODE: kFar  -- the tile is far from every i of the warp: hi parts alone
//                (r = x_j.hi - x_i.hi, within 2^-24 (|x_i|+|x_j|) of the exact
//                difference: relative error <= 2^-24 (1/theta + 1) at the
//                far-test distance);
//       kNear -- double-single difference;
//       kSelf -- double-single difference, pairs with j == i get 1/s = 0.
constexpr int kFar = 0, kNear = 1, kSelf = 2;
// far test: box gap >= theta * (|x|max_i + |x|max_j)
#ifndef NB_FAR_THETA
#define NB_FAR_THETA 0.125f
#endif
constexpr float kFarTheta = NB_FAR_THETA;

template <int IPT, int JT, int MODE>
__device__ __forceinline__ void mixed_tile_pass(const float4* __restrict__ sA, const float4* __restrict__ sB,
                                                const float2* __restrict__ sC, const float (&xh)[IPT][3],
                                                const float (&xl)[IPT][3], const float (&vi)[IPT][3],
                                                const int (&rel)[IPT], float eps2, float (&p)[IPT][7]) {
  NB_PRAGMA_UNROLL(NB_MIXED_UNROLL)
  for (int q = 0; q < JT; ++q) {
    const float4 A = sA[q];
    const float4 B = sB[q];
    const float2 C = sC[q];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const float dx = MODE == kFar ? A.x - xh[k][0] : (A.x - xh[k][0]) + (B.x - xl[k][0]);
      const float dy = MODE == kFar ? A.y - xh[k][1] : (A.y - xh[k][1]) + (B.y - xl[k][1]);
      const float dz = MODE == kFar ? A.z - xh[k][2] : (A.z - xh[k][2]) + (B.z - xl[k][2]);
      const float wx = B.w - vi[k][0];
      const float wy = C.x - vi[k][1];
      const float wz = C.y - vi[k][2];
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
      const float rw = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
#if NB_MIXED_NEWTON
      // hardware 1/sqrt + one Newton step: e = 1 - s^2 y0^2, y = y0 + y0 e / 2
      const float y0 = nb_rsqrt_approx(r2);
      const float e = fmaf(-r2, y0 * y0, 1.0f);
      float rinv = fmaf(0.5f, y0 * e, y0);
#else
      float rinv = nb_rsqrt_approx(r2);
#endif
      if (MODE == kSelf) rinv = (q == rel[k]) ? 0.0f : rinv;
      const float rinv2 = rinv * rinv;
      const float mr = A.w * rinv;
      const float mr3 = mr * rinv2;
      // jerk term formed before accumulation: u = w - 3 (r.w)/s^2 r; the two
      // parts cancel for close pairs, so they must not enter the sum apart
      const float a3 = (rw * -3.0f) * rinv2;
      p[k][6] += mr;
      p[k][0] = fmaf(mr3, dx, p[k][0]);
      p[k][1] = fmaf(mr3, dy, p[k][1]);
      p[k][2] = fmaf(mr3, dz, p[k][2]);
      p[k][3] = fmaf(mr3, fmaf(a3, dx, wx), p[k][3]);
      p[k][4] = fmaf(mr3, fmaf(a3, dy, wy), p[k][4]);
      p[k][5] = fmaf(mr3, fmaf(a3, dz, wz), p[k][5]);
    }
  }
}

// The same pass on the pair layout for IPT i per thread: every FP32
// operation acts on the pair (j, j+1) at once (packed FP32x2 add/mul/fma,
// each lane rounded exactly as its scalar counterpart), which halves the
// issue slots of the FP32 work.  ni* hold the NEGATED i coordinates and
// velocity in both lanes, so x_j + (-x_i) is the scalar x_j - x_i bit for
// bit.  The two lanes of p sum the even and the odd j of the tile.
template <int IPT, int JT, int MODE>
__device__ __forceinline__ void mixed_pair_pass(const PairTile<JT>& t, const float2 (&nxh)[IPT][3],
                                                const float2 (&nxl)[IPT][3], const float2 (&nv)[IPT][3],
                                                const int (&rel)[IPT], float2 eps2, float2 (&p)[IPT][7]) {
  const float4* __restrict__ P0 = (const float4*)t.p0;
  const float4* __restrict__ P1 = (const float4*)t.p1;
  const float4* __restrict__ P2 = (const float4*)t.p2;
  const float4* __restrict__ P3 = (const float4*)t.p3;
  const float4* __restrict__ P4 = (const float4*)t.p4;
  const float2 m3 = make_float2(-3.0f, -3.0f);
  NB_PRAGMA_UNROLL(NB_MIXED_UNROLL)
  for (int u = 0; u < JT / 2; ++u) {
    const float4 a = P0[u], b = P1[u], c = P2[u], d = P3[u];
    float4 e;
    if (MODE != kFar) e = P4[u];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      float2 dx = __fadd2_rn(make_float2(a.x, a.y), nxh[k][0]);
      float2 dy = __fadd2_rn(make_float2(a.z, a.w), nxh[k][1]);
      float2 dz = __fadd2_rn(make_float2(b.x, b.y), nxh[k][2]);
      if (MODE != kFar) {
        dx = __fadd2_rn(dx, __fadd2_rn(make_float2(d.z, d.w), nxl[k][0]));
        dy = __fadd2_rn(dy, __fadd2_rn(make_float2(e.x, e.y), nxl[k][1]));
        dz = __fadd2_rn(dz, __fadd2_rn(make_float2(e.z, e.w), nxl[k][2]));
      }
      const float2 wx = __fadd2_rn(make_float2(c.x, c.y), nv[k][0]);
      const float2 wy = __fadd2_rn(make_float2(c.z, c.w), nv[k][1]);
      const float2 wz = __fadd2_rn(make_float2(d.x, d.y), nv[k][2]);
      const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, eps2)));
      const float2 rw = __ffma2_rn(dz, wz, __ffma2_rn(dy, wy, __fmul2_rn(dx, wx)));
#if NB_MIXED_NEWTON
      const float2 y0 = make_float2(nb_rsqrt_approx(r2.x), nb_rsqrt_approx(r2.y));
      const float2 ee = __ffma2_rn(make_float2(-r2.x, -r2.y), __fmul2_rn(y0, y0), make_float2(1.0f, 1.0f));
      float2 rinv = __ffma2_rn(make_float2(0.5f, 0.5f), __fmul2_rn(y0, ee), y0);
#else
      float2 rinv = make_float2(nb_rsqrt_approx(r2.x), nb_rsqrt_approx(r2.y));
#endif
      if (MODE == kSelf) {
        rinv.x = (2 * u == rel[k]) ? 0.0f : rinv.x;
        rinv.y = (2 * u + 1 == rel[k]) ? 0.0f : rinv.y;
      }
      const float2 rinv2 = __fmul2_rn(rinv, rinv);
      const float2 mr = __fmul2_rn(make_float2(b.z, b.w), rinv);
      const float2 mr3 = __fmul2_rn(mr, rinv2);
      const float2 a3 = __fmul2_rn(__fmul2_rn(rw, m3), rinv2);
      p[k][6] = __fadd2_rn(p[k][6], mr);
      p[k][0] = __ffma2_rn(mr3, dx, p[k][0]);
      p[k][1] = __ffma2_rn(mr3, dy, p[k][1]);
      p[k][2] = __ffma2_rn(mr3, dz, p[k][2]);
      p[k][3] = __ffma2_rn(mr3, __ffma2_rn(a3, dx, wx), p[k][3]);
      p[k][4] = __ffma2_rn(mr3, __ffma2_rn(a3, dy, wy), p[k][4]);
      p[k][5] = __ffma2_rn(mr3, __ffma2_rn(a3, dz, wz), p[k][5]);
    }
  }
}

// (hi, lo) += (bh, bl): double-single sum (Knuth's TwoSum of the high parts,
// the low parts and the rounding error added without renormalisation, as the
// items' per-tile fold)
__device__ __forceinline__ void ds_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  lo = (lo + bl) + ((hi - (s - bb)) + (bh - bb));
  hi = s;
}

// an FP64 value as a double-single pair: hi = fl32(x), lo = fl32(x - hi)
__device__ __forceinline__ float2 ds_split(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

// Mixed-precision item: i-tile starting at list position ibase (n entries in
// list, entries clamped to [0, idx_hi)), j-range [jlo, jhi).  Writes 7 rows
// out[c * ostride + pos] (final: acc, jerk, pot with its sign) or raw sums.
// With FusedSmem the j-tiles come from the j-memory (fa) and are predicted
// to fa.T as they are staged; the i-particles always come from jA/jB/jC.
template <int NT, int IPT, int JT, typename SM>
__device__ __forceinline__ void mixed_item(SM& sm, const float4* __restrict__ jA,
                                           const float4* __restrict__ jB, const float2* __restrict__ jC,
                                           int64_t jlo, int64_t jhi, int64_t idx_hi,
                                           const int32_t* __restrict__ list, int64_t n, int64_t ibase,
                                           float eps2, double* __restrict__ out, int64_t ostride,
                                           bool finalize, const float4* __restrict__ tbox = nullptr,
                                           const int32_t* __restrict__ ord = nullptr, int64_t box_origin = 0,
                                           const FusedArgs fa = FusedArgs(), const ISrc is = ISrc(),
                                           bool ds_out = false) {
  constexpr bool kFusedLoad = SM::kFused;
  // list: j-store slots of the i-particles.  ord (optional): the list
  // positions in processing order (a caller's list visited in spatial
  // order); results always go to the list positions.  tbox (optional):
  // boxes of every NB_BOX_TILE slots from slot box_origin on (j-ranges start
  // at box_origin plus a multiple of JT), which allow the far-tile pass.
  const int tid = threadIdx.x;
  float xh[IPT][3], xl[IPT][3], vi[IPT][3];
  int64_t self[IPT];
#if NB_MIXED_DS_FOLD
  // double-single accumulators: the per-tile FP32 partial is added with
  // Knuth's TwoSum in FP32 (no FP64 instruction in the loop at all)
  float acc_hi[IPT][7], acc_lo[IPT][7];
#elif NB_MIXED_SMEM_ACC
  // FP64 accumulators in shared memory: fewer registers, more resident warps
  __shared__ double s_acc[IPT * 7 * NT];
#define NB_ACC(k, c) s_acc[((k) * 7 + (c)) * NT + tid]
#else
  double acc[IPT][7];
#define NB_ACC(k, c) acc[k][c]
#endif
#if NB_MIXED_DS_FOLD
#define NB_ACC_ZERO(k, c) (acc_hi[k][c] = acc_lo[k][c] = 0.0f)
#define NB_ACC_ADD(k, c, val)                                   \
  do {                                                          \
    const float a_ = acc_hi[k][c], b_ = (val);                  \
    const float s_ = a_ + b_;                                   \
    const float bb_ = s_ - a_;                                  \
    acc_lo[k][c] += (a_ - (s_ - bb_)) + (b_ - bb_);             \
    acc_hi[k][c] = s_;                                          \
  } while (0)
#define NB_ACC_GET(k, c) ((double)acc_hi[k][c] + (double)acc_lo[k][c])
#define NB_ACC_DS(k, c) make_float2(acc_hi[k][c], acc_lo[k][c])
#else
#define NB_ACC_ZERO(k, c) (NB_ACC(k, c) = 0.0)
#define NB_ACC_ADD(k, c, val) (NB_ACC(k, c) += (double)(val))
#define NB_ACC_GET(k, c) NB_ACC(k, c)
#define NB_ACC_DS(k, c) ds_split(NB_ACC(k, c))
#endif
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    int64_t pos = ibase + k * NT + tid;
    if (pos >= n) pos = n - 1;
    if (ord) pos = ord[pos];
    int64_t p = list[pos];
    float4 A, B;
    float2 C;
    if (is.A) {  // a particle held elsewhere: list positions index the i arrays (n long)
      p = p < 0 ? 0 : (p >= n ? n - 1 : p);
      A = is.A[p];
      B = is.B[p];
      C = is.C[p];
      self[k] = is.self ? is.self[pos] : -1;
    } else {
      p = p < 0 ? 0 : (p >= idx_hi ? idx_hi - 1 : p);  // a bad list never reads out of bounds
      self[k] = p;  // j-store slot of this i
      A = jA[p];
      B = jB[p];
      C = jC[p];
    }
    xh[k][0] = A.x; xh[k][1] = A.y; xh[k][2] = A.z;
    xl[k][0] = B.x; xl[k][1] = B.y; xl[k][2] = B.z;
    vi[k][0] = B.w; vi[k][1] = C.x; vi[k][2] = C.y;
#pragma unroll
    for (int c = 0; c < 7; ++c) NB_ACC_ZERO(k, c);
  }
  // box of this thread's i-particles (hi parts) and their largest
  // |coordinate|: the far test is taken per thread and the tile is far for
  // the warp when it is far for every lane (a warp of scattered particles,
  // as a small random block forms, still finds the tiles far from all of them)
  float wlo[3], whi[3], wr = 0.0f;
  if (tbox) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      wlo[c] = xh[0][c];
      whi[c] = xh[0][c];
#pragma unroll
      for (int k = 1; k < IPT; ++k) {
        wlo[c] = fminf(wlo[c], xh[k][c]);
        whi[c] = fmaxf(whi[c], xh[k][c]);
      }
      wr = fmaxf(wr, fmaxf(fabsf(wlo[c]), fabsf(whi[c])));
    }
  }

  // packed loop: each i-particle in both lanes, negated
  constexpr bool kPk = NB_MIXED_PACKED && IPT <= 2;
  static_assert(!kFusedLoad || kPk, "on-the-fly prediction fills the pair layout of the packed loop");
  float2 nxh[IPT][3], nxl[IPT][3], nv[IPT][3];
#pragma unroll
  for (int k = 0; k < IPT; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      nxh[k][c] = make_float2(-xh[k][c], -xh[k][c]);
      nxl[k][c] = make_float2(-xl[k][c], -xl[k][c]);
      nv[k][c] = make_float2(-vi[k][c], -vi[k][c]);
    }

  const int ntiles = (int)((jhi - jlo + JT - 1) / JT);
  if (ntiles > 0) {
    if constexpr (kFusedLoad)
      jm_load_tile<NT, JT>(sm, 0, fa, jlo, jhi);
    else if constexpr (kPk)
      mixed_load_tile_pairs<NT, JT>(sm.A[0], sm.B[0], sm.C[0], jA, jB, jC, jlo, jhi);
    else
      mixed_load_tile<NT, JT>(sm.A[0], sm.B[0], sm.C[0], jA, jB, jC, jlo, jhi);
  }
  cp_async_commit();

  for (int tile = 0; tile < ntiles; ++tile) {
    const int buf = tile & 1;
    const int64_t jt = jlo + (int64_t)tile * JT;
    if (tile + 1 < ntiles) {
      if constexpr (kFusedLoad)
        jm_load_tile<NT, JT>(sm, buf ^ 1, fa, jt + JT, jhi);
      else if constexpr (kPk)
        mixed_load_tile_pairs<NT, JT>(sm.A[buf ^ 1], sm.B[buf ^ 1], sm.C[buf ^ 1], jA, jB, jC, jt + JT, jhi);
      else
        mixed_load_tile<NT, JT>(sm.A[buf ^ 1], sm.B[buf ^ 1], sm.C[buf ^ 1], jA, jB, jC, jt + JT, jhi);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if constexpr (kFusedLoad) {
      // predict the staged tile (ragged tail included) into the pair tile
      jm_predict_tile<NT, JT>(sm, buf, fa.T, jt, jhi);
      __syncthreads();
    } else if (jt + JT > jhi) {  // ragged last tile: massless far-away particles past jhi
      for (int q = tid; q < JT; q += NT) {
        if (jt + q < jhi) continue;
        if constexpr (kPk) {
          const PairTile<JT> pt(sm.A[buf], sm.B[buf], sm.C[buf]);
          const int o = 4 * (q >> 1) + (q & 1);
          pt.p0[o] = kFarF;
          pt.p0[o + 2] = kFarF;
          pt.p1[o] = kFarF;
          pt.p1[o + 2] = 0.0f;
        } else {
          sm.A[buf][q] = make_float4(kFarF, kFarF, kFarF, 0.0f);
        }
      }
      __syncthreads();
    }

    int rel[IPT];
    bool hit = false;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int64_t d = self[k] - jt;
      rel[k] = (d >= 0 && d < JT) ? (int)d : -1;
      hit = hit || rel[k] >= 0;
    }
    float p[IPT][7];
#pragma unroll
    for (int k = 0; k < IPT; ++k)
#pragma unroll
      for (int c = 0; c < 7; ++c) p[k][c] = 0.0f;

    // far test: box gap >= theta (|x|max of the thread's i + |x|max of the
    // tile) bounds the hi-only difference error of each of its pairs by
    // 2^-24 (1/theta + 1); the warp takes the far pass when every lane passes.
    // Boxes cover NB_BOX_TILE slots: a longer tile needs all of its boxes
    // far, a shorter one uses the box that contains it.
    bool far = false;
    if (tbox) {
      constexpr int kBoxes = JT >= NB_BOX_TILE ? JT / NB_BOX_TILE : 1;
      far = true;
#pragma unroll
      for (int b = 0; b < kBoxes; ++b) {
        const int64_t t = (jt - box_origin) / NB_BOX_TILE + b;
        const float4 blo = tbox[2 * t], bhi = tbox[2 * t + 1];
        const float gx = fmaxf(0.0f, fmaxf(blo.x - whi[0], wlo[0] - bhi.x));
        const float gy = fmaxf(0.0f, fmaxf(blo.y - whi[1], wlo[1] - bhi.y));
        const float gz = fmaxf(0.0f, fmaxf(blo.z - whi[2], wlo[2] - bhi.z));
        const float lim = kFarTheta * (wr + blo.w);
        far = far && fmaf(gx, gx, fmaf(gy, gy, gz * gz)) >= lim * lim;
      }
    }
    if constexpr (kPk) {
      const PairTile<JT> pt = pair_tile(sm, buf);
      const float2 e2 = make_float2(eps2, eps2);
      float2 p2[IPT][7];
#pragma unroll
      for (int k = 0; k < IPT; ++k)
#pragma unroll
        for (int c = 0; c < 7; ++c) p2[k][c] = make_float2(0.0f, 0.0f);
      if (__any_sync(0xffffffffu, hit))
        mixed_pair_pass<IPT, JT, kSelf>(pt, nxh, nxl, nv, rel, e2, p2);
      else if (__all_sync(0xffffffffu, far))
        mixed_pair_pass<IPT, JT, kFar>(pt, nxh, nxl, nv, rel, e2, p2);
      else
        mixed_pair_pass<IPT, JT, kNear>(pt, nxh, nxl, nv, rel, e2, p2);
#pragma unroll
      for (int k = 0; k < IPT; ++k)
#pragma unroll
        for (int c = 0; c < 7; ++c) p[k][c] = p2[k][c].x + p2[k][c].y;
    } else {
      if (__any_sync(0xffffffffu, hit))
        mixed_tile_pass<IPT, JT, kSelf>(sm.A[buf], sm.B[buf], sm.C[buf], xh, xl, vi, rel, eps2, p);
      else if (__all_sync(0xffffffffu, far))
        mixed_tile_pass<IPT, JT, kFar>(sm.A[buf], sm.B[buf], sm.C[buf], xh, xl, vi, rel, eps2, p);
      else
        mixed_tile_pass<IPT, JT, kNear>(sm.A[buf], sm.B[buf], sm.C[buf], xh, xl, vi, rel, eps2, p);
    }

#pragma unroll
    for (int k = 0; k < IPT; ++k)
#pragma unroll
      for (int c = 0; c < 7; ++c) NB_ACC_ADD(k, c, p[k][c]);
    __syncthreads();
  }
  cp_async_wait<0>();

  // final results (one split): FP64 with the potential's sign; partial sums
  // of a split: FP64, or with ds_out the double-single pair (hi, lo) in the
  // same 8-byte slot (no FP64 instruction: the FP64 pipe issues a warp
  // instruction every 64 cycles per warp on this GPU), which the split
  // reduction sums in FP32 (split_reduce_ds)
  float2* out2 = reinterpret_cast<float2*>(out);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    int64_t pos = ibase + k * NT + tid;
    if (pos >= n) continue;
    if (ord) pos = ord[pos];
    if (ds_out && !finalize) {
#pragma unroll
      for (int c = 0; c < 7; ++c) out2[c * ostride + pos] = NB_ACC_DS(k, c);
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) out[c * ostride + pos] = NB_ACC_GET(k, c);
      out[6 * ostride + pos] = finalize ? -NB_ACC_GET(k, 6) : NB_ACC_GET(k, 6);
    }
  }
#undef NB_ACC
#undef NB_ACC_ZERO
#undef NB_ACC_ADD
#undef NB_ACC_GET
#undef NB_ACC_DS
}

template <int JT>
struct Fp64Smem {
  double x[3][JT], v[3][JT], m[JT];
};

// FP64 item: one i per thread (i-tile of NT), j-range [jlo, jhi) with a
// ragged tail filled by massless far-away particles.  xp, vp are SoA rows of
// stride n_pad.
template <int NT, int JT>
__device__ __forceinline__ void fp64_item(Fp64Smem<JT>& sm, const double* __restrict__ xp,
                                          const double* __restrict__ vp, const double* __restrict__ m,
                                          int64_t n_pad, int64_t jlo, int64_t jhi,
                                          const int32_t* __restrict__ list, int64_t n, int64_t ibase,
                                          double eps2, double* __restrict__ out, int64_t ostride,
                                          bool finalize, const ISrc is = ISrc()) {
  const int tid = threadIdx.x;
  const int64_t pos0 = ibase + tid;
  const int64_t pos = pos0 < n ? pos0 : n - 1;
  int64_t self = list[pos];
  double xi[3], vi[3];
  if (is.x) {  // a particle held elsewhere (see ISrc)
    self = self < 0 ? 0 : (self >= n ? n - 1 : self);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xi[c] = is.x[c * is.stride + self];
      vi[c] = is.v[c * is.stride + self];
    }
    self = is.self ? is.self[pos] : -1;
  } else {
    self = self < 0 ? 0 : (self >= n_pad ? n_pad - 1 : self);  // a bad list never reads out of bounds
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xi[c] = xp[c * n_pad + self];
      vi[c] = vp[c * n_pad + self];
    }
  }
  double hi[7], lo[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) hi[c] = lo[c] = 0.0;
  // a warp whose list positions all lie past n computes nothing (its
  // results are not written); it still loads its share of every j-tile
  const bool wact = ibase + (int64_t)(tid & ~31) < n;

  for (int64_t jt = jlo; jt < jhi; jt += JT) {
    __syncthreads();
    for (int q = tid; q < JT; q += NT) {
      const int64_t j = jt + q;
      if (j < jhi) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sm.x[c][q] = xp[c * n_pad + j];
          sm.v[c][q] = vp[c * n_pad + j];
        }
        sm.m[q] = m[j];
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sm.x[c][q] = (double)kFarF;
          sm.v[c][q] = 0.0;
        }
        sm.m[q] = 0.0;
      }
    }
    __syncthreads();
    if (!wact) continue;  // the next tile's leading barrier keeps the warp in step
    double p[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) p[c] = 0.0;
#pragma unroll 2
    for (int q = 0; q < JT; ++q) {
      const double dx = sm.x[0][q] - xi[0], dy = sm.x[1][q] - xi[1], dz = sm.x[2][q] - xi[2];
      const double wx = sm.v[0][q] - vi[0], wy = sm.v[1][q] - vi[1], wz = sm.v[2][q] - vi[2];
      const double r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
      const double rw = fma(dz, wz, fma(dy, wy, dx * wx));
      // the self pair (j == i) gets 1/s = 0, also when eps = 0
      const double rinv = (jt + q == self) ? 0.0 : nb_rsqrt_fp64(r2);
      const double rinv2 = rinv * rinv;
      const double mr = sm.m[q] * rinv;
      const double mr3 = mr * rinv2;
      const double a3 = (rw * -3.0) * rinv2;  // jerk term formed before accumulation
      p[6] += mr;
      p[0] = fma(mr3, dx, p[0]);
      p[1] = fma(mr3, dy, p[1]);
      p[2] = fma(mr3, dz, p[2]);
      p[3] = fma(mr3, fma(a3, dx, wx), p[3]);
      p[4] = fma(mr3, fma(a3, dy, wy), p[4]);
      p[5] = fma(mr3, fma(a3, dz, wz), p[5]);
    }
    // TwoSum fold (Knuth): hi + p = s + e exactly
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      const double s = hi[c] + p[c];
      const double bp = s - hi[c];
      const double e = (hi[c] - (s - bp)) + (p[c] - bp);
      hi[c] = s;
      lo[c] += e;
    }
  }
  __syncthreads();  // the caller may reuse shared memory for its next item
  if (pos0 >= n) return;
#pragma unroll
  for (int c = 0; c < 6; ++c) out[c * ostride + pos0] = hi[c] + lo[c];
  out[6 * ostride + pos0] = finalize ? -(hi[6] + lo[6]) : hi[6] + lo[6];
}

}  // namespace nbk
