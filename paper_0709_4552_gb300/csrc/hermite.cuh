// hermite.cuh -- per-particle arithmetic of the 4th-order Hermite block-step
// scheme, shared by every loop driver (the host-driven kernels, the body of
// the CUDA-graph loop and the persistent loop): the predictor of Sec. 4.1
// step 3 and the corrector with the power-of-two block-step rule of step 5
// (block steps of Sec. 2).  One definition, so every driver takes the same
// steps bit for bit.
#pragma once

#include <math.h>

#include "nb_internal.cuh"

namespace nbh {

// largest power of two <= x for positive finite x (clears the mantissa)
__device__ __forceinline__ double pow2_floor(double x) {
  if (!(x > 0.0)) return 0.0;
  if (isinf(x)) return x;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if ((b >> 52) == 0) return 0.0;  // subnormal: below any admissible step
  return __longlong_as_double((long long)(b & 0xFFF0000000000000ULL));
}

// y / x.  When x is a positive power of two (every block step, and h = t - t_i
// of every active particle) the quotient is y times 2^-k formed from the
// exponent bits: the same correctly rounded result without an FP64 divide
// (the FP64 pipe bounds the corrector).  Anything else takes the division.
__device__ __forceinline__ double div_pow2(double y, double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long e = b >> 52;  // sign 0 and biased exponent
  if ((b & 0x000FFFFFFFFFFFFFULL) == 0 && e >= 1 && e <= 2045)
    return y * __longlong_as_double((long long)((2046ULL - e) << 52));
  return y / x;
}

__device__ __forceinline__ double clamp_dt(double c, double dt_min, double dt_max) {
  if (c > dt_max) c = dt_max;
  if (c < dt_min) c = dt_min;
  return c;
}

// ---- exact integer forms of FP64 operations with exact results -------------
// On this GPU a warp's FP64 instruction occupies it for about 64 cycles, and
// the corrector's chain is the critical path of a small block step.  Where an
// FP64 operation's result is exact -- a power of two raised to a power, a
// constant scaled by a power of two, the power-of-two floor of a correctly
// rounded square root, comparisons -- it is formed from the exponent bits
// instead: the same bits, no FP64 instruction.  Outside the stated
// preconditions the FP64 expression is taken.

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// x a positive normal power of two: its exponent in e
__device__ __forceinline__ bool is_pow2(double x, int& e) {
  const unsigned long long b = dbits(x);
  const unsigned long long E = b >> 52;  // sign bit 0 and biased exponent
  e = (int)E - 1023;
  return (b & 0x000FFFFFFFFFFFFFULL) == 0 && E >= 1 && E <= 2046;
}

// 2^e, e in [-1022, 1023]
__device__ __forceinline__ double pow2i(int e) {
  return __longlong_as_double((long long)((unsigned long long)(e + 1023) << 52));
}

// c 2^k for a positive normal c whose scaled exponent stays normal (the
// callers' ranges guarantee it): exact, so equal to the FP64 product
__device__ __forceinline__ double scale_pow2(double c, int k) {
  return __longlong_as_double((long long)(dbits(c) + ((unsigned long long)(long long)k << 52)));
}

// powers of the step h = t - t_i and the constant multiples the corrector
// uses: from the exponent when h is a power of two 2^e with |e| <= 200 (every
// block step; all results normal), else by FP64 products
struct HPow {
  double ih, ih2, ih3, h2, h3, h4, h5;
  double h3_6, h4_24, h5_120, h6;  // h^3/6, h^4/24, h^5/120, 6h
  int e;                           // h = 2^e when pow2
  bool pow2;
};

// y 2^k, exact: from the exponent bits when y is finite and normal and the
// result stays normal, else the FP64 product y p2 with p2 = 2^k (the same
// value; infinities and NaNs take the product)
__device__ __forceinline__ double mul_pow2(double y, int k, double p2) {
  const unsigned long long b = dbits(y);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E >= 1 && E <= 2046 && E + k >= 1 && E + k <= 2046)  // y finite and normal, so is the result
    return __longlong_as_double((long long)(b + ((unsigned long long)(long long)k << 52)));
  return y * p2;
}

// y / h^2 and y / h^3 of the corrector (products by the exact inverse powers)
__device__ __forceinline__ double div_h2(const struct HPow& q, double y) {
  return q.pow2 ? mul_pow2(y, -2 * q.e, q.ih2) : y * q.ih2;
}
__device__ __forceinline__ double div_h3(const struct HPow& q, double y) {
  return q.pow2 ? mul_pow2(y, -3 * q.e, q.ih3) : y * q.ih3;
}
// the FP64 products (the reference of the exponent form, and its fallback)
__device__ __forceinline__ HPow h_powers_fp64(double h) {
  HPow q;
  q.ih = div_pow2(1.0, h);
  q.ih2 = q.ih * q.ih;
  q.ih3 = q.ih2 * q.ih;
  q.h2 = h * h;
  q.h3 = q.h2 * h;
  q.h4 = q.h3 * h;
  q.h5 = q.h4 * h;
  q.h3_6 = q.h3 * (1.0 / 6.0);
  q.h4_24 = q.h4 * (1.0 / 24.0);
  q.h5_120 = q.h5 * (1.0 / 120.0);
  q.h6 = 6.0 * h;
  q.e = 0;
  q.pow2 = false;
  return q;
}

__device__ __forceinline__ HPow h_powers(double h) {
  HPow q;
  int e;
  if (is_pow2(h, e) && e >= -200 && e <= 200) {
    q.e = e;
    q.pow2 = true;
    q.ih = pow2i(-e);
    q.ih2 = pow2i(-2 * e);
    q.ih3 = pow2i(-3 * e);
    q.h2 = pow2i(2 * e);
    q.h3 = pow2i(3 * e);
    q.h4 = pow2i(4 * e);
    q.h5 = pow2i(5 * e);
    q.h3_6 = scale_pow2(1.0 / 6.0, 3 * e);
    q.h4_24 = scale_pow2(1.0 / 24.0, 4 * e);
    q.h5_120 = scale_pow2(1.0 / 120.0, 5 * e);
    q.h6 = scale_pow2(6.0, e);
    return q;
  }
  return h_powers_fp64(h);
}

// t (>= 0) an integer multiple of 2^s: 1 yes, 0 no, -1 undecided here
// (negative, subnormal or non-finite t, or t 2^-s below the normal range)
__device__ __forceinline__ int multiple_of_pow2(double t, int s) {
  const unsigned long long b = dbits(t);
  if (b == 0) return 1;
  const unsigned long long E = b >> 52;
  if (E == 0 || E >= 2047) return -1;
  const int d = (int)E - 1023 - s;  // t 2^-s = 1.f 2^d
  if (d < -1000) return -1;
  if (d < 0) return 0;
  if (d >= 52) return 1;
  return (b & ((1ULL << (52 - d)) - 1ULL)) == 0 ? 1 : 0;
}

// The new step (Sec. 4.1 step 5; block steps of Sec. 2) of a particle at time
// t with step dt_old, from num = na n2 + nj^2 and den = nj n3 + n2^2 (na =
// |a1|, nj = |j1|, n2 = |a2 + a3 h|, n3 = |a3|): Aarseth criterion
// crit = sqrt(eta num / den), its power-of-two floor clamped to [dt_min,
// dt_max]; the step shrinks to that freely and doubles only when t is a
// multiple of the doubled step (and the doubled step is admissible).  Counts
// criteria below dt_min; crit_nan reports a NaN criterion.  This is the FP64
// expression: the reference of new_step_nd's exponent form and its fallback.
__device__ __forceinline__ double new_step_fp64(double t, double dt_old, double num, double den, double eta,
                                                double dt_min, double dt_max, nb_dev_status* st, bool& crit_nan) {
  const double crit = (den == 0.0) ? (double)INFINITY : sqrt(eta * num / den);
  if (crit < dt_min) atomicAdd(&st->dt_underflows, 1ULL);
  crit_nan = isnan(crit);
  const double c = clamp_dt(pow2_floor(crit), dt_min, dt_max);
  if (c < dt_old) return c;
  const double two = 2.0 * dt_old;
  const double qq = div_pow2(t, two);  // exact: two is a power of two
  return (c >= two && two <= dt_max && qq == floor(qq)) ? two : dt_old;
}

// new_step_fp64's result from exponents.  For positive normal N = fl(eta num)
// and D = den, fl(N / D) has exponent e_N - e_D, less one when N's
// significand is below D's (a quotient of 53-bit significands never rounds up
// to a power of two), and the power-of-two floor of the correctly rounded
// square root of q = fl(N / D) is 2^floor(e_q / 2) (the square root never
// rounds up to a power of two either); crit < dt_min = 2^m exactly when
// e_q < 2m.  So no division or square root is needed; they are taken (the
// FP64 expression) only when an operand is zero, subnormal or non-finite, a
// step bound or dt_old is not a power of two, or t is negative or subnormal.
__device__ __forceinline__ double new_step_nd(double t, double dt_old, double num, double den, double eta,
                                              double dt_min, double dt_max, nb_dev_status* st, bool& crit_nan) {
  crit_nan = false;
  int emin, emax, eo;
  if (den != 0.0 && is_pow2(dt_min, emin) && is_pow2(dt_max, emax) && is_pow2(dt_old, eo) && emin <= emax) {
    const double nq = eta * num;
    const unsigned long long bN = dbits(nq), bD = dbits(den);
    const unsigned long long EN = bN >> 52, ED = bD >> 52;  // sign bits 0 for positive operands
    if (EN >= 1 && EN <= 2046 && ED >= 1 && ED <= 2046) {
      const int eq = (int)EN - (int)ED - ((bN & 0x000FFFFFFFFFFFFFULL) < (bD & 0x000FFFFFFFFFFFFFULL) ? 1 : 0);
      const int s = eo + 1;  // the doubled step 2^s
      const int mt = eq >= -1022 && eq <= 1023 ? multiple_of_pow2(t, s) : -1;
      if (mt >= 0) {
        if (eq < 2 * emin) atomicAdd(&st->dt_underflows, 1ULL);  // crit < dt_min
        int ec = (eq - (eq & 1)) / 2;  // floor(eq / 2): exponent of the criterion's floor
        if (ec > emax) ec = emax;
        if (ec < emin) ec = emin;
        if (ec < eo) return pow2i(ec);
        return (ec >= s && s <= emax && mt == 1) ? pow2i(s) : dt_old;
      }
    }
  }
  return new_step_fp64(t, dt_old, num, den, eta, dt_min, dt_max, st, crit_nan);
}

// the step from the four norms' roots
__device__ __forceinline__ double new_step(double t, double dt_old, double na, double nj, double n2, double n3,
                                           double eta, double dt_min, double dt_max, nb_dev_status* st,
                                           bool& crit_nan) {
  const double num = na * n2 + nj * nj;
  const double den = nj * n3 + n2 * n2;
  return new_step_nd(t, dt_old, num, den, eta, dt_min, dt_max, st, crit_nan);
}

// Predictor (Sec. 4.1 step 3) of row i over h = t - t_i, Horner form:
//   xp = x + v h + a h^2/2 + jk h^3/6,   vp = v + a h + jk h^2/2
__device__ __forceinline__ void taylor(int64_t i, int64_t n_pad, double h, const double* __restrict__ x,
                                       const double* __restrict__ v, const double* __restrict__ a,
                                       const double* __restrict__ jk, double (&px)[3], double (&pv)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t q = d * n_pad + i;
    const double xv = x[q], vv = v[q], av = a[q], jv = jk[q];
    px[d] = xv + h * (vv + h * (0.5 * av + h * (jv * (1.0 / 6.0))));
    pv[d] = vv + h * (av + h * (0.5 * jv));
  }
}

// the predicted row in the FP64 j-store and/or the mixed one; the
// double-single split of a position is exact: hi = fl32(xp), lo = fl32(xp - hi)
__device__ __forceinline__ void store_predicted(int64_t i, int64_t n_pad, const double (&px)[3],
                                                const double (&pv)[3], double mi, double* __restrict__ xp,
                                                double* __restrict__ vp, float4* __restrict__ jA,
                                                float4* __restrict__ jB, float2* __restrict__ jC,
                                                bool write_fp64, bool write_mixed) {
  if (write_fp64) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xp[d * n_pad + i] = px[d];
      vp[d * n_pad + i] = pv[d];
    }
  }
  if (write_mixed) {
    float hi[3], lo[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      hi[d] = __double2float_rn(px[d]);
      lo[d] = __double2float_rn(px[d] - (double)hi[d]);
    }
    jA[i] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(mi));
    jB[i] = make_float4(lo[0], lo[1], lo[2], __double2float_rn(pv[0]));
    jC[i] = make_float2(__double2float_rn(pv[1]), __double2float_rn(pv[2]));
  }
}

// Corrector (Sec. 4.1 step 5) of row i at block time t from its new force
// f = (a1[3], j1[3], pot1), h = t - t_i.  Hermite interpolation of the
// acceleration through (a0, j0) and (a1, j1) gives at the start
//   a2 = [-6 (a0 - a1) - h (4 j0 + 2 j1)] / h^2,  a3 = [12 (a0 - a1) + 6 h (j0 + j1)] / h^3,
// and x1 = xp + a2 h^4/24 + a3 h^5/120,  v1 = vp + a2 h^3/6 + a3 h^4/24.
// New step: Aarseth criterion at the end of the step (a2e = a2 + a3 h),
// largest power of two below it within [dt_min, dt_max]; it may shrink
// freely and doubles only when t is a multiple of the doubled step.
// Returns the row's next due time t + dt_new.
__device__ __forceinline__ double correct_row(int64_t i, int64_t n_pad, double t, const double (&f)[7], double eta,
                                            double dt_min, double dt_max, double* __restrict__ x,
                                            double* __restrict__ v, double* __restrict__ a,
                                            double* __restrict__ jk, double* __restrict__ pot,
                                            double* __restrict__ ti, double* __restrict__ dt,
                                            const double* __restrict__ xp, const double* __restrict__ vp,
                                            nb_dev_status* __restrict__ st) {
  const double h = t - ti[i];
  const HPow hp = h_powers(h);
  double na2 = 0, nj2 = 0, n22 = 0, n32 = 0;
  bool finite = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t q = c * n_pad + i;
    const double a0 = a[q], j0 = jk[q];
    const double a1 = f[c], j1 = f[3 + c];
    const double da = a0 - a1;
    const double a2 = div_h2(hp, -6.0 * da - h * (4.0 * j0 + 2.0 * j1));
    const double a3 = div_h3(hp, 12.0 * da + hp.h6 * (j0 + j1));
    const double x1 = xp[q] + a2 * hp.h4_24 + a3 * hp.h5_120;
    const double v1 = vp[q] + a2 * hp.h3_6 + a3 * hp.h4_24;
    const double a2e = a2 + a3 * h;
    x[q] = x1;
    v[q] = v1;
    a[q] = a1;
    jk[q] = j1;
    na2 += a1 * a1;
    nj2 += j1 * j1;
    n22 += a2e * a2e;
    n32 += a3 * a3;
    finite = finite && isfinite(x1) && isfinite(v1) && isfinite(a1) && isfinite(j1);
  }
  const double p1 = f[6];
  pot[i] = p1;
  const double na = sqrt(na2), nj = sqrt(nj2), n2 = sqrt(n22), n3 = sqrt(n32);
  bool crit_nan;
  const double dnew = new_step(t, dt[i], na, nj, n2, n3, eta, dt_min, dt_max, st, crit_nan);
  if (!finite || !isfinite(p1) || crit_nan) atomicOr(&st->flags, NB_ST_NUMERIC);
  ti[i] = t;
  dt[i] = dnew;
  return t + dnew;
}

// Inputs of one lane's part of a correction: the row's time and step before
// it, and component `sub` (< 3; lane 3 takes component 0) of the old
// acceleration and jerk and of the predicted position and velocity.
struct CorrIn {
  double t0, dt0, a0, j0, xp, vp;
};

// The same correction spread over four lanes of a warp: lane `sub` < 3 of
// the group takes component `sub` (the same FP64 operations in the same order
// as correct_row), the squared norms are gathered by shuffles and summed in
// component order on every lane, lanes 0-3 take one square root each, and
// lane 0 applies the step rule.  The result is correct_row's, bit for bit;
// the dependent FP64 chain is about a third as long, which matters where one
// particle's correction is the critical path of a block step.
//
// Every lane of the warp must call this with the same control flow: the
// shuffles use the full mask and are taken unconditionally.  `base` is the
// warp lane of the group's lane 0; `write` says whether this group's row is
// real (lanes of groups without a row, and lanes sub >= 4, compute on a
// valid row and write nothing).  With jm the corrected row's j-memory record
// is written as well (write_jm_record's values; its mass word is left as it
// is): each lane its component, lane 0 the reach once the new step is known.
// Returns, on the group's lane 0 of a real row, the row's next due time
// t + dt_new (0 elsewhere).
__device__ __forceinline__ double correct_lanes4(int64_t i, int64_t n_pad, double t, const double (&f)[7],
                                                 const CorrIn& in, double eta, double dt_min, double dt_max,
                                                 double* __restrict__ x, double* __restrict__ v,
                                                 double* __restrict__ a, double* __restrict__ jk,
                                                 double* __restrict__ pot, double* __restrict__ ti,
                                                 double* __restrict__ dt, nb_dev_status* __restrict__ st, int sub,
                                                 int base, bool write, float4* __restrict__ jm = nullptr) {
  const double h = t - in.t0;
  const HPow hp = h_powers(h);
  double sq[4] = {0.0, 0.0, 0.0, 0.0};  // a1^2, j1^2, a2e^2, a3^2 of this lane's component
  double ab[3];                         // |v1|, |a1|, |j1| of this lane's component (the record's reach)
  int fin = 1;
  const int c = sub < 3 ? sub : 0;
  {
    const int64_t q = c * n_pad + i;
    const double a0 = in.a0, j0 = in.j0;
    // (selects, not an index: f stays in registers)
    const double a1 = c == 0 ? f[0] : (c == 1 ? f[1] : f[2]);
    const double j1 = c == 0 ? f[3] : (c == 1 ? f[4] : f[5]);
    const double da = a0 - a1;
    const double a2 = div_h2(hp, -6.0 * da - h * (4.0 * j0 + 2.0 * j1));
    const double a3 = div_h3(hp, 12.0 * da + hp.h6 * (j0 + j1));
    const double x1 = in.xp + a2 * hp.h4_24 + a3 * hp.h5_120;
    const double v1 = in.vp + a2 * hp.h3_6 + a3 * hp.h4_24;
    const double a2e = a2 + a3 * h;
    if (write && sub < 3) {
      x[q] = x1;
      v[q] = v1;
      a[q] = a1;
      jk[q] = j1;
      if (jm) {
        float* r = reinterpret_cast<float*>(jm + i);
        const float xh = __double2float_rn(x1), vh = __double2float_rn(v1);
        r[c] = xh;
        r[4 * n_pad + c] = __double2float_rn(x1 - (double)xh);
        r[8 * n_pad + c] = vh;
        r[12 * n_pad + c] = __double2float_rn(v1 - (double)vh);
        r[16 * n_pad + c] = __double2float_rn(0.5 * a1);
        r[4 * n_pad * (2 + c) + 3] = __double2float_rn(j1 * (1.0 / 6.0));
      }
    }
    sq[0] = a1 * a1;
    sq[1] = j1 * j1;
    sq[2] = a2e * a2e;
    sq[3] = a3 * a3;
    ab[0] = fabs(v1);
    ab[1] = fabs(a1);
    ab[2] = fabs(j1);
    fin = (isfinite(x1) && isfinite(v1) && isfinite(a1) && isfinite(j1)) ? 1 : 0;
  }
  // lane sub (< 4) sums squared norm `sub` in component order (0 + x^2 +
  // y^2 + z^2, as correct_row's running sums): three FP64 adds per lane
  // instead of all four norms on every lane; every shuffle is taken by every lane
  double own[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double t0 = __shfl_sync(0xffffffffu, sq[0], base + k);
    const double t1 = __shfl_sync(0xffffffffu, sq[1], base + k);
    const double t2 = __shfl_sync(0xffffffffu, sq[2], base + k);
    const double t3 = __shfl_sync(0xffffffffu, sq[3], base + k);
    own[k] = sub == 1 ? t1 : (sub == 2 ? t2 : (sub == 3 ? t3 : t0));
  }
  const double mine = ((0.0 + own[0]) + own[1]) + own[2];
  double sum_ab[3] = {0.0, 0.0, 0.0};  // write_jm_record's sums of |v|, |a|, |j| in component order
  if (jm) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double s0 = __shfl_sync(0xffffffffu, ab[r], base);
      const double s1 = __shfl_sync(0xffffffffu, ab[r], base + 1);
      const double s2 = __shfl_sync(0xffffffffu, ab[r], base + 2);
      sum_ab[r] = ((0.0 + s0) + s1) + s2;
    }
  }
  const int f0 = __shfl_sync(0xffffffffu, fin, base);
  const int f1 = __shfl_sync(0xffffffffu, fin, base + 1);
  const int f2 = __shfl_sync(0xffffffffu, fin, base + 2);
  // one square root per lane, gathered on lane 0
  const double root = sqrt(mine);
  const double na = __shfl_sync(0xffffffffu, root, base);
  const double nj = __shfl_sync(0xffffffffu, root, base + 1);
  const double n2 = __shfl_sync(0xffffffffu, root, base + 2);
  const double n3 = __shfl_sync(0xffffffffu, root, base + 3);
  if (!write || sub != 0) return 0.0;
  const double p1 = f[6];
  pot[i] = p1;
  bool crit_nan;
  const double dnew = new_step(t, in.dt0, na, nj, n2, n3, eta, dt_min, dt_max, st, crit_nan);
  const bool finite = f0 && f1 && f2;
  if (!finite || !isfinite(p1) || crit_nan) atomicOr(&st->flags, NB_ST_NUMERIC);
  ti[i] = t;
  dt[i] = dnew;
  if (jm) {
    const double d = dnew;
    const double rr = d * (sum_ab[0] + d * (0.5 * sum_ab[1] + d * (sum_ab[2] * (1.0 / 6.0))));
    reinterpret_cast<float*>(jm + n_pad + i)[3] = __double2float_ru(rr * (1.0 + 0x1p-20));
  }
  return t + dnew;
}

// correct_lanes4 with its inputs read from the state and the predicted rows
__device__ __forceinline__ double correct_row_lanes4(int64_t i, int64_t n_pad, double t, const double (&f)[7],
                                                   double eta, double dt_min, double dt_max, double* __restrict__ x,
                                                   double* __restrict__ v, double* __restrict__ a,
                                                   double* __restrict__ jk, double* __restrict__ pot,
                                                   double* __restrict__ ti, double* __restrict__ dt,
                                                   const double* __restrict__ xp, const double* __restrict__ vp,
                                                   nb_dev_status* __restrict__ st, int sub, int base, bool write) {
  const int64_t q = (sub < 3 ? sub : 0) * n_pad + i;
  const CorrIn in{ti[i], dt[i], a[q], jk[q], xp[q], vp[q]};
  return correct_lanes4(i, n_pad, t, f, in, eta, dt_min, dt_max, x, v, a, jk, pot, ti, dt, st, sub, base, write);
}

// j-memory record of row i (the on-the-fly j prediction's input, Sec. 4.4
// step 4; layout in force_common.cuh): double-single position and velocity,
// a/2 and jerk/6 in FP32, the mass, and the reach Rd >= |v_c| dt + |a_c| dt^2/2
// + |j_c| dt^3/6 summed over components (a bound on every coordinate's move
// within the row's current step), rounded up.  Rows >= N: padding.
__device__ __forceinline__ void write_jm_record(int64_t i, int64_t N, int64_t n_pad, const double* __restrict__ m,
                                                const double* __restrict__ x, const double* __restrict__ v,
                                                const double* __restrict__ a, const double* __restrict__ jk,
                                                const double* __restrict__ dt, float4* __restrict__ jm) {
  float xh[3], xl[3], vh[3], vl[3], a2[3], j6[3], mf = 0.0f, reach = 0.0f;
  if (i < N) {
    double sv = 0.0, sa = 0.0, sj = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t q = c * n_pad + i;
      const double xv = x[q], vv = v[q], av = a[q], jv = jk[q];
      xh[c] = __double2float_rn(xv);
      xl[c] = __double2float_rn(xv - (double)xh[c]);
      vh[c] = __double2float_rn(vv);
      vl[c] = __double2float_rn(vv - (double)vh[c]);
      a2[c] = __double2float_rn(0.5 * av);
      j6[c] = __double2float_rn(jv * (1.0 / 6.0));
      sv += fabs(vv);
      sa += fabs(av);
      sj += fabs(jv);
    }
    const double d = dt[i];
    const double r = d * (sv + d * (0.5 * sa + d * (sj * (1.0 / 6.0))));
    reach = __double2float_ru(r * (1.0 + 0x1p-20));
    mf = __double2float_rn(m[i]);
  } else {  // padding row: massless and far away
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xh[c] = (float)NB_PAD_POS;
      xl[c] = vh[c] = vl[c] = a2[c] = j6[c] = 0.0f;
    }
  }
  jm[i] = make_float4(xh[0], xh[1], xh[2], mf);
  jm[n_pad + i] = make_float4(xl[0], xl[1], xl[2], reach);
  jm[2 * n_pad + i] = make_float4(vh[0], vh[1], vh[2], j6[0]);
  jm[3 * n_pad + i] = make_float4(vl[0], vl[1], vl[2], j6[1]);
  jm[4 * n_pad + i] = make_float4(a2[0], a2[1], a2[2], j6[2]);
}

}  // namespace nbh
