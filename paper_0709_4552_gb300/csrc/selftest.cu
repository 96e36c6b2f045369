// selftest.cu -- device self-check of the corrector's exponent forms
// (hermite.cuh: h_powers, mul_pow2, new_step_nd) against their FP64
// expressions (h_powers_fp64, the product by 2^k, new_step_fp64) on seeded
// random operands, bit for bit.
// The operands cover the block-step regime and its edges: powers of two and
// other steps, significands of N = eta num and den equal or one unit apart
// (quotients at a power-of-two boundary), zero, subnormal, infinite and NaN
// norms, times that are and are not multiples of the doubled step.
#include <stdint.h>
#include <string.h>

#include "hermite.cuh"
#include "nb_internal.cuh"

namespace {

// SplitMix64 (Steele, Lea and Flood 2014): a counter-based 64-bit generator
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double from_bits(uint64_t b) { return __longlong_as_double((long long)b); }

// a positive double with biased exponent E and the given 52 fraction bits
__device__ __forceinline__ double make_pos(int E, uint64_t frac) {
  return from_bits(((uint64_t)E << 52) | (frac & 0x000FFFFFFFFFFFFFULL));
}

// a norm-like operand: mostly positive normal over a wide exponent range,
// sometimes zero, subnormal, infinite or NaN
__device__ double random_norm(uint64_t r, uint64_t r2) {
  switch (r & 63) {
    case 0: return 0.0;
    case 1: return make_pos(0, r2 | 1);                  // subnormal
    case 2: return (double)INFINITY;
    case 3: return (double)NAN;
    default: return make_pos(1023 - 80 + (int)((r >> 8) % 160), r2);
  }
}

__global__ void selftest_kernel(int64_t samples, uint64_t seed, unsigned long long* bad, nb_dev_status* st_fast,
                                nb_dev_status* st_ref) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < samples;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r0 = mix64(seed ^ (uint64_t)k * 0xD1B54A32D192ED03ULL);
    const uint64_t r1 = mix64(r0), r2 = mix64(r1), r3 = mix64(r2), r4 = mix64(r3), r5 = mix64(r4);
    // powers of a step: a power of two 2^e (e in [-215, 215], beyond the
    // exponent form's range at both ends) or a general step
    {
      const int e = -215 + (int)(r0 % 431);
      const double h = (r1 & 7) == 0 ? make_pos(1023 + (int)((r1 >> 8) % 40) - 30, r2) : nbh::pow2i(e);
      const nbh::HPow a = nbh::h_powers(h), b = nbh::h_powers_fp64(h);
      const double* pa = &a.ih;
      const double* pb = &b.ih;
      for (int q = 0; q < 11; ++q)
        if (nbh::dbits(pa[q]) != nbh::dbits(pb[q])) atomicAdd(bad, 1ULL);
    }
    // exact power-of-two scaling: y 2^k from the exponent bits against the
    // FP64 product (y normal, subnormal, zero, infinite or NaN; results that
    // stay normal, leave the normal range or overflow)
    {
      const int k = -600 + (int)((r2 >> 20) % 1201);
      const double y = (r3 & 3) == 0 ? random_norm(r4, r5) : make_pos(1 + (int)((r4 >> 8) % 2046), r5);
      const double ys = (r1 >> 63) ? -y : y;
      if (nbh::dbits(nbh::mul_pow2(ys, k, nbh::pow2i(k))) != nbh::dbits(ys * nbh::pow2i(k))) atomicAdd(bad, 1ULL);
    }
    // the step rule
    const int emin = -30 + (int)(r0 >> 40) % 12;           // dt_min = 2^emin
    const int emax = emin + (int)(r1 >> 40) % 22;           // dt_max = 2^emax
    const double dt_min = nbh::pow2i(emin), dt_max = nbh::pow2i(emax);
    const int eo = emin - 1 + (int)(r2 >> 40) % (emax - emin + 3);
    const double dt_old = (r3 & 15) == 0 ? make_pos(1023 + eo, r4) : nbh::pow2i(eo);
    double t;
    switch ((r3 >> 4) & 7) {
      case 0: t = 0.0; break;
      case 1: t = make_pos(1023 + (int)(r4 >> 50) % 8 - 4, r5); break;      // arbitrary
      case 2: t = make_pos(0, r5 | 1); break;                                 // subnormal
      default: t = (double)(r5 >> 44) * nbh::pow2i(eo + (int)(r4 >> 60) % 4 - 1);  // multiples of a nearby step
    }
    const double eta = (r4 & 1) ? 0.01 : make_pos(1023 - 7 + (int)((r4 >> 8) % 4), r5 >> 3);
    double num = random_norm(r1, r2), den = random_norm(r3, r4);
    if ((r5 & 3) == 0 && isfinite(num) && num > 0.0 && isfinite(den) && den > 0.0) {
      // den's significand equal to fl(eta num)'s, or one unit either side:
      // quotients at and next to a power-of-two boundary
      const uint64_t nb = nbh::dbits(eta * num);
      const int64_t off = (int64_t)((r5 >> 2) % 3) - 1;
      const uint64_t frac = (uint64_t)((int64_t)(nb & 0x000FFFFFFFFFFFFFULL) + off) & 0x000FFFFFFFFFFFFFULL;
      den = from_bits((nbh::dbits(den) & 0xFFF0000000000000ULL) | frac);
    }
    bool nan_a, nan_b;
    const double da = nbh::new_step_nd(t, dt_old, num, den, eta, dt_min, dt_max, st_fast, nan_a);
    const double db = nbh::new_step_fp64(t, dt_old, num, den, eta, dt_min, dt_max, st_ref, nan_b);
    if (nbh::dbits(da) != nbh::dbits(db) || nan_a != nan_b) atomicAdd(bad, 1ULL);
  }
}

}  // namespace

extern "C" int nb_selftest_corrector(int device, int64_t samples, uint64_t seed, int64_t* mismatches) {
  if (samples < 0 || !mismatches) return NB_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return NB_ECUDA;
  }
  unsigned long long* d = nullptr;  // [0] mismatches, then two status words
  if (cudaMalloc((void**)&d, sizeof(unsigned long long) + 2 * sizeof(nb_dev_status)) != cudaSuccess) {
    cudaGetLastError();
    return NB_ENOMEM;
  }
  nb_dev_status* st = reinterpret_cast<nb_dev_status*>(d + 1);
  int rc = NB_OK;
  if (cudaMemset(d, 0, sizeof(unsigned long long) + 2 * sizeof(nb_dev_status)) != cudaSuccess) rc = NB_ECUDA;
  if (rc == NB_OK && samples > 0) {
    selftest_kernel<<<1024, 256>>>(samples, seed, d, st, st + 1);
    if (cudaGetLastError() != cudaSuccess) rc = NB_ECUDA;
  }
  unsigned long long h[1 + 2 * sizeof(nb_dev_status) / sizeof(unsigned long long)] = {0};
  if (rc == NB_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = NB_ECUDA;
  cudaFree(d);
  if (rc != NB_OK) {
    cudaGetLastError();
    return rc;
  }
  nb_dev_status s[2];
  memcpy(s, h + 1, sizeof(s));
  // the criteria below dt_min count the same in both forms
  *mismatches = (int64_t)h[0] + (s[0].dt_underflows != s[1].dt_underflows ? 1 : 0);
  return NB_OK;
}
