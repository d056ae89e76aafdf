// nmfa_device.cuh -- device helpers shared by the NMFA kernels: the Philox4x32-10
// counter-based generator (Salmon et al., SC'11), the uniform mapping and the
// Box-Muller transform that turn it into the N(0, 1) draws of Algorithm 1's field update.
//
// Stream layout (fixed for every kernel of the library):
//   counter = (r / 4, t, i, stream_id), key = (seed low 32 bits, seed high 32 bits)
//   words 0,1 -> replicas 4p (cos) and 4p+1 (sin) of spin i at step t
//   words 2,3 -> replicas 4p+2 (cos) and 4p+3 (sin)
//   uniform(w) = (2 * (w >> 9) + 1) * 2^-24, in (0, 1) and exact in binary32.
// One generator call therefore serves four consecutive replicas of one spin.
#pragma once
#include <cstdint>

namespace nmfa {

struct NoiseKey {
  uint32_t lo, hi;
};

__host__ __device__ inline NoiseKey make_noise_key(uint64_t seed) {
  return NoiseKey{static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)};
}

// Ten Philox rounds: the products of words 0 and 2 with the two multipliers are
// split into high and low halves, the halves cross over and the round key is
// mixed into the high halves; the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, NoiseKey key) {
  uint32_t k0 = key.lo, k1 = key.hi;
#pragma unroll
  for (int rd = 0; rd < 10; ++rd) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    const uint32_t lo0 = m0 * c.x, hi0 = __umulhi(m0, c.x);
    const uint32_t lo1 = m1 * c.z, hi1 = __umulhi(m1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 noise_words(NoiseKey key, uint32_t stream, uint32_t rep4,
                                             uint32_t t, uint32_t i) {
  return philox4x32_10(make_uint4(rep4, t, i, stream), key);
}

__device__ __forceinline__ float u01_f32(uint32_t w) {
  return static_cast<float>(((w >> 9) << 1) | 1u) * 5.9604644775390625e-08f;  // 2^-24
}
__device__ __forceinline__ double u01_f64(uint32_t w) {
  return static_cast<double>(((w >> 9) << 1) | 1u) * 5.9604644775390625e-08;
}

// Four N(0,1) draws for replicas 4p..4p+3 from one block of words (binary32).
__device__ __forceinline__ float4 gauss4_f32(uint4 w) {
  const float ra = sqrtf(-2.0f * logf(u01_f32(w.x)));
  const float rb = sqrtf(-2.0f * logf(u01_f32(w.z)));
  float sa, ca, sb, cb;
  sincospif(2.0f * u01_f32(w.y), &sa, &ca);
  sincospif(2.0f * u01_f32(w.w), &sb, &cb);
  return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

// The same draws in binary64.
__device__ __forceinline__ void gauss4_f64(uint4 w, double z[4]) {
  const double ra = sqrt(-2.0 * log(u01_f64(w.x)));
  const double rb = sqrt(-2.0 * log(u01_f64(w.z)));
  double sa, ca, sb, cb;
  sincospi(2.0 * u01_f64(w.y), &sa, &ca);
  sincospi(2.0 * u01_f64(w.w), &sb, &cb);
  z[0] = ra * ca;
  z[1] = ra * sa;
  z[2] = rb * cb;
  z[3] = rb * sb;
}

// The same generator with the round keys precomputed (rk[2r], rk[2r+1] = key of
// round r) and each 32x32 -> 64-bit product formed in one wide multiply.
struct RoundKeys {
  uint32_t k[20];
};
__device__ __forceinline__ RoundKeys make_round_keys(NoiseKey key) {
  RoundKeys rk;
#pragma unroll
  for (int rd = 0; rd < 10; ++rd) {
    rk.k[2 * rd] = key.lo + static_cast<uint32_t>(rd) * 0x9E3779B9u;
    rk.k[2 * rd + 1] = key.hi + static_cast<uint32_t>(rd) * 0xBB67AE85u;
  }
  return rk;
}
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int rd = 0; rd < 10; ++rd) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ rk.k[2 * rd], static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ rk.k[2 * rd + 1], static_cast<uint32_t>(p0));
  }
  return c;
}

// The same uniform built from bits: 1 + k 2^-23 has k as its mantissa, and adding
// -(1 - 2^-24) gives (2k + 1) 2^-24 exactly (the sum has at most 24 significant bits).
__device__ __forceinline__ float u01_f32_bits(uint32_t w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) + (-1.0f + 5.9604644775390625e-08f);
}

// Four draws with the hardware transcendental units (lg2, rsqrt, sin, cos): the
// angle 2 pi u is evaluated as -(sin, cos) of 2 pi (u - 1/2), whose argument lies
// in (-pi, pi) where the sine/cosine approximations are most accurate; u - 1/2 is
// exact.  Absolute error of each draw is below 1e-5, far inside the BF16 path's
// rounding of the state.
__device__ __forceinline__ float4 gauss4_f32_fast(uint4 w) {
  // -2 ln u >= 0; the approximate log may round to 0 (or a hair below) for u next
  // to 1, so clamp before the reciprocal square root (sqrt(0) must stay 0).
  const float la = fmaxf(-1.3862943611198906f * __log2f(u01_f32_bits(w.x)), 0.0f);
  const float lc = fmaxf(-1.3862943611198906f * __log2f(u01_f32_bits(w.z)), 0.0f);
  const float ra = la * rsqrtf(fmaxf(la, 1e-30f));
  const float rc = lc * rsqrtf(fmaxf(lc, 1e-30f));
  const float aa = 6.283185307179586f * (u01_f32_bits(w.y) - 0.5f);
  const float ac = 6.283185307179586f * (u01_f32_bits(w.w) - 0.5f);
  float sa, ca, sc, cc;
  __sincosf(aa, &sa, &ca);
  __sincosf(ac, &sc, &cc);
  return make_float4(-ra * ca, -ra * sa, -rc * cc, -rc * sc);
}

__device__ __forceinline__ float get4(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

}  // namespace nmfa
