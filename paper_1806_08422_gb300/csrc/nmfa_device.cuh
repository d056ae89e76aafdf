// nmfa_device.cuh -- device helpers shared by the NMFA kernels: the Philox4x32-10
// counter-based generator (Salmon et al., SC'11), the uniform mapping and the
// Box-Muller transform that turn it into the N(0, 1) draws of Algorithm 1 line 6.
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

__device__ __forceinline__ float get4(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

}  // namespace nmfa
