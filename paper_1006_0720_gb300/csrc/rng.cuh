// Counter-based Gaussian draws on the device.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): a 128-bit counter and a 64-bit key, ten rounds of
// two 32x32->64 multiplications (multipliers 0xD2511F53, 0xCD9E8D57) with the
// key bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
//
// Uniforms: (floor(w / 2^9) + 1/2) / 2^23, exact in FP32, inside (0, 1).
// Gaussians: Box-Muller, evaluated in FP32 with explicitly rounded
// operations so that every implementation of this specification returns the
// same bits:
//   ln u  : u = m 2^e, m in [sqrt(1/2), sqrt(2)); s = (m-1)/(m+1);
//           ln m = 2 s (1 + z/3 + z^2/5 + z^3/7 + z^4/9), z = s^2 (Horner,
//           fused multiply-adds, innermost first: 1/9 * z + 1/7);
//           ln u = e * (1420/2048) + (e * tail + ln m)
//   sin/cos 2 pi u: t = 4u, q = rint(t), r = t - q, th = r * (pi/2);
//           sin th, cos th by Taylor polynomials in z = th^2 to degree 9 and
//           10; the result rotated by q quarter turns.
#pragma once
#include <stdint.h>

namespace pdfgb {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ float u01_from_word(uint32_t w) {
  return __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 0x1p-23f);
}

// ln u for u in [2^-24, 1): normal FP32 input only.
__device__ __forceinline__ float ln_unit(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 126;                                 // u = m 2^e, m in [0.5, 1)
  float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F000000u);
  if (m < 0.70710678f) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float z = __fmul_rn(s, s);
  float p = __fmaf_rn(z, 1.0f / 9.0f, 1.0f / 7.0f);
  p = __fmaf_rn(p, z, 1.0f / 5.0f);
  p = __fmaf_rn(p, z, 1.0f / 3.0f);
  p = __fmaf_rn(p, z, 1.0f);
  const float lnm = __fmul_rn(__fmul_rn(2.0f, s), p);
  const float fe = (float)e;
  return __fmaf_rn(fe, 1420.0f / 2048.0f, __fmaf_rn(fe, -2.12194440054690582e-4f, lnm));
}

__device__ __forceinline__ void sincos_2pi(float u, float* sn, float* cs) {
  const float t = __fmul_rn(4.0f, u);
  const float q = rintf(t);
  const float r = __fsub_rn(t, q);
  const float th = __fmul_rn(r, 1.57079632679489662f);
  const float z = __fmul_rn(th, th);
  float ps = __fmaf_rn(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = __fmaf_rn(ps, z, 1.0f / 120.0f);
  ps = __fmaf_rn(ps, z, -1.0f / 6.0f);
  ps = __fmaf_rn(ps, z, 1.0f);
  const float s = __fmul_rn(th, ps);
  float pc = __fmaf_rn(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = __fmaf_rn(pc, z, -1.0f / 720.0f);
  pc = __fmaf_rn(pc, z, 1.0f / 24.0f);
  pc = __fmaf_rn(pc, z, -0.5f);
  const float c = __fmaf_rn(pc, z, 1.0f);
  switch (((int)q) & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

__device__ __forceinline__ void box_muller(uint32_t w1, uint32_t w2, float* g0, float* g1) {
  const float rad = __fsqrt_rn(__fmul_rn(-2.0f, ln_unit(u01_from_word(w1))));
  float sn, cs;
  sincos_2pi(u01_from_word(w2), &sn, &cs);
  *g0 = __fmul_rn(rad, cs);
  *g1 = __fmul_rn(rad, sn);
}

// Four N(0,1) from the block with counter (c0, c1, c2, c3).
__device__ __forceinline__ void gauss4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                       uint32_t c3, float g[4]) {
  uint32_t c[4] = {c0, c1, c2, c3};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  box_muller(c[0], c[1], &g[0], &g[1]);
  box_muller(c[2], c[3], &g[2], &g[3]);
}

enum : uint32_t { kPurposeStep = 0, kPurposeInit = 1, kPurposeRedist = 2 };

}  // namespace pdfgb
