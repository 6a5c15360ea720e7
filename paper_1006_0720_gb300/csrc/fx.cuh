// FP64-accurate arithmetic without FP64 instructions.
//
// GB300 issues FP64 arithmetic, FP64 compares and every conversion to or
// from FP64 at about 2 per clock per SM, against ~128 FP32 and ~64-100
// integer operations.  The particle kernel therefore never executes an FP64
// instruction on its fast path:
//   - state values (FP64 in memory) are decoded from their bits into 64-bit
//     fixed point (exact additions), and encoded back with round-to-nearest-
//     even;
//   - products are formed as unevaluated sums of two FP32 numbers
//     ("double-float", Dekker 1971; Knuth's TwoSum; the FMA-based exact
//     product), about 48 significant bits;
//   - increments are summed in double-float and added to the fixed-point
//     state exactly.
// All helpers are host+device so that they can be checked on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDA_ARCH__
#define FX_HD __host__ __device__ __forceinline__
#define FX_CLZ64(x) __clzll((long long)(x))
#define FX_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define FX_ADD(a, b) __fadd_rn((a), (b))
#define FX_SUB(a, b) __fsub_rn((a), (b))
#define FX_MUL(a, b) __fmul_rn((a), (b))
#define FX_SQRT(a) __fsqrt_rn(a)
#define FX_RCP(a) __fdiv_rn(1.0f, (a))
#else
#include <math.h>
#define FX_HD inline
#define FX_CLZ64(x) __builtin_clzll((unsigned long long)(x))
#define FX_FMA(a, b, c) fmaf((a), (b), (c))
#define FX_ADD(a, b) ((float)((a) + (b)))
#define FX_SUB(a, b) ((float)((a) - (b)))
#define FX_MUL(a, b) ((float)((a) * (b)))
#define FX_SQRT(a) sqrtf(a)
#define FX_RCP(a) (1.0f / (a))
#endif

namespace fx {

FX_HD uint32_t f_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
FX_HD float bits_f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

// Exponent field of an FP64 bit pattern (0 for zero and subnormals).
FX_HD int d_exp(uint64_t b) { return (int)((b >> 52) & 0x7FF); }

// FP64 bits -> fixed point with F fraction bits, rounded to nearest (ties
// away from zero).  Exact when the value's ulp is >= 2^-F.  Requires
// |value| < 2^(63-F-1) (checked by the caller through d_exp).
FX_HD int64_t d2fix(uint64_t b, int F) {
  const int e = d_exp(b);
  if (e == 0) return 0;
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int s = e - 1075 + F;
  uint64_t r;
  if (s >= 0) r = m << s;
  else if (s > -64) r = (m + (1ull << (-s - 1))) >> (-s);
  else r = 0;
  return (b >> 63) ? -(int64_t)r : (int64_t)r;
}

// Fixed point (F fraction bits) -> FP64 bits, round to nearest even (IEEE).
FX_HD uint64_t fix2d(int64_t X, int F) {
  if (X == 0) return 0;
  uint64_t sign = 0, a = (uint64_t)X;
  if (X < 0) { sign = 1ull << 63; a = 0ull - (uint64_t)X; }
  int nb = 64 - FX_CLZ64(a);
  uint64_t m;
  if (nb <= 53) {
    m = a << (53 - nb);
  } else {
    const int sh = nb - 53;
    uint64_t q = a >> sh;
    const uint64_t rem = a & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) q += 1;
    if (q == (1ull << 53)) { q >>= 1; nb += 1; }
    m = q;
  }
  const uint64_t e = (uint64_t)(nb - 1 - F + 1023);
  return sign | (e << 52) | (m & 0xFFFFFFFFFFFFFull);
}

// FP32 -> fixed point, exact when the float's ulp >= 2^-F (else rounded).
// Requires |f| < 2^(63-F-1).
FX_HD int64_t f2fix(float f, int F) {
  const uint32_t b = f_bits(f);
  const int e = (int)((b >> 23) & 0xFF);
  if (e == 0) return 0;
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  const int s = e - 150 + F;
  uint64_t r;
  if (s >= 0) r = m << s;
  else if (s > -40) r = (m + (1ull << (-s - 1))) >> (-s);
  else r = 0;
  return (b >> 31) ? -(int64_t)r : (int64_t)r;
}

struct alignas(8) df {
  float h, l;
};

// FP64 <-> double-float with FP64 instructions (initialisation, state
// transfers and the FP64 fall-back only): h = x rounded to FP32, l = the
// exact remainder rounded to FP32; back as the FP64 sum, rounded once.
FX_HD df from_double(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}
FX_HD double to_double(df a) { return (double)a.h + (double)a.l; }

// The same two conversions without FP64 arithmetic (integer rounding of the
// mantissas), bit-identical to from_double / to_double; outside the range
// where every part is a normal FP32 number (|x| below 2^-73 or from 2^126
// on, a low part far below the high part's last bit) they take the FP64
// expressions.  Used by the state transfers, which would otherwise run five
// FP64 additions and ten FP64 conversions per particle on the slow FP64
// pipe.
FX_HD df d2df_rn(uint64_t b) {
  const int e = d_exp(b);
  if (e < 1023 - 73 || e >= 1023 + 126) {
    double x;
    memcpy(&x, &b, 8);
    return from_double(x);
  }
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53 bits
  uint64_t hm = M >> 29;                                        // 24 bits
  const uint64_t rem = M & ((1ull << 29) - 1);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (hm & 1))) hm += 1;  // nearest, ties to even
  const int64_t r = (int64_t)M - (int64_t)(hm << 29);  // x - h in units of 2^(e-1075), |r| <= 2^28
  int eh = e - 1023 + 127;
  if (hm == (1ull << 24)) {
    hm >>= 1;
    eh += 1;
  }
  df out;
  out.h = bits_f(sign | ((uint32_t)eh << 23) | ((uint32_t)hm & 0x7FFFFFu));
  if (r == 0) {
    out.l = 0.0f;  // x - h == +0 under round to nearest
    return out;
  }
  const uint32_t ls = sign ^ (r < 0 ? 0x80000000u : 0u);
  uint64_t a = (uint64_t)(r < 0 ? -r : r);
  const int nb = 64 - FX_CLZ64(a);  // <= 29
  int el = e - 1075 + (nb - 1) + 127;
  uint32_t lm;
  if (nb <= 24) {
    lm = (uint32_t)(a << (24 - nb));
  } else {
    const int sh = nb - 24;
    uint64_t q = a >> sh;
    const uint64_t rr = a & ((1ull << sh) - 1), hf = 1ull << (sh - 1);
    if (rr > hf || (rr == hf && (q & 1))) q += 1;
    if (q == (1ull << 24)) {
      q >>= 1;
      el += 1;
    }
    lm = (uint32_t)q;
  }
  out.l = bits_f(ls | ((uint32_t)el << 23) | (lm & 0x7FFFFFu));
  return out;
}

// An FP32 value's FP64 bits (exact), without an FP64 conversion for normal
// numbers and zeros.
FX_HD uint64_t f2d_bits(float f) {
  const uint32_t b = f_bits(f);
  const int e = (int)((b >> 23) & 0xFF);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  if ((b & 0x7FFFFFFFu) == 0) return sign;
  if (e == 0 || e == 255) {
    const double x = (double)f;
    uint64_t r;
    memcpy(&r, &x, 8);
    return r;
  }
  return sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
}

FX_HD uint64_t df2d_rn(df a) {
  const uint32_t hb = f_bits(a.h), lb = f_bits(a.l);
  const int eh = (int)((hb >> 23) & 0xFF), el = (int)((lb >> 23) & 0xFF);
  const bool lzero = (lb & 0x7FFFFFFFu) == 0;
  const int D = eh - el;
  if (eh == 0 || eh == 255 || (!lzero && (el == 0 || el == 255 || D < 0 || D > 38))) {
    const double x = to_double(a);
    uint64_t r;
    memcpy(&r, &x, 8);
    return r;
  }
  const uint64_t hsign = (uint64_t)(hb >> 31) << 63;
  const uint64_t H = (uint64_t)((hb & 0x7FFFFFu) | 0x800000u);
  if (lzero) return hsign | ((uint64_t)(eh - 127 + 1023) << 52) | ((H & 0x7FFFFFu) << 29);
  const uint64_t L = (uint64_t)((lb & 0x7FFFFFu) | 0x800000u);
  // the exact sum S 2^(eh - 188): h at bits 61..38, l aligned below it
  int64_t S = (int64_t)(H << 38);
  const int64_t La = (int64_t)(L << (38 - D));
  S = ((hb >> 31) == (lb >> 31)) ? S + La : S - La;
  uint64_t sgn = hsign;
  if (S < 0) {
    S = -S;
    sgn ^= 1ull << 63;
  }
  if (S == 0) return 0ull;
  const uint64_t u = (uint64_t)S;
  int nb = 64 - FX_CLZ64(u);
  uint64_t q;
  if (nb <= 53) {
    q = u << (53 - nb);
  } else {
    const int sh = nb - 53;
    q = u >> sh;
    const uint64_t rr = u & ((1ull << sh) - 1), hf = 1ull << (sh - 1);
    if (rr > hf || (rr == hf && (q & 1))) q += 1;
    if (q == (1ull << 53)) {
      q >>= 1;
      nb += 1;
    }
  }
  return sgn | ((uint64_t)(nb + eh + 834) << 52) | (q & 0xFFFFFFFFFFFFFull);
}

// Knuth's TwoSum: s + e == a + b exactly.
FX_HD df two_sum(float a, float b) {
  const float s = FX_ADD(a, b);
  const float bb = FX_SUB(s, a);
  const float e = FX_ADD(FX_SUB(a, FX_SUB(s, bb)), FX_SUB(b, bb));
  return {s, e};
}

// Fixed point -> double-float.  X = a 2^44 + b 2^22 + c with 22-bit unsigned
// b, c and a signed |a| < 2^19: each piece converts to FP32 exactly by adding
// and subtracting a power-of-two "magic" constant, is scaled exactly by a
// power of two, and the three are summed with TwoSum; |error| < 2^-46 |X|.
FX_HD float exp2i(int k) { return bits_f((uint32_t)(k + 127) << 23); }  // 2^k, -126 <= k <= 127

FX_HD df fix2df(int64_t X, int F) {
  const int32_t a = (int32_t)(X >> 44);
  const uint32_t b = (uint32_t)((uint64_t)X >> 22) & 0x3FFFFFu;
  const uint32_t c = (uint32_t)X & 0x3FFFFFu;
  const float fa = FX_SUB(bits_f(0x4B400000u + (uint32_t)a), 12582912.0f);  // exact, |a| < 2^22
  const float fb = FX_SUB(bits_f(0x4B000000u | b), 8388608.0f);             // exact, b < 2^22
  const float fc = FX_SUB(bits_f(0x4B000000u | c), 8388608.0f);
  const float ha = FX_MUL(fa, exp2i(44 - F));
  const float hb = FX_MUL(fb, exp2i(22 - F));
  const float hc = FX_MUL(fc, exp2i(-F));
  const df s = two_sum(ha, hb);
  return df{s.h, FX_ADD(s.l, hc)};
}

// FP64 bits -> double-float (leading 24 bits and the next 24, truncated);
// values below 2^-100 in magnitude become 0, and a low part that would
// fall below the FP32 normal range (|x| below about 2^-76) is dropped (an
// absolute error below 2^-126).
FX_HD df d2df(uint64_t b) {
  df r = {0.f, 0.f};
  const int e = d_exp(b);
  if (e < 1023 - 100) return r;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull);
  // top 23 explicit bits
  r.h = bits_f(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)(m >> 29));
  const uint64_t rem = m & ((1ull << 29) - 1);  // weight 2^(e-1075)
  if (rem) {
    const int nr = 64 - FX_CLZ64(rem);          // <= 29
    const int el = e - 1075 + nr - 1 + 127;     // FP32 exponent field of the low part
    const uint32_t mr = nr > 24 ? (uint32_t)(rem >> (nr - 24)) : (uint32_t)(rem << (24 - nr));
    if (el > 0) r.l = bits_f(sign | ((uint32_t)el << 23) | (mr & 0x7FFFFFu));
  }
  return r;
}

// Renormalize (|a| >= |b|).
FX_HD df fast_two_sum(float a, float b) {
  const float s = FX_ADD(a, b);
  return {s, FX_SUB(b, FX_SUB(s, a))};
}

FX_HD df df_norm(df a) { return two_sum(a.h, a.l); }

// Unnormalized products (the low part is not folded in).
FX_HD df mul_f(df a, float b) {
  const float p = FX_MUL(a.h, b);
  const float e = FX_FMA(a.h, b, -p);
  return {p, FX_FMA(a.l, b, e)};
}

FX_HD df mul(df a, df b) {
  const float p = FX_MUL(a.h, b.h);
  float e = FX_FMA(a.h, b.h, -p);
  e = FX_FMA(a.h, b.l, e);
  e = FX_FMA(a.l, b.h, e);
  return {p, e};
}

// Accumulator: the high parts are added exactly (TwoSum), the low parts and
// the rounding errors of the high sums in FP32.
struct acc {
  float h, l;
  FX_HD void init(df a) { h = a.h; l = a.l; }
  FX_HD void add(df a) {
    const df s = two_sum(h, a.h);
    h = s.h;
    l = FX_ADD(l, FX_ADD(s.l, a.l));
  }
  FX_HD void sub(df a) { add(df{-a.h, -a.l}); }
  FX_HD int64_t fix(int F) const { return f2fix(h, F) + f2fix(l, F); }
  FX_HD df value() const { return df_norm(df{h, l}); }
};

FX_HD df add(df a, df b) {
  acc s;
  s.init(a);
  s.add(b);
  return s.value();
}

FX_HD df sub(df a, df b) { return add(a, df{-b.h, -b.l}); }

// sqrt of a non-negative double-float: one Newton correction of the FP32
// root, r = s + (a - s^2) / (2 s).
FX_HD df sqrt_df(df a) {
  if (!(a.h > 0.f)) return {0.f, 0.f};
  const float s = FX_SQRT(a.h);
  const float p = FX_MUL(s, s);
  const float pe = FX_FMA(s, s, -p);            // s^2 = p + pe exactly
  const float d = FX_ADD(FX_SUB(FX_SUB(a.h, p), pe), a.l);
  const float c = FX_MUL(d, FX_MUL(0.5f, FX_RCP(s)));
  return fast_two_sum(s, c);
}

// Signed 128-bit integer (hi:lo) times 2^scale -> double-float (the top 63
// bits are kept; |error| < 2^-46 relative).
FX_HD df i128_to_df(uint64_t lo, int64_t hi, int scale) {
  const bool neg = hi < 0;
  uint64_t ml = lo, mh = (uint64_t)hi;
  if (neg) {
    ml = ~ml + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  uint64_t top;
  int sh;
  if (mh != 0) {
    const int nb = 128 - FX_CLZ64(mh);  // bit length, > 64
    sh = nb - 63;
    top = (mh << (64 - sh)) | (ml >> sh);
  } else if (ml >> 63) {
    sh = 1;
    top = ml >> 1;
  } else {
    sh = 0;
    top = ml;
  }
  const df r = fix2df((int64_t)top, -(sh + scale));
  return neg ? df{-r.h, -r.l} : r;
}

// 1/n for an integer 1 <= n < 2^24 as a double-float (one Newton step).
FX_HD df recip_df(int n) {
  const float fn = (float)n;
  const float r = FX_RCP(fn);
  const float e = FX_FMA(-fn, r, 1.0f);  // exact residual
  return fast_two_sum(r, FX_MUL(r, e));
}

// Double-float -> FP64 bits, rounded to nearest (error < 2^-61 relative).
FX_HD uint64_t df2d(df a) {
  if (a.h == 0.0f) return 0ull;
  const int eh = (int)((f_bits(a.h) >> 23) & 0xFF) - 127;
  const int F = 60 - eh;
  return fix2d(f2fix(a.h, F) + f2fix(a.l, F), F);
}

// Sign and ordering of normalized double-floats.
FX_HD bool lt(df a, df b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
FX_HD bool ge0(df a) { return a.h > 0.f || (a.h == 0.f && a.l >= 0.f); }

}  // namespace fx
