// divint.cuh -- the correctly rounded binary64 quotient RN(x / y) computed on the integer
// pipes.  GB300 retires binary64 arithmetic at about 1/64 of its binary32 rate and an IEEE
// binary64 division costs the FP64 pipe about seven fused multiply-adds (measured), so in
// the edge weights of Sec. 2.2 the division is most of the FP64 work.  Here it costs no
// binary64 instruction on the common path:
//
//   x = mx 2^(ex-52), y = my 2^(ey-52) with 53-bit integer significands mx, my.  With
//   k = 53 when mx >= my and 54 otherwise, Q = floor(mx 2^k / my) lies in [2^53, 2^54) and
//   holds the 53 result bits plus one guard bit; the remainder mx 2^k - Q my gives the
//   sticky bit, and round-to-nearest-even on (Q, remainder) is exact integer logic.
//
// Q comes from a fixed-point reciprocal v ~ 2^116 / my refined by Newton-Raphson iteration
// v <- v + v (2^126 - d v) / 2^126 (d = my 2^10; the classical quadratically convergent
// reciprocal iteration, e.g. Knuth, TAOCP Vol. 2, Sec. 4.3.3), seeded from a binary32
// reciprocal of the top 24 bits of my: two steps take the relative error from about 2^-22
// to about 2^-62, so mx v / 2^(116-k) is within one unit of Q.  The remainder is formed
// exactly (modulo 2^64, and its magnitude is below 2^55), Q is corrected by one unit when
// the remainder leaves [0, my), and a remainder still outside [0, my) -- which the error
// bound excludes -- hands the operands to the hardware division, as do operands that are
// zero, subnormal, infinite or NaN and quotients outside the normal range, so the function
// returns RN(x / y) bit for bit on every input.
#pragma once

namespace cwm {

// One Newton step for v ~ 2^126 / d, d in [2^62, 2^63): e = 2^126 - d v is formed exactly
// as a 128-bit two's-complement value; SH is chosen so that e / 2^SH fits a signed 64-bit
// word at the step's accuracy (|e| < 2^(62 + SH)).  The correction v e / 2^126 is
// (v |e / 2^SH|) / 2^64 / 2^(62 - SH).  The sum saturates at 2^64 - 1 (v = 2^64 exactly
// is the reciprocal of d = 2^62, which the quotient step then corrects by one unit).
template <int SH>
__device__ __forceinline__ unsigned long long divint_newton(unsigned long long d, unsigned long long v) {
  const unsigned long long plo = d * v, phi = __umul64hi(d, v);
  const unsigned long long elo = 0ull - plo;
  const unsigned long long ehi = (1ull << 62) - phi - (plo != 0ull ? 1ull : 0ull);
  const long long t = (long long)((ehi << (64 - SH)) | (elo >> SH));
  const unsigned long long at = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const unsigned long long c = __umul64hi(v, at) >> (62 - SH);
  if (t < 0) return v - c;
  const unsigned long long s = v + c;
  return s < v ? ~0ull : s;
}

__device__ __forceinline__ double div_rn_int(double x, double y) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
  const unsigned long long by = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((bx >> 52) & 0x7ff), ey = (int)((by >> 52) & 0x7ff);
  const unsigned long long frac = (1ull << 52) - 1ull;
  const unsigned long long mx = (bx & frac) | (1ull << 52), my = (by & frac) | (1ull << 52);
  const int lt = mx < my ? 1 : 0;
  int E = ex - ey + 1023 - lt;  // biased exponent of the quotient
  if (ex == 0 || ex == 0x7ff || ey == 0 || ey == 0x7ff || E < 1 || E > 2045) return __ddiv_rn(x, y);
  // seed: 2^87 / (my >> 29) from a binary32 reciprocal of the top 24 bits of my (exactly
  // representable), taken to 32 bits (a 32-bit conversion: 64-bit ones are slow) and shifted
  const float s = __frcp_rn((float)(unsigned)(my >> 29)) * 0x1p55f;  // in (2^31, 2^32]
  unsigned long long v = (unsigned long long)(s >= 0x1p32f ? 0xffffffffu : __float2uint_rz(s)) << 32;
  const unsigned long long d = my << 10;
  v = divint_newton<42>(d, v);  // |e| < 2^104: the seed's relative error is below 2^-22
  v = divint_newton<21>(d, v);  // |e| < 2^83: below 2^-44 after the first step
  // Q ~ mx v / 2^(116 - k): the 117-bit product shifted right by 63 (k = 53) or 62 (k = 54)
  const unsigned long long plo = mx * v, phi = __umul64hi(mx, v);
  unsigned long long q = lt ? ((phi << 2) | (plo >> 62)) : ((phi << 1) | (plo >> 63));
  const long long dm = (long long)my;
  long long rem = (long long)((mx << (53 + lt)) - q * my);  // mx 2^k - q my, exact mod 2^64
  if (rem < 0) {
    --q;
    rem += dm;
  } else if (rem >= dm) {
    ++q;
    rem -= dm;
  }
  if (rem < 0 || rem >= dm) return __ddiv_rn(x, y);
  // round to nearest, ties to even: guard bit q & 1, sticky bit rem != 0
  unsigned long long m = q >> 1;
  if ((q & 1ull) && (rem != 0 || (m & 1ull))) ++m;
  if (m == (1ull << 53)) {
    m >>= 1;
    ++E;
  }
  const unsigned long long sign = (bx ^ by) & (1ull << 63);
  return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (m & frac)));
}

}  // namespace cwm
