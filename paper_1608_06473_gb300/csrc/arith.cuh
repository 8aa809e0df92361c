// Hand-written arithmetic helpers of the surrogate kernels: exact integer
// multiply-adds, int64 -> FP64 conversion on the integer pipe, a reciprocal
// on the integer pipe, and an FP32 divide by a reciprocal estimate refined
// with a Newton-Raphson step.  GB300 issues FP64
// operations (conversions included) on a narrow pipe, so the FP64 kernels
// move what they can to the integer pipe.  Each helper is checked against
// the IEEE operation it stands for by a diagnostic entry point (diag.cu).
#pragma once

#include <cstdint>

namespace hhg {

// v * i + c (mod 2^64) for a 32-bit multiplier i >= 0: the low word times i
// widened to 64 bits plus c, then the high word times i added to the top
// half (two integer multiply-adds instead of a full 64 x 64 product).
__device__ __forceinline__ long long mad_i64_u32(long long v, unsigned i, long long c) {
  const unsigned long long vu = (unsigned long long)v;
  unsigned long long r = (unsigned long long)(unsigned)vu * i + (unsigned long long)c;
  r += (unsigned long long)((unsigned)(vu >> 32) * i) << 32;
  return (long long)r;
}

// v 2^-E for int64 v on the integer pipe (GB300 issues FP64 conversions on
// its narrow FP64 pipe): magnitude, leading-zero count, normalising shift,
// and the biased exponent, lowered by E, added to the top bits, where the
// leading one of the shifted magnitude carries into the exponent field.  The
// weights of the FP64 surrogate are stored as integers scaled by 2^E, so
// this also undoes the scale for free.  Truncated toward zero (relative
// error below 2^-52); |v| 2^-E must be a normal FP64 number (or v = 0).
__device__ __forceinline__ double i64_to_f64_scaled(long long v, int E) {
  const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  unsigned long long m;
  asm("shl.b64 %0, %1, %2;" : "=l"(m) : "l"(a), "r"(lz));
  const unsigned long long bits = ((unsigned long long)(1085 - lz - E) << 52) + (m >> 11);
  return a ? __longlong_as_double((long long)(bits | sign)) : 0.0;
}

// 2^E / W for W != 0, as FP64, on the integer pipe.  With Wn = |W| shifted
// to [2^63, 2^64), R ~ 2^126 / Wn in (2^62, 2^63] is seeded from the FP32
// reciprocal estimate of Wn's leading 24 bits (relative error about 2^-22)
// and refined by two Newton-Raphson steps for the reciprocal,
// R <- R + R (2^126 - Wn R) / 2^126, in 64 x 64 -> 128-bit integer products;
// each step squares the relative error, so R ends within a few units of
// 2^126 / Wn (relative error below 2^-60).  R is then truncated to 53 bits and
// given the exponent of 2^(E + lz - 126) (lz = leading zeros of |W|).  The
// result is within 2^-51 of 2^E / W.
__device__ __forceinline__ double rcp_i64_scaled(long long W, int E) {
  const unsigned long long sign = (unsigned long long)W & 0x8000000000000000ull;
  const unsigned long long a = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  const int lz = __clzll((long long)a);
  const unsigned long long an = a << lz;
  const float m = __uint_as_float(0x3F800000u | ((unsigned)(an >> 40) & 0x7FFFFFu));  // an / 2^63, truncated
  float x;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(m));  // 1 / m in (0.5, 1]
  const unsigned xb = __float_as_uint(x);
  // R = x 2^63 with x = (2^23 + frac) 2^(e - 150), e = biased exponent (126 or 127)
  unsigned long long R = (unsigned long long)((xb & 0x7FFFFFu) | 0x800000u) << ((int)(xb >> 23) - 87);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // e = 2^126 - an R as a signed 128-bit value; its top word eh (the low
    // word is dropped: an error below 2^64 in e, 2^-62 relative)
    const unsigned long long lo = an * R;
    const unsigned long long hi = __umul64hi(an, R);
    const long long eh = (long long)((1ull << 62) - hi - (lo != 0ull ? 1ull : 0ull));
    // correction R eh / 2^62 from the unsigned 128-bit product R |eh|
    const unsigned long long ea = eh < 0 ? 0ull - (unsigned long long)eh : (unsigned long long)eh;
    const unsigned long long plo = R * ea, phi = __umul64hi(R, ea);
    const unsigned long long corr = (phi << 2) | (plo >> 62);
    R = eh < 0 ? R - corr : R + corr;
  }
  const int lz2 = __clzll((long long)R);
  const unsigned long long mR = R << lz2;
  const unsigned long long bits = ((unsigned long long)(959 - lz2 + lz + E) << 52) + (mR >> 11);
  return __longlong_as_double((long long)(bits | sign));
}

// n / d in FP32: the hardware reciprocal estimate refined by one
// Newton-Raphson step x <- x + x (1 - d x), then the product.
__device__ __forceinline__ float div_nr32(float n, float d) {
  float x;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(d));
  x = fmaf(x, fmaf(-d, x, 1.0f), x);
  return n * x;
}

}  // namespace hhg
